"""Seeded synthetic initial fields for the LB-MHD workloads.

This module holds no arithmetic of the lattice Boltzmann method: it only
draws the macroscopic fields (rho, u, B) that a run starts from.  Both the
CUDA path and the CPU oracle are fed from it, so a parity test compares the
two on identical inputs.  All arrays are float64 of shape (ny, nx), x
fastest; derivatives are periodic central differences, so the magnetic
fields built as a discrete curl have zero discrete divergence.

Workloads (the paper itself runs none; these follow its setting, 2D MHD
with a direct cascade, Sec. 1 and Sec. 3):
  * ``orszag_tang``: the Orszag-Tang vortex with a small seeded perturbation.
  * ``turbulence``: decaying 2D MHD turbulence, random-phase Fourier modes in
    a band of integer wavenumbers, divergence-free by construction.
  * ``ensemble``: a seeded list of independent runs of uneven sizes and
    Smagorinsky constants, for the batched form.
  * ``turbulence3d``: decaying 3D MHD turbulence for the 3D extension,
    arrays of shape (nz, ny, nx), u and B discrete curls of band-limited
    random vector potentials.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _dx(a: np.ndarray) -> np.ndarray:
    """Periodic central difference along x (axis 1)."""
    return 0.5 * (np.roll(a, -1, axis=1) - np.roll(a, 1, axis=1))


def _dy(a: np.ndarray) -> np.ndarray:
    """Periodic central difference along y (axis 0)."""
    return 0.5 * (np.roll(a, -1, axis=0) - np.roll(a, 1, axis=0))


def curl_z(psi: np.ndarray):
    """(d_y psi, -d_x psi): a discretely divergence-free planar field."""
    return _dy(psi), -_dx(psi)


def orszag_tang(nx: int, ny: int, u0: float = 0.05, b0: float = 0.05, amp: float = 1e-4,
                seed: int = 0):
    """Orszag-Tang vortex: rho = 1, u = u0(-sin y, sin x), B = b0(-sin y, sin 2x)
    on x = 2 pi i / nx, y = 2 pi j / ny.  A seeded uniform perturbation in
    [-amp, amp] is added to each component of u; B is perturbed by the
    discrete curl of a seeded uniform potential, scaled so that its largest
    magnitude is amp (a cellwise draw on B would break div B = 0)."""
    x = 2.0 * np.pi * np.arange(nx) / nx
    y = 2.0 * np.pi * np.arange(ny) / ny
    X, Y = np.meshgrid(x, y)
    rho = np.ones((ny, nx))
    ux = -u0 * np.sin(Y)
    uy = u0 * np.sin(X)
    bx = -b0 * np.sin(Y)
    by = b0 * np.sin(2.0 * X)
    if amp > 0.0:
        g = _rng(seed)
        ux = ux + g.uniform(-amp, amp, size=(ny, nx))
        uy = uy + g.uniform(-amp, amp, size=(ny, nx))
        a = g.uniform(-1.0, 1.0, size=(ny, nx))
        dbx, dby = curl_z(a)
        m = np.sqrt(dbx * dbx + dby * dby).max()
        if m > 0.0:
            bx = bx + dbx * (amp / m)
            by = by + dby * (amp / m)
    return rho, ux, uy, bx, by


def band_field(nx: int, ny: int, kmin: float, kmax: float, g: np.random.Generator) -> np.ndarray:
    """Real field with equal amplitude and a uniform random phase on every
    integer mode (n_x, n_y) with kmin <= |n| <= kmax (one draw per +/- pair)."""
    kk = int(np.ceil(kmax))
    spec = np.zeros((ny, nx // 2 + 1), dtype=np.complex128)
    for my in range(-kk, kk + 1):
        for mx in range(0, kk + 1):
            if mx == 0 and my <= 0:
                continue  # one representative per conjugate pair
            r2 = mx * mx + my * my
            if r2 < kmin * kmin or r2 > kmax * kmax:
                continue
            ph = np.exp(1j * g.uniform(0.0, 2.0 * np.pi))
            if mx == 0:
                spec[my % ny, 0] += ph
                spec[(-my) % ny, 0] += np.conj(ph)
            else:
                spec[my % ny, mx % (nx // 2 + 1)] += ph
    return np.fft.irfft2(spec, s=(ny, nx))


def turbulence(nx: int, ny: int, kmin: float = 4.0, kmax: float = 8.0, rms: float = 0.04,
               seed: int = 1):
    """Decaying 2D MHD turbulence: rho = 1; u and B are discrete curls of
    random-phase stream function and flux function in the band
    kmin <= |k| <= kmax, each scaled to sqrt(<|u|^2>) = sqrt(<|B|^2>) = rms."""
    g = _rng(seed)
    psi = band_field(nx, ny, kmin, kmax, g)
    az = band_field(nx, ny, kmin, kmax, g)
    ux, uy = curl_z(psi)
    bx, by = curl_z(az)
    su = np.sqrt(np.mean(ux * ux + uy * uy))
    sb = np.sqrt(np.mean(bx * bx + by * by))
    ux, uy = ux * (rms / su), uy * (rms / su)
    bx, by = bx * (rms / sb), by * (rms / sb)
    return np.ones((ny, nx)), ux, uy, bx, by


def ensemble(nruns: int = 256, seed: int = 7, sizes=(128, 256, 512, 1024),
             cs_range=(0.05, 0.2), tau_range=(0.51, 0.7)):
    """Independent runs for the batched form: square sizes drawn uniformly
    from ``sizes``, one seed each, C_S and tau (= tau_nu = tau_eta) drawn
    uniformly from their ranges."""
    g = _rng(seed)
    n = g.choice(np.asarray(sizes), size=nruns)
    seeds = g.integers(0, 2**31 - 1, size=nruns)
    cs = g.uniform(*cs_range, size=nruns)
    tau = g.uniform(*tau_range, size=nruns)
    return [dict(nx=int(n[r]), ny=int(n[r]), seed=int(seeds[r]), C_S=float(cs[r]),
                 tau=float(tau[r])) for r in range(nruns)]


def _band_field3(nx: int, ny: int, nz: int, kmin: float, kmax: float,
                 g: np.random.Generator) -> np.ndarray:
    """A real periodic field of shape (nz, ny, nx) with equal amplitude on
    every integer wavevector kmin <= |n| <= kmax and random phases."""
    nzf, nyf, nxf = np.fft.fftfreq(nz) * nz, np.fft.fftfreq(ny) * ny, np.fft.fftfreq(nx) * nx
    kz, ky, kx = np.meshgrid(nzf, nyf, nxf, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    mask = (kk >= kmin) & (kk <= kmax)
    spec = np.where(mask, np.exp(2j * np.pi * g.random(kk.shape)), 0.0)
    return np.real(np.fft.ifftn(spec))


def _d3(a: np.ndarray, axis: int) -> np.ndarray:
    """Periodic central difference along array axis (0 z, 1 y, 2 x)."""
    return 0.5 * (np.roll(a, -1, axis=axis) - np.roll(a, 1, axis=axis))


def curl3(ax: np.ndarray, ay: np.ndarray, az: np.ndarray):
    """Central-difference curl of a periodic vector field (arrays (nz, ny,
    nx)); its central-difference divergence is zero."""
    return (_d3(az, 1) - _d3(ay, 0), _d3(ax, 0) - _d3(az, 2), _d3(ay, 2) - _d3(ax, 1))


def turbulence3d(nx: int, ny: int, nz: int, kmin: float = 2.0, kmax: float = 4.0,
                 rms: float = 0.04, seed: int = 1):
    """Decaying 3D MHD turbulence: u and B the discrete curls of band-limited
    random vector potentials, each scaled to sqrt(<|.|^2>) = rms; rho = 1.
    Returns (rho, ux, uy, uz, bx, by, bz), each (nz, ny, nx)."""
    g = _rng(seed)
    out = []
    for _ in range(2):
        pot = [_band_field3(nx, ny, nz, kmin, kmax, g) for _ in range(3)]
        v = curl3(*pot)
        norm = np.sqrt(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
        out.append([c * (rms / norm) if norm > 0 else c for c in v])
    rho = np.ones((nz, ny, nx))
    return (rho, *out[0], *out[1])
