"""The largest lattice the ABI accepts (nx * ny = 2^30 nodes) and a
one-long-row lattice, in the benchmark's FP32 launch shape: every index of
the step, the initialisation, the moments and the diagnostics reductions at
its maximum.  Two GPU steps from an analytic field, then the moments at
sampled nodes against the oracle stepping a 5 x 5 patch around each node
(after two steps the centre depends only on nodes within distance 2, so the
patch's own periodic wrap never reaches it), and mass conservation over the
whole lattice.  Peak device memory 203 GB (FP32 state 163 GB + five FP64
fields)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KW = dict(tau_nu=0.51, tau_eta=0.51, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3)


def fields_at(i, j, nx, ny, xp):
    """rho, ux, uy, bx, by of an Orszag-Tang-like field with a density wave
    at integer coordinates (i, j) (numpy or torch)."""
    x = (2.0 * np.pi / nx) * i
    y = (2.0 * np.pi / ny) * j
    return (1.0 + 0.01 * xp.sin(x + y), -0.05 * xp.sin(y), 0.05 * xp.sin(x),
            -0.05 * xp.sin(y), 0.05 * xp.sin(2.0 * x))


@pytest.mark.parametrize("nx,ny", [(32768, 32768), (1 << 24, 4)])
def test_maximum_size_lattice_sampled(orc, nx, ny):
    import torch

    assert torch.cuda.is_available()
    from paper_1607_08675_gb300 import build, lbmhd as L

    build.build()
    need = 19 * 4 * 2 * nx * ny + 5 * 8 * nx * ny
    free, _ = torch.cuda.mem_get_info()
    if free < need + (8 << 30):
        pytest.skip(f"needs {need / 2**30:.0f} GiB free on the device")
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision="fp32", **KW))
    try:
        dev = torch.device("cuda")
        jj = torch.arange(ny, dtype=torch.float64, device=dev)[:, None]
        ii = torch.arange(nx, dtype=torch.float64, device=dev)[None, :]
        f = [t.expand(ny, nx).contiguous() for t in fields_at(ii, jj, nx, ny, torch)]
        torch.cuda.synchronize()  # the fields are complete before the handle's stream reads them
        mass0 = float(f[0].sum())
        L.lbmhd_init_device(h, *f)
        L.lbmhd_sync(h)
        mass_init = L.lbmhd_diagnostics(h)["mass"]
        del f, ii, jj
        torch.cuda.empty_cache()
        L.lbmhd_step(h, 2)
        m = [torch.empty((ny, nx), dtype=torch.float64, device=dev) for _ in range(5)]
        L.lbmhd_moments_device(h, *m)
        L.lbmhd_sync(h)
        d = L.lbmhd_diagnostics(h)
        rng = np.random.default_rng(3)
        pts = [(0, 0), (nx - 1, ny - 1), (nx - 1, 0), (0, ny - 1), (nx // 2, ny // 2)]
        pts += list(zip(rng.integers(0, nx, 200).tolist(), rng.integers(0, ny, 200).tolist()))
        xs = torch.tensor([p[0] for p in pts], device=dev)
        ys = torch.tensor([p[1] for p in pts], device=dev)
        got = np.stack([t[ys, xs].cpu().numpy() for t in m], axis=1)
        del m
    finally:
        L.lbmhd_destroy(h)
        torch.cuda.empty_cache()
    off = np.arange(-2, 3)
    p = orc.params(**KW)
    for k, (x, y) in enumerate(pts):
        pi = (x + off[None, :]) % nx
        pj = (y + off[:, None]) % ny
        patch = [np.ascontiguousarray(np.broadcast_to(a, (5, 5)))
                 for a in fields_at(pi.astype(np.float64), pj.astype(np.float64), nx, ny, np)]
        ref = orc.moments(orc.step(orc.init(*patch), p, 2))
        want = np.array([r[2, 2] for r in ref])
        assert np.max(np.abs(got[k] - want)) < 1e-6, ((x, y), got[k], want)
    # the steps conserve the stored mass (FP32 rounding random-walks to
    # ~1e-13 relative over 2^30 nodes)
    assert abs(d["mass"] - mass_init) <= 1e-10 * mass_init, (d["mass"], mass_init)
    # FP32 storage holds f itself while the arithmetic measures deviations
    # from the FP32-rounded weights, which sum to 1 + 7.45e-9: the stored
    # mass sits that far below the FP64 input's
    assert abs(mass_init - mass0) <= 1e-8 * mass0, (mass_init, mass0)
