"""The largest 3D lattice the ABI accepts (nx * ny * nz = 2^30 nodes), as a
cube and as one long x-row of planes, in FP16 deviation storage (the one
format whose two buffers, 193 GB, fit beside seven FP64 fields), in the
default launch shape: every index of the step, the initialisation and the
moments at its maximum.  Two GPU steps from an analytic field, then the
moments at sampled nodes against the 3D oracle stepping a 5 x 5 x 5 patch
around each node (after two steps the centre depends only on nodes within
distance 2, so the patch's own periodic wrap never reaches it), and mass
conservation over the whole lattice.  Peak device memory 253 GB."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KW = dict(tau_nu=0.55, tau_eta=0.6, C_S=0.1, delta=1.0, les=1)


def fields_at(i, j, k, nx, ny, nz, xp):
    """rho, ux, uy, uz, bx, by, bz at integer coordinates (i, j, k), each a
    function of at most two of them (numpy or torch)."""
    x = (2.0 * np.pi / nx) * i
    y = (2.0 * np.pi / ny) * j
    z = (2.0 * np.pi / nz) * k
    return (1.0 + 0.01 * xp.sin(x + z), -0.05 * xp.sin(y), 0.05 * xp.sin(z), 0.05 * xp.sin(x),
            -0.05 * xp.sin(z), 0.05 * xp.sin(2.0 * x), 0.04 * xp.sin(y + z))


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3

    oracle3.build()
    return oracle3


@pytest.mark.parametrize("nx,ny,nz", [(1024, 1024, 1024), (1 << 22, 16, 16)])
def test_maximum_size_3d_lattice_sampled(o3, nx, ny, nz):
    import torch

    assert torch.cuda.is_available()
    from paper_1607_08675_gb300 import build, lbmhd as L

    build.build()
    n = nx * ny * nz
    need = 45 * 2 * 2 * n + 7 * 8 * n
    free, _ = torch.cuda.mem_get_info()
    if free < need + (8 << 30):
        pytest.skip(f"needs {need / 2**30:.0f} GiB free on the device")
    h = L.lbmhd3_create(nx, ny, nz, L.lbmhd_params_default(precision="fp16_dev", **KW))
    dev = torch.device("cuda")
    try:
        ii = torch.arange(nx, dtype=torch.float64, device=dev)[None, None, :]
        jj = torch.arange(ny, dtype=torch.float64, device=dev)[None, :, None]
        kk = torch.arange(nz, dtype=torch.float64, device=dev)[:, None, None]
        f = [t.expand(nz, ny, nx).contiguous() for t in fields_at(ii, jj, kk, nx, ny, nz, torch)]
        # the handle reads the fields on its own stream: they must be complete
        torch.cuda.synchronize()
        L.lbmhd3_init_device(h, *f)
        L.lbmhd3_sync(h)  # the fields are read on the handle's stream
        del f, ii, jj, kk
        torch.cuda.empty_cache()
        out = [torch.empty((nz, ny, nx), dtype=torch.float64, device=dev) for _ in range(7)]
        # mass of the stored initial state (after the FP16 rounding)
        L.lbmhd3_moments_device(h, *out)
        L.lbmhd3_sync(h)
        mass0 = float(out[0].sum())
        L.lbmhd3_step(h, 2)
        L.lbmhd3_moments_device(h, *out)
        L.lbmhd3_sync(h)
        mass2 = float(out[0].sum())
        rng = np.random.default_rng(5)
        pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, nz - 1), (0, ny - 1, 0),
               (nx // 2, ny // 2, nz // 2)]
        pts += list(zip(rng.integers(0, nx, 120).tolist(), rng.integers(0, ny, 120).tolist(),
                        rng.integers(0, nz, 120).tolist()))
        xs = torch.tensor([p[0] for p in pts], device=dev)
        ys = torch.tensor([p[1] for p in pts], device=dev)
        zs = torch.tensor([p[2] for p in pts], device=dev)
        got = np.stack([t[zs, ys, xs].cpu().numpy() for t in out], axis=1)
        del out
    finally:
        L.lbmhd3_destroy(h)
        torch.cuda.empty_cache()
    off = np.arange(-2, 3)
    p = o3.params(**KW)
    for q, (x, y, z) in enumerate(pts):
        pi = ((x + off) % nx).astype(np.float64)[None, None, :]
        pj = ((y + off) % ny).astype(np.float64)[None, :, None]
        pk = ((z + off) % nz).astype(np.float64)[:, None, None]
        patch = [np.ascontiguousarray(np.broadcast_to(a, (5, 5, 5)))
                 for a in fields_at(pi, pj, pk, nx, ny, nz, np)]
        ref = o3.moments(o3.step(o3.init(*patch), p, 2))
        want = np.array([r[2, 2, 2] for r in ref])
        # FP16 storage: each stored deviation rounded to 2^-11 of itself
        # (|d| <= ~0.03 here) at init and after each step, summed over the
        # populations of a moment: well under 2e-4 absolute
        assert np.max(np.abs(got[q] - want)) < 2e-4, ((x, y, z), got[q], want)
    # the steps conserve mass to the FP16 rounding of the stored deviations
    assert abs(mass2 - mass0) <= 1e-6 * mass0, (mass2, mass0)
