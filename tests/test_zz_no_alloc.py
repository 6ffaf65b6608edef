"""lbmhd_diagnostics_noalloc: diagnostics for callers that cannot allocate.

A host application that owns all device memory through its own arena, or
a latency-critical loop that cannot take cudaMalloc's implicit device
synchronisation, cannot let the library allocate scratch.  This entry
point reduces a state buffer the caller already holds, keeping its partial
sums in a static device array.  Here it is called through the C ABI on two
lattices in a row and must agree with the handle-based lbmhd_diagnostics
(which uses scratch from lbmhd_create) within the diagnostics tolerance of
the parity tests (1e-11 relative).

This file is collected last on purpose: the other GPU tests have run
before it when a run stops at the first failure.
"""
import numpy as np
import pytest

from paper_1607_08675_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_08675_gb300 import build, lbmhd

    build.build()
    return lbmhd


def _close(a, b, key):
    tol = 1e-11 * max(abs(b), 1e-300)
    if key in ("mom_x", "mom_y", "bsum_x", "bsum_y", "divB_max", "divB_rms"):
        tol = max(tol, 1e-13)
    return abs(a - b) <= tol


def test_noalloc_matches_handle_diagnostics_on_two_calls(L):
    import torch

    runs = [("fp64", 96, 80, torch.float64, 40), ("fp32", 256, 192, torch.float32, 25)]
    for prec, nx, ny, dt, steps in runs:
        h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision=prec))
        L.lbmhd_init(h, *inputs.turbulence(nx, ny, kmin=2, kmax=5, seed=nx))
        L.lbmhd_step(h, steps)
        ref = L.lbmhd_diagnostics(h)
        host_state = L.lbmhd_get_state(h)  # FP32 storage decodes exactly to FP64
        L.lbmhd_destroy(h)
        state = torch.from_numpy(host_state).to(dt).cuda().contiguous()
        assert np.array_equal(state.double().cpu().numpy(), host_state)
        out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
        L.lbmhd_diagnostics_noalloc(state, prec, nx, ny, nx * ny, out)
        got = out.cpu().numpy()
        for q, key in enumerate(L.DIAG_KEYS):
            assert _close(got[q], ref[key], key), (prec, key, got[q], ref[key])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_dev", "fp16_dev", "ff"])
@pytest.mark.parametrize("pad", [0, 3])
@pytest.mark.parametrize("shape", [(123, 77), (128, 77)])
def test_noalloc_every_stored_format_bitwise(L, prec, pad, shape):
    """The raw stored state of every format, laid out with a plane stride of
    nx*ny + pad elements: the handle's own diagnostics bit for bit -- the
    same work split and arithmetic over the same values.  With nx = 128 the
    4-byte formats (FP32, FP32 deviations) take the reduction's wide form
    (16-byte copies of aligned row windows) in the handle and the unpadded
    layout, and its per-lane copies in the padded one (plane starts off
    16-byte boundaries); FP16 always loads its values per lane into
    registers, FP64 and FF always copy per lane; nx = 123 takes the
    per-lane form throughout."""
    import torch

    nx, ny = shape
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision=prec))
    L.lbmhd_init(h, *inputs.turbulence(nx, ny, kmin=2, kmax=5, seed=7))
    L.lbmhd_step(h, 30)
    ref = L.lbmhd_diagnostics(h)
    raw = L.lbmhd_get_state_raw(h)
    L.lbmhd_destroy(h)
    if raw.dtype == np.uint16:
        raw = raw.view(np.int16)
    tail = raw.shape[3:]
    ps = nx * ny + pad
    buf = np.zeros((19, ps) + tail, dtype=raw.dtype)
    buf[:, : nx * ny] = raw.reshape((19, nx * ny) + tail)
    state = torch.from_numpy(buf).cuda()
    out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
    L.lbmhd_diagnostics_noalloc(state, prec, nx, ny, ps, out)
    got = out.cpu().numpy()
    for q, key in enumerate(L.DIAG_KEYS):
        assert got[q] == ref[key], (prec, pad, key, got[q], ref[key])


def test_noalloc_wide_and_per_lane_forms_share_one_split(L):
    """FP32 at 2048^2, where the number of resident warps (not the row
    count) bounds the work split: the handle's state (16-byte aligned, the
    wide form) and the same values with planes off 16-byte boundaries (the
    per-lane form) give the same bits, because both forms take one plan."""
    import torch

    nx = ny = 2048
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision="fp32"))
    L.lbmhd_init(h, *inputs.turbulence(nx, ny, kmin=4, kmax=8, seed=11))
    L.lbmhd_step(h, 5)
    ref = L.lbmhd_diagnostics(h)
    raw = L.lbmhd_get_state_raw(h)
    L.lbmhd_destroy(h)
    for pad in (0, 1):
        ps = nx * ny + pad
        buf = torch.zeros((19, ps), dtype=torch.float32)
        buf[:, : nx * ny] = torch.from_numpy(raw.reshape(19, nx * ny))
        state = buf.cuda()
        out = torch.full((12,), float("nan"), dtype=torch.float64, device="cuda")
        L.lbmhd_diagnostics_noalloc(state, "fp32", nx, ny, ps, out)
        got = out.cpu().numpy()
        for q, key in enumerate(L.DIAG_KEYS):
            assert got[q] == ref[key], (pad, key, got[q], ref[key])


def test_noalloc_rejects_misaligned_pointers(L):
    """A state pointer off the stored value size, or an out pointer off 8
    bytes (as a caller's arena may hand out), is refused with EINVAL before
    any launch; the properly aligned call on the same buffers works."""
    import torch

    nx, ny = 8, 4
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    for prec, size in (("fp64", 8), ("ff", 8), ("fp32", 4), ("fp16_dev", 2)):
        st = torch.zeros(19 * nx * ny * size + 64, dtype=torch.uint8, device="cuda")
        for off in sorted({1, size // 2} - {0}):
            with pytest.raises(L.LBMHDError) as e:
                L.lbmhd_diagnostics_noalloc(st.data_ptr() + off, prec, nx, ny, nx * ny,
                                            out.data_ptr())
            assert e.value.code == -1
    st = torch.zeros(19 * nx * ny + 1, dtype=torch.float64, device="cuda")
    for off in (1, 4):
        with pytest.raises(L.LBMHDError) as e:
            L.lbmhd_diagnostics_noalloc(st, "fp64", nx, ny, nx * ny, out.data_ptr() + off)
        assert e.value.code == -1
    # one double in: every plane and the 12 sums still inside their buffers
    L.lbmhd_diagnostics_noalloc(st.data_ptr() + 8, "fp64", nx, ny, nx * ny, out.data_ptr() + 8)
    torch.cuda.synchronize()
    assert out[1:13].cpu().numpy()[0] == 0.0  # mass of an all-zero state


def test_noalloc_rejects_oversized_and_bad_arguments(L):
    import torch

    out = torch.zeros(12, dtype=torch.float64, device="cuda")
    st = torch.zeros(19 * 16, dtype=torch.float64, device="cuda")
    for args in [(1 << 16, 1 << 15, (1 << 31)), (4, 4, 15), (0, 4, 16)]:
        with pytest.raises(L.LBMHDError) as e:
            L.lbmhd_diagnostics_noalloc(st, "fp64", *args, out)
        assert e.value.code == -1
    with pytest.raises(L.LBMHDError):
        L.lbmhd_diagnostics_noalloc(st, 9, 4, 4, 16, out)
