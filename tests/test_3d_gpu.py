"""The 3D step (D3Q27 + D3Q7) on the GPU against the 3D oracle, through the
lbmhd3_* C ABI: every population plane and the moments after many steps on
ragged lattices (FP64 to the 1e-12 bar, FP32 and FP16 deviation storage to
their storage bars), with LES
off, the local LES rates, the paper's filtered equilibria (kinetic LES) and
the cross-helicity closure; identical bits across launch shapes; the
diagnostics; one step at sampled nodes of a larger lattice in the default
launch shape; the refused configurations."""
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


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3

    oracle3.build()
    return oracle3


KW = dict(tau_nu=0.58, tau_eta=0.62, C_S=0.15, delta=1.5)


def gpu3(L, fields, steps, vec=None, block=None, **kw):
    nz, ny, nx = fields[0].shape
    h = L.lbmhd3_create(nx, ny, nz, L.lbmhd_params_default(**kw))
    if vec is not None:
        L.lbmhd3_set_launch(h, vec, block)
    L.lbmhd3_init(h, *fields)
    L.lbmhd3_step(h, steps)
    m = L.lbmhd3_moments(h)
    st = L.lbmhd3_get_state(h)
    d = L.lbmhd3_diagnostics(h)
    assert L.lbmhd3_step_count(h) == steps
    L.lbmhd3_destroy(h)
    return m, st, d


def okw(kw):
    return dict(tau_nu=kw["tau_nu"], tau_eta=kw["tau_eta"], C_S=kw["C_S"], delta=kw["delta"],
                les=kw.get("les", 1))


def rel_fields(m, ref):
    """Per field: max |gpu - oracle| / max |oracle|.  rho is measured as
    itself: in these divergence-free starts rho - 1 is only pressure
    fluctuation that the sound damping takes from 1e-2 to 3e-4 in 100
    steps, while the FP64 rounding of rho ~ 1 stays ~1e-14 (measured: every
    population within 3.2e-15 of the oracle), so a bar relative to
    max |rho - 1| would measure that damping, not the step."""
    out = {}
    for name, a, b in zip(("rho", "ux", "uy", "uz", "bx", "by", "bz"), m, ref):
        out[name] = np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
    return out


@pytest.mark.parametrize("les", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(12, 10, 8), (16, 6, 9), (20, 14, 12)])
def test_fp64_matches_oracle(L, o3, les, shape):
    """Moments relative to their maxima at the 1e-12 bar after 100 steps, on
    lattices whose largest scales survive that long (band 1 <= |n| <= 2),
    and every population plane to 1e-14."""
    nx, ny, nz = shape
    fields = inputs.turbulence3d(nx, ny, nz, kmin=1, kmax=2, rms=0.05, seed=nx)
    kw = dict(KW, les=les, precision="fp64")
    steps = 100
    ref = o3.step(o3.init(*fields), o3.params(**okw(kw)), steps)
    m, st, _ = gpu3(L, fields, steps, **kw)
    e = rel_fields(m, o3.moments(ref))
    assert max(e.values()) < 1e-12, e
    assert np.max(np.abs(st - ref)) < 1e-14


@pytest.mark.parametrize("les", [1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 6, 5), (9, 1, 4), (5, 3, 1), (7, 5, 3),
                                   (2, 2, 2)])
def test_fp64_degenerate_shapes(L, o3, les, shape):
    """One-node, one-row, one-column and one-plane lattices (every neighbour
    along a size-1 axis is the node itself; along a size-2 axis both
    neighbours are the same node) and a small odd lattice: every population
    to 1e-14 after 25 steps."""
    nx, ny, nz = shape
    rng = np.random.default_rng(4)
    fields = (1 + 0.01 * rng.random((nz, ny, nx)),) + tuple(
        0.02 * rng.standard_normal((nz, ny, nx)) for _ in range(6))
    kw = dict(KW, les=les, precision="fp64")
    ref = o3.step(o3.init(*fields), o3.params(**okw(kw)), 25)
    _, st, _ = gpu3(L, fields, 25, **kw)
    assert np.max(np.abs(st - ref)) < 1e-14


@pytest.mark.parametrize("les", [0, 1, 2, 3])
def test_fp32_matches_oracle(L, o3, les):
    fields = inputs.turbulence3d(16, 12, 10, kmin=1, kmax=3, rms=0.05, seed=9)
    kw = dict(KW, les=les, precision="fp32")
    steps = 100
    ref = o3.step(o3.init(*fields), o3.params(**okw(kw)), steps)
    m, _, _ = gpu3(L, fields, steps, **kw)
    e = rel_fields(m, o3.moments(ref))
    assert max(e.values()) < 2e-4, e


@pytest.mark.parametrize("les", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(12, 10, 8), (16, 6, 9)])
def test_double_word_matches_oracle(L, o3, les, shape):
    """Double-word deviations (hi + lo of two FP32 numbers, unit roundoff
    2^-48) on the FP32 pipes: the FP64 bars times 2^5, the ratio of the
    unit roundoffs -- moments 3.2e-11 relative to their maxima after 100
    steps, every population 3.2e-13."""
    nx, ny, nz = shape
    fields = inputs.turbulence3d(nx, ny, nz, kmin=1, kmax=2, rms=0.05, seed=nx)
    kw = dict(KW, les=les, precision="ff")
    ref = o3.step(o3.init(*fields), o3.params(**okw(kw)), 100)
    m, st, _ = gpu3(L, fields, 100, **kw)
    e = rel_fields(m, o3.moments(ref))
    assert max(e.values()) < 3.2e-11, e
    assert np.max(np.abs(st - ref)) < 3.2e-13, np.max(np.abs(st - ref))


@pytest.mark.parametrize("les", [0, 1, 2, 3])
def test_fp16_deviations_match_oracle(L, o3, les):
    """FP16 storage of the deviations f - w (g itself) times the storage
    scale 1024, FP32 arithmetic: 100 steps within 2e-3 of the FP64 oracle
    per field relative to its maximum (measured up to 7.8e-4: the binary16
    rounding, 2^-11 relative, of every stored deviation each step)."""
    fields = inputs.turbulence3d(16, 12, 10, kmin=1, kmax=3, rms=0.05, seed=9)
    kw = dict(KW, les=les, precision="fp16_dev")
    ref = o3.step(o3.init(*fields), o3.params(**okw(kw)), 100)
    m, _, _ = gpu3(L, fields, 100, **kw)
    e = rel_fields(m, o3.moments(ref))
    assert max(e.values()) < 2e-3, e


def test_fp16_one_step_is_the_rounded_oracle_step(L, o3):
    """One step from a developed FP16 state: every population of every
    node is the oracle's step of the same stored state (decoded exactly)
    up to the binary16 rounding of its deviation (half an ulp, 2^-11
    relative) and the FP32 arithmetic."""
    nx, ny, nz = 24, 10, 8
    fields = inputs.turbulence3d(nx, ny, nz, kmin=1, kmax=3, rms=0.05, seed=3)
    c, w, _, _ = o3.lattice()
    rest = np.concatenate([w, np.zeros(18)])[:, None, None, None]
    for les in (1, 2, 3):
        kw = dict(KW, les=les, precision="fp16_dev")
        h = L.lbmhd3_create(nx, ny, nz, L.lbmhd_params_default(**kw))
        L.lbmhd3_init(h, *fields)
        L.lbmhd3_step(h, 10)
        before = L.lbmhd3_get_state(h)
        L.lbmhd3_step(h, 1)
        after = L.lbmhd3_get_state(h)
        L.lbmhd3_destroy(h)
        ref = o3.step(before, o3.params(**okw(kw)), 1)
        bound = 2.0 ** -11 * np.abs(ref - rest) + 2e-7
        assert np.all(np.abs(after - ref) <= bound), (les, np.max(np.abs(after - ref) - bound))


@pytest.mark.parametrize("les", [1, 2, 3])
def test_launch_shapes_give_identical_bits(L, les):
    fields = inputs.turbulence3d(32, 8, 6, seed=2)
    shapes = ((1, 128), (2, 128), (1, 64), (2, 256))
    if les >= 2:  # and the fused one-pass kernel
        shapes += ((0, 8),)
    for prec in ("fp64", "fp32", "fp16_dev", "ff"):
        sts = [gpu3(L, fields, 30, vec, block, precision=prec, **dict(KW, les=les))[1]
               for vec, block in shapes]
        assert all(np.array_equal(sts[0], s) for s in sts[1:]), (prec, les)


@pytest.mark.parametrize("les", [2, 3])
@pytest.mark.parametrize("shape", [(33, 17, 5), (70, 9, 3), (5, 3, 1), (1, 1, 1), (2, 2, 2),
                                   (40, 40, 40)])
def test_fused_closure_kernel_is_the_two_pass_kernel(L, les, shape):
    """Ragged tiles (x not a multiple of 32, y not of 4), planes fewer than
    the ring, one-node and size-2 axes, and a lattice of many segments: the
    fused kernel's bits are the two-pass kernel's."""
    nx, ny, nz = shape
    rng = np.random.default_rng(nx + ny + nz)
    fields = (1 + 0.01 * rng.random((nz, ny, nx)),) + tuple(
        0.02 * rng.standard_normal((nz, ny, nx)) for _ in range(6))
    for prec in ("fp32", "fp64", "fp16_dev", "ff"):
        kw = dict(KW, les=les, precision=prec)
        ref = gpu3(L, fields, 12, 1, 128, **kw)[1]
        got = gpu3(L, fields, 12, 0, 8, **kw)[1]
        assert np.array_equal(got, ref), prec


@pytest.mark.parametrize("les", [2, 3])
@pytest.mark.parametrize("shape", [(33, 17, 5), (70, 9, 3), (5, 3, 1), (1, 1, 1), (2, 2, 2),
                                   (40, 40, 40), (96, 40, 48), (4, 3, 2), (36, 11, 7), (8, 1, 1),
                                   (12, 5, 3)])
def test_warp_specialised_kernel_is_the_two_pass_kernel(L, les, shape):
    """The warp-specialised kernel (vec 3, tiles of 32 x 8 columns) on ragged
    tiles, one-node and size-2 axes, planes fewer than its rings, and a
    lattice of many units (96 x 40 x 48: 15 tiles, segments of a few planes,
    so each persistent CTA runs units one after another and its producer and
    consumer counters wrap the rings across units): bit for bit the two-pass
    kernel's result after 12 steps, in FP32 and FP16 storage (4 x 3 x 2: one
    tile wrapping on both sides; 36 x 11 x 7: a last tile of 4 columns)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(nx + ny + nz)
    fields = (1 + 0.01 * rng.random((nz, ny, nx)),) + tuple(
        0.02 * rng.standard_normal((nz, ny, nx)) for _ in range(6))
    for prec in ("fp32", "fp16_dev"):
        kw = dict(KW, les=les, precision=prec)
        ref = gpu3(L, fields, 12, 1, 128, **kw)[1]
        got = gpu3(L, fields, 12, 3, 8, **kw)[1]
        assert np.array_equal(got, ref), prec


def test_warp_specialised_kernel_timeout_is_reported_not_hung(L):
    """Host-requested fault: the producer warps stop announcing their planes,
    so the consumers' bounded waits expire; the step returns, the next
    synchronising call reports ETIMEOUT, and after a fresh init the handle
    steps correctly again."""
    fields = inputs.turbulence3d(64, 24, 20, seed=5)
    kw = dict(KW, les=2, precision="fp32")
    ref = gpu3(L, fields, 3, 1, 128, **kw)[1]
    h = L.lbmhd3_create(64, 24, 20, L.lbmhd_params_default(**kw))
    assert L.lbmhd3_get_launch(h) == (3, 8)
    L.lbmhd3_init(h, *fields)
    L.lbmhd3_debug(h, L.DEBUG_DROP_BARRIER_ARRIVAL)
    L.lbmhd3_step(h, 1)
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd3_sync(h)
    assert e.value.code == -5
    L.lbmhd3_debug(h, 0)
    L.lbmhd3_init(h, *fields)
    L.lbmhd3_step(h, 3)
    got = L.lbmhd3_get_state(h)
    L.lbmhd3_destroy(h)
    assert np.array_equal(got, ref)


def test_warp_specialised_kernel_on_a_plane_range(L):
    """Plane ranges (the z-slab step) through the warp-specialised kernel:
    three ranges and a commit equal one whole step."""
    fields = inputs.turbulence3d(64, 24, 20, seed=4)
    kw = dict(KW, les=2, precision="fp32")
    ref = gpu3(L, fields, 1, 1, 128, **kw)[1]
    h = L.lbmhd3_create(64, 24, 20, L.lbmhd_params_default(**kw))
    L.lbmhd3_set_launch(h, 3, 8)
    L.lbmhd3_init(h, *fields)
    for z0, z1 in ((0, 7), (7, 8), (8, 20)):
        L.lbmhd3_step_planes(h, z0, z1)
    L.lbmhd3_step_commit(h)
    got = L.lbmhd3_get_state(h)
    assert L.lbmhd3_launch_count(h) == 3
    L.lbmhd3_destroy(h)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("les", [2, 3])
def test_gradient_closure_launches_per_step(L, les):
    """Two launches per step in the two-pass form, one in the fused form."""
    fields = inputs.turbulence3d(8, 6, 4, seed=3)
    for vec, block, per_step in ((1, 128, 2), (0, 128, 1), (3, 8, 1)):
        h = L.lbmhd3_create(8, 6, 4, L.lbmhd_params_default(precision="fp32", les=les, **KW))
        L.lbmhd3_set_launch(h, vec, block)
        L.lbmhd3_init(h, *fields)
        L.lbmhd3_step(h, 5)
        assert L.lbmhd3_launch_count(h) == 5 * per_step and L.lbmhd3_step_count(h) == 5
        L.lbmhd3_destroy(h)


def test_diagnostics_match_oracle(L, o3):
    fields = inputs.turbulence3d(12, 10, 8, kmin=1, kmax=3, seed=5)
    kw = dict(KW, les=1, precision="fp64")
    _, st, d = gpu3(L, fields, 20, **kw)
    ref = o3.diagnostics(st)
    for k, v in ref.items():
        tol = 1e-12 * max(abs(v), 1.0) if k in ("mass",) else 1e-11 * max(abs(v), 1e-3)
        if k.startswith(("mom", "bsum")):
            tol = 1e-12 * ref["mass"]
        if k.startswith("divB"):
            tol = 1e-12 * max(abs(v), 1e-6)
        assert abs(d[k] - v) <= tol, (k, d[k], v)


@pytest.mark.parametrize("les", [1, 2, 3])
def test_sampled_step_of_a_larger_lattice(L, o3, les):
    """128 x 96 x 64 (786,432 nodes, the default launch shape), FP32: one
    step from a developed state, 3,000 sampled nodes against the oracle's
    step of the same stored state (decoded exactly)."""
    nx, ny, nz = 128, 96, 64
    fields = inputs.turbulence3d(nx, ny, nz, seed=11)
    kw = dict(KW, les=les, precision="fp32")
    h = L.lbmhd3_create(nx, ny, nz, L.lbmhd_params_default(**kw))
    L.lbmhd3_init(h, *fields)
    L.lbmhd3_step(h, 10)
    before = L.lbmhd3_get_state(h)
    L.lbmhd3_step(h, 1)
    after = L.lbmhd3_get_state(h).reshape(45, -1)
    L.lbmhd3_destroy(h)
    idx = np.random.default_rng(1).integers(0, nx * ny * nz, 3000)
    ref = o3.step_cells(before, o3.params(**okw(kw)), idx)
    got = after[:, idx].T
    # FP32 arithmetic of one collision on values of size ~0.3: a few ulp
    assert np.max(np.abs(got - ref)) < 2e-7, np.max(np.abs(got - ref))


def test_refused_configurations(L):
    for bad in (dict(les=4), dict(les=-1), dict(precision="fp32_dev"), dict(tau_nu=0.5),
                dict(precision="fp16_dev", fp16_scale=0.0)):
        with pytest.raises(L.LBMHDError) as e:
            L.lbmhd3_create(8, 8, 8, L.lbmhd_params_default(**dict(dict(precision="fp32"), **bad)))
        assert e.value.code == -1
    h = L.lbmhd3_create(6, 4, 4, L.lbmhd_params_default(precision="fp32"))
    with pytest.raises(L.LBMHDError):
        L.lbmhd3_step(h, 1)  # before init
    with pytest.raises(L.LBMHDError):
        L.lbmhd3_set_launch(h, 4, 128)
    with pytest.raises(L.LBMHDError):
        L.lbmhd3_set_launch(h, 0, 8)  # the fused kernel is for les 2, 3
    with pytest.raises(L.LBMHDError):
        L.lbmhd3_set_launch(h, 3, 8)  # and so is the warp-specialised one
    L.lbmhd3_destroy(h)
    h = L.lbmhd3_create(6, 4, 4, L.lbmhd_params_default(precision="fp32", les=2))
    assert L.lbmhd3_get_launch(h) == (3, 8)  # FP32 closures: the warp-specialised kernel
    for block in (2, 4, 16):
        with pytest.raises(L.LBMHDError):
            L.lbmhd3_set_launch(h, 3, block)  # 8 tile rows
    L.lbmhd3_destroy(h)
    for prec in ("fp64", "ff"):  # FP32 arithmetic only
        h = L.lbmhd3_create(6, 4, 4, L.lbmhd_params_default(precision=prec, les=3))
        with pytest.raises(L.LBMHDError):
            L.lbmhd3_set_launch(h, 3, 8)
        L.lbmhd3_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16_dev", "ff"])
def test_checkpoint_resume_and_device_io(L, prec):
    """Checkpoint / resume: a run interrupted after 17 steps, its state read
    out and written into a fresh handle, continues bit for bit as the
    uninterrupted run -- through the raw stored values for every format,
    through FP64 planes for FP64, FP32 and FP16 storage.  Initialisation
    and moments through device fields equal the host-array calls."""
    import torch

    shape = (18, 10, 7)
    nx, ny, nz = shape
    fields = inputs.turbulence3d(*shape, kmin=1, kmax=3, rms=0.05, seed=12)
    kw = dict(KW, les=1, precision=prec)
    ref = gpu3(L, fields, 30, **kw)[1]
    a = L.lbmhd3_create(*shape, L.lbmhd_params_default(**kw))
    L.lbmhd3_init(a, *fields)
    L.lbmhd3_step(a, 17)
    raw, fp = L.lbmhd3_get_state_raw(a), L.lbmhd3_get_state(a)
    L.lbmhd3_destroy(a)
    routes = [("raw", raw)] + ([("fp64", fp)] if prec != "ff" else [])
    for name, st in routes:
        b = L.lbmhd3_create(*shape, L.lbmhd_params_default(**kw))
        (L.lbmhd3_set_state_raw if name == "raw" else L.lbmhd3_set_state)(b, st)
        L.lbmhd3_step(b, 13)
        assert np.array_equal(L.lbmhd3_get_state(b), ref), name
        L.lbmhd3_destroy(b)
    # device fields
    dev = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in fields]
    torch.cuda.synchronize()  # complete before the handle's stream reads them
    c = L.lbmhd3_create(*shape, L.lbmhd_params_default(**kw))
    L.lbmhd3_init_device(c, *dev)
    L.lbmhd3_step(c, 30)
    out = [torch.empty_like(dev[0]) for _ in range(7)]
    L.lbmhd3_moments_device(c, *out)
    torch.cuda.synchronize()
    assert np.array_equal(L.lbmhd3_get_state(c), ref)
    host = L.lbmhd3_moments(c)
    for q in range(7):
        assert np.array_equal(out[q].cpu().numpy(), host[q])
    with pytest.raises(ValueError):
        L.lbmhd3_set_state_raw(c, raw[:-1])
    import ctypes
    assert L.lib().lbmhd3_set_state_raw(c.ptr, raw.ctypes.data_as(ctypes.c_void_p), raw.nbytes - 1) == -1
    L.lbmhd3_destroy(c)


@pytest.mark.parametrize("prec", ["fp32", "fp16_dev"])
def test_non_finite_detection(L, prec):
    """check_finite_every = 1: a clean run is unchanged and reports nothing;
    a NaN written into one population of one node (a host-side injection)
    is reported as ENONFINITE by the next synchronising call; a new init
    clears the report."""
    shape = (16, 8, 6)
    fields = inputs.turbulence3d(*shape, seed=13)
    kw = dict(KW, les=1, precision=prec)
    ref = gpu3(L, fields, 12, **kw)[1]
    h = L.lbmhd3_create(*shape, L.lbmhd_params_default(check_finite_every=1, **kw))
    L.lbmhd3_init(h, *fields)
    L.lbmhd3_step(h, 12)
    L.lbmhd3_sync(h)
    assert np.array_equal(L.lbmhd3_get_state(h), ref)
    st = L.lbmhd3_get_state(h)
    st[13, 3, 4, 5] = np.nan
    L.lbmhd3_set_state(h, st)
    L.lbmhd3_step(h, 2)
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd3_sync(h)
    assert "non-finite" in str(e.value)
    with pytest.raises(L.LBMHDError):
        L.lbmhd3_moments(h)
    L.lbmhd3_init(h, *fields)
    L.lbmhd3_step(h, 2)
    L.lbmhd3_sync(h)
    L.lbmhd3_destroy(h)
    with pytest.raises(L.LBMHDError):
        L.lbmhd3_create(*shape, L.lbmhd_params_default(check_finite_every=-1, **kw))
