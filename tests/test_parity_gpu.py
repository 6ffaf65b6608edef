"""CUDA path vs the FP64 CPU oracle, through the C ABI.

Tolerances (per field F in {rho - 1, u_x, u_y, B_x, B_y} and per population
plane, relative to max|F_oracle|):
  * FP64 storage and arithmetic: 1e-12 after 200 steps.  The only
    differences are rounding order and FMA contraction (~1e-16 per step).
  * FP32 storage / arithmetic: FP32 rounding of populations of size ~0.4
    (f) is ~3e-8 absolute per step; against fields of size ~5e-2 that is
    a few 1e-6 relative after 200 steps -> 2e-4 stated with margin.
  * FP32 deviation storage: the stored deviations are ~1e-2, so rounding
    drops ~40x -> 3e-5.
  * FP16 deviation storage: 11-bit mantissa, ~5e-4 relative per stored
    value -> 2e-2 on u and B, 5e-2 on rho - 1 (a small difference of large
    terms).
"""
import numpy as np
import pytest

from paper_1607_08675_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("rho-1", "ux", "uy", "bx", "by")


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_08675_gb300 import build, lbmhd

    build.build()
    return lbmhd


def rel_errs(got, ref):
    out = {}
    for name, a, b in zip(FIELDS, got, ref):
        if name == "rho-1":
            a, b = a - 1.0, b - 1.0
        out[name] = float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
    return out


def run_gpu(L, fields, steps, **kw):
    ny, nx = fields[0].shape
    launch = kw.pop("launch", None)
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(**kw))
    try:
        if launch:
            L.lbmhd_set_launch(h, *launch)
        L.lbmhd_init(h, *fields)
        L.lbmhd_step(h, steps)
        return L.lbmhd_moments(h), L.lbmhd_get_state(h), L.lbmhd_diagnostics(h)
    finally:
        L.lbmhd_destroy(h)


def oracle_kw(kw):
    keys = ("tau_nu", "tau_eta", "C_S", "delta", "s5", "s6", "s7", "s8", "les")
    return {k: v for k, v in kw.items() if k in keys}


PRESETS = {
    "les": dict(tau_nu=0.6, tau_eta=0.6, C_S=0.1),
    "les_mrt": dict(tau_nu=0.6, tau_eta=0.7, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3),
    "les_off": dict(tau_nu=0.6, tau_eta=0.6, C_S=0.0, les=0),
    "les_strong": dict(tau_nu=0.52, tau_eta=0.55, C_S=0.5, delta=2.0),
}


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("preset", list(PRESETS))
def test_fp64_orszag_tang_64_200_steps(L, orc, preset, seed):
    """Orszag-Tang 64^2, 200 steps, FP64: every field and every population
    plane within 1e-12 relative of the oracle."""
    kw = PRESETS[preset]
    fields = inputs.orszag_tang(64, 64, seed=seed)
    ref = orc.step(orc.init(*fields), orc.params(**oracle_kw(kw)), 200)
    m, st, _ = run_gpu(L, fields, 200, precision="fp64", **kw)
    errs = rel_errs(m, orc.moments(ref))
    assert max(errs.values()) < 1e-12, errs
    for p in range(19):
        e = np.max(np.abs(st[p] - ref[p])) / np.max(np.abs(ref[p] - ref[p].mean()))
        assert e < 1e-12, (p, e)


@pytest.mark.parametrize("shape", [(37, 23), (5, 3), (1, 9), (9, 1), (130, 67), (1, 1), (64, 2)])
def test_fp64_ragged_and_degenerate_shapes(L, orc, shape):
    nx, ny = shape
    fields = inputs.orszag_tang(nx, ny, seed=4, amp=1e-3)
    kw = PRESETS["les_mrt"]
    ref = orc.step(orc.init(*fields), orc.params(**oracle_kw(kw)), 50)
    _, st, _ = run_gpu(L, fields, 50, precision="fp64", **kw)
    assert np.max(np.abs(st - ref)) < 1e-14


SHAPES = ((1, 256), (2, 128), (4, 64), (4, 256), (1, 32), (2, 96), (8, 64), (8, 32), (0, 128),
          (0, 256), (0, 512))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_dev", "fp16_dev", "ff"])
@pytest.mark.parametrize("shape", [(512, 40), (256, 3), (128, 1), (1024, 2)])
def test_launch_shapes_give_identical_results(L, prec, shape):
    """The result does not depend on the kernel or its launch shape: the
    register kernel at every vector width and block size and the TMA-staged
    kernel at every tile width (including one tile per row, where both
    periodic granules wrap, and one-row lattices) give the same bits."""
    nx, ny = shape
    fields = inputs.orszag_tang(nx, ny, seed=1)
    base, n = None, 0
    for launch in SHAPES:
        if prec == "fp64" and launch[0] in (0, 4):
            continue
        if launch[0] == 8 and prec != "fp16_dev":
            continue
        if launch[0] == 0 and prec == "ff":
            continue
        if launch[0] == 0 and nx % launch[1]:
            continue
        _, st, _ = run_gpu(L, fields, 70, precision=prec, launch=launch, **PRESETS["les"])
        n += 1
        if base is None:
            base = st
        else:
            assert np.array_equal(st, base), launch
    assert n >= 4


def test_graph_replay_equals_single_launches(L):
    """lbmhd_step(n) with n >= 64 replays a captured graph; splitting the same
    run into short calls must give the same bits."""
    fields = inputs.orszag_tang(64, 48, seed=3)
    nx, ny = 64, 48
    outs = []
    for chunks in ([200], [1] * 7 + [63, 1, 129], [33] * 6 + [2]):
        h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision="fp32", **PRESETS["les"]))
        L.lbmhd_init(h, *fields)
        for c in chunks:
            L.lbmhd_step(h, c)
        assert L.lbmhd_step_count(h) == 200
        outs.append(L.lbmhd_get_state(h))
        L.lbmhd_destroy(h)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


TOL32 = {"fp32": 2e-4, "fp32_dev": 3e-5}


@pytest.mark.parametrize("prec", ["fp32", "fp32_dev", "fp16_dev"])
def test_reduced_precision_against_fp64_oracle(L, orc, prec):
    kw = PRESETS["les"]
    fields = inputs.orszag_tang(64, 64, seed=0)
    ref = orc.step(orc.init(*fields), orc.params(**oracle_kw(kw)), 200)
    m, _, _ = run_gpu(L, fields, 200, precision=prec, **kw)
    errs = rel_errs(m, orc.moments(ref))
    if prec == "fp16_dev":
        assert errs["rho-1"] < 5e-2 and max(errs[k] for k in FIELDS[1:]) < 2e-2, errs
    else:
        assert max(errs.values()) < TOL32[prec], errs


def test_moments_and_diagnostics_match_oracle(L, orc):
    kw = PRESETS["les_mrt"]
    fields = inputs.turbulence(96, 80, kmin=2, kmax=5, seed=2)
    ref = orc.step(orc.init(*fields), orc.params(**oracle_kw(kw)), 60)
    m, _, d = run_gpu(L, fields, 60, precision="fp64", **kw)
    for a, b in zip(m, orc.moments(ref)):
        assert np.max(np.abs(a - b)) < 1e-14
    dref = orc.diagnostics(ref)
    for k, v in dref.items():
        scale = max(abs(v), 1e-3 * abs(dref["E_kin"]) if k.startswith("divB") else abs(v))
        if k in ("mom_x", "mom_y", "bsum_x", "bsum_y"):
            scale = dref["mass"] * 1e-3
        assert abs(d[k] - v) <= 1e-11 * max(scale, 1e-300), (k, d[k], v)
    assert d["step"] == 60


DIAG_TOL = {"fp64": 1e-11, "ff": 32 * 1e-11, "fp32": 1e-6, "fp32_dev": 1e-6, "fp16_dev": 1e-6}


@pytest.mark.parametrize("prec", ["fp64", "ff", "fp32", "fp16_dev"])
@pytest.mark.parametrize("shape", [(1, 1), (2, 1), (1, 2), (9, 1), (1, 9), (5, 3), (31, 7),
                                   (61, 2), (30, 30), (30007, 53), (4, 5), (8, 3), (248, 9)])
def test_diagnostics_ragged_shapes_match_oracle(L, orc, prec, shape):
    """The diagnostics of the stored state against the oracle's of the same
    state (decoded exactly): lattices narrower than one 30-column strip, one
    node wide or high (both neighbours of a node are one node), strips with
    a ragged last set of columns, and a 30007 x 53 lattice whose 1001
    strips are cut into segments of several rows with a shorter last one
    (53 is prime), so a warp's row ring wraps several times per segment;
    and 16-byte aligned rows (nx = 4, 8, 248), where the FP32 form copies
    aligned windows whose granules wrap around short rows more than once,
    with a ragged last strip at 248 (FP16 loads per lane whatever the
    alignment).  Bars: the format's relative
    bar on every quantity; the sums of rho u and B to that bar times the
    mass (FP32 forms: 1e-9 of it); div B to the bar times the rms B."""
    nx, ny = shape
    kw = PRESETS["les_mrt"]
    fields = inputs.orszag_tang(nx, ny, seed=6)
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision=prec, **kw))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, 20)
    got = L.lbmhd_diagnostics(h)
    ref = orc.diagnostics(L.lbmhd_get_state(h))
    L.lbmhd_destroy(h)
    tol = DIAG_TOL[prec]
    floor = tol * (ref["E_kin"] + ref["E_mag"])
    for k in ("mass", "E_kin", "E_mag", "enstrophy", "cross_helicity", "current_sq"):
        assert abs(got[k] - ref[k]) <= tol * abs(ref[k]) + floor, (k, got[k], ref[k])
    sums = 1e-9 if prec in ("fp32", "fp32_dev", "fp16_dev") else tol
    for k in ("mom_x", "mom_y", "bsum_x", "bsum_y"):
        assert abs(got[k] - ref[k]) <= sums * ref["mass"], (k, got[k], ref[k])
    brms = np.sqrt(2.0 * ref["E_mag"])
    for k in ("divB_max", "divB_rms"):
        assert abs(got[k] - ref[k]) <= tol * brms, (k, got[k], ref[k])


def test_diagnostics_deterministic(L):
    fields = inputs.turbulence(256, 256, seed=5)
    h = L.lbmhd_create(256, 256, L.lbmhd_params_default(precision="fp32"))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, 10)
    a = L.lbmhd_diagnostics(h)
    b = L.lbmhd_diagnostics(h)
    L.lbmhd_destroy(h)
    assert a == b


def test_full_size_turbulence_sampled_one_step(L, orc):
    """1024^2 decaying turbulence in the launch shape the benchmark times:
    after 100 GPU steps, one more GPU step is compared with the oracle's
    step at 4096 sampled nodes (FP64: 1e-13 absolute; FP32: from the FP32
    state, 2e-7 absolute on populations)."""
    n = 1024
    fields = inputs.turbulence(n, n, seed=1)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.integers(0, n * n, 4000),
                          [0, n - 1, n * n - 1, n * (n - 1), n * 512 + 1023, 1023 * n + 511]])
    kw = dict(tau_nu=0.51, tau_eta=0.51, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3)
    for prec, tol in (("fp64", 1e-13), ("fp32", 2e-7)):
        h = L.lbmhd_create(n, n, L.lbmhd_params_default(precision=prec, **kw))
        L.lbmhd_init(h, *fields)
        L.lbmhd_step(h, 100)
        before = L.lbmhd_get_state(h)
        L.lbmhd_step(h, 1)
        after = L.lbmhd_get_state(h)
        L.lbmhd_destroy(h)
        ref = orc.step_cells(before, orc.params(**kw), idx)
        got = after.reshape(19, -1)[:, idx].T
        assert np.max(np.abs(got - ref)) < tol, prec


def test_checkpoint_resume_is_bitwise(L):
    fields = inputs.orszag_tang(64, 64, seed=7)
    for prec in ("fp64", "fp16_dev"):
        p = L.lbmhd_params_default(precision=prec)
        a = L.lbmhd_create(64, 64, p)
        L.lbmhd_init(a, *fields)
        L.lbmhd_step(a, 150)
        ref = L.lbmhd_get_state(a)
        b = L.lbmhd_create(64, 64, p)
        L.lbmhd_init(b, *fields)
        L.lbmhd_step(b, 70)
        ck = L.lbmhd_get_state(b)
        L.lbmhd_destroy(b)
        c = L.lbmhd_create(64, 64, p)
        L.lbmhd_set_state(c, ck)
        L.lbmhd_step(c, 80)
        assert np.array_equal(L.lbmhd_get_state(c), ref), prec
        L.lbmhd_destroy(a)
        L.lbmhd_destroy(c)


def test_conservation_and_div_b_on_gpu(L):
    fields = inputs.orszag_tang(64, 64, seed=1)
    h = L.lbmhd_create(64, 64, L.lbmhd_params_default(tau_nu=0.6, tau_eta=1.0, les=0, C_S=0.0))
    L.lbmhd_init(h, *fields)
    d0 = L.lbmhd_diagnostics(h)
    L.lbmhd_step(h, 300)
    d1 = L.lbmhd_diagnostics(h)
    L.lbmhd_destroy(h)
    assert abs(d1["mass"] - d0["mass"]) < 1e-12 * d0["mass"]
    for k in ("mom_x", "mom_y", "bsum_x", "bsum_y"):
        assert abs(d1[k] - d0[k]) < 1e-12 * d0["mass"]
    assert d1["divB_max"] < 1e-15  # s_m = 1: machine zero (central differences)


def test_nonfinite_detection_and_errors(L):
    fields = inputs.orszag_tang(32, 32, seed=0)
    h = L.lbmhd_create(32, 32, L.lbmhd_params_default(precision="fp32", check_finite_every=5))
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd_step(h, 1)
    assert e.value.code == -7  # ESTATE before init
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, 10)
    L.lbmhd_sync(h)
    st = L.lbmhd_get_state(h)
    st[3, 5, 7] = np.nan  # injected on the host
    L.lbmhd_set_state(h, st)
    L.lbmhd_step(h, 10)
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd_sync(h)
    assert e.value.code == -4
    # the handle stays usable: a clean re-init clears the report
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, 10)
    L.lbmhd_sync(h)
    bad = [f.copy() for f in fields]
    bad[0][0, 0] = -1.0
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd_init(h, *bad)
    assert e.value.code == -1
    L.lbmhd_destroy(h)


def test_device_entry_points_match_host(L):
    import torch

    fields = inputs.orszag_tang(64, 32, seed=2)
    dev = [torch.from_numpy(f).cuda() for f in fields]
    torch.cuda.synchronize()
    a = L.lbmhd_create(64, 32)
    L.lbmhd_init_device(a, *dev)
    L.lbmhd_step(a, 20)
    out = [torch.empty_like(t) for t in dev]
    L.lbmhd_moments_device(a, *out)
    L.lbmhd_sync(a)
    m, _, _ = run_gpu(L, fields, 20)
    for t, ref in zip(out, m):
        assert np.array_equal(t.cpu().numpy(), ref)
    L.lbmhd_destroy(a)


def test_pinned_and_pageable_host_fields_give_the_same_bits(L):
    """lbmhd_init / lbmhd_moments read and write pinned host arrays in place
    and stage pageable ones through device copies: same bits either way."""
    import torch

    nx, ny = 96, 80
    fields = inputs.turbulence(nx, ny, kmin=2, kmax=5, seed=5)
    pinned = [torch.from_numpy(a).pin_memory().numpy() for a in fields]
    outs = []
    for src in (fields, pinned):
        h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision="fp32", **PRESETS["les"]))
        L.lbmhd_init(h, *src)
        L.lbmhd_step(h, 20)
        pg = L.lbmhd_moments(h)
        pn = [torch.empty((ny, nx), dtype=torch.float64).pin_memory().numpy() for _ in range(5)]
        L.lbmhd_moments_into(h, *pn)
        outs.append((L.lbmhd_get_state(h), pg, pn))
        L.lbmhd_destroy(h)
    assert np.array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][2]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
@pytest.mark.parametrize("pin", [False, True])
def test_init_rejects_bad_density_on_the_device(L, bad, pin):
    import torch

    nx, ny = 40, 24
    fields = [a.copy() for a in inputs.orszag_tang(nx, ny, seed=2)]
    good = [a.copy() for a in fields]
    fields[0][7, 13] = bad
    if pin:
        fields = [torch.from_numpy(a).pin_memory().numpy() for a in fields]
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision="fp64"))
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd_init(h, *fields)
    assert e.value.code == -1
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd_step(h, 1)
    assert e.value.code == -7  # ESTATE: not initialised
    L.lbmhd_init(h, *good)
    L.lbmhd_step(h, 3)
    m = L.lbmhd_moments(h)
    assert np.isfinite(m[0]).all() and L.lbmhd_step_count(h) == 3
    L.lbmhd_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_dev", "fp16_dev", "ff"])
def test_raw_checkpoint_resume_is_bitwise(L, prec):
    """lbmhd_get_state_raw / lbmhd_set_state_raw keep every format bit for bit
    (the FP64 view of lbmhd_get_state rounds double-word pairs)."""
    fields = inputs.orszag_tang(64, 48, seed=7)
    p = L.lbmhd_params_default(precision=prec, **PRESETS["les_mrt"])
    a = L.lbmhd_create(64, 48, p)
    L.lbmhd_init(a, *fields)
    L.lbmhd_step(a, 150)
    ref = L.lbmhd_get_state_raw(a)
    b = L.lbmhd_create(64, 48, p)
    L.lbmhd_init(b, *fields)
    L.lbmhd_step(b, 70)
    ck = L.lbmhd_get_state_raw(b)
    assert ck.nbytes == 64 * 48 * L.lbmhd_bytes_per_cell(prec) // 2
    L.lbmhd_destroy(b)
    c = L.lbmhd_create(64, 48, p)
    L.lbmhd_set_state_raw(c, ck)
    L.lbmhd_step(c, 80)
    got = L.lbmhd_get_state_raw(c)
    assert got.view(np.uint8).tobytes() == ref.view(np.uint8).tobytes()
    # the raw values decode to the FP64 view
    st = L.lbmhd_get_state(c)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4 + [0.0] * 10)[:, None, None]
    if prec in ("fp64", "fp32"):
        dec = got.astype(np.float64)
    elif prec == "fp32_dev":
        dec = w + got.astype(np.float64)
    elif prec == "fp16_dev":
        dec = w + got.astype(np.float64) / 1024.0
    else:
        dec = w + (got[..., 0].astype(np.float64) + got[..., 1].astype(np.float64))
    assert np.max(np.abs(dec - st)) <= 1e-15
    rc = L.lib().lbmhd_set_state_raw(c.ptr, got.ctypes.data_as(__import__("ctypes").c_void_p),
                                     got.nbytes - 1)
    assert rc == -1  # EINVAL: wrong byte count
    L.lbmhd_destroy(a)
    L.lbmhd_destroy(c)


@pytest.mark.parametrize("prec", ["fp32", "fp32_dev", "fp16_dev"])
def test_reduced_precision_diagnostics_match_fp64_of_the_same_state(L, orc, prec):
    """The diagnostics of the FP32 and FP16 forms form each node's terms in
    FP32 and sum them in double-word: against the oracle's FP64 diagnostics
    of the same stored state (decoded exactly) the energies, enstrophy,
    cross helicity and <j^2> agree to 1e-6 relative, the sums of rho, rho u
    and B and the div B norms to FP32 rounding of the terms."""
    n = 256
    fields = inputs.turbulence(n, n, kmin=2, kmax=6, seed=4)
    h = L.lbmhd_create(n, n, L.lbmhd_params_default(precision=prec, **PRESETS["les_mrt"]))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, 40)
    got = L.lbmhd_diagnostics(h)
    ref = orc.diagnostics(L.lbmhd_get_state(h))
    L.lbmhd_destroy(h)
    for k in ("mass", "E_kin", "E_mag", "enstrophy", "cross_helicity", "current_sq"):
        assert abs(got[k] - ref[k]) <= 1e-6 * abs(ref[k]), (k, got[k], ref[k])
    for k in ("mom_x", "mom_y", "bsum_x", "bsum_y"):
        assert abs(got[k] - ref[k]) <= 1e-9 * ref["mass"], (k, got[k], ref[k])
    # central differences of B formed in FP32: ~1e-7 of |B| each
    brms = np.sqrt(2.0 * ref["E_mag"])
    for k in ("divB_max", "divB_rms"):
        assert abs(got[k] - ref[k]) <= 1e-6 * brms, (k, got[k], ref[k])
