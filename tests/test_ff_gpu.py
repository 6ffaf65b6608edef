"""Double-word ("float-float") storage and arithmetic against the FP64 oracle.

LBMHD_FF keeps every deviation as an FP32 pair (hi, lo) and computes the
collision in double-word arithmetic: unit roundoff 2^-48 against FP64's
2^-53.  The bars below are the FP64 bars of test_parity_gpu.py scaled by
that ratio, 2^5 = 32: 3.2e-11 relative after 200 steps, 3.2e-13 absolute on
populations after 50 steps of a small-amplitude state, 3.2e-12 absolute for
one step of the full-size turbulence workload.
"""
import numpy as np
import pytest

from paper_1607_08675_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("rho-1", "ux", "uy", "bx", "by")
RATIO = 2.0 ** 5  # unit roundoff of double-word over FP64


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


def run_gpu(L, fields, steps, launch=None, **kw):
    ny, nx = fields[0].shape
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(**kw))
    try:
        if launch:
            L.lbmhd_set_launch(h, *launch)
        L.lbmhd_init(h, *fields)
        L.lbmhd_step(h, steps)
        return L.lbmhd_moments(h), L.lbmhd_get_state(h)
    finally:
        L.lbmhd_destroy(h)


def okw(kw):
    keys = ("tau_nu", "tau_eta", "C_S", "delta", "s5", "s6", "s7", "s8", "les")
    return {k: v for k, v in kw.items() if k in keys}


PRESETS = {
    "les": dict(tau_nu=0.6, tau_eta=0.6, C_S=0.1),
    "les_mrt": dict(tau_nu=0.6, tau_eta=0.7, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3),
    "les_off": dict(tau_nu=0.6, tau_eta=0.6, C_S=0.0, les=0),
    "les_strong": dict(tau_nu=0.52, tau_eta=0.55, C_S=0.5, delta=2.0),
}


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("preset", list(PRESETS))
def test_ff_orszag_tang_64_200_steps(L, orc, preset, seed):
    kw = PRESETS[preset]
    fields = inputs.orszag_tang(64, 64, seed=seed)
    ref = orc.step(orc.init(*fields), orc.params(**okw(kw)), 200)
    m, st = run_gpu(L, fields, 200, precision="ff", **kw)
    errs = rel_errs(m, orc.moments(ref))
    assert max(errs.values()) < RATIO * 1e-12, errs
    for p in range(19):
        e = np.max(np.abs(st[p] - ref[p])) / np.max(np.abs(ref[p] - ref[p].mean()))
        assert e < RATIO * 1e-12, (p, e)


def test_ff_is_far_more_accurate_than_fp32(L, orc):
    """The double-word mode sits with FP64, orders of magnitude below the
    FP32 deviation mode on the same run."""
    kw = PRESETS["les_mrt"]
    fields = inputs.orszag_tang(96, 64, seed=2)
    ref = orc.moments(orc.step(orc.init(*fields), orc.params(**okw(kw)), 200))
    e_ff = max(rel_errs(run_gpu(L, fields, 200, precision="ff", **kw)[0], ref).values())
    e_32 = max(rel_errs(run_gpu(L, fields, 200, precision="fp32_dev", **kw)[0], ref).values())
    assert e_ff < 1e-4 * e_32, (e_ff, e_32)


@pytest.mark.parametrize("shape", [(37, 23), (5, 3), (1, 9), (9, 1), (130, 67), (1, 1), (64, 2)])
def test_ff_ragged_and_degenerate_shapes(L, orc, shape):
    nx, ny = shape
    fields = inputs.orszag_tang(nx, ny, seed=4, amp=1e-3)
    kw = PRESETS["les_mrt"]
    ref = orc.step(orc.init(*fields), orc.params(**okw(kw)), 50)
    _, st = run_gpu(L, fields, 50, precision="ff", **kw)
    assert np.max(np.abs(st - ref)) < RATIO * 1e-14


def test_ff_rest_state_is_exact(L):
    """At rest every deviation is zero and the double-word step keeps it
    exactly zero (sqrt at 0, rcp at rho = 1)."""
    n = 32
    z = np.zeros((n, n))
    fields = (np.ones((n, n)), z, z, z, z)
    _, st = run_gpu(L, fields, 10, precision="ff", **PRESETS["les"])
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4 + [0.0] * 10)
    assert np.array_equal(st, np.broadcast_to(w[:, None, None], st.shape))


def test_ff_full_size_turbulence_sampled_one_step(L, orc):
    """1024^2 decaying turbulence in the benchmark's launch shape: after 100
    GPU steps one more step is compared with the oracle's step from the same
    state at 4096 sampled nodes."""
    n = 1024
    fields = inputs.turbulence(n, n, seed=1)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.integers(0, n * n, 4000),
                          [0, n - 1, n * n - 1, n * (n - 1), n * 512 + 1023, 1023 * n + 511]])
    kw = dict(tau_nu=0.51, tau_eta=0.51, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3)
    h = L.lbmhd_create(n, n, L.lbmhd_params_default(precision="ff", **kw))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, 100)
    before = L.lbmhd_get_state(h)
    L.lbmhd_step(h, 1)
    after = L.lbmhd_get_state(h)
    L.lbmhd_destroy(h)
    ref = orc.step_cells(before, orc.params(**kw), idx)
    got = after.reshape(19, -1)[:, idx].T
    assert np.max(np.abs(got - ref)) < RATIO * 1e-13


def test_ff_diagnostics_match_fp64(L, orc):
    """FP64 diagnostics of a double-word state: the conserved sums and the
    energies agree with the oracle's at the double-word bar."""
    kw = PRESETS["les"]
    fields = inputs.orszag_tang(64, 48, seed=3)
    ref = orc.diagnostics(orc.step(orc.init(*fields), orc.params(**okw(kw)), 60))
    h = L.lbmhd_create(64, 48, L.lbmhd_params_default(precision="ff", **kw))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, 60)
    d = L.lbmhd_diagnostics(h)
    L.lbmhd_destroy(h)
    for k in ("mass", "E_kin", "E_mag", "enstrophy", "cross_helicity", "current_sq"):
        assert abs(d[k] - ref[k]) <= RATIO * 1e-11 * abs(ref[k]), (k, d[k], ref[k])


U2 = 2.0 ** -48  # double-word unit roundoff


def _ff_round(x):
    """The nearest double-word (FP32 hi + FP32 lo) to each double, as an
    exact double: the input the device operation actually sees."""
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi.astype(np.float64) + lo.astype(np.float64)


def test_ff_primitives_within_their_error_bounds(L):
    """Each double-word operation against FP64 on 2e5 random operands
    spanning 11 decades and both signs.  Bounds (u^2 = 2^-48), from the
    analyses of the methods named in lbmhd_ff.cuh plus the FP64 reference's
    own rounding: sum 4u^2 (|x| + |y|); product 6u^2 |xy|; reciprocal
    4u^2; square root 8u^2; product by an FP32 constant 3u^2 (exact for a
    power of two); every result normalised, |lo| <= ulp(hi) / 2."""
    rng = np.random.default_rng(11)
    n = 200_000
    mag = lambda: 10.0 ** rng.uniform(-8, 3, n) * rng.choice([-1.0, 1.0], n)
    x, y = mag(), mag()
    # cancellation and special operands
    x[:6] = [1.0, 0.5, 3.0, 1e-3, 2.0 / 3.0, 0.1]
    y[:6] = [-1.0, -0.5, 1.0, -1e-3, -2.0 / 3.0, 0.2]
    xf, yf = _ff_round(x), _ff_round(y)

    r = L.lbmhd_ff_eval("add", x, y)
    assert np.all(np.abs(r - (xf + yf)) <= 4 * U2 * (np.abs(xf) + np.abs(yf)))
    assert np.all(r[[0, 1, 3, 4]] == 0.0)
    r = L.lbmhd_ff_eval("sub", x, y)
    assert np.all(np.abs(r - (xf - yf)) <= 4 * U2 * (np.abs(xf) + np.abs(yf)))
    r = L.lbmhd_ff_eval("mul", x, y)
    assert np.all(np.abs(r - xf * yf) <= 6 * U2 * np.abs(xf * yf))
    r = L.lbmhd_ff_eval("rcp", x)
    assert np.all(np.abs(r * xf - 1.0) <= 4 * U2)
    ax = np.abs(x)
    axf = _ff_round(ax)
    r = L.lbmhd_ff_eval("sqrt", ax)
    assert np.all(np.abs(r - np.sqrt(axf)) <= 8 * U2 * np.sqrt(axf))
    squares = np.array([0.0, 1.0, 4.0, 0.25, 16.0, 2.0 ** -40])
    assert np.array_equal(L.lbmhd_ff_eval("sqrt", squares), np.sqrt(squares))
    pow2 = np.array([1.0, 2.0, 4.0, 0.25, -0.5, 2.0 ** 20])
    assert np.array_equal(L.lbmhd_ff_eval("rcp", pow2), 1.0 / pow2)
    for k in (2.0, 0.25, 0.5, 4.0):
        r = L.lbmhd_ff_eval("kmul", x, np.full(n, k))
        assert np.array_equal(r, xf * k), k
    for k in (3.0, 5.0, 1.0 / 3.0):
        kf = float(np.float32(k))
        r = L.lbmhd_ff_eval("kmul", x, np.full(n, kf))
        assert np.all(np.abs(r - xf * kf) <= 3 * U2 * np.abs(xf * kf)), k
    assert np.max(L.lbmhd_ff_eval("norm", x, y)) <= 0.5
