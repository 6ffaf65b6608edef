"""The hand-written CUDA adjoint against the brute-force FP64 tape oracle
(oracle/tape.py, PyTorch autograd on a from-the-paper step), against
central finite differences of the CUDA forward, and across checkpoint
spacings.  Tolerances: FP64 adjoint vs tape 1e-10 relative (the two differ
only in rounding order); vs finite differences 1e-6 relative (h = 1e-6:
truncation ~1e-12, rounding ~1e-10); FP32 adjoint vs FP64 adjoint 5e-3
relative on the parameter gradients and 1e-2 on the field gradients
(FP32 arithmetic over the whole backward sweep)."""
import numpy as np
import pytest

from paper_1607_08675_gb300 import inputs

pytestmark = pytest.mark.gpu

MRT = dict(s5=1.2, s6=1.25, s7=1.3, s8=1.35)


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_08675_gb300 import autograd, build, lbmhd

    build.build()
    return lbmhd, autograd, torch


def cuda(torch, arrs):
    return [torch.tensor(a, dtype=torch.float64, device="cuda") for a in arrs]


def adjoint(L, torch, fields, weights, th, steps, every, prec="fp64", rates=None):
    ny, nx = fields[0].shape
    p = L.lbmhd_params_default(precision=prec, tau_nu=th[1], tau_eta=th[2], C_S=th[0],
                               **(rates or {}))
    h = L.lbmhd_create(nx, ny, p)
    L.lbmhd_adjoint_record(h, *cuda(torch, fields), steps, every)
    dth, df = L.lbmhd_adjoint_backward(h, cuda(torch, weights))
    out = [t.cpu().numpy() for t in df]
    L.lbmhd_destroy(h)
    return np.array(dth), out


def forward_value(L, torch, fields, weights, th, steps, prec="fp64", rates=None):
    ny, nx = fields[0].shape
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(precision=prec, tau_nu=th[1],
                                                      tau_eta=th[2], C_S=th[0], **(rates or {})))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, steps)
    m = L.lbmhd_moments(h)
    L.lbmhd_destroy(h)
    return sum(float((a * w).sum()) for a, w in zip(m, weights))


@pytest.mark.parametrize("rates", [None, MRT])
def test_fp64_adjoint_equals_tape_oracle(env, rates):
    from oracle import tape

    L, _, torch = env
    fields = inputs.orszag_tang(16, 16, seed=2, amp=1e-3)
    rng = np.random.default_rng(3)
    weights = [rng.standard_normal((16, 16)) for _ in range(5)]
    th = (0.15, 0.6, 0.65)
    steps = 20
    kw = {} if rates is None else dict(rates=(rates["s5"], rates["s6"], rates["s7"], rates["s8"]))
    _, ref = tape.gradients(fields, th[1], th[2], th[0], steps, weights, **kw)
    dth, df = adjoint(L, torch, fields, weights, th, steps, 7, rates=rates)
    for got, key in zip(dth, ("C_S", "tau_nu", "tau_eta")):
        assert abs(got - ref[key]) <= 1e-10 * abs(ref[key]), (key, got, ref[key])
    for got, key in zip(df, ("rho0", "ux0", "uy0", "bx0", "by0")):
        scale = np.max(np.abs(ref[key]))
        assert np.max(np.abs(got - ref[key])) <= 1e-10 * scale, key


def test_fp64_adjoint_equals_finite_differences(env):
    L, _, torch = env
    n, steps = 48, 60
    fields = inputs.orszag_tang(n, n, seed=5)
    rng = np.random.default_rng(4)
    weights = [rng.standard_normal((n, n)) for _ in range(5)]
    th = (0.1, 0.6, 0.6)
    dth, df = adjoint(L, torch, fields, weights, th, steps, 16, rates=MRT)
    for i in range(3):
        h = 1e-6 * th[i]
        up = list(th)
        dn = list(th)
        up[i] += h
        dn[i] -= h
        fd = (forward_value(L, torch, fields, weights, up, steps, rates=MRT) -
              forward_value(L, torch, fields, weights, dn, steps, rates=MRT)) / (2 * h)
        assert abs(fd - dth[i]) <= 1e-6 * abs(fd), (i, fd, dth[i])
    d = [rng.standard_normal((n, n)) * s for s in (1e-3, 1.0, 1.0, 1.0, 1.0)]
    h = 1e-7
    up = [a + h * b for a, b in zip(fields, d)]
    dn = [a - h * b for a, b in zip(fields, d)]
    fd = (forward_value(L, torch, up, weights, th, steps, rates=MRT) -
          forward_value(L, torch, dn, weights, th, steps, rates=MRT)) / (2 * h)
    ad = sum(float((g * b).sum()) for g, b in zip(df, d))
    assert abs(fd - ad) <= 1e-6 * abs(fd)


def test_checkpoint_spacing_does_not_change_gradients(env):
    L, _, torch = env
    fields = inputs.orszag_tang(64, 40, seed=6)
    rng = np.random.default_rng(5)
    weights = [rng.standard_normal((40, 64)) for _ in range(5)]
    th = (0.1, 0.55, 0.6)
    base = adjoint(L, torch, fields, weights, th, 45, 45)
    for every in (1, 7, 100):
        got = adjoint(L, torch, fields, weights, th, 45, every)
        assert np.array_equal(got[0], base[0])
        for a, b in zip(got[1], base[1]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp32", "fp32_dev"])
def test_fp32_adjoint_against_fp64_adjoint(env, prec):
    L, _, torch = env
    n = 64
    fields = inputs.orszag_tang(n, n, seed=8)
    rng = np.random.default_rng(6)
    weights = [rng.standard_normal((n, n)) for _ in range(5)]
    th = (0.1, 0.6, 0.6)
    d64, f64 = adjoint(L, torch, fields, weights, th, 100, 25, rates=MRT)
    d32, f32 = adjoint(L, torch, fields, weights, th, 100, 25, prec=prec, rates=MRT)
    assert np.max(np.abs(d32 - d64) / np.abs(d64)) < 5e-3, (d32, d64)
    for a, b in zip(f32, f64):
        assert np.max(np.abs(a - b)) < 1e-2 * np.max(np.abs(b))


def test_autograd_function_misfit_gradients(env):
    """loss = 1/2 sum |u - u_ref|^2 + |B - B_ref|^2 with the reference run at
    C_S = 0.12: torch.autograd through Rollout equals the direct ABI call."""
    L, AG, torch = env
    n, steps = 32, 40
    fields = inputs.orszag_tang(n, n, seed=9)
    f = cuda(torch, fields)
    with torch.no_grad():
        ref = AG.rollout(*f, 0.12, 0.6, 0.6, steps, every=10)
    leaves = [t.clone().requires_grad_(True) for t in f]
    th = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (0.1, 0.6, 0.6)]
    out = AG.rollout(*leaves, *th, steps, every=10)
    loss = 0.5 * sum(((o - r) ** 2).sum() for o, r in zip(out[1:], ref[1:]))
    loss.backward()
    weights = [np.zeros((n, n))] + [(o - r).detach().cpu().numpy() for o, r in zip(out[1:], ref[1:])]
    dth, df = adjoint(L, torch, fields, weights, (0.1, 0.6, 0.6), steps, 10)
    got = [float(t.grad) for t in th]
    assert np.allclose(got, dth, rtol=1e-12, atol=0)
    for leaf, b in zip(leaves, df):
        assert np.allclose(leaf.grad.cpu().numpy(), b, rtol=1e-12, atol=1e-300)
    assert loss.item() > 0


def test_adjoint_errors(env):
    L, _, torch = env
    h = L.lbmhd_create(16, 16, L.lbmhd_params_default(precision="fp16_dev"))
    f = cuda(torch, inputs.orszag_tang(16, 16))
    with pytest.raises(L.LBMHDError):
        L.lbmhd_adjoint_record(h, *f, 10, 5)
    L.lbmhd_destroy(h)
    h = L.lbmhd_create(16, 16, L.lbmhd_params_default(precision="fp64"))
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd_adjoint_backward(h, [None] * 5)
    assert e.value.code == -7
    L.lbmhd_adjoint_record(h, *f, 10, 5)
    L.lbmhd_step(h, 1)
    with pytest.raises(L.LBMHDError) as e:
        L.lbmhd_adjoint_backward(h, [None] * 5)
    assert e.value.code == -7
    L.lbmhd_destroy(h)


# Double-word (FF) adjoint: the FP64 bars scaled by the ratio of the unit
# roundoffs, 2^-48 / 2^-53 = 32.
FF_RATIO = 2.0 ** 5


@pytest.mark.parametrize("rates", [None, MRT])
def test_ff_adjoint_equals_tape_oracle(env, rates):
    """Double-word storage and adjoint against the brute-force FP64 tape
    oracle: the FP64 adjoint's 1e-10 bar times 32."""
    from oracle import tape

    L, _, torch = env
    fields = inputs.orszag_tang(16, 16, seed=2, amp=1e-3)
    rng = np.random.default_rng(3)
    weights = [rng.standard_normal((16, 16)) for _ in range(5)]
    th = (0.15, 0.6, 0.65)
    steps = 20
    kw = {} if rates is None else dict(rates=(rates["s5"], rates["s6"], rates["s7"], rates["s8"]))
    _, ref = tape.gradients(fields, th[1], th[2], th[0], steps, weights, **kw)
    dth, df = adjoint(L, torch, fields, weights, th, steps, 7, prec="ff", rates=rates)
    for got, key in zip(dth, ("C_S", "tau_nu", "tau_eta")):
        assert abs(got - ref[key]) <= FF_RATIO * 1e-10 * abs(ref[key]), (key, got, ref[key])
    for got, key in zip(df, ("rho0", "ux0", "uy0", "bx0", "by0")):
        scale = np.max(np.abs(ref[key]))
        assert np.max(np.abs(got - ref[key])) <= FF_RATIO * 1e-10 * scale, key


def test_ff_adjoint_against_fp64_adjoint(env):
    """On the 64^2 case of the FP32 comparison: the double-word adjoint sits
    with FP64 (3.2e-9), orders of magnitude below FP32's 5e-3."""
    L, _, torch = env
    n = 64
    fields = inputs.orszag_tang(n, n, seed=8)
    rng = np.random.default_rng(6)
    weights = [rng.standard_normal((n, n)) for _ in range(5)]
    th = (0.1, 0.6, 0.6)
    d64, f64 = adjoint(L, torch, fields, weights, th, 100, 25, rates=MRT)
    dff, fff = adjoint(L, torch, fields, weights, th, 100, 25, prec="ff", rates=MRT)
    assert np.max(np.abs(dff - d64) / np.abs(d64)) < FF_RATIO * 1e-10, (dff, d64)
    for a, b in zip(fff, f64):
        assert np.max(np.abs(a - b)) < FF_RATIO * 1e-10 * np.max(np.abs(b))
