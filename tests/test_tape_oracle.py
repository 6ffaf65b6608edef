"""Pins of the brute-force FP64 gradient oracle (oracle/tape.py): its
forward must equal the C oracle's step, and its tape gradients must equal
central finite differences of the C oracle (an independent code path)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import tape  # noqa: E402
from paper_1607_08675_gb300 import inputs  # noqa: E402

KW = dict(tau_nu=0.6, tau_eta=0.65, C_S=0.15)
RATES = (1.2, 1.25, 1.3, 1.35)


def oracle_final(orc, fields, steps, tau_nu, tau_eta, C_S, rates=(0, 0, 0, 0)):
    p = orc.params(tau_nu=tau_nu, tau_eta=tau_eta, C_S=C_S, s5=rates[0], s6=rates[1],
                   s7=rates[2], s8=rates[3])
    return orc.moments(orc.step(orc.init(*fields), p, steps))


@pytest.mark.parametrize("rates", [(0, 0, 0, 0), RATES])
def test_tape_forward_equals_c_oracle(orc, rates):
    fields = inputs.orszag_tang(16, 12, seed=3, amp=1e-3)
    ref = oracle_final(orc, fields, 12, **KW, rates=rates)
    t = [torch.tensor(a) for a in fields]
    out = tape.rollout(*t, torch.tensor(KW["tau_nu"], dtype=torch.float64),
                       torch.tensor(KW["tau_eta"], dtype=torch.float64),
                       torch.tensor(KW["C_S"], dtype=torch.float64), 12, rates=rates)
    for a, b in zip(out, ref):
        assert np.max(np.abs(a.numpy() - b)) < 1e-14


def test_tape_gradients_equal_finite_differences_of_c_oracle(orc):
    fields = inputs.orszag_tang(12, 12, seed=4, amp=1e-3)
    rng = np.random.default_rng(1)
    weights = [rng.standard_normal((12, 12)) for _ in range(5)]
    steps = 8
    val, grads = tape.gradients(fields, KW["tau_nu"], KW["tau_eta"], KW["C_S"], steps, weights)

    def F(fl, tn, te, cs):
        out = oracle_final(orc, fl, steps, tn, te, cs)
        return sum(float((o * w).sum()) for o, w in zip(out, weights))

    assert abs(F(fields, **{"tn": KW["tau_nu"], "te": KW["tau_eta"], "cs": KW["C_S"]}) - val) < 1e-12
    for name, key in (("tau_nu", "tn"), ("tau_eta", "te"), ("C_S", "cs")):
        base = dict(tn=KW["tau_nu"], te=KW["tau_eta"], cs=KW["C_S"])
        h = 1e-6
        up, dn = dict(base), dict(base)
        up[key] += h
        dn[key] -= h
        fd = (F(fields, **up) - F(fields, **dn)) / (2 * h)
        assert abs(fd - grads[name]) < 1e-6 * max(abs(fd), 1e-3), (name, fd, grads[name])
    # a random direction in the initial velocity and field
    d = [np.zeros((12, 12))] + [rng.standard_normal((12, 12)) for _ in range(4)]
    h = 1e-7
    up = [a + h * b for a, b in zip(fields, d)]
    dn = [a - h * b for a, b in zip(fields, d)]
    fd = (F(up, KW["tau_nu"], KW["tau_eta"], KW["C_S"]) -
          F(dn, KW["tau_nu"], KW["tau_eta"], KW["C_S"])) / (2 * h)
    ad = sum(float((grads[n] * b).sum()) for n, b in zip(("rho0", "ux0", "uy0", "bx0", "by0"), d))
    assert abs(fd - ad) < 1e-6 * abs(fd)
