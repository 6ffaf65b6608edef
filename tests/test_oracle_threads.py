"""The oracle's OpenMP split (streaming, the kinetic closures' moment and
collision loops, the local-rate collision loop) changes only which thread
computes a node, never how: one thread and several give the same bits,
for the local rates (les 1), the paper's filtered equilibria (les 2) and
the cross-helicity closure (les 3), on a lattice whose rows do not divide
evenly among the threads."""
import numpy as np
import pytest

from paper_1607_08675_gb300 import inputs


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle

    oracle.build()
    return oracle


@pytest.mark.parametrize("les", [1, 2, 3])
def test_thread_count_does_not_change_the_bits(orc, les):
    fields = inputs.orszag_tang(37, 29, seed=4, amp=1e-3)
    p = orc.params(tau_nu=0.6, tau_eta=0.65, C_S=0.1, delta=2.0, les=les)
    st = orc.init(*fields)
    one = orc.step(st, p, 12, nthreads=1)
    for threads in (2, 3, 8):
        assert np.array_equal(orc.step(st, p, 12, nthreads=threads), one), threads
