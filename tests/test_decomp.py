"""y-slab domain decomposition: the halo plan on CPU, the exchange over
gloo send/recv between two CPU ranks stepping their slabs with the oracle,
and k slabs on one GPU through lbmhd_copy_rows -- all bit for bit equal to
the undivided lattice."""
import os
import socket
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_1607_08675_gb300 import decomp, inputs


def test_split_and_plan():
    assert decomp.split_rows(10, 3) == [(0, 4), (4, 7), (7, 10)]
    mv = decomp.plan(10, 3)
    # every ghost row of every slab is written exactly once
    targets = sorted((d, r) for _, _, d, r in mv)
    assert targets == [(0, 0), (0, 5), (1, 0), (1, 4), (2, 0), (2, 4)]
    # global row identities: the row sent is the global row the ghost mirrors
    rows = decomp.split_rows(10, 3)
    for s, sr, d, dr in mv:
        g_src = rows[s][0] + sr - 1
        g_dst = (rows[d][0] + dr - 1) % 10
        assert g_src == g_dst
    with pytest.raises(ValueError):
        decomp.split_rows(3, 4)


@pytest.mark.parametrize("ghost", [1, 2])
@pytest.mark.parametrize("ny,k", [(10, 3), (12, 1), (9, 4), (7, 2)])
def test_plan_with_ghost_depth(ghost, ny, k):
    """Two ghost rows per side (kinetic closures): every ghost row of every
    slab is written exactly once, by the global row it mirrors."""
    if min(b - a for a, b in decomp.split_rows(ny, k)) < ghost:
        with pytest.raises(ValueError):
            decomp.plan(ny, k, ghost)
        return
    rows = decomp.split_rows(ny, k)
    mv = decomp.plan(ny, k, ghost)
    want = sorted([(s, i) for s in range(k) for i in range(ghost)] +
                  [(s, ghost + (b - a) + i) for s, (a, b) in enumerate(rows) for i in range(ghost)])
    assert sorted((d, r) for _, _, d, r in mv) == want
    for s, sr, d, dr in mv:
        assert ghost <= sr < ghost + rows[s][1] - rows[s][0]  # an interior row
        assert (rows[s][0] + sr - ghost) % ny == (rows[d][0] + dr - ghost) % ny


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nx, ny, steps, q, les=1):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from oracle import oracle
    from paper_1607_08675_gb300 import decomp as D, inputs as I

    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = oracle.params(tau_nu=0.6, tau_eta=0.65, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3,
                      les=les, delta=2.0)
    g = D.ghost_rows(les)
    fields = D.slab_fields(I.orszag_tang(nx, ny, seed=3), ny, world, g)[rank]
    st = oracle.init(*fields)
    moves = D.plan(ny, world, g)
    for _ in range(steps):
        st = oracle.step(st, p, 1)
        reqs, recv = [], []
        for s, sr, d, dr in moves:
            if s == rank and d == rank:
                st[:, dr] = st[:, sr]
            elif s == rank:
                reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(st[:, sr])), d))
            elif d == rank:
                buf = torch.empty((19, nx), dtype=torch.float64)
                reqs.append(dist.irecv(buf, s))
                recv.append((dr, buf))
        for r in reqs:
            r.wait()
        for dr, buf in recv:
            st[:, dr] = buf.numpy()
    q.put((rank, st[:, g:-g].copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("les", [1, 2])
def test_gloo_two_ranks_match_undivided_oracle(orc, les):
    """Two ranks, each stepping its slab with the oracle, exchanging ghost
    rows by send/recv: the undivided oracle run bit for bit -- one ghost row
    per side with local rates, two with the paper's kinetic LES."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    nx, ny, steps = 16, 13, 12
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, nx, ny, steps, q, les))
             for r in range(2)]
    for p in procs:
        p.start()
    parts = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([parts[0], parts[1]], axis=1)
    ref = orc.step(orc.init(*inputs.orszag_tang(nx, ny, seed=3)),
                   orc.params(tau_nu=0.6, tau_eta=0.65, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3,
                              les=les, delta=2.0),
                   steps)
    assert np.array_equal(got, ref)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16_dev", "ff"])
@pytest.mark.parametrize("k", [1, 3, 4])
def test_slabs_on_one_gpu_match_monolithic(prec, k):
    import torch

    assert torch.cuda.is_available()
    from paper_1607_08675_gb300 import build, lbmhd as L

    build.build()
    nx, ny, steps = 128, 50, 60
    kw = dict(precision=prec, tau_nu=0.6, tau_eta=0.65, C_S=0.1)
    fields = inputs.orszag_tang(nx, ny, seed=5)
    sl = decomp.SlabLattice(nx, ny, k, **kw)
    sl.init(*fields)
    sl.step(steps)
    got = sl.state()
    sl.close()
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(**kw))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, steps)
    ref = L.lbmhd_get_state(h)
    L.lbmhd_destroy(h)
    assert np.array_equal(got, ref)


@pytest.mark.gpu
@pytest.mark.parametrize("les", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16_dev", "ff"])
@pytest.mark.parametrize("k", [1, 3])
def test_kinetic_slabs_on_one_gpu_match_monolithic(prec, k, les):
    """The kinetic closures with two ghost rows per side: bit for bit the
    undivided lattice."""
    import torch

    assert torch.cuda.is_available()
    from paper_1607_08675_gb300 import build, lbmhd as L

    build.build()
    nx, ny, steps = 96, 50, 40
    kw = dict(precision=prec, tau_nu=0.6, tau_eta=0.65, C_S=0.1, les=les, delta=2.0)
    fields = inputs.orszag_tang(nx, ny, seed=8)
    sl = decomp.SlabLattice(nx, ny, k, **kw)
    sl.init(*fields)
    sl.step(steps)
    got = sl.state()
    sl.close()
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(**kw))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, steps)
    ref = L.lbmhd_get_state(h)
    L.lbmhd_destroy(h)
    assert np.array_equal(got, ref)
