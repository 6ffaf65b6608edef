"""y-slab domain decomposition: the halo messages on CPU, the exchange of
decomp.exchange over gloo between two CPU ranks stepping their slabs with
the oracle, and k slabs on one GPU through the same exchange with the
device store (lbmhd_pack_row / lbmhd_unpack_row, lbmhd_step_rows) -- all
bit for bit equal to the undivided lattice."""
import os
import socket
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_1607_08675_gb300 import decomp, inputs

CY = {p: c for p, c in enumerate(decomp.PLANE_CY)}


def test_plane_sets():
    """The planes that stream up, down and along x: the D2Q9 and D2Q5 lists
    of Sec. 3 (f_2, f_5, f_6 and g_2 up; f_4, f_7, f_8 and g_4 down)."""
    assert decomp.planes_of(decomp.UP) == [2, 5, 6, 13, 14]
    assert decomp.planes_of(decomp.DOWN) == [4, 7, 8, 17, 18]
    assert decomp.planes_of(decomp.REST) == [0, 1, 3, 9, 10, 11, 12, 15, 16]
    assert decomp.UP | decomp.DOWN | decomp.REST == (1 << 19) - 1


def _needed(les, ghost):
    """Brute force: for every interior row of a slab, the (ghost row, plane)
    pairs its step reads -- the pull of the row itself and, with the kinetic
    closures, the pulls of the rows whose moments its gradients use."""
    need = set()
    n = 2 * ghost + 3
    interior = range(ghost, ghost + n)
    reach = 1 if les < 2 else 2
    for y in interior:
        pulled_rows = {y} if les < 2 else {y - 1, y, y + 1}
        for r in pulled_rows:
            for p in range(19):
                src = r - CY[p]
                if src < ghost or src >= ghost + n:
                    need.add((src, p))
    assert all(abs(r - ghost) <= reach or abs(r - (ghost + n - 1)) <= reach for r, _ in need)
    return need, n


@pytest.mark.parametrize("les", [1, 2])
def test_messages_carry_exactly_what_the_ghost_rows_feed(les):
    """The message parts received by a slab write exactly the (ghost row,
    plane) pairs its interior rows read (brute force over the pull), nothing
    more; the rows sent are the global rows the ghosts mirror."""
    g = decomp.ghost_rows(les)
    need, n = _needed(les, g)
    ny, k = 3 * n, 3
    rows = decomp.split_rows(ny, k)
    msgs = decomp.halo_messages(ny, k, g)
    got = {}
    for m in msgs:
        for sr, dr, mask in m.parts:
            assert g <= sr < g + rows[m.src][1] - rows[m.src][0]  # an interior row
            gs = (rows[m.src][0] + sr - g) % ny
            gd = (rows[m.dst][0] + dr - g) % ny
            assert gs == gd
            for p in decomp.planes_of(mask):
                key = (m.dst, dr, p)
                assert key not in got
                got[key] = m
    for s in range(k):
        assert {(r, p) for (d, r, p) in got if d == s} == need, (les, s)
    vals = sum(m.nvalues(10) for m in msgs) // (2 * k * 10)
    assert vals == (5 if les < 2 else 19)  # values per cut and direction, in nx units


@pytest.mark.parametrize("ny,k,ghost", [(10, 3, 1), (12, 1, 1), (9, 4, 2), (7, 2, 2), (3, 4, 1)])
def test_message_plan_shapes(ny, k, ghost):
    if k > ny or min(b - a for a, b in decomp.split_rows(ny, k)) < ghost:
        with pytest.raises(ValueError):
            decomp.halo_messages(ny, k, ghost)
        return
    msgs = decomp.halo_messages(ny, k, ghost)
    assert len(msgs) == 2 * k
    assert all(len(m.parts) == ghost for m in msgs)
    assert decomp.halo_bytes_per_step(64, ny, k, 2 * (ghost - 1) + 1, 4) == \
        sum(m.nvalues(64) for m in msgs) * 4


def test_exchange_on_host_slabs_matches_global_rows():
    """decomp.exchange with the host store and no communicator fills every
    ghost plane the messages name with the mirrored global row's values, and
    leaves every other value alone."""
    nx, ny, k = 6, 11, 3
    for les in (1, 2):
        g = decomp.ghost_rows(les)
        glob = np.arange(19 * ny * nx, dtype=np.float64).reshape(19, ny, nx)
        rows = decomp.split_rows(ny, k)
        slabs = {}
        for s, (a, b) in enumerate(rows):
            st = np.full((19, b - a + 2 * g, nx), -1.0)
            st[:, g:g + b - a] = glob[:, a:b]
            slabs[s] = st
        decomp.exchange(decomp.halo_messages(ny, k, g), slabs, decomp.HostStore(nx))
        for m in decomp.halo_messages(ny, k, g):
            for _, dr, mask in m.parts:
                gy = (rows[m.dst][0] + dr - g) % ny
                p = decomp.planes_of(mask)
                assert np.array_equal(slabs[m.dst][p, dr], glob[p, gy])
        for s, st in slabs.items():
            n = rows[s][1] - rows[s][0]
            assert np.array_equal(st[:, g:g + n], glob[:, rows[s][0]:rows[s][1]])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, nx, ny, steps, q, les=1, k=2):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from oracle import oracle
    from paper_1607_08675_gb300 import decomp as D, inputs as I

    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = oracle.params(tau_nu=0.6, tau_eta=0.65, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3,
                      les=les, delta=2.0)
    g = D.ghost_rows(les)
    owner = [s * world // k for s in range(k)]
    mine = [s for s in range(k) if owner[s] == rank]
    parts = D.slab_fields(I.orszag_tang(nx, ny, seed=3), ny, k, g)
    slabs = {s: oracle.init(*parts[s]) for s in mine}
    msgs = D.halo_messages(ny, k, g)
    comm, store = D.DistComm(owner), D.HostStore(nx)
    for _ in range(steps):
        D.exchange(msgs, slabs, store, comm)
        for s in mine:
            slabs[s] = oracle.step(slabs[s], p, 1)
    q.put((rank, {s: slabs[s][:, g:-g].copy() for s in mine}))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("les,k", [(1, 2), (2, 2), (1, 4), (3, 3)])
def test_gloo_ranks_match_undivided_oracle(orc, les, k):
    """Two gloo ranks holding k slabs between them, each slab stepped by the
    oracle, the halos moved by decomp.exchange over torch.distributed
    (several messages between one pair of ranks, and between slabs of one
    rank): the undivided oracle run bit for bit -- one ghost row per side
    with local rates, two with the kinetic closures."""
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    nx, ny, steps = 16, 13, 12
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, nx, ny, steps, q, les, k))
             for r in range(2)]
    for p in procs:
        p.start()
    parts = {}
    for _ in procs:
        parts.update(q.get(timeout=300)[1])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([parts[s] for s in range(k)], axis=1)
    ref = orc.step(orc.init(*inputs.orszag_tang(nx, ny, seed=3)),
                   orc.params(tau_nu=0.6, tau_eta=0.65, C_S=0.1, s5=1.2, s6=1.2, s7=1.3, s8=1.3,
                              les=les, delta=2.0),
                   steps)
    assert np.array_equal(got, ref)


def _monolithic(L, nx, ny, steps, fields, **kw):
    h = L.lbmhd_create(nx, ny, L.lbmhd_params_default(**kw))
    L.lbmhd_init(h, *fields)
    L.lbmhd_step(h, steps)
    ref = L.lbmhd_get_state(h)
    L.lbmhd_destroy(h)
    return ref


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_08675_gb300 import build, lbmhd

    build.build()
    return lbmhd


@pytest.mark.gpu
@pytest.mark.parametrize("overlap", [True, False])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16_dev", "ff"])
@pytest.mark.parametrize("k", [1, 3, 4])
def test_slabs_on_one_gpu_match_monolithic(L, prec, k, overlap):
    """k slabs of one lattice on this GPU, halos through decomp.exchange with
    the device store (only the planes a ghost row feeds), the interior rows
    stepped while the exchange runs on a side stream, the rows next to the
    ghosts after it: the undivided lattice bit for bit (k = 1: a slab that is
    its own neighbour)."""
    nx, ny, steps = 128, 50, 60
    kw = dict(precision=prec, tau_nu=0.6, tau_eta=0.65, C_S=0.1)
    fields = inputs.orszag_tang(nx, ny, seed=5)
    sl = decomp.SlabLattice(nx, ny, k, overlap=overlap, **kw)
    sl.init(*fields)
    sl.step(steps)
    got = sl.state()
    sl.close()
    assert np.array_equal(got, _monolithic(L, nx, ny, steps, fields, **kw))


@pytest.mark.gpu
@pytest.mark.parametrize("les", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16_dev", "ff"])
@pytest.mark.parametrize("k,ny", [(1, 50), (3, 50), (4, 10)])
def test_kinetic_slabs_on_one_gpu_match_monolithic(L, prec, k, ny, les):
    """The kinetic closures with two ghost rows per side (the nearer one
    also carries the planes moving along x): bit for bit the undivided
    lattice; slabs of 2 and 3 rows (fewer than the 4 that leave interior
    rows free of ghosts) take the exchange-then-step path."""
    nx, steps = 96, 40
    kw = dict(precision=prec, tau_nu=0.6, tau_eta=0.65, C_S=0.1, les=les, delta=2.0)
    fields = inputs.orszag_tang(nx, ny, seed=8)
    sl = decomp.SlabLattice(nx, ny, k, **kw)
    sl.init(*fields)
    sl.step(steps)
    got = sl.state()
    sl.close()
    assert np.array_equal(got, _monolithic(L, nx, ny, steps, fields, **kw))


@pytest.mark.gpu
def test_step_rows_and_row_planes_through_the_abi(L):
    """lbmhd_step_rows over two row ranges plus one commit equals one
    lbmhd_step; pack / unpack move exactly the masked planes of one row; bad
    ranges, rows, masks and misaligned buffers are refused."""
    import torch

    nx, ny = 64, 20
    fields = inputs.orszag_tang(nx, ny, seed=9)
    for prec in ("fp32", "fp64"):
        kw = dict(precision=prec, tau_nu=0.6, tau_eta=0.65, C_S=0.1)
        a = L.lbmhd_create(nx, ny, L.lbmhd_params_default(**kw))
        L.lbmhd_init(a, *fields)
        L.lbmhd_step_rows(a, 0, 7)
        L.lbmhd_step_rows(a, 7, ny)
        L.lbmhd_step_commit(a)
        assert L.lbmhd_step_count(a) == 1
        assert np.array_equal(L.lbmhd_get_state(a), _monolithic(L, nx, ny, 1, fields, **kw))
        raw = L.lbmhd_get_state_raw(a)
        vb = L.lbmhd_bytes_per_cell(prec) // 38
        dt = {4: torch.int32, 8: torch.int64}[vb]
        mask = decomp.UP | (1 << 0)
        planes = decomp.planes_of(mask)
        buf = torch.zeros(len(planes) * nx, dtype=dt, device="cuda")
        L.lbmhd_pack_row(a, 5, mask, buf)
        torch.cuda.synchronize()
        rawi = raw.view({4: np.int32, 8: np.int64}[vb]).reshape(19, ny, nx)
        assert np.array_equal(buf.cpu().numpy().reshape(len(planes), nx), rawi[planes, 5])
        L.lbmhd_unpack_row(a, 11, mask, buf)
        torch.cuda.synchronize()
        after = L.lbmhd_get_state_raw(a).view(rawi.dtype).reshape(19, ny, nx)
        want = rawi.copy()
        want[planes, 11] = rawi[planes, 5]
        assert np.array_equal(after, want)
        for bad in ((-1, 3), (3, 3), (5, ny + 1)):
            with pytest.raises(L.LBMHDError):
                L.lbmhd_step_rows(a, *bad)
        for row, m, off in ((ny, mask, 0), (-1, mask, 0), (0, 1 << 19, 0), (0, mask, 2)):
            with pytest.raises(L.LBMHDError):
                L.lbmhd_pack_row(a, row, m, buf.data_ptr() + off)
        # lbmhd_copy_rows: every plane of a block of rows from one handle to another
        b = L.lbmhd_create(nx, ny, L.lbmhd_params_default(**kw))
        L.lbmhd_init(b, *fields)
        L.lbmhd_copy_rows(b, 2, a, 10, 3)
        L.lbmhd_sync(b)
        got = L.lbmhd_get_state_raw(b).view(rawi.dtype).reshape(19, ny, nx)
        assert np.array_equal(got[:, 2:5], after[:, 10:13])
        L.lbmhd_destroy(b)
        L.lbmhd_destroy(a)
