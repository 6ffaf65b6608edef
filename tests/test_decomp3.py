"""z-slab domain decomposition of a 3D lattice: the halo messages on CPU,
the exchange of decomp.exchange over gloo between two CPU ranks stepping
their slabs with the 3D oracle, and k slabs on one GPU through the same
exchange with the device store (lbmhd3_pack_plane / lbmhd3_unpack_plane,
lbmhd3_step_planes) -- all bit for bit equal to the undivided lattice."""
import os
import socket
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_1607_08675_gb300 import decomp, inputs

MASKS3 = (decomp.UP3, decomp.DOWN3, decomp.REST3)


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3

    oracle3.build()
    return oracle3


def test_plane_sets3(o3):
    """The planes that stream towards +z, -z and within a plane, from the
    3D oracle's own lattice (27 velocities c in {-1, 0, 1}^3, then the six
    axes of the magnetic lattice, three components each)."""
    c, _, cm, _ = o3.lattice()
    cz = [int(v[2]) for v in c] + [int(cm[q][2]) for q in range(6) for _ in range(3)]
    assert tuple(cz) == decomp.PLANE_CZ3
    assert decomp.planes_of3(decomp.UP3) == [p for p in range(45) if cz[p] > 0]
    assert len(decomp.planes_of3(decomp.UP3)) == 12 and len(decomp.planes_of3(decomp.REST3)) == 21
    assert decomp.UP3 | decomp.DOWN3 | decomp.REST3 == (1 << 45) - 1


def _needed3(les, ghost):
    """Brute force: the (ghost plane, storage plane) pairs the interior
    planes of a slab read -- the pull of the plane itself and, with the
    kinetic closures, the pulls of the planes whose fields its gradients
    use."""
    need = set()
    n = 2 * ghost + 3
    for z in range(ghost, ghost + n):
        pulled = {z} if les < 2 else {z - 1, z, z + 1}
        for r in pulled:
            for p in range(45):
                src = r - decomp.PLANE_CZ3[p]
                if src < ghost or src >= ghost + n:
                    need.add((src, p))
    return need, n


@pytest.mark.parametrize("les", [1, 2])
def test_messages3_carry_exactly_what_the_ghost_planes_feed(les):
    g = decomp.ghost_rows(les)
    need, n = _needed3(les, g)
    nz, k = 3 * n, 3
    planes = decomp.split_rows(nz, k)
    msgs = decomp.halo_messages(nz, k, g, MASKS3)
    got = set()
    for m in msgs:
        for sz, dz, mask in m.parts:
            assert g <= sz < g + planes[m.src][1] - planes[m.src][0]
            assert (planes[m.src][0] + sz - g) % nz == (planes[m.dst][0] + dz - g) % nz
            for p in decomp.planes_of3(mask):
                assert (m.dst, dz, p) not in got
                got.add((m.dst, dz, p))
    for s in range(k):
        assert {(z, p) for (d, z, p) in got if d == s} == need, (les, s)
    per = sum(m.nvalues(1) for m in msgs) // (2 * k)
    assert per == (12 if les < 2 else 33 + 12)  # planes per cut and direction
    assert decomp.halo_bytes_per_step3(8, 4, nz, k, les, 4) == sum(m.nvalues(32) for m in msgs) * 4


def test_exchange_on_host_slabs3_matches_global_planes():
    nx, ny, nz, k = 4, 3, 11, 3
    for les in (1, 2):
        g = decomp.ghost_rows(les)
        glob = np.arange(45 * nz * ny * nx, dtype=np.float64).reshape(45, nz, ny, nx)
        planes = decomp.split_rows(nz, k)
        slabs = {}
        for s, (a, b) in enumerate(planes):
            st = np.full((45, b - a + 2 * g, ny, nx), -1.0)
            st[:, g:g + b - a] = glob[:, a:b]
            slabs[s] = st
        msgs = decomp.halo_messages(nz, k, g, MASKS3)
        decomp.exchange(msgs, slabs, decomp.HostStore3(nx, ny))
        for m in msgs:
            for _, dz, mask in m.parts:
                gz = (planes[m.dst][0] + dz - g) % nz
                p = decomp.planes_of3(mask)
                assert np.array_equal(slabs[m.dst][p, dz], glob[p, gz])
        for s, st in slabs.items():
            n = planes[s][1] - planes[s][0]
            assert np.array_equal(st[:, g:g + n], glob[:, planes[s][0]:planes[s][1]])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _params3(o3, les):
    return o3.params(tau_nu=0.6, tau_eta=0.65, C_S=0.2, delta=2.0, les=les)


def _rank3(rank, world, port, shape, steps, q, les, k):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from oracle import oracle3
    from paper_1607_08675_gb300 import decomp as D, inputs as I

    dist.init_process_group("gloo", rank=rank, world_size=world)
    nx, ny, nz = shape
    p = _params3(oracle3, les)
    g = D.ghost_rows(les)
    owner = [s * world // k for s in range(k)]
    mine = [s for s in range(k) if owner[s] == rank]
    parts = D.slab_fields3(I.turbulence3d(nx, ny, nz, kmin=1, kmax=2, rms=0.05, seed=3), nz, k, g)
    slabs = {s: oracle3.init(*parts[s]) for s in mine}
    msgs = D.halo_messages(nz, k, g, (D.UP3, D.DOWN3, D.REST3))
    comm, store = D.DistComm(owner), D.HostStore3(nx, ny)
    for _ in range(steps):
        D.exchange(msgs, slabs, store, comm)
        for s in mine:
            slabs[s] = oracle3.step(slabs[s], p, 1)
    q.put((rank, {s: slabs[s][:, g:-g].copy() for s in mine}))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("les,k", [(1, 2), (2, 2), (3, 3), (1, 3)])
def test_gloo_ranks_match_undivided_3d_oracle(o3, les, k):
    """Two gloo ranks holding k z-slabs between them, each slab stepped by
    the 3D oracle, the halos moved by decomp.exchange over
    torch.distributed: the undivided oracle run bit for bit."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    shape, steps = (6, 5, 13), 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank3, args=(r, 2, port, shape, steps, q, les, k)) for r in range(2)]
    for p in procs:
        p.start()
    parts = {}
    for _ in procs:
        parts.update(q.get(timeout=300)[1])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([parts[s] for s in range(k)], axis=1)
    nx, ny, nz = shape
    ref = o3.step(o3.init(*inputs.turbulence3d(nx, ny, nz, kmin=1, kmax=2, rms=0.05, seed=3)),
                  _params3(o3, les), steps)
    assert np.array_equal(got, ref)


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_08675_gb300 import build, lbmhd

    build.build()
    return lbmhd


def _monolithic3(L, shape, steps, fields, launch=None, **kw):
    nx, ny, nz = shape
    h = L.lbmhd3_create(nx, ny, nz, L.lbmhd_params_default(**kw))
    if launch is not None:
        L.lbmhd3_set_launch(h, *launch)
    L.lbmhd3_init(h, *fields)
    L.lbmhd3_step(h, steps)
    ref = L.lbmhd3_get_state(h)
    L.lbmhd3_destroy(h)
    return ref


@pytest.mark.gpu
@pytest.mark.parametrize("les", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16_dev", "ff"])
@pytest.mark.parametrize("k,nz,overlap", [(1, 12, True), (3, 20, True), (4, 13, False), (5, 11, True)])
def test_slabs3_on_one_gpu_match_monolithic(L, prec, les, k, nz, overlap):
    """k z-slabs of one lattice on this GPU, halos through decomp.exchange
    with the device store (only the planes a ghost plane feeds), the
    interior planes stepped while the exchange runs on a side stream: the
    undivided lattice bit for bit, in every storage format and closure
    (k = 1: a slab that is its own neighbour; slabs thinner than 2 g planes
    take the exchange-then-step path)."""
    shape, steps = (40, 12, nz), 15
    kw = dict(precision=prec, tau_nu=0.6, tau_eta=0.65, C_S=0.2, delta=2.0, les=les)
    fields = inputs.turbulence3d(*shape, kmin=1, kmax=3, rms=0.05, seed=8)
    sl = decomp.SlabRunner3(*shape, k, overlap=overlap, **kw)
    sl.init(*fields)
    sl.step(steps)
    got = sl.state()
    sl.close()
    assert np.array_equal(got, _monolithic3(L, shape, steps, fields, **kw))


@pytest.mark.gpu
@pytest.mark.parametrize("launch", [(2, 128), (0, 4)])
def test_two_pass_slabs3_match_monolithic(L, launch):
    """The two-pass closure kernels (their moments pass around a plane
    range) and the barrier-per-plane fused kernel under slabs, against the
    default (warp-specialised) kernel on the undivided lattice."""
    shape, steps = (32, 10, 14), 12
    fields = inputs.turbulence3d(*shape, kmin=1, kmax=3, rms=0.05, seed=9)
    for les in (2, 3):
        kw = dict(precision="fp32", tau_nu=0.6, tau_eta=0.65, C_S=0.2, delta=2.0, les=les)
        sl = decomp.SlabRunner3(*shape, 3, launch=launch, **kw)
        sl.init(*fields)
        sl.step(steps)
        got = sl.state()
        sl.close()
        assert np.array_equal(got, _monolithic3(L, shape, steps, fields, **kw))


@pytest.mark.gpu
def test_step_planes_and_plane_messages_through_the_abi(L):
    """lbmhd3_step_planes over two plane ranges plus one commit equals one
    lbmhd3_step; pack / unpack move exactly the masked planes of one
    z-plane; bad ranges, planes, masks and misaligned buffers are refused."""
    import torch

    shape = (16, 6, 9)
    nx, ny, nz = shape
    fields = inputs.turbulence3d(*shape, seed=4)
    for prec in ("fp32", "fp64", "fp16_dev"):
        kw = dict(precision=prec, tau_nu=0.6, tau_eta=0.65, C_S=0.2)
        a = L.lbmhd3_create(nx, ny, nz, L.lbmhd_params_default(**kw))
        L.lbmhd3_init(a, *fields)
        L.lbmhd3_step_planes(a, 0, 4)
        L.lbmhd3_step_planes(a, 4, nz)
        L.lbmhd3_step_commit(a)
        assert L.lbmhd3_step_count(a) == 1
        assert np.array_equal(L.lbmhd3_get_state(a), _monolithic3(L, shape, 1, fields, **kw))
        vb = L.lbmhd3_bytes_per_cell(prec) // 90
        dt = {2: torch.int16, 4: torch.int32, 8: torch.int64}[vb]
        mask = decomp.UP3 | 1
        planes = decomp.planes_of3(mask)
        buf = torch.zeros(len(planes) * nx * ny, dtype=dt, device="cuda")
        L.lbmhd3_pack_plane(a, 5, mask, buf)
        buf2 = buf.clone()
        L.lbmhd3_unpack_plane(a, 2, mask, buf)
        buf3 = torch.zeros_like(buf)
        L.lbmhd3_pack_plane(a, 2, mask, buf3)
        torch.cuda.synchronize()
        assert torch.equal(buf3, buf2)
        st = L.lbmhd3_get_state(a)
        assert np.array_equal(st[planes, 2], st[planes, 5])
        for bad in ((a, 0, 0), (a, 3, 2), (a, -1, 4), (a, 0, nz + 1)):
            with pytest.raises(L.LBMHDError):
                L.lbmhd3_step_planes(*bad)
        with pytest.raises(L.LBMHDError):
            L.lbmhd3_pack_plane(a, nz, mask, buf)
        with pytest.raises(L.LBMHDError):
            L.lbmhd3_pack_plane(a, 0, 1 << 45, buf)
        with pytest.raises(L.LBMHDError):
            L.lbmhd3_pack_plane(a, 0, mask, buf.data_ptr() + 1)
        L.lbmhd3_destroy(a)
