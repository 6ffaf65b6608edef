"""y-slab domain decomposition of one periodic lattice (the sharding of the
step across devices or ranks).

The step streams every population by a shift (Sec. 1.2) and collides
locally (Sec. 3), so a lattice cut into k row slabs can be advanced slab by
slab.  Each slab holds its own rows plus g ghost rows above and below that
mirror its neighbours' boundary rows: g = 1 with local rates (les 0, 1),
whose step reads rows y - 1 .. y + 1; g = 2 with the kinetic closures
(les 2, 3), whose moment gradients pull from two rows away.

Only the planes a ghost row feeds travel (``halo_messages``): the ghost row
below a slab feeds the pull of the slab's first row with the planes that
stream upwards (c_y = +1: f_2, f_5, f_6, g_2); with g = 2 it also feeds the
moments of the ghost row itself, which pull the c_y = 0 planes from it and
the upward planes from the second ghost row.  Per cut and direction that is
5 x nx values with local rates (19 x nx when every plane of one row is
copied) and 14 + 5 = 19 x nx with the kinetic closures (38 x nx).

A 3D lattice is cut the same way into z-slabs of planes (``SlabRunner3``):
the ghost plane below a slab carries the populations streaming upwards
(c_z = +1: the nine f_i with k_z = 1 and g_{+z}, 12 of the 45 planes), with
g = 2 also the 21 planes with c_z = 0 for its own moments: 12 x nx x ny
values per cut and direction with local rates, 33 + 12 with the kinetic
closures.

``exchange`` moves one round of these messages through any transport: it
packs the outgoing rows of the slabs a rank holds, delivers messages
between its own slabs directly, and hands the rest to a communicator
(``DistComm``: torch.distributed send/recv, NCCL between GPUs or gloo on
CPU).  ``SlabRunner`` advances the slabs one process holds on its GPU: the
exchange runs on a side stream while the rows that need no ghost row are
computed (lbmhd_step_rows), then the rows next to the ghosts, then the
commit; ghost rows are never computed.  The same ``exchange`` moves the
halos of slabs held as host arrays (``HostStore``) between gloo ranks.
"""
from __future__ import annotations

import numpy as np

from . import lbmhd as L

# c_y of the 19 stored planes: f_0..f_8, then g_k (x, y) for k = 0..4
PLANE_CY = (0, 0, 1, 0, -1, 1, 1, -1, -1) + tuple(c for c in (0, 0, 1, 0, -1) for _ in (0, 1))
UP = sum(1 << p for p, c in enumerate(PLANE_CY) if c > 0)     # streaming towards +y
DOWN = sum(1 << p for p, c in enumerate(PLANE_CY) if c < 0)   # towards -y
REST = sum(1 << p for p, c in enumerate(PLANE_CY) if c == 0)  # along x or at rest


def planes_of(mask: int):
    return [p for p in range(19) if mask >> p & 1]


def split_rows(ny: int, k: int):
    """Row ranges [start, stop) of k slabs covering ny rows (sizes differ by
    at most one)."""
    if not 1 <= k <= ny:
        raise ValueError("need 1 <= k <= ny")
    base, extra = divmod(ny, k)
    out, y = [], 0
    for s in range(k):
        n = base + (1 if s < extra else 0)
        out.append((y, y + n))
        y += n
    return out


def ghost_rows(les: int) -> int:
    """Ghost rows per side the step needs: 1 with local rates, 2 with the
    kinetic closures (moment gradients of pulled populations)."""
    return 2 if les >= 2 else 1


class Message:
    """One slab-to-slab halo message: parts (src_row, dst_row, plane_mask)
    in local rows (0 .. g - 1 the lower ghosts, g .. g + n - 1 the interior,
    then the upper ghosts)."""

    __slots__ = ("src", "dst", "parts", "direction")

    def __init__(self, src, dst, parts, direction):
        self.src, self.dst, self.parts, self.direction = src, dst, parts, direction

    def nvalues(self, nx: int) -> int:
        return sum(bin(m).count("1") for _, _, m in self.parts) * nx

    def __repr__(self):
        return f"Message({self.src}->{self.dst} {self.direction} {self.parts})"


# c_z of the 45 stored planes of a 3D state: f_i with i = 9 kz + 3 ky + kx
# (c_z = 0, +1, -1 for kz = 0, 1, 2), then g_q (x, y, z) for q = +x, -x,
# +y, -y, +z, -z
PLANE_CZ3 = tuple((0, 1, -1)[i // 9] for i in range(27)) + tuple(
    (1 if q == 4 else (-1 if q == 5 else 0)) for q in range(6) for _ in range(3))
UP3 = sum(1 << p for p, c in enumerate(PLANE_CZ3) if c > 0)
DOWN3 = sum(1 << p for p, c in enumerate(PLANE_CZ3) if c < 0)
REST3 = sum(1 << p for p, c in enumerate(PLANE_CZ3) if c == 0)


def halo_messages(ny: int, k: int, ghost: int = 1, masks=None):
    """Every message of one exchange, in one global order (every rank walks
    the same list, so matching sends and receives are posted in the same
    order).  Slab s sends upwards to s + 1 and downwards to s - 1 (periodic);
    with k = 1 a slab is its own neighbour.  masks: the (up, down, rest)
    plane masks -- the 2D lattice's by default, (UP3, DOWN3, REST3) for
    z-slabs of a 3D lattice (rows are then planes)."""
    UP_, DOWN_, REST_ = masks if masks is not None else (UP, DOWN, REST)
    rows = split_rows(ny, k)
    g = ghost
    if min(b - a for a, b in rows) < g:
        raise ValueError("every slab needs at least as many rows as ghost rows")
    msgs = []
    for s, (a, b) in enumerate(rows):
        n = b - a
        up, down = (s + 1) % k, (s - 1) % k
        n_down = rows[down][1] - rows[down][0]
        # part j: the ghost row at distance j + 1 from the receiver's interior;
        # the nearer ghost row (j < g - 1) also feeds its own moments
        msgs.append(Message(s, up, [(g + n - 1 - j, g - 1 - j, UP_ | (REST_ if j < g - 1 else 0))
                                    for j in range(g)], "up"))
        msgs.append(Message(s, down, [(g + j, g + n_down + j, DOWN_ | (REST_ if j < g - 1 else 0))
                                      for j in range(g)], "down"))
    return msgs


def halo_bytes_per_step(nx: int, ny: int, k: int, les: int, value_bytes: int) -> int:
    """Bytes one exchange moves between slabs (all messages)."""
    return sum(m.nvalues(nx) for m in halo_messages(ny, k, ghost_rows(les))) * value_bytes


def slab_fields(fields, ny: int, k: int, ghost: int = 1):
    """Per slab, the five initial fields of its rows plus ghost rows (periodic
    rows of the global fields)."""
    out = []
    for a, b in split_rows(ny, k):
        idx = np.arange(a - ghost, b + ghost) % ny
        out.append([np.ascontiguousarray(f[idx]) for f in fields])
    return out


def exchange(msgs, slabs, store, comm=None):
    """One round of halo messages.

    slabs: {slab index: slab object} for the slabs this rank holds.
    store: packs and unpacks message parts for those slab objects --
      ``new_buffer(nvalues)``, ``pack(slab_obj, row, mask, buf, offset)``,
      ``unpack(slab_obj, row, mask, buf, offset)`` (offset in values).
    comm: None when every slab is local; otherwise ``rank_of(slab)`` and
      ``transfer(sends, recvs)`` with lists of (peer rank, buffer) in the
      global message order.
    Messages between two local slabs are unpacked straight from the packed
    buffer.  Every part is packed before any is unpacked, so a slab that is
    its own neighbour (k = 1) reads its boundary rows before its ghost rows
    change."""
    sends, recvs, ready = [], [], []
    for m in msgs:
        src_here, dst_here = m.src in slabs, m.dst in slabs
        if not (src_here or dst_here):
            continue
        buf = store.new_buffer(m.nvalues(store.nx))
        if src_here:
            off = 0
            for row, _, mask in m.parts:
                store.pack(slabs[m.src], row, mask, buf, off)
                off += bin(mask).count("1") * store.nx
        if src_here and dst_here:
            ready.append((m, buf))
        elif src_here:
            sends.append((comm.rank_of(m.dst), buf))
        else:
            recvs.append((comm.rank_of(m.src), buf))
            ready.append((m, buf))
    if comm is not None and (sends or recvs):
        comm.transfer(sends, recvs)
    for m, buf in ready:
        off = 0
        for _, row, mask in m.parts:
            store.unpack(slabs[m.dst], row, mask, buf, off)
            off += bin(mask).count("1") * store.nx


class DistComm:
    """torch.distributed point-to-point transport: slab s lives on rank
    owner[s].  The sends and receives of one exchange go out as one batch
    (NCCL groups them; gloo posts them), then all are waited for."""

    def __init__(self, owner):
        self.owner = list(owner)

    def rank_of(self, slab):
        return self.owner[slab]

    def transfer(self, sends, recvs):
        import torch.distributed as dist

        ops = [dist.P2POp(dist.isend, buf, peer) for peer, buf in sends]
        ops += [dist.P2POp(dist.irecv, buf, peer) for peer, buf in recvs]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class HostStore:
    """Message buffers and packing for slabs held as host arrays of shape
    (19, rows, nx) (FP64 populations): torch CPU tensors, for gloo."""

    def __init__(self, nx: int):
        self.nx = nx

    def new_buffer(self, nvalues):
        import torch

        return torch.empty(nvalues, dtype=torch.float64)

    def pack(self, st, row, mask, buf, off):
        p = planes_of(mask)
        buf.numpy()[off:off + len(p) * self.nx] = st[p, row, :].reshape(-1)

    def unpack(self, st, row, mask, buf, off):
        p = planes_of(mask)
        st[p, row, :] = buf.numpy()[off:off + len(p) * self.nx].reshape(len(p), self.nx)


_RAW = {2: "int16", 4: "int32", 8: "int64"}


class DeviceStore:
    """Message buffers and packing for lbmhd_t slabs: the stored values are
    moved as raw integers of their width (lbmhd_pack_row / lbmhd_unpack_row)
    on the current torch stream."""

    def __init__(self, nx: int, precision: str):
        import torch

        self.nx = nx
        self.vb = L.lbmhd_bytes_per_cell(precision) // 38
        self.dtype = getattr(torch, _RAW[self.vb])

    def new_buffer(self, nvalues):
        import torch

        return torch.empty(nvalues, dtype=self.dtype, device="cuda")

    def pack(self, h, row, mask, buf, off):
        import torch

        L.lbmhd_pack_row(h, row, mask, buf.data_ptr() + off * self.vb,
                         torch.cuda.current_stream())

    def unpack(self, h, row, mask, buf, off):
        import torch

        L.lbmhd_unpack_row(h, row, mask, buf.data_ptr() + off * self.vb,
                           torch.cuda.current_stream())


class SlabRunner:
    """The slabs of one nx x ny lattice that this process holds, each an
    lbmhd_t of its rows plus ghost rows on the current GPU.

    slabs: the slab indices held here (default: all k).  comm: a transport
    for the other slabs (None: every slab is here).  overlap: exchange on a
    side stream while the rows that need no ghost row are computed."""

    def __init__(self, nx: int, ny: int, k: int, slabs=None, comm=None, overlap=True,
                 **params):
        import torch

        self.nx, self.ny, self.k = nx, ny, k
        self.les = params.get("les", 1)
        self.g = ghost_rows(self.les)
        self.rows = split_rows(ny, k)
        self.msgs = halo_messages(ny, k, self.g)
        self.mine = list(range(k)) if slabs is None else list(slabs)
        self.comm, self.overlap = comm, overlap
        self.main = torch.cuda.Stream()
        self.side = torch.cuda.Stream() if overlap else self.main
        prec = params.get("precision", "fp64")
        self.store = DeviceStore(nx, prec)
        p = dict(params, stream=self.main)
        self.h = {s: L.lbmhd_create(nx, self.rows[s][1] - self.rows[s][0] + 2 * self.g,
                                    L.lbmhd_params_default(**p)) for s in self.mine}

    def halo_bytes(self) -> int:
        """Bytes this rank's slabs receive per step."""
        return sum(m.nvalues(self.nx) for m in self.msgs if m.dst in self.h) * self.store.vb

    def init(self, rho, ux, uy, bx, by):
        parts = slab_fields((rho, ux, uy, bx, by), self.ny, self.k, self.g)
        for s, h in self.h.items():
            L.lbmhd_init(h, *parts[s])
        self.main.synchronize()

    def _ranges(self, s):
        """(interior rows that read no ghost row, rows next to the ghosts)."""
        g, n = self.g, self.rows[s][1] - self.rows[s][0]
        if n < 2 * g:
            return [], [(g, g + n)]
        inner = [(2 * g, n)] if n > 2 * g else []
        return inner, [(g, 2 * g), (n, g + n)]

    def step(self, nsteps: int = 1):
        import torch

        for _ in range(nsteps):
            # the exchange reads the state the last step wrote
            self.side.wait_stream(self.main)
            with torch.cuda.stream(self.side):
                exchange(self.msgs, self.h, self.store, self.comm)
            for s, h in self.h.items():
                for y0, y1 in self._ranges(s)[0]:
                    L.lbmhd_step_rows(h, y0, y1)
            self.main.wait_stream(self.side)
            for s, h in self.h.items():
                for y0, y1 in self._ranges(s)[1]:
                    L.lbmhd_step_rows(h, y0, y1)
                L.lbmhd_step_commit(h)

    def sync(self):
        self.main.synchronize()
        self.side.synchronize()

    def state(self):
        """FP64 populations of the interior rows, slab after slab (the
        rows this process holds)."""
        g = self.g
        return np.concatenate([L.lbmhd_get_state(self.h[s])[:, g:-g] for s in self.mine], axis=1)

    def moments(self):
        g = self.g
        parts = [L.lbmhd_moments(self.h[s]) for s in self.mine]
        return tuple(np.concatenate([p[q][g:-g] for p in parts]) for q in range(5))

    def close(self):
        for h in self.h.values():
            L.lbmhd_destroy(h)
        self.h = {}


class SlabLattice(SlabRunner):
    """k slabs of one nx x ny lattice, all on the current GPU."""

    def __init__(self, nx: int, ny: int, k: int, **params):
        super().__init__(nx, ny, k, **params)


# ---- z-slabs of a 3D lattice --------------------------------------------------


def halo_bytes_per_step3(nx: int, ny: int, nz: int, k: int, les: int, value_bytes: int) -> int:
    """Bytes one exchange of a 3D lattice cut into k z-slabs moves."""
    msgs = halo_messages(nz, k, ghost_rows(les), (UP3, DOWN3, REST3))
    return sum(m.nvalues(nx * ny) for m in msgs) * value_bytes


def slab_fields3(fields, nz: int, k: int, ghost: int = 1):
    """Per z-slab, the seven initial fields (nz, ny, nx) of its planes plus
    ghost planes (periodic planes of the global fields)."""
    out = []
    for a, b in split_rows(nz, k):
        idx = np.arange(a - ghost, b + ghost) % nz
        out.append([np.ascontiguousarray(f[idx]) for f in fields])
    return out


class HostStore3:
    """Message buffers and packing for 3D slabs held as host arrays of shape
    (45, planes, ny, nx) (FP64 populations): torch CPU tensors, for gloo.
    nx here is the length of one message row: nx * ny values."""

    def __init__(self, nx: int, ny: int):
        self.nx = nx * ny

    def new_buffer(self, nvalues):
        import torch

        return torch.empty(nvalues, dtype=torch.float64)

    def pack(self, st, z, mask, buf, off):
        p = planes_of3(mask)
        buf.numpy()[off:off + len(p) * self.nx] = st[p, z].reshape(-1)

    def unpack(self, st, z, mask, buf, off):
        p = planes_of3(mask)
        st[p, z] = buf.numpy()[off:off + len(p) * self.nx].reshape((len(p),) + st.shape[2:])


def planes_of3(mask: int):
    return [p for p in range(45) if mask >> p & 1]


class DeviceStore3:
    """Message buffers and packing for lbmhd3_t slabs: stored values moved as
    raw integers of their width (lbmhd3_pack_plane / lbmhd3_unpack_plane) on
    the current torch stream."""

    def __init__(self, nx: int, ny: int, precision: str):
        import torch

        self.nx = nx * ny
        self.vb = L.lbmhd3_bytes_per_cell(precision) // 90
        self.dtype = getattr(torch, _RAW[self.vb])

    def new_buffer(self, nvalues):
        import torch

        return torch.empty(nvalues, dtype=self.dtype, device="cuda")

    def pack(self, h, z, mask, buf, off):
        import torch

        L.lbmhd3_pack_plane(h, z, mask, buf.data_ptr() + off * self.vb, torch.cuda.current_stream())

    def unpack(self, h, z, mask, buf, off):
        import torch

        L.lbmhd3_unpack_plane(h, z, mask, buf.data_ptr() + off * self.vb, torch.cuda.current_stream())


class SlabRunner3:
    """The z-slabs of one nx x ny x nz lattice that this process holds, each
    an lbmhd3_t of its planes plus ghost planes on the current GPU; the
    exchange, overlap and commit of ``SlabRunner`` with planes for rows."""

    def __init__(self, nx: int, ny: int, nz: int, k: int, slabs=None, comm=None, overlap=True,
                 **params):
        import torch

        self.nx, self.ny, self.nz, self.k = nx, ny, nz, k
        self.les = params.get("les", 1)
        self.g = ghost_rows(self.les)
        self.planes = split_rows(nz, k)
        self.msgs = halo_messages(nz, k, self.g, (UP3, DOWN3, REST3))
        self.mine = list(range(k)) if slabs is None else list(slabs)
        self.comm, self.overlap = comm, overlap
        self.main = torch.cuda.Stream()
        self.side = torch.cuda.Stream() if overlap else self.main
        prec = params.get("precision", "fp64")
        self.store = DeviceStore3(nx, ny, prec)
        launch = params.pop("launch", None)
        p = dict(params, stream=self.main)
        self.h = {}
        for s in self.mine:
            n = self.planes[s][1] - self.planes[s][0] + 2 * self.g
            self.h[s] = L.lbmhd3_create(nx, ny, n, L.lbmhd_params_default(**p))
            if launch is not None:
                L.lbmhd3_set_launch(self.h[s], *launch)

    def halo_bytes(self) -> int:
        """Bytes this rank's slabs receive per step."""
        return sum(m.nvalues(self.nx * self.ny) for m in self.msgs if m.dst in self.h) * self.store.vb

    def init(self, rho, ux, uy, uz, bx, by, bz):
        parts = slab_fields3((rho, ux, uy, uz, bx, by, bz), self.nz, self.k, self.g)
        for s, h in self.h.items():
            L.lbmhd3_init(h, *parts[s])
        self.main.synchronize()

    def _ranges(self, s):
        """(interior planes that read no ghost plane, planes next to the
        ghosts)."""
        g, n = self.g, self.planes[s][1] - self.planes[s][0]
        if n < 2 * g:
            return [], [(g, g + n)]
        inner = [(2 * g, n)] if n > 2 * g else []
        return inner, [(g, 2 * g), (n, g + n)]

    def step(self, nsteps: int = 1):
        import torch

        for _ in range(nsteps):
            self.side.wait_stream(self.main)
            with torch.cuda.stream(self.side):
                exchange(self.msgs, self.h, self.store, self.comm)
            for s, h in self.h.items():
                for z0, z1 in self._ranges(s)[0]:
                    L.lbmhd3_step_planes(h, z0, z1)
            self.main.wait_stream(self.side)
            for s, h in self.h.items():
                for z0, z1 in self._ranges(s)[1]:
                    L.lbmhd3_step_planes(h, z0, z1)
                L.lbmhd3_step_commit(h)

    def sync(self):
        self.main.synchronize()
        self.side.synchronize()

    def state(self):
        """FP64 populations (45, planes, ny, nx) of the interior planes, slab
        after slab (the planes this process holds)."""
        g = self.g
        return np.concatenate([L.lbmhd3_get_state(self.h[s])[:, g:-g] for s in self.mine], axis=1)

    def moments(self):
        g = self.g
        parts = [L.lbmhd3_moments(self.h[s]) for s in self.mine]
        return tuple(np.concatenate([p[q][g:-g] for p in parts]) for q in range(7))

    def close(self):
        for h in self.h.values():
            L.lbmhd3_destroy(h)
        self.h = {}
