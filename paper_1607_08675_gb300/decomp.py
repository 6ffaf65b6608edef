"""y-slab domain decomposition of one periodic lattice (the sharding of the
step across devices or ranks).

The lattice's ny rows are cut into k slabs.  Each slab is stepped as a
lattice of its own rows plus one ghost row above and below; the step reads
only rows y - 1, y, y + 1, so the interior rows of every slab come out
exactly as in the undivided lattice provided the ghost rows hold the
neighbouring slabs' boundary rows (post-collision) before each step.  After
each step every slab sends its last interior row to the lower ghost row of
the slab above it and its first interior row to the upper ghost row of the
slab below it (periodic in y).  One ghost row suffices for les = 0 and 1;
les = 2 and 3 take gradients of moments of the neighbouring rows and would
need two, so SlabLattice refuses them.

``plan`` gives the row bookkeeping (pure host logic, shared by any
transport); ``SlabLattice`` runs k slabs on one GPU through the C ABI, the
exchange being lbmhd_copy_rows (device-to-device copies).  A multi-GPU run
would move the same rows with peer copies or NCCL send/recv.
"""
from __future__ import annotations

import numpy as np

from . import lbmhd as L


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


def plan(ny: int, k: int):
    """Halo exchange after a step, as (src_slab, src_local_row, dst_slab,
    dst_local_row) copies of one row.  Local rows: 0 is the lower ghost, 1..n
    the interior, n + 1 the upper ghost."""
    rows = split_rows(ny, k)
    moves = []
    for s, (a, b) in enumerate(rows):
        n = b - a
        up, down = (s + 1) % k, (s - 1) % k
        n_down = rows[down][1] - rows[down][0]
        moves.append((s, n, up, 0))            # last interior row -> ghost below `up`
        moves.append((s, 1, down, n_down + 1))  # first interior row -> ghost above `down`
    return moves


def slab_fields(fields, ny: int, k: int):
    """Per slab, the five initial fields of its rows plus ghost rows (periodic
    rows of the global fields)."""
    out = []
    for a, b in split_rows(ny, k):
        idx = np.arange(a - 1, b + 1) % ny
        out.append([np.ascontiguousarray(f[idx]) for f in fields])
    return out


class SlabLattice:
    """k slabs of one nx x ny lattice on the current GPU."""

    def __init__(self, nx: int, ny: int, k: int, **params):
        if params.get("les", 1) >= 2:
            raise ValueError("slab decomposition with one ghost row supports les 0 and 1")
        self.nx, self.ny, self.k = nx, ny, k
        self.rows = split_rows(ny, k)
        self.moves = plan(ny, k)
        self.h = [L.lbmhd_create(nx, b - a + 2, L.lbmhd_params_default(**params))
                  for a, b in self.rows]

    def init(self, rho, ux, uy, bx, by):
        for h, f in zip(self.h, slab_fields((rho, ux, uy, bx, by), self.ny, self.k)):
            L.lbmhd_init(h, *f)

    def step(self, n: int = 1):
        for _ in range(n):
            for h in self.h:
                L.lbmhd_step(h, 1)
            for src, srow, dst, drow in self.moves:
                L.lbmhd_copy_rows(self.h[dst], drow, self.h[src], srow, 1)

    def moments(self):
        parts = [L.lbmhd_moments(h) for h in self.h]
        return tuple(np.concatenate([p[q][1:-1] for p in parts]) for q in range(5))

    def state(self):
        return np.concatenate([L.lbmhd_get_state(h)[:, 1:-1] for h in self.h], axis=1)

    def close(self):
        for h in self.h:
            L.lbmhd_destroy(h)
