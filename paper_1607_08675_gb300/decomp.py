"""y-slab domain decomposition of one periodic lattice (the sharding of the
step across devices or ranks).

The lattice's ny rows are cut into k slabs.  Each slab is stepped as a
lattice of its own rows plus g ghost rows above and below.  The step with
local rates (les = 0, 1) reads rows y - 1, y, y + 1; the kinetic closures
(les = 2, 3) take central differences of moments that are themselves
pulled from the neighbouring rows, so they read rows y - 2 .. y + 2.  With
g = 1 or g = 2 rows of ghosts respectively, the interior rows of every
slab come out exactly as in the undivided lattice provided the ghost rows
hold the neighbouring slabs' boundary rows (post-collision) before each
step; the ghost rows' own results are wrong and are overwritten.  After
each step every slab sends its last g interior rows to the lower ghost
rows of the slab above it and its first g interior rows to the upper ghost
rows of the slab below it (periodic in y).  Every slab needs at least g
rows.

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


def ghost_rows(les: int) -> int:
    """Ghost rows per side the step needs: 1 with local rates, 2 with the
    kinetic closures (moment gradients of pulled populations)."""
    return 2 if les >= 2 else 1


def plan(ny: int, k: int, ghost: int = 1):
    """Halo exchange after a step, as (src_slab, src_local_row, dst_slab,
    dst_local_row) copies of one row.  Local rows: 0 .. ghost - 1 are the
    lower ghosts, ghost .. ghost + n - 1 the interior, then the upper
    ghosts."""
    rows = split_rows(ny, k)
    if min(b - a for a, b in rows) < ghost:
        raise ValueError("every slab needs at least as many rows as ghost rows")
    g = ghost
    moves = []
    for s, (a, b) in enumerate(rows):
        n = b - a
        up, down = (s + 1) % k, (s - 1) % k
        n_down = rows[down][1] - rows[down][0]
        for i in range(g):
            moves.append((s, n + i, up, i))              # last g interior rows -> below `up`
            moves.append((s, g + i, down, g + n_down + i))  # first g rows -> above `down`
    return moves


def slab_fields(fields, ny: int, k: int, ghost: int = 1):
    """Per slab, the five initial fields of its rows plus ghost rows (periodic
    rows of the global fields)."""
    out = []
    for a, b in split_rows(ny, k):
        idx = np.arange(a - ghost, b + ghost) % ny
        out.append([np.ascontiguousarray(f[idx]) for f in fields])
    return out


class SlabLattice:
    """k slabs of one nx x ny lattice on the current GPU."""

    def __init__(self, nx: int, ny: int, k: int, **params):
        self.nx, self.ny, self.k = nx, ny, k
        self.g = ghost_rows(params.get("les", 1))
        self.rows = split_rows(ny, k)
        self.moves = plan(ny, k, self.g)
        self.h = [L.lbmhd_create(nx, b - a + 2 * self.g, L.lbmhd_params_default(**params))
                  for a, b in self.rows]

    def init(self, rho, ux, uy, bx, by):
        for h, f in zip(self.h, slab_fields((rho, ux, uy, bx, by), self.ny, self.k, self.g)):
            L.lbmhd_init(h, *f)

    def step(self, n: int = 1):
        for _ in range(n):
            for h in self.h:
                L.lbmhd_step(h, 1)
            for src, srow, dst, drow in self.moves:
                L.lbmhd_copy_rows(self.h[dst], drow, self.h[src], srow, 1)

    def moments(self):
        g = self.g
        parts = [L.lbmhd_moments(h) for h in self.h]
        return tuple(np.concatenate([p[q][g:-g] for p in parts]) for q in range(5))

    def state(self):
        g = self.g
        return np.concatenate([L.lbmhd_get_state(h)[:, g:-g] for h in self.h], axis=1)

    def close(self):
        for h in self.h:
            L.lbmhd_destroy(h)
