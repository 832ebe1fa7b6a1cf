"""Spatial decomposition of one film over ranks: the bookkeeping and the messages.

The paper splits its atoms over MPI processes (atom decomposition, Sec. 3.1) and, per time
step, makes every process's positions known to all others after Task 3 and every F'(rho),
M'(P) known to all others before the force pass (two Allgathervs, Sec. 3.3.2, Figs. 7-8).
For one film spread over several GPUs this module restates that as a spatial
decomposition, so that each rank receives only what its own atoms can reach:

  * the film is cut into a px x py grid of bricks in x and y (z is not cut); rank
    r = ix + px * iy owns the atoms whose positions, wrapped into the periodic box, fall in
    brick (ix, iy);
  * at every list rebuild (Task 1, Sec. 2.6) each rank picks, for every other brick, the
    owned atoms within `halo` (= rc + skin) of it -- with the periodic shift that places
    them next to it -- and atoms that left their brick migrate to the new owner;
  * per step, exchange 1 (after the drift of Task 3): the positions of those atoms, shifted,
    go to the ranks that hold them as ghosts; exchange 2 (after the density pass of Task
    4a): the same atoms' F'(rho), M'(P).  A pair within rc at any step before the next
    rebuild was within rc + skin at the rebuild, so the ghost sets chosen then suffice;
  * energies and the indenter load are summed over ranks (all-reduce).

This module holds no arithmetic of the method: each rank's density, force and
integration passes belong to its engine (on a GPU, the CUDA kernels of libmd, which would
receive the ghosts as atoms whose positions and F', M' are set from outside).  Messages are
torch.distributed point-to-point sends of CPU tensors (gloo); a GPU engine would pass
device tensors over NCCL, each rank's halo copied into its own memory before any kernel
reads it.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class Brick:
    lo: np.ndarray   # (3,) lower corner (z: the whole domain)
    hi: np.ndarray   # (3,)


class BrickGrid:
    """A px x py grid of bricks over the box [box_lo, box_hi) in x and y."""

    def __init__(self, box_lo, box_hi, periodic, px: int, py: int, halo: float):
        self.lo = np.asarray(box_lo, float)
        self.hi = np.asarray(box_hi, float)
        self.L = self.hi - self.lo
        self.per = np.asarray(periodic, int)
        self.px, self.py = int(px), int(py)
        self.n = self.px * self.py
        self.halo = float(halo)
        if self.px < 1 or self.py < 1:
            raise ValueError("px, py >= 1")
        self.w = np.array([self.L[0] / self.px, self.L[1] / self.py, self.L[2]])
        for k, m in ((0, self.px), (1, self.py)):
            if m > 1 and self.w[k] < self.halo:
                raise ValueError(f"bricks along axis {k} ({self.w[k]:.3f} A) narrower than the halo {self.halo:.3f} A")

    def coords(self, r: int) -> Tuple[int, int]:
        return r % self.px, r // self.px

    def brick(self, r: int) -> Brick:
        ix, iy = self.coords(r)
        lo = self.lo + np.array([ix * self.w[0], iy * self.w[1], 0.0])
        hi = lo + self.w
        if ix == self.px - 1:
            hi[0] = self.hi[0]
        if iy == self.py - 1:
            hi[1] = self.hi[1]
        return Brick(lo, hi)

    def wrap(self, x: np.ndarray) -> np.ndarray:
        """Positions wrapped into the box along periodic x, y (as a list build does)."""
        x = np.array(x, float, copy=True)
        for k in (0, 1, 2):
            if self.per[k]:
                x[:, k] = x[:, k] - np.floor((x[:, k] - self.lo[k]) / self.L[k]) * self.L[k]
        return x

    def owner(self, x: np.ndarray) -> np.ndarray:
        """Owning rank of each position (wrapped first); positions outside a non-periodic
        extent belong to the nearest brick."""
        xw = self.wrap(x)
        ix = np.clip(np.floor((xw[:, 0] - self.lo[0]) / self.w[0]).astype(np.int64), 0, self.px - 1)
        iy = np.clip(np.floor((xw[:, 1] - self.lo[1]) / self.w[1]).astype(np.int64), 0, self.py - 1)
        return ix + self.px * iy

    def _shifts(self, k: int, m: int) -> Sequence[float]:
        # a ghost crosses a periodic face of a cut axis with a shift of -+L
        return (-self.L[k], 0.0, self.L[k]) if (m > 1 and self.per[k]) else (0.0,)

    def local_box(self, r: int, reach: float = 0.0):
        """The box a rank's engine works in: along a cut axis its brick widened by the halo
        or by `reach` (the indenter's interaction range), whichever is larger, plus 1 A
        (non-periodic: the ghosts stand in for the neighbours), elsewhere the film's box."""
        b = self.brick(r)
        lo, hi, per = self.lo.copy(), self.hi.copy(), self.per.copy()
        m_ = max(self.halo, reach) + 1.0
        for k, m in ((0, self.px), (1, self.py)):
            if m > 1:
                lo[k] = b.lo[k] - m_
                hi[k] = b.hi[k] + m_
                per[k] = 0
        return lo, hi, per

    def ghost_plan(self, x_owned: np.ndarray, r: int) -> Dict[int, Tuple[np.ndarray, np.ndarray]]:
        """For every other rank d: (indices into x_owned, (m, 3) shifts) of the owned atoms
        within the halo of d's brick, each with the periodic shift that places it there (an
        atom can go to one rank under two shifts when that rank borders this one on both
        sides).  Chosen at list rebuilds."""
        plan: Dict[int, Tuple[np.ndarray, np.ndarray]] = {}
        x = np.asarray(x_owned, float)
        h = self.halo
        for d in range(self.n):
            if d == r:
                continue
            b = self.brick(d)
            idx_all: List[np.ndarray] = []
            sh_all: List[np.ndarray] = []
            for sx in self._shifts(0, self.px):
                for sy in self._shifts(1, self.py):
                    s = np.array([sx, sy, 0.0])
                    y = x + s
                    inside = np.ones(len(x), bool)
                    for k, m in ((0, self.px), (1, self.py)):
                        if m > 1:
                            inside &= (y[:, k] >= b.lo[k] - h) & (y[:, k] < b.hi[k] + h)
                    sel = np.nonzero(inside)[0]
                    if len(sel):
                        idx_all.append(sel)
                        sh_all.append(np.repeat(s[None, :], len(sel), 0))
            if idx_all:
                plan[d] = (np.concatenate(idx_all), np.concatenate(sh_all))
        return plan


class Exchange:
    """Variable-size messages between all pairs of ranks over torch.distributed: the counts
    go first (one all-gather of a world-sized row), then one send per non-empty part, every
    receive posted before any send."""

    def __init__(self, dist, rank: int, world: int):
        self.dist, self.rank, self.world = dist, rank, world

    def all_to_all(self, parts: Dict[int, np.ndarray], width: int, dtype=np.float64) -> Dict[int, np.ndarray]:
        import torch
        d = self.dist
        counts = torch.zeros(self.world, dtype=torch.int64)
        for dst, a in parts.items():
            counts[dst] = len(a)
        rows = [torch.zeros(self.world, dtype=torch.int64) for _ in range(self.world)]
        d.all_gather(rows, counts)
        tdt = torch.float64 if dtype == np.float64 else torch.int64
        recv, reqs = {}, []
        for src in range(self.world):
            m = int(rows[src][self.rank])
            if src != self.rank and m > 0:
                buf = torch.empty((m, width), dtype=tdt)
                recv[src] = buf
                reqs.append(d.irecv(buf, src))
        for dst, a in parts.items():
            if dst != self.rank and len(a) > 0:
                reqs.append(d.isend(torch.from_numpy(np.ascontiguousarray(a, dtype=dtype).reshape(len(a), width)), dst))
        for q in reqs:
            q.wait()
        return {src: buf.numpy() for src, buf in recv.items()}

    def sum(self, values: Sequence[float]) -> np.ndarray:
        """Sum over ranks of a few scalars (energies, load), FP64."""
        import torch
        t = torch.tensor(np.asarray(values, float), dtype=torch.float64)
        self.dist.all_reduce(t)
        return t.numpy()

    def max(self, value: float) -> float:
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


class Halo:
    """The ghost sets of one rank between two rebuilds and the two per-step exchanges.

    Local atom order for the engine: the owned atoms, then the ghosts grouped by source rank
    (ascending) in the order their owner sent them."""

    def __init__(self, grid: BrickGrid, ex: Exchange, x_owned: np.ndarray):
        self.grid, self.ex = grid, ex
        self.plan = grid.ghost_plan(x_owned, ex.rank)
        self.n_ghost = None

    def positions(self, x_owned: np.ndarray) -> np.ndarray:
        """Exchange 1: ghost positions (shifted) from their owners, (n_ghost, 3)."""
        parts = {d: x_owned[idx] + sh for d, (idx, sh) in self.plan.items()}
        got = self.ex.all_to_all(parts, 3)
        g = np.concatenate([got[s] for s in sorted(got)]) if got else np.zeros((0, 3))
        self.n_ghost = len(g)
        return g

    def values(self, v_owned: np.ndarray) -> np.ndarray:
        """Exchange 2 (or any per-atom values of the owned atoms, e.g. F'(rho), M'(P)): the
        ghosts' values, in the order of `positions`."""
        v_owned = np.asarray(v_owned, float)
        w = 1 if v_owned.ndim == 1 else v_owned.shape[1]
        parts = {d: v_owned[idx].reshape(len(idx), w) for d, (idx, _) in self.plan.items()}
        got = self.ex.all_to_all(parts, w)
        g = np.concatenate([got[s] for s in sorted(got)]) if got else np.zeros((0, w))
        return g if v_owned.ndim > 1 else g[:, 0]


def migrate(grid: BrickGrid, ex: Exchange, ids: np.ndarray, arrays: Sequence[np.ndarray]):
    """Atoms whose wrapped positions (arrays[0], (n, 3)) left this rank's brick go to their
    new owners.  Returns (ids, arrays) of the atoms owned afterwards, positions wrapped,
    sorted by global id (so the local order does not depend on the history)."""
    x = grid.wrap(arrays[0])
    arrays = [x] + [np.asarray(a) for a in arrays[1:]]
    cols = [a.reshape(len(ids), -1).astype(np.float64) for a in arrays]
    widths = [c.shape[1] for c in cols]
    table = np.concatenate([np.asarray(ids, np.float64)[:, None]] + cols, axis=1)
    own = grid.owner(x)
    keep = own == ex.rank
    parts = {int(d): table[own == d] for d in np.unique(own[~keep])}
    got = ex.all_to_all(parts, table.shape[1])
    table = np.concatenate([table[keep]] + [got[s] for s in sorted(got)])
    table = table[np.argsort(table[:, 0], kind="stable")]
    out, c = [], 1
    for a, wdt in zip(arrays, widths):
        col = table[:, c:c + wdt]
        out.append(col.astype(a.dtype).reshape((len(table),) + a.shape[1:]))
        c += wdt
    return table[:, 0].astype(np.int64), out
