"""Autotuner of the launch shape and the Verlet-list schedule.

For a given set of replicas it times md_step on the GPU for candidate settings and
returns the fastest:
  - threads per atom (tpa) and threads per block of the pair kernels,
  - the Verlet skin (list radius rc + skin; a thinner skin means shorter lists but more
    frequent rebuilds, Sec. 2.6),
  - the rebuild rule: the displacement test (rebuild_every = 0) or a fixed interval, the
    interval being the mean interval the displacement test chose, shortened by a safety
    factor (a fixed interval that is too long is reported as MD_ERR_SKIN_VIOLATION).

Every candidate runs from the same initial state, so the choice depends on the
workload only; the tuned options are plain md_options fields.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Iterable, List, Optional, Sequence, Tuple

from . import md


@dataclasses.dataclass
class Tuned:
    tpa: int
    block: int
    skin: float
    rebuild_every: int
    ms_per_step: float
    table: List[Tuple[dict, float]]


def _time_steps(sim: "md.MD", warmup: int, steps: int) -> float:
    import torch
    sim.step(warmup)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def autotune(replicas: Sequence, params: Optional[dict] = None, precision: str = "mixed",
             shapes: Iterable[Tuple[int, int]] = ((1, 64), (1, 128), (2, 128), (4, 128)),
             skins: Iterable[float] = (0.3, 0.6, 1.0, 1.1), steps: int = 60, warmup: int = 5,
             base_skin: float = 0.3,
             interval_safety: float = 0.7, log=None) -> Tuned:
    """Time each (tpa, block) at base_skin, then each skin with the best shape, then
    a fixed rebuild interval derived from the best skin's observed rebuild rate."""
    params = params or md.load_params()
    table: List[Tuple[dict, float]] = []

    def trial(**opt) -> float:
        t0 = time.perf_counter()
        try:
            sim = md.MD(replicas, params, precision=precision, **opt)
            try:
                ms = _time_steps(sim, warmup, steps)
                e = sim.energy(0)
                opt = dict(opt, rebuilds=e["rebuilds"])
            finally:
                sim.close()
        except md.MDError as err:
            ms = float("inf")
            opt = dict(opt, error=str(err))
        table.append((opt, ms))
        if log:
            log(f"autotune {opt}: {ms:.4f} ms/step ({time.perf_counter() - t0:.1f} s)")
        return ms

    best_shape = min(shapes, key=lambda sb: trial(tpa=sb[0], block=sb[1], skin=base_skin))
    tpa, block = best_shape
    best_skin, best_ms = base_skin, None
    for skin in skins:
        ms = trial(tpa=tpa, block=block, skin=skin) if skin != base_skin else \
            next(m for o, m in table if o.get("tpa") == tpa and o.get("block") == block and o.get("skin") == base_skin)
        if best_ms is None or ms < best_ms:
            best_skin, best_ms = skin, ms
    # fixed interval from the displacement test's own rebuild rate at the chosen skin
    rebuilds = next((o.get("rebuilds", 0) for o, m in table
                     if o.get("skin") == best_skin and o.get("tpa") == tpa and o.get("block") == block), 0)
    rebuild_every = 0
    if rebuilds > 0:
        interval = max(1, int(interval_safety * (warmup + steps) / rebuilds))
        ms = trial(tpa=tpa, block=block, skin=best_skin, rebuild_every=interval)
        if ms < best_ms:
            rebuild_every, best_ms = interval, ms
    return Tuned(tpa=tpa, block=block, skin=best_skin, rebuild_every=rebuild_every, ms_per_step=best_ms, table=table)
