#!/usr/bin/env python3
"""Benchmark of the per-timestep short-range force evaluation (EAM Cr-Cr + Morse Cr-C +
velocity Verlet) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 1M] [--impl reference]

Metric: Cr atom-timesteps/s of md_step on the named workload (whole job over all ranks;
replicas shard across ranks with no data-path collective: "scaling": "weak").  Prints ONE
JSON line on rank 0.  --impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import md_inputs as mi  # noqa: E402

METRIC = "atom-timesteps/s (Cr), md_step on one GB300"
UNIT = "atom-steps/s"

WORKLOAD_TEXT = {
    "tiny": "tiny: Cr film 8x8x8 cells (1,024 atoms) + C hemisphere R=0.6 nm, 300 K, 20 m/s, dt=1 fs",
    "64k": "64k: Cr film 40x40x20 cells (64,000 atoms) + C hemisphere R=1.5 nm, 3 fixed planes, 300 K",
    "1M": "1M: Cr film 100x100x50 cells (1,000,000 atoms) + C hemisphere R=3 nm, 300 K, 20 m/s, dt=1 fs",
    "8M": "8M: Cr film 200x200x100 cells (8,000,000 atoms) + C hemisphere R=6 nm, 300 K, 20 m/s, dt=1 fs",
    "batched": "batched: 256 uneven replicas (6..24 x 6..24 x 6..12 cells, R 0.5-1.5 nm, 100-500 K)",
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 50):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.lines = []
        self._t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", str(self.period)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self._t:
                self._t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(name: str, rank: int):
    """The replicas rank `rank` runs.  Weak scaling: every rank runs the whole workload on
    its own GPU, rank 0 with the preset seed, other ranks with their own velocity draw
    (and, for the batched set, their own replica draw); ranks never exchange data."""
    if rank == 0:
        wl = mi.make_workload(name)
        return wl, wl.replicas
    if name == "batched":
        reps = mi.batched_replicas(256, seed_base=1507 * 1000 + 100000 * rank)
        return mi.Workload("batched", reps, steps=1000), reps
    nx, ny, nz, R, nf, steps = mi.PRESETS[name]
    reps = [mi.make_replica(name, nx, ny, nz, R, 300.0, seed=1507 * 1000 + 97 * rank, n_fixed_planes=nf)]
    return mi.Workload(name, reps, steps=steps), reps


def max_over_ranks(ms: float, dist) -> float:
    """The job's time: the slowest rank's (ranks start together after a barrier)."""
    if dist is None:
        return ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_cr_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job throughput: atoms of all ranks times steps over the slowest rank's time."""
    return n_cr_per_rank * world * steps / (ms_max * 1e-3)


def algorithmic_bytes(kernel: str, kmean: float, kin: float, kskin: float, precision: str) -> float:
    """Bytes per Cr atom the method must move in one launch of the kernel (int32 lists,
    neighbour data counted once, assuming reuse in cell order), K_in = pairs within rc (the
    paper's inner list, Sec. 2.6), K = Verlet-list length:
      mixed k_density  cnt 4 + list 4K_in + own position 16 + (F', M') out 8     = 4K_in + 28
      mixed k_force    cnt 4 + list 4K_in + position 16 + (F', M') 8 + force out 16 = 4K_in + 44,
                       plus the integrator fused in its epilogue: x, v FP64 in and out 96,
                       the FP32 position out 16, the fixed flag 1                  = 4K_in + 157
    The FP64 form walks the Verlet list with FP64 coordinates: k_density 4K + 44,
    k_force 4K + 121 (coordinates 24, (F', M') 16, force 24, v 48, flags 5)."""
    if precision == "mixed":
        if kernel == "density":
            return 4 * kin + 28
        return 4 * kin + 44 + 113
    if kernel == "density":
        return 4 * kmean + 44
    return 4 * kmean + 121


def verlet1_bytes(precision: str) -> int:
    """k_verlet1 per atom: x, v, F in (72), x, v(t+dt/2) out (48), cell 4, fixed 1; mixed adds
    the positions at the two list builds in (32) and pos4 out (16), FP64 reads x_build (24).
    In mixed precision it runs only on steps that rebuild the lists (the force epilogue makes
    the drift otherwise)."""
    return 125 + (48 if precision == "mixed" else 24)


def moved_bytes(kernel: str, kin: float, kskin: float) -> float:
    """Bytes per Cr atom this implementation's mixed kernels actually stream: the inner
    list they walk (K_skin entries within rc + inner skin), and in k_force the separate
    v(t + dt/2) array, the FP64 force store and the positions at the two list builds that
    the fused displacement tests read."""
    if kernel == "density":
        return 4 * kskin + 28
    # icnt 4 + inner list 4K_skin + position 16 + (F', M') 8 + F out 24 + v(t+dt/2) in 24 +
    # v out 24 + fixed 1 + cntc 4, and the next step's drift: x in 24, x and v(t+3dt/2) out 48,
    # position out 16, the positions at the two list builds in 32, cell 4
    return 4 * kskin + 229


def inner_mean(sim, rep, radii, sample: int = 20000, seed: int = 0):
    """Mean number of Verlet-list entries within each radius at the current positions,
    from a random sample of atoms of replica 0."""
    x = sim.state(0)[0]
    _, cnt, nbr = sim.neighbors(0, 0)
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(x), min(sample, len(x)), replace=False)
    nb = nbr[idx]
    valid = np.arange(nb.shape[1])[None, :] < cnt[idx][:, None]
    d = x[np.where(valid, nb, 0)] - x[idx][:, None, :]
    L = rep.box_hi - rep.box_lo
    for k in range(3):
        if rep.periodic[k]:
            d[..., k] -= np.round(d[..., k] / L[k]) * L[k]
    r2 = (d * d).sum(-1)
    return [float(((r2 < r * r) & valid).sum(1).mean()) for r in radii]


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("md_kernels.cu", "md_internal.h"):
        with open(os.path.join(ROOT, "paper_1507_07068_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dram_traffic(workload: str, precision: str, kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled to this
    workload; None when absent or taken from a different kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as fh:
            tr = json.load(fh)
        rec = tr.get(f"{workload}:{precision}:k_{kernel}")
        if not rec or rec.get("source_hash") != kernel_source_hash():
            return None
        return rec.get("bytes_per_launch")
    except (OSError, ValueError):
        return None


def run_gpu(args):
    import torch
    from paper_1507_07068_gb300 import md

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    params = md.load_params()
    wl, reps = make_workload(args.workload, rank)
    n_cr = sum(r.n_cr for r in reps)
    n_c = sum(r.n_c for r in reps)
    stream = torch.cuda.current_stream()
    tuned = None
    if args.autotune if args.autotune is not None else args.workload == "8M":
        # the launch shape, Verlet skin and rebuild rule chosen by timing candidates on this
        # workload (each candidate from the same initial state)
        from paper_1507_07068_gb300.autotune import autotune
        t = autotune(reps, params, precision=args.precision,
                     shapes=((1, 64), (1, 128), (1, 256), (2, 128)), skins=(0.8, 1.0, 1.1, 1.2),
                     steps=60, warmup=5, base_skin=args.skin)
        args.tpa, args.block, args.skin, args.rebuild_every = t.tpa, t.block, t.skin, t.rebuild_every
        tuned = {"chosen": {"tpa": t.tpa, "block": t.block, "skin_A": t.skin, "rebuild_every": t.rebuild_every,
                            "ms_per_step": t.ms_per_step},
                 "table": [dict(o, ms_per_step=m) for o, m in t.table]}
    sim = md.MD(reps, params, precision=args.precision, skin=args.skin, rebuild_every=args.rebuild_every,
                tpa=args.tpa, block=args.block, use_graph=not args.no_graph, inner_skin=args.inner_skin)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timed region (graph replay)
    sim.step(args.warmup)
    e0 = sim.energy(0)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    e1 = sim.energy(0)
    rebuilds = e1["rebuilds"] - e0["rebuilds"]
    t_max = max_over_ranks(ms, dist)
    value = job_value(n_cr, ws, args.steps, t_max)

    # ---- per-kernel device time (direct launches with CUDA events around each phase);
    # profiled until at least one list rebuild has been timed (for the amortised rate)
    prof = sim.step_profiled(args.profile_steps)
    while prof["rebuilds"] == 0 and prof["steps"] < 8 * args.profile_steps:
        more = sim.step_profiled(args.profile_steps)
        prof = {k: prof[k] + more[k] for k in prof}
    # rebuild rate of the displacement rule, over an untimed stretch of steps
    r0 = sim.energy(0)["rebuilds"]
    sim.step(args.rate_steps)
    rate = (sim.energy(0)["rebuilds"] - r0) / args.rate_steps
    # one rebuild costs the list build plus the k_verlet1 that redoes the step's drift
    ms_rebuild = ((prof["rebuild"] + prof["verlet1"]) / prof["rebuilds"]) if prof["rebuilds"] else None
    value_amortised = None
    if ms_rebuild is not None:
        t_amort = t_max + (rate * args.steps - rebuilds) * ms_rebuild
        value_amortised = {"value": job_value(n_cr, ws, args.steps, t_amort), "unit": UNIT,
                           "rebuilds_per_step": rate, "ms_per_rebuild": ms_rebuild,
                           "how": "timed steps + (rebuild rate x steps - rebuilds in the timed region) "
                                  "x measured rebuild time"}
    _, cnt, _ = sim.neighbors(0, 0, kmax=1)
    kmean = float(cnt.mean())
    inner_skin = args.inner_skin if args.inner_skin > 0 else (0.0 if args.inner_skin < 0 else 0.1)
    kin, kskin = inner_mean(sim, reps[0], (params["rc"], params["rc"] + inner_skin))
    phases = {k: prof[k] / prof["steps"] for k in ("skin", "rebuild", "verlet1", "density", "morse", "force", "reduce")}
    dom = "force" if phases["force"] >= phases["density"] else "density"
    peak, peak_kind = load_peaks()
    bytes_per_launch = algorithmic_bytes(dom, kmean, kin, kskin, args.precision) * n_cr
    achieved = bytes_per_launch / (phases[dom] * 1e-3) / 1e9
    traffic = dram_traffic(args.workload, args.precision, dom)
    # the whole step: the per-step kernels' algorithmic bytes (rebuilds excluded) over the
    # measured time per step
    every_step_v1 = args.precision != "mixed"
    step_bytes = (algorithmic_bytes("density", kmean, kin, kskin, args.precision)
                  + algorithmic_bytes("force", kmean, kin, kskin, args.precision)
                  + (verlet1_bytes(args.precision) if every_step_v1 else 0)) * n_cr
    step_gbs = step_bytes / (t_max / args.steps * 1e-3) / 1e9
    step_roofline = {"bytes_per_atom": step_bytes / n_cr, "achieved": step_gbs, "peak": peak, "unit": "GB/s",
                     "frac": step_gbs / peak,
                     "kernels": ("k_verlet1 + k_density + k_force" if every_step_v1 else
                                 "k_density + k_force (drift fused; k_verlet1 only on list-build steps)")
                     + " (rebuilds excluded)"}

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timing
    e2e = None
    if not args.no_e2e and len(reps) >= 1:
        r0 = reps[0]
        n0 = r0.n_cr
        hx = torch.empty((n0, 3), dtype=torch.float64, pin_memory=True).numpy()
        hv = torch.empty((n0, 3), dtype=torch.float64, pin_memory=True).numpy()
        x, v, z, st = sim.state(0)
        hx[:] = x; hv[:] = v

        def exchange():
            # H2D of this step's inputs, one step, D2H of its result and energies (in place)
            _, _, en = md.md_step_io(sim.h, 0, hx, hv, z, st, 1, hx, hv)
            return en["z_indenter"], en["step"]

        def in_turn():
            sim.set_state(0, hx, hv, z, st)
            sim.step(1)
            md.md_get_state(sim.h, 0, n0, hx, hv)
            en = sim.energy(0)
            return en["z_indenter"], en["step"]

        rates = {}
        for name, fn in (("in_turn", in_turn), ("step_io", exchange)):
            for _ in range(2):
                z, st = fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                z, st = fn()
            rates[name] = n0 * args.e2e_steps / (time.perf_counter() - t0)
        e2e = {"value": rates["step_io"], "unit": UNIT,
               "h2d_bytes_per_step": int(hx.nbytes + hv.nbytes + 16),
               "d2h_bytes_per_step": int(hx.nbytes + hv.nbytes + md.C.sizeof(md.md_energy)),
               "path": "md_step_io(replica 0, n = 1): H2D of x, v; one step; D2H of x, v, energies",
               "value_calls_in_turn": rates["in_turn"],
               "calls_in_turn": "md_set_state + md_step(1) + md_get_state + md_get_energy"}

    # ---- variants on the same GPU: plain FP64 form on this workload, batched replicas
    variants = {}
    if not args.no_variants and rank == 0:
        if args.precision != "fp64":
            s64 = md.MD(reps, params, precision="fp64", skin=0.3)   # the FP64 loops walk the Verlet list: a thin skin
            s64.step(3)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
            k64 = max(5, min(args.steps, args.fp64_steps))
            a0.record(stream); s64.step(k64); a1.record(stream); torch.cuda.synchronize()
            variants["fp64"] = {"value": n_cr * k64 / (a0.elapsed_time(a1) * 1e-3), "steps": k64, "skin_A": 0.3,
                                "ms_per_step": a0.elapsed_time(a1) / k64,
                                # the bound of this form: the CUDA cores' FP64 FMA rate, measured here
                                "fp64_fma_peak_tflops": md.md_probe_fp64_fma() * 1e-12}
            s64.close()
        if args.workload != "batched":
            bw = mi.make_workload("batched")
            sb = md.MD(bw.replicas, params, precision="mixed", skin=args.skin)
            sb.step(10)
            torch.cuda.synchronize()
            b0 = torch.cuda.Event(enable_timing=True); b1 = torch.cuda.Event(enable_timing=True)
            kb = max(10, min(args.steps, args.batched_steps))
            b0.record(stream); sb.step(kb); b1.record(stream); torch.cuda.synchronize()
            variants["batched_mixed"] = {"value": bw.n_cr * kb / (b0.elapsed_time(b1) * 1e-3), "steps": kb, "skin_A": args.skin,
                                         "replicas": len(bw.replicas), "n_cr": bw.n_cr,
                                         "ms_per_step": b0.elapsed_time(b1) / kb}
            sb.close()
        if not args.no_paper_cubes:
            variants["paper_table2_rstar"] = paper_cubes()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, params, args.cpu_seconds, args.skin)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic (seeded BCC film + diamond hemisphere, Maxwell-Boltzmann velocities)",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "n_cr": n_cr * ws, "n_c": n_c * ws,
                   "precision": args.precision,
                   "potential": ("analytic FP32 forms in the pair loops, FP64 state" if args.precision == "mixed"
                                 else "cubic Hermite tables (FP64)") + ", shifted-force cut-offs",
                   "skin_A": args.skin,
                   "inner_list": ("rebuilt every step (radius rc)" if args.inner_skin < 0 else
                                  "skin %.3g A, rebuilt when an atom moved half of it" % (args.inner_skin or 0.1)),
                   "rebuild": ("every %d steps" % args.rebuild_every) if args.rebuild_every
                   else "displacement rule 2 max|dx| > skin (conditional graph node)",
                   "rebuilds_in_timed_region": rebuilds, "tpa": args.tpa or 1, "block": args.block or 128,
                   "l2": "working set larger than L2 (neighbour list alone %.0f MB)" % (n_cr * kmean * 4 / 1e6),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "autotuned": tuned},
        "roofline": {"bound": "hbm", "kernel": f"k_{dom}", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_atom": algorithmic_bytes(dom, kmean, kin, kskin, args.precision),
                     "moved_bytes_per_atom": (moved_bytes(dom, kin, kskin) if args.precision == "mixed"
                                              else algorithmic_bytes(dom, kmean, kin, kskin, args.precision)),
                     "mean_list_length": kmean, "mean_pairs_within_rc": kin, "mean_inner_length": kskin,
                     "launch_ms": phases[dom], "launches_timed": prof["steps"]},
        "phases_ms_per_step": phases,
        "clocks": clk.summary(),
        "e2e": e2e,
        # per step: k_decide, k_density, k_force, and k_morse_mixed (mixed) or k_verlet1 (FP64);
        # per list build 14 kernels, and in mixed precision k_verlet1; one k_reduce; the
        # checkpoint md_step keeps for a list overflow (calls of >= 16 steps: k_ckpt_save)
        "gpu_launches": int(4 * args.steps + (15 if args.precision == "mixed" else 14) * rebuilds + 1
                            + (1 if args.steps >= 16 else 0)),
        "value_incl_c": (n_cr + n_c) * ws * args.steps / (t_max * 1e-3),
        "value_amortised": value_amortised,
        "step_roofline": step_roofline,
        "variants": variants,
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    sim.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# the paper's timing runs (Table 2: time per step of its best MPI x OpenMP layout on 48
# Xeon cores, indenter disabled, r* = 8.262 A); context only: another machine, and the
# potential here is the derived set fitted with the same cut-off
PAPER_TABLE2_S_PER_STEP = {10: 0.0077, 20: 0.0567, 40: 0.4110}


def paper_cubes() -> dict:
    """The paper's timing workload on this GPU: cubes of n^3 unit cells with free faces
    (2331 / 17261 / 132921 atoms), the r* = 8.262 A parameter set, mixed and FP64, with two
    list schemes: a thin Verlet skin (1.0 A) over Hermite tables, and the paper's own
    (Sec. 2.6: outer list of radius 1.7 r*, skin 0.7 r*, inner list of radius r* rebuilt
    every step; analytic forms, Sec. 2.4)."""
    import torch
    import md_inputs as mi
    from paper_1507_07068_gb300 import md
    prs = md.load_params(os.path.join(ROOT, "paper_1507_07068_gb300", "cr_c_params_rstar.json"))
    rstar = prs["rc"]
    schemes = {"": dict(skin=1.0),
               " paper-lists": dict(skin=0.7 * rstar, inner_skin=-1.0, tabulated=0)}
    out = {"potential": "r* = 8.262 A (cr_c_params_rstar.json)", "skin_A": 1.0,
           "paper-lists": "outer list 1.7 r* (skin 0.7 r* = %.3f A), inner list r* every step, analytic forms"
                          % (0.7 * rstar)}
    for n, t_paper in PAPER_TABLE2_S_PER_STEP.items():
        rep = mi.paper_cube(n)
        for tag, kw in schemes.items():
            for prec, k in (("mixed", 200), ("fp64", 20)):
                sim = md.MD([rep], prs, precision=prec, **kw)
                sim.step(5)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
                a.record(); sim.step(k); b.record(); torch.cuda.synchronize()
                ms = a.elapsed_time(b) / k
                out[f"{n}^3 {prec}{tag}"] = {"n_cr": rep.n_cr, "steps": k, "ms_per_step": ms,
                                             "value": rep.n_cr / (ms * 1e-3), "paper_s_per_step": t_paper,
                                             "speedup_vs_paper": t_paper / (ms * 1e-3)}
                sim.close()
    return out


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample_replica(workload: str, target_atoms: int):
    """A film of the workload's kind, thinned in z to about target_atoms (same lateral size)."""
    if workload == "batched":
        return mi.batched_replicas(1)[0], "one replica of the batched set"
    nx, ny, nz, R, nf, _ = mi.PRESETS[workload]
    full = 2 * nx * ny * nz
    if target_atoms >= full:
        rep = mi.make_workload(workload).replicas[0]
        return rep, f"the full {workload} film ({full} Cr)"
    nz_s = max(4, int(target_atoms / (2 * nx * ny)))
    while 2 * nx * ny * nz_s > target_atoms and nz_s > 4:
        nz_s -= 1
    if 2 * nx * ny * nz_s > target_atoms * 2:
        # lateral thinning too (keeps the film periodic and the indenter inside)
        s = max(0.2, (target_atoms / (2 * nx * ny * nz_s)) ** 0.5)
        nx = max(int(2 * R / mi.A_CR) + 6, int(nx * s)); ny = nx
    rep = mi.make_replica(workload, nx, ny, nz_s, R, 300.0, seed=1507 + 7, n_fixed_planes=nf)
    return rep, f"{nx}x{ny}x{nz_s}-cell slab of the {workload} film ({rep.n_cr} Cr), same indenter"


def oracle_rate(params, rep, steps: int, skin: float = 0.3):
    import oracle
    pot = oracle.Potential(params)
    sim = oracle.Sim(pot, rep, skin=skin)
    t0 = time.perf_counter()
    sim.step(steps)
    return rep.n_cr * steps / (time.perf_counter() - t0)


def cpu_baseline(workload: str, params, seconds: float, skin: float = 0.3):
    """The oracle on the host cores, built -O2 (the paper's flags, Sec. 2.3: `value`) and -O3
    (`value_O3`), each on a bounded sample of the workload of about seconds / 2."""
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    probe = mi.make_replica("probe", 24, 24, 10, 6.0, 300.0, seed=3)
    rate = oracle_rate(params, probe, 2)
    target = int(rate * seconds / 12)
    rep, desc = oracle_sample_replica(workload, max(target, 20000))
    n = max(2, min(6, int(rate * seconds / 2 / max(rep.n_cr, 1))))
    v = oracle_rate(params, rep, n, skin)
    oracle.select("O3")
    try:
        v3 = oracle_rate(params, rep, n, skin)
    finally:
        oracle.select("O2")
    # one thread (-O2), on a sample sized for about seconds / 8 at the all-core rate / cores
    oracle.set_threads(1)
    try:
        rep1, desc1 = oracle_sample_replica(workload, max(int(rate / max(cores, 1) * seconds / 16), 5000))
        v1 = oracle_rate(params, rep1, 2, skin)
    finally:
        oracle.set_threads(cores)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "value_O3": v3, "value_1core": v1,
            "sample": f"{n} FP64 oracle time steps (list build excluded) on {desc}, OpenMP over {cores} threads; "
                      "value: built -O2 (the paper's flags), value_O3: the same at -O3; "
                      f"value_1core: -O2 on one thread, 2 steps on {desc1}"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    params = oracle.load_params()
    cores = oracle.set_threads(os.cpu_count() or 1)
    probe = mi.make_replica("probe", 24, 24, 10, 6.0, 300.0, seed=3)
    rate = oracle_rate(params, probe, 2)
    budget = args.ref_seconds
    per_step = budget / max(args.steps + args.warmup, 1)
    rep, desc = oracle_sample_replica(args.workload, max(int(rate * per_step), 5000))
    pot = oracle.Potential(params)
    sim = oracle.Sim(pot, rep, skin=args.skin, rebuild_every=args.rebuild_every)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    dt = time.perf_counter() - t0
    value = rep.n_cr * args.steps / dt
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded BCC film + diamond hemisphere, Maxwell-Boltzmann velocities)",
           "config": {"workload": WORKLOAD_TEXT[args.workload], "precision": "fp64 (oracle)",
                      "skin_A": args.skin, "n_cr": rep.n_cr, "sample": desc},
           "impl": "reference",
           "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                            "sample": f"each step one FP64 oracle time step on {desc}"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--workload", default="1M", choices=list(WORKLOAD_TEXT))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--tpa", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--skin", type=float, default=1.1,
                    help="Verlet skin (A); 1.1 measured fastest on the 1M film (0.2-1.2 swept)")
    ap.add_argument("--inner-skin", type=float, default=0.0,
                    help="skin of the inner list (0 = library default 0.1 A; < 0 = rebuilt every step)")
    ap.add_argument("--rebuild-every", type=int, default=0)
    ap.add_argument("--autotune", dest="autotune", action="store_true", default=None,
                    help="choose tpa, block, skin and the rebuild rule by timing (default: on for the 8M film)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--no-paper-cubes", action="store_true",
                    help="skip the variant timing the paper's Table 2 workload (r* = 8.262 A cubes)")
    ap.add_argument("--no-graph", action="store_true",
                    help="direct launches instead of graph replay (for launch-list profiling)")
    ap.add_argument("--profile-steps", type=int, default=50)
    ap.add_argument("--rate-steps", type=int, default=400,
                    help="untimed steps over which the list-rebuild rate is counted")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--fp64-steps", type=int, default=40)
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=120.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
