"""Nano-indentation run on the library and the analysis of its load-depth curve.

The run follows the paper's protocol (Sec. 2.5, Sec. 4.3): the rigid indenter is held
while the film relaxes, driven into the film at constant speed to a maximum depth, then
withdrawn at the same speed; the load on the indenter and its depth are sampled along
the way.  The analysis gives the reduced modulus from the loading branch by the Hertz
contact law of a sphere, and the reduced modulus and hardness from the unloading branch
by the method of W. C. Oliver and G. M. Pharr (J. Mater. Res. 7, 1564 (1992)).

Units: depth in A, load in eV/A, moduli and hardness in eV/A^3 (times EV_A3_IN_GPA for GPa).
Depth is that of the indenter's lowest atom below the film's top plane at t = 0, so it
starts at minus the initial gap.
"""
from __future__ import annotations

import math
import os
from typing import Optional

import numpy as np

EV_A3_IN_GPA = 160.21766208   # 1 eV/A^3 in GPa


def run(sim, replica: int = 0, relax_steps: int = 0, depth_max: float = 3.08, speed: float = 1e-4,
        sample_every: int = 10, unload_to: Optional[float] = None, max_steps: int = 10_000_000) -> dict:
    """Drive replica `replica` of the MD handle `sim` (paper_1507_07068_gb300.md.MD) through
    relax (indenter at rest), load (downwards at `speed` A/fs until the depth reaches
    `depth_max`) and unload (upwards at `speed` until the depth is back to `unload_to`,
    default the depth at the start of loading).  Every `sample_every` steps the step,
    indenter displacement, depth, load, temperature and potential energy are recorded
    (the time histories of Sec. 3.1).  Returns the samples as arrays
    and the index of the first unloading sample."""
    if speed <= 0 or sample_every < 1:
        raise ValueError("speed > 0 and sample_every >= 1 are required")
    rec = {"step": [], "z_ind": [], "depth": [], "load": [], "temperature": [], "potential": [], "phase": []}

    def sample(phase):
        e = sim.energy(replica)
        rec["step"].append(e["step"]); rec["z_ind"].append(e["z_indenter"])
        rec["depth"].append(e["depth"]); rec["load"].append(e["load"]); rec["phase"].append(phase)
        rec["temperature"].append(e["temperature"]); rec["potential"].append(e["potential"])
        return e

    sim.set_indenter_velocity(replica, 0.0)
    done = 0
    while done < relax_steps:
        k = min(sample_every, relax_steps - done)
        sim.step(k); done += k
        sample(0)
    e = sample(0) if not rec["step"] else sim.energy(replica)
    depth0 = e["depth"]
    sim.set_indenter_velocity(replica, -speed)
    steps = 0
    while e["depth"] < depth_max:
        if steps >= max_steps:
            raise RuntimeError("loading did not reach depth_max")
        sim.step(sample_every); steps += sample_every
        e = sample(1)
    i_unload = len(rec["step"])
    target = depth0 if unload_to is None else unload_to
    sim.set_indenter_velocity(replica, speed)
    while e["depth"] > target:
        if steps >= 2 * max_steps:
            raise RuntimeError("unloading did not reach its end depth")
        sim.step(sample_every); steps += sample_every
        e = sample(2)
    sim.set_indenter_velocity(replica, 0.0)
    out = {k: np.asarray(v) for k, v in rec.items()}
    out["i_unload"] = i_unload
    return out


def hertz_modulus(depth: np.ndarray, load: np.ndarray, R: float) -> float:
    """Reduced modulus E* of the Hertz law of a sphere of radius R pressed to depth h,
    P = (4/3) E* R^(1/2) h^(3/2), by least squares through the origin over the samples
    with h > 0."""
    h = np.asarray(depth, float)
    P = np.asarray(load, float)
    m = h > 0
    if not m.any():
        raise ValueError("no sample in contact (depth > 0)")
    g = (4.0 / 3.0) * math.sqrt(R) * h[m] ** 1.5
    return float(np.dot(g, P[m]) / np.dot(g, g))


def contact_area(h_c: float, R: float) -> float:
    """Projected contact area of a sphere of radius R at contact depth h_c (< R)."""
    if not (0.0 < h_c < R):
        raise ValueError("contact depth outside (0, R)")
    return math.pi * (2.0 * R * h_c - h_c * h_c)


def oliver_pharr(depth: np.ndarray, load: np.ndarray, R: float, top: float = 0.6, eps: float = 0.75) -> dict:
    """Oliver-Pharr analysis of an unloading branch (samples ordered from maximum depth
    outwards).  The upper `top` fraction of the load range is fitted by
    P = alpha (h - h_f)^m; the contact stiffness is S = dP/dh at the maximum depth, the
    contact depth h_c = h_max - eps P_max / S (eps = 0.75 for a paraboloid), the area that
    of a sphere's cap at h_c, the reduced modulus E_r = sqrt(pi) S / (2 sqrt(A)) and the
    hardness H = P_max / A."""
    from scipy.optimize import curve_fit

    h = np.asarray(depth, float)
    P = np.asarray(load, float)
    i = int(np.argmax(P))
    h_max, P_max = h[i], P[i]
    keep = P >= (1.0 - top) * P_max
    hf, Pf = h[keep], P[keep]
    if len(hf) < 4:
        raise ValueError("too few unloading samples in the fitted range")

    def law(x, alpha, h_f, m):
        return alpha * np.clip(x - h_f, 1e-12, None) ** m

    h_f0 = float(hf.min()) - 0.5 * float(hf.max() - hf.min()) - 1e-3
    m0 = 1.5
    alpha0 = P_max / max(h_max - h_f0, 1e-6) ** m0
    (alpha, h_f, m), _ = curve_fit(law, hf, Pf, p0=(alpha0, h_f0, m0), maxfev=20000)
    S = alpha * m * (h_max - h_f) ** (m - 1.0)
    h_c = h_max - eps * P_max / S
    A = contact_area(h_c, R)
    E_r = math.sqrt(math.pi) * S / (2.0 * math.sqrt(A))
    return {"alpha": float(alpha), "h_f": float(h_f), "m": float(m), "h_max": float(h_max), "P_max": float(P_max),
            "S": float(S), "h_c": float(h_c), "A": float(A), "E_r": float(E_r), "H": float(P_max / A)}


def main(argv=None) -> int:
    """Run the protocol on one of the seeded synthetic films and print the analysis as one
    JSON line (the potential parameters are the derived set the library ships with, not
    the paper's, so the moduli are not the paper's)."""
    import argparse
    import json

    import md_inputs as mi
    from paper_1507_07068_gb300 import md

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--workload", default="p11k",
                    help="p11k: the paper's 11k system (Sec. 2.5), or a preset film (tiny, 64k, 1M, 8M)")
    ap.add_argument("--params", default="",
                    help="parameter JSON (default: cr_c_params_indent.json for p11k, else cr_c_params.json)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--relax", type=int, default=10000, help="steps with the indenter at rest")
    ap.add_argument("--depth", type=float, default=3.08, help="maximum depth (A)")
    ap.add_argument("--speed-ms", type=float, default=10.0, help="indenter speed (m/s)")
    ap.add_argument("--sample-every", type=int, default=100)
    ap.add_argument("--skin", type=float, default=1.1)
    ap.add_argument("--kcmax", type=int, default=512,
                    help="Cr-C list capacity (a deep indent puts many C atoms in reach of one Cr atom)")
    ap.add_argument("--curve", default="", help="write the samples to this .npz file")
    args = ap.parse_args(argv)
    if args.workload == "p11k":
        rep, R = mi.paper_indentation_film(), 9.78
        pfile = args.params or os.path.join(os.path.dirname(os.path.abspath(__file__)), "cr_c_params_indent.json")
    elif args.workload in mi.PRESETS:
        rep = mi.make_workload(args.workload).replicas[0]
        R = float(mi.PRESETS[args.workload][3])   # the hemisphere's radius (A)
        pfile = args.params or None
    else:
        raise SystemExit(f"--workload: p11k or one of {sorted(mi.PRESETS)}")
    params = md.load_params(pfile) if pfile else md.load_params()
    sim = md.MD([rep], params, precision=args.precision, skin=args.skin, kcmax=args.kcmax)
    out = run(sim, 0, relax_steps=args.relax, depth_max=args.depth, speed=args.speed_ms * 1e-5,
              sample_every=args.sample_every)
    sim.close()
    if args.curve:
        np.savez(args.curve, **{k: v for k, v in out.items() if k != "i_unload"}, i_unload=out["i_unload"])
    iu = out["i_unload"]
    res = {"workload": args.workload, "n_cr": int(rep.n_cr), "n_c": int(rep.n_c), "precision": args.precision,
           "params": os.path.basename(pfile) if pfile else "cr_c_params.json",
           "steps": int(out["step"][-1]), "max_load": float(out["load"].max()), "min_load": float(out["load"].min()),
           "depth_at_max_load": float(out["depth"][int(np.argmax(out["load"]))])}
    if R > 0 and out["load"][:iu].max() <= 0:
        # the Hertz law and the Oliver-Pharr analysis describe a repulsive contact
        res["analysis_error"] = "no repulsive load while loading (the Cr-C attraction dominates)"
    elif R > 0:
        res["R"] = R
        try:
            res["hertz_E"] = hertz_modulus(out["depth"][:iu], out["load"][:iu], R)
            res["hertz_E_GPa"] = res["hertz_E"] * EV_A3_IN_GPA
            op = oliver_pharr(out["depth"][iu - 1:], out["load"][iu - 1:], R)
            res.update({"op_" + k: v for k, v in op.items()})
            res["op_E_r_GPa"] = op["E_r"] * EV_A3_IN_GPA
            res["op_H_GPa"] = op["H"] * EV_A3_IN_GPA
        except (ValueError, RuntimeError) as e:
            res["analysis_error"] = str(e)
    print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
