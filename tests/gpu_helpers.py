"""Shared helpers of the GPU parity tests (no method arithmetic: metrics and inputs only)."""
import numpy as np

import md_inputs as mi


def rel_force_err(F, ref):
    """Per-atom ||dF_i|| / max(||F_i||, F_rms), F_rms the system RMS force (a per-atom ratio
    is ill-posed for the near-zero net forces of a lattice)."""
    F = np.asarray(F).reshape(-1, 3); ref = np.asarray(ref).reshape(-1, 3)
    nrm = np.sqrt((ref ** 2).sum(1))
    frms = np.sqrt((ref ** 2).sum(1).mean())
    return np.sqrt(((F - ref) ** 2).sum(1)) / np.maximum(nrm, frms)


def jitter(rep, amp=0.1, seed=0):
    rng = np.random.default_rng(seed)
    rep.x_cr = np.ascontiguousarray(rep.x_cr + rng.uniform(-amp, amp, rep.x_cr.shape))
    return rep


def tiny(seed=1507, gap=1.5, T=300.0, R=6.0, amp=0.1, n=8, nz=8, **kw):
    rep = mi.make_replica("tiny", n, n, nz, R, T, seed=seed, gap=gap, **kw)
    return jitter(rep, amp, seed)


def min_image_r(x, i, j, lo, hi, per):
    d = x[j] - x[i]
    L = hi - lo
    for k in range(3):
        if per[k]:
            if d[k] > 0.5 * L[k]:
                d[k] -= L[k]
            elif d[k] < -0.5 * L[k]:
                d[k] += L[k]
    return float(np.sqrt((d * d).sum()))


def compare_sets(gpu_cnt, gpu_nbr, off, idx, near_cut):
    """Exact set equality per atom, except pairs for which near_cut(i, j) is True."""
    n = len(gpu_cnt)
    bad = []
    for i in range(n):
        g = set(gpu_nbr[i, :gpu_cnt[i]].tolist())
        o = set(idx[off[i]:off[i + 1]].tolist())
        for j in g ^ o:
            if not near_cut(i, j):
                bad.append((i, j))
    return bad
