"""Dynamics on the GPU: NVE energy conservation of the FP64 and mixed-precision forms
(static indenter, no fixed atoms, periodic x, y: nothing does work on the film), the mixed
form's trajectory against the FP64 form, and the autotuner."""
import json
import os

import numpy as np
import pytest

import md_inputs as mi
import oracle
from gpu_helpers import rel_force_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1507_07068_gb300 import md as mdmod
    mdmod.lib()
    return mdmod


def nve_film():
    return mi.make_replica("nve", 16, 16, 8, 8.0, 300.0, seed=11, n_fixed_planes=0, v_ind_ms=0.0, gap=2.0)


def energy_series(md, params, rep, precision, steps=1000, every=50):
    sim = md.MD([rep], params, precision=precision)
    E = [sim.energy(0)["total"]]
    for _ in range(steps // every):
        sim.step(every)
        E.append(sim.energy(0)["total"])
    rebuilds = sim.energy(0)["rebuilds"]
    sim.close()
    return np.array(E), rebuilds


def test_nve_energy_drift(md, params):
    rep = nve_film()
    N = rep.n_cr
    out = {}
    for prec in ("fp64", "mixed"):
        E, nreb = energy_series(md, params, rep, prec)
        dev = np.abs(E - E[0]).max() / N
        # drift per 1000 steps: least-squares slope of E(t)
        t = np.arange(len(E)) * 50.0
        slope = np.polyfit(t, E, 1)[0] * 1000.0 / N
        out[prec] = dict(max_dev_per_atom=float(dev), drift_per_1000_steps_per_atom=float(slope), rebuilds=int(nreb))
        assert dev < 5e-5, (prec, dev)
        assert abs(slope) < 2e-5, (prec, slope)
    print("NVE", json.dumps(out))
    res = os.environ.get("MD_RESULTS_DIR")   # optional: keep the numbers as a file
    if res:
        os.makedirs(res, exist_ok=True)
        with open(os.path.join(res, "nve_drift.json"), "w") as fh:
            json.dump(out, fh, indent=1)


def test_mixed_trajectory_tracks_fp64(md, params):
    rep = mi.make_replica("traj", 12, 12, 8, 8.0, 300.0, seed=5, gap=2.0)
    a = md.MD([rep], params, precision="fp64")
    b = md.MD([rep], params, precision="mixed")
    a.step(200); b.step(200)
    xa = a.state(0)[0]; xb = b.state(0)[0]
    L = rep.box_hi - rep.box_lo
    d = xb - xa
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-4
    ea, eb = a.energy(0), b.energy(0)
    assert eb["total"] == pytest.approx(ea["total"], abs=1e-5 * rep.n_cr)


def test_autotune_picks_a_valid_configuration(md, params):
    from paper_1507_07068_gb300.autotune import autotune
    rep = mi.make_replica("tune", 16, 16, 8, 8.0, 300.0, seed=3, gap=2.0)
    best = autotune([rep], params, steps=20, warmup=3, shapes=((1, 128), (2, 128)), skins=(0.2, 0.3))
    assert best.tpa in (1, 2) and best.block == 128 and best.skin in (0.2, 0.3)
    assert np.isfinite(best.ms_per_step) and best.ms_per_step > 0
    assert len(best.table) >= 3
    sim = md.MD([rep], params, precision="mixed", tpa=best.tpa, block=best.block, skin=best.skin,
                rebuild_every=best.rebuild_every)
    o = oracle.forces(oracle.Potential(params), rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c)
    # the perfect lattice at t = 0: interior forces vanish by symmetry, F_rms is small
    assert rel_force_err(sim.forces(0), o["F"]).max() <= 1e-5
    sim.step(50)
