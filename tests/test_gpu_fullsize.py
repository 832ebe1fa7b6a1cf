"""Parity at full size in the launch configuration the benchmark times (mixed precision,
default launch shape, cell order and lists as built by the library): the 1,000,000- and
8,000,000-atom films and the 256-replica batch against the FP64 oracle over every atom."""
import dataclasses

import numpy as np
import pytest

import md_inputs as mi
import oracle
from gpu_helpers import rel_force_err

pytestmark = pytest.mark.gpu

SKIN = 1.1   # the Verlet skin of the benchmark's configuration


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1507_07068_gb300 import md as mdmod
    mdmod.lib()
    return mdmod


@pytest.fixture(scope="module")
def film_1m():
    oracle.set_threads(0)
    return mi.make_workload("1M").replicas[0]


@pytest.fixture(scope="module")
def thermal_1m(md, params, film_1m):
    """The 1M film after 100 FP64 steps on the GPU (a thermal configuration)."""
    sim = md.MD([film_1m], params, precision="fp64", skin=SKIN)
    sim.step(100)
    x, v, z, st = sim.state(0)
    F64 = sim.forces(0)
    sim.close()
    return dataclasses.replace(film_1m, x_cr=x, v_cr=v, z_indenter0=z), F64


def test_fullsize_fp64_forces_and_lists(md, params, thermal_1m):
    rep, F64 = thermal_1m
    ref = oracle.forces(oracle.Potential(params), rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic,
                        rep.x_c + np.array([0.0, 0.0, rep.z_indenter0]))
    assert rel_force_err(F64, ref["F"]).max() <= 1e-11
    sim = md.MD([rep], params, precision="fp64", skin=SKIN)
    e = sim.energy(0)
    assert e["potential"] == pytest.approx(ref["potential"], rel=1e-12)
    assert e["load"] == pytest.approx(ref["load"], rel=1e-9, abs=1e-9)
    # neighbour sets of a sample of atoms, bit-exact
    cut = params["rc"] + SKIN
    cell, cnt, nbr = sim.neighbors(0, 0)
    ocell = oracle.cell_coords(rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, cut)
    assert np.array_equal(cell, ocell)
    off, idx = oracle.neighbors(rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, cut, method=1)
    rng = np.random.default_rng(0)
    for i in rng.choice(rep.n_cr, 3000, replace=False):
        assert set(nbr[i, :cnt[i]].tolist()) == set(idx[off[i]:off[i + 1]].tolist())
    sim.close()


def test_fullsize_mixed_forces(md, params, thermal_1m):
    rep, _ = thermal_1m
    sim = md.MD([rep], params, precision="mixed", skin=SKIN)
    Fm = sim.forces(0)
    ref = oracle.forces(oracle.Potential(params), rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic,
                        rep.x_c + np.array([0.0, 0.0, rep.z_indenter0]))
    assert all(v == 0 for v in sim.check_lists().values())
    err = rel_force_err(Fm, ref["F"])
    print("1M mixed: max %.2e p99 %.2e median %.2e F_rms %.3f" % (err.max(), np.quantile(err, 0.99),
                                                                   np.median(err), np.sqrt((ref["F"] ** 2).sum(1).mean())))
    assert err.max() <= 1e-5
    e = sim.energy(0)
    assert e["potential"] == pytest.approx(ref["potential"], rel=1e-6)
    sim.close()


def test_fullsize_load_curve_and_energy_against_oracle(md, params, film_1m):
    """The 1M configuration's load-displacement curve and energy history over 1 000 steps
    from the seeded state (indenter coming down at 20 m/s inside the Morse range of the
    surface), mixed precision against the FP64 oracle's own run of the same steps (OpenMP
    over the host's cores), sampled every 100 steps; the GPU's FP64 form beside it."""
    oracle.set_threads(0)
    osim = oracle.Sim(oracle.Potential(params), film_1m, skin=SKIN)
    sims = {p: md.MD([film_1m], params, precision=p, skin=SKIN) for p in ("fp64", "mixed")}
    hist = {p: [] for p in ("oracle", "fp64", "mixed")}
    for _ in range(10):
        osim.step(100)
        st = osim.state()
        hist["oracle"].append((st["z_ind"], st["load"], st["total"]))
        for p, sim in sims.items():
            sim.step(100)
            e = sim.energy(0)
            hist[p].append((e["z_indenter"], e["load"], e["total"]))
    for sim in sims.values():
        sim.close()
    o, a, b = (np.array(hist[k]) for k in ("oracle", "fp64", "mixed"))
    assert np.array_equal(o[:, 0], b[:, 0]) and np.array_equal(o[:, 0], a[:, 0])   # the same indenter path
    scale = np.abs(o[:, 1]).max()
    assert scale > 0.1                                              # the film pulls on the indenter
    assert np.abs(b[:, 1] - o[:, 1]).max() <= 2e-3 * scale          # load curves agree
    assert np.abs(a[:, 1] - o[:, 1]).max() <= 1e-6 * scale
    n = film_1m.n_cr
    drift_o, driftm = (o[-1, 2] - o[0, 2]) / n, (b[-1, 2] - b[0, 2]) / n
    print("1M load max %.3f eV/A, mixed |d load| max %.2e; energy change per atom over 900 steps: "
          "oracle %.3e, mixed %.3e eV" % (scale, np.abs(b[:, 1] - o[:, 1]).max(), drift_o, driftm))
    assert abs(driftm - drift_o) < 1e-5                             # same energy history per atom
    assert np.abs(b[:, 2] - o[:, 2]).max() / n < 1e-5


def test_fullsize_batched_mixed_against_oracle(md, params):
    """The 256-replica batch (film sizes 6..24 x 6..24 x 6..12 cells, 100-500 K): after
    200 FP64 steps (thermal configurations), every replica's mixed-precision forces at that
    state against the FP64 oracle's forces at the same positions, at the flat 1e-5 bar."""
    oracle.set_threads(0)
    w = mi.make_workload("batched")
    b64 = md.MD(w.replicas, params, precision="fp64", skin=0.3)
    b64.step(200)
    bm = md.MD(w.replicas, params, precision="mixed", skin=SKIN)
    states = []
    for r in range(len(w.replicas)):
        x, v, z, st = b64.state(r)
        bm.set_state(r, x, v, z, st)
        states.append((x, z))
    b64.close()
    pot = oracle.Potential(params)
    worst, worst_r = 0.0, -1
    for r, rep in enumerate(w.replicas):
        x, z = states[r]
        ref = oracle.forces(pot, x, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c + np.array([0.0, 0.0, z]))
        err = float(rel_force_err(bm.forces(r), ref["F"]).max())
        if err > worst:
            worst, worst_r = err, r
        assert err <= 1e-5, (r, rep.temperature, err)
    bm.close()
    print("batched: worst per-atom mixed force error over 256 replicas %.2e (replica %d, %.0f K)"
          % (worst, worst_r, w.replicas[worst_r].temperature))


def test_fullsize_8m_mixed_forces_and_lists(md, params):
    """The 8,000,000-atom film (200 x 200 x 100 cells, the largest configuration) after
    100 mixed-precision steps: cells and a sample of neighbour sets bit-exact, and every
    atom's mixed-precision force within 1e-5 of the FP64 oracle."""
    oracle.set_threads(0)
    rep0 = mi.make_workload("8M").replicas[0]
    sim = md.MD([rep0], params, precision="mixed", skin=SKIN)
    sim.step(100)
    x, v, z, st = sim.state(0)
    sim.close()
    rep = dataclasses.replace(rep0, x_cr=x, v_cr=v, z_indenter0=z)
    sim = md.MD([rep], params, precision="mixed", skin=SKIN)   # lists built from x
    Fm = sim.forces(0)
    cut = params["rc"] + SKIN
    cell, cnt, nbr = sim.neighbors(0, 0)
    sim.close()
    assert np.array_equal(cell, oracle.cell_coords(rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, cut))
    off, idx = oracle.neighbors(rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, cut, method=1)
    rng = np.random.default_rng(8)
    for i in rng.choice(rep.n_cr, 3000, replace=False):
        assert set(nbr[i, :cnt[i]].tolist()) == set(idx[off[i]:off[i + 1]].tolist())
    del off, idx, nbr
    ref = oracle.forces(oracle.Potential(params), rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic,
                        rep.x_c + np.array([0.0, 0.0, rep.z_indenter0]))
    err = rel_force_err(Fm, ref["F"])
    print("8M mixed: max %.2e p99 %.2e" % (err.max(), np.quantile(err, 0.99)))
    assert err.max() <= 1e-5


def test_fullsize_step_io_against_oracle(md, params, thermal_1m):
    """md_step_io on the whole 1M film from a state the host changed (velocities scaled,
    so the drift is made afresh), page-locked arrays written in place, 10 steps, mixed
    precision: positions and velocities against the FP64 oracle started at that state
    (every atom), energies per atom; the call's result is the calls in turn's bit for bit."""
    torch = pytest.importorskip("torch")
    rep, _ = thermal_1m
    x, v, z = rep.x_cr, np.ascontiguousarray(0.9 * rep.v_cr), rep.z_indenter0
    hx = torch.empty(x.shape, dtype=torch.float64, pin_memory=True).numpy()
    hv = torch.empty(v.shape, dtype=torch.float64, pin_memory=True).numpy()
    a = md.MD([rep], params, precision="mixed", skin=SKIN)
    b = md.MD([rep], params, precision="mixed", skin=SKIN)
    hx[:] = x; hv[:] = v
    _, _, e = a.step_io(0, hx, hv, z, 0, 10, x_out=hx, v_out=hv)
    b.set_state(0, x, v, z, 0)
    b.step(10)
    xb, vb, _, _ = b.state(0)
    assert np.array_equal(hx, xb) and np.array_equal(hv, vb)
    oracle.set_threads(0)
    osim = oracle.Sim(oracle.Potential(params), dataclasses.replace(rep, v_cr=v), skin=SKIN)
    osim.step(10)
    o = osim.state()
    d = hx - o["x"]
    L = rep.box_hi - rep.box_lo
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-5
    assert np.abs(hv - o["v"]).max() < 1e-5
    assert abs(e["potential"] - o["potential"]) / rep.n_cr < 1e-5
    assert e["step"] == 10 and e["z_indenter"] == o["z_ind"]
    a.close(); b.close()
