"""Parity at the full size of the 1,000,000-atom film in the launch configuration the
benchmark times (mixed precision, default launch shape, cell order and lists as built by
the library), against the FP64 oracle over every atom."""
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
    err = rel_force_err(Fm, ref["F"])
    print("1M mixed: max %.2e p99 %.2e median %.2e F_rms %.3f" % (err.max(), np.quantile(err, 0.99),
                                                                   np.median(err), np.sqrt((ref["F"] ** 2).sum(1).mean())))
    assert err.max() <= 1e-5
    e = sim.energy(0)
    assert e["potential"] == pytest.approx(ref["potential"], rel=1e-6)
    sim.close()
