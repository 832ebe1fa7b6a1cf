"""The paper's timing workload (Table 2, Sec. 4): BCC cubes with free faces and the
potential fitted with the long cut-off r* = 8.262 A (Sec. 2.6), ~180 neighbours within it.
CUDA path against the oracle, with a thin Verlet skin and with the paper's own list scheme
(outer list of radius 1.7 r*, i.e. skin 0.7 r*, rebuilt when an atom moved half the skin;
inner list of radius r* rebuilt from it every step; analytic forms, Sec. 2.4)."""
import numpy as np
import pytest

import md_inputs as mi
import oracle
from gpu_helpers import jitter, rel_force_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1507_07068_gb300 import md as mdmod
    mdmod.lib()
    return mdmod


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_long_cutoff_forces(md, params_rstar, precision, tol):
    rep = jitter(mi.paper_cube(10), 0.05, 3)
    sim = md.MD([rep], params_rstar, precision=precision, skin=1.0)
    o = oracle.forces(oracle.Potential(params_rstar), rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic)
    assert rel_force_err(sim.forces(0), o["F"]).max() <= tol
    e = sim.energy(0)
    rt = 1e-12 if precision == "fp64" else 1e-5
    for k in ("embed", "pair", "mterm"):
        assert e[k] == pytest.approx(o[k], rel=rt, abs=1e-9 if precision == "fp64" else 1e-4)
    _, cnt, _ = sim.neighbors(0, 0, kmax=1)
    assert cnt.max() > 200   # the list reaches r* + skin
    sim.close()


def test_long_cutoff_trajectory(md, params_rstar):
    rep = jitter(mi.paper_cube(10), 0.05, 4)
    sim = md.MD([rep], params_rstar, precision="fp64", skin=1.0)
    o = oracle.Sim(oracle.Potential(params_rstar), rep, skin=1.0)
    sim.step(40)
    o.step(40)
    x, _, _, _ = sim.state(0)
    assert np.abs(x - o.state()["x"]).max() < 1e-10
    assert sim.energy(0)["rebuilds"] == o.state()["rebuilds"]
    sim.close()


def paper_lists(params_rstar):
    """md.MD options of the paper's two-tier list (Sec. 2.6) with its analytic forms."""
    return dict(skin=0.7 * params_rstar["rc"], inner_skin=-1.0, tabulated=0)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_paper_list_scheme_forces(md, params_rstar, precision, tol):
    rep = jitter(mi.paper_cube(10), 0.05, 5)
    sim = md.MD([rep], params_rstar, precision=precision, **paper_lists(params_rstar))
    o = oracle.forces(oracle.Potential(params_rstar, tabulated=0), rep.x_cr, rep.box_lo, rep.box_hi,
                      rep.periodic)
    assert rel_force_err(sim.forces(0), o["F"]).max() <= tol
    e = sim.energy(0)
    rt = 1e-12 if precision == "fp64" else 1e-5
    for k in ("embed", "pair", "mterm"):
        assert e[k] == pytest.approx(o[k], rel=rt, abs=1e-9 if precision == "fp64" else 1e-4)
    _, cnt, _ = sim.neighbors(0, 0, kmax=1)
    assert cnt.max() > 600   # the outer list reaches 1.7 r* = 14.0 A
    sim.close()


def test_paper_list_scheme_trajectory(md, params_rstar):
    """40 FP64 steps with the paper's list scheme against the oracle's run with the same
    outer list (skin 0.7 r*) and analytic forms."""
    rep = jitter(mi.paper_cube(10), 0.05, 6)
    kw = paper_lists(params_rstar)
    sim = md.MD([rep], params_rstar, precision="fp64", **kw)
    o = oracle.Sim(oracle.Potential(params_rstar, tabulated=0), rep, skin=kw["skin"])
    sim.step(40)
    o.step(40)
    x, _, _, _ = sim.state(0)
    assert np.abs(x - o.state()["x"]).max() < 1e-10
    assert sim.energy(0)["rebuilds"] == o.state()["rebuilds"]
    sim.close()
