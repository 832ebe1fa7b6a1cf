"""The device check of the neighbour lists (md_check_lists, and the debug mode that runs it
after every list build): lists as built pass every check, in both precisions, for ragged
replicas and after steps with rebuilds; checked against a smaller radius it counts exactly
the listed pairs between that radius and the list radius, which the oracle counts
independently."""
import numpy as np
import pytest

import md_inputs as mi
import oracle
from gpu_helpers import jitter, tiny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1507_07068_gb300 import md as mdmod
    mdmod.lib()
    return mdmod


def ragged():
    reps = []
    for r, (nxy, nz, R, T) in enumerate([(6, 6, 5.0, 100.0), (9, 7, 6.0, 450.0), (7, 11, 5.5, 250.0)]):
        reps.append(jitter(mi.make_replica(f"c{r}", nxy, nxy, nz, R, T, seed=300 + r, gap=1.2), 0.08, r))
    return reps


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lists_as_built_pass_every_check(md, params, precision):
    sim = md.MD(ragged(), params, precision=precision, skin=0.4)
    assert all(v == 0 for v in sim.check_lists().values())
    sim.step(120)
    assert sim.energy(0)["rebuilds"] > 0
    assert all(v == 0 for v in sim.check_lists().values())
    sim.close()


def test_smaller_radius_counts_the_skin_pairs(md, params):
    rep = tiny(amp=0.1, gap=1.5)
    skin = 0.3
    sim = md.MD([rep], params, precision="fp64", skin=skin)
    c = sim.check_lists(radius=params["rc"])
    x = rep.x_cr
    off1, _ = oracle.neighbors(x, rep.box_lo, rep.box_hi, rep.periodic, params["rc"] + skin)
    off0, _ = oracle.neighbors(x, rep.box_lo, rep.box_hi, rep.periodic, params["rc"])
    assert c["beyond_radius"] == int(off1[-1] - off0[-1]) > 0
    assert c["missing"] == 0
    assert all(v == 0 for k, v in c.items() if k not in ("beyond_radius",))
    # the check's violation is reported by the call, not left to the next step
    sim.step(5)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_debug_mode_checks_every_build(md, params, precision):
    rep = tiny(amp=0.05, gap=1.0, T=900.0)
    a = md.MD([rep], params, precision=precision, skin=0.3, debug_checks=True)
    b = md.MD([rep], params, precision=precision, skin=0.3)
    a.step(100); b.step(100)
    assert a.energy(0)["rebuilds"] == b.energy(0)["rebuilds"] > 2
    xa, xb = a.state(0)[0], b.state(0)[0]
    assert np.array_equal(xa, xb)   # the checks read only
    a.close(); b.close()


@pytest.mark.parametrize("tpa", [2, 4, 8])
def test_inner_list_capacity_with_lane_groups(md, params, tpa):
    """With several threads per atom the inner list's rows are lane-interleaved and padded to
    the longest lane's count times the threads per atom, which can pass kmax by up to
    tpa - 1 rows when the Verlet lists are nearly full (the list check found it): with kmax
    equal to the longest Verlet list the lists pass the check and the run is bit for bit
    the run with room."""
    rep = tiny(amp=0.05, gap=1.0, T=900.0)
    rep.v_indenter = -2e-3
    roomy = md.MD([rep], params, precision="mixed", skin=0.42, kmax=200, kcmax=400, tpa=tpa)
    k0 = roomy.info()["max_cnt"]
    tight = md.MD([rep], params, precision="mixed", skin=0.42, kmax=k0, kcmax=400, tpa=tpa)
    assert all(v == 0 for v in tight.check_lists().values())
    assert np.array_equal(tight.forces(0), roomy.forces(0))
    tight.step(50)
    roomy.step(50)
    assert np.array_equal(tight.state(0)[0], roomy.state(0)[0])
    assert all(v == 0 for v in tight.check_lists().values())
    tight.close(); roomy.close()


def test_batched_lists_pass_the_check(md, params):
    """The 256-replica batch (uneven films, 128-slot tiles) after steps with rebuilds."""
    w = mi.make_workload("batched")
    b = md.MD(w.replicas, params, precision="mixed", skin=1.1)
    b.step(150)
    assert b.energy(0)["rebuilds"] > 0
    assert all(v == 0 for v in b.check_lists().values())
    b.close()
