"""md_step recovering from a neighbour-list overflow inside the call: a hot film (900 K)
under a fast indenter (200 m/s, 1.0 A gap), with list capacities equal to the longest
lists of the first build, Verlet skin 0.42 A (the list radius just below BCC's fifth shell,
so thermal motion and compression lengthen both lists at later rebuilds)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import tiny

pytestmark = pytest.mark.gpu

SKIN = 0.42


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1507_07068_gb300 import md as mdmod
    mdmod.lib()
    return mdmod


def compressed_film():
    rep = tiny(amp=0.05, gap=1.0, T=900.0)
    rep.v_indenter = -2e-3
    return rep


def first_build_capacity(md, params, rep, precision):
    probe = md.MD([rep], params, precision=precision, skin=SKIN, kmax=200, kcmax=400)
    info = probe.info()
    probe.close()
    return info["max_cnt"], info["max_cntc"]


def test_fp64_run_through_overflow_matches_oracle(md, params):
    rep = compressed_film()
    k0, kc0 = first_build_capacity(md, params, rep, "fp64")
    sim = md.MD([rep], params, precision="fp64", skin=SKIN, kmax=k0, kcmax=kc0)
    assert sim.info()["kmax"] == k0 and sim.info()["kcmax"] == kc0
    osim = oracle.Sim(oracle.Potential(params), rep, skin=SKIN)
    sim.step(100)
    osim.step(100)
    info = sim.info()
    assert info["kmax"] > k0 or info["kcmax"] > kc0    # a build inside the call overflowed
    x, v, z, step = sim.state(0)
    o = osim.state()
    assert step == 100 and z == o["z_ind"]
    d = x - o["x"]
    L = rep.box_hi - rep.box_lo
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-10
    np.testing.assert_allclose(v, o["v"], rtol=0, atol=1e-12)
    sim.close()


def test_mixed_run_through_overflow_equals_run_with_room(md, params):
    """The call goes back to its own start, where the lists are rebuilt from the same
    positions as before: the steps then repeat those of a run that never overflowed, bit
    for bit."""
    rep = compressed_film()
    k0, kc0 = first_build_capacity(md, params, rep, "mixed")
    tight = md.MD([rep], params, precision="mixed", skin=SKIN, kmax=k0, kcmax=kc0)
    roomy = md.MD([rep], params, precision="mixed", skin=SKIN, kmax=200, kcmax=400)
    tight.step(100)
    roomy.step(100)
    info = tight.info()
    assert info["kmax"] > k0 or info["kcmax"] > kc0
    xa, va, za, _ = tight.state(0)
    xb, vb, zb, _ = roomy.state(0)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and za == zb
    assert tight.energy(0)["total"] == roomy.energy(0)["total"]
    # one build more per restart (a redo can meet another list's overflow and restart again)
    assert tight.energy(0)["rebuilds"] >= roomy.energy(0)["rebuilds"] + 1
    assert all(v == 0 for v in tight.check_lists().values())   # the lists after the restart
    tight.close(); roomy.close()


def test_short_call_without_headroom_still_recovers(md, params):
    """A call of 5 steps (below the length that always keeps a copy) when the last build
    filled the capacity: the copy is kept because the lists are near capacity."""
    rep = compressed_film()
    k0, kc0 = first_build_capacity(md, params, rep, "fp64")
    sim = md.MD([rep], params, precision="fp64", skin=SKIN, kmax=k0, kcmax=kc0)
    osim = oracle.Sim(oracle.Potential(params), rep, skin=SKIN)
    for _ in range(20):
        sim.step(5)
        osim.step(5)
    d = sim.state(0)[0] - osim.state()["x"]
    L = rep.box_hi - rep.box_lo   # a list build wraps positions into the periodic box
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-9
    sim.close()
