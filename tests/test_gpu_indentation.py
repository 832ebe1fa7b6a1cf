"""The indentation run through the C ABI: indenter velocity changes between steps (the
loading and unloading legs, Sec. 2.5) against the oracle, and a short full run."""
import numpy as np
import pytest

import oracle
from gpu_helpers import tiny

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1507_07068_gb300 import md as mdmod
    mdmod.lib()
    return mdmod


def test_velocity_switches_follow_the_oracle(md, params):
    """Load, hold and unload legs with the velocity set between steps: the indenter path
    is bit for bit the oracle's (the same z += v dt), the film and its load follow the
    oracle's FP64 trajectory."""
    rep = tiny(amp=0.02, gap=0.5)
    sim = md.MD([rep], params, precision="fp64", skin=0.3)
    o = oracle.Sim(oracle.Potential(params), rep, skin=0.3)
    loads = []
    for v, n in ((-1e-2, 60), (0.0, 15), (1e-2, 40), (-5e-3, 10)):
        sim.set_indenter_velocity(0, v)
        o.set_indenter_velocity(v)
        sim.step(n)
        o.step(n)
        os_ = o.state()
        x, _, z, _ = sim.state(0)
        assert z == os_["z_ind"]
        d = x - os_["x"]
        L = rep.box_hi - rep.box_lo
        d -= np.round(d / L) * L * (rep.periodic == 1)
        assert np.abs(d).max() < 1e-9
        e = sim.energy(0)
        assert e["load"] == pytest.approx(os_["load"], rel=1e-8, abs=1e-10)
        loads.append(e["load"])
    assert max(abs(l) for l in loads) > 1e-3   # the indenter reached the film
    sim.close()


def test_short_indentation_run_and_its_analysis(md, params):
    from paper_1507_07068_gb300 import indentation as ind
    rep = tiny(amp=0.02, gap=0.8, n=12, nz=8, R=6.0)
    sim = md.MD([rep], params, precision="mixed", skin=0.6)
    out = ind.run(sim, 0, relax_steps=40, depth_max=1.2, speed=2e-3, sample_every=5)
    sim.close()
    iu = out["i_unload"]
    assert out["depth"][0] == pytest.approx(-0.8, abs=0.05)
    assert out["depth"][iu - 1] >= 1.2 and out["depth"][-1] <= out["depth"][0] + 0.02
    load = out["load"]
    assert np.all(np.isfinite(load)) and np.abs(load).max() > 0.1   # the indenter met the film
    # past the snap-in (the Morse well pulls the indenter down: negative load) the film's
    # repulsion grows with depth
    assert load[iu - 1] > load[:iu].min() + 0.1
    assert np.all(np.diff(out["step"]) > 0)
    assert set(np.unique(out["phase"])) == {0, 1, 2}
