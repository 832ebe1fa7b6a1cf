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


@pytest.fixture(scope="module")
def params_indent():
    import os
    return oracle.load_params(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                           "paper_1507_07068_gb300", "cr_c_params_indent.json"))


def test_paper_system_leg_in_contact_follows_the_oracle(md, params_indent):
    """The paper's 11k system (19 x 19 x 14 cells, free faces, R = 9.78 A) with the Cr-C
    reading of the indentation run, the indenter started 0.5 A below the top plane: a hold
    and a loading leg at 10 m/s in FP64 against the oracle's run."""
    import md_inputs as mi
    rep = mi.paper_indentation_film()
    rep.z_indenter0 = -3.5
    sim = md.MD([rep], params_indent, precision="fp64", skin=0.3, kcmax=512)
    o = oracle.Sim(oracle.Potential(params_indent), rep, skin=0.3)
    for v, n in ((0.0, 30), (-1e-4, 70)):
        sim.set_indenter_velocity(0, v)
        o.set_indenter_velocity(v)
        sim.step(n)
        o.step(n)
        os_ = o.state()
        x, _, z, _ = sim.state(0)
        assert z == os_["z_ind"]
        assert np.abs(x - os_["x"]).max() < 1e-9
        e = sim.energy(0)
        assert e["load"] == pytest.approx(os_["load"], rel=1e-8, abs=1e-10)
    assert e["load"] > 1.0   # a repulsive contact
    sim.close()


def test_paper_protocol_gives_modulus_and_hardness(md, params_indent):
    """The paper's protocol on its 11k system (Sec. 4.3: 10 000 steps of relaxation, loading
    at 10 m/s to a depth of 3.08 A, unloading) in mixed precision, and the analysis: a
    repulsive loading branch, a Hertz modulus, the Oliver-Pharr reduced modulus and
    hardness.  Their values are this parameter reading's, not the paper's."""
    import md_inputs as mi
    from paper_1507_07068_gb300 import indentation as ind
    rep = mi.paper_indentation_film()
    sim = md.MD([rep], params_indent, precision="mixed", skin=1.1, kcmax=768)
    out = ind.run(sim, 0, relax_steps=10000, depth_max=3.08, speed=1e-4, sample_every=100)
    sim.close()
    iu = out["i_unload"]
    P = out["load"]
    assert P.max() > 5.0 and P[:iu].min() > -0.1 * P.max()
    E_h = ind.hertz_modulus(out["depth"][:iu], P[:iu], 9.78) * ind.EV_A3_IN_GPA
    op = ind.oliver_pharr(out["depth"][iu - 1:], P[iu - 1:], 9.78)
    E_r, H = op["E_r"] * ind.EV_A3_IN_GPA, op["H"] * ind.EV_A3_IN_GPA
    print("11k indentation: P_max %.2f eV/A, Hertz E* %.1f GPa, Oliver-Pharr E_r %.1f GPa, H %.1f GPa"
          % (P.max(), E_h, E_r, H))
    assert 10.0 < E_h < 1000.0 and 10.0 < E_r < 1000.0 and 1.0 < H < 200.0
