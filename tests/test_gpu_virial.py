"""Per-atom virial through the C ABI against the oracle (the potential part of per-atom
stress times volume, Sec. 2.1)."""
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


def rel_tensor_err(W, Wref):
    """per-atom |dW_i| / max(|W_i|, W_rms) over the 6 components"""
    nrm = np.sqrt((Wref ** 2).sum(1))
    rms = np.sqrt((nrm ** 2).mean())
    return np.sqrt(((W - Wref) ** 2).sum(1)) / np.maximum(nrm, rms)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_virial_matches_oracle_with_indenter(md, params, precision, tol):
    rep = tiny(amp=0.06, gap=0.3)        # the indenter within the Morse range of the surface
    sim = md.MD([rep], params, precision=precision)
    W = sim.virial(0)
    _, _, z, _ = sim.state(0)
    o = oracle.virial(oracle.Potential(params), rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic,
                      rep.x_c + np.array([0.0, 0.0, z]))
    assert np.abs(o["morse"]) > 1e-3          # Cr-C pairs contribute
    assert rel_tensor_err(W, o["W"]).max() <= tol
    assert np.isfinite(sim.energy(0)["total"])
    sim.close()


def test_virial_after_steps_follows_the_oracle(md, params):
    rep = tiny(amp=0.05, gap=0.5)
    sim = md.MD([rep], params, precision="fp64")
    o = oracle.Sim(oracle.Potential(params), rep, skin=0.3)
    sim.step(30)
    o.step(30)
    W = sim.virial(0)
    Wo = o.virial()
    assert rel_tensor_err(W, Wo).max() < 1e-8       # trajectories agree to ~1e-10 A
    # the call re-evaluates the forces to the same values and leaves the run unchanged
    F = sim.forces(0)
    sim.step(5); o.step(5)
    assert np.abs(sim.state(0)[0] - o.state()["x"]).max() < 1e-9
    assert np.isfinite(F).all()
    sim.close()
