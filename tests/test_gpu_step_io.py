"""md_step_io, the exchange of one replica's state with the host around n steps: the same
values, bit for bit, as md_set_state + md_step(n) + md_get_state + md_get_energy made in
turn, on every path the state takes (the same positions, positions moved within the skin,
a move that rebuilds the lists, a rebuild inside the steps, calls of 16 steps or more that
take md_step's recovery path, one replica of a batch, outputs written over the inputs);
and one exchange against the oracle started at that state."""
import dataclasses

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


def in_turn(sim, r, x, v, z, st, n):
    sim.set_state(r, x, v, z, st)
    sim.step(n)
    xo, vo, _, _ = sim.state(r)
    return xo, vo, sim.energy(r)


def same(a, b):
    xa, va, ea = a
    xb, vb, eb = b
    assert np.array_equal(xa, xb)
    assert np.array_equal(va, vb)
    for k in ("embed", "pair", "mterm", "morse", "kinetic", "load", "z_indenter", "step", "rebuilds"):
        assert ea[k] == eb[k], k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_io_equals_the_calls_in_turn(md, params, precision):
    rep = tiny(amp=0.05, gap=1.5, T=600.0)
    rep.v_indenter = -1e-3
    a = md.MD([rep], params, precision=precision, skin=0.3)
    b = md.MD([rep], params, precision=precision, skin=0.3)
    a.step(5); b.step(5)
    x, v, z, st = a.state(0)
    rng = np.random.default_rng(7)
    for it, (dx, n) in enumerate([(0.0, 1), (0.0, 1), (0.02, 1), (0.0, 3), (0.3, 1), (0.0, 9),
                                  (0.01, 2), (0.0, 20), (0.0, 1)]):
        x = np.ascontiguousarray(x + rng.uniform(-dx, dx, x.shape)) if dx else x
        v = np.ascontiguousarray(v * (1.0 + 0.01 * it))
        ra = in_turn(a, 0, x, v, z, st, n)
        rb = b.step_io(0, x, v, z, st, n)
        same(ra, rb)
        x, v = rb[0], rb[1]
        z, st = rb[2]["z_indenter"], rb[2]["step"]
    assert b.energy(0)["rebuilds"] >= 2      # the 0.3 A move, and builds inside the steps
    a.close(); b.close()


def test_step_io_one_replica_of_a_batch_in_place(md, params):
    reps = []
    for r, (nxy, nz, R, T) in enumerate([(6, 6, 5.0, 100.0), (9, 7, 6.0, 450.0), (7, 11, 5.5, 250.0)]):
        reps.append(jitter(mi.make_replica(f"b{r}", nxy, nxy, nz, R, T, seed=40 + r, gap=1.5), 0.08, r))
    a = md.MD(reps, params, precision="mixed", skin=0.6)
    b = md.MD(reps, params, precision="mixed", skin=0.6)
    a.step(4); b.step(4)
    x, v, z, st = a.state(1)
    for _ in range(6):
        ra = in_turn(a, 1, x, v, z, st, 2)
        xb, vb = x.copy(), v.copy()
        rb = b.step_io(1, xb, vb, z, st, 2, x_out=xb, v_out=vb)   # outputs over the inputs
        assert rb[0] is xb and rb[1] is vb
        same(ra, rb)
        x, v, z, st = rb[0], rb[1], rb[2]["z_indenter"], rb[2]["step"]
    for r in (0, 2):   # the replicas not exchanged stepped on alike
        sa, sb = a.state(r), b.state(r)
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
    a.close(); b.close()


def test_step_io_against_the_oracle(md, params):
    """FP64: an exchange of 10 steps from a state set by the host, against the oracle
    started at that state (positions within 1e-10 A, energies within 1e-9 relative)."""
    rep = tiny(amp=0.05, gap=2.0, T=300.0)
    sim = md.MD([rep], params, precision="fp64", skin=0.3)
    sim.step(15)
    x, v, z, st = sim.state(0)
    v2 = np.ascontiguousarray(0.9 * v)
    xo, vo, e = sim.step_io(0, x, v2, z, st, 10)
    o = oracle.Sim(oracle.Potential(params), dataclasses.replace(rep, x_cr=x, v_cr=v2, z_indenter0=z), skin=0.3)
    o.step(10)
    s = o.state()
    d = xo - s["x"]
    L = rep.box_hi - rep.box_lo
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-10
    assert np.abs(vo - s["v"]).max() < 1e-10
    assert abs(e["potential"] - s["potential"]) <= 1e-9 * abs(s["potential"])
    assert abs(e["kinetic"] - s["kinetic"]) <= 1e-9 * abs(s["kinetic"])
    assert e["step"] == st + 10
    sim.close()


def test_step_io_arguments(md, params):
    rep = tiny()
    sim = md.MD([rep], params, precision="mixed")
    x, v, z, st = sim.state(0)
    with pytest.raises(md.MDError):
        md.md_step_io(sim.h, 0, x, v, z, st, 0)
    with pytest.raises(ValueError):
        sim.step_io(0, x[:-1], v[:-1], z, st)
    with pytest.raises(md.MDError):
        md.md_step_io(sim.h, 5, x, v, z, st, 1)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_io_recovers_an_overflow_as_md_step(md, params, precision):
    """A hot film under a fast indenter with list capacities equal to the first build's
    longest lists (skin 0.42 A, just below BCC's fifth shell): builds inside the exchanges
    overflow; md_step_io goes back to the state it set and redoes the steps as md_step does,
    so every exchange equals the calls in turn bit for bit."""
    rep = tiny(amp=0.05, gap=1.0, T=900.0)
    rep.v_indenter = -2e-3
    probe = md.MD([rep], params, precision=precision, skin=0.42, kmax=200, kcmax=400)
    k0, kc0 = probe.info()["max_cnt"], probe.info()["max_cntc"]
    probe.close()
    a = md.MD([rep], params, precision=precision, skin=0.42, kmax=k0, kcmax=kc0)
    b = md.MD([rep], params, precision=precision, skin=0.42, kmax=k0, kcmax=kc0)
    x, v, z, st = a.state(0)
    for n in [1, 4, 1, 7, 1, 3] * 5:
        ra = in_turn(a, 0, x, v, z, st, n)
        rb = b.step_io(0, x, v, z, st, n)
        same(ra, rb)
        x, v, z, st = rb[0], rb[1], rb[2]["z_indenter"], rb[2]["step"]
    info = b.info()
    assert info["kmax"] > k0 or info["kcmax"] > kc0    # an exchange met an overflow
    assert (info["kmax"], info["kcmax"]) == (a.info()["kmax"], a.info()["kcmax"])
    a.close(); b.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_one_changed_velocity_remakes_the_drift(md, params, use_graph):
    """md_set_state with every position and all velocities but one atom's the held ones:
    the device's comparison must void the drift the last force pass made (it used the old
    velocity), so the run follows the oracle started at the new state; with the drift kept
    that atom would move 1.5e-3 A off in the first step alone."""
    rep = tiny(amp=0.05, gap=2.0, T=300.0)
    sim = md.MD([rep], params, precision="mixed", skin=0.3, use_graph=use_graph)
    sim.step(12)
    x, v, z, st = sim.state(0)
    v2 = v.copy()
    k = int(np.argmax(np.abs(v[:, 0])))
    v2[k] *= 1.5
    if use_graph:
        sim.step_io(0, x, v2, z, st, 1)
    else:   # direct launches: k_decide's DEC_AUTO read back by the host
        sim.set_state(0, x, v2, z, st)
        sim.step(1)
    sim.step(9)
    o = oracle.Sim(oracle.Potential(params), dataclasses.replace(rep, x_cr=x, v_cr=v2, z_indenter0=z), skin=0.3)
    o.step(10)
    d = sim.state(0)[0] - o.state()["x"]
    L = rep.box_hi - rep.box_lo
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-5
    sim.close()


def _pinned(a):
    """A page-locked copy of a (the array and the tensor that owns its memory)."""
    torch = pytest.importorskip("torch")
    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
    p = t.numpy()
    p[:] = a
    return p, t


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_page_locked_arrays_move_the_same_bits(md, params, precision):
    """Page-locked host arrays (copied asynchronously by the copy engines; md_set_state
    waits until its velocities are read) and pageable ones give the same state, forces and
    energies bit for bit, through state changes that keep and rebuild the lists, on a
    replica that is not the first of its batch."""
    reps = []
    for r, (nxy, nz, R, T) in enumerate([(6, 6, 5.0, 100.0), (9, 7, 6.0, 600.0)]):
        reps.append(jitter(mi.make_replica(f"p{r}", nxy, nxy, nz, R, T, seed=70 + r, gap=1.5), 0.05, r))
    a = md.MD(reps, params, precision=precision, skin=0.3)
    b = md.MD(reps, params, precision=precision, skin=0.3)
    a.step(3); b.step(3)
    x, v, z, st = a.state(1)
    rng = np.random.default_rng(5)
    keep = []
    for it, (dx, n) in enumerate([(0.0, 1), (0.02, 1), (0.0, 4), (0.3, 1), (0.0, 20), (0.0, 1)]):
        x = np.ascontiguousarray(x + rng.uniform(-dx, dx, x.shape)) if dx else x
        v = np.ascontiguousarray(v * (1.0 + 0.01 * it))
        ra = a.step_io(1, x, v, z, st, n)                       # pageable: staged copies
        xp, t1 = _pinned(x); vp, t2 = _pinned(v)
        xo, t3 = _pinned(np.zeros_like(x)); vo, t4 = _pinned(np.zeros_like(v))
        keep += [t1, t2, t3, t4]
        rb = b.step_io(1, xp, vp, z, st, n, x_out=xo, v_out=vo)  # page-locked: in place
        same(ra, rb)
        x, v, z, st = ra[0], ra[1], ra[2]["z_indenter"], ra[2]["step"]
    assert b.energy(1)["rebuilds"] >= 2
    # the separate calls with page-locked arrays
    xp, t1 = _pinned(x); vp, t2 = _pinned(v)
    a.set_state(1, x, v, z, st); b.set_state(1, xp, vp, z, st)
    a.step(3); b.step(3)
    xo, t3 = _pinned(np.zeros_like(x)); vo, t4 = _pinned(np.zeros_like(v)); fo, t5 = _pinned(np.zeros_like(x))
    md.md_get_state(b.h, 1, len(x), xo, vo)
    md.md_get_forces(b.h, 1, len(x), fo)
    xa, va, _, _ = a.state(1)
    assert np.array_equal(xa, xo) and np.array_equal(va, vo) and np.array_equal(a.forces(1), fo)
    a.close(); b.close()
