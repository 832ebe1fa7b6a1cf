"""Pins of the oracle's time loop (Fig. 5; Tasks 1-5 of Sec. 2.1; Eqs. A11-A13).

Velocity Verlet is time reversible and, with conservative forces, conserves energy
and (for free atoms, no external field) momentum; the rigid indenter's travel is
v_ind * t; the neighbour-list schedule must not change the trajectory.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle


def small_film(T=300.0, R=5.0, v_ms=0.0, fixed=0, seed=21, n=6, nz=5):
    rep = mi.make_replica("t", n, n, nz, R, T, seed=seed, n_fixed_planes=fixed, v_ind_ms=v_ms, gap=1.0)
    return rep


def test_time_reversibility(params):
    pot = oracle.Potential(params)
    rep = small_film(T=600.0, fixed=2)
    sim = oracle.Sim(pot, rep, skin=0.3)
    sim.step(150)
    st = sim.state()
    back = oracle.Sim(pot, rep, skin=0.3, x=st["x"], v=-st["v"])
    back.step(150)
    x0 = np.mod(rep.x_cr, rep.box_hi - rep.box_lo) * (rep.periodic == 1) + rep.x_cr * (rep.periodic == 0)
    xb = back.state()["x"]
    L = rep.box_hi - rep.box_lo
    d = xb - x0
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-9
    assert sim.state()["rebuilds"] >= 0


def test_nve_energy_conservation(params):
    """Static indenter, no fixed atoms: |E(t) - E(0)| / N stays small with no trend."""
    pot = oracle.Potential(params)
    rep = small_film(T=300.0, v_ms=0.0, fixed=0, R=5.0)
    sim = oracle.Sim(pot, rep, skin=0.3)
    N = rep.n_cr
    E = [sim.state()["total"]]
    for _ in range(20):
        sim.step(50)
        E.append(sim.state()["total"])
    E = np.array(E)
    assert np.abs(E - E[0]).max() / N < 2e-5
    # no secular drift: first and second half means agree
    assert abs(E[1:11].mean() - E[11:].mean()) / N < 1e-5
    assert sim.state()["rebuilds"] > 0


def test_momentum_conservation(params):
    pot = oracle.Potential(params)
    rep = small_film(T=500.0, R=0.0, fixed=0)
    sim = oracle.Sim(pot, rep, skin=0.3)
    p0 = (rep.v_cr * rep.mass_cr).sum(0)
    sim.step(200)
    p1 = (sim.state()["v"] * rep.mass_cr).sum(0)
    assert np.abs(p0).max() < 1e-12
    assert np.abs(p1 - p0).max() < 1e-11


def test_indenter_travel_and_load_sign(params):
    pot = oracle.Potential(params)
    rep = small_film(T=10.0, v_ms=2000.0, fixed=2, R=5.0)
    sim = oracle.Sim(pot, rep, skin=0.3)
    sim.step(400)
    st = sim.state()
    assert st["z_ind"] == pytest.approx(400 * rep.v_indenter * rep.dt, rel=1e-12)
    # 0.8 A of travel from a 1 A gap brings the indenter into the repulsive range
    assert st["load"] > 0.0


def test_rebuild_schedule_does_not_change_trajectory(params):
    pot = oracle.Potential(params)
    rep = small_film(T=300.0, v_ms=20.0, fixed=2)
    a = oracle.Sim(pot, rep, skin=0.3)
    b = oracle.Sim(pot, rep, skin=0.3, rebuild_every=1)
    a.step(120); b.step(120)
    sa, sb = a.state(), b.state()
    assert sb["rebuilds"] == 119 and sa["rebuilds"] < 119   # initial build + one before every later step
    L = rep.box_hi - rep.box_lo
    d = sa["x"] - sb["x"]
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-9
    assert sa["total"] == pytest.approx(sb["total"], rel=1e-11)


def test_first_step_matches_hand_verlet(params):
    """One step against Eqs. A11-A13 written out with the oracle's own forces."""
    pot = oracle.Potential(params)
    rep = small_film(T=300.0, v_ms=20.0, fixed=2)
    f0 = oracle.forces(pot, rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c)["F"]
    acc = 9.6485332e-3 / rep.mass_cr
    mob = (rep.fixed == 0)[:, None]
    x1 = rep.x_cr + mob * (rep.v_cr * rep.dt + 0.5 * acc * f0 * rep.dt ** 2)
    xc1 = rep.x_c + np.array([0, 0, rep.v_indenter * rep.dt])
    f1 = oracle.forces(pot, x1, rep.box_lo, rep.box_hi, rep.periodic, xc1)["F"]
    v1 = rep.v_cr + mob * 0.5 * acc * (f0 + f1) * rep.dt
    sim = oracle.Sim(pot, rep, skin=0.3)
    sim.step(1)
    st = sim.state()
    np.testing.assert_allclose(st["x"], x1, rtol=0, atol=1e-13)
    np.testing.assert_allclose(st["v"], v1, rtol=0, atol=1e-15)
    np.testing.assert_allclose(st["F"], f1, rtol=0, atol=1e-10)
