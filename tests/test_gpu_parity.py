"""CUDA path (through the C ABI) against the FP64 CPU oracle, element by element.

Bars: cell coordinates and neighbour sets built in FP64 bit-exact (pairs within 1e-12 A of
the list cut-off excluded); per-atom forces within 1e-12 (FP64 mode) and 1e-5 (mixed mode)
of the metric ||dF_i|| / max(||F_i||, F_rms); energies likewise.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle
from gpu_helpers import compare_sets, jitter, min_image_r, rel_force_err, tiny

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12   # per-atom force bar, FP64 mode
MIXED_TOL = 1e-5   # per-atom force bar, mixed mode


@pytest.fixture(scope="module")
def md():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1507_07068_gb300 import md as mdmod
    mdmod.lib()
    return mdmod


def oracle_eval(params, rep, z_ind=0.0, **ov):
    pot = oracle.Potential(params, **ov)
    xc = rep.x_c + np.array([0.0, 0.0, z_ind]) if rep.n_c else None
    return oracle.forces(pot, rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, xc)


def energy_close(e, o, rtol, atol):
    for k in ("embed", "pair", "mterm", "morse", "load"):
        assert e[k] == pytest.approx(o[k], rel=rtol, abs=atol), k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cells_and_lists_bit_exact(md, params, precision):
    rep = tiny(amp=0.12, gap=1.0)
    skin = 0.3
    sim = md.MD([rep], params, precision=precision, skin=skin)
    cut = params["rc"] + skin
    cell, cnt, nbr = sim.neighbors(0, 0)
    ocell = oracle.cell_coords(rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, cut)
    assert np.array_equal(cell, ocell)
    off, idx = oracle.neighbors(rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, cut, method=0)
    near = lambda i, j: abs(min_image_r(rep.x_cr, i, j, rep.box_lo, rep.box_hi, rep.periodic) - cut) < 1e-12
    assert compare_sets(cnt, nbr, off, idx, near) == []
    assert cnt.sum() == off[-1]
    # Cr-C list
    cutc = params["rc_m"] + skin
    _, cntc, nbrc = sim.neighbors(0, 1)
    offc, idxc = oracle.cneighbors(rep.x_cr, rep.x_c, rep.box_lo, rep.box_hi, rep.periodic, cutc)
    assert offc[-1] > 0
    assert compare_sets(cntc, nbrc, offc, idxc, lambda i, j: False) == []
    sim.close()


def test_cells_on_cell_faces_bit_exact(md, params):
    """Coordinates exactly on cell faces and one ulp either side, and periodic coordinates
    shifted by whole periods (the cases where the quotient floors of the binning are decided
    by rounding): cell coordinates and neighbour sets equal the oracle's."""
    rep = tiny(amp=0.12, gap=1.0)
    skin = 0.3
    cut = params["rc"] + skin
    lo, hi, per = rep.box_lo, rep.box_hi, rep.periodic
    L = hi - lo
    n = np.maximum(1, np.floor(L / cut)).astype(int)
    w = L / n
    x = rep.x_cr.copy()
    rng = np.random.default_rng(7)
    moved = 0
    for i in range(len(x)):
        for k in range(3):
            q = (x[i, k] - lo[k]) / w[k]
            kb = np.round(q)
            if abs(q - kb) * w[k] < 0.2 and 0 < kb < n[k]:
                b = lo[k] + kb * w[k]
                x[i, k] = (b, np.nextafter(b, np.inf), np.nextafter(b, -np.inf))[rng.integers(3)]
                moved += 1
            elif per[k] and rng.random() < 0.1:
                x[i, k] += L[k] * rng.choice([-2.0, -1.0, 1.0, 3.0])
    assert moved > 50
    rep.x_cr = x
    sim = md.MD([rep], params, precision="mixed", skin=skin)
    cell, cnt, nbr = sim.neighbors(0, 0)
    assert np.array_equal(cell, oracle.cell_coords(x, lo, hi, per, cut))
    # the oracle's cell-list build wraps the positions first (its brute-force form takes a
    # single minimum-image shift, so it wants positions within one period)
    off, idx = oracle.neighbors(x, lo, hi, per, cut, method=1)
    xw = np.where(per == 1, x - np.floor((x - lo) / L) * L, x)
    near = lambda i, j: abs(min_image_r(xw, i, j, lo, hi, per) - cut) < 1e-12
    assert compare_sets(cnt, nbr, off, idx, near) == []
    sim.close()


def test_cr_c_list_periodic_z_tall_indenter(md, params):
    """Periodic z with an indenter taller than half the period minus the Morse reach: the
    Cr-C candidates are found through either z image (the list equals the oracle's)."""
    rep = mi.make_replica("pz", 8, 8, 6, 10.0, 300.0, seed=3, gap=1.0, periodic_z=True)
    rep = jitter(rep, 0.1, 3)
    skin = 0.3
    cutc = params["rc_m"] + skin
    L = rep.box_hi - rep.box_lo
    assert 0.5 * (rep.x_c[:, 2].max() - rep.x_c[:, 2].min()) + cutc > 0.5 * L[2]
    sim = md.MD([rep], params, precision="mixed", skin=skin)
    _, cntc, nbrc = sim.neighbors(0, 1)
    offc, idxc = oracle.cneighbors(rep.x_cr, rep.x_c, rep.box_lo, rep.box_hi, rep.periodic, cutc)
    assert offc[-1] > 0
    assert compare_sets(cntc, nbrc, offc, idxc, lambda i, j: False) == []
    sim.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_rebuild_after_steps_bit_exact(md, params, precision):
    """Cells and lists of a rebuild after time steps (the mixed path bins from the FP32
    cell-relative positions it keeps current; atoms cross cells and periodic faces) equal
    the oracle's on the positions of that moment."""
    rep = tiny(amp=0.12, gap=2.0, T=900.0)
    skin = 0.3
    sim = md.MD([rep], params, precision=precision, skin=skin)
    cut = params["rc"] + skin
    lo, hi, per = rep.box_lo, rep.box_hi, rep.periodic
    for _ in range(3):
        sim.step(40)
        sim.build_neighbors()
        x = sim.state(0)[0]
        cell, cnt, nbr = sim.neighbors(0, 0)
        assert np.array_equal(cell, oracle.cell_coords(x, lo, hi, per, cut))
        off, idx = oracle.neighbors(x, lo, hi, per, cut, method=1)
        near = lambda i, j: abs(min_image_r(x, i, j, lo, hi, per) - cut) < 1e-12
        assert compare_sets(cnt, nbr, off, idx, near) == []
    assert sim.energy(0)["rebuilds"] >= 3
    sim.close()


@pytest.mark.parametrize("tab,shifted", [(1, 1), (0, 1), (1, 0), (0, 0)])
def test_forces_fp64(md, params, tab, shifted):
    rep = tiny(amp=0.12, gap=1.0)
    sim = md.MD([rep], params, precision="fp64", tabulated=tab, shifted=shifted)
    F = sim.forces(0)
    e = sim.energy(0)
    o = oracle_eval(params, rep, tabulated=tab, shifted=shifted)
    err = rel_force_err(F, o["F"])
    assert err.max() <= FP64_TOL, err.max()
    energy_close(e, o, 1e-12, 1e-10)
    sim.close()


@pytest.mark.parametrize("tab", [1, 0])
def test_forces_mixed(md, params, tab):
    rep = tiny(amp=0.12, gap=1.0)
    sim = md.MD([rep], params, precision="mixed", tabulated=tab)
    F = sim.forces(0)
    e = sim.energy(0)
    o = oracle_eval(params, rep, tabulated=tab)
    err = rel_force_err(F, o["F"])
    assert err.max() <= MIXED_TOL, err.max()
    energy_close(e, o, 1e-5, 1e-4)
    sim.close()


@pytest.mark.parametrize("beta", [5.5, 8.0])
def test_forces_mixed_other_exponents(md, params, beta):
    """beta other than 6: the pair loops' generic form of f (exp2/log2 for a non-even beta,
    the runtime integer power for an even one) against the oracle."""
    rep = tiny(amp=0.12, gap=1.0)
    sim = md.MD([rep], params, precision="mixed", beta=beta, tabulated=0)
    o = oracle_eval(params, rep, beta=beta, tabulated=0)
    assert rel_force_err(sim.forces(0), o["F"]).max() <= MIXED_TOL
    energy_close(sim.energy(0), o, 1e-5, 1e-4)
    sim.close()


@pytest.mark.parametrize("tpa,block", [(1, 128), (2, 256), (4, 128), (8, 256), (8, 64)])
def test_launch_shapes_agree(md, params, tpa, block):
    rep = tiny(amp=0.1)
    o = oracle_eval(params, rep)
    for prec, tol in (("fp64", FP64_TOL), ("mixed", MIXED_TOL)):
        sim = md.MD([rep], params, precision=prec, tpa=tpa, block=block)
        assert rel_force_err(sim.forces(0), o["F"]).max() <= tol
        sim.close()


@pytest.mark.parametrize("gap", [1.0, 2.5])
def test_trajectory_fp64_fixed_rebuilds(md, params, gap):
    """50 FP64 steps with rebuilds every 7 steps against the oracle's run.  gap 1.0 A puts
    the indenter's lowest atoms 1.8 A from the film (inside the Cr-C repulsive wall, 857
    Cr-C pairs within the Morse cut-off); gap 2.5 A near the Morse minimum (321 pairs)."""
    rep = tiny(amp=0.05, gap=gap, T=400.0)
    sim = md.MD([rep], params, precision="fp64", rebuild_every=7)
    osim = oracle.Sim(oracle.Potential(params), rep, skin=0.3, rebuild_every=7)
    for chunk in (1, 9, 40):
        sim.step(chunk)
        osim.step(chunk)
        x, v, z, step = sim.state(0)
        o = osim.state()
        assert step == o["step"]
        assert z == o["z_ind"]
        np.testing.assert_allclose(x, o["x"], rtol=0, atol=1e-10)
        np.testing.assert_allclose(v, o["v"], rtol=0, atol=1e-12)
        assert rel_force_err(sim.forces(0), o["F"]).max() <= 1e-9
        e = sim.energy(0)
        assert e["total"] == pytest.approx(o["total"], abs=1e-9 * rep.n_cr)
        assert e["kinetic"] == pytest.approx(o["kinetic"], rel=1e-11)
        assert e["load"] == pytest.approx(o["load"], rel=1e-9, abs=1e-10)
        assert e["rebuilds"] == o["rebuilds"]


def test_trajectory_skin_mode_matches_oracle_schedule(md, params):
    rep = tiny(amp=0.02, gap=2.0, T=600.0)
    sim = md.MD([rep], params, precision="fp64", rebuild_every=0)
    osim = oracle.Sim(oracle.Potential(params), rep, skin=0.3, rebuild_every=0)
    sim.step(250)
    osim.step(250)
    e = sim.energy(0)
    o = osim.state()
    assert o["rebuilds"] > 1
    assert e["rebuilds"] == o["rebuilds"]
    x, v, z, _ = sim.state(0)
    np.testing.assert_allclose(x, o["x"], rtol=0, atol=1e-9)


def test_trajectory_mixed_tracks_oracle(md, params):
    rep = tiny(amp=0.05, gap=1.0, T=300.0)
    sim = md.MD([rep], params, precision="mixed", rebuild_every=0)
    osim = oracle.Sim(oracle.Potential(params), rep, skin=0.3)
    sim.step(100)
    osim.step(100)
    x, v, z, _ = sim.state(0)
    o = osim.state()
    np.testing.assert_allclose(x, o["x"], rtol=0, atol=1e-5)
    assert rel_force_err(sim.forces(0), o["F"]).max() < 1e-3
    assert sim.energy(0)["total"] == pytest.approx(o["total"], abs=1e-5 * rep.n_cr)


@pytest.mark.parametrize("inner_skin", [0.1, 0.02])
def test_inner_list_schedule_bitwise_equal(md, params, inner_skin):
    """The inner list rebuilt every step with radius rc (the paper's schedule) and the
    inner list with a skin, rebuilt only when an atom has moved half of it: the density and
    force loops take the same pairs in the same order, so trajectories agree bit for bit."""
    rep = tiny(amp=0.05, gap=2.0, T=600.0)
    a = md.MD([rep], params, precision="mixed", inner_skin=-1.0)
    b = md.MD([rep], params, precision="mixed", inner_skin=inner_skin)
    for _ in range(4):
        a.step(50); b.step(50)
        xa, va, za, _ = a.state(0)
        xb, vb, zb, _ = b.state(0)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
        assert np.array_equal(a.forces(0), b.forces(0))
    assert a.energy(0)["total"] == b.energy(0)["total"]
    a.close(); b.close()


def test_graph_and_direct_launch_bitwise_equal(md, params):
    rep = tiny(amp=0.05)
    a = md.MD([rep], params, precision="mixed", use_graph=True)
    b = md.MD([rep], params, precision="mixed", use_graph=False)
    a.step(37); b.step(37)
    xa, va, _, _ = a.state(0)
    xb, vb, _, _ = b.state(0)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert a.energy(0) == b.energy(0)
    t = b.step_profiled(5)
    assert t["steps"] == 5 and t["force"] > 0 and t["density"] > 0 and t["morse"] > 0
    # the profiled steps (direct launches, the Morse kernel in its own timed phase) take
    # the same trajectory
    a.step(5)
    xa, va, _, _ = a.state(0)
    xb, vb, _, _ = b.state(0)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


def test_interleaved_calls_keep_the_trajectory(md, params):
    """The mixed-precision force kernel makes the next step's drift; forces recomputed or
    lists rebuilt between steps make it again, and a state set from the host keeps it when
    positions, velocities and indenter are bit for bit the ones held (even with another
    step count; the first step then reads the device's drift flag), else the next step
    drifts afresh.  A run interrupted by such calls that do not change the state follows
    the uninterrupted run bit for bit, with graphs (unrolled and single steps) and with
    direct launches alike."""
    rep = tiny(amp=0.05, gap=2.0, T=600.0)
    ref = md.MD([rep], params, precision="mixed")
    ref.step(3 + 1 + 2 + 9 + 4)
    runs = [md.MD([rep], params, precision="mixed", use_graph=g) for g in (True, False)]
    for sim in runs:
        sim.step(3)
        x, v, z, st = sim.state(0)
        sim.set_state(0, x, v, z, st)          # same state: lists kept
        sim.step(1)
        sim.compute_forces()
        sim.step(2)
        sim.step(9)                            # one unrolled graph and one single step
        x, v, z, st = sim.state(0)
        sim.set_state(0, x, v, z, st + 1)      # another step count (the buffers keep their parity)
        sim.step(4)
        assert sim.energy(0)["step"] == 3 + 1 + 2 + 9 + 4 + 1
    xr, vr, zr, _ = ref.state(0)
    for sim in runs:
        x, v, z, _ = sim.state(0)
        assert np.array_equal(x, xr) and np.array_equal(v, vr) and z == zr
        assert np.array_equal(sim.forces(0), ref.forces(0))
    # an explicit list build reorders the pair sums: graph and direct runs still agree
    for sim in runs:
        sim.build_neighbors()
        sim.step(6)
    ref.step(6)
    xa, va, _, _ = runs[0].state(0)
    xb, vb, _, _ = runs[1].state(0)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    d = xa - ref.state(0)[0]   # the explicit build wrapped positions into the periodic box
    L = rep.box_hi - rep.box_lo
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-3
    for sim in runs + [ref]:
        sim.close()


def _uneven_replicas(n=5, gap=2.0):
    reps = []
    for r, (nxy, nz, R, T) in enumerate([(6, 6, 5.0, 100.0), (9, 7, 6.0, 450.0), (7, 11, 5.5, 250.0),
                                         (11, 6, 8.0, 300.0), (8, 9, 6.5, 500.0)][:n]):
        rep = mi.make_replica(f"r{r}", nxy, nxy, nz, R, T, seed=100 + r, gap=gap)
        reps.append(jitter(rep, 0.08, r))
    return reps


@pytest.mark.parametrize("gap", [1.2, 2.0])
@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_batched_replicas_match_oracle(md, params, precision, tol, gap):
    reps = _uneven_replicas(gap=gap)
    sim = md.MD(reps, params, precision=precision)
    info = sim.info()
    assert info["replicas"] == len(reps) and info["n_cr"] == sum(r.n_cr for r in reps)
    assert info["slots"] % 128 == 0 and info["slots"] >= info["n_cr"]
    for r, rep in enumerate(reps):
        o = oracle_eval(params, rep)
        assert rel_force_err(sim.forces(r), o["F"]).max() <= tol
        energy_close(sim.energy(r), o, 1e-12 if precision == "fp64" else 1e-5, 1e-10 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("gap", [1.2, 2.0])
def test_batched_trajectory_equals_replicas_alone(md, params, gap):
    reps = _uneven_replicas(3, gap=gap)
    batch = md.MD(reps, params, precision="fp64", rebuild_every=5)
    batch.step(30)
    for r, rep in enumerate(reps):
        osim = oracle.Sim(oracle.Potential(params), rep, skin=0.3, rebuild_every=5)
        osim.step(30)
        x, v, z, _ = batch.state(r)
        np.testing.assert_allclose(x, osim.state()["x"], rtol=0, atol=1e-10)
        assert z == osim.state()["z_ind"]


def test_ragged_free_cluster_and_no_indenter(md, params):
    rep = mi.small_cluster(3, jitter=0.1)          # 91 atoms: not a multiple of the tile
    rep.v_cr = np.random.default_rng(1).normal(0, 2e-3, rep.x_cr.shape)
    for prec, tol in (("fp64", FP64_TOL), ("mixed", MIXED_TOL)):
        sim = md.MD([rep], params, precision=prec)
        o = oracle_eval(params, rep)
        assert rel_force_err(sim.forces(0), o["F"]).max() <= tol
        e = sim.energy(0)
        assert e["morse"] == 0.0 and e["load"] == 0.0
        sim.step(20)
        sim.close()


def test_single_atom(md, params):
    rep = mi.small_cluster(1, jitter=0.0)
    rep.x_cr = rep.x_cr[:1].copy(); rep.v_cr = rep.v_cr[:1].copy(); rep.fixed = rep.fixed[:1].copy()
    sim = md.MD([rep], params, precision="mixed")
    assert np.all(sim.forces(0) == 0.0)
    e = sim.energy(0)
    assert e["potential"] == 0.0
    sim.step(5)


def test_bcc_closed_form_on_gpu(md, params):
    n = 6
    x = mi.bcc_film(n, n, n)
    rep = mi.Replica("bcc", x, np.zeros_like(x), np.zeros(len(x), np.uint8), np.zeros((0, 3)),
                     np.zeros(3), np.full(3, n * mi.A_CR), np.ones(3, np.int32), 0.0, 0.0, 1.0, mi.MASS_CR,
                     0.0, float(x[:, 2].max()))
    for prec, tol in (("fp64", 1e-9), ("mixed", 2e-6)):
        sim = md.MD([rep], params, precision=prec)
        e = sim.energy(0)
        assert e["potential"] / len(x) == pytest.approx(-params["_targets"]["E_c"], abs=tol)
        assert np.abs(sim.forces(0)).max() < (1e-11 if prec == "fp64" else 1e-5)


def test_state_roundtrip(md, params):
    rep = tiny(amp=0.05)
    sim = md.MD([rep], params, precision="fp64")
    sim.step(10)
    x, v, z, step = sim.state(0)
    e0 = sim.energy(0)
    sim.set_state(0, x, v, z, step)
    x2, v2, z2, step2 = sim.state(0)
    # positions come back wrapped into the periodic box (the list build wraps them)
    L = rep.box_hi - rep.box_lo
    d = x2 - x
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-12
    assert np.array_equal(v, v2) and z == z2 and step == step2
    e1 = sim.energy(0)
    assert e1["potential"] == pytest.approx(e0["potential"], rel=1e-13)
    # a state set from elsewhere is what the next step starts from
    import dataclasses
    o = oracle.Sim(oracle.Potential(params), dataclasses.replace(rep, z_indenter0=z), skin=0.3, x=x, v=v)
    sim.step(5)
    o.step(5)
    # positions are wrapped into the box only at list builds, and the two sides build on
    # their own schedules: compare modulo the period
    d = sim.state(0)[0] - o.state()["x"]
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-10


def test_set_state_of_one_replica_in_a_batch(md, params):
    """md_set_state on one replica of a batch: its new positions get the oracle's forces,
    and the other replicas, whose state is unchanged, step on exactly as in a batch that
    was never interrupted (no list rebuild: the change is within the skin)."""
    import dataclasses
    reps = _uneven_replicas(3)
    a = md.MD(reps, params, precision="mixed", skin=1.1)   # no rebuild in either run
    b = md.MD(reps, params, precision="mixed", skin=1.1)
    a.step(12); b.step(12)
    x, v, z, st = a.state(1)
    nreb = a.energy(1)["rebuilds"]
    rng = np.random.default_rng(11)
    x1 = x + rng.uniform(-0.02, 0.02, x.shape)
    a.set_state(1, x1, v, z, st)
    assert a.energy(1)["rebuilds"] == nreb
    o = oracle_eval(params, dataclasses.replace(reps[1], x_cr=x1), z_ind=z)
    assert rel_force_err(a.forces(1), o["F"]).max() <= MIXED_TOL
    a.step(9); b.step(9)
    for r in (0, 2):
        xa, va, za, sa = a.state(r)
        xb, vb, zb, sb = b.state(r)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and za == zb and sa == sb
        assert np.array_equal(a.forces(r), b.forces(r))
    assert np.isfinite(a.state(1)[0]).all()
    a.close(); b.close()


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_set_state_keeps_or_rebuilds_lists(md, params, precision, tol):
    """Positions replaced within the skin rule keep the lists (no rebuild counted) and give
    the oracle's forces at the new positions; larger moves rebuild them."""
    import dataclasses
    rep = tiny(amp=0.05, gap=2.0)
    sim = md.MD([rep], params, precision=precision)
    sim.step(10)
    sim.build_neighbors()
    x, v, z, step = sim.state(0)
    nreb = sim.energy(0)["rebuilds"]
    rng = np.random.default_rng(3)
    x1 = x + rng.uniform(-0.03, 0.03, x.shape)
    sim.set_state(0, x1, v, z, step)
    assert sim.energy(0)["rebuilds"] == nreb
    o = oracle_eval(params, dataclasses.replace(rep, x_cr=x1), z_ind=z)
    assert rel_force_err(sim.forces(0), o["F"]).max() <= tol
    x2 = x + rng.uniform(-0.4, 0.4, x.shape)
    sim.set_state(0, x2, v, z, step)
    assert sim.energy(0)["rebuilds"] == nreb + 1
    o = oracle_eval(params, dataclasses.replace(rep, x_cr=x2), z_ind=z)
    assert rel_force_err(sim.forces(0), o["F"]).max() <= tol
    sim.step(20)   # and the run goes on from there
    assert np.isfinite(sim.state(0)[0]).all()
    sim.close()


def test_lost_atom_reported(md, params):
    rep = tiny(amp=0.0)
    rep.x_cr = rep.x_cr.copy()
    rep.x_cr[5, 2] = rep.box_hi[2] + 1.0
    with pytest.raises(md.MDError) as ei:
        md.MD([rep], params, precision="mixed")
    assert ei.value.code == md.MD_ERR_LOST_ATOM


def test_blown_up_state_reported_without_quadratic_rebuild(md, params):
    """Every position non-finite (a blown-up run): all atoms bin into one cell; the rebuild
    must still be linear in the atoms and the call must end with MD_ERR_LOST_ATOM."""
    import time
    rep = mi.make_workload("64k").replicas[0]
    sim = md.MD([rep], params, precision="mixed")
    sim.step(5)
    x = np.full_like(rep.x_cr, np.nan)
    t0 = time.perf_counter()
    with pytest.raises(md.MDError) as ei:
        sim.set_state(0, x, None, 0.0, 5)
    assert ei.value.code == md.MD_ERR_LOST_ATOM
    assert time.perf_counter() - t0 < 10.0
    sim.close()


def test_neighbour_capacity_grows_at_build(md, params):
    rep = tiny(amp=0.05)
    sim = md.MD([rep], params, precision="mixed", kmax=20, kcmax=8)
    info = sim.info()
    assert info["kmax"] >= info["max_cnt"] > 20
    o = oracle_eval(params, rep)
    assert rel_force_err(sim.forces(0), o["F"]).max() <= MIXED_TOL


def test_skin_violation_reported_in_fixed_interval_mode(md, params):
    rep = tiny(amp=0.0, T=3000.0, gap=3.0)
    sim = md.MD([rep], params, precision="mixed", rebuild_every=100000)
    with pytest.raises(md.MDError) as ei:
        sim.step(200)
    assert ei.value.code == md.MD_ERR_SKIN_VIOLATION


def test_bad_periodic_box_rejected(md, params):
    rep = mi.make_replica("small", 4, 4, 4, 0.0, 10.0, seed=1)   # 11.5 A < 3 cells of 4.84 A
    with pytest.raises(md.MDError) as ei:
        md.MD([rep], params)
    assert ei.value.code == md.MD_ERR_ARG


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-6)])
def test_set_state_same_positions_keeps_forces(md, params, precision, tol):
    """md_set_state with the positions the handle holds and new velocities: the forces of
    the state stay (they do not depend on velocities; nothing is re-evaluated) and the run
    goes on from the new velocities, as the oracle started at that state does."""
    import dataclasses
    rep = tiny(amp=0.05, gap=2.0, T=300.0)
    sim = md.MD([rep], params, precision=precision)
    sim.step(20)
    x, v, z, st = sim.state(0)
    F = sim.forces(0)
    v2 = np.ascontiguousarray(0.8 * v)
    sim.set_state(0, x, v2, z, st)
    assert np.array_equal(sim.forces(0), F)
    sim.step(30)
    o = oracle.Sim(oracle.Potential(params), dataclasses.replace(rep, x_cr=x, v_cr=v2, z_indenter0=z), skin=0.3)
    o.step(30)
    d = sim.state(0)[0] - o.state()["x"]
    L = rep.box_hi - rep.box_lo
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < tol
    sim.close()
