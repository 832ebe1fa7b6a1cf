"""Pins of the oracle's neighbour sets, energy and forces (Eq. A1, Eq. (1), Eqs. A6-A10).

Each check is fixed by the mathematics rather than by the oracle itself:
brute force == cell list, forces == -grad E by central differences (per energy term
and in total), Newton's third law, the BCC closed form at the fitted lattice constant,
and the Cr dimer / Cr-C pair special cases.
"""
import numpy as np
import pytest

import md_inputs as mi
import oracle


def jittered_bcc(n, a=mi.A_CR, jitter=0.08, seed=1, periodic=(1, 1, 1)):
    rng = np.random.default_rng(seed)
    x = mi.bcc_film(n, n, n, a)
    x = x + rng.uniform(-jitter, jitter, x.shape)
    lo = np.zeros(3); hi = np.full(3, n * a)
    per = np.array(periodic, np.int32)
    for k in range(3):
        if not per[k]:
            lo[k] = x[:, k].min() - 5.0; hi[k] = x[:, k].max() + 5.0
    x = np.where(per[None, :] == 1, np.mod(x, hi[None, :]), x)
    return x, lo, hi, per


def as_sets(off, idx):
    return [frozenset(idx[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


@pytest.mark.parametrize("per", [(1, 1, 1), (1, 1, 0), (0, 0, 0)])
@pytest.mark.parametrize("cut", [4.5441, 4.8441, 6.3])
def test_brute_force_equals_cell_list(per, cut):
    x, lo, hi, per = jittered_bcc(8, periodic=per)
    ob, ib = oracle.neighbors(x, lo, hi, per, cut, method=0)
    oc, ic = oracle.neighbors(x, lo, hi, per, cut, method=1)
    assert np.array_equal(ob, oc) and np.array_equal(ib, ic)
    s = as_sets(ob, ib)
    for i, si in enumerate(s):        # symmetric, no self pairs
        assert i not in si
        for j in si:
            assert i in s[j]


def test_bcc_shell_counts():
    x, lo, hi, per = jittered_bcc(6, jitter=0.0)
    for cut, expect in ((2.6, 8), (3.0, 14), (4.5441, 26), (4.8441, 50)):
        off, _ = oracle.neighbors(x, lo, hi, per, cut)
        assert np.all(np.diff(off) == expect)


def test_cell_coords_in_range_and_wrapped():
    x, lo, hi, per = jittered_bcc(6)
    x = x.copy(); x[0, 0] = -0.3; x[1, 1] = hi[1] + 0.2
    c = oracle.cell_coords(x, lo, hi, per, 4.8441)
    n, w = oracle.grid(lo, hi, per, 4.8441)
    assert np.all(c >= 0) and np.all(c < n[None, :])
    assert c[0, 0] == n[0] - 1 and c[1, 1] == 0


@pytest.mark.parametrize("tab", [0, 1])
def test_bcc_closed_form(params, tab):
    """Perfect fully periodic BCC at a = 2.885 A: E/atom = -E_c, F = 0, dE/da = 0 (derived set)."""
    pot = oracle.Potential(params, tabulated=tab)
    n = 6

    def energy(a):
        x = mi.bcc_film(n, n, n, a)
        lo = np.zeros(3); hi = np.full(3, n * a)
        r = oracle.forces(pot, x, lo, hi, np.ones(3, np.int32))
        return r, len(x)

    r, N = energy(mi.A_CR)
    tol = 1e-12 if tab == 0 else 1e-9
    assert r["potential"] / N == pytest.approx(-params["_targets"]["E_c"], abs=tol)
    assert np.abs(r["F"]).max() < 1e-12
    assert abs(r["mterm"]) < 1e-12 * N      # M(P_e) = 0
    d = 1e-5
    ep = energy(mi.A_CR + d)[0]["potential"]; em = energy(mi.A_CR - d)[0]["potential"]
    assert abs((ep - em) / (2 * d) / N) < 1e-7


@pytest.mark.parametrize("tab", [0, 1])
def test_bcc_closed_form_long_cutoff(params_rstar, tab):
    """The set fitted with r* = 8.262 A (Sec. 2.6): the same lattice targets hold with the
    fifth and sixth neighbour shells inside the cut-off of f."""
    params = params_rstar
    assert params["rc"] == 8.262
    pot = oracle.Potential(params, tabulated=tab)
    n = 9   # three cells of r* per periodic axis

    def energy(a):
        x = mi.bcc_film(n, n, n, a)
        lo = np.zeros(3); hi = np.full(3, n * a)
        r = oracle.forces(pot, x, lo, hi, np.ones(3, np.int32))
        return r, len(x)

    r, N = energy(mi.A_CR)
    tol = 1e-12 if tab == 0 else 1e-9
    assert r["potential"] / N == pytest.approx(-params["_targets"]["E_c"], abs=tol)
    assert np.abs(r["F"]).max() < 1e-12
    assert abs(r["mterm"]) < 1e-12 * N
    d = 1e-5
    ep = energy(mi.A_CR + d)[0]["potential"]; em = energy(mi.A_CR - d)[0]["potential"]
    assert abs((ep - em) / (2 * d) / N) < 1e-7
    # rho_e is the density of a lattice atom: the shifted-force f summed over the BCC
    # lattice points within r* (enumerated here directly: 8, 6, 12, 24, 8, 6, 24, 24, 24 ...)
    m = 4
    g = np.arange(-m, m + 1)
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(float)
    pts = np.concatenate([c, c + 0.5]) * mi.A_CR
    rr = np.sqrt((pts ** 2).sum(1))
    rc = params["rc"]
    rr = rr[(rr > 0) & (rr < rc)]
    f = lambda q: params["f_e"] * (params["r_e"] / q) ** params["beta"]
    fs = f(rr) - f(rc) - (rr - rc) * (-params["beta"] * f(rc) / rc)   # shifted-force form
    assert len(rr) == 8 + 6 + 12 + 24 + 8 + 6 + 24 + 24 + 24 + 32 + 12
    assert params["rho_e"] == pytest.approx(float(fs.sum()), rel=1e-12)


def _isolate(params, term):
    p = dict(params)
    zero_pair = dict(a0=0.0, a1=0.0, a2=0.0, a3=0.0)
    if term == "pair":
        p.update(F_o=0.0, alpha=0.0)
    elif term == "embed":
        p.update(alpha=0.0, **zero_pair)
    elif term == "mterm":
        p.update(F_o=0.0, **zero_pair)
    elif term == "morse":
        p.update(F_o=0.0, alpha=0.0, **zero_pair)
    return p


@pytest.mark.parametrize("term", ["pair", "embed", "mterm", "morse", "all"])
@pytest.mark.parametrize("tab", [0, 1])
def test_forces_are_minus_energy_gradient(params, term, tab):
    """Central differences of E (Eq. A1 + Morse) against F, per term (Eq. (1), A6-A10)."""
    pot = oracle.Potential(_isolate(params, term), tabulated=tab)
    rng = np.random.default_rng(2)
    x = mi.bcc_film(3, 3, 3, free_lateral=True) + rng.uniform(-0.15, 0.15, (91, 3))
    lo = x.min(0) - 8.0; hi = x.max(0) + 8.0
    per = np.zeros(3, np.int32)
    xc = mi.diamond_hemisphere(4.0) + np.array([4.3, 4.3, x[:, 2].max() + 1.9 - 0.0])
    base = oracle.forces(pot, x, lo, hi, per, xc)
    h = 1e-5
    assert np.abs(base["F"]).max() > 1e-3
    for i in rng.choice(len(x), 12, replace=False):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            ep = oracle.forces(pot, xp, lo, hi, per, xc)["potential"]
            em = oracle.forces(pot, xm, lo, hi, per, xc)["potential"]
            fd = -(ep - em) / (2 * h)
            assert base["F"][i, k] == pytest.approx(fd, rel=1e-6, abs=2e-8)


def test_forces_minus_gradient_periodic(params):
    pot = oracle.Potential(params, tabulated=1)
    x, lo, hi, per = jittered_bcc(6, jitter=0.12, seed=9)
    base = oracle.forces(pot, x, lo, hi, per)
    h = 1e-5
    rng = np.random.default_rng(4)
    for i in rng.choice(len(x), 6, replace=False):
        for k in range(3):
            xp = x.copy(); xp[i, k] += h
            xm = x.copy(); xm[i, k] -= h
            fd = -(oracle.forces(pot, xp, lo, hi, per)["potential"] - oracle.forces(pot, xm, lo, hi, per)["potential"]) / (2 * h)
            assert base["F"][i, k] == pytest.approx(fd, rel=1e-6, abs=5e-8)


def test_newton_third_law(params):
    pot = oracle.Potential(params)
    rep = mi.make_replica("t", 6, 6, 6, 6.0, 300.0, seed=3, gap=0.5)
    rng = np.random.default_rng(0)
    x = rep.x_cr + rng.uniform(-0.1, 0.1, rep.x_cr.shape)
    r0 = oracle.forces(pot, x, rep.box_lo, rep.box_hi, rep.periodic)
    assert np.abs(r0["F"].sum(0)).max() < 1e-11
    r1 = oracle.forces(pot, x, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c)
    assert r1["load"] != 0.0
    # the indenter feels +load along z; the film the opposite
    assert r1["F"][:, 2].sum() == pytest.approx(-r1["load"], abs=1e-11)


def test_brute_and_cell_forces_identical(params):
    pot = oracle.Potential(params)
    x, lo, hi, per = jittered_bcc(6, periodic=(1, 1, 0), seed=5)
    a = oracle.forces(pot, x, lo, hi, per, method=0)
    b = oracle.forces(pot, x, lo, hi, per, method=1)
    assert np.array_equal(a["F"], b["F"])
    assert a["potential"] == b["potential"]


@pytest.mark.parametrize("tab", [0, 1])
def test_dimer_energy(params, tab):
    pot = oracle.Potential(params, tabulated=tab)
    for r in (2.2, 2.6, 3.3, 4.2):
        x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]]) + 20.0
        res = oracle.forces(pot, x, np.zeros(3), np.full(3, 40.0), np.zeros(3, np.int32), method=0)
        f, _ = pot.eval(oracle.OR_F, r)
        phi, _ = pot.eval(oracle.OR_PHI, r)
        E = 2 * pot.eval(oracle.OR_EMBED, f)[0] + phi + 2 * pot.eval(oracle.OR_MTERM, f * f)[0]
        assert res["potential"] == pytest.approx(E, rel=1e-13, abs=1e-14)
        assert res["F"][0, 0] == pytest.approx(-res["F"][1, 0], rel=1e-14)


def test_cr_c_pair(params):
    pot = oracle.Potential(params, tabulated=0, shifted=0)
    ys = np.linspace(1.8, 3.5, 341)
    E = []
    for y in ys:
        x = np.array([[20.0, 20.0, 20.0]])
        xc = np.array([[20.0, 20.0, 20.0 + y]])
        r = oracle.forces(pot, x, np.zeros(3), np.full(3, 40.0), np.zeros(3, np.int32), xc, method=0)
        E.append(r["morse"])
        _, dm = pot.eval(oracle.OR_MORSE_RAW, xc[0, 2] - x[0, 2])   # y as rounded in the positions
        assert r["F"][0, 2] == pytest.approx(dm, rel=1e-13, abs=1e-15)   # pushed down when repulsive
        assert r["load"] == pytest.approx(-dm, rel=1e-13, abs=1e-15)
    k = int(np.argmin(E))
    assert abs(ys[k] - params["y_eq"]) < 0.006
    assert min(E) == pytest.approx(-params["D_o"], rel=1e-4)


def test_cr_c_list_in_narrow_periodic_box_matches_plain_minimum_image():
    """Cr-C pairs by a plain numpy minimum-image double loop, in a box where the indenter
    plus twice the reach is wider than the period (pairs through the periodic image)."""
    # indenter sunk into the film so that its equator meets film atoms (a geometry test)
    rep = mi.make_replica("narrow", 8, 8, 6, 6.0, 300.0, seed=4, gap=-6.0)
    L = rep.box_hi - rep.box_lo
    cut = 6.3
    assert (rep.x_c[:, 0].max() - rep.x_c[:, 0].min()) + 2 * cut > L[0]
    off, idx = oracle.cneighbors(rep.x_cr, rep.x_c, rep.box_lo, rep.box_hi, rep.periodic, cut)
    d = rep.x_c[None, :, :] - rep.x_cr[:, None, :]
    for k in range(2):
        d[..., k] = np.where(d[..., k] > 0.5 * L[k], d[..., k] - L[k], d[..., k])
        d[..., k] = np.where(d[..., k] < -0.5 * L[k], d[..., k] + L[k], d[..., k])
    r2 = (d ** 2).sum(-1)
    for i in range(rep.n_cr):
        expect = set(np.nonzero(r2[i] < cut * cut)[0].tolist())
        assert set(idx[off[i]:off[i + 1]].tolist()) == expect, i
    # some pairs are reached only through the periodic image
    direct = rep.x_c[None, :, :2] - rep.x_cr[:, None, :2]
    assert np.any((r2 < cut * cut) & (np.abs(direct).max(-1) > 0.5 * L[0]))


def test_forces_given_passes_equal_the_single_evaluation(params):
    """The two passes of Task 4 with an exchange between them (oracle.forces_given): fed
    back its own first-pass F'(rho), M'(P) for every atom, the second pass gives the forces
    and energies of oracle.forces; a changed F' of one atom changes only the forces of the
    atoms within rc of it."""
    import md_inputs as mi
    rep = mi.make_replica("given", 6, 6, 5, 5.0, 300.0, seed=4, gap=1.5)
    x = rep.x_cr + np.random.default_rng(2).uniform(-0.1, 0.1, rep.x_cr.shape)
    pot = oracle.Potential(params)
    ref = oracle.forces(pot, x, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c)
    a = oracle.forces_given(pot, x, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c)
    b = oracle.forces_given(pot, x, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c,
                            given=np.ones(len(x), np.uint8), fm_in=a["fm"])
    assert np.array_equal(a["F"], ref["F"]) and np.array_equal(b["F"], ref["F"])
    assert a["pair"] == ref["pair"] and a["embed"] == ref["embed"]
    assert a["e_atom"].sum() == pytest.approx(ref["potential"], rel=1e-12)
    k = 17
    fm = a["fm"].copy(); fm[k, 0] += 0.05
    g = np.zeros(len(x), np.uint8); g[k] = 1
    c = oracle.forces_given(pot, x, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c, given=g, fm_in=fm)
    changed = np.nonzero(np.abs(c["F"] - ref["F"]).max(1) > 0)[0]
    off, idx = oracle.neighbors(x, rep.box_lo, rep.box_hi, rep.periodic, params["rc"])
    assert set(changed.tolist()) <= set(idx[off[k]:off[k + 1]].tolist()) | {k}
    assert len(changed) > 5
