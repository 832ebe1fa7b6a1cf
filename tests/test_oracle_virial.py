"""Pins of the oracle's per-atom virial (the potential part of per-atom stress times
volume; Sec. 2.1 lists stresses among Task 4's outputs).  Summed over the atoms the virial
is the derivative of the energy with respect to a homogeneous deformation x -> (I + e) x,
checked here by central differences of the oracle's energy."""
import numpy as np
import pytest

import md_inputs as mi
import oracle

COMP = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def strained(x, e):
    return x @ (np.eye(3) + e).T


def fd(energy, h=1e-6):
    out = []
    for (i, j) in COMP:
        e = np.zeros((3, 3)); e[i, j] = h
        out.append((energy(e) - energy(-e)) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("tab", [0, 1])
def test_periodic_virial_is_the_strain_derivative(params, tab):
    pot = oracle.Potential(params, tabulated=tab)
    n, a = 6, mi.A_CR
    rng = np.random.default_rng(1)
    x0 = mi.bcc_film(n, n, n, a) + rng.uniform(-0.08, 0.08, (2 * n ** 3, 3))
    lo = np.zeros(3); L = np.full(3, n * a); per = np.ones(3, np.int32)
    W = oracle.virial(pot, x0, lo, L, per)["W"].sum(0)

    def energy(e):   # orthorhombic boxes only: the diagonal strains
        return oracle.forces(pot, strained(x0, e), lo, L * np.diag(np.eye(3) + e), per)["potential"]

    for k in range(3):
        (i, j) = COMP[k]
        e = np.zeros((3, 3)); h = 1e-6; e[i, j] = h
        d = (energy(e) - energy(-e)) / (2 * h)
        assert W[k] == pytest.approx(d, rel=1e-6)


def test_free_cluster_virial_all_components(params):
    """A free cluster (no periodicity): the full tensor, shears included; it is symmetric
    because a rotation does not change the energy."""
    pot = oracle.Potential(params, tabulated=0)
    rep = mi.small_cluster(n_side=4, jitter=0.1, seed=5)
    lo, hi, per = rep.box_lo, rep.box_hi, rep.periodic
    W = oracle.virial(pot, rep.x_cr, lo, hi, per)["W"].sum(0)
    energy = lambda e: oracle.forces(pot, strained(rep.x_cr, e), lo - 5, hi + 5, per)["potential"]
    d = fd(energy)
    np.testing.assert_allclose(W, d, rtol=1e-6, atol=1e-8 * np.abs(d).max())
    for (i, j), k in ((COMP[3], 3), (COMP[4], 4), (COMP[5], 5)):
        e = np.zeros((3, 3)); h = 1e-6; e[j, i] = h   # the transposed shear gives the same
        assert (energy(e) - energy(-e)) / (2 * h) == pytest.approx(d[k], rel=1e-6, abs=1e-8)


def test_virial_of_a_dimer_and_the_cr_c_half(params):
    """Two Cr atoms: each holds half of c d (x) d with c = (dE/dr)/r, dE/dr from the
    energy at r +- h.  A Cr-C pair gives the Cr atom half of its term: the virial added by
    an indenter atom is half the strain derivative it adds when both move."""
    pot = oracle.Potential(params, tabulated=0)
    lo, hi, per = np.full(3, -20.0), np.full(3, 20.0), np.zeros(3, np.int32)
    u = np.array([0.48, -0.36, 0.8]); u /= np.linalg.norm(u)
    r0 = 2.6
    x = np.stack([np.zeros(3), r0 * u])
    W = oracle.virial(pot, x, lo, hi, per)["W"]
    E = lambda r: oracle.forces(pot, np.stack([np.zeros(3), r * u]), lo, hi, per)["potential"]
    h = 1e-6
    c = (E(r0 + h) - E(r0 - h)) / (2 * h) / r0
    d = r0 * u
    want = 0.5 * c * np.array([d[0] * d[0], d[1] * d[1], d[2] * d[2], d[0] * d[1], d[0] * d[2], d[1] * d[2]])
    np.testing.assert_allclose(W[0], want, rtol=1e-7, atol=1e-12)
    np.testing.assert_allclose(W[1], want, rtol=1e-7, atol=1e-12)
    # Cr cluster + two C atoms within the Morse range
    rep = mi.small_cluster(n_side=3, jitter=0.05, seed=9)
    xc = np.array([[rep.x_cr[:, 0].mean(), rep.x_cr[:, 1].mean(), rep.x_cr[:, 2].max() + 2.3],
                   [rep.x_cr[:, 0].mean() + 1.4, rep.x_cr[:, 1].mean(), rep.x_cr[:, 2].max() + 2.6]])
    lo2, hi2 = rep.box_lo - 5, rep.box_hi + 5
    W_with = oracle.virial(pot, rep.x_cr, lo2, hi2, rep.periodic, xc)["W"].sum(0)
    W_without = oracle.virial(pot, rep.x_cr, lo2, hi2, rep.periodic)["W"].sum(0)
    e_with = lambda e: oracle.forces(pot, strained(rep.x_cr, e), lo2, hi2, rep.periodic, strained(xc, e))["potential"]
    e_without = lambda e: oracle.forces(pot, strained(rep.x_cr, e), lo2, hi2, rep.periodic)["potential"]
    morse_full = fd(e_with) - fd(e_without)
    assert np.abs(morse_full).max() > 1e-3
    np.testing.assert_allclose(W_with - W_without, 0.5 * morse_full, rtol=1e-6, atol=1e-7)   # FD noise ~1e-8
