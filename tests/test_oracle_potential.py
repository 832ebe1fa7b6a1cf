"""Pins of the oracle's potential functions (Appendix Eqs. A2-A9).

The oracle differentiates Eqs. A2-A5 by the product and chain rules; the paper prints
the resulting force terms as Eqs. A6-A9.  Evaluating those printed expressions
literally pins every derivative (with A6/A7 read as +F' f' and +M' 2 f f', and A8/A9 as
-Phi' and -phi', the reading F = -grad E).
"""
import math

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def pot_an(params):
    return oracle.Potential(params, tabulated=0)


@pytest.fixture(scope="module")
def pot_tab(params):
    return oracle.Potential(params, tabulated=1)


def test_A6_embedding_force_term(params, pot_an):
    p = params
    for rho in (0.7 * p["rho_e"], 0.95 * p["rho_e"], 1.3 * p["rho_e"], 3.0):
        for r in (2.3, 2.9, 3.7):
            _, Fd = pot_an.eval(oracle.OR_EMBED, rho)
            _, fd = pot_an.eval(oracle.OR_F_RAW, r)
            s = rho / p["rho_e"]
            T1 = -(p["n"] ** 2 * p["F_o"] * p["beta"] * p["f_e"] / (r * rho)) * (p["r_e"] / r) ** p["beta"] \
                * s ** p["n"] * math.log(s)
            assert Fd * fd == pytest.approx(T1, rel=1e-13, abs=1e-15)


def test_A7_mterm_force_term(params, pot_an):
    p = params
    for P in (0.5 * p["P_e"], 0.9 * p["P_e"], 1.2 * p["P_e"], 1.9 * p["P_e"]):
        for r in (2.3, 2.9, 3.7):
            _, Md = pot_an.eval(oracle.OR_MTERM, P)
            f, fd = pot_an.eval(oracle.OR_F_RAW, r)
            u = P / p["P_e"]
            T2 = -(4 * p["alpha"] * p["beta"] * p["f_e"] ** 2 * P / (p["P_e"] ** 2 * r)) \
                * (p["r_e"] / r) ** (2 * p["beta"]) * (2 - u) * (u - 1) * math.exp(-(u - 1) ** 2)
            assert Md * 2 * f * fd == pytest.approx(T2, rel=1e-12, abs=1e-15)


def test_A8_pair_force_term(params, pot_an):
    p = params
    for r in np.linspace(1.5, p["d"] * p["r_e"] - 1e-3, 17):
        _, dphi = pot_an.eval(oracle.OR_PHI_AN, r)
        x, d = r / p["r_e"], p["d"]
        T3 = -((x - d) / p["r_e"]) * (5 * p["a3"] * x ** 3 + (4 * p["a2"] - 3 * p["a3"] * d) * x ** 2
                                      + (3 * p["a1"] - 2 * p["a2"] * d) * x + (2 * p["a0"] - p["a1"] * d))
        assert -dphi == pytest.approx(T3, rel=1e-11, abs=1e-12)
    # Phi = 0 beyond x = d (Eq. A4)
    assert pot_an.eval(oracle.OR_PHI_AN, p["d"] * p["r_e"] * 1.001) == (0.0, 0.0)


def test_A9_morse_force_term(params, pot_an):
    p = params
    for y in (1.6, 2.0, 2.2, 2.9, 4.5):
        _, dm = pot_an.eval(oracle.OR_MORSE_RAW, y)
        q = y / p["y_eq"] - 1
        T4 = p["D_o"] * p["alpha_x"] / p["y_eq"] * (math.exp(-p["alpha_x"] * q) - math.exp(-p["alpha_x"] / 2 * q))
        assert -dm == pytest.approx(T4, rel=1e-13, abs=1e-16)


def test_special_values(params, pot_an):
    p = params
    Fv, Fd = pot_an.eval(oracle.OR_EMBED, p["rho_e"])
    assert Fv == pytest.approx(-p["F_o"], rel=1e-15) and abs(Fd) < 1e-15
    Mv, Md = pot_an.eval(oracle.OR_MTERM, p["P_e"])
    assert Mv == 0.0 and Md == 0.0
    # M extrema at u^2 = 1 (P = 2 P_e): M = alpha / e
    assert pot_an.eval(oracle.OR_MTERM, 2 * p["P_e"])[0] == pytest.approx(p["alpha"] / math.e, rel=1e-14)
    # Morse: minimum -D_o at y_eq (Eq. A5 unshifted)
    v, d = pot_an.eval(oracle.OR_MORSE_RAW, p["y_eq"])
    assert v == pytest.approx(-p["D_o"], rel=1e-15) and abs(d) < 1e-15
    # f(r_e) = f_e (Eq. A2)
    assert pot_an.eval(oracle.OR_F_RAW, p["r_e"])[0] == pytest.approx(p["f_e"], rel=1e-15)
    # an isolated atom: F(0) = M(0) = 0
    assert pot_an.eval(oracle.OR_EMBED, 0.0) == (0.0, 0.0)
    assert pot_an.eval(oracle.OR_MTERM, 0.0) == (0.0, 0.0)


def test_shifted_force_cutoff_is_C1(params, pot_an):
    rc = params["rc"]
    v, d = pot_an.eval(oracle.OR_F, rc - 1e-9)
    assert abs(v) < 1e-12 and abs(d) < 1e-8
    assert pot_an.eval(oracle.OR_F, rc) == (0.0, 0.0)
    v, d = pot_an.eval(oracle.OR_MORSE, params["rc_m"] - 1e-9)
    assert abs(v) < 1e-12 and abs(d) < 1e-9
    # literal mode truncates without shifting
    lit = oracle.Potential(params, tabulated=0, shifted=0)
    assert lit.eval(oracle.OR_F, rc - 1e-9)[0] == pytest.approx(lit.eval(oracle.OR_F_RAW, rc - 1e-9)[0])


@pytest.mark.parametrize("which,lo,hi", [(oracle.OR_F, 1.6, 4.5), (oracle.OR_PHI, 1.6, 4.5),
                                         (oracle.OR_MORSE, 1.3, 5.95), (oracle.OR_EMBED, 2.0, 40.0),
                                         (oracle.OR_MTERM, 3.0, 60.0)])
@pytest.mark.parametrize("tab", [0, 1])
def test_derivatives_by_central_differences(params, which, lo, hi, tab):
    pot = oracle.Potential(params, tabulated=tab)
    for x in np.linspace(lo, hi, 23):
        h = 1e-6 * max(1.0, x)
        vp, _ = pot.eval(which, x + h)
        vm, _ = pot.eval(which, x - h)
        _, d = pot.eval(which, x)
        fd = (vp - vm) / (2 * h)
        assert d == pytest.approx(fd, rel=2e-6, abs=5e-8)


def _fourth_derivative_bound(pot, which, a, b):
    # max |g''''| on [a, b] from a coarse 4th difference of the analytic function
    hh = 2e-3
    xs = np.linspace(a + 2 * hh, b - 2 * hh, 400)
    g = lambda x: pot.eval(which, x)[0]
    vals = [abs(g(x - 2 * hh) - 4 * g(x - hh) + 6 * g(x) - 4 * g(x + hh) + g(x + 2 * hh)) / hh ** 4 for x in xs]
    return max(vals)


@pytest.mark.parametrize("which,lo,hi", [(oracle.OR_F, 1.5, 4.54), (oracle.OR_PHI, 1.5, 4.54),
                                         (oracle.OR_MORSE, 1.5, 5.99)])
def test_hermite_within_error_bound(params, pot_an, pot_tab, which, lo, hi):
    """Cubic Hermite interpolation error <= h^4 max|g''''| / 384 on each interval."""
    h = params["h"]
    rng = np.random.default_rng(11)
    for a in np.arange(lo, hi - 0.05, 0.25):
        b = a + 0.25
        bound = h ** 4 * _fourth_derivative_bound(pot_an, which, a, b) / 384.0
        for x in rng.uniform(a, b, 40):
            err = abs(pot_tab.eval(which, x)[0] - pot_an.eval(which, x)[0])
            assert err <= 2.0 * bound + 1e-15


def test_hermite_reproduces_knots(params, pot_an, pot_tab):
    h = params["h"]
    for k in (0, 1, 500, 2000, 3500):
        r = params["r_min"] + k * (params["rc"] - params["r_min"]) / math.ceil((params["rc"] - params["r_min"]) / h - 1e-9)
        assert pot_tab.eval(oracle.OR_F, r)[0] == pytest.approx(pot_an.eval(oracle.OR_F, r)[0], rel=1e-13, abs=1e-15)


def test_neumaier_is_order_independent():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(10000) * 1e-8, [1e8, -1e8], rng.standard_normal(10000)])
    exact = math.fsum(x)  # correctly rounded sum
    s1 = oracle.neumaier(x)
    s2 = oracle.neumaier(x[::-1])
    assert abs(s1 - exact) <= 1e-13 * abs(exact) and abs(s2 - exact) <= 1e-13 * abs(exact)
    assert abs(float(np.sum(x)) - exact) > abs(s1 - exact)  # plain summation is worse here


def _knot_ext(params, which, r):
    """Value and slope at a knot in extended precision: Eq. A2 (shifted), A4, A5 (shifted)."""
    L = np.longdouble
    p = {k: L(v) for k, v in params.items() if isinstance(v, (int, float))}
    r = L(r)
    if which == oracle.OR_F:
        f = lambda q: p["f_e"] * np.power(p["r_e"] / q, p["beta"])
        frc = f(p["rc"]); dfrc = -p["beta"] * frc / p["rc"]
        return f(r) - frc - (r - p["rc"]) * dfrc, -p["beta"] * f(r) / r - dfrc
    if which == oracle.OR_PHI:
        x = r / p["r_e"]; t = x - p["d"]
        poly = ((p["a3"] * x + p["a2"]) * x + p["a1"]) * x + p["a0"]
        dpoly = (3 * p["a3"] * x + 2 * p["a2"]) * x + p["a1"]
        return t * t * poly, (2 * t * poly + t * t * dpoly) / p["r_e"]
    def m(y):
        q = y / p["y_eq"] - 1
        e1 = np.exp(-p["alpha_x"] * q); e2 = np.exp(-p["alpha_x"] * q / 2)
        return p["D_o"] * (e1 - 2 * e2), p["D_o"] * p["alpha_x"] * (e2 - e1) / p["y_eq"]
    mrc, dmrc = m(p["rc_m"])
    v, dv = m(r)
    return v - mrc - (r - p["rc_m"]) * dmrc, dv - dmrc


@pytest.mark.parametrize("which", [oracle.OR_F, oracle.OR_PHI, oracle.OR_MORSE])
def test_hermite_rounding_against_extended_precision(params, pot_tab, which):
    """Tables: knots are the extended-precision values rounded once to FP64, and the
    tabulated value and slope equal the cubic Hermite through those knots evaluated in
    extended precision to ~1e-14 (the oracle's grouping does not cancel)."""
    L = np.longdouble
    rc = params["rc_m"] if which == oracle.OR_MORSE else params["rc"]
    N = math.ceil((rc - params["r_min"]) / params["h"] - 1e-9)
    h = (rc - params["r_min"]) / N
    rng = np.random.default_rng(3)
    for r in rng.uniform(1.8, rc - 1e-3, 400):
        k = min(int(math.floor((r - params["r_min"]) / h)), N - 1)

        def knot(q):
            g, d = _knot_ext(params, which, rc if q == N else params["r_min"] + q * h)
            return float(g), float(d)
        g0, d0 = knot(k); g1, d1 = knot(k + 1)
        t = (L(r) - L(params["r_min"])) / L(h) - L(k)
        hh = L(h)
        v = (2 * t**3 - 3 * t**2 + 1) * L(g0) + (t**3 - 2 * t**2 + t) * hh * L(d0) + (-2 * t**3 + 3 * t**2) * L(g1) \
            + (t**3 - t**2) * hh * L(d1)
        dv = ((6 * t**2 - 6 * t) * L(g0) + (3 * t**2 - 4 * t + 1) * hh * L(d0) + (-6 * t**2 + 6 * t) * L(g1)
              + (3 * t**2 - 2 * t) * hh * L(d1)) / hh
        tv, td = pot_tab.eval(which, r)
        assert abs(tv - float(v)) <= 1e-14 * max(1.0, abs(float(v)))
        assert abs(td - float(dv)) <= 5e-14 * max(1.0, abs(float(dv)))
