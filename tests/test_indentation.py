"""Analysis of a load-depth curve (host logic, no GPU): the Hertz fit and the Oliver-Pharr
analysis against curves whose answers are known in closed form."""
import math

import numpy as np
import pytest

from paper_1507_07068_gb300 import indentation as ind


def test_hertz_fit_recovers_the_modulus():
    R, E = 30.0, 0.85
    h = np.linspace(-1.0, 3.0, 81)        # samples before contact are ignored
    P = np.where(h > 0, (4.0 / 3.0) * E * math.sqrt(R) * np.clip(h, 0, None) ** 1.5, 0.0)
    assert ind.hertz_modulus(h, P, R) == pytest.approx(E, rel=1e-12)


def test_contact_area_is_the_circle_cut_by_the_contact_plane():
    R = 12.0
    for hc in (0.1, 1.0, 5.0, 11.5):
        a2 = R * R - (R - hc) ** 2          # radius of the circle at depth hc below the apex
        assert ind.contact_area(hc, R) == pytest.approx(math.pi * a2, rel=1e-14)
    with pytest.raises(ValueError):
        ind.contact_area(0.0, R)


def test_oliver_pharr_on_a_power_law_unloading_curve():
    R, alpha, h_f, m = 30.0, 0.9, 1.2, 1.35
    h = np.linspace(3.08, 1.25, 60)        # from the maximum depth outwards
    P = alpha * (h - h_f) ** m
    out = ind.oliver_pharr(h, P, R, top=0.8)
    assert out["alpha"] == pytest.approx(alpha, rel=1e-6)
    assert out["h_f"] == pytest.approx(h_f, rel=1e-6)
    assert out["m"] == pytest.approx(m, rel=1e-6)
    h_max, P_max = 3.08, alpha * (3.08 - h_f) ** m
    S = alpha * m * (h_max - h_f) ** (m - 1)                  # dP/dh at h_max
    h_c = h_max - 0.75 * P_max / S
    A = math.pi * (R * R - (R - h_c) ** 2)
    assert out["S"] == pytest.approx(S, rel=1e-6)
    assert out["h_c"] == pytest.approx(h_c, rel=1e-6)
    assert out["E_r"] == pytest.approx(math.sqrt(math.pi) * S / (2 * math.sqrt(A)), rel=1e-6)
    assert out["H"] == pytest.approx(P_max / A, rel=1e-6)


def test_oliver_pharr_on_an_elastic_hertz_contact_gives_its_modulus():
    """Unloading along the Hertz curve itself (no residual depth): the contact depth is
    half the depth and the method returns E* up to the cap's h_c^2 term of the area,
    E_r = E* / sqrt(1 - h_max / (4R))."""
    R, E, h_max = 100.0, 0.6, 1.0
    h = np.linspace(h_max, 0.05, 80)
    P = (4.0 / 3.0) * E * math.sqrt(R) * h ** 1.5
    out = ind.oliver_pharr(h, P, R, top=0.9)
    assert out["m"] == pytest.approx(1.5, rel=1e-6)
    assert out["h_c"] == pytest.approx(0.5 * h_max, rel=1e-6)
    assert out["E_r"] == pytest.approx(E / math.sqrt(1.0 - h_max / (4.0 * R)), rel=1e-6)
