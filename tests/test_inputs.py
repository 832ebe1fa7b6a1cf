"""The seeded input generators against the sizes the paper prints (Sec. 2.5, Sec. 4)."""
import json
import os

import numpy as np
import pytest

import md_inputs as mi

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


@pytest.mark.parametrize("case", GOLD["bcc_free_lateral_counts"], ids=lambda c: "x".join(map(str, c["cells"])))
def test_free_lateral_film_counts(case):
    nx, ny, nz = case["cells"]
    x = mi.bcc_film(nx, ny, nz, free_lateral=True)
    assert len(x) == case["atoms"] == mi.bcc_count(nx, ny, nz, True)
    # no duplicate sites
    assert len(np.unique(np.round(x, 6), axis=0)) == len(x)


def test_film_extent_matches_paper():
    x = mi.bcc_film(19, 19, 14, free_lateral=True)
    ext = x.max(0) - x.min(0)
    # 19 x 2.885 = 54.8 A of lattice plus the surface layer reach the paper's ~61 A only with
    # its own lattice constant/vacuum convention; the paper rounds, so check the order only.
    assert np.all(ext[:2] > 50) and np.all(ext[:2] < 62)
    assert 35 < ext[2] < 46


def test_periodic_film_count_and_spacing():
    x = mi.bcc_film(8, 8, 8)
    assert len(x) == 1024 == mi.bcc_count(8, 8, 8, False)
    d = np.diff(np.unique(np.round(x[:, 2], 9)))
    np.testing.assert_allclose(d, mi.A_CR / 2, rtol=0, atol=1e-12)


def test_indenter_count_near_paper():
    c = mi.diamond_hemisphere(GOLD["indenter"]["R_A"])
    # the paper's 394 for R = 9.78 A (Sec. 2.5, 4.3); the lattice registration is not printed
    assert abs(len(c) - GOLD["indenter"]["atoms"]) / GOLD["indenter"]["atoms"] < 0.1
    r = np.sqrt((c ** 2).sum(1))
    assert r.max() <= 9.78 + 1e-9 and c[:, 2].max() <= 1e-9


def test_fixed_planes():
    x = mi.bcc_film(4, 4, 4)
    for k in (1, 2, 3):
        m = mi.fixed_planes_mask(x, mi.A_CR, k)
        assert m.sum() == k * 16


def test_velocities_com_and_temperature():
    rng = np.random.default_rng(3)
    n = 20000
    fixed = np.zeros(n, np.uint8); fixed[:100] = 1
    v = mi.maxwell_velocities(n, 300.0, mi.MASS_CR, fixed, rng)
    assert np.all(v[:100] == 0)
    np.testing.assert_allclose(v[100:].mean(0), 0, atol=1e-15)
    ke = 0.5 * mi.MASS_CR * (v ** 2).sum() * mi.EV_PER_U_A2_FS2
    T = 2 * ke / (3 * (n - 100) * mi.KB_EV)
    assert abs(T - 300) < 10


def test_replica_geometry():
    rep = mi.make_replica("t", 8, 8, 8, 6.0, 300.0, seed=1)
    assert rep.n_cr == 1024 and rep.n_c > 50
    # indenter lowest atom 3 A above the top plane, centred laterally
    assert abs(rep.x_c[:, 2].min() - (rep.z_surface0 + 3.0)) < 1e-12
    np.testing.assert_allclose(rep.x_c[:, :2].mean(0), [4 * mi.A_CR, 4 * mi.A_CR], atol=1.0)
    assert rep.v_indenter == pytest.approx(-2e-4)


def test_batched_replicas_valid_minimum_image():
    reps = mi.batched_replicas(16)
    for r in reps:
        L = r.box_hi[0] - r.box_lo[0]
        R = np.sqrt((r.x_c[:, :2] - r.x_c[:, :2].mean(0)) ** 2).max() if r.n_c else 0
        assert L >= 2 * 5.0 + 2 * mi.RC_MORSE_DEFAULT
        assert 6 * mi.A_CR <= L <= 24 * mi.A_CR + 1e-9
    tot = sum(r.n_cr for r in mi.batched_replicas(256))
    assert 0.8e6 < tot < 1.6e6
