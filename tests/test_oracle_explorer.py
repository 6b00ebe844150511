"""Pins of the explorer oracle: the masked perturbation against its defining
properties (inactive sites untouched, unit spins, first-order agreement with
x0 + P_Omega P delta), pairwise L1 against scipy's cityblock distance, the
diversity and population figures against brute force on tiny inputs."""
import numpy as np
import pytest

import inputs
from oracle import explorer, spin, topo


def _disk_mask(L, r):
    i2, i1 = np.mgrid[0:L, 0:L]
    return ((i1 - L / 2) ** 2 + (i2 - L / 2) ** 2 <= r * r).astype(np.uint8)


def test_perturbation_keeps_inactive_sites_and_unit_spins():
    L = 12
    x0 = inputs.skyrmion(L, L, 3.0)
    mask = _disk_mask(L, 3.5)
    delta = 0.3 * inputs.gaussian_field(41, L, L)
    x = explorer.masked_perturbation(x0, mask, delta)
    off = mask == 0
    assert np.array_equal(x[:, off], x0[:, off])
    np.testing.assert_allclose(np.sum(x * x, axis=0), 1.0, atol=1e-14)
    assert np.max(np.abs(x[:, ~off] - x0[:, ~off])) > 1e-3


def test_perturbation_is_first_order_x0_plus_masked_tangent_step():
    L = 8
    x0 = inputs.add_noise(inputs.ferromagnet(L, L), 0.2, 3)
    mask = _disk_mask(L, 3.0)
    delta = inputs.gaussian_field(42, L, L)
    for eps in (1e-3, 1e-4):
        x = explorer.masked_perturbation(x0, mask, eps * delta)
        lin = x0 + eps * spin.project(x0, delta) * mask[None]
        # the retraction agrees with the linear step to second order
        assert np.max(np.abs(x - lin)) <= 2.0 * (eps * np.max(np.abs(delta))) ** 2 * 3


def test_pairwise_l1_matches_scipy_cityblock():
    scipy_distance = pytest.importorskip("scipy.spatial.distance")
    X = [inputs.gaussian_field(50 + j, 5, 7) for j in range(6)]
    D = explorer.pairwise_l1(X)
    ref = scipy_distance.cdist(np.stack([x.ravel() for x in X]), np.stack([x.ravel() for x in X]), "cityblock")
    np.testing.assert_allclose(D, ref, rtol=1e-13, atol=1e-12)


def test_diversity_and_population_figures_by_brute_force():
    # four points on a line at 0, 1, 3, 7 (one component): pairwise L1 are
    # the absolute differences; each point's nearest neighbour distance is
    # 1, 1, 2, 4; maximin 1; total 1+3+7+2+6+4 = 23; an archive point at 6.5
    # makes the last candidate's diversity 0.5
    pts = [0.0, 1.0, 3.0, 7.0]
    X = [np.array([[[p]]]) for p in pts]
    D = explorer.pairwise_l1(X)
    np.testing.assert_allclose(explorer.diversity(D), [1.0, 1.0, 2.0, 4.0])
    total, maximin = explorer.population_figures(D)
    assert total == pytest.approx(23.0) and maximin == pytest.approx(1.0)
    Da = np.array([[abs(p - 6.5)] for p in pts])
    np.testing.assert_allclose(explorer.diversity(D, Da), [1.0, 1.0, 2.0, 0.5])


def test_feasibility_and_separability():
    assert explorer.feasibility(2.0 + 1e-9, 2.0) == pytest.approx(0.5e-9)
    assert explorer.feasibility(0.0, 2.0) == pytest.approx(1.0)
    assert explorer.feasibility(1.0, 0.0) == pytest.approx(1.0)
    assert explorer.separability(-0.5, 0.25) == pytest.approx(0.75)
    # a skyrmion seed meets its charge target
    assert explorer.feasibility(topo.topo_charge(inputs.skyrmion(24, 24, 4.0)), 1.0) < 1e-6
