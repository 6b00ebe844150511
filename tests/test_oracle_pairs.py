"""Pins of the pair-list oracle: the shell model written as a pair list
reproduces the shell oracle (energy, gradient, HVP); for a random closed list
the energy is a quadratic whose central differences give the gradient and
whose gradient differences give the HVP exactly; the HVP is symmetric; the
energy is translation invariant; an unclosed list is detected."""
import numpy as np
import pytest

import inputs
from oracle import pairs, spin
from oracle.model import Model

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


def _vdot(a, b):
    return float(np.sum(a * b))


def test_shell_model_as_pairs_reproduces_the_shell_oracle():
    M = Model(9, 7, **FULL)
    pm = pairs.PairModel(9, 7, pairs.pairs_from_model(M), K=M.K, muB=M.muB)
    assert pairs.closed(pm.pairs)
    m = inputs.add_noise(inputs.skyrmion(9, 7, 2.0), 0.2, 3)
    v = inputs.gaussian_field(4, 9, 7)
    assert pairs.energy(pm, m) == pytest.approx(spin.energy(M, m), rel=1e-13)
    np.testing.assert_allclose(pairs.euclid_grad(pm, m), spin.euclid_grad(M, m), atol=1e-12)
    g, s = spin.riemann_grad(M, m)
    np.testing.assert_allclose(pairs.hvp(pm, m, s, v), spin.hvp(M, m, s, v), atol=1e-12)


@pytest.fixture(scope="module")
def random_model():
    L1, L2 = 13, 11
    pl = inputs.random_pairs(71, reach=3, n_offsets=12)
    return pairs.PairModel(L1, L2, pl, K=0.07, muB=0.03)


def test_random_list_is_closed_and_nonempty(random_model):
    assert len(random_model.pairs) >= 10 and pairs.closed(random_model.pairs)
    broken = list(random_model.pairs)
    d1, d2, J, D = broken[0]
    broken[0] = (d1, d2, J + 0.1, D)
    assert not pairs.closed(broken)


def test_gradient_is_the_central_difference_of_the_quadratic_energy(random_model):
    pm = random_model
    m = inputs.gaussian_field(72, pm.L1, pm.L2)
    g = pairs.euclid_grad(pm, m)
    for seed in range(73, 76):
        v = inputs.gaussian_field(seed, pm.L1, pm.L2)
        h = 0.25
        fd = (pairs.energy(pm, m + h * v) - pairs.energy(pm, m - h * v)) / (2 * h)
        assert fd == pytest.approx(_vdot(g, v), rel=1e-10, abs=1e-9)


def test_hvp_is_the_gradient_difference_and_symmetric(random_model):
    pm = random_model
    m = inputs.gaussian_field(80, pm.L1, pm.L2)
    v = inputs.gaussian_field(81, pm.L1, pm.L2)
    w = inputs.gaussian_field(82, pm.L1, pm.L2)
    hv = pairs.euclid_hvp(pm, v)
    h = 0.5
    fd = (pairs.euclid_grad(pm, m + h * v) - pairs.euclid_grad(pm, m - h * v)) / (2 * h)
    np.testing.assert_allclose(hv, fd, atol=1e-11)
    assert _vdot(w, hv) == pytest.approx(_vdot(v, pairs.euclid_hvp(pm, w)), rel=1e-12)


def test_energy_is_translation_invariant(random_model):
    pm = random_model
    m = inputs.add_noise(inputs.skyrmion(pm.L1, pm.L2, 3.0), 0.1, 90)
    moved = np.roll(m, shift=(2, 5), axis=(1, 2))
    assert pairs.energy(pm, moved) == pytest.approx(pairs.energy(pm, m), rel=1e-12)
