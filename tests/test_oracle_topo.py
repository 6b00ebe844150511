"""Pins of the oracle's lattice topological charge."""
import math
import os

import numpy as np
import pytest

import inputs
from oracle import topo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "charges.txt")


def golden_charges():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = int(v)
    return out


def test_solid_angle_of_an_octant():
    x, y, z = (np.array(v, dtype=float).reshape(3, 1) for v in ((1, 0, 0), (0, 1, 0), (0, 0, 1)))
    assert topo.solid_angle(x, y, z)[0] == pytest.approx(math.pi / 2, rel=1e-15)
    assert topo.solid_angle(x, z, y)[0] == pytest.approx(-math.pi / 2, rel=1e-15)
    # a degenerate (coplanar great-circle) triangle has zero area
    w = np.array([1.0, 1.0, 0.0]).reshape(3, 1) / math.sqrt(2)
    assert topo.solid_angle(x, w, y)[0] == pytest.approx(0.0, abs=1e-15)


def test_charges_printed_in_the_paper():
    g = golden_charges()
    L = 48
    cases = {
        "skyrmion": inputs.skyrmion(L, L, 5.0),
        "antiskyrmion": inputs.skyrmion(L, L, 5.0, anti=True),
        "biskyrmion": inputs.biskyrmion(L, L, 5.0),
        "bi-antiskyrmion": inputs.multi_texture(L, L, -2, 4.0, 77),
    }
    for name, m in cases.items():
        q, frac = topo.integer_charge(m)
        assert q == g[name], name
        assert frac < 1e-9


def test_charge_of_uniform_state_and_translations():
    assert topo.topo_charge(inputs.ferromagnet(10, 10)) == pytest.approx(0.0, abs=1e-15)
    m = inputs.skyrmion(40, 36, 4.5, c=(10.3, 20.7))
    q = topo.topo_charge(m)
    assert q == pytest.approx(1.0, abs=1e-9)
    assert topo.topo_charge(np.roll(m, (5, 11), axis=(1, 2))) == pytest.approx(q, abs=1e-12)


@pytest.mark.parametrize("charge", [-2, -1, 0, 1, 2])
def test_random_charge_textures(charge):
    m = inputs.multi_texture(64, 64, charge, 4.0, 1234 + charge)
    q, frac = topo.integer_charge(m)
    assert q == charge
    assert frac < 1e-9


def test_charge_is_integer_on_noisy_states():
    m = inputs.add_noise(inputs.biskyrmion(64, 64, 6.0), 0.2, 99)
    q, frac = topo.integer_charge(m)
    assert frac < 1e-9
