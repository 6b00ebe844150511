"""Lattice topological charge Q (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper labels minima and saddles by their skyrmion number (Results,
Pd/Fe/Ir(111) networks: Neel skyrmion Q = +1, antiskyrmion Q = -1, biskyrmion
Q = 2) but does not define it on the lattice.  Reading R10: the Berg-Luescher
charge, a sum over all 2N elementary triangles of the signed solid angle
spanned by the three spins,

    Omega(a, b, c) = 2 atan2(a . (b x c), 1 + a.b + b.c + c.a),
    Q = -(1 / 4 pi) sum_triangles Omega,

with up triangles (i, i+a1, i+a2) and down triangles (i+a1, i+a1+a2, i+a2), both
counter-clockwise in the plane.  The overall minus sign makes a core-down
skyrmion in a +z background count +1.  On a periodic lattice Q is an integer
away from exceptional configurations (a triangle with a vanishing atan2
argument pair).
"""
from __future__ import annotations

import math

import numpy as np

from .spin import nb


def solid_angle(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Signed solid angle of the spherical triangle (a, b, c), field-wise."""
    bxc = np.stack([b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]])
    num = np.sum(a * bxc, axis=0)
    den = 1.0 + np.sum(a * b, axis=0) + np.sum(b * c, axis=0) + np.sum(c * a, axis=0)
    return 2.0 * np.arctan2(num, den)


def topo_charge(m: np.ndarray) -> float:
    m0 = m
    m1 = nb(m, 1, 0)
    m2 = nb(m, 0, 1)
    m3 = nb(m, 1, 1)
    up = solid_angle(m0, m1, m2)
    down = solid_angle(m1, m3, m2)
    return -math.fsum(np.concatenate([up.ravel(), down.ravel()])) / (4.0 * math.pi)


def integer_charge(m: np.ndarray):
    """(round(Q), |Q - round(Q)|)."""
    q = topo_charge(m)
    r = int(round(q))
    return r, abs(q - r)
