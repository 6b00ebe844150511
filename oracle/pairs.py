"""General pair-list Hamiltonian (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's Pd/Fe/Ir(111) model (Supplementary Note 4 tables) has many
exchange shells and full DMI vectors; its moment, anisotropy and field
conversion are not given, so this module carries the general form with the
parameters as inputs:

    E = - sum_i sum_p [ J_p m_i . m_{i+d_p} + D_p . (m_i x m_{i+d_p}) ]
        - muB sum_i m_iz - K sum_i m_iz^2

over a list of ordered pairs p = (d1, d2, J, D) closed under d -> -d with
J_{-d} = J_d and D_{-d} = -D_d (every bond counted twice, as in Eq.
param-hamiltonian).  The derivatives are taken term by term from this sum
(the i-th spin appears as the first member of the pairs (i, i+d) and the
second member of the pairs (i-d, i)); nothing assumes the closure except the
validity check.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import spin
from .model import SHELLS, Model


@dataclass
class PairModel:
    L1: int
    L2: int
    pairs: list = field(default_factory=list)   # [(d1, d2, J, (Dx, Dy, Dz))]
    K: float = 0.0
    muB: float = 0.0

    @property
    def N(self) -> int:
        return self.L1 * self.L2


def closed(pairs) -> bool:
    """Every (d, J, D) has exactly one partner (-d, J, -D)."""
    for d1, d2, J, D in pairs:
        partners = [q for q in pairs if q[0] == -d1 and q[1] == -d2 and q[2] == J
                    and all(q[3][c] == -D[c] for c in range(3))]
        if len(partners) != 1:
            return False
    return True


def pairs_from_model(model: Model):
    """The shell model of Eq. param-hamiltonian written as a pair list."""
    out = []
    for Js, shell in zip(model.J, SHELLS):
        for d1, d2 in shell:
            D = model.D * spin.dmi_vector(d1, d2) if (model.D != 0.0 and shell is SHELLS[0]) else np.zeros(3)
            out.append((d1, d2, float(Js), tuple(float(x) for x in D)))
    if model.D != 0.0 and len(model.J) < 1:
        raise ValueError
    return out


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def _vec(D, like):
    return np.asarray(D, dtype=float)[:, None, None] * np.ones_like(like)


def energy(pm: PairModel, m: np.ndarray) -> float:
    e = 0.0
    for d1, d2, J, D in pm.pairs:
        mj = spin.nb(m, d1, d2)
        e -= J * float(np.sum(m * mj))
        e -= float(np.sum(_vec(D, m) * _cross(m, mj)))
    e -= pm.muB * float(np.sum(m[2])) + pm.K * float(np.sum(m[2] ** 2))
    return e


def linear_field(pm: PairModel, x: np.ndarray) -> np.ndarray:
    """Gradient of the pair terms at x: the i-th spin as first member of
    (i, i+d) gives -J x_{i+d} - x_{i+d} x D; as second member of (i-d, i),
    -J x_{i-d} - D x x_{i-d}."""
    h = np.zeros_like(x)
    for d1, d2, J, D in pm.pairs:
        xp = spin.nb(x, d1, d2)
        xm = spin.nb(x, -d1, -d2)
        Dv = _vec(D, x)
        h -= J * (xp + xm) + _cross(xp, Dv) + _cross(Dv, xm)
    return h


def euclid_grad(pm: PairModel, m: np.ndarray) -> np.ndarray:
    g = linear_field(pm, m)
    g[2] -= pm.muB + 2.0 * pm.K * m[2]
    return g


def riemann_grad(pm: PairModel, m: np.ndarray):
    ge = euclid_grad(pm, m)
    s = np.sum(m * ge, axis=0)
    return ge - s[None] * m, s


def euclid_hvp(pm: PairModel, v: np.ndarray) -> np.ndarray:
    h = linear_field(pm, v)
    h[2] -= 2.0 * pm.K * v[2]
    return h


def hvp(pm: PairModel, m: np.ndarray, s: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Tangent HVP P_i[(hess E v)_i - s_i v_i] (reading R3)."""
    return spin.project(m, euclid_hvp(pm, v) - s[None] * v)
