"""Lattice and model description for the oracle.

Periodic 2D triangular lattice with primitive vectors a1 = (1, 0) and
a2 = (1/2, sqrt(3)/2); site (i1, i2) sits at i1*a1 + i2*a2.  A neighbour offset
(d1, d2) in index space has length |r|^2 = d1^2 + d1*d2 + d2^2.  The three
shells at |r| = 1, sqrt(3), 2 each hold six neighbours; the paper's parameter
tables (Supplementary Note 4) list distance ratios 1 : sqrt(3) : 2 with six
pairs per shell, which identifies the triangular lattice.

Energy parameters (meV): J_s per shell, Neel DMI strength D on the first shell
with D_ij = D (z x r_hat_ij), uniaxial anisotropy K along e_z and a Zeeman term
mu*B along +z (Eq. param-hamiltonian).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

# (d1, d2) offsets of each shell, listed so that every offset and its negative
# both appear.
SHELLS = (
    ((1, 0), (0, 1), (-1, 1), (-1, 0), (0, -1), (1, -1)),        # |r| = 1
    ((1, 1), (-1, 2), (-2, 1), (-1, -1), (1, -2), (2, -1)),      # |r| = sqrt(3)
    ((2, 0), (0, 2), (-2, 2), (-2, 0), (0, -2), (2, -2)),        # |r| = 2
)


def offset_vector(d1: int, d2: int):
    """Cartesian vector of an index-space offset."""
    return (d1 + 0.5 * d2, 0.5 * math.sqrt(3.0) * d2)


@dataclass(frozen=True)
class Model:
    L1: int
    L2: int
    J: tuple = (1.0,)
    D: float = 0.0
    K: float = 0.0
    muB: float = 0.0

    def __post_init__(self):
        if len(self.J) < 1 or len(self.J) > len(SHELLS):
            raise ValueError("1..3 exchange shells supported")
        if self.L1 < 5 or self.L2 < 5:
            # shell-3 offsets (+-2) must stay distinct modulo L
            raise ValueError("lattice sides must be >= 5")

    @property
    def N(self) -> int:
        return self.L1 * self.L2


def model_from_workload(p: dict) -> Model:
    return Model(L1=p["L1"], L2=p["L2"], J=tuple(p["J"]), D=p["D"], K=p["K"], muB=p["muB"])
