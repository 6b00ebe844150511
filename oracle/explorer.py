"""Explorer front-end of the bilayer kernel: masked perturbations and the
objectives the multi-objective selection ranks (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Results, "Multi-objective initial-configuration explorer": an initial
configuration is x = x0 + P_Omega delta over the active set Omega (the mask),
optionally projected back to the admissible manifold (the spin-tangent
retraction); the selection uses (i) diversity (similarity among candidates and
to an archive; Fig. 2e-f report the population's total pairwise L1 distance and
its maximin L1 distance), (ii) feasibility (normalised violations, e.g. of the
initial topological charge) and (iii) minimum-mode separability
Delta lambda = lambda_2 - lambda_1.  Readings where the paper gives no rule:

* [R17] For spins, delta holds a 3-vector per site; its tangent part at x0 is
  kept on the active sites (mask byte 1) and zeroed elsewhere, and the spins
  are rotated by it (the Rodrigues retraction of R7); inactive sites keep x0
  exactly.
* [R18] Distances are L1 over all 3N components.  The diversity of candidate a
  is d_a = min_b |x_a - x_b|_1 over the other candidates and the archive (to
  be maximised); the population's maximin is min_a d_a (over candidates only)
  and its total pairwise L1 the sum over pairs a < b.
* [R19] Feasibility violation of a candidate: |Q(x_a) - Q_target| /
  max(1, |Q_target|), 0 when feasible.
"""
from __future__ import annotations

import numpy as np

from . import spin, topo


def masked_perturbation(x0: np.ndarray, mask: np.ndarray, delta: np.ndarray) -> np.ndarray:
    """x = R_x0(P_Omega P_x0 delta) (R17); mask: (L2, L1) of 0/1."""
    active = mask.astype(bool)
    t = spin.project(x0, delta) * active[None]
    out = spin.retract(x0, t)
    out[:, ~active] = x0[:, ~active]
    return out


def pairwise_l1(X) -> np.ndarray:
    """D[a, b] = sum_e |X_a[e] - X_b[e]| for a list of configurations."""
    P = len(X)
    D = np.zeros((P, P))
    for a in range(P):
        for b in range(a + 1, P):
            D[a, b] = D[b, a] = float(np.sum(np.abs(X[a] - X[b])))
    return D


def diversity(D: np.ndarray, D_archive: np.ndarray | None = None) -> np.ndarray:
    """d_a = min over the other candidates (and the archive columns) (R18)."""
    P = D.shape[0]
    d = np.full(P, np.inf)
    for a in range(P):
        for b in range(P):
            if b != a:
                d[a] = min(d[a], D[a, b])
        if D_archive is not None:
            for c in range(D_archive.shape[1]):
                d[a] = min(d[a], D_archive[a, c])
    return d


def population_figures(D: np.ndarray):
    """(total pairwise L1, maximin L1) of a population (Fig. 2e-f)."""
    P = D.shape[0]
    total = sum(D[a, b] for a in range(P) for b in range(a + 1, P))
    return total, float(np.min(diversity(D)))


def feasibility(Q: float, Q_target: float) -> float:
    """Normalised charge violation (R19)."""
    return abs(Q - Q_target) / max(1.0, abs(Q_target))


def separability(lam1: float, lam2: float) -> float:
    """Delta lambda = lambda_2 - lambda_1."""
    return lam2 - lam1


def objectives(X, Q_target: float, lams, X_archive=None):
    """Per-candidate (diversity, violation, separability) from the
    configurations and their two lowest curvatures."""
    D = pairwise_l1(X)
    Da = None
    if X_archive:
        Da = np.array([[float(np.sum(np.abs(x - y))) for y in X_archive] for x in X])
    d = diversity(D, Da)
    v = np.array([feasibility(topo.topo_charge(x), Q_target) for x in X])
    s = np.array([separability(l1, l2) for l1, l2 in lams])
    return d, v, s
