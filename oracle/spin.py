"""Energy, gradients and tangent Hessian of the spin Hamiltonian (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper used here:

* [R1] The exchange and DMI sums of Eq. param-hamiltonian run over ordered
  pairs i != j exactly as printed, so every bond is counted twice.
* [R2] Neel DMI on the first shell only: D_ij = D (z x r_hat_ij), which is
  antisymmetric (D_ji = -D_ij) as an ordered-pair sum requires.
* The force is "understood as tangent-projected" (Methods, gradient section):
  F = -g with the Riemannian gradient g_i = grad_i E - (m_i . grad_i E) m_i.
* [R3] The HVP operator acts on the tangent bundle: for tangent v,
  (H v)_i = P_i (hess E v)_i - s_i v_i with s_i = m_i . grad_i E, the Riemannian
  Hessian on a product of unit spheres (Absil, Mahony & Sepulchre, 2008).  It is
  the tangent block of the Hermitian part of the Jacobian of the projected
  gradient that the paper assembles for its explicit-Hessian benchmark.

Arrays are (3, L2, L1) float64; ``nb(x, d1, d2)[:, i2, i1] = x[:, i2+d2, i1+d1]``
with periodic wrap.
"""
from __future__ import annotations

import math

import numpy as np

from .model import SHELLS, Model, offset_vector

ZHAT = np.array([0.0, 0.0, 1.0])


def nb(x: np.ndarray, d1: int, d2: int) -> np.ndarray:
    """Field of the neighbour at offset (d1, d2) of every site (periodic)."""
    return np.roll(x, shift=(-d2, -d1), axis=(-2, -1))


def dmi_vector(d1: int, d2: int) -> np.ndarray:
    """D_ij / D = z x r_hat for a first-shell offset (Neel, reading R2)."""
    rx, ry = offset_vector(d1, d2)
    n = math.hypot(rx, ry)
    return np.array([-ry / n, rx / n, 0.0])


def _dot(a, b):
    return np.sum(a * b, axis=0)


def _cross(a, b):
    return np.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


# ----------------------------------------------------------------------------
# energy (Eq. param-hamiltonian)
# ----------------------------------------------------------------------------
def site_energy(model: Model, m: np.ndarray) -> np.ndarray:
    """Per-site share of E: every ordered pair (i, j) is attributed to i."""
    e = np.zeros(m.shape[1:])
    for Js, shell in zip(model.J, SHELLS):
        for d1, d2 in shell:
            e -= Js * _dot(m, nb(m, d1, d2))
    if model.D != 0.0:
        for d1, d2 in SHELLS[0]:
            Dv = model.D * dmi_vector(d1, d2)
            e -= _dot(Dv[:, None, None] * np.ones_like(m), _cross(m, nb(m, d1, d2)))
    e -= model.muB * m[2]
    e -= model.K * m[2] ** 2
    return e


def energy(model: Model, m: np.ndarray) -> float:
    """E(m) of Eq. param-hamiltonian, summed with correct rounding (fsum)."""
    return math.fsum(site_energy(model, m).ravel())


# ----------------------------------------------------------------------------
# gradients
# ----------------------------------------------------------------------------
def euclid_grad(model: Model, m: np.ndarray) -> np.ndarray:
    """grad_i E of the unconstrained E (reverse-mode gradient of the paper):
    -2 sum_s J_s sum_d m_{i+d} - 2 D sum_{d in s1} [z (m_{i+d}.d_hat) - d_hat m_{i+d,z}]
    - muB z - 2 K m_iz z."""
    g = np.zeros_like(m)
    for Js, shell in zip(model.J, SHELLS):
        for d1, d2 in shell:
            g -= 2.0 * Js * nb(m, d1, d2)
    if model.D != 0.0:
        for d1, d2 in SHELLS[0]:
            # d/dm_i of -D_ij.(m_i x m_j), both orderings: -2 (m_j x D_ij)
            Dv = model.D * dmi_vector(d1, d2)
            mj = nb(m, d1, d2)
            g -= 2.0 * _cross(mj, Dv[:, None, None] * np.ones_like(m))
    g[2] -= model.muB
    g[2] -= 2.0 * model.K * m[2]
    return g


def riemann_grad(model: Model, m: np.ndarray):
    """(g, s): Riemannian gradient g_i = grad_i E - s_i m_i, s_i = m_i . grad_i E.
    The force of the paper is F = -g."""
    ge = euclid_grad(model, m)
    s = _dot(m, ge)
    return ge - s[None] * m, s


def project(m: np.ndarray, v: np.ndarray) -> np.ndarray:
    """P_i v_i = v_i - (m_i . v_i) m_i for every site."""
    return v - _dot(m, v)[None] * m


def euclid_hvp(model: Model, v: np.ndarray) -> np.ndarray:
    """(hess E) v; E is quadratic in m so this does not depend on m:
    -2 sum_s J_s sum_d v_{i+d} - 2 D sum_{d in s1}[z (v_{i+d}.d_hat) - d_hat v_{i+d,z}]
    - 2 K v_iz z."""
    h = np.zeros_like(v)
    for Js, shell in zip(model.J, SHELLS):
        for d1, d2 in shell:
            h -= 2.0 * Js * nb(v, d1, d2)
    if model.D != 0.0:
        for d1, d2 in SHELLS[0]:
            Dv = model.D * dmi_vector(d1, d2)
            h -= 2.0 * _cross(nb(v, d1, d2), Dv[:, None, None] * np.ones_like(v))
    h[2] -= 2.0 * model.K * v[2]
    return h


def hvp(model: Model, m: np.ndarray, s: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Riemannian Hessian-vector product for tangent v (reading R3):
    (H v)_i = P_i (hess E v)_i - s_i v_i.

    Evaluated as P_i[(hess E v)_i - s_i v_i], which is the same for tangent v and
    keeps the output exactly tangent: a rounding-level normal component of v is
    then not multiplied by -s_i ~ 10 meV and amplified by the normalisations of
    an eigensolver."""
    return project(m, euclid_hvp(model, v) - s[None] * v)


# ----------------------------------------------------------------------------
# retraction (exponential map on each unit sphere)
# ----------------------------------------------------------------------------
def retract(m: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Rodrigues rotation of every spin by its tangent step d_i (reading R7):
    m_i <- m_i cos|d_i| + (d_i/|d_i|) sin|d_i|, then rescaled to unit length."""
    th = np.sqrt(_dot(d, d))
    safe = np.where(th > 0.0, th, 1.0)
    out = m * np.cos(th)[None] + d * (np.sin(th) / safe)[None]
    return out / np.sqrt(_dot(out, out))[None]


# ----------------------------------------------------------------------------
# explicit dense Hessian (small lattices only)
# ----------------------------------------------------------------------------
def _site(model: Model, i1: int, i2: int) -> int:
    return (i2 % model.L2) * model.L1 + (i1 % model.L1)


def _cross_matrix(a: np.ndarray) -> np.ndarray:
    """[a]_x with [a]_x b = a x b."""
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def dense_euclid_hessian(model: Model):
    """(A, b) with E(m) = 1/2 m^T A m + b^T m, built term by term from
    Eq. param-hamiltonian.  Flat index 3*site + component, site = i2*L1 + i1."""
    n = 3 * model.N
    A = np.zeros((n, n))
    b = np.zeros(n)
    for i2 in range(model.L2):
        for i1 in range(model.L1):
            i = _site(model, i1, i2)
            for Js, shell in zip(model.J, SHELLS):
                for d1, d2 in shell:
                    j = _site(model, i1 + d1, i2 + d2)
                    # -J m_i.m_j: d^2/dm_i dm_j = -J I (and the transpose block)
                    A[3 * i:3 * i + 3, 3 * j:3 * j + 3] -= Js * np.eye(3)
                    A[3 * j:3 * j + 3, 3 * i:3 * i + 3] -= Js * np.eye(3)
            if model.D != 0.0:
                for d1, d2 in SHELLS[0]:
                    j = _site(model, i1 + d1, i2 + d2)
                    Dv = model.D * dmi_vector(d1, d2)
                    # -D.(m_i x m_j) = m_i^T [D]_x m_j
                    C = _cross_matrix(Dv)
                    A[3 * i:3 * i + 3, 3 * j:3 * j + 3] += C
                    A[3 * j:3 * j + 3, 3 * i:3 * i + 3] += C.T
            A[3 * i + 2, 3 * i + 2] -= 2.0 * model.K
            b[3 * i + 2] -= model.muB
    return A, b


def flat(x: np.ndarray) -> np.ndarray:
    """(3, L2, L1) -> flat vector with index 3*site + component."""
    return np.ascontiguousarray(np.moveaxis(x, 0, -1)).reshape(-1)


def unflat(x: np.ndarray, L1: int, L2: int) -> np.ndarray:
    return np.moveaxis(x.reshape(L2, L1, 3), -1, 0).copy()


def tangent_frame(m: np.ndarray) -> np.ndarray:
    """Per-spin orthonormal tangent basis, shape (N, 3, 2): e1 by Gram-Schmidt of
    x (or y where m is close to x), e2 = m x e1."""
    mf = flat(m).reshape(-1, 3)
    out = np.empty((mf.shape[0], 3, 2))
    for i, mi in enumerate(mf):
        ref = np.array([1.0, 0.0, 0.0]) if abs(mi[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        e1 = ref - np.dot(ref, mi) * mi
        e1 /= np.linalg.norm(e1)
        e2 = np.cross(mi, e1)
        out[i, :, 0] = e1
        out[i, :, 1] = e2
    return out


def dense_tangent_hessian(model: Model, m: np.ndarray):
    """(Ht, B): the 2N x 2N Riemannian Hessian in the tangent frame,
    Ht = B^T A B - diag(s), and the 3N x 2N frame matrix B."""
    A, b = dense_euclid_hessian(model)
    mflat = flat(m)
    ge = A @ mflat + b
    s = np.einsum("ij,ij->i", mflat.reshape(-1, 3), ge.reshape(-1, 3))
    fr = tangent_frame(m)
    N = model.N
    B = np.zeros((3 * N, 2 * N))
    for i in range(N):
        B[3 * i:3 * i + 3, 2 * i:2 * i + 2] = fr[i]
    Ht = B.T @ A @ B - np.diag(np.repeat(s, 2))
    return 0.5 * (Ht + Ht.T), B
