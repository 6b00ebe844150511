"""Krylov eigensolvers for the k smallest tangent eigenpairs (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The inner layer of the bilayer MMF kernel finds the k smallest eigenpairs of
the tangent Hessian with HVP-driven Lanczos or LOBPCG in operator mode (Results,
"Bilayer MMF"; Methods, "HVP operator mode"; Supplementary Note 1, layer (ii)).
The paper calls library solvers and caps them at 200 iterations in its
benchmarks; it does not state the variant, so the oracle takes textbook forms:

* Lanczos (Lanczos 1950) with full reorthogonalisation by classical
  Gram-Schmidt applied twice after the three-term recurrence, a fixed number
  of steps, early stop on beta <= 1e-12 |T| (reading R4); the tridiagonal
  eigenproblem is solved by a library routine (``numpy.linalg.eigh``).
* Block Lanczos with block size b (Golub & Van Loan, sec. 10.3.6): the same
  recurrence on blocks, blocks orthonormalised by Cholesky QR applied twice.
  With b = 1 it is the Lanczos above.
* LOBPCG (Knyazev 2001): trial subspace [X, W, P] with W the residuals, a
  Rayleigh-Ritz step on it in FP64 made robust by SVQB orthonormalisation of the
  subspace (Stathopoulos & Wu 2002; reading R5), stopped when every residual
  |H x_j - theta_j x_j| <= tol * max|theta| of the subspace problem.

Ritz vectors are projected on the tangent bundle, normalised and signed so that
their entry of largest magnitude is positive, ties going to the lowest flat
index of the (3, L2, L1) layout (reading R4).

Vectors are (3, L2, L1) arrays; a block is a list of such arrays.
"""
from __future__ import annotations

import numpy as np

from . import spin


def _dot(a, b) -> float:
    return float(np.dot(a.ravel(), b.ravel()))


def fix_sign(v: np.ndarray) -> np.ndarray:
    flat = v.ravel()
    i = int(np.argmax(np.abs(flat)))  # first index among equal magnitudes
    return v if flat[i] >= 0.0 else -v


def finish_ritz(m: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Project on the tangent planes, normalise, fix the sign (R4)."""
    v = spin.project(m, v)
    v = v / np.sqrt(_dot(v, v))
    return fix_sign(v)


# ----------------------------------------------------------------------------
# Lanczos
# ----------------------------------------------------------------------------
def lanczos(op, q0: np.ndarray, nsteps: int, breakdown: float = 1e-12, proj=None):
    """Lanczos with full CGS2 reorthogonalisation.

    ``proj`` (optional) maps a vector onto the subspace the operator lives on;
    it is applied after the three-term recurrence, since a small beta would
    otherwise magnify rounding-level components outside that subspace.

    Returns (theta, Y, Q): Ritz values ascending, eigenvectors of T (columns),
    and the orthonormal Krylov basis as an (nq, n) matrix."""
    n = q0.size
    Q = np.zeros((nsteps, n))
    Q[0] = q0.ravel() / np.sqrt(_dot(q0, q0))
    alpha, beta = [], []
    tnorm = 0.0
    for j in range(nsteps):
        w = op(Q[j].reshape(q0.shape)).ravel()
        a = float(np.dot(Q[j], w))
        alpha.append(a)
        w = w - a * Q[j]
        if j > 0:
            w = w - beta[j - 1] * Q[j - 1]
        if proj is not None:
            w = proj(w.reshape(q0.shape)).ravel()
        for _ in range(2):
            c = Q[: j + 1] @ w
            w = w - Q[: j + 1].T @ c
        b = float(np.sqrt(np.dot(w, w)))
        tnorm = max(tnorm, abs(a) + b + (beta[j - 1] if j > 0 else 0.0))
        if j == nsteps - 1 or b <= breakdown * tnorm:
            break
        beta.append(b)
        Q[j + 1] = w / b
    nq = len(alpha)
    T = np.diag(alpha) + np.diag(beta[: nq - 1], 1) + np.diag(beta[: nq - 1], -1)
    theta, Y = np.linalg.eigh(T)
    return theta, Y, Q[:nq]


def lanczos_modes(model, m, s, q0, nsteps: int, k: int = 1):
    """k lowest tangent eigenpairs by Lanczos from start vector q0 (projected).

    Returns (lam, V): the nsteps-bounded Ritz values (all of them, ascending) and
    the first k finished Ritz vectors."""
    op = lambda v: spin.hvp(model, m, s, v)
    theta, Y, Q = lanczos(op, spin.project(m, q0), nsteps, proj=lambda v: spin.project(m, v))
    V = []
    for i in range(k):
        v = (Q.T @ Y[:, i]).reshape(m.shape)
        V.append(finish_ritz(m, v))
    return theta, V


# ----------------------------------------------------------------------------
# block Lanczos
# ----------------------------------------------------------------------------
def _chol_factor(W: np.ndarray):
    """Lower Cholesky factor of W W^T (rows of W are vectors), or None."""
    try:
        return np.linalg.cholesky(W @ W.T)
    except np.linalg.LinAlgError:
        return None


def _dependent(L, G) -> bool:
    """A column whose new direction is below 1e-6 of its own length."""
    return bool(np.any(np.diag(L) <= 1e-6 * np.sqrt(np.clip(np.diag(G), 0.0, None))))


def cholqr2(W: np.ndarray):
    """Cholesky QR applied twice: W = Q R with Q Q^T = I (rows are vectors).
    Returns (Q, R), or None when W is numerically rank deficient (a factor
    fails or a column keeps less than 1e-6 of its length)."""
    R = np.eye(W.shape[0])
    Qm = W
    for _ in range(2):
        G = Qm @ Qm.T
        Lc = _chol_factor(Qm)
        if Lc is None or _dependent(Lc, G):
            return None
        Qm = np.linalg.solve(Lc, Qm)          # L^{-1} W  (rows)
        R = Lc.T @ R
    return Qm, R


def block_lanczos(op_block, X0: np.ndarray, nsteps: int, breakdown: float = 1e-12, proj=None):
    """Block Lanczos with full CGS2 reorthogonalisation of each new block.

    op_block maps a (b, n) block to H applied row-wise.  Returns (theta, Y, Q)
    with Q the (b * steps, n) orthonormal basis and T = Q H Q^T block tridiagonal."""
    b = X0.shape[0]
    first = cholqr2(X0)
    if first is None:
        raise ValueError("start block is rank deficient")
    blocks = [first[0]]
    T = np.zeros((b * nsteps, b * nsteps))
    Rprev = None
    nb_used = 0
    tnorm = 0.0
    for j in range(nsteps):
        Qj = blocks[j]
        W = op_block(Qj)
        A = Qj @ W.T
        A = 0.5 * (A + A.T)
        T[j * b:(j + 1) * b, j * b:(j + 1) * b] = A
        nb_used = j + 1
        W = W - A.T @ Qj                       # W - Q_j A (rows)
        if j > 0:
            W = W - Rprev @ blocks[j - 1]      # W - Q_{j-1} R_j^T (rows)
        if proj is not None:
            W = proj(W)
        Qall = np.concatenate(blocks, axis=0)
        for _ in range(2):
            C = W @ Qall.T
            W = W - C @ Qall
        if j == nsteps - 1:
            break
        # Cholesky QR of the new block; breakdown when its smallest diagonal
        # is below rel * |T| (|T| estimated by the largest row sum seen, as for
        # beta_j <= 1e-12 |T| in the plain Lanczos above)
        L1 = _chol_factor(W)
        if L1 is None:
            break
        rows = np.abs(A).sum(axis=1) + (np.abs(Rprev).sum(axis=1) if Rprev is not None else 0.0)
        tnorm = max(tnorm, float(np.max(rows)) + float(np.max(np.diag(L1))))
        if np.min(np.diag(L1)) <= breakdown * tnorm:
            break
        Q1 = np.linalg.solve(L1, W)
        L2 = _chol_factor(Q1)
        if L2 is None or _dependent(L2, Q1 @ Q1.T):
            break
        Qn = np.linalg.solve(L2, Q1)
        Rn = L2.T @ L1.T
        T[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b] = Rn
        T[j * b:(j + 1) * b, (j + 1) * b:(j + 2) * b] = Rn.T
        blocks.append(Qn)
        Rprev = Rn
    nT = b * nb_used
    theta, Y = np.linalg.eigh(T[:nT, :nT])
    return theta, Y, np.concatenate(blocks[:nb_used], axis=0)


def block_lanczos_modes(model, m, s, X0_list, nsteps: int, k: int):
    shape = m.shape
    op_block = lambda B: np.stack([spin.hvp(model, m, s, r.reshape(shape)).ravel() for r in B])
    proj = lambda B: np.stack([spin.project(m, r.reshape(shape)).ravel() for r in B])
    X0 = np.stack([spin.project(m, x).ravel() for x in X0_list])
    theta, Y, Q = block_lanczos(op_block, X0, nsteps, proj=proj)
    V = [finish_ritz(m, (Q.T @ Y[:, i]).reshape(shape)) for i in range(k)]
    return theta, V


# ----------------------------------------------------------------------------
# LOBPCG
# ----------------------------------------------------------------------------
def svqb(G: np.ndarray, drop: float = 1e-12):
    """Stathopoulos-Wu SVQB: Z with Z^T G Z = I, dropping directions whose scaled
    Gram eigenvalue is below drop * largest."""
    d = np.sqrt(np.clip(np.diag(G), 1e-300, None))
    Dinv = 1.0 / d
    Gs = Dinv[:, None] * G * Dinv[None, :]
    w, U = np.linalg.eigh(Gs)
    keep = w > drop * w[-1]
    return (Dinv[:, None] * U[:, keep]) / np.sqrt(w[keep])[None, :]


def lobpcg(op_block, X0: np.ndarray, tol: float = 1e-6, max_iter: int = 200, drop: float = 1e-12, proj=None):
    """LOBPCG for the k lowest eigenpairs of a symmetric operator.

    X0: (k, n) start block.  ``proj`` (optional) maps a block onto the subspace
    the operator lives on; the residual block is projected before it is
    normalised, since normalising a small residual would otherwise magnify the
    rounding-level components outside that subspace every iteration.
    Returns (theta, X, iters, converged) with X (k, n)."""
    k = X0.shape[0]
    Z = svqb(X0 @ X0.T, drop)
    X = Z.T @ X0
    AX = op_block(X)
    M = X @ AX.T
    theta, C = np.linalg.eigh(0.5 * (M + M.T))
    X = C.T @ X
    AX = C.T @ AX
    P = AP = None
    it = 0
    converged = False
    hnorm = float(np.max(np.abs(theta)))
    for it in range(1, max_iter + 1):
        R = AX - theta[:, None] * X
        rn = np.sqrt(np.sum(R * R, axis=1))
        if np.all(rn <= tol * hnorm):
            converged = True
            it -= 1
            break
        # residual block, orthogonalised against X and orthonormalised, its
        # image computed afresh so that no large coefficient multiplies a
        # recurrence-updated block
        if proj is not None:
            R = proj(R)
        W = R - (R @ X.T) @ X
        qr = cholqr2(W)
        if qr is None:
            Zw = svqb(W @ W.T, drop)
            W = Zw.T @ W
        else:
            W = qr[0]
        AW = op_block(W)
        if P is not None:
            pn = np.sqrt(np.sum(P * P, axis=1))
            pn = np.where(pn > 0.0, pn, 1.0)
            P, AP = P / pn[:, None], AP / pn[:, None]
        S = [X, W] + ([P] if P is not None else [])
        AS = [AX, AW] + ([AP] if AP is not None else [])
        S = np.concatenate(S, axis=0)
        AS = np.concatenate(AS, axis=0)
        G = S @ S.T
        M = S @ AS.T
        M = 0.5 * (M + M.T)
        Z = svqb(G, drop)
        Mr = Z.T @ M @ Z
        w, U = np.linalg.eigh(0.5 * (Mr + Mr.T))
        hnorm = max(hnorm, float(np.max(np.abs(w))))
        Cx = Z @ U[:, :k]                 # (p, k)
        Cp = Cx.copy()
        Cp[:k] = 0.0                       # directions outside the old X
        X, AX = Cx.T @ S, Cx.T @ AS
        P, AP = Cp.T @ S, Cp.T @ AS
        theta = w[:k]
    return theta, X, it, converged


def lobpcg_modes(model, m, s, X0_list, k: int, tol: float = 1e-6, max_iter: int = 200):
    shape = m.shape
    op_block = lambda B: np.stack([spin.hvp(model, m, s, r.reshape(shape)).ravel() for r in B])
    proj = lambda B: np.stack([spin.project(m, r.reshape(shape)).ravel() for r in B])
    X0 = proj(np.stack([x.ravel() for x in X0_list[:k]]))
    theta, X, it, conv = lobpcg(op_block, X0, tol, max_iter, proj=proj)
    V = [finish_ritz(m, X[i].reshape(shape)) for i in range(k)]
    return theta, V, it, conv
