"""Pins of the oracle's eigensolvers: known spectra, the dense explicit Hessian
(the paper's own accuracy protocol: cosine similarity of the minimum mode with
the explicit-Hessian eigenvector), and agreement between solvers."""
import math

import numpy as np
import pytest

import inputs
from oracle import krylov, spin
from oracle.model import Model

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


def vdot(a, b):
    return float(np.dot(a.ravel(), b.ravel()))


def test_lanczos_diagonal_operator_exact_spectrum():
    n = 40
    d = np.linspace(-1.0, 3.0, n) ** 3
    op = lambda v: d * v
    q0 = inputs.normal(5, n)
    theta, Y, Q = krylov.lanczos(op, q0, n)
    np.testing.assert_allclose(theta, np.sort(d), atol=1e-12)
    np.testing.assert_allclose(Q @ Q.T, np.eye(Q.shape[0]), atol=1e-13)


def test_lanczos_breakdown_on_invariant_subspace():
    d = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    q0 = np.array([1.0, 1.0, 0.0, 0.0, 0.0, 0.0])
    theta, Y, Q = krylov.lanczos(lambda v: d * v, q0, 6)
    assert Q.shape[0] == 2
    np.testing.assert_allclose(theta, [1.0, 2.0], atol=1e-14)


def test_block_lanczos_with_block_size_one_is_lanczos():
    n = 50
    rng = inputs.normal(9, n * n).reshape(n, n)
    A = rng + rng.T
    q0 = inputs.normal(10, n)
    t1, _, _ = krylov.lanczos(lambda v: A @ v, q0, 20)
    t2, _, _ = krylov.block_lanczos(lambda B: B @ A.T, q0.reshape(1, -1), 20)
    np.testing.assert_allclose(t1, t2, atol=1e-11)


def test_block_lanczos_full_space_recovers_spectrum():
    n = 48
    rng = inputs.normal(19, n * n).reshape(n, n)
    A = rng + rng.T
    X0 = inputs.normal(20, 4 * n).reshape(4, n)
    theta, Y, Q = krylov.block_lanczos(lambda B: B @ A.T, X0, n // 4)
    np.testing.assert_allclose(theta, np.linalg.eigvalsh(A), atol=1e-10)
    np.testing.assert_allclose(Q @ Q.T, np.eye(n), atol=1e-12)


def test_lobpcg_diagonal_operator():
    n = 300
    d = np.arange(1, n + 1, dtype=float) ** 1.5
    theta, X, it, conv = krylov.lobpcg(lambda B: B * d[None], inputs.normal(3, 4 * n).reshape(4, n), tol=1e-10, max_iter=1000)
    assert conv
    np.testing.assert_allclose(theta, d[:4], rtol=1e-12)


def small_state(L1=6, L2=6, seed=101):
    m = inputs.add_noise(inputs.skyrmion(L1, L2, 1.5), 0.3, seed)
    return m


@pytest.mark.parametrize("L1,L2", [(6, 6), (7, 5)])
def test_min_mode_matches_explicit_hessian(L1, L2):
    M = Model(L1, L2, **FULL)
    m = small_state(L1, L2)
    _, s = spin.riemann_grad(M, m)
    Ht, B = spin.dense_tangent_hessian(M, m)
    w, U = np.linalg.eigh(Ht)
    n = 2 * L1 * L2
    q0 = inputs.gaussian_field(1, L1, L2)
    lam, V = krylov.lanczos_modes(M, m, s, q0, n, k=1)
    assert lam[0] == pytest.approx(w[0], abs=1e-10)
    assert lam[1] == pytest.approx(w[1], abs=1e-10)
    vdense = spin.unflat(B @ U[:, 0], L1, L2)
    assert abs(vdot(V[0], vdense)) == pytest.approx(1.0, abs=1e-10)
    # LOBPCG with k = 3
    X0 = [inputs.gaussian_field(2 + j, L1, L2) for j in range(3)]
    th, VV, it, conv = krylov.lobpcg_modes(M, m, s, X0, 3, tol=1e-9, max_iter=500)
    assert conv
    np.testing.assert_allclose(th, w[:3], atol=1e-9)
    # block Lanczos with b = 3 over the whole space
    th2, VB = krylov.block_lanczos_modes(M, m, s, X0, n // 3 + 1, 3)
    np.testing.assert_allclose(th2[:3], w[:3], atol=1e-9)
    for v in VV + VB + V:
        assert np.max(np.abs(np.sum(v * m, axis=0))) < 1e-12
        assert vdot(v, v) == pytest.approx(1.0, abs=1e-12)


def test_ritz_sign_rule():
    v = np.zeros((3, 5, 5))
    v[1, 2, 3] = -0.9
    v[0, 0, 0] = 0.3
    assert krylov.fix_sign(v)[1, 2, 3] > 0
    w = np.zeros((3, 5, 5))
    w[0, 1, 1] = -0.5
    w[2, 4, 4] = 0.5
    assert krylov.fix_sign(w)[0, 1, 1] > 0  # tie -> lowest flat index decides


def test_lanczos_and_lobpcg_agree_on_config1_state():
    p = inputs.WORKLOADS[1]
    M = Model(p["L1"], p["L2"], J=p["J"], D=p["D"], K=p["K"], muB=p["muB"])
    m = inputs.workload1_state()
    _, s = spin.riemann_grad(M, m)
    lam, V = krylov.lanczos_modes(M, m, s, inputs.gaussian_field(7, 32, 32), 200, k=1)
    th, VV, it, conv = krylov.lobpcg_modes(M, m, s, [inputs.gaussian_field(8 + j, 32, 32) for j in range(2)], 2, tol=1e-8, max_iter=400)
    assert conv
    assert th[0] == pytest.approx(lam[0], rel=1e-6)
    assert abs(vdot(V[0], VV[0])) == pytest.approx(1.0, abs=1e-6)


def _block_with_dependent_row(rel: float):
    """Four rows: three independent ones, and a fourth that is a combination
    of them plus a new direction of relative size ``rel`` (the sine of its
    angle to the span of the others)."""
    n = 300
    W = np.stack([inputs.normal(40 + j, n) for j in range(3)])
    comb = 0.7 * W[0] - 1.3 * W[1] + 0.4 * W[2]
    Qo, _ = np.linalg.qr(W.T)
    new = inputs.normal(50, n)
    new = new - Qo @ (Qo.T @ new)
    new *= rel * np.linalg.norm(comb) / np.linalg.norm(new)
    return np.vstack([W, comb + new])


def test_cholqr2_rank_rule():
    """The rank rule of Cholesky QR applied twice (reading R4): a row whose new
    direction is below 1e-6 of its length makes cholqr2 report a dependent
    block, since then the condition number of the block is at least 1e6,
    within two orders of magnitude of the u^(-1/2) ~ 1e8 beyond which CholQR2
    no longer delivers an orthonormal factor (Yamamoto, Nakatsukasa,
    Yanagisawa & Fukaya 2015).  Above it, the factor is orthonormal to FP64
    rounding and reproduces the block."""
    assert krylov.cholqr2(_block_with_dependent_row(1e-7)) is None
    W = _block_with_dependent_row(1e-5)
    res = krylov.cholqr2(W)
    assert res is not None
    Q, R = res
    assert np.linalg.norm(Q @ Q.T - np.eye(4)) <= 1e-12
    assert np.linalg.norm(W - R.T @ Q) <= 1e-12 * np.linalg.norm(W)
    # the rule reads the fourth diagonal of the factor: the relative new
    # direction itself
    L = np.linalg.cholesky(W @ W.T)
    assert L[3, 3] / np.linalg.norm(W[3]) == pytest.approx(1e-5, rel=1e-3)
