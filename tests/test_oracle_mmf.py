"""Pins of the oracle's outer layer: the L-BFGS two-loop against the explicit
BFGS inverse-Hessian update, the reflection, and the end points of ascent and
descent against the dense spectrum (index-1 saddle, index-0 minima)."""
import math

import numpy as np
import pytest

import inputs
from oracle import krylov, mmf, spin, topo
from oracle.model import Model


def vdot(a, b):
    return float(np.dot(a.ravel(), b.ravel()))


def test_two_loop_equals_explicit_bfgs_matrix():
    # vectors with zero z component are tangent at the +z ferromagnet, so the
    # tangent projection inside the optimiser is the identity here
    L = 6
    m = inputs.ferromagnet(L, L)
    n = L * L
    rng = inputs.normal(3, 9 * 3 * n).reshape(9, 3, L, L)
    rng[:, 2] = 0.0
    opt = mmf.LBFGS(mem=3, gamma0=0.5, theta_max=1e9)
    # feed steps with positive curvature: y = A s for an SPD A on the xy plane
    Adiag = 1.0 + np.arange(2 * n, dtype=float).reshape(2, L, L) / n
    S, Y = [], []
    G = rng[0].copy()
    opt.direction(m, G)
    for k in range(1, 5):
        s = opt.d_prev.copy()
        Gn = G.copy()
        Gn[:2] = G[:2] + Adiag * s[:2]
        S.append(s)
        Y.append(Gn - G)
        G = Gn
        d = opt.direction(m, G)
        Sk, Yk = S[-3:], Y[-3:]
        Hm = (vdot(Sk[-1], Yk[-1]) / vdot(Yk[-1], Yk[-1])) * np.eye(3 * n)
        for s_, y_ in zip(Sk, Yk):
            sf, yf = s_.ravel(), y_.ravel()
            rho = 1.0 / (yf @ sf)
            V = np.eye(3 * n) - rho * np.outer(yf, sf)
            Hm = V.T @ Hm @ V + rho * np.outer(sf, sf)
        np.testing.assert_allclose(d.ravel(), -Hm @ G.ravel(), rtol=1e-10, atol=1e-12)


def test_reflection_inverts_the_mode_component():
    F = inputs.gaussian_field(1, 5, 5)
    v = inputs.gaussian_field(2, 5, 5)
    v /= math.sqrt(vdot(v, v))
    Fm = mmf.reflected_force(F, v)
    assert vdot(Fm, v) == pytest.approx(-vdot(F, v), rel=1e-13)
    perp = F - vdot(F, v) * v
    np.testing.assert_allclose(Fm + vdot(F, v) * v, perp, atol=1e-13)


def test_step_cap_limits_rotation():
    m = inputs.add_noise(inputs.ferromagnet(6, 6), 0.3, 5)
    G = 50.0 * spin.project(m, inputs.gaussian_field(6, 6, 6))
    opt = mmf.LBFGS(mem=5, gamma0=0.02, theta_max=0.2)
    d = opt.direction(m, G)
    assert mmf.max_torque(d) == pytest.approx(0.2, rel=1e-14)
    assert vdot(d, G) < 0


@pytest.fixture(scope="module")
def config1_run():
    p = inputs.WORKLOADS[1]
    M = Model(p["L1"], p["L2"], J=p["J"], D=p["D"], K=p["K"], muB=p["muB"])
    m0 = inputs.workload1_state()
    q0 = inputs.gaussian_field(inputs.workload_seed(1, 0), 32, 32, offset=10**6)
    P = mmf.MMFParams()
    res = mmf.ascend(M, m0, [q0], P)
    return M, P, res


@pytest.mark.slow
def test_config1_ascent_reaches_an_index1_saddle(config1_run):
    M, P, res = config1_run
    assert res.converged
    g, s = spin.riemann_grad(M, res.m)
    assert mmf.max_torque(g) <= 2 * P.tau_F
    Ht, _ = spin.dense_tangent_hessian(M, res.m)
    w = np.linalg.eigvalsh(Ht)
    assert w[0] < 0.0 < w[1]
    assert res.lam[0] == pytest.approx(w[0], abs=1e-7)


@pytest.mark.slow
def test_config1_descent_reaches_two_minima(config1_run):
    M, P, res = config1_run
    plus, minus = mmf.descend(M, res.m, res.v1, P)
    seeds = mmf.descent_seeds(res.m, res.v1, P)
    for r, seed in zip((plus, minus), seeds):
        assert r.converged
        # relaxation never ends above its seed (the saddle itself is only
        # resolved to tau_F, so its energy is no sharp bound on this flat path)
        assert r.E <= spin.energy(M, seed) + 1e-9
        g, _ = spin.riemann_grad(M, r.m)
        assert mmf.max_torque(g) <= P.tau_F
        assert abs(r.Q - r.Qint) < 1e-9
        # the skyrmion's translation mode is nearly flat (curvature ~1e-5 meV),
        # so at force resolution tau_F the end point is a minimum only up to a
        # curvature of that order
        Ht, _ = spin.dense_tangent_hessian(M, r.m)
        assert np.linalg.eigvalsh(Ht)[0] > -1e-4
