"""Pins of the oracle's energy, gradients and tangent Hessian against closed
forms, finite differences, invariants and an explicit term-by-term Hessian."""
import math

import numpy as np
import pytest

import inputs
from oracle import spin
from oracle.model import SHELLS, Model

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


def rand_spins(L1, L2, seed):
    m = inputs.gaussian_field(seed, L1, L2)
    return m / np.sqrt(np.sum(m * m, axis=0))[None]


def rand_tangent(m, seed):
    L2, L1 = m.shape[1:]
    return spin.project(m, inputs.gaussian_field(seed, L1, L2, offset=10**5))


def vdot(a, b):
    return float(np.dot(a.ravel(), b.ravel()))


@pytest.mark.parametrize("L1,L2", [(5, 5), (6, 7)])
def test_energy_equals_dense_quadratic_form(L1, L2):
    M = Model(L1, L2, **FULL)
    m = rand_spins(L1, L2, 11)
    A, b = spin.dense_euclid_hessian(M)
    x = spin.flat(m)
    assert spin.energy(M, m) == pytest.approx(0.5 * x @ A @ x + b @ x, rel=1e-13, abs=1e-12)
    ge = spin.flat(spin.euclid_grad(M, m))
    np.testing.assert_allclose(ge, A @ x + b, rtol=0, atol=1e-12)
    v = inputs.gaussian_field(5, L1, L2)
    np.testing.assert_allclose(spin.flat(spin.euclid_hvp(M, v)), A @ spin.flat(v), rtol=0, atol=1e-12)


def test_gradient_central_differences():
    # E is a polynomial of degree 2 in the unconstrained m: central differences
    # are exact up to rounding for any step.
    M = Model(8, 9, **FULL)
    m = rand_spins(8, 9, 3)
    ge = spin.euclid_grad(M, m)
    for k in range(4):
        u = inputs.gaussian_field(100 + k, 8, 9)
        h = 1e-3
        fd = (spin.energy(M, m + h * u) - spin.energy(M, m - h * u)) / (2 * h)
        assert vdot(ge, u) == pytest.approx(fd, rel=1e-9, abs=1e-8)
        sec = (spin.energy(M, m + h * u) - 2 * spin.energy(M, m) + spin.energy(M, m - h * u)) / h**2
        assert vdot(u, spin.euclid_hvp(M, u)) == pytest.approx(sec, rel=1e-5, abs=1e-5)


def test_gradient_each_component_small_lattice():
    M = Model(5, 6, **FULL)
    m = rand_spins(5, 6, 4)
    ge = spin.euclid_grad(M, m)
    h = 1e-4
    for c in range(3):
        for i2 in range(6):
            for i1 in range(5):
                e = np.zeros_like(m)
                e[c, i2, i1] = 1.0
                fd = (spin.energy(M, m + h * e) - spin.energy(M, m - h * e)) / (2 * h)
                assert ge[c, i2, i1] == pytest.approx(fd, abs=1e-8)


def test_riemannian_gradient_and_hvp_along_geodesics():
    M = Model(6, 6, **FULL)
    m = rand_spins(6, 6, 21)
    g, s = spin.riemann_grad(M, m)
    for k in range(3):
        v = rand_tangent(m, 30 + k)
        v /= math.sqrt(vdot(v, v))
        h = 2e-2
        f = {j: spin.energy(M, spin.retract(m, j * h * v)) for j in (-2, -1, 0, 1, 2)}
        d1 = (f[-2] - 8 * f[-1] + 8 * f[1] - f[2]) / (12 * h)
        d2 = (-f[2] + 16 * f[1] - 30 * f[0] + 16 * f[-1] - f[-2]) / (12 * h * h)
        assert vdot(g, v) == pytest.approx(d1, rel=1e-6, abs=1e-6)
        assert vdot(v, spin.hvp(M, m, s, v)) == pytest.approx(d2, rel=1e-5, abs=1e-5)
    # g is tangent
    assert np.max(np.abs(np.sum(g * m, axis=0))) < 1e-12


def test_hvp_symmetric_on_tangent_vectors():
    M = Model(16, 12, **FULL)
    m = rand_spins(16, 12, 7)
    _, s = spin.riemann_grad(M, m)
    u = rand_tangent(m, 8)
    v = rand_tangent(m, 9)
    a = vdot(u, spin.hvp(M, m, s, v))
    b = vdot(v, spin.hvp(M, m, s, u))
    assert a == pytest.approx(b, rel=1e-12)
    # output is tangent
    hv = spin.hvp(M, m, s, v)
    assert np.max(np.abs(np.sum(hv * m, axis=0))) < 1e-12


def test_hvp_equals_dense_tangent_hessian():
    M = Model(5, 7, **FULL)
    m = rand_spins(5, 7, 12)
    _, s = spin.riemann_grad(M, m)
    Ht, B = spin.dense_tangent_hessian(M, m)
    v = rand_tangent(m, 13)
    c = B.T @ spin.flat(v)
    np.testing.assert_allclose(B.T @ spin.flat(spin.hvp(M, m, s, v)), Ht @ c, atol=1e-11)


def spin_wave_eigs(L1, L2, J, K, muB):
    out = []
    for n2 in range(L2):
        for n1 in range(L1):
            lam = muB + 2 * K
            for Js, shell in zip(J, SHELLS):
                for d1, d2 in shell:
                    lam += 2 * Js * (1 - math.cos(2 * math.pi * (n1 * d1 / L1 + n2 * d2 / L2)))
            out += [lam, lam]
    return np.sort(np.array(out))


@pytest.mark.parametrize("L1,L2", [(5, 5), (6, 6), (7, 5)])
def test_ferromagnet_spin_wave_spectrum(L1, L2):
    M = Model(L1, L2, **FULL)
    m = inputs.ferromagnet(L1, L2)
    Ht, _ = spin.dense_tangent_hessian(M, m)
    np.testing.assert_allclose(np.linalg.eigvalsh(Ht), spin_wave_eigs(L1, L2, M.J, M.K, M.muB), atol=1e-11)
    N = L1 * L2
    assert spin.energy(M, m) == pytest.approx(-N * (6 * sum(M.J) + M.muB + M.K), rel=1e-14)


def test_plane_waves_are_hvp_eigenvectors():
    L = 32
    M = Model(L, L, **FULL)
    m = inputs.ferromagnet(L, L)
    _, s = spin.riemann_grad(M, m)
    i2, i1 = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    for n1, n2 in [(0, 0), (1, 0), (3, 5), (16, 7)]:
        ph = 2 * math.pi * (n1 * i1 + n2 * i2) / L
        lam = M.muB + 2 * M.K
        for Js, shell in zip(M.J, SHELLS):
            for d1, d2 in shell:
                lam += 2 * Js * (1 - math.cos(2 * math.pi * (n1 * d1 + n2 * d2) / L))
        for comp in (0, 1):
            v = np.zeros_like(m)
            v[comp] = np.cos(ph)
            np.testing.assert_allclose(spin.hvp(M, m, s, v), lam * v, atol=1e-12)


def cycloid(L, n1, n2):
    """sin(q.r) q_hat + cos(q.r) z with q.r_i = 2 pi (n1 i1 + n2 i2) / L."""
    # q = (2 pi / L)(n1 b1 + n2 b2), b1 = (1, -1/sqrt3), b2 = (0, 2/sqrt3)
    qx = 2 * math.pi / L * n1
    qy = 2 * math.pi / L * (-n1 / math.sqrt(3) + 2 * n2 / math.sqrt(3))
    qn = math.hypot(qx, qy)
    i2, i1 = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    ph = 2 * math.pi * (n1 * i1 + n2 * i2) / L
    m = np.stack([np.sin(ph) * qx / qn, np.sin(ph) * qy / qn, np.cos(ph)])
    return m, (qx / qn, qy / qn)


@pytest.mark.parametrize("n1,n2", [(1, 0), (2, 1), (3, -1)])
def test_neel_cycloid_energy_closed_form(n1, n2):
    L = 24
    M = Model(L, L, **FULL)
    m, qhat = cycloid(L, n1, n2)
    e = -M.K / 2
    for Js, shell in zip(M.J, SHELLS):
        for d1, d2 in shell:
            e -= Js * math.cos(2 * math.pi * (n1 * d1 + n2 * d2) / L)
    for d1, d2 in SHELLS[0]:
        dx, dy = d1 + 0.5 * d2, 0.5 * math.sqrt(3) * d2
        e -= M.D * math.sin(2 * math.pi * (n1 * d1 + n2 * d2) / L) * (dx * qhat[0] + dy * qhat[1])
    assert spin.energy(M, m) / (L * L) == pytest.approx(e, rel=1e-12, abs=1e-12)


def test_mirror_cycloid_is_stationary():
    L = 24
    M = Model(L, L, J=FULL["J"], D=FULL["D"], K=0.0, muB=0.0)
    m, _ = cycloid(L, 2, 0)
    g, _ = spin.riemann_grad(M, m)
    assert np.max(np.abs(g)) < 1e-12
    # the favoured rotation sense lowers the energy below the opposite one
    mr = m.copy()
    mr[:2] *= -1
    assert spin.energy(M, m) < spin.energy(M, mr)


def test_translation_and_c6_invariance():
    L = 12
    M = Model(L, L, **FULL)
    m = rand_spins(L, L, 40)
    E = spin.energy(M, m)
    assert spin.energy(M, np.roll(m, (3, -5), axis=(1, 2))) == pytest.approx(E, rel=1e-13)
    # rotate sites and spins by 60 degrees: (i1, i2) -> (-i2, i1 + i2)
    c, s_ = 0.5, math.sqrt(3) / 2
    rot = np.empty_like(m)
    for i2 in range(L):
        for i1 in range(L):
            j1, j2 = (-i2) % L, (i1 + i2) % L
            x, y, z = m[:, i2, i1]
            rot[:, j2, j1] = (c * x - s_ * y, s_ * x + c * y, z)
    assert spin.energy(M, rot) == pytest.approx(E, rel=1e-13)
    g = spin.euclid_grad(M, m)
    gr = spin.euclid_grad(M, rot)
    for i2 in range(L):
        for i1 in range(L):
            j1, j2 = (-i2) % L, (i1 + i2) % L
            x, y, z = g[:, i2, i1]
            np.testing.assert_allclose(gr[:, j2, j1], (c * x - s_ * y, s_ * x + c * y, z), atol=1e-12)


def test_helicity_pi_is_favoured():
    M = Model(32, 32, J=(1.0,), D=0.3, K=0.05, muB=0.02)
    assert spin.energy(M, inputs.skyrmion(32, 32, 4.0)) < spin.energy(M, inputs.skyrmion(32, 32, 4.0, helicity=0.0))


def test_retraction_is_rotation():
    m = rand_spins(6, 6, 50)
    d = rand_tangent(m, 51) * 0.3
    r = spin.retract(m, d)
    np.testing.assert_allclose(np.sum(r * r, axis=0), 1.0, atol=1e-15)
    th = np.sqrt(np.sum(d * d, axis=0))
    np.testing.assert_allclose(np.sum(r * m, axis=0), np.cos(th), atol=1e-14)
