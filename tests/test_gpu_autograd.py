"""GPU parity of the autograd.Function (energy -> grad E -> hess E v) against
the oracle, plus identities that hold at any size.

Bars: FP64 energies to 1e-12 relative, gradients and Hessian products to 1e-12
of the field's norm; FP32 fields (energies still in double arithmetic) to
1e-6 of the norm (rounding of the stored inputs and outputs)."""
import numpy as np
import pytest
import torch

import inputs
from oracle import spin
from oracle.model import Model
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


def _energy():
    from paper_2509_26269_gb300 import energy
    return energy


def rel(a, b):
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_energy_grad_hvp_match_oracle_workload5(dtype):
    require_gpu()
    M = workload_model(5)
    m_np = inputs.workload5_state()
    ctx = context(M, dtype)
    m = to_dev(m_np, dtype).requires_grad_(True)
    E = _energy()(m, ctx)
    assert E.dtype == torch.float64
    mo = to_np(m)  # the stored (possibly rounded) spins
    E_ref = spin.energy(M, mo)
    assert float(E.detach()) == pytest.approx(E_ref, rel=1e-12)
    (g,) = torch.autograd.grad(E, m, create_graph=True)
    tol = 1e-12 if dtype == torch.float64 else 1e-6
    assert rel(to_np(g), spin.euclid_grad(M, mo)) < tol
    for k in range(3):
        v_np = inputs.gaussian_field(inputs.workload_seed(5, 100 + k), M.L1, M.L2)
        v = to_dev(v_np, dtype)
        (hv,) = torch.autograd.grad(g, m, v, retain_graph=True)
        assert rel(to_np(hv), spin.euclid_hvp(M, to_np(v))) < tol
    ctx.close()


def test_fd_identities_of_the_quadratic_energy_10000_directions():
    """E is a polynomial of degree 2, so along any v
         E(m + h v) - E(m - h v) = 2 h grad E . v,
         E(m + h v) - 2 E(m) + E(m - h v) = h^2 v . hess E v
    hold up to rounding for every h (no truncation error), so h is chosen to
    keep the rounding of E (|E| ~ 1e6 meV, ~1e-7 absolute in double) small
    against both sides.  10,000 seeded directions at 512 x 512 (FP64), the
    energies from the forward kernel, the derivatives from the backward and
    double-backward kernels."""
    require_gpu()
    M = workload_model(5)
    ctx = context(M, torch.float64)
    m = to_dev(inputs.workload5_state(), torch.float64).requires_grad_(True)
    energy = _energy()
    E0 = energy(m, ctx)
    (g,) = torch.autograd.grad(E0, m, create_graph=True)
    gen = torch.Generator(device="cuda").manual_seed(inputs.workload_seed(5, 1))
    h = 0.05
    err1, err2 = [], []
    for _ in range(10000):
        v = torch.randn(m.shape, dtype=torch.float64, device="cuda", generator=gen)
        with torch.no_grad():
            Ep = energy(m + h * v, ctx)
            Em = energy(m - h * v, ctx)
        (hv,) = torch.autograd.grad(g, m, v, retain_graph=True)
        with torch.no_grad():
            gv = (g * v).sum()
            vhv = (v * hv).sum()
            err1.append(((Ep - Em) / (2 * h) - gv).abs() / (gv.abs() + 1.0))
            err2.append(((Ep - 2 * E0 + Em) / (h * h) - vhv).abs() / (vhv.abs() + 1.0))
    # rounding of E ~1e-7: the first difference is good to ~3e-6 against
    # |g.v| ~ 1e3-1e4, the second to ~2e-4 against |v.Hv| ~ 1e7
    assert float(torch.stack(err1).max()) < 1e-8
    assert float(torch.stack(err2).max()) < 1e-8
    ctx.close()


def test_gradcheck_and_gradgradcheck_on_a_small_lattice():
    require_gpu()
    M = Model(6, 5, **FULL)
    ctx = context(M, torch.float64)
    m = to_dev(inputs.add_noise(inputs.skyrmion(6, 5, 1.5), 0.2, 7), torch.float64).requires_grad_(True)
    f = lambda x: _energy()(x, ctx)
    assert torch.autograd.gradcheck(f, (m,), eps=1e-6, atol=1e-6, rtol=1e-6)
    assert torch.autograd.gradgradcheck(f, (m,), eps=1e-6, atol=1e-6, rtol=1e-6)
    ctx.close()


def test_third_derivative_vanishes_and_hessian_is_symmetric():
    require_gpu()
    M = Model(7, 6, **FULL)
    ctx = context(M, torch.float64)
    m = to_dev(inputs.add_noise(inputs.skyrmion(7, 6, 1.5), 0.2, 8), torch.float64).requires_grad_(True)
    u = to_dev(inputs.gaussian_field(11, 7, 6), torch.float64)
    v = to_dev(inputs.gaussian_field(12, 7, 6), torch.float64)
    E = _energy()(m, ctx)
    (g,) = torch.autograd.grad(E, m, create_graph=True)
    (hv,) = torch.autograd.grad(g, m, v, create_graph=True)
    (hu,) = torch.autograd.grad(g, m, u, retain_graph=True)
    assert float((u * hv).sum()) == pytest.approx(float((v * hu).sum()), rel=1e-12)
    # d/dm (u . hess E v) = 0: hess E does not depend on m, so the product
    # carries no graph back to m
    if hv.requires_grad:
        third = torch.autograd.grad((u * hv).sum(), m, allow_unused=True)[0]
        assert third is None or float(third.abs().max()) == 0.0
    ctx.close()
