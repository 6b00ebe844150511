"""GPU parity of the explorer front-end: masked perturbations against the
oracle (inactive sites bit-equal to x0), pairwise L1 distances against the
oracle at sizes from one partial tile to many blocks and population sizes 2
to MOTO_MAX_POP, and the three objectives of a perturbed population
(diversity from the distances, charge violation, spectral gap) against the
oracle's, the gap pinned by the dense tangent spectrum."""
import numpy as np
import pytest
import torch

import inputs
from oracle import explorer, spin, topo
from oracle.model import Model
from gpu_util import context, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


def _disk_mask(L1, L2, r):
    i2, i1 = np.mgrid[0:L2, 0:L1]
    return ((i1 - L1 / 2) ** 2 + (i2 - L2 / 2) ** 2 <= r * r).astype(np.uint8)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-14), (torch.float32, 2e-6)])
@pytest.mark.parametrize("L1,L2", [(12, 12), (37, 29)])
def test_perturbation_matches_the_oracle(dtype, tol, L1, L2):
    require_gpu()
    ctx = context(Model(L1, L2, **FULL), dtype)
    x0 = inputs.skyrmion(L1, L2, 3.0)
    mask = _disk_mask(L1, L2, min(L1, L2) / 3)
    deltas = np.stack([0.4 * inputs.gaussian_field(700 + j, L1, L2) for j in range(5)])
    # both sides start from the same (rounded) inputs
    x0_in = to_np(to_dev(x0, dtype))
    d_in = to_np(to_dev(deltas, dtype))
    out = to_np(ctx.perturb(to_dev(x0, dtype), to_dev(deltas, dtype).contiguous(),
                            torch.from_numpy(mask).cuda()))
    for j in range(5):
        ref = explorer.masked_perturbation(x0_in, mask, d_in[j])
        assert np.max(np.abs(out[j] - ref)) <= tol
        assert np.array_equal(out[j][:, mask == 0], x0_in[:, mask == 0])
    # no mask: every site moves
    out = to_np(ctx.perturb(to_dev(x0, dtype), to_dev(deltas[:1], dtype).contiguous()))
    ref = explorer.masked_perturbation(x0_in, np.ones((L2, L1), np.uint8), d_in[0])
    assert np.max(np.abs(out[0] - ref)) <= tol
    ctx.close()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("L1,L2,P", [(7, 6, 2), (37, 29, 3), (64, 64, 24), (256, 256, 24), (48, 40, 64)])
def test_pairwise_l1_matches_the_oracle(dtype, tol, L1, L2, P):
    require_gpu()
    ctx = context(Model(L1, L2, **FULL), dtype)
    X = np.stack([inputs.gaussian_field(900 + j, L1, L2) for j in range(P)])
    Xd = to_dev(X, dtype).contiguous()
    D = to_np(ctx.pairwise_l1(Xd))
    ref = explorer.pairwise_l1(list(to_np(Xd)))
    scale = np.maximum(ref, 1.0)
    assert np.max(np.abs(D - ref) / scale) <= tol
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0.0)
    ctx.close()


def test_population_objectives_match_the_oracle():
    require_gpu()
    L = 12
    M = Model(L, L, **FULL)
    ctx = context(M, torch.float64)
    x0 = inputs.skyrmion(L, L, 2.5)
    mask = _disk_mask(L, L, 4.0)
    deltas = np.stack([0.3 * inputs.gaussian_field(1100 + j, L, L) for j in range(6)])
    Xg = ctx.perturb(to_dev(x0, torch.float64), to_dev(deltas, torch.float64).contiguous(),
                     torch.from_numpy(mask).cuda())
    X = to_np(Xg)
    D = to_np(ctx.pairwise_l1(Xg))
    d_gpu = explorer.diversity(D)
    lams = []
    for j in range(6):
        starts = np.stack([inputs.gaussian_field(1200 + 2 * j + q, L, L) for q in range(2)])
        lam, V, info = ctx.lowest_modes(Xg[j].contiguous(), to_dev(starts, torch.float64).contiguous(),
                                        k=2, block=2, krylov_steps=40)
        lam = to_np(lam)
        lams.append((lam[0], lam[1]))
        w = np.linalg.eigvalsh(spin.dense_tangent_hessian(M, X[j])[0])
        assert lam[0] == pytest.approx(w[0], abs=1e-8) and lam[1] == pytest.approx(w[1], abs=1e-8)
    Q = [float(to_np(ctx.topo_charge(Xg[j].contiguous()))[0]) for j in range(6)]
    d, v, s = explorer.objectives(list(X), 1.0, lams)
    np.testing.assert_allclose(d_gpu, d, rtol=1e-12)
    np.testing.assert_allclose([explorer.feasibility(q, 1.0) for q in Q], v, atol=1e-12)
    np.testing.assert_allclose([explorer.separability(a, b) for a, b in lams], s, rtol=1e-15)
    ctx.close()
