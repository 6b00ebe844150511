"""GPU parity of the general pair-list Hamiltonian: energy, Riemannian
gradient, tangent HVP and the Euclidean derivatives against the pair-list
oracle (FP64, FP32; ragged lattices, reach 3 and 8, and the paper's own
Pd/Fe/Ir(111) parameter tables: 360 ordered pairs out to reach 11 on a
100 x 100 lattice), the
shell model entered as a pair list matching the built-in stencils, and the
eigensolver running on a pair-list context against the dense spectrum."""
import numpy as np
import pytest
import torch

import inputs
from oracle import pairs, spin
from oracle.model import Model
from gpu_util import context, require_gpu, to_dev, to_np
import paper_2509_26269_gb300 as mo

pytestmark = pytest.mark.gpu

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


def _pair_ctx(L1, L2, pl, dtype, K=0.07, muB=0.03):
    ctx = context(Model(L1, L2, J=(1.0,), D=0.0, K=K, muB=muB), dtype)
    ctx.set_pairs(pl)
    return ctx, pairs.PairModel(L1, L2, pl, K=K, muB=muB)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
@pytest.mark.parametrize("L1,L2,reach,nofs", [(37, 29, 3, 12), (40, 36, 8, 40), (100, 100, 11, "paper")])
def test_pair_stencils_match_the_oracle(dtype, tol, L1, L2, reach, nofs):
    require_gpu()
    if nofs == "paper":
        # the Supplementary Note 4 tables (reading R23), K and muB at stated readings
        pl = inputs.pdfeir_pairs()
        assert len(pl) == 360 and max(max(abs(p[0]), abs(p[1])) for p in pl) == reach
    else:
        pl = inputs.random_pairs(300 + reach, reach=reach, n_offsets=nofs)
    ctx, pm = _pair_ctx(L1, L2, pl, dtype)
    m = inputs.add_noise(inputs.skyrmion(L1, L2, 4.0), 0.1, 310 + reach)
    md = to_dev(m, dtype)
    m_in = to_np(md)
    ge = pairs.euclid_grad(pm, m_in)
    scale = np.linalg.norm(ge)
    out, g, s = ctx.energy_grad(md)
    g_ref, s_ref = pairs.riemann_grad(pm, m_in)
    assert np.linalg.norm(to_np(g) - g_ref) / scale <= tol
    E = float(to_np(ctx.energy(md))[0])
    assert E == pytest.approx(pairs.energy(pm, m_in), rel=max(tol, 1e-12), abs=1e-9)
    V = np.stack([spin.project(m_in, inputs.gaussian_field(320 + j, L1, L2)) for j in range(3)])
    Vd = to_dev(V, dtype).contiguous()
    hv = to_np(ctx.hvp(md, s, Vd))
    s_in = to_np(s)
    for j in range(3):
        ref = pairs.hvp(pm, m_in, s_in, to_np(Vd[j]))
        assert np.linalg.norm(hv[j] - ref) / np.linalg.norm(pairs.euclid_hvp(pm, to_np(Vd[j]))) <= tol
    # Euclidean derivatives (the autograd entry points)
    gE = torch.empty_like(md)
    o2 = torch.empty(2, dtype=torch.float64, device="cuda")
    mo.moto_energy_euclid_grad(ctx.handle, md, gE, o2)
    assert np.linalg.norm(to_np(gE) - ge) / scale <= tol
    hE = torch.empty_like(Vd)
    mo.moto_euclid_hvp(ctx.handle, Vd, 3 * L1 * L2, hE, 3 * L1 * L2, 3)
    for j in range(3):
        ref = pairs.euclid_hvp(pm, to_np(Vd[j]))
        assert np.linalg.norm(to_np(hE[j]) - ref) / np.linalg.norm(ref) <= tol
    ctx.close()


def test_shell_model_as_pairs_matches_the_builtin_stencils():
    require_gpu()
    L1, L2 = 33, 27
    M = Model(L1, L2, **FULL)
    pl = pairs.pairs_from_model(M)
    a = context(M, torch.float64)
    b, _ = _pair_ctx(L1, L2, pl, torch.float64, K=M.K, muB=M.muB)
    m = to_dev(inputs.add_noise(inputs.skyrmion(L1, L2, 3.0), 0.1, 5), torch.float64)
    oa, ga, sa = a.energy_grad(m)
    ob, gb, sb = b.energy_grad(m)
    assert float(oa[0]) == pytest.approx(float(ob[0]), rel=1e-13)
    assert np.max(np.abs(to_np(ga) - to_np(gb))) <= 1e-12
    v = to_dev(inputs.gaussian_field(6, L1, L2), torch.float64)
    assert np.max(np.abs(to_np(a.hvp(m, sa, v)) - to_np(b.hvp(m, sb, v)))) <= 1e-12
    b.set_pairs([])  # back to the context's own shell model (J = (1,), no DMI)
    c = context(Model(L1, L2, J=(1.0,), D=0.0, K=M.K, muB=M.muB), torch.float64)
    ob2, gb2, _ = b.energy_grad(m)
    oc, gc, _ = c.energy_grad(m)
    assert float(ob2[0]) == float(oc[0]) and torch.equal(gb2, gc)
    a.close()
    b.close()
    c.close()


def test_eigensolver_on_a_pair_list_context_matches_the_dense_spectrum():
    require_gpu()
    L1, L2 = 12, 10
    pl = inputs.random_pairs(400, reach=3, n_offsets=10)
    ctx, pm = _pair_ctx(L1, L2, pl, torch.float64)
    # a relaxed-ish state: the ferromagnet is not a critical point of a random
    # list, but the tangent spectrum is defined at any configuration
    m = inputs.add_noise(inputs.ferromagnet(L1, L2), 0.05, 401)
    md = to_dev(m, torch.float64)
    starts = np.stack([inputs.gaussian_field(402 + q, L1, L2) for q in range(2)])
    lam, V, info = ctx.lowest_modes(md, to_dev(starts, torch.float64).contiguous(), k=2, block=2, krylov_steps=48)
    # dense tangent Hessian of the pair model, column by column from the oracle HVP
    g, s = pairs.riemann_grad(pm, m)
    n = 3 * L1 * L2
    H = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        H[:, c] = pairs.hvp(pm, m, s, spin.project(m, e.reshape(3, L2, L1))).ravel()
    # restrict to the tangent space: an orthonormal tangent basis per site
    B = []
    for i in range(L1 * L2):
        mi = m.reshape(3, -1)[:, i]
        a = np.cross(mi, [0.0, 0.0, 1.0] if abs(mi[2]) < 0.9 else [1.0, 0.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(mi, a)
        for t in (a, b):
            col = np.zeros((3, L1 * L2))
            col[:, i] = t
            B.append(col.ravel())
    B = np.array(B).T
    w = np.linalg.eigvalsh(B.T @ H @ B)
    lam = to_np(lam)
    assert lam[0] == pytest.approx(w[0], abs=1e-8) and lam[1] == pytest.approx(w[1], abs=1e-8)
    ctx.close()


def test_invalid_pair_lists_are_refused():
    require_gpu()
    ctx = context(Model(12, 12, **FULL), torch.float64)
    bad = [[(1, 0, 1.0, (0.0, 0.0, 0.0))],                                   # no partner
           [(1, 0, 1.0, (0.1, 0, 0)), (-1, 0, 1.0, (0.1, 0, 0))],           # D not antisymmetric
           [(0, 0, 1.0, (0, 0, 0))],                                          # d = 0
           [(9, 0, 1.0, (0, 0, 0)), (-9, 0, 1.0, (0, 0, 0))],               # beyond the reach
           [(6, 0, 1.0, (0, 0, 0)), (-6, 0, 1.0, (0, 0, 0))]]               # lattice too small
    for pl in bad:
        with pytest.raises(mo.MotoError):
            ctx.set_pairs(pl)
    ctx.close()
