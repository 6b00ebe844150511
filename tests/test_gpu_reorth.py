"""Reorthogonalisation of block Lanczos on the GPU: the orthogonality of the
whole Krylov basis (not only of the returned Ritz vectors), for the full
scheme and for the selective one (Simon's omega estimate in block form), and
the agreement of the selective scheme's eigenvalues with the oracle.

Bars.  Full reorthogonalisation keeps every entry of Q^T Q - I at the size of
the rounding of the stored fields times a small factor: <= 1e-5 for FP32
fields (unit roundoff 6e-8), <= 1e-12 for FP64.  The selective scheme keeps
the basis semi-orthogonal: the estimate triggers the full pass once it
crosses sqrt(eps) (2.4e-4 in FP32), so the measured entries stay within a
small multiple of it (<= 2e-3); semi-orthogonality keeps the Ritz values as
accurate as full reorthogonalisation (Simon 1984), so they meet the same
eigenvalue bars as the full scheme: 1e-9 relative to the oracle in FP64,
1e-4 |lam| + 1e-6 |H| in FP32."""
import numpy as np
import pytest
import torch

import inputs
from oracle import krylov, spin
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu


def basis_gram(mo, ctx):
    """(Q^T Q of the last solve's basis, full passes taken)."""
    ptr, ld, nv, nr = mo.moto_krylov_basis(ctx.handle)
    esz = 4 if ctx.dtype == torch.float32 else 8
    G = np.zeros((nv, nv))
    for c0 in range(0, nv, 8):
        ny = min(8, nv - c0)
        out = torch.empty(nv * ny, dtype=torch.float64, device="cuda")
        mo.moto_gram(ctx.handle, ptr, ld, nv, ptr + c0 * ld * esz, ld, ny, out)
        G[:, c0:c0 + ny] = to_np(out).reshape(nv, ny)
    return G, nr


def test_selective_lanczos_fp64_matches_the_oracle():
    """32 x 32 workload, Lanczos k = 1, 60 steps: the selective scheme skips
    most full passes and still matches the oracle's fully reorthogonalised
    run."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = workload_model(1)
    m = inputs.workload1_state()
    q0 = inputs.gaussian_field(inputs.workload_seed(1, 0), 32, 32, offset=10**6)
    ctx = context(M, torch.float64, k=1, block=1, krylov_steps=60, reorth=mo.MOTO_REORTH_SELECTIVE)
    md = to_dev(m, torch.float64)
    lam, V, info = ctx.lowest_modes(md, to_dev(q0, torch.float64)[None].contiguous())
    G, nr = basis_gram(mo, ctx)
    _, s_ref = spin.riemann_grad(M, m)
    th, Vr = krylov.lanczos_modes(M, m, s_ref, q0, 60, k=1)
    lam = to_np(lam)
    assert int(to_np(info)[0]) == 60
    assert nr < 59
    assert np.max(np.abs(G - np.eye(G.shape[0]))) <= 1e-7  # semi-orthogonal: sqrt(eps) = 1.05e-8
    np.testing.assert_allclose(lam[:8], th[:8], rtol=1e-9, atol=1e-12)
    assert abs(float(np.dot(to_np(V[0]).ravel(), Vr[0].ravel()))) == pytest.approx(1.0, abs=1e-8)
    ctx.close()


@pytest.mark.parametrize("L", [256, 1024])
def test_basis_orthogonality_fp32_full_and_selective(L):
    """The roofline workload's solver (3 shells, FP32, block Lanczos 8 x 12,
    biskyrmion start) at L x L: the whole 96-field basis, full vs selective,
    and the eight lowest eigenvalues of both."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = workload_model(4, L, L)
    m = inputs.add_noise(inputs.biskyrmion(L, L, 8.0), 0.01, inputs.workload_seed(4, 0))
    V0 = np.stack([inputs.gaussian_field(inputs.workload_seed(4, 17), L, L, offset=j * 3 * L * L) for j in range(8)])
    md = to_dev(m, torch.float32)
    res = {}
    for name, mode in (("full", mo.MOTO_REORTH_FULL), ("selective", mo.MOTO_REORTH_SELECTIVE)):
        ctx = context(M, torch.float32, k=8, block=8, krylov_steps=12, reorth=mode)
        lam, V, info = ctx.lowest_modes(md, to_dev(V0, torch.float32))
        assert mo.moto_status(ctx.handle) == mo.MOTO_OK
        G, nr = basis_gram(mo, ctx)
        res[name] = dict(lam=to_np(lam), dev=float(np.max(np.abs(G - np.eye(G.shape[0])))), nr=nr,
                         nv=G.shape[0])
        ctx.close()
    f, s = res["full"], res["selective"]
    assert f["nv"] == s["nv"] == 96
    assert f["nr"] == 11
    assert f["dev"] <= 1e-5, f["dev"]
    assert s["dev"] <= 2e-3, s["dev"]
    assert s["nr"] < 11
    # |H| <= 2 sum_s 6 |J_s| max(1 - cos) + |muB| + 2 K + DMI < 30 meV for these strengths
    hn = 30.0
    for i in range(8):
        assert abs(s["lam"][i] - f["lam"][i]) <= 1e-4 * abs(f["lam"][i]) + 1e-6 * hn, (i, s["lam"][i], f["lam"][i])
    print(f"L={L}: full |QtQ-I|={f['dev']:.2e}, selective |QtQ-I|={s['dev']:.2e} with {s['nr']} of 11 full passes")
