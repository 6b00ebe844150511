"""The strip HVP's variants (strip length, warps per block, spins held in
registers, FP32 pair arithmetic packed or scalar) must give bit-identical
results, so that the autotuner's choice, which depends on timing, never
changes a result; each is checked against the oracle too."""
import numpy as np
import pytest
import torch

import inputs
from oracle import spin
from oracle.model import Model
from gpu_util import context, rand_spins, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("L1,L2", [(128, 64), (37, 29), (200, 72), (6, 7)])
def test_hvp_variants_are_bit_identical(dtype, L1, L2):
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = Model(L1, L2, **FULL)
    m = rand_spins(L1, L2, 7000 + L1)
    ctx = context(M, dtype, k=3, block=3, krylov_steps=4)
    variant, ms = mo.moto_hvp_tuning(ctx.handle)
    assert 0 <= variant < len(ms)
    md = to_dev(m, dtype)
    _, _, s = ctx.energy_grad(md)
    mo_ = to_np(md)
    _, s_ref = spin.riemann_grad(M, mo_)
    vs = np.stack([spin.project(mo_, inputs.gaussian_field(7100 + j, L1, L2)) for j in range(3)])
    vd = to_dev(vs, dtype)
    outs = []
    for v in range(len(ms)):
        mo.moto_set_hvp_variant(ctx.handle, v)
        outs.append(to_np(ctx.hvp(md, s, vd)))
    mo.moto_set_hvp_variant(ctx.handle, -1)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    np.testing.assert_array_equal(to_np(ctx.hvp(md, s, vd)), outs[0])
    for j in range(3):
        v = to_np(vd[j])
        ref = spin.hvp(M, mo_, s_ref, v)
        err = np.linalg.norm(outs[0][j] - ref) / np.linalg.norm(spin.euclid_hvp(M, v))
        assert err <= TOL[dtype]
    with pytest.raises(mo.MotoError):
        mo.moto_set_hvp_variant(ctx.handle, len(ms))
    ctx.close()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("L1,L2", [(128, 64), (37, 29), (6, 7)])
def test_energy_stencil_variants(dtype, L1, L2):
    """The energy / gradient stencil's variants (two or three staged tiles,
    four or five blocks an SM, FP32 pair arithmetic packed or scalar) give
    bit-identical g and s and energies within the rounding of a differently
    partitioned sum; each matches the oracle."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = Model(L1, L2, **FULL)
    m = rand_spins(L1, L2, 7300 + L1)
    ctx = context(M, dtype)
    variant, ms = mo.moto_stencil_tuning(ctx.handle)
    assert 0 <= variant < len(ms) == 4
    md = to_dev(m, dtype)
    res = []
    for v in range(len(ms)):
        mo.moto_set_stencil_variant(ctx.handle, v)
        out, g, s = ctx.energy_grad(md)
        res.append((to_np(out), to_np(g), to_np(s)))
    mo.moto_set_stencil_variant(ctx.handle, -1)
    for o, g, s in res[1:]:
        np.testing.assert_array_equal(g, res[0][1])
        np.testing.assert_array_equal(s, res[0][2])
        assert o[0] == pytest.approx(res[0][0][0], rel=1e-13 if dtype == torch.float64 else 1e-6)
        assert o[1] == res[0][0][1]
    mo_ = to_np(md)
    g_ref, _ = spin.riemann_grad(M, mo_)
    err = np.linalg.norm(res[0][1] - g_ref) / np.linalg.norm(spin.euclid_grad(M, mo_))
    assert err <= TOL[dtype]
    ctx.close()
