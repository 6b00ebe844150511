"""GPU parity of the stencil kernels (energy + Riemannian gradient, tangent
HVP, topological charge) against the FP64 oracle, through the C ABI.

Tolerances (reading of the stated gradient bar): the Riemannian gradient error
is measured against the Euclidean gradient norm, |dg|_2 <= 1e-12 |grad E|_2 in
FP64 and <= 1e-5 in FP32; the same bars for the HVP relative to |(hess E) v|."""
import math

import numpy as np
import pytest
import torch

import inputs
from oracle import spin, topo
from oracle.model import Model
from gpu_util import context, rand_spins, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}

# lattices: tile-aligned, ragged, smaller than a tile, odd primes
SIZES = [(32, 32), (37, 29), (5, 5), (6, 7), (13, 64), (96, 33)]


def rel(a, b, ref):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(ref.ravel()))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("L1,L2", SIZES)
def test_energy_grad_parity(dtype, L1, L2):
    require_gpu()
    M = Model(L1, L2, **FULL)
    m = rand_spins(L1, L2, 1000 + L1 * L2)
    ctx = context(M, dtype)
    md = to_dev(m, dtype)
    out, g, s = ctx.energy_grad(md)
    mo = to_np(md)  # the rounded input the kernel saw
    g_ref, s_ref = spin.riemann_grad(M, mo)
    ge = spin.euclid_grad(M, mo)
    assert rel(to_np(g), g_ref, ge) <= TOL[dtype]
    assert rel(to_np(s), s_ref, np.sqrt(np.sum(ge * ge, axis=0))) <= TOL[dtype]
    E_ref = spin.energy(M, mo)
    scale = math.fsum(np.abs(spin.site_energy(M, mo)).ravel())
    E, gmax = to_np(out)
    assert abs(E - E_ref) <= (1e-13 if dtype == torch.float64 else 2e-6) * scale
    assert gmax == pytest.approx(math.sqrt(np.max(np.sum(g_ref ** 2, axis=0))), rel=10 * TOL[dtype])
    # FP64-arithmetic energy of the same (rounded) spins
    E64 = to_np(ctx.energy(md))[0]
    assert abs(E64 - E_ref) <= 1e-13 * scale
    ctx.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("L1,L2", SIZES)
def test_hvp_parity(dtype, L1, L2):
    require_gpu()
    M = Model(L1, L2, **FULL)
    m = rand_spins(L1, L2, 2000 + L1 * L2)
    ctx = context(M, dtype)
    md = to_dev(m, dtype)
    _, _, s = ctx.energy_grad(md)
    mo = to_np(md)
    _, s_ref = spin.riemann_grad(M, mo)
    vs = np.stack([spin.project(mo, inputs.gaussian_field(3000 + j, L1, L2)) for j in range(3)])
    vd = to_dev(vs, dtype)
    hv = to_np(ctx.hvp(md, s, vd))
    for j in range(3):
        v = to_np(vd[j])
        ref = spin.hvp(M, mo, s_ref, v)
        assert rel(hv[j], ref, spin.euclid_hvp(M, v)) <= TOL[dtype]
    # one vector at a time equals the batched call
    hv1 = to_np(ctx.hvp(md, s, vd[1].contiguous()))
    np.testing.assert_array_equal(hv1, hv[1])
    ctx.close()


def test_hvp_symmetry_fp64():
    require_gpu()
    M = Model(40, 24, **FULL)
    m = rand_spins(40, 24, 5)
    ctx = context(M, torch.float64)
    md = to_dev(m, torch.float64)
    _, _, s = ctx.energy_grad(md)
    u = to_dev(spin.project(m, inputs.gaussian_field(6, 40, 24)), torch.float64)
    v = to_dev(spin.project(m, inputs.gaussian_field(7, 40, 24)), torch.float64)
    a = float(torch.sum(u * ctx.hvp(md, s, v)))
    b = float(torch.sum(v * ctx.hvp(md, s, u)))
    assert a == pytest.approx(b, rel=1e-12)
    ctx.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_ferromagnet_plane_waves_through_gpu(dtype):
    """Closed-form spin-wave eigenpairs of the uniform state, on the GPU."""
    require_gpu()
    L = 48
    M = Model(L, L, **FULL)
    ctx = context(M, dtype)
    md = to_dev(inputs.ferromagnet(L, L), dtype)
    _, _, s = ctx.energy_grad(md)
    i2, i1 = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    from oracle.model import SHELLS
    for n1, n2 in [(0, 0), (1, 0), (5, 3), (24, 11)]:
        lam = M.muB + 2 * M.K
        for Js, shell in zip(M.J, SHELLS):
            for d1, d2 in shell:
                lam += 2 * Js * (1 - math.cos(2 * math.pi * (n1 * d1 + n2 * d2) / L))
        v = np.zeros((3, L, L))
        v[1] = np.cos(2 * math.pi * (n1 * i1 + n2 * i2) / L)
        hv = to_np(ctx.hvp(md, s, to_dev(v, dtype)))
        assert np.max(np.abs(hv - lam * v)) <= 20 * TOL[dtype] * max(lam, 1.0)
    ctx.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_topological_charge(dtype):
    require_gpu()
    L = 64
    M = Model(L, L, **FULL)
    ctx = context(M, dtype)
    cases = [(inputs.skyrmion(L, L, 5.0), 1), (inputs.skyrmion(L, L, 5.0, anti=True), -1),
             (inputs.biskyrmion(L, L, 5.0), 2), (inputs.multi_texture(L, L, -2, 4.0, 77), -2),
             (inputs.multi_texture(L, L, 0, 4.0, 78), 0), (inputs.ferromagnet(L, L), 0)]
    for m, q in cases:
        md = to_dev(m, dtype)
        Q = to_np(ctx.topo_charge(md))[0]
        Qref = topo.topo_charge(to_np(md))
        assert int(round(Q)) == q == int(round(Qref))
        assert abs(Q - Qref) <= (1e-10 if dtype == torch.float64 else 1e-4)
    ctx.close()


def test_workload2_size_fp32_vs_oracle():
    require_gpu()
    M = workload_model(2)
    m = inputs.workload2_states(1)[0]
    ctx = context(M, torch.float32)
    md = to_dev(m, torch.float32)
    out, g, s = ctx.energy_grad(md)
    mo = to_np(md)
    g_ref, s_ref = spin.riemann_grad(M, mo)
    assert rel(to_np(g), g_ref, spin.euclid_grad(M, mo)) <= 1e-5
    v = spin.project(mo, inputs.gaussian_field(11, 256, 256))
    vd = to_dev(v, torch.float32)
    ref = spin.hvp(M, mo, s_ref, to_np(vd))
    assert rel(to_np(ctx.hvp(md, s, vd)), ref, spin.euclid_hvp(M, to_np(vd))) <= 1e-5
    ctx.close()


def test_nonfinite_input_is_reported_not_trapped():
    """A NaN spin made on the host: the kernel flags it in the status word."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = Model(16, 16, **FULL)
    m = rand_spins(16, 16, 9)
    m[0, 3, 4] = np.nan
    ctx = context(M, torch.float64)
    ctx.energy_grad(to_dev(m, torch.float64))
    assert mo.moto_status(ctx.handle) == mo.MOTO_ERR_NONFINITE
    mo.moto_clear_status(ctx.handle)
    assert mo.moto_status(ctx.handle) == mo.MOTO_OK
    ctx.close()
