"""GPU parity at the full benchmark size: the 2048 x 2048 three-shell
workload (4,194,304 spins, FP32 fields, biskyrmion start) in the launch
configuration the benchmark times (8 HVPs a launch, k = 8 block Lanczos with
8 x 12 steps, one MMF outer step).  The FP64 oracle evaluates the same
(FP32-rounded) fields on the host: energy, gradient and HVPs element by
element; the Krylov output is checked by properties that hold at any size
(tangency, orthonormality, each Ritz value the oracle's Rayleigh quotient of
its vector, within the FP32 bar |dlam| <= 1e-4 |lam| + 1e-6 |H|)."""
import math

import numpy as np
import pytest
import torch

import inputs
from oracle import spin, topo
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 fields, relative to the Euclidean counterpart's norm


def hnorm(M):
    """Gershgorin-type bound on |H| for the shell model: each of the six
    bonds of a shell couples with weight 2 |J_s| twice (ordered pairs), the
    DMI bonds with 2 |D|, plus the anisotropy and Zeeman diagonal."""
    return sum(24.0 * abs(J) for J in M.J) + 12.0 * abs(M.D) + 2.0 * abs(M.K) + abs(M.muB)


def rel(a, b, ref):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(ref.ravel()))


def vdot(a, b):
    return float(np.dot(a.ravel(), b.ravel()))


def fp32_ok(M, lam_gpu, lam_ref):
    return abs(lam_gpu - lam_ref) <= 1e-4 * abs(lam_ref) + 1e-6 * hnorm(M)


def start_block(L1, L2):
    seed = inputs.workload_seed(4, 0) + 17
    return np.stack([inputs.gaussian_field(seed, L1, L2, offset=j * 3 * L1 * L2) for j in range(8)])


@pytest.fixture(scope="module")
def full():
    require_gpu()
    M = workload_model(4)
    ctx = context(M, torch.float32, k=8, block=8, krylov_steps=12)
    md = to_dev(inputs.workload4_state(), torch.float32)
    mo = to_np(md)  # the rounded state the kernels see
    _, s_ref = spin.riemann_grad(M, mo)
    yield M, ctx, md, mo, s_ref
    ctx.close()


def test_fullsize_energy_gradient_and_hvps(full):
    M, ctx, md, mo, s_ref = full
    out, g, s = ctx.energy_grad(md)
    g_ref, _ = spin.riemann_grad(M, mo)
    ge = spin.euclid_grad(M, mo)
    assert rel(to_np(g), g_ref, ge) <= TOL
    scale = math.fsum(np.abs(spin.site_energy(M, mo)).ravel())
    assert abs(to_np(out)[0] - spin.energy(M, mo)) <= 2e-6 * scale
    # eight tangent vectors in one launch, as the Krylov solver issues them
    vs = np.stack([spin.project(mo, inputs.gaussian_field(7000 + j, M.L1, M.L2)) for j in range(8)])
    vd = to_dev(vs, torch.float32)
    hv = to_np(ctx.hvp(md, s, vd))
    for j in (0, 3, 7):
        v = to_np(vd[j])
        assert rel(hv[j], spin.hvp(M, mo, s_ref, v), spin.euclid_hvp(M, v)) <= TOL


def test_fullsize_block_lanczos_properties(full):
    M, ctx, md, mo, s_ref = full
    _, _, s = ctx.energy_grad(md)
    lam, V, info = ctx.lowest_modes(md, to_dev(start_block(M.L1, M.L2), torch.float32), s)
    assert int(to_np(info)[1]) == 0  # no device status bits
    lam = to_np(lam)
    Vh = to_np(V)
    G = Vh.reshape(8, -1) @ Vh.reshape(8, -1).T
    np.testing.assert_allclose(G, np.eye(8), atol=1e-4)
    for j in range(8):
        assert np.max(np.abs(np.sum(Vh[j] * mo, axis=0))) <= 1e-5
        # sign rule: the entry of largest magnitude is positive
        flat = Vh[j].ravel()
        assert flat[np.argmax(np.abs(flat))] > 0
    assert np.all(np.diff(lam[:16]) >= -1e-7)
    for j in (0, 1, 7):
        v = Vh[j]
        rq = vdot(v, spin.hvp(M, mo, s_ref, v)) / vdot(v, v)
        assert fp32_ok(M, lam[j], rq), (j, lam[j], rq)


def test_fullsize_mmf_step(full):
    """One outer step as the benchmark runs it: the reported energy, lowest
    curvatures and force norm belong to the input state (oracle), the new
    state keeps unit spins and the biskyrmion's charge."""
    M, ctx, md, mo, s_ref = full
    m = md.clone()
    V = to_dev(start_block(M.L1, M.L2), torch.float32)
    ctx.reset()
    out, _ = ctx.mmf_step(m, V)
    out = to_np(out)
    scale = math.fsum(np.abs(spin.site_energy(M, mo)).ravel())
    assert abs(out[0] - spin.energy(M, mo)) <= 2e-6 * scale
    Vh = to_np(V)
    for j, lam in ((0, out[2]), (1, out[3])):
        v = Vh[j]
        rq = vdot(v, spin.hvp(M, mo, s_ref, v)) / vdot(v, v)
        assert fp32_ok(M, lam, rq), (j, lam, rq)
    # |F_mmf| = max_i |g_i - 2 (g . v1) v1_i| at the input state
    g_ref, _ = spin.riemann_grad(M, mo)
    v1 = Vh[0] / np.linalg.norm(Vh[0])
    f = g_ref - 2.0 * vdot(g_ref, v1) * v1
    fmax_ref = math.sqrt(float(np.max(np.sum(f * f, axis=0))))
    assert out[1] == pytest.approx(fmax_ref, rel=1e-3)
    mn = to_np(m)
    assert np.max(np.abs(np.sum(mn * mn, axis=0) - 1.0)) <= 1e-5
    assert not np.array_equal(mn, mo)
    assert int(round(topo.topo_charge(mn))) == 2
