"""The 256 x 256 FP32 workload (3 shells; seeded skyrmion, antiskyrmion and
meron starts; k = 6 modes) taken to saddles on the GPU, each saddle certified
by the FP64 oracle.  MMF is path-dependent, so the check is the rule for a
saddle found in another precision: at the GPU's spins the oracle computes
the gradient and its own six lowest modes (block Lanczos from the GPU's
modes), so the reflected force and the index-1 signature are the oracle's;
its own MMF ascent started there must converge within 50 steps to a saddle
within 1e-4 meV and 1e-3 rad.  The signature uses the curvature threshold
tau_lambda = 1e-4 meV (R22): soft translation modes (|lambda| ~ 1e-5 meV) are
below the resolution of FP32 curvatures against |H| ~ 20 meV.  At the saddle,
the GPU's k = 6 LOBPCG (FP64 Rayleigh-Ritz) gives lambda_1 within the FP32
eigenvalue bar of the oracle's, and lambda_2 within tau_lambda."""
import numpy as np
import pytest
import torch

import inputs
from oracle import krylov, mmf, spin
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu

TAU_L = 1e-4
HNORM = 30.0  # bound of |H| for these strengths (meV)


@pytest.mark.parametrize("w", [0, 7, 15])  # a skyrmion, an antiskyrmion, a meron start
def test_config2_fp32_saddle_certified_by_the_oracle(w):
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = workload_model(2)
    m0 = inputs.workload2_states(w + 1)[w]
    V0 = np.stack([inputs.gaussian_field(inputs.workload_seed(2, 100 + 10 * w + j), 256, 256) for j in range(6)])
    ctx = context(M, torch.float32, k=6, block=6, krylov_steps=16, max_steps=8000, tau_lambda=TAU_L)
    m = to_dev(m0, torch.float32)
    V = to_dev(V0, torch.float32)
    rc, steps, trace = ctx.ascend(m, V, check_every=50)
    assert rc == mo.MOTO_OK, (w, rc, steps, to_np(trace[-1]))
    last = to_np(trace[-1])
    assert last[1] <= 1e-3 and last[2] < -TAU_L < last[3]
    E_gpu = float(to_np(ctx.energy(m))[0])  # FP64 sum over the FP32 spins
    mg, Vg = to_np(m), to_np(V)
    assert E_gpu == pytest.approx(spin.energy(M, mg), abs=1e-6)
    # the oracle at the GPU's saddle
    g, s = spin.riemann_grad(M, mg)
    lam, Vo = krylov.block_lanczos_modes(M, mg, s, [Vg[j] for j in range(6)], 16, 6)
    assert mmf.max_torque(mmf.reflected_force(-g, Vo[0])) <= 5e-3
    assert lam[0] < -TAU_L and lam[1] > -TAU_L, lam[:3]
    P = mmf.MMFParams(k=6, solver="block_lanczos", krylov_steps=16, max_steps=50, tau_F=1e-3, tau_lambda=TAU_L)
    res = mmf.ascend(M, mg, list(Vo[:6]), P)
    assert res.converged and res.steps <= 50
    assert abs(spin.energy(M, res.m) - E_gpu) <= 1e-4
    assert float(np.sqrt(np.max(np.sum((res.m - mg) ** 2, axis=0)))) < 1e-3
    # k = 6 LOBPCG on the GPU at the saddle
    lamL, VL, info = ctx.lowest_modes(m, V, solver=mo.MOTO_SOLVER_LOBPCG, max_iter=200, tol=1e-4)
    lamL = to_np(lamL)
    assert mo.moto_status(ctx.handle) == mo.MOTO_OK
    assert abs(lamL[0] - lam[0]) <= 1e-4 * abs(lam[0]) + 1e-6 * HNORM, (lamL[:2], lam[:2])
    assert abs(lamL[1] - lam[1]) <= TAU_L, (lamL[:2], lam[:2])
    ctx.close()
