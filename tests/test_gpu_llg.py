"""GPU parity of the dynamic certifier (damped Landau-Lifshitz-Gilbert
descent, Heun): a fixed 50-step trajectory from both descent seeds against
the oracle (FP64 and FP32, ragged lattice), and the two-sided descent from the
32 x 32 workload's saddle reaching the oracle's minima and charges."""
import numpy as np
import pytest
import torch

import inputs
from oracle import mmf, spin, topo
from oracle.model import Model
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 2e-4)])
def test_llg_trajectory_matches_the_oracle(dtype, tol):
    require_gpu()
    L1, L2 = 24, 20
    M = Model(L1, L2, **FULL)
    m = inputs.add_noise(inputs.skyrmion(L1, L2, 3.5), 0.05, 17)
    v = spin.project(m, inputs.gaussian_field(18, L1, L2))
    v /= np.sqrt(np.sum(v * v))
    kw = dict(descent=1, llg_alpha=1.0, llg_dt=0.01, llg_time=0.5, tau_F=1e-12)
    ctx = context(M, dtype, **kw)
    md, vd = to_dev(m, dtype), to_dev(v, dtype)
    rc, mp, mm, out = ctx.descend(md, vd)
    P = mmf.MMFParams(descent="llg", llg_alpha=1.0, llg_dt=0.01, llg_time=0.5, tau_F=1e-12)
    seeds = mmf.descent_seeds(to_np(md), to_np(vd), P)
    o = to_np(out)
    for x_gpu, seed, steps in ((mp, seeds[0], o[4]), (mm, seeds[1], o[5])):
        ref, conv, nsteps = mmf.llg_relax(M, seed, P)
        assert not conv and nsteps == 50 and int(steps) == 50
        assert np.max(np.abs(to_np(x_gpu) - ref)) <= tol
    ctx.close()


def test_llg_descent_reaches_the_oracle_minima():
    require_gpu()
    M = workload_model(1)
    m0 = inputs.workload1_state()
    q0 = inputs.gaussian_field(inputs.workload_seed(1, 0), 32, 32, offset=10**6)
    res = mmf.ascend(M, m0, [q0], mmf.MMFParams())
    P = mmf.MMFParams(descent="llg")
    plus, minus = mmf.descend(M, res.m, res.v1, P)
    ctx = context(M, torch.float64, descent=1)
    rc, mp, mm, out = ctx.descend(to_dev(res.m, torch.float64), to_dev(res.v1, torch.float64))
    assert rc == 0 and plus.converged and minus.converged
    E_p, Q_p, E_m, Q_m, s_p, s_m = to_np(out)
    assert int(round(Q_p)) == plus.Qint and int(round(Q_m)) == minus.Qint
    assert E_p == pytest.approx(plus.E, abs=1e-6) and E_m == pytest.approx(minus.E, abs=1e-6)
    assert abs(int(s_p) - plus.steps) <= 1 and abs(int(s_m) - minus.steps) <= 1
    for x in (mp, mm):
        g, _ = spin.riemann_grad(M, to_np(x))
        assert mmf.max_torque(g) <= 1e-3 * (1 + 1e-9)
    ctx.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_llg_graph_replay_matches_plain_launches(monkeypatch, dtype):
    """The Heun steps are replayed as a captured CUDA graph after the first;
    launching every kernel (MOTO_GRAPHS=0) must give the same end states,
    energies, charges and step counts bit for bit."""
    require_gpu()
    L1, L2 = 24, 20
    M = Model(L1, L2, **FULL)
    m = inputs.add_noise(inputs.skyrmion(L1, L2, 3.5), 0.05, 21)
    v = spin.project(m, inputs.gaussian_field(22, L1, L2))
    v /= np.sqrt(np.sum(v * v))
    res = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("MOTO_GRAPHS", graphs)
        ctx = context(M, dtype, descent=1, llg_alpha=1.0, llg_dt=0.01, llg_time=0.6, tau_F=1e-12)
        rc, mp, mm, out = ctx.descend(to_dev(m, dtype), to_dev(v, dtype))
        res.append((rc, to_np(mp), to_np(mm), to_np(out)))
        ctx.close()
    (rc_a, mp_a, mm_a, o_a), (rc_b, mp_b, mm_b, o_b) = res
    assert rc_a == rc_b and int(o_a[4]) == int(o_a[5]) == 60
    np.testing.assert_array_equal(mp_a, mp_b)
    np.testing.assert_array_equal(mm_a, mm_b)
    np.testing.assert_array_equal(o_a, o_b)
