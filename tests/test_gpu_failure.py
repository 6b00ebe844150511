"""Failure detection without a GPU fault: every device wait is bounded and
reports through the context's status word; iteration caps report
MOTO_NOT_CONVERGED.  Nothing here faults, traps or hangs the GPU: the
timeout is provoked by lowering the bound of the streaming kernel's waits
from the host (a handful of non-blocking tests), and the copies in flight
are still drained with the full bound."""
import numpy as np
import pytest
import torch

import inputs
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu


def _solve(ctx, m, v0):
    lam, V, info = ctx.lowest_modes(m, v0)
    torch.cuda.synchronize()
    return to_np(lam), to_np(V), to_np(info)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_bounded_wait_reports_timeout_and_the_context_recovers(dtype):
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = workload_model(2, 64, 48)
    params = dict(k=2, block=2, krylov_steps=10)
    m = to_dev(inputs.add_noise(inputs.skyrmion(M.L1, M.L2, 5.0), 0.05, 71), dtype)
    v0 = to_dev(np.stack([inputs.gaussian_field(72 + j, M.L1, M.L2) for j in range(2)]), dtype)
    ctx = context(M, dtype, **params)
    lam_ref, V_ref, info_ref = _solve(ctx, m, v0)
    assert mo.moto_status(ctx.handle) == mo.MOTO_OK
    # one non-blocking test per stage: the consumers give up on the first
    # stage whose copies have not landed yet
    mo.moto_set_wait_limit(ctx.handle, 1)
    _solve(ctx, m, v0)
    assert mo.moto_status(ctx.handle) == mo.MOTO_ERR_TIMEOUT
    # the host restores the bound and clears the status: the same solve again
    # gives exactly the first result
    mo.moto_set_wait_limit(ctx.handle, 0)
    mo.moto_clear_status(ctx.handle)
    lam, V, info = _solve(ctx, m, v0)
    assert mo.moto_status(ctx.handle) == mo.MOTO_OK
    np.testing.assert_array_equal(lam, lam_ref)
    np.testing.assert_array_equal(V, V_ref)
    np.testing.assert_array_equal(info, info_ref)
    ctx.close()


def test_wait_limit_rejects_negative_bounds():
    require_gpu()
    import paper_2509_26269_gb300 as mo
    ctx = context(workload_model(1), torch.float64)
    with pytest.raises(mo.MotoError):
        mo.moto_set_wait_limit(ctx.handle, -1)
    ctx.close()


def test_ascent_step_cap_reports_not_converged():
    """A 3-step cap on the 32 x 32 ascent (which needs ~100 steps) ends with
    MOTO_NOT_CONVERGED, three steps taken and no device error."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = workload_model(1)
    ctx = context(M, torch.float64)
    m = to_dev(inputs.workload1_state(), torch.float64)
    q0 = inputs.gaussian_field(inputs.workload_seed(1, 0), 32, 32, offset=10**6)
    V = to_dev(q0, torch.float64)[None].contiguous()
    rc, steps, trace = ctx.ascend(m, V, check_every=1, max_steps=3)
    assert rc == mo.MOTO_NOT_CONVERGED
    assert steps == 3
    tr = to_np(trace)
    assert tr.shape[0] == 4 and np.isfinite(tr).all()
    assert tr[-1, 1] > 1e-3  # the force is still above tau_F
    assert mo.moto_status(ctx.handle) == mo.MOTO_OK
    ctx.close()


def test_batch_step_cap_reports_not_converged_per_walker():
    require_gpu()
    from paper_2509_26269_gb300 import Batch, MOTO_NOT_CONVERGED
    FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)
    walkers = []
    for w, L in enumerate((24, 32)):
        m = inputs.add_noise(inputs.skyrmion(L, L, 0.2 * L), 0.05, 300 + w)
        V = inputs.gaussian_field(310 + w, L, L)[None]
        walkers.append((to_dev(m, torch.float32), to_dev(V, torch.float32)))
    b = Batch(walkers, dtype=torch.float32, n_streams=2, k=1, block=1, krylov_steps=20, max_steps=3, **FULL)
    rc, status, steps, rec = b.ascend(check_every=1)
    assert rc == MOTO_NOT_CONVERGED
    assert list(status) == [MOTO_NOT_CONVERGED] * 2
    assert list(steps) == [3, 3]
    assert np.isfinite(to_np(rec)).all()
    b.close()
