"""The allocation-free energy + gradient entry point, for callers that cannot
allocate device memory (and so cannot create a moto_ctx), must give the same
outputs as the context path, call after call: its scratch is a fixed array
inside the library that every call reuses.  Collected last on purpose."""
import ctypes
import gc

import numpy as np
import pytest
import torch

import inputs
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,code,tol", [(torch.float64, 1, 1e-12), (torch.float32, 0, 1e-5)])
def test_noalloc_matches_context_path_twice(dtype, code, tol):
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = workload_model(2, 96, 72)
    model = mo.make_model(M.L1, M.L2, J=M.J, D=M.D, K=M.K, muB=M.muB)
    ctx = context(M, dtype)
    for call, seed in enumerate((11, 12)):
        m = to_dev(inputs.add_noise(inputs.skyrmion(M.L1, M.L2, 6.0), 0.1, seed), dtype)
        out_ref, g_ref, s_ref = ctx.energy_grad(m)
        g = torch.full_like(g_ref, float("nan"))
        s = torch.full_like(s_ref, float("nan"))
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        mo.moto_energy_grad_noalloc(model, code, m, g, s, out)
        torch.cuda.synchronize()
        gr = to_np(g_ref)
        assert np.linalg.norm(to_np(g) - gr) <= tol * max(np.linalg.norm(gr), 1.0), call
        assert np.max(np.abs(to_np(s) - to_np(s_ref))) <= tol * float(torch.max(torch.abs(s_ref))), call
        o, r = to_np(out), to_np(out_ref)
        assert abs(o[0] - r[0]) <= tol * abs(r[0]) and abs(o[1] - r[1]) <= tol * abs(r[1]), call
    ctx.close()


def test_noalloc_rejects_lattices_beyond_its_fixed_scratch():
    require_gpu()
    import paper_2509_26269_gb300 as mo
    for L1, L2 in ((8192, 4097), (2147483616, 1056)):
        big = mo.make_model(L1, L2, J=(1.0,))
        rc = mo._lib.moto_energy_grad_noalloc(ctypes.byref(big), 0, 1, None, None, None, None)
        assert rc == mo.MOTO_ERR_ARG


def test_noalloc_allocates_no_device_memory():
    """The defining property: after a first call (which looks up the fixed
    array), further calls leave the device's free memory unchanged."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    M = workload_model(2, 64, 48)
    model = mo.make_model(M.L1, M.L2, J=M.J, D=M.D, K=M.K, muB=M.muB)
    m = to_dev(inputs.add_noise(inputs.skyrmion(M.L1, M.L2, 5.0), 0.1, 21), torch.float32)
    g = torch.empty_like(m)
    s = torch.empty(M.L1 * M.L2, dtype=torch.float32, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    # the binding raises MotoError on any non-OK return code
    mo.moto_energy_grad_noalloc(model, 0, m, g, s, out)
    torch.cuda.synchronize()
    # contexts of earlier tests may still be released by the garbage
    # collector; do that now and keep it off while measuring
    gc.collect()
    gc.disable()
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(5):
            mo.moto_energy_grad_noalloc(model, 0, m, g, s, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
    finally:
        gc.enable()
    assert free1 == free0
