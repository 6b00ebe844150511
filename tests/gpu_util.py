"""Helpers for the GPU parity tests: numpy <-> torch and a context factory."""
import numpy as np
import pytest
import torch

import inputs
from oracle.model import Model


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def to_np(t):
    return t.detach().to("cpu", torch.float64).numpy()


def context(model: Model, dtype, **params):
    from paper_2509_26269_gb300 import Context
    return Context(model.L1, model.L2, J=model.J, D=model.D, K=model.K, muB=model.muB, dtype=dtype, **params)


def workload_model(c, L1=None, L2=None):
    p = inputs.WORKLOADS[c]
    return Model(L1 or p["L1"], L2 or p["L2"], J=tuple(p["J"]), D=p["D"], K=p["K"], muB=p["muB"])


def rand_spins(L1, L2, seed):
    m = inputs.gaussian_field(seed, L1, L2)
    return m / np.sqrt(np.sum(m * m, axis=0))[None]
