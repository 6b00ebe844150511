"""Python binding of ``libmoto.so``, the GB300 (sm_103a) minimum-mode kernel
for atomistic spin systems (arXiv 2509.26269).

Every entry point of ``include/moto.h`` is exposed under the same name; the
functions only marshal arguments (torch CUDA tensors or raw device pointers
as ints) into the C ABI.  All computation runs in the library's CUDA kernels;
there is no CPU path: importing this package fails if ``libmoto.so`` has not
been built (``python paper_2509_26269_gb300/build.py``).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmoto.so")

MOTO_F32, MOTO_F64 = 0, 1
MOTO_OK, MOTO_NOT_CONVERGED = 0, 1
MOTO_ERR_ARG, MOTO_ERR_CUDA, MOTO_ERR_NUMERIC = -1, -2, -3
MOTO_ERR_NONFINITE, MOTO_ERR_TIMEOUT, MOTO_ERR_NOMEM = -4, -5, -6
MOTO_SOLVER_LANCZOS, MOTO_SOLVER_LOBPCG = 0, 1
MOTO_OPT_LBFGS, MOTO_OPT_CG = 0, 1
MOTO_DESCENT_OPT, MOTO_DESCENT_LLG = 0, 1
MOTO_REORTH_FULL, MOTO_REORTH_SELECTIVE = 0, 1
MOTO_MAX_POP = 64
MOTO_MAX_PAIRS, MOTO_MAX_REACH = 512, 12
MOTO_MAX_K, MOTO_MAX_BASIS, MOTO_MAX_MEM = 8, 96, 8


class moto_model(ctypes.Structure):
    _fields_ = [
        ("L1", ctypes.c_int), ("L2", ctypes.c_int), ("n_shells", ctypes.c_int),
        ("J", ctypes.c_double * 3), ("D", ctypes.c_double), ("K", ctypes.c_double), ("muB", ctypes.c_double),
    ]


class moto_params(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int), ("solver", ctypes.c_int), ("block", ctypes.c_int), ("krylov_steps", ctypes.c_int),
        ("max_iter", ctypes.c_int), ("tol", ctypes.c_double), ("lbfgs_mem", ctypes.c_int),
        ("theta_max", ctypes.c_double), ("gamma0", ctypes.c_double), ("tau_F", ctypes.c_double),
        ("eta_theta", ctypes.c_double), ("max_steps", ctypes.c_int), ("descent_max_steps", ctypes.c_int),
        ("optimizer", ctypes.c_int), ("subspace", ctypes.c_int), ("descent", ctypes.c_int),
        ("llg_alpha", ctypes.c_double), ("llg_dt", ctypes.c_double), ("llg_time", ctypes.c_double),
        ("reorth", ctypes.c_int), ("tau_lambda", ctypes.c_double),
    ]


class moto_pair(ctypes.Structure):
    _fields_ = [("d1", ctypes.c_int), ("d2", ctypes.c_int), ("J", ctypes.c_double), ("D", ctypes.c_double * 3)]


class moto_walker(ctypes.Structure):
    _fields_ = [("L1", ctypes.c_int), ("L2", ctypes.c_int), ("m_dev", ctypes.c_void_p), ("V_dev", ctypes.c_void_p)]


class MotoError(RuntimeError):
    pass


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_2509_26269_gb300/build.py` "
            "(this package has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, Z = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t
    sig = {
        "moto_default_params": (None, [ctypes.POINTER(moto_params)]),
        "moto_create": (I, [ctypes.POINTER(moto_model), I, ctypes.POINTER(moto_params), ctypes.POINTER(P)]),
        "moto_destroy": (None, [P]),
        "moto_energy_grad": (I, [P, P, P, P, P, P]),
        "moto_energy": (I, [P, P, P, P]),
        "moto_hvp": (I, [P, P, P, P, Z, P, Z, I, P]),
        "moto_energy_euclid_grad": (I, [P, P, P, P, P]),
        "moto_euclid_hvp": (I, [P, P, Z, P, Z, I, P]),
        "moto_lowest_modes": (I, [P, P, P, ctypes.POINTER(moto_params), P, P, P, P, P]),
        "moto_topo_charge": (I, [P, P, P, P]),
        "moto_lbfgs_reset": (I, [P, P]),
        "moto_mmf_step": (I, [P, P, ctypes.POINTER(moto_params), P, P, P, P]),
        "moto_ascend": (I, [P, P, ctypes.POINTER(moto_params), P, P, I, ctypes.POINTER(I), P]),
        "moto_descend": (I, [P, P, P, ctypes.POINTER(moto_params), P, P, P, P]),
        "moto_status": (I, [P, P]),
        "moto_clear_status": (I, [P, P]),
        "moto_status_string": (ctypes.c_char_p, [I]),
        "moto_workspace_bytes": (Z, [P]),
        "moto_profile_begin": (I, [P, I]),
        "moto_energy_grad_noalloc": (I, [ctypes.POINTER(moto_model), I, P, P, P, P, P]),
        "moto_gram": (I, [P, P, Z, I, P, Z, I, P, P]),
        "moto_perturb": (I, [P, P, P, P, Z, I, P, Z, P]),
        "moto_set_pairs": (I, [P, ctypes.POINTER(moto_pair), I]),
        "moto_set_wait_limit": (I, [P, I]),
        "moto_hvp_tuning": (I, [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float), I]),
        "moto_set_hvp_variant": (I, [P, I]),
        "moto_stencil_tuning": (I, [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float), I]),
        "moto_set_stencil_variant": (I, [P, I]),
        "moto_krylov_basis": (I, [P, ctypes.POINTER(P), ctypes.POINTER(Z), ctypes.POINTER(I), ctypes.POINTER(I),
                                  P]),
        "moto_pairwise_l1": (I, [P, P, Z, I, P, P]),
        "moto_profile_end": (I, [P, I, P, P, P]),
        "moto_batch_create": (I, [ctypes.POINTER(moto_model), I, ctypes.POINTER(moto_params),
                                  ctypes.POINTER(moto_walker), I, I, ctypes.POINTER(P)]),
        "moto_batch_destroy": (None, [P]),
        "moto_batch_ascend": (I, [P, I, P, P, P, P]),
        "moto_batch_descend": (I, [P, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
EXPORTED = (
    "moto_default_params", "moto_create", "moto_destroy", "moto_energy_grad", "moto_energy", "moto_hvp",
    "moto_lowest_modes", "moto_topo_charge", "moto_lbfgs_reset", "moto_mmf_step", "moto_ascend", "moto_descend",
    "moto_status", "moto_clear_status", "moto_status_string", "moto_workspace_bytes", "moto_profile_begin",
    "moto_profile_end", "moto_energy_grad_noalloc", "moto_gram", "moto_energy_euclid_grad", "moto_euclid_hvp",
    "moto_perturb", "moto_pairwise_l1", "moto_set_pairs", "moto_set_wait_limit",
    "moto_hvp_tuning", "moto_set_hvp_variant", "moto_krylov_basis", "moto_stencil_tuning",
    "moto_set_stencil_variant",
    "moto_batch_create", "moto_batch_destroy", "moto_batch_ascend", "moto_batch_descend",
)
PROFILE_KINDS = ("hvp", "gram", "combine", "stencil", "small", "vec", "eig", "reorth_gram", "reorth_update",
                 "chol2_gram")


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _ptr(x):
    """Device address of a torch CUDA tensor (checked contiguous), an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise MotoError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise MotoError("expected a contiguous tensor")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc, what, ok=(MOTO_OK,)):
    if rc not in ok:
        raise MotoError(f"{what}: {_lib.moto_status_string(rc).decode()} ({rc})")
    return rc


def make_model(L1, L2, J=(1.0,), D=0.0, K=0.0, muB=0.0) -> moto_model:
    mm = moto_model()
    mm.L1, mm.L2, mm.n_shells = int(L1), int(L2), len(J)
    for i in range(3):
        mm.J[i] = float(J[i]) if i < len(J) else 0.0
    mm.D, mm.K, mm.muB = float(D), float(K), float(muB)
    return mm


def make_params(**kw) -> moto_params:
    p = moto_params()
    _lib.moto_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise MotoError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------
# the C ABI, same names
# ---------------------------------------------------------------------------
def moto_default_params() -> moto_params:
    return make_params()


def moto_create(model: moto_model, dtype: int, params: moto_params | None = None) -> int:
    h = ctypes.c_void_p()
    p = params if params is not None else make_params()
    _check(_lib.moto_create(ctypes.byref(model), int(dtype), ctypes.byref(p), ctypes.byref(h)), "moto_create")
    return h.value


def moto_destroy(ctx: int) -> None:
    _lib.moto_destroy(ctx)


def moto_energy_grad(ctx, m, g=None, s=None, out=None, stream=None):
    _check(_lib.moto_energy_grad(ctx, _ptr(m), _ptr(g), _ptr(s), _ptr(out), _stream(stream)), "moto_energy_grad")


def moto_energy(ctx, m, E, stream=None):
    _check(_lib.moto_energy(ctx, _ptr(m), _ptr(E), _stream(stream)), "moto_energy")


def moto_hvp(ctx, m, s, v, ldv, hv, ldhv, nvec=1, stream=None):
    _check(_lib.moto_hvp(ctx, _ptr(m), _ptr(s), _ptr(v), int(ldv), _ptr(hv), int(ldhv), int(nvec),
                         _stream(stream)), "moto_hvp")


def moto_energy_euclid_grad(ctx, m, grad, out, stream=None):
    _check(_lib.moto_energy_euclid_grad(ctx, _ptr(m), _ptr(grad), _ptr(out), _stream(stream)),
           "moto_energy_euclid_grad")


def moto_euclid_hvp(ctx, v, ldv, hv, ldhv, nvec=1, stream=None):
    _check(_lib.moto_euclid_hvp(ctx, _ptr(v), int(ldv), _ptr(hv), int(ldhv), int(nvec), _stream(stream)),
           "moto_euclid_hvp")


def moto_lowest_modes(ctx, m, s, params, v0, V, lam, info=None, stream=None):
    _check(_lib.moto_lowest_modes(ctx, _ptr(m), _ptr(s), ctypes.byref(params), _ptr(v0), _ptr(V), _ptr(lam),
                                  _ptr(info), _stream(stream)), "moto_lowest_modes")


def moto_gram(ctx, X, ldx, nx, Y, ldy, ny, out, stream=None):
    _check(_lib.moto_gram(ctx, _ptr(X), int(ldx), int(nx), _ptr(Y), int(ldy), int(ny), _ptr(out),
                          _stream(stream)), "moto_gram")


def moto_set_pairs(ctx, pairs):
    """pairs: sequence of (d1, d2, J, (Dx, Dy, Dz)); empty restores the shells."""
    arr = (moto_pair * max(len(pairs), 1))()
    for i, (d1, d2, J, D) in enumerate(pairs):
        arr[i].d1, arr[i].d2, arr[i].J = int(d1), int(d2), float(J)
        for c in range(3):
            arr[i].D[c] = float(D[c])
    _check(_lib.moto_set_pairs(ctx, arr, len(pairs)), "moto_set_pairs")


def moto_perturb(ctx, x0, mask, delta, ld_delta, count, out, ld_out, stream=None):
    _check(_lib.moto_perturb(ctx, _ptr(x0), _ptr(mask), _ptr(delta), int(ld_delta), int(count), _ptr(out),
                             int(ld_out), _stream(stream)), "moto_perturb")


def moto_pairwise_l1(ctx, X, ldx, count, D, stream=None):
    _check(_lib.moto_pairwise_l1(ctx, _ptr(X), int(ldx), int(count), _ptr(D), _stream(stream)),
           "moto_pairwise_l1")


def moto_topo_charge(ctx, m, Q, stream=None):
    _check(_lib.moto_topo_charge(ctx, _ptr(m), _ptr(Q), _stream(stream)), "moto_topo_charge")


def moto_lbfgs_reset(ctx, stream=None):
    _check(_lib.moto_lbfgs_reset(ctx, _stream(stream)), "moto_lbfgs_reset")


def moto_mmf_step(ctx, m, params, V, out=None, status=None, stream=None):
    _check(_lib.moto_mmf_step(ctx, _ptr(m), ctypes.byref(params), _ptr(V), _ptr(out), _ptr(status),
                              _stream(stream)), "moto_mmf_step")


def moto_ascend(ctx, m, params, V, trace=None, check_every=10, stream=None):
    """Returns (code, steps); code is MOTO_OK at a saddle, MOTO_NOT_CONVERGED at the cap."""
    steps = ctypes.c_int(0)
    rc = _lib.moto_ascend(ctx, _ptr(m), ctypes.byref(params), _ptr(V), _ptr(trace), int(check_every),
                          ctypes.byref(steps), _stream(stream))
    _check(rc, "moto_ascend", ok=(MOTO_OK, MOTO_NOT_CONVERGED))
    return rc, steps.value


def moto_descend(ctx, m_saddle, v1, params, m_plus, m_minus, out, stream=None):
    rc = _lib.moto_descend(ctx, _ptr(m_saddle), _ptr(v1), ctypes.byref(params), _ptr(m_plus), _ptr(m_minus),
                           _ptr(out), _stream(stream))
    _check(rc, "moto_descend", ok=(MOTO_OK, MOTO_NOT_CONVERGED))
    return rc


def moto_hvp_tuning(ctx):
    """(variant in use, [ms per launch of each variant, zeros unless this
    context ran the autotuner])."""
    v = ctypes.c_int()
    ms = (ctypes.c_float * 16)()
    n = _lib.moto_hvp_tuning(ctx, ctypes.byref(v), ms, 16)
    if n < 0:
        raise MotoError(f"moto_hvp_tuning: {moto_status_string(n)}")
    return v.value, [float(ms[i]) for i in range(n)]


def moto_krylov_basis(ctx, stream=None):
    """(device address of the last block Lanczos basis, element stride,
    number of basis fields, steps with a full reorthogonalisation pass)."""
    b, ld, nv, nr = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.moto_krylov_basis(ctx, ctypes.byref(b), ctypes.byref(ld), ctypes.byref(nv), ctypes.byref(nr),
                                  _stream(stream)), "moto_krylov_basis")
    return b.value, ld.value, nv.value, nr.value


def moto_stencil_tuning(ctx):
    """(energy-stencil variant in use, [ms per launch of each variant, zeros
    unless this context ran the autotuner])."""
    v = ctypes.c_int()
    ms = (ctypes.c_float * 8)()
    n = _lib.moto_stencil_tuning(ctx, ctypes.byref(v), ms, 8)
    if n < 0:
        raise MotoError(f"moto_stencil_tuning: {moto_status_string(n)}")
    return v.value, [float(ms[i]) for i in range(n)]


def moto_set_stencil_variant(ctx, variant: int):
    _check(_lib.moto_set_stencil_variant(ctx, int(variant)), "moto_set_stencil_variant")


def moto_set_hvp_variant(ctx, variant: int):
    _check(_lib.moto_set_hvp_variant(ctx, int(variant)), "moto_set_hvp_variant")


def moto_set_wait_limit(ctx, polls: int):
    """Bound of the streaming kernel's consumer waits (0 = default); a test
    hook for the timeout path."""
    _check(_lib.moto_set_wait_limit(ctx, int(polls)), "moto_set_wait_limit")


def moto_status(ctx, stream=None) -> int:
    return _lib.moto_status(ctx, _stream(stream))


def moto_clear_status(ctx, stream=None):
    _check(_lib.moto_clear_status(ctx, _stream(stream)), "moto_clear_status")


def moto_status_string(code: int) -> str:
    return _lib.moto_status_string(int(code)).decode()


def moto_workspace_bytes(ctx) -> int:
    return int(_lib.moto_workspace_bytes(ctx))


def moto_energy_grad_noalloc(model: moto_model, dtype: int, m, g=None, s=None, out=None, stream=None):
    """Energy and Riemannian gradient without a context: for callers that
    cannot allocate device memory (see include/moto.h)."""
    _check(_lib.moto_energy_grad_noalloc(ctypes.byref(model), int(dtype), _ptr(m), _ptr(g), _ptr(s), _ptr(out),
                                         _stream(stream)), "moto_energy_grad_noalloc")


def moto_batch_create(model: moto_model, dtype: int, params: moto_params, walkers, n_streams=8) -> int:
    """walkers: sequence of (L1, L2, m, V) with m, V CUDA tensors or device pointers."""
    arr = (moto_walker * len(walkers))()
    for i, (L1, L2, m, V) in enumerate(walkers):
        arr[i].L1, arr[i].L2, arr[i].m_dev, arr[i].V_dev = int(L1), int(L2), _ptr(m), _ptr(V)
    h = ctypes.c_void_p()
    _check(_lib.moto_batch_create(ctypes.byref(model), int(dtype), ctypes.byref(params), arr, len(walkers),
                                  int(n_streams), ctypes.byref(h)), "moto_batch_create")
    return h.value


def moto_batch_destroy(batch: int) -> None:
    _lib.moto_batch_destroy(batch)


def moto_batch_ascend(batch, n, rec, check_every=10, stream=None):
    """Returns (code, per-walker codes, per-walker steps)."""
    status = (ctypes.c_int * n)()
    steps = (ctypes.c_int * n)()
    rc = _lib.moto_batch_ascend(batch, int(check_every), _ptr(rec), ctypes.cast(status, ctypes.c_void_p),
                                ctypes.cast(steps, ctypes.c_void_p), _stream(stream))
    _check(rc, "moto_batch_ascend", ok=(MOTO_OK, MOTO_NOT_CONVERGED))
    return rc, list(status), list(steps)


def moto_batch_descend(batch, m_plus, m_minus, out, stream=None):
    """m_plus, m_minus: sequences of CUDA tensors; returns (code, per-walker codes)."""
    n = len(m_plus)
    mp = (ctypes.c_void_p * n)(*[_ptr(x) for x in m_plus])
    mm = (ctypes.c_void_p * n)(*[_ptr(x) for x in m_minus])
    status = (ctypes.c_int * n)()
    rc = _lib.moto_batch_descend(batch, ctypes.cast(mp, ctypes.c_void_p), ctypes.cast(mm, ctypes.c_void_p),
                                 _ptr(out), ctypes.cast(status, ctypes.c_void_p), _stream(stream))
    _check(rc, "moto_batch_descend", ok=(MOTO_OK, MOTO_NOT_CONVERGED))
    return rc, list(status)


def moto_profile_begin(ctx, capacity=8192):
    _check(_lib.moto_profile_begin(ctx, int(capacity)), "moto_profile_begin")


def moto_profile_end(ctx):
    """Returns {kind: (launches, ms, algorithmic bytes)} for the recorded launches."""
    n = len(PROFILE_KINDS)
    launches = (ctypes.c_int * n)()
    ms = (ctypes.c_double * n)()
    nbytes = (ctypes.c_double * n)()
    _check(_lib.moto_profile_end(ctx, n, ctypes.cast(launches, ctypes.c_void_p), ctypes.cast(ms, ctypes.c_void_p),
                                 ctypes.cast(nbytes, ctypes.c_void_p)), "moto_profile_end")
    return {k: (launches[i], ms[i], nbytes[i]) for i, k in enumerate(PROFILE_KINDS)}


from .context import Batch, Context  # noqa: E402,F401
from .autograd import MotoEnergy, energy  # noqa: E402,F401
