"""A small convenience wrapper that owns one ``moto_ctx`` and allocates the
output tensors of each call.  Fields are torch CUDA tensors of shape
(3, L2, L1) (component-major, site (i1, i2) at [:, i2, i1]); scalars come back
as float64 CUDA tensors.  No arithmetic happens here."""
from __future__ import annotations

import torch

from . import (MOTO_F32, MOTO_F64, MOTO_MAX_BASIS, make_model, make_params, moto_ascend, moto_batch_ascend,
               moto_batch_create, moto_batch_descend, moto_batch_destroy, moto_create, moto_descend, moto_destroy,
               moto_energy, moto_energy_grad, moto_hvp, moto_lbfgs_reset, moto_lowest_modes, moto_mmf_step,
               moto_pairwise_l1, moto_perturb, moto_set_pairs, moto_topo_charge, moto_workspace_bytes)


class Context:
    def __init__(self, L1, L2, J=(1.0,), D=0.0, K=0.0, muB=0.0, dtype=torch.float32, device="cuda", **params):
        self.L1, self.L2 = int(L1), int(L2)
        self.N = self.L1 * self.L2
        self.dtype = dtype
        dev = torch.device(device)
        if dev.type == "cuda" and dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.params = make_params(**params)
        code = MOTO_F64 if dtype == torch.float64 else MOTO_F32
        with torch.cuda.device(self.device):
            self.handle = moto_create(make_model(L1, L2, J, D, K, muB), code, self.params)

    # -- helpers ---------------------------------------------------------------
    def field(self, n=None):
        shape = (3, self.L2, self.L1) if n is None else (n, 3, self.L2, self.L1)
        return torch.empty(shape, dtype=self.dtype, device=self.device)

    def _p(self, **kw):
        if not kw:
            return self.params
        p = make_params()
        for name, _ in type(p)._fields_:
            setattr(p, name, getattr(self.params, name))
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    @property
    def workspace_bytes(self):
        return moto_workspace_bytes(self.handle)

    # -- calls -----------------------------------------------------------------
    def energy_grad(self, m):
        g = self.field()
        s = torch.empty((self.L2, self.L1), dtype=self.dtype, device=self.device)
        out = torch.empty(2, dtype=torch.float64, device=self.device)
        moto_energy_grad(self.handle, m, g, s, out)
        return out, g, s

    def energy(self, m):
        E = torch.empty(1, dtype=torch.float64, device=self.device)
        moto_energy(self.handle, m, E)
        return E

    def hvp(self, m, s, v):
        """v: (3, L2, L1) or (n, 3, L2, L1) tangent fields."""
        many = v.dim() == 4
        hv = torch.empty_like(v)
        n = v.shape[0] if many else 1
        moto_hvp(self.handle, m, s, v, 3 * self.N, hv, 3 * self.N, n)
        return hv

    def lowest_modes(self, m, v0, s=None, **kw):
        p = self._p(**kw)
        V = self.field(p.k)
        lam = torch.empty(MOTO_MAX_BASIS, dtype=torch.float64, device=self.device)
        info = torch.zeros(2, dtype=torch.int32, device=self.device)
        moto_lowest_modes(self.handle, m, s, p, v0, V, lam, info)
        return lam, V, info

    def topo_charge(self, m):
        Q = torch.empty(1, dtype=torch.float64, device=self.device)
        moto_topo_charge(self.handle, m, Q)
        return Q

    def set_pairs(self, pairs):
        """Use a general pair-list Hamiltonian (``moto_set_pairs``): pairs is
        a sequence of (d1, d2, J, (Dx, Dy, Dz)); [] restores the shells."""
        moto_set_pairs(self.handle, list(pairs))

    def perturb(self, x0, delta, mask=None):
        """Masked perturbations R_x0(P_mask P_x0 delta_j) of x0 for a stack
        delta (count, 3, L2, L1); mask: (L2, L1) uint8 or None (all sites)."""
        count = delta.shape[0]
        out = self.field(count)
        n3 = 3 * self.N
        moto_perturb(self.handle, x0, mask, delta, n3, count, out, n3)
        return out

    def pairwise_l1(self, X):
        """count x count L1 distances of a stack X (count, 3, L2, L1)."""
        count = X.shape[0]
        D = torch.empty((count, count), dtype=torch.float64, device=self.device)
        moto_pairwise_l1(self.handle, X, 3 * self.N, count, D)
        return D

    def reset(self):
        moto_lbfgs_reset(self.handle)

    def mmf_step(self, m, V, **kw):
        p = self._p(**kw)
        out = torch.empty(6, dtype=torch.float64, device=self.device)
        status = torch.zeros(1, dtype=torch.int32, device=self.device)
        moto_mmf_step(self.handle, m, p, V, out, status)
        return out, status

    def ascend(self, m, V, check_every=10, **kw):
        p = self._p(**kw)
        trace = torch.full((p.max_steps + 1, 6), float("nan"), dtype=torch.float64, device=self.device)
        rc, steps = moto_ascend(self.handle, m, p, V, trace, check_every)
        return rc, steps, trace[: steps + 1]

    def descend(self, m_saddle, v1, **kw):
        p = self._p(**kw)
        mp, mm = self.field(), self.field()
        out = torch.empty(6, dtype=torch.float64, device=self.device)
        rc = moto_descend(self.handle, m_saddle, v1, p, mp, mm, out)
        return rc, mp, mm, out

    def close(self):
        if getattr(self, "handle", None):
            moto_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent MMF walkers advanced together (``moto_batch_*``).  ``walkers``
    is a list of (m, V): spins (3, L2, L1) and start block (nv, 3, L2, L1), all
    of one dtype on one device; both are updated in place."""

    def __init__(self, walkers, J=(1.0,), D=0.0, K=0.0, muB=0.0, dtype=torch.float32, n_streams=8, **params):
        self.walkers = [(m, V) for m, V in walkers]
        self.dtype = dtype
        self.device = self.walkers[0][0].device
        self.params = make_params(**params)
        code = MOTO_F64 if dtype == torch.float64 else MOTO_F32
        desc = []
        for m, V in self.walkers:
            if m.dtype != dtype or V.dtype != dtype or not m.is_contiguous() or not V.is_contiguous():
                raise TypeError("walker tensors must be contiguous and of the batch dtype")
            desc.append((m.shape[-1], m.shape[-2], m, V))
        with torch.cuda.device(self.device):
            self.handle = moto_batch_create(make_model(5, 5, J, D, K, muB), code, self.params, desc, n_streams)

    def ascend(self, check_every=10):
        rec = torch.full((len(self.walkers), 6), float("nan"), dtype=torch.float64, device=self.device)
        rc, status, steps = moto_batch_ascend(self.handle, len(self.walkers), rec, check_every)
        return rc, status, steps, rec

    def descend(self):
        mp = [torch.empty_like(m) for m, _ in self.walkers]
        mm = [torch.empty_like(m) for m, _ in self.walkers]
        out = torch.full((len(self.walkers), 6), float("nan"), dtype=torch.float64, device=self.device)
        rc, status = moto_batch_descend(self.handle, mp, mm, out)
        return rc, status, mp, mm, out

    def close(self):
        if getattr(self, "handle", None):
            moto_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
