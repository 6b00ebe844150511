"""Batched walkers on the GPU: a batch of independent walkers (mixed lattice
sizes, one CUDA graph per outer step) must give exactly what each walker
gives alone through the one-walker entry points (same kernels in the same
order per walker), and its certified saddles must pass the oracle's checks."""
import numpy as np
import pytest
import torch

import inputs
from oracle import spin
from oracle.model import Model
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


def _walkers(sizes, dtype, nv, seed0):
    out = []
    for w, (L1, L2) in enumerate(sizes):
        m = inputs.add_noise(inputs.skyrmion(L1, L2, 0.2 * min(L1, L2)), 0.05, seed0 + w)
        V = np.stack([inputs.gaussian_field(seed0 + 100 * w + j, L1, L2) for j in range(nv)])
        out.append((m, V))
    return out


def _run_batch(walkers, dtype, params):
    from paper_2509_26269_gb300 import Batch
    dev = [(to_dev(m, dtype), to_dev(V, dtype)) for m, V in walkers]
    b = Batch(dev, J=FULL["J"], D=FULL["D"], K=FULL["K"], muB=FULL["muB"], dtype=dtype, n_streams=4, **params)
    rc, status, steps, rec = b.ascend(check_every=10)
    rc2, status2, mp, mm, out = b.descend()
    res = dict(status=status, steps=steps, rec=to_np(rec), m=[to_np(m) for m, _ in dev], V=[to_np(V) for _, V in dev],
               status2=status2, mp=[to_np(x) for x in mp], mm=[to_np(x) for x in mm], out=to_np(out))
    b.close()
    return res


def _run_single(walkers, dtype, params):
    res = dict(status=[], steps=[], rec=[], m=[], V=[], status2=[], mp=[], mm=[], out=[])
    for m_np, V_np in walkers:
        L2, L1 = m_np.shape[1:]
        ctx = context(Model(L1, L2, **FULL), dtype, **params)
        m, V = to_dev(m_np, dtype), to_dev(V_np, dtype)
        rc, steps, trace = ctx.ascend(m, V, check_every=10)
        rc2, mp, mm, out = ctx.descend(m, V[0].contiguous())
        res["status"].append(rc)
        res["steps"].append(steps)
        res["rec"].append(to_np(trace[-1]))
        res["m"].append(to_np(m))
        res["V"].append(to_np(V))
        res["status2"].append(rc2)
        res["mp"].append(to_np(mp))
        res["mm"].append(to_np(mm))
        res["out"].append(to_np(out))
        ctx.close()
    return res


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batch_equals_walkers_run_alone(dtype):
    """Walkers of equal lattices form one group whose every kernel runs once
    for all of them (walker = blockIdx.z): three 20 x 20 walkers, two 24 x 18,
    one 16 x 16.  Each walker's per-walker grids are those of a lone walker,
    so the results are bit-equal."""
    require_gpu()
    sizes = [(20, 20), (24, 18), (16, 16), (20, 20), (20, 20), (24, 18)]
    params = dict(k=1, block=1, krylov_steps=40, max_steps=120, descent_max_steps=400)
    walkers = _walkers(sizes, dtype, 1, 4100)
    b = _run_batch(walkers, dtype, params)
    s = _run_single(walkers, dtype, params)
    assert b["status"] == s["status"]
    assert b["steps"] == s["steps"]
    for i in range(len(sizes)):
        np.testing.assert_array_equal(b["m"][i], s["m"][i])
        np.testing.assert_array_equal(b["V"][i], s["V"][i])
        np.testing.assert_array_equal(b["rec"][i], s["rec"][i])
        np.testing.assert_array_equal(b["mp"][i], s["mp"][i])
        np.testing.assert_array_equal(b["mm"][i], s["mm"][i])
        np.testing.assert_array_equal(b["out"][i][:4], s["out"][i][:4])


@pytest.mark.parametrize("dtype", [torch.float32])
def test_batch_block_lanczos_selective_group(dtype):
    """A group of four equal walkers with k = 2 block Lanczos and selective
    reorthogonalisation (the saddle-search configuration of the batched
    explorer) equals the walkers run alone."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    sizes = [(24, 24)] * 4
    params = dict(k=2, block=2, krylov_steps=12, max_steps=60, descent_max_steps=200,
                  reorth=mo.MOTO_REORTH_SELECTIVE, tau_lambda=1e-4)
    walkers = _walkers(sizes, dtype, 2, 4300)
    b = _run_batch(walkers, dtype, params)
    s = _run_single(walkers, dtype, params)
    assert b["status"] == s["status"]
    assert b["steps"] == s["steps"]
    for i in range(len(sizes)):
        np.testing.assert_array_equal(b["m"][i], s["m"][i])
        np.testing.assert_array_equal(b["V"][i], s["V"][i])
        np.testing.assert_array_equal(b["rec"][i], s["rec"][i])
        np.testing.assert_array_equal(b["mp"][i], s["mp"][i])
        np.testing.assert_array_equal(b["out"][i][:4], s["out"][i][:4])


def test_batch_with_cg_runs_walkers_alone():
    """Nonlinear CG has no walker dimension: each walker is a group of one,
    and the batch still equals the walkers run alone."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    sizes = [(20, 20), (20, 20)]
    params = dict(k=2, block=2, krylov_steps=15, max_steps=80, descent_max_steps=200, optimizer=mo.MOTO_OPT_CG)
    walkers = _walkers(sizes, torch.float64, 2, 4500)
    b = _run_batch(walkers, torch.float64, params)
    s = _run_single(walkers, torch.float64, params)
    assert b["status"] == s["status"] and b["steps"] == s["steps"]
    for i in range(len(sizes)):
        np.testing.assert_array_equal(b["m"][i], s["m"][i])
        np.testing.assert_array_equal(b["rec"][i], s["rec"][i])


def oracle_certify(M, m_gpu, V_gpu, steps=30, dense_max_sites=1600, max_refine=50, tau_lambda=0.0):
    """The saddle rule for a saddle found in FP32 (MMF is path-dependent, so
    the oracle checks the end point rather than the trajectory): at the GPU's
    spins, in FP64, the oracle recomputes the gradient, its own two lowest
    modes (block Lanczos from the GPU modes) and the reflected force; then
    refines with its own MMF ascent (at most 50 steps) from the GPU's spins.
    Returns a dict of what the checks need."""
    from oracle import krylov, mmf
    g, s = spin.riemann_grad(M, m_gpu)
    lam, V = krylov.block_lanczos_modes(M, m_gpu, s, [V_gpu[0], V_gpu[1]], steps, 2)
    Fm = mmf.reflected_force(-g, V[0])
    P = mmf.MMFParams(k=2, solver="block_lanczos", krylov_steps=steps, max_steps=max_refine, tau_F=1e-3,
                      tau_lambda=tau_lambda)
    res = mmf.ascend(M, m_gpu, [V_gpu[0], V_gpu[1]], P)
    out = dict(lam=lam, fmax=mmf.max_torque(Fm), refine=res,
               dE=abs(spin.energy(M, res.m) - spin.energy(M, m_gpu)),
               dev=float(np.sqrt(np.max(np.sum((res.m - m_gpu) ** 2, axis=0)))))
    if M.N <= dense_max_sites:
        out["dense"] = np.linalg.eigvalsh(spin.dense_tangent_hessian(M, res.m)[0])[:3]
    return out


def test_batched_walkers_certify_saddles_fp32():
    """Explorer-style walkers (random charge, masked perturbation) on mixed
    lattices, k = 2 block Lanczos, FP32.  Every walker the batch reports at a
    saddle is certified by the oracle in FP64 on its stored spins: the oracle's
    own minimum modes give the index-1 signature and a reflected force within
    a few times tau_F, and its own MMF ascent started there converges within 50
    steps to a saddle within 1e-4 meV and 1e-3 rad of the GPU's, index 1 in the
    dense spectrum where the lattice is small enough (N <= 1600).  The
    signature is read with the curvature threshold tau_lambda = 1e-4 meV (R22):
    these textures have a soft translation mode, |lambda_2| ~ 1e-5 meV, below
    what FP32 curvatures resolve against |H| ~ 20 meV."""
    require_gpu()
    sides = [32, 40, 48, 32, 40, 48]
    # these walkers reach their saddles in a few hundred to a few thousand outer steps
    tl = 1e-4
    params = dict(k=2, block=2, krylov_steps=30, max_steps=4000, tau_F=1e-3, tau_lambda=tl)
    walkers = []
    for w, L in enumerate(sides):
        m = inputs.workload3_walker(w, L)
        V = np.stack([inputs.gaussian_field(inputs.workload_seed(3, 500 + 10 * w + j), L, L) for j in range(2)])
        walkers.append((m, V))
    from paper_2509_26269_gb300 import Batch
    dev = [(to_dev(m, torch.float32), to_dev(V, torch.float32)) for m, V in walkers]
    b = Batch(dev, J=FULL["J"], D=FULL["D"], K=FULL["K"], muB=FULL["muB"], dtype=torch.float32, n_streams=3,
              **params)
    rc, status, steps, rec = b.ascend(check_every=10)
    rec = to_np(rec)
    ok = 0
    for i, (L, code) in enumerate(zip(sides, status)):
        assert code in (0, 1)
        if code != 0:
            continue
        ok += 1
        M = Model(L, L, **FULL)
        mo = to_np(dev[i][0])
        Vo = to_np(dev[i][1])
        # the GPU's record describes the stored spins (FP32 force below tau_F)
        assert rec[i, 1] <= params["tau_F"]
        assert spin.energy(M, mo) == pytest.approx(rec[i, 0], rel=1e-6)
        c = oracle_certify(M, mo, Vo, tau_lambda=tl)
        assert c["lam"][0] < -tl and c["lam"][1] > -tl, (i, c["lam"][:3])
        assert c["fmax"] <= 5 * params["tau_F"], (i, c["fmax"])
        assert c["refine"].converged and c["refine"].steps <= 50, (i, c["refine"].steps)
        assert c["dE"] <= 1e-4, (i, c["dE"])
        assert c["dev"] < 1e-3, (i, c["dev"])
        if "dense" in c:
            assert c["dense"][0] < -tl and c["dense"][1] > -tl, (i, c["dense"])
    assert ok >= 4
    b.close()
