"""GPU parity of the outer layer on the 32 x 32 single-walker workload (FP64):
the reflected-force ascent must retrace the oracle's trajectory step by step,
stop at the same index-1 saddle, and the two-sided descent must reach the same
two minima with bit-equal integer Q."""
import numpy as np
import pytest
import torch

import inputs
from oracle import mmf, spin, topo
from gpu_util import context, require_gpu, to_dev, to_np, workload_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def oracle_run():
    M = workload_model(1)
    m0 = inputs.workload1_state()
    q0 = inputs.gaussian_field(inputs.workload_seed(1, 0), 32, 32, offset=10**6)
    P = mmf.MMFParams()
    res = mmf.ascend(M, m0, [q0], P)
    plus, minus = mmf.descend(M, res.m, res.v1, P)
    return M, m0, q0, P, res, plus, minus


@pytest.fixture(scope="module")
def gpu_run(oracle_run):
    require_gpu()
    M, m0, q0, P, res, plus, minus = oracle_run
    ctx = context(M, torch.float64)
    m = to_dev(m0, torch.float64)
    V = to_dev(q0, torch.float64)[None].contiguous()
    rc, steps, trace = ctx.ascend(m, V, check_every=10)
    rc2, mp, mm, out = ctx.descend(m, V[0].contiguous())
    r = dict(rc=rc, steps=steps, trace=to_np(trace), m=to_np(m), v1=to_np(V[0]), rc2=rc2, mp=to_np(mp),
             mm=to_np(mm), out=to_np(out))
    ctx.close()
    return r


def test_ascent_retraces_the_oracle(oracle_run, gpu_run):
    M, m0, q0, P, res, plus, minus = oracle_run
    assert res.converged and gpu_run["rc"] == 0
    assert gpu_run["steps"] == res.steps
    tr = gpu_run["trace"]
    for t, row in enumerate(res.trace):
        assert tr[t, 0] == pytest.approx(row["E"], abs=1e-7)
        assert tr[t, 1] == pytest.approx(row["fmax"], rel=1e-5, abs=1e-9)
        assert tr[t, 2] == pytest.approx(row["lam1"], rel=1e-5, abs=1e-9)
        assert tr[t, 3] == pytest.approx(row["lam2"], rel=1e-5, abs=1e-9)


def test_saddle_matches_and_is_index1(oracle_run, gpu_run):
    M, m0, q0, P, res, plus, minus = oracle_run
    E_gpu = spin.energy(M, gpu_run["m"])
    assert E_gpu == pytest.approx(spin.energy(M, res.m), abs=1e-4)
    dev = np.sqrt(np.max(np.sum((gpu_run["m"] - res.m) ** 2, axis=0)))
    assert dev < 1e-3
    w = np.linalg.eigvalsh(spin.dense_tangent_hessian(M, gpu_run["m"])[0])
    assert w[0] < 0.0 < w[1]


def test_descent_minima_and_charges(oracle_run, gpu_run):
    M, m0, q0, P, res, plus, minus = oracle_run
    out = gpu_run["out"]
    assert gpu_run["rc2"] == 0
    E_p, Q_p, E_m, Q_m = out[:4]
    assert int(round(Q_p)) == plus.Qint and int(round(Q_m)) == minus.Qint
    assert E_p == pytest.approx(plus.E, abs=1e-4)
    assert E_m == pytest.approx(minus.E, abs=1e-4)
    assert E_p == pytest.approx(spin.energy(M, gpu_run["mp"]), abs=1e-9)
    assert Q_p == pytest.approx(topo.topo_charge(gpu_run["mp"]), abs=1e-9)
    for mm in (gpu_run["mp"], gpu_run["mm"]):
        g, _ = spin.riemann_grad(M, mm)
        assert mmf.max_torque(g) <= P.tau_F * (1 + 1e-9)


@pytest.mark.parametrize("dtype,L,extra", [
    (torch.float64, 32, dict()),
    (torch.float32, 64, dict(k=2, block=2, krylov_steps=20, reorth=1)),
])
def test_graph_replay_matches_plain_launches(monkeypatch, dtype, L, extra):
    """The outer loop replays a captured step as a CUDA graph, the records
    indexed on the device; launching every kernel one by one (MOTO_GRAPHS=0)
    must give the same trajectory bit for bit, ascent and descent."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    if extra.get("reorth") == 1:
        extra = dict(extra, reorth=mo.MOTO_REORTH_SELECTIVE)
    M = workload_model(1, L, L)
    m0 = inputs.add_noise(inputs.skyrmion(L, L, 4.0), 0.01, inputs.workload_seed(1, 7))
    nv = extra.get("block", 1)
    V0 = np.stack([inputs.gaussian_field(inputs.workload_seed(1, 30 + j), L, L) for j in range(nv)])
    runs = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("MOTO_GRAPHS", graphs)
        ctx = context(M, dtype, max_steps=25, descent_max_steps=40, **extra)
        m = to_dev(m0, dtype)
        V = to_dev(V0, dtype).contiguous()
        rc, steps, trace = ctx.ascend(m, V, check_every=7)
        rc2, mp, mm, out = ctx.descend(m, V[0].contiguous())
        runs.append(dict(rc=rc, steps=steps, trace=to_np(trace), m=to_np(m), V=to_np(V), mp=to_np(mp),
                         mm=to_np(mm), out=to_np(out)))
        ctx.close()
    a, b = runs
    assert a["steps"] == b["steps"] and a["rc"] == b["rc"] and a["steps"] >= 3
    assert np.isfinite(a["trace"]).all()
    for key in ("trace", "m", "V", "mp", "mm", "out"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_repeated_mmf_step_replays_bit_identically(monkeypatch):
    """moto_mmf_step called again with the same arguments replays a captured
    CUDA graph of the step; the states, records and status words must equal
    those of the kernel-by-kernel launches (MOTO_GRAPHS=0) bit for bit, also
    across a change of parameters between calls."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    L = 64
    M = workload_model(1, L, L)
    m0 = inputs.add_noise(inputs.skyrmion(L, L, 4.0), 0.01, inputs.workload_seed(1, 9))
    V0 = np.stack([inputs.gaussian_field(inputs.workload_seed(1, 40 + j), L, L) for j in range(2)])
    runs = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("MOTO_GRAPHS", graphs)
        ctx = context(M, torch.float32, k=2, block=2, krylov_steps=16)
        m = to_dev(m0, torch.float32)
        V = to_dev(V0, torch.float32).contiguous()
        out = torch.empty(6, dtype=torch.float64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        p2 = mo.make_params(**{f: getattr(ctx.params, f) for f, _ in ctx.params._fields_})
        p2.reorth = mo.MOTO_REORTH_SELECTIVE
        recs = []
        for t in range(10):
            mo.moto_mmf_step(ctx.handle, m, ctx.params if t < 6 else p2, V, out, status)
            recs.append(np.concatenate([to_np(out), to_np(status)]))
        runs.append(dict(recs=np.stack(recs), m=to_np(m), V=to_np(V)))
        ctx.close()
    a, b = runs
    assert np.isfinite(a["recs"]).all()
    for key in ("recs", "m", "V"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_step_graph_follows_a_change_of_model(monkeypatch):
    """A captured moto_mmf_step graph bakes in the model; moto_set_pairs must
    discard it, so steps after the switch to a pair-list Hamiltonian equal
    those of a context that launched every kernel (bit for bit), and differ
    from the shell model's."""
    require_gpu()
    import paper_2509_26269_gb300 as mo
    L = 64
    M = workload_model(1, L, L)
    pl = inputs.random_pairs(41, reach=3, n_offsets=12)
    m0 = inputs.add_noise(inputs.skyrmion(L, L, 4.0), 0.01, inputs.workload_seed(1, 11))
    V0 = np.stack([inputs.gaussian_field(inputs.workload_seed(1, 50 + j), L, L) for j in range(2)])
    runs = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("MOTO_GRAPHS", graphs)
        ctx = context(M, torch.float32, k=2, block=2, krylov_steps=16)
        m = to_dev(m0, torch.float32)
        V = to_dev(V0, torch.float32).contiguous()
        out = torch.empty(6, dtype=torch.float64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        recs = []
        for t in range(6):
            if t == 3:
                ctx.set_pairs(pl)
            mo.moto_mmf_step(ctx.handle, m, ctx.params, V, out, status)
            recs.append(to_np(out).copy())
        runs.append(dict(recs=np.stack(recs), m=to_np(m)))
        ctx.close()
    a, b = runs
    np.testing.assert_array_equal(a["recs"], b["recs"])
    np.testing.assert_array_equal(a["m"], b["m"])
    # the energy of step 3 is the pair model's, not a continuation of the shells'
    assert abs(a["recs"][3, 0] - a["recs"][2, 0]) > 1e-3 * abs(a["recs"][2, 0])
