"""HYB spill: rows with more in-domain successors than the row cap.

The paper sizes the neighbouring sub-grid so that every landing fits
(Sec. III-B); under a high-sigma field a (state, action) row then reaches more
distinct successor cells than the sliced-ELL width keeps (64 by default).  The
build keeps a row's first row_cap successors in the slice's ELL columns and
the rest, in the same ascending order, in the slice's spill block; every sweep
sums the ELL columns and then the spill entries, i.e. the row in its plain
ascending order.

  check mode     spilled models (the default cap with rows of up to ~115
                 successors, and a cap of 6 where most rows spill) against the
                 oracle's build (Alg. 2) and value iteration (Sec. II-B):
                 counts and successor lists bit-identical, R and V within
                 1e-12, policy equal; 32 actions (the warp-specialized sweep),
                 16 actions (two states per slice) and 12 actions (padding
                 lanes), fused objectives, Jacobi and the layered pass.
  FP32           a model whose rows spill equals the same model built with a
                 cap above every row bit for bit (export, values, policies),
                 through the warp kernel and through the full-window kernel;
                 the FP32 build gate against the oracle.
  around it      the allocation-free solve, a served request (charged again
                 for its spill area, never above its charge) and the batch's
                 refusal.
"""
import numpy as np
import pytest

import oracle
from conftest import device_pool_meter, policy_tie_check
from paper_2109_00857_gb300 import inputs

pytestmark = pytest.mark.gpu

# sigma of the modes large against a cell: rows of up to ~115 in-domain
# successors, a quarter of the rows beyond 64; the 41x41 sub-grid holds every
# landing
HIGH_SIGMA = dict(nx=20, ny=18, nt=4, K=3, N=600, L=41, sigma=(2.0, 1.5, 1.0), seed=41,
                  amplitude=1.0, obstacle="squares", square=4)


def high_sigma(n_headings=16, n_speeds=2, **kw):
    args = dict(HIGH_SIGMA, n_headings=n_headings, n_speeds=n_speeds)
    args.update(kw)
    return inputs.make_env(**args)


@pytest.fixture(scope="module")
def mdp():
    import torch
    torch.cuda.set_device(0)
    from paper_2109_00857_gb300 import build_native, mdp as m
    build_native.build()
    m.load()
    return m


def build(mdp, env, precision, row_cap=0, hist_cap=0, objs=None):
    opts = mdp.MdpBuildOpts(row_cap=row_cap, hist_cap=hist_cap)
    return mdp.mdp_build(mdp.DeviceEnv(env, precision), objs=objs or env.objectives, opts=opts)


def export_np(mdp, model, obj=0):
    rp, col, cnt, R = mdp.mdp_export_csr(model, obj)
    return rp.cpu().numpy(), col.cpu().numpy(), cnt.cpu().numpy(), R.cpu().numpy()


def domain_lengths(ref, nS):
    """In-domain successors per row of an oracle model (the sink, col = |S|, apart)."""
    dom = (ref.col < nS).astype(np.int64)
    return np.add.reduceat(dom, ref.rowptr[:-1]) * (np.diff(ref.rowptr) > 0)


ACTIONS = {"A32": (16, 2), "A16": (16, 1), "A12": (12, 1)}


@pytest.mark.parametrize("row_cap", [0, 6])
@pytest.mark.parametrize("actions", sorted(ACTIONS))
def test_check_mode_spilled_model_matches_the_oracle(mdp, actions, row_cap):
    env = high_sigma(*ACTIONS[actions], with_gbar=True, objectives=(0, 1, 2))
    objs = env.objectives
    ref = oracle.build(env, objs=objs)
    assert ref.overflow == 0
    dl = domain_lengths(ref, env.nS)
    cap = row_cap or 64
    assert (dl > cap).sum() > 100   # the case really spills
    model = build(mdp, env, mdp.MDP_FP64_CHECK, row_cap=row_cap)
    info = model.info()
    assert info.spill_rows == int((dl > cap).sum())
    assert info.max_row_nnz == min(cap, int(dl.max())) and info.max_row_len == int(dl.max())
    assert info.nnz == len(ref.col)
    for o in range(len(objs)):
        rp, col, cnt, R = export_np(mdp, model, o)
        assert np.array_equal(rp, ref.rowptr)
        assert np.array_equal(col, ref.col)
        assert np.array_equal(cnt, ref.cnt)
        np.testing.assert_allclose(R, ref.R[o], rtol=1e-12, atol=1e-12)
    fx = oracle.fixed_mask(env)
    Vf, pf, sf = mdp.mdp_solve_multi(model, tuple(range(3)), method=mdp.MDP_SOLVE_JACOBI, tol=0.0)
    Vl, pl, sl = mdp.mdp_solve_multi(model, tuple(range(3)), method=mdp.MDP_SOLVE_LAYERED)
    for o in range(len(objs)):
        Vo, pio, sw, res = oracle.vi_jacobi(ref, ref.R[o], fx, tol=0.0, nt=env.nt)
        V1, p1, s1 = mdp.mdp_solve(model, o, tol=0.0)
        assert s1.sweeps == sw and sf[o].sweeps == sw
        for V, pi in ((V1, p1), (Vf[o], pf[o]), (Vl[o], pl[o])):
            np.testing.assert_allclose(V.cpu().numpy(), Vo, rtol=1e-12, atol=1e-12)
            assert np.array_equal(pi.cpu().numpy(), pio)


@pytest.mark.parametrize("actions", ["A32", "A16"])
def test_fp32_spilled_model_equals_the_unspilled_model_bit_for_bit(mdp, actions):
    """Against a build with a cap above every row: the same export; the same
    values and policies (32 actions: the unspilled model's solve; 16 actions,
    whose warp-per-slice sweep stages at most ~110 columns per slice: the
    default-cap model's, and every cap and kernel must agree with it)."""
    env = high_sigma(*ACTIONS[actions], with_gbar=True, objectives=(0, 1, 2))
    whole = build(mdp, env, mdp.MDP_FP32, row_cap=255)   # every row in the ELL columns
    assert whole.info().spill_rows == 0 and whole.info().max_row_nnz > 64
    ex_whole = [export_np(mdp, whole, o) for o in range(3)]
    ref_model = whole if actions == "A32" else build(mdp, env, mdp.MDP_FP32)
    Vw, pw, sw = mdp.mdp_solve_multi(ref_model, (0, 1, 2), tol=0.0)
    # the warp kernel (default fine tables) and the full-window kernel (every
    # sampled slice deferred) with a small cap and the default cap
    for row_cap, hist_cap in ((5, 0), (0, 0), (5, 1)):
        m = build(mdp, env, mdp.MDP_FP32, row_cap=row_cap, hist_cap=hist_cap)
        info = m.info()
        assert info.spill_rows > 0 and info.max_row_nnz <= (row_cap or 64)
        assert info.max_row_len == whole.info().max_row_nnz and info.nnz == whole.info().nnz
        for o in range(3):
            for x, y in zip(export_np(mdp, m, o), ex_whole[o]):
                assert np.array_equal(x, y), (row_cap, hist_cap, o)
        for method in (mdp.MDP_SOLVE_JACOBI, mdp.MDP_SOLVE_LAYERED, mdp.MDP_SOLVE_JACOBI_FULL):
            V, p, st = mdp.mdp_solve_multi(m, (0, 1, 2), method=method, tol=0.0)
            for o in range(3):
                assert np.array_equal(V[o].cpu().numpy(), Vw[o].cpu().numpy()), (row_cap, hist_cap, method, o)
                assert np.array_equal(p[o].cpu().numpy(), pw[o].cpu().numpy()), (row_cap, hist_cap, method, o)
        V1, p1, _ = mdp.mdp_solve(m, 1, tol=0.0)
        assert np.array_equal(V1.cpu().numpy(), Vw[1].cpu().numpy())


def test_fp32_spilled_build_and_solve_within_the_gates(mdp):
    """FP32 against the oracle: |d count| <= 2 per entry and full row sums;
    the solve on the exported model within the solver gate."""
    env = high_sigma()
    ref = oracle.build(env, objs=(0,))
    m = build(mdp, env, mdp.MDP_FP32, row_cap=8)
    assert m.info().spill_rows > 0
    rp, col, cnt, R = export_np(mdp, m, 0)
    for r in range(0, env.nS * env.A, 7):
        a = dict(zip(ref.col[ref.rowptr[r]:ref.rowptr[r + 1]].tolist(),
                     ref.cnt[ref.rowptr[r]:ref.rowptr[r + 1]].tolist()))
        for c_, n_ in zip(col[rp[r]:rp[r + 1]].tolist(), cnt[rp[r]:rp[r + 1]].tolist()):
            a[c_] = a.get(c_, 0) - n_
        assert all(abs(v) <= 2 for v in a.values()), r
        if rp[r + 1] > rp[r]:
            assert cnt[rp[r]:rp[r + 1]].sum() == env.N
    V, pi, st = mdp.mdp_solve(m, 0, tol=0.0)
    om = oracle.model_from_csr(env.nS, env.A, env.N, rp, col, cnt)
    R64 = R.astype(np.float64)
    Vo, pio, sw, res = oracle.vi_jacobi(om, R64, oracle.fixed_mask(env), tol=0.0, nt=env.nt)
    V = V.cpu().numpy().astype(np.float64)
    scale = np.maximum(1.0, np.abs(Vo))
    assert np.all(np.abs(V - Vo) <= 1e-5 * scale)
    policy_tie_check(pi.cpu().numpy(), pio, oracle.q_values(om, R64, Vo))


def test_allocation_free_solve_of_a_spilled_model(mdp):
    env = high_sigma()
    m = build(mdp, env, mdp.MDP_FP32, row_cap=6)
    V, pi, st = mdp.mdp_solve(m, 0, tol=0.0)
    Vn, pn, sn = mdp.mdp_solve_noalloc(m, 0, tol=0.0)
    assert np.array_equal(V.cpu().numpy(), Vn.cpu().numpy())
    assert np.array_equal(pi.cpu().numpy(), pn.cpu().numpy())
    assert st.sweeps == sn.sweeps


def test_served_request_with_spilled_rows(mdp):
    """A request whose rows spill: charged first without a spill area, charged
    again for the exact spill words and rebuilt; its device-memory peak stays
    within its charge and the result equals a direct build + solve."""
    import torch
    env = high_sigma()
    kw = dict(start=(3, 3), target=(15, 12), seed=9, N=600, objective=0)
    reset, read = device_pool_meter()
    srv = mdp.Server(8 << 30, 1)
    eid = srv.register(mdp.DeviceEnv(env, mdp.MDP_FP32))
    torch.cuda.synchronize()
    used0, _ = read()
    reset()
    res, V, pi = srv.poll(srv.submit(eid, **kw), timeout_ms=60000, env_id=eid, want_V=True)
    assert res.status == 0, mdp.load().mdp_last_error().decode()
    _, high = read()
    assert high - used0 <= res.device_bytes
    srv.close()
    e = inputs.Environment(**{**env.__dict__})
    e.target = inputs.target_block(env.nx, env.ny, *kw["target"])
    e.seed, e.N, e.mdp_id = kw["seed"], kw["N"], 0
    m = mdp.mdp_build(mdp.DeviceEnv(e, mdp.MDP_FP32), objs=(0,))
    assert m.info().spill_rows > 0
    Vd, pid, _ = mdp.mdp_solve(m, 0, tol=0.0)
    assert np.array_equal(V, Vd.cpu().numpy()) and np.array_equal(pi, pid.cpu().numpy())


def test_batch_refuses_a_member_with_spilled_rows(mdp):
    with pytest.raises(mdp.MdpError) as ex:
        mdp.Batch([mdp.DeviceEnv(high_sigma(), mdp.MDP_FP32)])
    assert "MDP_ERR_ELL_OVERFLOW" in str(ex.value)
