"""Parity at the large workload's own geometry: 200x200 cells, nt = 120,
K = 8 DO modes, N = 5000 realizations, 32 actions (16 headings x 2 speeds),
a 21x21 sub-grid and all three objectives from one build -- the sizes and the
launch configuration the benchmark times (warp-per-slice build, fused
three-objective active-layer Jacobi solve).

  build, two-layer cut   layers 60 and 61 of the large environment (with those
                         layers' coefficients), so layer 0 of the cut builds
                         exactly the large model's layer 60: 2,000 cells of it
                         (a band crossing an obstacle's edge and a band holding
                         the target) compared row by row with the oracle's
                         build (Alg. 2 in FP64): FP64 check mode bit for bit,
                         FP32 |d count| <= 2 and R within the count bound.
  solver, four-layer cut the FP32 model of layers 60..63 solved by the fused
                         solve and by the layered pass; the oracle's value
                         iteration (Sec. II-B) on the GPU's exported P/R:
                         |dV| <= 1e-5 max(1, |V|), policy equal up to ties.
  full model             the whole 120-layer model: 240 sampled (t, cell) units
                         against the oracle's build of the same units, and the
                         solved values on 3,000 sampled states against one
                         FP64 Bellman backup of the GPU's own values (the fixed
                         point property V = T V, Sec. II-B).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from conftest import policy_tie_check
from paper_2109_00857_gb300 import inputs

pytestmark = pytest.mark.gpu

T_CUT = 60
# 2,000 cells of one layer: rows 60-65 (the lower moving square's edge is at
# rows 60-79 of these layers) and rows 159-162 (the 2x2 target at row 160)
BANDS = ((60 * 200, 66 * 200), (159 * 200, 163 * 200))


@pytest.fixture(scope="module")
def mdp():
    import torch
    torch.cuda.set_device(0)
    from paper_2109_00857_gb300 import build_native, mdp as m
    build_native.build()
    m.load()
    return m


@pytest.fixture(scope="module")
def large():
    env = inputs.large()
    env.Y = oracle.coeffs_for(env)   # the large model's own draw, all 120 layers
    return env


def cut(env, t0, n):
    """Layers t0..t0+n-1 of env with those layers' coefficients."""
    sl = slice(t0, t0 + n)
    return dataclasses.replace(env, nt=n, vbar=np.ascontiguousarray(env.vbar[sl]),
                               modes=np.ascontiguousarray(env.modes[sl]),
                               obstacle=np.ascontiguousarray(env.obstacle[sl]),
                               gbar=np.ascontiguousarray(env.gbar[sl]),
                               Y=np.ascontiguousarray(env.Y[sl]))


def export_np(mdp, model, obj=0):
    rp, col, cnt, R = mdp.mdp_export_csr(model, obj)
    return rp.cpu().numpy(), col.cpu().numpy(), cnt.cpu().numpy(), R.cpu().numpy()


def compare_units(env, ref, u0, gpu_rows, exact, obj_slots):
    """Rows of units u0.. (oracle local layout: row (u - u0) * A + a) against
    the GPU's paper-layout rows.  gpu_rows(u, a, o) -> (cols, counts, R)."""
    A, N = env.A, env.N
    rmax = max(abs(env.r_outbound), 1.0 + abs(env.r_term) + 4.0 * (1.0 + env.c_r))
    nunits = len(ref["nnz"]) // A
    worst = 0
    for k in range(nunits):
        u = u0 + k
        for a in range(A):
            lr = k * A + a
            n = ref["nnz"][lr]
            oc, on = ref["col"][lr, :n], ref["cnt"][lr, :n]
            for o in obj_slots:
                gc, gn, gR = gpu_rows(u, a, o)
                if exact:
                    assert np.array_equal(gc, oc) and np.array_equal(gn, on), (u, a)
                    assert abs(gR - ref["R"][o][lr]) <= 1e-12 * max(1.0, abs(ref["R"][o][lr])), (u, a, o)
                    continue
                d = dict(zip(oc.tolist(), on.tolist()))
                for c_, n_ in zip(gc.tolist(), gn.tolist()):
                    d[c_] = d.get(c_, 0) - n_
                diff = np.abs(np.fromiter(d.values(), dtype=np.int64)) if d else np.zeros(1, np.int64)
                worst = max(worst, int(diff.max()))
                assert diff.max() <= 2, (u, a, "|d count| > 2")
                if n:
                    assert gn.sum() == N and on.sum() == N
                bound = diff.sum() / N * rmax + 1e-5 * max(1.0, abs(ref["R"][o][lr]))
                assert abs(float(gR) - ref["R"][o][lr]) <= bound, (u, a, o)
    return worst


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_layer_cut_of_the_large_model_matches_the_oracle(mdp, large, precision):
    es = cut(large, T_CUT, 2)
    objs = es.objectives
    prec = mdp.MDP_FP64_CHECK if precision == "fp64" else mdp.MDP_FP32
    model = mdp.mdp_build(mdp.DeviceEnv(es, prec), objs=objs)
    info = model.info()
    assert info.L == 21 and info.max_row_nnz <= 64
    ex = [export_np(mdp, model, o) for o in range(len(objs))]
    rp, col, cnt = ex[0][:3]
    nS = es.nS

    def gpu_rows(u, a, o):
        r = a * nS + u
        lo, hi = rp[r], rp[r + 1]
        return col[lo:hi], cnt[lo:hi], ex[o][3][r]

    for (u0, u1) in BANDS:
        ref = oracle.build_units(es, objs, u0, u1, with_literal=False)
        assert ref["status"] == 0 and ref["overflow"] == 0
        # the stored successor offsets dj*200 + di take both signs beyond 8 bits
        lr, k = np.nonzero(ref["cnt"] > 0)
        cols = ref["col"][lr, k]
        dom = cols < nS
        offs = cols[dom] - (u0 + lr[dom] // es.A + es.Nc)
        assert offs.min() < -128 and offs.max() > 127
        compare_units(es, ref, u0, gpu_rows, precision == "fp64", range(len(objs)))


def test_four_layer_cut_solves_match_the_oracle_on_identical_P_R(mdp, large):
    es = cut(large, T_CUT, 4)
    objs = es.objectives
    model = mdp.mdp_build(mdp.DeviceEnv(es, mdp.MDP_FP32), objs=objs)
    assert model.info().max_row_nnz <= 13   # rows as narrow as on the full model
    Vs, ps, sts = mdp.mdp_solve_multi(model, tuple(range(3)), method=mdp.MDP_SOLVE_JACOBI, tol=0.0)
    Vl, pl, stl = mdp.mdp_solve_multi(model, tuple(range(3)), method=mdp.MDP_SOLVE_LAYERED)
    fx = oracle.fixed_mask(es)
    for o in range(3):
        assert np.array_equal(Vs[o].cpu().numpy(), Vl[o].cpu().numpy())
        assert np.array_equal(ps[o].cpu().numpy(), pl[o].cpu().numpy())
        rp, col, cnt, R = export_np(mdp, model, o)
        om = oracle.model_from_csr(es.nS, es.A, es.N, rp, col, cnt)
        R64 = R.astype(np.float64)
        Vo, pio, sw, res = oracle.vi_jacobi(om, R64, fx, tol=0.0, nt=es.nt)
        assert sts[o].sweeps == sw and sts[o].residual == 0.0
        V = Vs[o].cpu().numpy().astype(np.float64)
        scale = np.maximum(1.0, np.abs(Vo))
        assert np.all(np.abs(V - Vo) <= 1e-5 * scale), np.max(np.abs(V - Vo) / scale)
        policy_tie_check(ps[o].cpu().numpy(), pio, oracle.q_values(om, R64, Vo))


def test_full_model_sampled_units_and_bellman_fixed_point(mdp, large):
    import torch
    objs = large.objectives
    model = mdp.mdp_build(mdp.DeviceEnv(large, mdp.MDP_FP32), objs=objs)
    info = model.info()
    assert info.rows == large.nS * 32 and info.L == 21
    nS, Nc, A, N = large.nS, large.Nc, large.A, large.N
    Vs, ps, sts = mdp.mdp_solve_multi(model, tuple(range(3)), method=mdp.MDP_SOLVE_JACOBI, tol=0.0)
    rp_d, col_d, cnt_d, R0 = mdp.mdp_export_csr(model, 0)
    R_d = [R0] + [mdp.mdp_export_csr(model, o, with_entries=False)[3] for o in (1, 2)]

    def rows_of(idx):
        """(lengths, cols, counts, R per objective) of paper-layout rows idx,
        gathered on the device."""
        it = torch.as_tensor(idx, device=rp_d.device)
        lo, hi = rp_d[it], rp_d[it + 1]
        ln = hi - lo
        first = torch.repeat_interleave(torch.cumsum(ln, 0) - ln, ln)
        pos = torch.repeat_interleave(lo, ln) + torch.arange(int(ln.sum()), device=rp_d.device) - first
        return (ln.cpu().numpy(), col_d[pos].cpu().numpy(), cnt_d[pos].cpu().numpy(),
                [r[it].cpu().numpy() for r in R_d])

    rng = np.random.default_rng(60)
    # (t, cell) units: 8 layers x 30 consecutive cells, against the oracle's build
    for t in (0, 1, 37, 60, 61, 90, 118, 119):
        c0 = int(rng.integers(0, Nc - 30))
        u0, u1 = t * Nc + c0, t * Nc + c0 + 30
        ref = oracle.build_units(large, objs, u0, u1, with_literal=False)
        assert ref["status"] == 0 and ref["overflow"] == 0
        pairs = [(u, a) for u in range(u0, u1) for a in range(A)]
        idx = np.array([a * nS + u for u, a in pairs], np.int64)
        ln, cc, nn, Rs = rows_of(idx)
        off = np.concatenate([[0], np.cumsum(ln)])
        where = {p: k for k, p in enumerate(pairs)}

        def gpu_rows(u, a, o):
            k = where[(u, a)]
            return cc[off[k]:off[k + 1]], nn[off[k]:off[k + 1]], Rs[o][k]
        compare_units(large, ref, u0, gpu_rows, False, range(3))
    # the fixed point: V(s) = max_a [R(s,a) + sum_j (c_j / N) V(s'_j)] in FP64
    # on the GPU's own values and rows, at 3,000 states over every layer; the
    # policy is an argmax of that Q up to ties
    states = np.unique(rng.integers(0, nS, 3000))
    idx = (np.arange(A)[:, None] * nS + states[None, :]).reshape(-1)
    ln, cc, nn, Rs = rows_of(idx)
    seg = np.repeat(np.arange(len(idx)), ln)
    fixed = oracle.fixed_mask(large)[states] != 0
    for o in range(3):
        V = Vs[o].cpu().numpy().astype(np.float64)
        pi = ps[o].cpu().numpy().astype(np.int64)
        acc = np.zeros(len(idx))
        np.add.at(acc, seg, nn / N * V[cc])
        Q = (Rs[o].astype(np.float64) + acc).reshape(A, len(states))
        Tv = Q.max(axis=0)
        err = np.abs(V[states] - Tv) / np.maximum(1.0, np.abs(Tv))
        assert err.max() <= 1e-5, (o, float(err.max()))
        assert np.all(pi[states[fixed]] == -1)
        free = ~fixed
        policy_tie_check(pi[states[free]], Q[:, free].argmax(axis=0), Q[:, free])
