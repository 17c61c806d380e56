"""Policy rollouts on the GPU (mdp_rollout) through the C ABI.

Gates: FP64 check mode equals the oracle's rollouts bit for bit (returns,
steps, statuses) under the same policy; in both precisions the first moves
of the N paths reproduce the GPU build's own row counts for (s0, pi(s0))
exactly (each move is one of the samples the build counted); the summaries
equal the path outputs' means."""
import numpy as np
import pytest

import oracle
from conftest import custom_env
from paper_2109_00857_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdp():
    import torch
    torch.cuda.set_device(0)
    from paper_2109_00857_gb300 import build_native, mdp as m
    build_native.build()
    m.load()
    return m


STARTS = [(3, 4), (12, 10), (20, 2), (7, 17), (0, 0)]


def test_check_mode_rollouts_equal_the_oracle_bitwise(mdp):
    env = inputs.energy(nx=24, ny=20, nt=7, N=150, L=15,
                        objectives=(inputs.OBJ_TIME, inputs.OBJ_ENERGY, inputs.OBJ_NET_ENERGY))
    d = mdp.DeviceEnv(env, mdp.MDP_FP64_CHECK)
    model = mdp.mdp_build(d, objs=(2,))
    V, pi, st = mdp.mdp_solve(model, 0, tol=0.0)
    pol = pi.cpu().numpy().astype(np.int32)
    ret, steps, status, summ = mdp.mdp_rollout(d, pi, STARTS, objs=(0, 1, 2))
    ret, steps, status = ret.cpu().numpy(), steps.cpu().numpy(), status.cpu().numpy()
    for q, start in enumerate(STARTS):
        r_o, s_o, st_o, _ = oracle.rollout(env, pol, start, objs=(0, 1, 2))
        assert np.array_equal(ret[q].view(np.uint64), r_o.view(np.uint64)), start
        assert np.array_equal(steps[q], s_o) and np.array_equal(status[q], st_o), start
        np.testing.assert_allclose([summ[q].mean_return[o] for o in range(3)], r_o.mean(axis=0), rtol=1e-12)
        assert summ[q].p_target == pytest.approx(np.mean(st_o == 0))
        arr = s_o[st_o == 0]
        assert summ[q].mean_steps_target == pytest.approx(arr.mean() if len(arr) else 0.0)
        assert summ[q].paths == env.N


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_first_moves_reproduce_the_build_row(mdp, precision):
    """Two layers, so every path makes exactly one move and then takes the
    sink from the last layer; the net-energy reward with gbar(t=1, c) = c + 1
    (c_f = 0, c_r = 2, dt = 1) makes the return r_out + c' + 1 identify the
    landing cell c' (r_out alone: the move itself took the sink)."""
    nx, ny, nt = 15, 13, 2
    rng = np.random.default_rng(8)
    vbar = np.zeros((nt, ny, nx, 2))
    vbar[..., 0], vbar[..., 1] = 0.4, -0.3
    K = 2
    modes = np.zeros((nt, K, ny, nx, 2))
    modes[:, 0, ..., 0] = 1.0
    modes[:, 1, ..., 1] = 1.0
    gbar = np.zeros((nt, ny, nx))
    gbar[1] = np.arange(ny * nx).reshape(ny, nx) + 1.0
    obst = np.zeros((nt, ny, nx), np.uint8)
    obst[1, 5:7, 6:9] = 1
    env = custom_env(nx=nx, ny=ny, nt=nt, K=K, N=2000, L=15, vbar=vbar, modes=modes, sigma=[0.9, 0.7],
                     obstacle=obst, gbar=gbar, c_f=0.0, c_r=2.0, r_term=0.0, r_outbound=-1000.0,
                     actions=inputs.action_table(16, 2, 1.0), seed=4)
    prec = mdp.MDP_FP32 if precision == "fp32" else mdp.MDP_FP64_CHECK
    d = mdp.DeviceEnv(env, prec)
    model = mdp.mdp_build(d, objs=(2,))
    V, pi, st = mdp.mdp_solve(model, 0, tol=0.0)
    rp, col, cnt, R = (x.cpu().numpy() for x in mdp.mdp_export_csr(model, 0))
    pol = pi.cpu().numpy()
    starts = [(7, 6), (2, 2), (13, 11), (7, 1), (0, 12), (14, 0)]
    ret, steps, status, summ = mdp.mdp_rollout(d, pi, starts, objs=(2,))
    ret = ret.cpu().numpy()[..., 0].astype(np.float64)
    sink_seen = 0
    for q, (i0, j0) in enumerate(starts):
        s0 = j0 * nx + i0
        a = int(pol[s0])
        r = a * env.nS + s0
        row = dict(zip(col[rp[r]:rp[r + 1]].tolist(), cnt[rp[r]:rp[r + 1]].tolist()))
        c_land = np.rint(ret[q] + 1000.0).astype(np.int64) - 1   # -1: the move took the sink
        landed = np.where(c_land < 0, env.nS, env.Nc + c_land)
        got = dict(zip(*(x.tolist() for x in np.unique(landed, return_counts=True))))
        assert got == row, (precision, (i0, j0))
        sink_seen += env.nS in row
    assert sink_seen >= 1   # some first moves leave the domain


def test_fp32_rollouts_track_the_fp64_oracle(mdp):
    env = inputs.energy(nx=26, ny=22, nt=8, N=800, L=15)
    d32 = mdp.DeviceEnv(env, mdp.MDP_FP32)
    m32 = mdp.mdp_build(d32, objs=(2,))
    V, pi, st = mdp.mdp_solve(m32, 0, tol=0.0)
    pol = pi.cpu().numpy().astype(np.int32)
    starts = [(5, 4), (20, 15), (12, 11)]
    ret, steps, status, summ = mdp.mdp_rollout(d32, pi, starts, objs=(2,))
    ret, steps, status = ret.cpu().numpy(), steps.cpu().numpy(), status.cpu().numpy()
    for q, start in enumerate(starts):
        r_o, s_o, st_o, _ = oracle.rollout(env, pol, start, objs=(2,))
        same = (steps[q] == s_o) & (status[q] == st_o)
        assert same.mean() >= 0.99, (start, same.mean())
        np.testing.assert_allclose(ret[q][same, 0], r_o[same, 0], rtol=1e-5, atol=1e-4)


def test_rollout_argument_errors(mdp):
    env = inputs.tiny(nx=8, ny=8, nt=3, N=20)
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    m = mdp.mdp_build(d)
    V, pi, st = mdp.mdp_solve(m, 0, tol=0.0)
    for kw in (dict(starts=[(8, 0)]), dict(starts=[(0, -1)]), dict(starts=[(1, 1)], objs=(3,)),
               dict(starts=[(1, 1)], N=0), dict(starts=[(1, 1)], objs=(0, 0, 0, 0))):
        with pytest.raises(mdp.MdpError) as ei:
            mdp.mdp_rollout(d, pi, **kw)
        assert ei.value.code == -1
