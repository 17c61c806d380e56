"""Pins of the oracle's policy rollouts (Sec. IV: the optimal policy applied to
every flow realization from the start) against facts fixed independently of
the rollout code: the build's own transition counts, value iteration on
deterministic flows, a closed form for zero flow, and the absorbing rules."""
import numpy as np
import pytest

import oracle
from conftest import custom_env
from paper_2109_00857_gb300 import inputs


def solved(env, obj_slot=0, objs=(0,)):
    m = oracle.build(env, objs=objs)
    V, pi, sw, res = oracle.vi_jacobi(m, m.R[obj_slot], oracle.fixed_mask(env), tol=0.0, nt=env.nt)
    return m, V, pi


def row_counts(m, s, a):
    r = a * m.nS + s
    lo, hi = m.rowptr[r], m.rowptr[r + 1]
    return dict(zip(m.col[lo:hi].tolist(), m.cnt[lo:hi].tolist()))


def test_first_step_histogram_is_the_build_row():
    """Path w's first move uses realization w of time 0, exactly the samples
    the build counted for (s0, pi(s0)): the first landings over the N paths
    reproduce that row's counts exactly (sink included)."""
    env = inputs.energy(nx=24, ny=20, nt=5, N=300, L=15)
    m, V, pi = solved(env, objs=(2,))
    checked = 0
    for (i0, j0) in [(3, 4), (12, 10), (20, 2), (7, 17)]:
        s0 = j0 * env.nx + i0
        if pi[s0] < 0:
            continue
        ret, steps, status, traj = oracle.rollout(env, pi, (i0, j0), objs=(2,), with_traj=True)
        land, n = np.unique(traj[:, 1], return_counts=True)
        assert dict(zip(land.tolist(), n.tolist())) == row_counts(m, s0, int(pi[s0]))
        checked += 1
    assert checked >= 3


def test_every_move_is_a_counted_transition():
    """Each move s -> s' of every path has a nonzero count in the build's row
    (s, pi(s)); returns are finite and steps match the trajectory length."""
    env = inputs.tiny(nx=14, ny=12, nt=9, N=120, r_term=5.0)
    m, V, pi = solved(env)
    ret, steps, status, traj = oracle.rollout(env, pi, (2, 3), with_traj=True)
    for w in range(env.N):
        for k in range(steps[w]):
            s, sp = int(traj[w, k]), int(traj[w, k + 1])
            assert row_counts(m, s, int(pi[s])).get(sp, 0) > 0, (w, k, s, sp)
        assert traj[w, steps[w] + 1:].tolist() == [-1] * (env.nt - steps[w])
    assert np.all(np.isfinite(ret))


@pytest.mark.parametrize("obj", [0, 1, 2])
def test_deterministic_flow_return_equals_value(obj):
    """With zero coefficient variance every realization moves alike, so the
    rollout return from any free start is the value V(s) of value iteration
    (summed forward instead of backward: equal to rounding)."""
    nx, ny, nt = 11, 9, 8
    rng = np.random.default_rng(3)
    vbar = np.zeros((nt, ny, nx, 2))
    vbar[..., 0] = 0.3 * np.sin(np.arange(nx) / 3.0)[None, None, :]
    vbar[..., 1] = -0.2
    tgt = np.zeros((ny, nx), np.uint8)
    tgt[6:8, 8:10] = 1
    obst = np.zeros((nt, ny, nx), np.uint8)
    obst[:, 2:4, 4] = 1
    gbar = rng.uniform(0.0, 1.0, (nt, ny, nx))
    env = custom_env(nx=nx, ny=ny, nt=nt, K=1, N=6, L=7, vbar=vbar, sigma=[0.0], target=tgt,
                     obstacle=obst, gbar=gbar, actions=inputs.action_table(8, 2, 1.0), r_term=2.0,
                     r_outbound=-40.0)
    m, V, pi = solved(env, objs=(obj,))
    checked = 0
    for j0 in range(ny):
        for i0 in range(nx):
            s0 = j0 * nx + i0
            ret, steps, status, _ = oracle.rollout(env, pi, (i0, j0), objs=(obj,))
            assert np.all(ret == ret[0]) and np.all(steps == steps[0])
            assert ret[0, 0] == pytest.approx(V[s0], rel=1e-12, abs=1e-12), (i0, j0)
            checked += 1
    assert checked == nx * ny


def test_zero_flow_paths_take_chebyshev_distance_steps():
    """Zero flow, F = 1, 16 headings: the time-optimal path from a start
    within reach lands on the target after d_inf steps, return r_term - dt d."""
    nx = ny = 9
    nt = 7
    tgt = np.zeros((ny, nx), np.uint8)
    tgt[6:8, 4:6] = 1
    env = custom_env(nx=nx, ny=ny, nt=nt, N=5, L=5, target=tgt, r_term=3.0, r_outbound=-500.0)
    m, V, pi = solved(env)
    tj, ti = np.nonzero(tgt)
    checked = 0
    for j0 in range(ny):
        for i0 in range(nx):
            d = min(max(abs(i0 - a), abs(j0 - b)) for a, b in zip(ti, tj))
            if d > nt - 1:
                continue
            ret, steps, status, _ = oracle.rollout(env, pi, (i0, j0))
            assert np.all(status == 0) and np.all(steps == d), (i0, j0, d, steps[0])
            assert np.all(ret[:, 0] == pytest.approx(3.0 - d if d else 0.0, abs=1e-12))
            checked += 1
    assert checked > 40


def test_absorbing_rules():
    """A target start stays (0 steps, return 0); an obstacle start and any
    move from the last layer end in the sink with r_outbound."""
    nx = ny = 6
    tgt = np.zeros((ny, nx), np.uint8)
    tgt[0, 0] = 1
    obst = np.zeros((3, ny, nx), np.uint8)
    obst[0, 4, 4] = 1
    env = custom_env(nx=nx, ny=ny, nt=3, N=4, L=5, target=tgt, obstacle=obst, r_term=1.0,
                     r_outbound=-9.0)
    m, V, pi = solved(env)
    ret, steps, status, traj = oracle.rollout(env, pi, (0, 0), with_traj=True)
    assert np.all(steps == 0) and np.all(status == 0) and np.all(ret == 0.0)
    ret, steps, status, traj = oracle.rollout(env, pi, (4, 4), with_traj=True)
    assert np.all(steps == 1) and np.all(status == 1) and np.all(ret == -9.0)
    assert np.all(traj[:, 1] == env.nS)
    one = custom_env(nx=nx, ny=ny, nt=1, N=4, L=5, target=tgt, r_outbound=-9.0)
    m1, V1, pi1 = solved(one)
    ret, steps, status, _ = oracle.rollout(one, pi1, (3, 3))
    assert np.all(steps == 1) and np.all(status == 1) and np.all(ret == -9.0)


def test_mean_return_estimates_the_value():
    """Path w reuses realization w at every step, and the draws are
    independent over t, so each path is a sample of the Markov chain: the
    mean return agrees with V(s0) within its sampling error."""
    env = inputs.energy(nx=26, ny=22, nt=8, N=1500, L=15)
    m, V, pi = solved(env, objs=(2,))
    i0, j0 = 5, 4
    ret, steps, status, _ = oracle.rollout(env, pi, (i0, j0), objs=(2,))
    r = ret[:, 0]
    se = r.std(ddof=1) / np.sqrt(len(r))
    assert abs(r.mean() - V[j0 * env.nx + i0]) <= 5.0 * se + 1e-9, (r.mean(), V[j0 * env.nx + i0], se)
