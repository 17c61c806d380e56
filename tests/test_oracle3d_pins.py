"""Pins of the 3-D oracle build (Sec. II-A with n = 3) against facts fixed
independently of it: the already pinned 2-D oracle (a one-layer 3-D grid with
no vertical motion is the 2-D problem), closed forms for zero and uniform
flow, and the model invariants."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2109_00857_gb300 import inputs


def lift(env2):
    """The 2-D environment as a 3-D one with a single layer and no vertical motion."""
    vb = np.concatenate([env2.vbar, np.zeros(env2.vbar.shape[:3] + (1,))], axis=-1)[:, None]
    md = np.concatenate([env2.modes, np.zeros(env2.modes.shape[:4] + (1,))], axis=-1)[:, :, None]
    act = np.stack([env2.actions[:, 0], env2.actions[:, 1], np.zeros(env2.A), env2.actions[:, 2]], axis=1)
    return inputs.Environment3D(nx=env2.nx, ny=env2.ny, nz=1, nt=env2.nt, K=env2.K, N=env2.N, L=env2.L,
                                vbar=vb, modes=md, sigma=env2.sigma, seed=env2.seed,
                                obstacle=env2.obstacle[:, None], target=env2.target[None], actions=act,
                                gbar=None if env2.gbar is None else env2.gbar[:, None], Y=env2.Y,
                                mdp_id=env2.mdp_id, c_f=env2.c_f, c_r=env2.c_r, r_term=env2.r_term,
                                r_outbound=env2.r_outbound)


@pytest.mark.parametrize("objs", [(0,), (0, 1, 2)])
def test_single_layer_grid_is_the_2d_problem(objs):
    env2 = inputs.energy(nx=14, ny=12, nt=4, N=120, L=9)
    m2 = oracle.build(env2, objs=objs)
    m3 = oracle.build3d(lift(env2), objs=objs, max_nnz=9 * 9 + 1)
    assert np.array_equal(m3.rowptr, m2.rowptr)
    assert np.array_equal(m3.col, m2.col)
    assert np.array_equal(m3.cnt, m2.cnt)
    assert np.array_equal(m3.R, m2.R)
    assert m3.overflow == m2.overflow


def unit_moves():
    """The 26 unit moves to the neighbouring cells, speed |d|."""
    rows = [(dx, dy, dz, float(np.sqrt(dx * dx + dy * dy + dz * dz)))
            for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3) if (dx, dy, dz) != (0, 0, 0)]
    return np.asarray(rows, dtype=np.float64)


def env3(nx, ny, nz, nt, N=4, L=3, vbar=None, target=None, obstacle=None, **kw):
    K = 1
    return inputs.Environment3D(
        nx=nx, ny=ny, nz=nz, nt=nt, K=K, N=N, L=L,
        vbar=np.zeros((nt, nz, ny, nx, 3)) if vbar is None else vbar,
        modes=np.zeros((nt, K, nz, ny, nx, 3)), sigma=np.zeros(K), seed=3,
        obstacle=np.zeros((nt, nz, ny, nx), np.uint8) if obstacle is None else obstacle,
        target=np.zeros((nz, ny, nx), np.uint8) if target is None else target,
        actions=kw.pop("actions", unit_moves()), **kw)


def test_zero_flow_value_is_3d_chebyshev_distance():
    """Zero flow, the 26 unit moves: V(s) = r_term - dt d_inf(s, target) (3-D
    Chebyshev distance) wherever the target is reachable within the horizon."""
    nx, ny, nz, nt = 7, 6, 5, 6
    tgt = np.zeros((nz, ny, nx), np.uint8)
    tgt[3:5, 4:6, 5:7] = 1
    e = env3(nx, ny, nz, nt, target=tgt, r_term=4.0, r_outbound=-300.0)
    m = oracle.build3d(e)
    V, pi, sw, res = oracle.vi_jacobi(m, m.R[0], oracle.fixed_mask3d(e), tol=0.0, nt=nt)
    tk, tj, ti = np.nonzero(tgt)
    checked = 0
    for t in range(nt):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    s = t * e.Nc + (k * ny + j) * nx + i
                    d = min(max(abs(i - a), abs(j - b), abs(k - c)) for a, b, c in zip(ti, tj, tk))
                    if d == 0:
                        assert V[s] == 0.0 and pi[s] == -1
                    elif d <= nt - 1 - t:
                        assert V[s] == pytest.approx(4.0 - d, abs=1e-12), (t, k, j, i)
                        checked += 1
    assert checked > 300


def test_uniform_flow_rows_are_one_hot_at_the_predicted_cell():
    """Uniform flow c, no variance: action d from the centre of (i, j, k)
    lands in floor(i + 1/2 + c_x + d_x) etc. with all N realizations (or in
    the sink outside the domain / on an obstacle)."""
    nx, ny, nz, nt = 8, 7, 5, 3
    c = np.array([0.7, -0.4, 0.3])
    vb = np.broadcast_to(c, (nt, nz, ny, nx, 3)).copy()
    obst = np.zeros((nt, nz, ny, nx), np.uint8)
    obst[1, 2, 3, 4] = 1
    act = np.array([[1.0, 0.0, 0.0, 1.0], [0.0, 0.5, -0.5, 0.7], [-0.3, -0.3, 0.9, 1.0]])
    e = env3(nx, ny, nz, nt, N=9, L=5, vbar=vb, obstacle=obst, actions=act, r_outbound=-7.0)
    m = oracle.build3d(e)
    for a in range(e.A):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    s = (k * ny + j) * nx + i        # t = 0
                    r = a * e.nS + s
                    cols = m.col[m.rowptr[r]:m.rowptr[r + 1]]
                    cnts = m.cnt[m.rowptr[r]:m.rowptr[r + 1]]
                    ip, jp, kp = (int(np.floor(x + 0.5 + cc + dd))
                                  for x, cc, dd in zip((i, j, k), c, act[a, :3]))
                    inside = 0 <= ip < nx and 0 <= jp < ny and 0 <= kp < nz
                    if inside and not obst[1, kp, jp, ip]:
                        want = e.Nc + (kp * ny + jp) * nx + ip
                    else:
                        want = e.nS
                    assert cols.tolist() == [want] and cnts.tolist() == [9], (a, k, j, i)


def test_model_invariants():
    e = inputs.cube(nx=10, ny=9, nz=4, nt=4, N=150)
    m = oracle.build3d(e, objs=(0,))
    assert m.overflow == 0
    nS, A, Nc = e.nS, e.A, e.Nc
    for r in range(A * nS):
        s = r % nS
        lo, hi = m.rowptr[r], m.rowptr[r + 1]
        t, c = divmod(s, Nc)
        if e.target.reshape(-1)[c]:
            assert hi == lo                      # terminal rows are empty
            continue
        assert m.cnt[lo:hi].sum() == e.N          # every realization lands somewhere
        cols = m.col[lo:hi]
        assert np.all(np.diff(cols) > 0)         # ascending, sink last
        inner = cols[cols < nS]
        assert np.all(inner // Nc == t + 1)      # one step forward in time
        assert not np.any(e.obstacle.reshape(-1)[inner])   # never onto an obstacle


def test_overflow_is_counted():
    nx, ny, nz, nt = 6, 6, 3, 2
    vb = np.zeros((nt, nz, ny, nx, 3))
    vb[..., 2] = 2.6                              # lands 3 layers up: outside a 3x3x3 window
    e = env3(nx, ny, nz, nt, N=5, L=3, vbar=vb, actions=np.array([[0.0, 0.0, 0.0, 0.0]]))
    m = oracle.build3d(e)
    assert m.overflow > 0


def test_vertical_mode_gives_gaussian_layer_offsets():
    """One unit mode along z with coefficient variance sigma^2 and mean vertical
    velocity mu, an action with no displacement: the layer offset
    floor(1/2 + mu + Y) of a landing is n with probability
    Phi((n + 1/2 - mu) / sigma) - Phi((n - 1/2 - mu) / sigma).  Counts of every
    start state are checked against it within 5 standard errors (+1)."""
    from math import erf, sqrt
    nx, ny, nz, nt, N = 3, 3, 15, 2, 4000
    mu, sig = 0.3, 1.1
    vb = np.zeros((nt, nz, ny, nx, 3))
    vb[..., 2] = mu
    e = env3(nx, ny, nz, nt, N=N, L=11, vbar=vb, actions=np.array([[0.0, 0.0, 0.0, 0.0]]))
    e.modes = np.zeros((nt, 1, nz, ny, nx, 3))
    e.modes[..., 2] = 1.0
    e.sigma = np.array([sig])
    m = oracle.build3d(e)
    assert m.overflow == 0

    def Phi(x):
        return 0.5 * (1.0 + erf(x / sqrt(2.0)))

    checked = 0
    for k in range(5, 10):   # interior layers: every offset within +-5 stays inside
        s = (k * ny + 1) * nx + 1           # t = 0, centre column
        lo, hi = m.rowptr[s], m.rowptr[s + 1]
        got = dict(zip(m.col[lo:hi].tolist(), m.cnt[lo:hi].tolist()))
        for n in range(-5, 6):
            p = Phi((n + 0.5 - mu) / sig) - Phi((n - 0.5 - mu) / sig)
            c = got.get(e.Nc + s + n * nx * ny, 0)
            assert abs(c - N * p) <= 5 * sqrt(N * p * (1 - p)) + 1, (k, n, c, N * p)
            checked += 1
    assert checked == 55
