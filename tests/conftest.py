import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def custom_env(nx=7, ny=7, nt=5, K=1, N=64, L=5, vbar=None, modes=None, sigma=None, seed=1,
               obstacle=None, target=None, actions=None, gbar=None, Y=None, **kw):
    """A small hand-made environment for closed-form checks."""
    from paper_2109_00857_gb300 import inputs
    if vbar is None:
        vbar = np.zeros((nt, ny, nx, 2))
    if modes is None:
        modes = np.zeros((nt, K, ny, nx, 2))
    if sigma is None:
        sigma = np.zeros(K)
    if obstacle is None:
        obstacle = np.zeros((nt, ny, nx), np.uint8)
    if target is None:
        target = np.zeros((ny, nx), np.uint8)
    if actions is None:
        actions = inputs.action_table(16, 1, 1.0)
    return inputs.Environment(nx=nx, ny=ny, nt=nt, K=K, N=N, L=L, vbar=np.asarray(vbar, float),
                              modes=np.asarray(modes, float), sigma=np.asarray(sigma, float),
                              seed=seed, obstacle=np.asarray(obstacle, np.uint8),
                              target=np.asarray(target, np.uint8), actions=np.asarray(actions, float),
                              gbar=gbar, Y=Y, **kw)


def device_pool_meter():
    """(reset the high-water mark, read (used now, high-water mark)) of the
    current device's default memory pool, through the CUDA driver API."""
    import ctypes as C
    cu = C.CDLL("libcuda.so.1")
    dev = C.c_int()
    assert cu.cuCtxGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    USED, USED_HIGH = 7, 8   # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def reset():
        zero = C.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, USED_HIGH, C.byref(zero)) == 0

    def read():
        a, b = C.c_uint64(), C.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, USED, C.byref(a)) == 0
        assert cu.cuMemPoolGetAttribute(pool, USED_HIGH, C.byref(b)) == 0
        return a.value, b.value
    return reset, read


@pytest.fixture
def make_env():
    return custom_env


# The stated tie tolerance of the policy gate: where a policy entry differs
# from the oracle's, the oracle's Q values of the two actions must lie within
# TIE_REL * max(1, |Q|) of each other.
TIE_REL = 1e-6


def policy_tie_check(pi, pio, Q, rel=TIE_REL):
    """Assert pi equals the oracle's pio except at ties: for every differing
    state both are actions (not -1) and Q[pio] - Q[pi] <= rel * max(1, |Q[pio]|)
    with Q the oracle's [A][nS] Q table.  Returns the number of ties taken."""
    pi = np.asarray(pi).astype(np.int64)
    pio = np.asarray(pio).astype(np.int64)
    bad = np.nonzero(pi != pio)[0]
    if len(bad) == 0:
        return 0
    assert np.all(pio[bad] >= 0) and np.all(pi[bad] >= 0), "a fixed state has a different policy"
    q0 = Q[pio[bad], bad]
    q1 = Q[pi[bad], bad]
    gap = q0 - q1
    lim = rel * np.maximum(1.0, np.abs(q0))
    worst = int(np.argmax(gap - lim))
    assert np.all(gap <= lim), (f"policy differs beyond a tie at state {bad[worst]}: "
                                f"Q gap {gap[worst]:.3e} > {lim[worst]:.3e}")
    return len(bad)


def oracle_end_to_end(mdp, env, obj, V, pi, tol_rel=1e-5):
    """Compare an FP32 result (V [nS+1], pi [nS] as numpy) for objective `obj`
    of env, produced by some path over the library's FP32 build of env (a
    served request, a batch member), with the oracle's own build (Alg. 2) and
    value iteration (Sec. II-B), end to end.

    The FP32 build may differ from the oracle's by a few counts per row
    (|d count| <= 2, the build gate).  Their effect is bounded exactly: with
    the oracle's fixed point V*, row r of the FP32 model (P', R') differs by
    e_r = |R'_r - R_r| + |sum_j (P'_rj - P_rj) V*(s'_j)| in its one-step
    backup, so |V' - V*| <= B_t on layer t with B_t = max_{rows of t} e_r +
    B_{t+1}, B_nt = 0 (transitions go to layer t+1 or the sink).  The gate
    is |V - V*| <= B_t + tol_rel max(1, |V*|); a policy entry may differ from
    the oracle's only where the oracle's Q gap is within the same bound
    (2 (max_rows e + B_{t+1}) + 1e-6 max(1, |Q|)).  The result must also equal
    the direct FP32 build + Jacobi solve of env bit for bit."""
    import oracle
    ref = oracle.build(env, objs=(obj,))
    m = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=(obj,))
    Vd, pid, _ = mdp.mdp_solve(m, 0, tol=0.0)
    assert np.array_equal(np.asarray(V, np.float32), Vd.cpu().numpy()), "differs from the direct solve"
    assert np.array_equal(np.asarray(pi), pid.cpu().numpy())
    rp, col, cnt, R = (x.cpu().numpy() for x in mdp.mdp_export_csr(m, 0))
    fx = oracle.fixed_mask(env)
    Vo, pio, sw, res = oracle.vi_jacobi(ref, ref.R[0], fx, tol=0.0, nt=env.nt)
    nS, A, N, Nc, nt = env.nS, env.A, env.N, env.Nc, env.nt

    def backup_part(rowptr, c, n):
        vals = n / N * Vo[c]
        out = np.zeros(len(rowptr) - 1)
        nz = np.diff(rowptr) > 0
        out[nz] = np.add.reduceat(vals, rowptr[:-1][nz])
        return out
    e = np.abs(R.astype(np.float64) - ref.R[0]) + \
        np.abs(backup_part(rp, col, cnt) - backup_part(ref.rowptr, ref.col, ref.cnt))
    layer = (np.arange(A * nS) % nS) // Nc
    E = np.zeros(nt + 1)
    np.maximum.at(E, layer, e)
    B = np.zeros(nt + 1)
    for t in range(nt - 1, -1, -1):
        B[t] = E[t] + B[t + 1]
    V = np.asarray(V, dtype=np.float64)
    Bs = np.concatenate([B[np.arange(nS) // Nc], [0.0]])
    err = np.abs(V - Vo) - Bs - tol_rel * np.maximum(1.0, np.abs(Vo))
    assert err.max() <= 0.0, f"|dV| exceeds the count-difference bound by {err.max():.3e}"
    Q = oracle.q_values(ref, ref.R[0], Vo)
    pi = np.asarray(pi).astype(np.int64)
    bad = np.nonzero(pi != pio)[0]
    if len(bad):
        assert np.all(pio[bad] >= 0) and np.all(pi[bad] >= 0)
        t = bad // Nc
        gap = Q[pio[bad], bad] - Q[pi[bad], bad]
        lim = 2.0 * (E[t] + B[t + 1]) + TIE_REL * np.maximum(1.0, np.abs(Q[pio[bad], bad]))
        assert np.all(gap <= lim), "a policy entry differs beyond the bound"
    return float(B[0])
