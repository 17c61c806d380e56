"""FP64 CPU oracle for the MDP build and value iteration (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library under
``paper_2109_00857_gb300`` never calls it, and the two share no code: the only
thing both sides consume is the seeded input arrays of
``paper_2109_00857_gb300.inputs``.

The arithmetic lives in ``oracle.c`` (plain C, IEEE binary64, no contraction);
this module compiles it with gcc and marshals numpy arrays through ctypes.

Parity-pin status per function (what fixes each one other than itself) is in
the docstrings below; every function here is pinned by a ``-m "not gpu"`` test.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OBJ_TIME, OBJ_ENERGY, OBJ_NET_ENERGY = 0, 1, 2


def compile_lib(force: bool = False) -> str:
    """Compile oracle.c -> _lib/liboracle.so (gcc -O2 -ffp-contract=off)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src),
                                             os.path.getmtime(os.path.join(_HERE, "oracle.h")))):
        return _SO
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nt", C.c_int32),
        ("dx", C.c_double), ("dt", C.c_double),
        ("K", C.c_int32), ("N", C.c_int32), ("A", C.c_int32), ("L", C.c_int32),
        ("vbar", C.c_void_p), ("modes", C.c_void_p), ("Y", C.c_void_p), ("gbar", C.c_void_p),
        ("obstacle", C.c_void_p), ("target", C.c_void_p), ("act", C.c_void_p),
        ("c_f", C.c_double), ("c_r", C.c_double), ("r_term", C.c_double),
        ("r_outbound", C.c_double),
    ]


class Problem3D(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nt", C.c_int32),
                ("dx", C.c_double), ("dt", C.c_double),
                ("K", C.c_int32), ("N", C.c_int32), ("A", C.c_int32), ("L", C.c_int32),
                ("vbar", C.c_void_p), ("modes", C.c_void_p), ("Y", C.c_void_p), ("gbar", C.c_void_p),
                ("obstacle", C.c_void_p), ("target", C.c_void_p), ("act", C.c_void_p),
                ("c_f", C.c_double), ("c_r", C.c_double), ("r_term", C.c_double),
                ("r_outbound", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(compile_lib())
            P = C.c_void_p
            l.orc_philox4x64_10.argtypes = [P, P, P]
            l.orc_ln.argtypes = [C.c_double]
            l.orc_ln.restype = C.c_double
            l.orc_polar_pair.argtypes = [C.c_uint64] * 5 + [P, P]
            l.orc_polar_pair.restype = C.c_int
            l.orc_sample_coeffs.argtypes = [C.c_int32, C.c_int32, C.c_int32, P, C.c_uint64,
                                            C.c_uint64, P]
            l.orc_sample_coeffs.restype = C.c_int64
            l.orc_build.argtypes = [C.POINTER(Problem), C.c_int64, C.c_int64, C.c_int32, P,
                                    C.c_int32, P, P, P, P, P, P]
            l.orc_build.restype = C.c_int
            l.orc_vi_jacobi.argtypes = [C.c_int64, C.c_int32, P, P, P, P, P, P, C.c_double,
                                        C.c_int32, P, P, P, P]
            l.orc_vi_jacobi.restype = C.c_int
            l.orc_vi_backward.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.c_int64, P, P, P, P,
                                          P, P, P]
            l.orc_vi_backward.restype = C.c_int
            l.orc_q_values.argtypes = [C.c_int64, C.c_int32, P, P, P, P, P, P]
            l.orc_rollout.argtypes = [C.POINTER(Problem), P, C.c_int32, C.c_int32, P, C.c_int32, P, P, P, P]
            l.orc_build3d.argtypes = [C.POINTER(Problem3D), C.c_int64, C.c_int64, C.c_int32, P,
                                      C.c_int32, P, P, P, P, P]
            l.orc_build3d.restype = C.c_int
            l.orc_rollout.restype = C.c_int
            _lib = l
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------- sampling --
def philox4x64_10(ctr, key) -> np.ndarray:
    """Philox4x64-10 block (Salmon et al. 2011).  Pinned against numpy.random.Philox."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def ln(x: float) -> float:
    """Self-written natural log.  Pinned against math.log (ulp bound)."""
    return lib().orc_ln(float(x))


def polar_pair(seed, mdp_id, t, w, j):
    z1, z2 = C.c_double(), C.c_double()
    n = lib().orc_polar_pair(seed, mdp_id, t, w, j, C.byref(z1), C.byref(z2))
    return z1.value, z2.value, n


def sample_coeffs(nt: int, N: int, K: int, sigma, seed: int, mdp_id: int = 0) -> np.ndarray:
    """DO coefficients Y[t][w][k] ~ N(0, sigma_k^2).  Pinned by moment / KS tests."""
    sig = _c(sigma, np.float64)
    assert sig.shape == (K,)
    Y = np.zeros((nt, N, K), dtype=np.float64)
    capped = lib().orc_sample_coeffs(nt, N, K, _p(sig), seed, mdp_id, _p(Y))
    assert capped == 0
    return Y


# -------------------------------------------------------------------- build --
class OracleModel:
    """Oracle build output in the paper's layout: rows appended over actions
    (row = a*|S| + s), CSR with successors ascending and the sink (= |S|) last."""

    def __init__(self, nS, A, rowptr, col, cnt, N, R, R_lit, overflow):
        self.nS, self.A, self.N = nS, A, N
        self.rowptr, self.col, self.cnt = rowptr, col, cnt
        self.prob = cnt.astype(np.float64) / float(N)
        self.R, self.R_lit, self.overflow = R, R_lit, overflow


_coeff_cache = {}


def coeffs_for(env) -> np.ndarray:
    """The oracle's own coefficient draw for an environment without an external table."""
    key = (env.nt, env.N, env.K, tuple(np.asarray(env.sigma).tolist()), env.seed, env.mdp_id)
    if key not in _coeff_cache:
        if len(_coeff_cache) > 8:
            _coeff_cache.clear()
        _coeff_cache[key] = sample_coeffs(env.nt, env.N, env.K, env.sigma, env.seed, env.mdp_id)
    return _coeff_cache[key]


def make_problem(env, keep):
    """Fill the ctypes Problem from an inputs.Environment (arrays kept alive in `keep`)."""
    def hold(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    p = Problem()
    p.nx, p.ny, p.nt = env.nx, env.ny, env.nt
    p.dx, p.dt = env.dx, env.dt
    p.K, p.N, p.A, p.L = env.K, env.N, env.A, env.L
    p.vbar = _p(hold(env.vbar, np.float64))
    p.modes = _p(hold(env.modes, np.float64))
    Y = env.Y if env.Y is not None else coeffs_for(env)
    p.Y = _p(hold(Y, np.float64))
    p.gbar = _p(hold(env.gbar, np.float64))
    p.obstacle = _p(hold(env.obstacle, np.uint8))
    p.target = _p(hold(env.target, np.uint8))
    p.act = _p(hold(env.actions, np.float64))
    p.c_f, p.c_r, p.r_term, p.r_outbound = env.c_f, env.c_r, env.r_term, env.r_outbound
    return p


def build_units(env, objs, u_begin, u_end, max_nnz=None, with_literal=True):
    """Run the oracle build over units [u_begin, u_end) (unit = t*Nc + c).
    Returns the raw local-row arrays (nnz, col, cnt, R, R_lit, overflow, status)."""
    keep = []
    p = make_problem(env, keep)
    A = env.A
    if max_nnz is None:
        max_nnz = env.L * env.L + 1
    nunits = u_end - u_begin
    rows = nunits * A
    ob = np.ascontiguousarray(objs, dtype=np.int32)
    nnz = np.zeros(rows, dtype=np.int32)
    col = np.zeros(rows * max_nnz, dtype=np.int64)
    cnt = np.zeros(rows * max_nnz, dtype=np.int32)
    R = np.zeros(len(ob) * rows, dtype=np.float64)
    R_lit = np.zeros(len(ob) * rows, dtype=np.float64) if with_literal else None
    ovf = C.c_int64(0)
    st = lib().orc_build(C.byref(p), u_begin, u_end, max_nnz, _p(ob), len(ob), _p(nnz), _p(col),
                         _p(cnt), _p(R), _p(R_lit), C.byref(ovf))
    return dict(nnz=nnz, col=col.reshape(rows, max_nnz), cnt=cnt.reshape(rows, max_nnz),
                R=R.reshape(len(ob), rows), R_lit=None if R_lit is None else R_lit.reshape(len(ob), rows),
                overflow=ovf.value, status=st)


def build(env, objs=(OBJ_TIME,)) -> OracleModel:
    """Full MDP build (all units), reordered into the paper's appended layout."""
    Nc = env.nx * env.ny
    nS = env.nt * Nc
    A = env.A
    out = build_units(env, objs, 0, nS)
    if out["status"] != 0:
        raise RuntimeError(f"oracle build failed with status {out['status']}")
    nnz_local = out["nnz"].reshape(nS, A)               # [s][a]
    nnz_paper = np.ascontiguousarray(nnz_local.T).reshape(-1)   # [a][s]
    rowptr = np.zeros(A * nS + 1, dtype=np.int64)
    np.cumsum(nnz_paper, out=rowptr[1:])
    col = np.zeros(rowptr[-1], dtype=np.int64)
    cnt = np.zeros(rowptr[-1], dtype=np.int32)
    colL = out["col"].reshape(nS, A, -1)
    cntL = out["cnt"].reshape(nS, A, -1)
    for a in range(A):
        for s_idx in np.nonzero(nnz_local[:, a])[0]:
            r = a * nS + s_idx
            n = nnz_local[s_idx, a]
            col[rowptr[r]:rowptr[r] + n] = colL[s_idx, a, :n]
            cnt[rowptr[r]:rowptr[r] + n] = cntL[s_idx, a, :n]
    nobj = len(objs)
    R = np.ascontiguousarray(out["R"].reshape(nobj, nS, A).transpose(0, 2, 1)).reshape(nobj, A * nS)
    R_lit = np.ascontiguousarray(out["R_lit"].reshape(nobj, nS, A).transpose(0, 2, 1)).reshape(nobj, A * nS)
    return OracleModel(nS, A, rowptr, col, cnt, env.N, R, R_lit, out["overflow"])


# ---------------------------------------------------------- value iteration --
def fixed_mask(env) -> np.ndarray:
    """1 for start states whose policy is undefined (terminal target cells, obstacles)."""
    tgt = np.broadcast_to(env.target[None, :, :], env.obstacle.shape)
    return ((env.obstacle != 0) | (tgt != 0)).astype(np.uint8).reshape(-1)


def vi_jacobi(m, R, fixed, tol=0.0, max_sweeps=None, nt=None, V0=None):
    """Jacobi value iteration (Sec. II-B) from v_0 = V0 (length nS or nS + 1;
    the sink entry is 0 regardless) or from 0.  Pinned by backward induction,
    dense brute force, and a dense one-sweep Bellman operator from random V0."""
    nS, A = m.nS, m.A
    if max_sweeps is None:
        max_sweeps = (nt + 1) if nt is not None else 10 ** 6
    V = np.zeros(nS + 1, dtype=np.float64)
    pi = np.zeros(nS, dtype=np.int32)
    sw, res = C.c_int32(0), C.c_double(0.0)
    Rc = np.ascontiguousarray(R, dtype=np.float64)
    fx = np.ascontiguousarray(fixed, dtype=np.uint8)
    v0 = None
    if V0 is not None:
        v0 = np.ascontiguousarray(np.asarray(V0, dtype=np.float64)[:nS])
        assert v0.shape == (nS,)
    lib().orc_vi_jacobi(nS, A, _p(m.rowptr), _p(m.col), _p(m.prob), _p(Rc), _p(fx), _p(v0), tol,
                        max_sweeps, _p(V), _p(pi), C.byref(sw), C.byref(res))
    return V, pi, sw.value, res.value


def vi_backward(m, R, fixed, nt, Nc):
    V = np.zeros(m.nS + 1, dtype=np.float64)
    pi = np.zeros(m.nS, dtype=np.int32)
    Rc = np.ascontiguousarray(R, dtype=np.float64)
    fx = np.ascontiguousarray(fixed, dtype=np.uint8)
    lib().orc_vi_backward(m.nS, m.A, nt, Nc, _p(m.rowptr), _p(m.col), _p(m.prob), _p(Rc), _p(fx),
                          _p(V), _p(pi))
    return V, pi


def q_values(m, R, V) -> np.ndarray:
    Q = np.zeros(m.A * m.nS, dtype=np.float64)
    Rc = np.ascontiguousarray(R, dtype=np.float64)
    Vc = np.ascontiguousarray(V, dtype=np.float64)
    lib().orc_q_values(m.nS, m.A, _p(m.rowptr), _p(m.col), _p(m.prob), _p(Rc), _p(Vc), _p(Q))
    return Q.reshape(m.A, m.nS)


def model_from_csr(nS, A, N, rowptr, col, cnt, R=None) -> OracleModel:
    """Wrap an externally produced paper-layout CSR (e.g. an exported model) for the
    oracle's value iteration, so that solvers can be compared on identical P/R."""
    m = OracleModel(nS, A, np.ascontiguousarray(rowptr, dtype=np.int64),
                    np.ascontiguousarray(col, dtype=np.int64),
                    np.ascontiguousarray(cnt, dtype=np.int32), N, R, None, 0)
    return m


# ----------------------------------------------------------------- rollouts --
def rollout(env, policy, start, objs=(OBJ_TIME,), with_traj=False):
    """Policy rollouts from start = (i0, j0) at t = 0 over the env's N
    realizations (Sec. IV).  policy: [nS] (-1 where undefined).  Returns
    (ret [N][n_obj], steps [N], status [N] (0 target, 1 sink), traj
    [N][nt+1] state after k steps (sink = nS, -1 after the end) or None)."""
    keep = []
    p = make_problem(env, keep)
    pol = np.ascontiguousarray(policy, dtype=np.int32)
    ob = np.ascontiguousarray(objs, dtype=np.int32)
    N = env.N
    ret = np.zeros((N, len(ob)), dtype=np.float64)
    steps = np.zeros(N, dtype=np.int32)
    status = np.zeros(N, dtype=np.int32)
    traj = np.zeros((N, env.nt + 1), dtype=np.int64) if with_traj else None
    st = lib().orc_rollout(C.byref(p), _p(pol), int(start[0]), int(start[1]), _p(ob), len(ob), _p(ret),
                           _p(steps), _p(status), _p(traj))
    if st != 0:
        raise ValueError(f"oracle rollout rejected its arguments ({st})")
    return ret, steps, status, traj


# ---------------------------------------------------------------- 3-D grid --
def build3d_units(env, objs, s_begin, s_end, max_nnz=None):
    """Run the 3-D oracle build over start states [s_begin, s_end) (s = t*Nc + c).
    Returns the raw local-row arrays (nnz, col, cnt, R, overflow, status)."""
    p, keep = _problem3d(env)
    A = env.A
    if max_nnz is None:
        max_nnz = env.L ** 3 + 1
    rows = (s_end - s_begin) * A
    ob = np.ascontiguousarray(objs, dtype=np.int32)
    nnz = np.zeros(rows, dtype=np.int32)
    col = np.zeros(rows * max_nnz, dtype=np.int64)
    cnt = np.zeros(rows * max_nnz, dtype=np.int32)
    R = np.zeros(len(ob) * rows, dtype=np.float64)
    ovf = C.c_int64(0)
    st = lib().orc_build3d(C.byref(p), s_begin, s_end, max_nnz, _p(ob), len(ob), _p(nnz), _p(col),
                           _p(cnt), _p(R), C.byref(ovf))
    return dict(nnz=nnz, col=col.reshape(rows, max_nnz), cnt=cnt.reshape(rows, max_nnz),
                R=R.reshape(len(ob), rows), overflow=ovf.value, status=st)


def _problem3d(env):
    """The ctypes Problem3D of an inputs.Environment3D and the arrays it points into."""
    keep = []

    def hold(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    p = Problem3D()
    p.nx, p.ny, p.nz, p.nt = env.nx, env.ny, env.nz, env.nt
    p.dx, p.dt = env.dx, env.dt
    p.K, p.N, p.A, p.L = env.K, env.N, env.A, env.L
    p.vbar = _p(hold(env.vbar, np.float64))
    p.modes = _p(hold(env.modes, np.float64))
    Y = env.Y if env.Y is not None else coeffs_for(env)
    p.Y = _p(hold(Y, np.float64))
    p.gbar = _p(hold(env.gbar, np.float64))
    p.obstacle = _p(hold(env.obstacle, np.uint8))
    p.target = _p(hold(env.target, np.uint8))
    p.act = _p(hold(env.actions, np.float64))
    p.c_f, p.c_r, p.r_term, p.r_outbound = env.c_f, env.c_r, env.r_term, env.r_outbound
    return p, keep


def build3d(env, objs=(OBJ_TIME,), max_nnz=None) -> OracleModel:
    """The 3-D build (inputs.Environment3D), reordered into the paper layout
    row = a*|S| + s."""
    p, keep = _problem3d(env)
    nS, A = env.nS, env.A
    if max_nnz is None:
        max_nnz = env.L ** 3 + 1
    rows = nS * A
    ob = np.ascontiguousarray(objs, dtype=np.int32)
    nnz = np.zeros(rows, dtype=np.int32)
    col = np.zeros(rows * max_nnz, dtype=np.int64)
    cnt = np.zeros(rows * max_nnz, dtype=np.int32)
    R = np.zeros(len(ob) * rows, dtype=np.float64)
    ovf = C.c_int64(0)
    st = lib().orc_build3d(C.byref(p), 0, nS, max_nnz, _p(ob), len(ob), _p(nnz), _p(col), _p(cnt), _p(R),
                           C.byref(ovf))
    if st != 0:
        raise RuntimeError(f"oracle 3-D build failed with status {st}")
    nnz_local = nnz.reshape(nS, A)
    rowptr = np.zeros(A * nS + 1, dtype=np.int64)
    np.cumsum(np.ascontiguousarray(nnz_local.T).reshape(-1), out=rowptr[1:])
    colp = np.zeros(rowptr[-1], dtype=np.int64)
    cntp = np.zeros(rowptr[-1], dtype=np.int32)
    colL = col.reshape(nS, A, max_nnz)
    cntL = cnt.reshape(nS, A, max_nnz)
    for a in range(A):
        for s_idx in np.nonzero(nnz_local[:, a])[0]:
            r = a * nS + s_idx
            n = nnz_local[s_idx, a]
            colp[rowptr[r]:rowptr[r] + n] = colL[s_idx, a, :n]
            cntp[rowptr[r]:rowptr[r] + n] = cntL[s_idx, a, :n]
    nobj = len(objs)
    Rp = np.ascontiguousarray(R.reshape(nobj, nS, A).transpose(0, 2, 1)).reshape(nobj, A * nS)
    return OracleModel(nS, A, rowptr, colp, cntp, env.N, Rp, None, ovf.value)


def fixed_mask3d(env) -> np.ndarray:
    """1 for 3-D start states whose policy is undefined (targets, obstacles)."""
    tgt = np.broadcast_to(env.target[None], env.obstacle.shape)
    return ((env.obstacle != 0) | (tgt != 0)).astype(np.uint8).reshape(-1)
