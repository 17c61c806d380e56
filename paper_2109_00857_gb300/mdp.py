"""Thin ctypes binding of libmdp_gb300.so (include/mdp.h), same names as the C ABI.

Argument marshalling only: every step of the build and the solve runs in the
library's CUDA kernels.  torch provides device memory and streams.  There is no
CPU fallback: if the library is missing or no CUDA device is present, the calls
raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmdp_gb300.so")

MDP_OK = 0
STATUS = {0: "MDP_OK", -1: "MDP_ERR_ARG", -2: "MDP_ERR_OOM", -3: "MDP_ERR_SUBGRID_OVERFLOW",
          -4: "MDP_ERR_ELL_OVERFLOW", -5: "MDP_ERR_TIMEOUT", -6: "MDP_ERR_CUDA",
          -7: "MDP_ERR_BUDGET", -8: "MDP_ERR_CANCELLED", -9: "MDP_ERR_NOT_FOUND",
          -10: "MDP_ERR_PENDING"}
MDP_OBJ_TIME, MDP_OBJ_ENERGY, MDP_OBJ_NET_ENERGY = 0, 1, 2
MDP_FP32, MDP_FP64_CHECK = 0, 1
MDP_SOLVE_JACOBI, MDP_SOLVE_LAYERED, MDP_SOLVE_JACOBI_FULL = 0, 1, 2
MDP_SOLVE_WARM = 16   # flag: Jacobi starts from the given V

P = C.c_void_p


class MdpGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nt", C.c_int32),
                ("dx", C.c_double), ("dt", C.c_double)]


class MdpActions(C.Structure):
    _fields_ = [("n_headings", C.c_int32), ("n_speeds", C.c_int32), ("f_max", C.c_double),
                ("table_h", P), ("c_f", C.c_double), ("c_r", C.c_double),
                ("r_term", C.c_double), ("r_outbound", C.c_double)]


class MdpEnv(C.Structure):
    _fields_ = [("K", C.c_int32), ("precision", C.c_int32), ("vbar", P), ("modes", P),
                ("coeffs", P), ("sigma_h", P), ("seed", C.c_uint64), ("mdp_id", C.c_uint64),
                ("gbar", P), ("obstacle", P), ("target", P)]


class MdpBuildOpts(C.Structure):
    _fields_ = [("row_cap", C.c_int32), ("no_compact", C.c_int32), ("threads", C.c_int32),
                ("chunk", C.c_int32), ("hist_cap", C.c_int32)]


class MdpModelInfo(C.Structure):
    _fields_ = [("n_states", C.c_int64), ("A", C.c_int32), ("N", C.c_int32), ("L", C.c_int32),
                ("n_obj", C.c_int32), ("objs", C.c_int32 * 3), ("precision", C.c_int32),
                ("rows", C.c_int64), ("nnz", C.c_int64), ("max_row_nnz", C.c_int32),
                ("pool_columns", C.c_int64), ("device_bytes", C.c_int64), ("samples", C.c_int64),
                ("build_ms", C.c_double), ("kernel_ms", C.c_double), ("launches", C.c_int32),
                ("wide_slices", C.c_int64), ("nnz_domain", C.c_int64), ("spill_rows", C.c_int64),
                ("spill_words", C.c_int64), ("max_row_len", C.c_int32)]


class MdpSolveStats(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("residual", C.c_double), ("solve_ms", C.c_double),
                ("backups", C.c_int64)]


class MdpGrid3D(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nt", C.c_int32),
                ("dx", C.c_double), ("dt", C.c_double)]


class MdpEnv3D(C.Structure):
    _fields_ = [("K", C.c_int32), ("precision", C.c_int32), ("vbar", P), ("modes", P), ("coeffs", P),
                ("sigma_h", P), ("seed", C.c_uint64), ("mdp_id", C.c_uint64), ("gbar", P),
                ("obstacle", P), ("target", P)]


class MdpActions3D(C.Structure):
    _fields_ = [("A", C.c_int32), ("table_h", P), ("c_f", C.c_double), ("c_r", C.c_double),
                ("r_term", C.c_double), ("r_outbound", C.c_double)]


class MdpRolloutSummary(C.Structure):
    _fields_ = [("mean_return", C.c_double * 3), ("p_target", C.c_double),
                ("mean_steps_target", C.c_double), ("paths", C.c_int64)]


class MdpTuning(C.Structure):
    _fields_ = [("build_warps", C.c_int32), ("hist_cap", C.c_int32), ("threads", C.c_int32),
                ("chunk", C.c_int32), ("sweep_smem_kb", C.c_int32), ("build_kernel_ms", C.c_double),
                ("sweep_ms", C.c_double), ("candidates", C.c_int32), ("calibration_layers", C.c_int32),
                ("key", C.c_char * 64)]

    def as_dict(self):
        return {"class": self.key.decode(), "build_warps": self.build_warps, "hist_cap": self.hist_cap,
                "threads": self.threads, "chunk": self.chunk, "sweep_smem_kb": self.sweep_smem_kb,
                "build_kernel_ms": self.build_kernel_ms, "sweep_ms": self.sweep_ms,
                "candidates": self.candidates, "calibration_layers": self.calibration_layers}


class MdpBatchItem(C.Structure):
    _fields_ = [("env", MdpEnv), ("grid", MdpGrid), ("actions", MdpActions), ("N", C.c_int32),
                ("subgrid_L", C.c_int32), ("objective", C.c_int32), ("V", P), ("policy", P)]


class MdpRequest(C.Structure):
    _fields_ = [("env_id", C.c_int32), ("start_i", C.c_int32), ("start_j", C.c_int32),
                ("target_i", C.c_int32), ("target_j", C.c_int32), ("target_w", C.c_int32),
                ("target_h", C.c_int32), ("sigma_scale", C.c_double), ("seed", C.c_uint64),
                ("N", C.c_int32), ("objective", C.c_int32), ("tol", C.c_double),
                ("start_t", C.c_int32), ("V0_h", P)]


class MdpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("V_start", C.c_float), ("pi_start", C.c_int16),
                ("sweeps", C.c_int32), ("latency_ms", C.c_double), ("queue_ms", C.c_double),
                ("device_bytes", C.c_int64)]


# name -> (restype, argtypes); every symbol include/mdp.h declares
SIGNATURES = {
    "mdp_build": (C.c_int, [P, P, P, C.c_int32, C.c_int32, P, C.c_int32, P, P, P]),
    "mdp_model_info": (C.c_int, [P, P]),
    "mdp_export_csr": (C.c_int, [P, C.c_int32, P, P, P, P, P]),
    "mdp_solve": (C.c_int, [P, C.c_int32, C.c_int32, C.c_double, C.c_int32, P, P, P, P]),
    "mdp_model_free": (None, [P]),
    "mdp_solve_multi": (C.c_int, [P, C.c_int32, P, C.c_int32, C.c_double, C.c_int32, P, P, P, P]),
    "mdp_solve_noalloc": (C.c_int, [P, C.c_int32, C.c_double, C.c_int32, P, P, P, P]),
    "mdp_build3d": (C.c_int, [P, P, P, C.c_int32, C.c_int32, P, C.c_int32, P, P]),
    "mdp_build3d_ex": (C.c_int, [P, P, P, C.c_int32, C.c_int32, P, C.c_int32, P, P, P]),
    "mdp_rollout": (C.c_int, [P, P, P, C.c_int32, P, P, C.c_int32, P, C.c_int32, P, P, P, P, P]),
    "mdp_sample_coeffs": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, C.c_uint64, C.c_uint64,
                                    C.c_int32, P, P]),
    "mdp_batch_create": (C.c_int, [P, C.c_int32, C.c_double, P]),
    "mdp_batch_run": (C.c_int, [P, P, P, P]),
    "mdp_batch_free": (None, [P]),
    "mdp_serve_create": (C.c_int, [C.c_size_t, C.c_int32, P]),
    "mdp_env_register": (C.c_int, [P, P, P, P, C.c_int32, P]),
    "mdp_serve_submit": (C.c_int, [P, P, P]),
    "mdp_serve_poll": (C.c_int, [P, C.c_uint64, C.c_int32, P, P, P]),
    "mdp_serve_stats": (C.c_int, [P, P, P, P]),
    "mdp_serve_destroy": (C.c_int, [P]),
    "mdp_last_error": (C.c_char_p, []),
    "mdp_test_inject": (C.c_int, [C.c_int32, C.c_int64]),
    "mdp_autotune": (C.c_int, [P, P, P, C.c_int32, C.c_int32, P, C.c_int32, C.c_char_p, P, P]),
    "mdp_tuning_load": (C.c_int, [C.c_char_p]),
    "mdp_version": (C.c_char_p, []),
}

_lib = None


class MdpError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the CUDA library.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libmdp_gb300.so not found at {path}; run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(code: int, where: str):
    if code != MDP_OK:
        raise MdpError(code, where, load().mdp_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return int(t.data_ptr())


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------- marshalling --
class DeviceEnv:
    """Device copies (torch tensors) of an inputs.Environment in one precision."""

    def __init__(self, env, precision: int = MDP_FP32, device="cuda", with_coeffs: bool = False):
        import torch
        ft = torch.float64 if precision == MDP_FP64_CHECK else torch.float32
        self.env, self.precision = env, precision
        self.vbar = torch.as_tensor(np.ascontiguousarray(env.vbar)).to(device, ft).contiguous()
        self.modes = torch.as_tensor(np.ascontiguousarray(env.modes)).to(device, ft).contiguous()
        self.gbar = (torch.as_tensor(np.ascontiguousarray(env.gbar)).to(device, ft).contiguous()
                     if env.gbar is not None else None)
        self.obstacle = torch.as_tensor(np.ascontiguousarray(env.obstacle, dtype=np.uint8)).to(device)
        self.target = torch.as_tensor(np.ascontiguousarray(env.target, dtype=np.uint8)).to(device)
        self.coeffs = None
        if env.Y is not None:
            self.coeffs = torch.as_tensor(np.ascontiguousarray(env.Y)).to(device, ft).contiguous()
        self.sigma = np.ascontiguousarray(env.sigma, dtype=np.float64)
        self.table = np.ascontiguousarray(env.actions, dtype=np.float64)

    def c_env(self) -> MdpEnv:
        e = MdpEnv()
        e.K = self.env.K
        e.precision = self.precision
        e.vbar, e.modes = _ptr(self.vbar), _ptr(self.modes)
        e.coeffs = _ptr(self.coeffs)
        e.sigma_h = self.sigma.ctypes.data_as(P).value
        e.seed, e.mdp_id = int(self.env.seed), int(self.env.mdp_id)
        e.gbar = _ptr(self.gbar)
        e.obstacle, e.target = _ptr(self.obstacle), _ptr(self.target)
        return e

    def c_grid(self) -> MdpGrid:
        g = MdpGrid()
        g.nx, g.ny, g.nt, g.dx, g.dt = self.env.nx, self.env.ny, self.env.nt, self.env.dx, self.env.dt
        return g

    def c_actions(self) -> MdpActions:
        a = MdpActions()
        a.n_headings, a.n_speeds = self.env.A, 1
        a.f_max = float(self.table[:, 2].max())
        a.table_h = self.table.ctypes.data_as(P).value
        a.c_f, a.c_r = self.env.c_f, self.env.c_r
        a.r_term, a.r_outbound = self.env.r_term, self.env.r_outbound
        return a


class DeviceEnv3D:
    """Device copies (torch tensors) of an inputs.Environment3D in one precision."""

    def __init__(self, env, precision: int = MDP_FP32, device="cuda"):
        import torch
        ft = torch.float64 if precision == MDP_FP64_CHECK else torch.float32
        self.env, self.precision = env, precision
        self.vbar = torch.as_tensor(np.ascontiguousarray(env.vbar)).to(device, ft).contiguous()
        self.modes = torch.as_tensor(np.ascontiguousarray(env.modes)).to(device, ft).contiguous()
        self.gbar = (torch.as_tensor(np.ascontiguousarray(env.gbar)).to(device, ft).contiguous()
                     if env.gbar is not None else None)
        self.obstacle = torch.as_tensor(np.ascontiguousarray(env.obstacle, dtype=np.uint8)).to(device)
        self.target = torch.as_tensor(np.ascontiguousarray(env.target, dtype=np.uint8)).to(device)
        self.coeffs = None
        if env.Y is not None:
            self.coeffs = torch.as_tensor(np.ascontiguousarray(env.Y)).to(device, ft).contiguous()
        self.sigma = np.ascontiguousarray(env.sigma, dtype=np.float64)
        self.table = np.ascontiguousarray(env.actions, dtype=np.float64)

    def c_env(self) -> MdpEnv3D:
        e = MdpEnv3D()
        e.K, e.precision = self.env.K, self.precision
        e.vbar, e.modes, e.coeffs = _ptr(self.vbar), _ptr(self.modes), _ptr(self.coeffs)
        e.sigma_h = self.sigma.ctypes.data_as(P).value
        e.seed, e.mdp_id = int(self.env.seed), int(self.env.mdp_id)
        e.gbar = _ptr(self.gbar)
        e.obstacle, e.target = _ptr(self.obstacle), _ptr(self.target)
        return e

    def c_grid(self) -> MdpGrid3D:
        g = MdpGrid3D()
        g.nx, g.ny, g.nz, g.nt = self.env.nx, self.env.ny, self.env.nz, self.env.nt
        g.dx, g.dt = self.env.dx, self.env.dt
        return g

    def c_actions(self) -> MdpActions3D:
        a = MdpActions3D()
        a.A = self.env.A
        a.table_h = self.table.ctypes.data_as(P).value
        a.c_f, a.c_r, a.r_term, a.r_outbound = self.env.c_f, self.env.c_r, self.env.r_term, self.env.r_outbound
        return a


class Model:
    """Owner of an mdp_model handle."""

    def __init__(self, handle: int, precision: int):
        self.handle = handle
        self.precision = precision

    def info(self) -> MdpModelInfo:
        return mdp_model_info(self)

    def free(self):
        if self.handle:
            load().mdp_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- calls --
def mdp_build(denv: DeviceEnv, N: Optional[int] = None, subgrid_L: Optional[int] = None,
              objs: Sequence[int] = (MDP_OBJ_TIME,), opts: Optional[MdpBuildOpts] = None,
              stream=None) -> Model:
    lib = load()
    e, g, a = denv.c_env(), denv.c_grid(), denv.c_actions()
    ob = np.ascontiguousarray(objs, dtype=np.int32)
    h = P()
    N = denv.env.N if N is None else N
    L = denv.env.L if subgrid_L is None else subgrid_L
    code = lib.mdp_build(C.byref(e), C.byref(g), C.byref(a), N, L, ob.ctypes.data_as(P), len(ob),
                         C.byref(opts) if opts is not None else None, _stream(stream), C.byref(h))
    _check(code, "mdp_build")
    return Model(h.value, denv.precision)


class MdpBuild3DOpts(C.Structure):
    _fields_ = [("per_action", C.c_int32)]


def mdp_build3d(denv: DeviceEnv3D, objs: Sequence[int] = (MDP_OBJ_TIME,), N: Optional[int] = None,
                subgrid_L: Optional[int] = None, stream=None, per_action: bool = False) -> Model:
    """The build on a 3-D grid; the model works with mdp_solve / mdp_export_csr.
    per_action=True counts one increment per (realization, action) on every
    slice (mdp_build3d_opts.per_action; the same model)."""
    e, g, a = denv.c_env(), denv.c_grid(), denv.c_actions()
    ob = np.ascontiguousarray(objs, dtype=np.int32)
    h = P()
    N = denv.env.N if N is None else N
    L = denv.env.L if subgrid_L is None else subgrid_L
    o = MdpBuild3DOpts(1 if per_action else 0)
    _check(load().mdp_build3d_ex(C.byref(e), C.byref(g), C.byref(a), N, L, ob.ctypes.data_as(P), len(ob),
                                 C.byref(o), _stream(stream), C.byref(h)), "mdp_build3d")
    return Model(h.value, denv.precision)


def mdp_model_info(model: Model) -> MdpModelInfo:
    info = MdpModelInfo()
    _check(load().mdp_model_info(model.handle, C.byref(info)), "mdp_model_info")
    return info


def mdp_export_csr(model: Model, obj: int = 0, stream=None, with_entries: bool = True):
    """Paper-layout CSR (row = a*|S| + s) as torch device tensors (rowptr, col, count, R);
    with_entries=False skips col and count (returned as None)."""
    import torch
    info = mdp_model_info(model)
    rows = info.rows
    rowptr = torch.empty(rows + 1, dtype=torch.int64, device="cuda")
    col = cnt = None
    if with_entries:
        col = torch.empty(max(info.nnz, 1), dtype=torch.int64, device="cuda")
        cnt = torch.empty(max(info.nnz, 1), dtype=torch.int32, device="cuda")
    R = torch.empty(rows, dtype=torch.float64 if model.precision else torch.float32, device="cuda")
    _check(load().mdp_export_csr(model.handle, obj, _ptr(rowptr), _ptr(col), _ptr(cnt), _ptr(R),
                                 _stream(stream)), "mdp_export_csr")
    if not with_entries:
        return rowptr, None, None, R
    return rowptr, col[:info.nnz], cnt[:info.nnz], R


def mdp_solve(model: Model, obj: int = 0, method: int = MDP_SOLVE_JACOBI, tol: float = 0.0,
              max_sweeps: int = 0, V=None, policy=None, stream=None, warm: bool = False):
    """Returns (V, policy, MdpSolveStats); V / policy are torch device tensors.
    warm=True (MDP_SOLVE_WARM): Jacobi starts from the given V instead of 0."""
    if warm:
        if V is None:
            raise ValueError("a warm start needs V")
        method |= MDP_SOLVE_WARM
    import torch
    info = mdp_model_info(model)
    if V is None:
        V = torch.empty(info.n_states + 1, dtype=torch.float64 if model.precision else torch.float32,
                        device="cuda")
    if policy is None:
        policy = torch.empty(info.n_states, dtype=torch.int16, device="cuda")
    st = MdpSolveStats()
    _check(load().mdp_solve(model.handle, obj, method, float(tol), int(max_sweeps), _ptr(V),
                            _ptr(policy), _stream(stream), C.byref(st)), "mdp_solve")
    return V, policy, st


def mdp_solve_multi(model: Model, objs=(0,), method: int = MDP_SOLVE_JACOBI, tol: float = 0.0,
                    max_sweeps: int = 0, V=None, policy=None, stream=None):
    """Solves 1..3 objective slots in one fused pass over P per sweep.
    Returns (list of V, list of policy, list of MdpSolveStats), one per slot."""
    import torch
    info = mdp_model_info(model)
    n = len(objs)
    dt = torch.float64 if model.precision else torch.float32
    if V is None:
        V = [torch.empty(info.n_states + 1, dtype=dt, device="cuda") for _ in range(n)]
    if policy is None:
        policy = [torch.empty(info.n_states, dtype=torch.int16, device="cuda") for _ in range(n)]
    if len(V) != n or len(policy) != n:
        raise ValueError("V and policy need one tensor per objective")
    o_arr = (C.c_int32 * max(n, 1))(*objs)
    v_arr = (C.c_void_p * max(n, 1))(*[_ptr(x) for x in V])
    p_arr = (C.c_void_p * max(n, 1))(*[_ptr(x) for x in policy])
    st = (MdpSolveStats * max(n, 1))()
    _check(load().mdp_solve_multi(model.handle, n, o_arr, method, float(tol), int(max_sweeps), v_arr,
                                  p_arr, _stream(stream), st), "mdp_solve_multi")
    return list(V), list(policy), [st[i] for i in range(n)]


def mdp_solve_noalloc(model: Model, obj: int = 0, tol: float = 0.0, max_sweeps: int = 0, V=None,
                      policy=None, stream=None):
    """Jacobi solve whose scratch is a fixed array inside the library: no device
    allocation happens in the call (V and policy must be passed in by a caller
    that cannot allocate; they are allocated here only for convenience when
    omitted).  Returns (V, policy, MdpSolveStats)."""
    import torch
    info = mdp_model_info(model)
    if V is None:
        V = torch.empty(info.n_states + 1, dtype=torch.float64 if model.precision else torch.float32,
                        device="cuda")
    if policy is None:
        policy = torch.empty(info.n_states, dtype=torch.int16, device="cuda")
    st = MdpSolveStats()
    _check(load().mdp_solve_noalloc(model.handle, obj, float(tol), int(max_sweeps), _ptr(V),
                                    _ptr(policy), _stream(stream), C.byref(st)), "mdp_solve_noalloc")
    return V, policy, st


def mdp_rollout(denv: "DeviceEnv", policy, starts, objs=(MDP_OBJ_TIME,), N: Optional[int] = None,
                paths: bool = True, stream=None):
    """Policy rollouts from each start (i, j) at t = 0 over N realizations.
    Returns (ret [n_starts][N][n_obj], steps [n_starts][N], status [n_starts][N])
    as torch device tensors (None unless paths) and a list of MdpRolloutSummary."""
    import torch
    st = np.ascontiguousarray(starts, dtype=np.int32).reshape(-1, 2)
    ob = np.ascontiguousarray(objs, dtype=np.int32)
    N = denv.env.N if N is None else N
    n = st.shape[0]
    ret = steps = status = None
    if paths:
        dt = torch.float64 if denv.precision else torch.float32
        ret = torch.empty((n, N, len(ob)), dtype=dt, device="cuda")
        steps = torch.empty((n, N), dtype=torch.int32, device="cuda")
        status = torch.empty((n, N), dtype=torch.int8, device="cuda")
    e, g, a = denv.c_env(), denv.c_grid(), denv.c_actions()
    summ = (MdpRolloutSummary * n)()
    _check(load().mdp_rollout(C.byref(e), C.byref(g), C.byref(a), int(N), _ptr(policy), st.ctypes.data_as(P), n,
                              ob.ctypes.data_as(P), len(ob), _ptr(ret), _ptr(steps), _ptr(status), summ,
                              _stream(stream)), "mdp_rollout")
    return ret, steps, status, [summ[q] for q in range(n)]


def mdp_sample_coeffs(nt: int, N: int, K: int, sigma, seed: int, mdp_id: int = 0,
                      precision: int = MDP_FP32, stream=None):
    import torch
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    Y = torch.empty((nt, N, K), dtype=torch.float64 if precision else torch.float32, device="cuda")
    _check(load().mdp_sample_coeffs(nt, N, K, sig.ctypes.data_as(P), seed, mdp_id, precision,
                                    _ptr(Y), _stream(stream)), "mdp_sample_coeffs")
    return Y


def mdp_autotune(denv: DeviceEnv, objs: Sequence[int] = (MDP_OBJ_TIME,), N: Optional[int] = None,
                 subgrid_L: Optional[int] = None, json_path: Optional[str] = None, stream=None) -> MdpTuning:
    """Times the launch-shape candidates on a calibration cut of denv's
    environment, records the fastest for its workload class (and in json_path)."""
    lib = load()
    e, g, a = denv.c_env(), denv.c_grid(), denv.c_actions()
    ob = np.ascontiguousarray(objs, dtype=np.int32)
    out = MdpTuning()
    N = denv.env.N if N is None else N
    L = denv.env.L if subgrid_L is None else subgrid_L
    _check(lib.mdp_autotune(C.byref(e), C.byref(g), C.byref(a), N, L, ob.ctypes.data_as(P), len(ob),
                            json_path.encode() if json_path else None, _stream(stream), C.byref(out)),
           "mdp_autotune")
    return out


def mdp_tuning_load(json_path: str):
    _check(load().mdp_tuning_load(json_path.encode()), "mdp_tuning_load")


def mdp_version() -> str:
    return load().mdp_version().decode()


# ---------------------------------------------------------------- serving --
class Server:
    """Replanning server (mdp_serve_*): resident environments, FIFO admission
    under an HBM budget, concurrent requests on per-slot streams."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int):
        h = P()
        _check(load().mdp_serve_create(int(hbm_budget_bytes), int(max_slots), C.byref(h)),
               "mdp_serve_create")
        self.handle = h.value
        self._envs = []
        self._start_t = {}
        self._keep = {}   # ticket -> host starting values the server reads

    def register(self, denv: DeviceEnv, subgrid_L: Optional[int] = None) -> int:
        e, g, a = denv.c_env(), denv.c_grid(), denv.c_actions()
        e.coeffs = None
        eid = C.c_int32()
        L = denv.env.L if subgrid_L is None else subgrid_L
        _check(load().mdp_env_register(self.handle, C.byref(e), C.byref(g), C.byref(a), L,
                                       C.byref(eid)), "mdp_env_register")
        self._envs.append(denv.env)
        return eid.value

    def submit(self, env_id, start, target, target_size=(2, 2), sigma_scale=1.0, seed=0, N=1000,
               objective=MDP_OBJ_TIME, tol=0.0, start_t=0, V0=None) -> int:
        """V0: host float32 array [|S|+1] starting a Jacobi request (tol > 0), e.g.
        the V polled from an earlier request; kept alive until the poll."""
        r = MdpRequest()
        r.env_id = env_id
        r.start_i, r.start_j = start
        r.target_i, r.target_j = target
        r.target_w, r.target_h = target_size
        r.sigma_scale, r.seed, r.N, r.objective, r.tol = sigma_scale, seed, N, objective, tol
        r.start_t = start_t
        v0 = None
        if V0 is not None:
            v0 = np.ascontiguousarray(V0, dtype=np.float32)
            env = self._envs[env_id]
            if v0.size != (env.nt - start_t) * env.Nc + 1:
                raise ValueError("V0 must hold |S| + 1 values of the request's horizon")
            r.V0_h = v0.ctypes.data_as(P)
        t = C.c_uint64()
        _check(load().mdp_serve_submit(self.handle, C.byref(r), C.byref(t)), "mdp_serve_submit")
        self._start_t[t.value] = start_t
        if v0 is not None:
            self._keep[t.value] = v0
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0, env_id: Optional[int] = None, want_V=False):
        """Returns (MdpResult, V, policy) or None while pending; V/policy are
        numpy arrays when want_V (env_id gives their size)."""
        res = MdpResult()
        V = pi = None
        if want_V:
            env = self._envs[env_id]
            nS = (env.nt - self._start_t.get(int(ticket), 0)) * env.Nc
            V = np.empty(nS + 1, dtype=np.float32)
            pi = np.empty(nS, dtype=np.int16)
        code = load().mdp_serve_poll(self.handle, int(ticket), int(timeout_ms), C.byref(res),
                                     V.ctypes.data_as(P) if V is not None else None,
                                     pi.ctypes.data_as(P) if pi is not None else None)
        if code == -10:
            return None
        self._keep.pop(int(ticket), None)
        _check(code, "mdp_serve_poll")
        return res, V, pi

    def stats(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().mdp_serve_stats(self.handle, C.byref(a), C.byref(b), C.byref(c)),
               "mdp_serve_stats")
        return a.value, b.value, c.value

    def close(self):
        if self.handle:
            load().mdp_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------- batching --
class Batch:
    """Many MDPs built and solved together (mdp_batch_*): persistent build
    launches, then per batched step (a Jacobi sweep for tol > 0, a time layer
    of the layered pass for tol = 0) one plan and one Bellman launch per solve
    class over all items, captured in a CUDA graph on the first run.  Keeps
    the DeviceEnvs and outputs alive."""

    def __init__(self, denvs, objectives=None, tol: float = 0.0):
        import torch
        self.denvs = list(denvs)
        n = len(self.denvs)
        arr = (MdpBatchItem * n)()
        self.V, self.policy = [], []
        for i, d in enumerate(self.denvs):
            it = arr[i]
            it.env, it.grid, it.actions = d.c_env(), d.c_grid(), d.c_actions()
            it.N, it.subgrid_L = d.env.N, d.env.L
            it.objective = (objectives[i] if objectives is not None else d.env.objectives[0])
            V = torch.empty(d.env.nS + 1, dtype=torch.float32, device="cuda")
            pi = torch.empty(d.env.nS, dtype=torch.int16, device="cuda")
            self.V.append(V)
            self.policy.append(pi)
            it.V, it.policy = _ptr(V), _ptr(pi)
        h = P()
        _check(load().mdp_batch_create(arr, n, float(tol), C.byref(h)), "mdp_batch_create")
        self.handle = h.value
        self.n = n

    def run(self, stream=None):
        """Returns (sweeps per item, device ms of the run)."""
        sw = (C.c_int32 * self.n)()
        ms = C.c_double()
        _check(load().mdp_batch_run(self.handle, _stream(stream), sw, C.byref(ms)), "mdp_batch_run")
        return list(sw), ms.value

    def close(self):
        if self.handle:
            load().mdp_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
