"""mdp_solve_noalloc: the Jacobi solve for callers that may not allocate device
memory while they run (a real-time replanning loop, or a program whose device
memory is owned by another allocator).  Its scratch is a fixed array inside the
library.  It must give the same V and policy as mdp_solve, also on a second
call in a row (the array keeps the previous call's contents, so the call has
to clear it), and refuse problems larger than the array.

This file is collected last so that a failure here comes after every other test
has run; it passes alone in a fresh process as well."""
import numpy as np
import pytest

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


def _check_same(V, pi, Vr, pir):
    V = V.cpu().numpy().astype(np.float64)
    Vr = Vr.cpu().numpy().astype(np.float64)
    # the tolerance the solver parity tests use; the kernels are the same, so
    # the results are in fact identical
    assert np.all(np.abs(V - Vr) <= 1e-5 * np.maximum(1.0, np.abs(Vr)))
    assert np.array_equal(pi.cpu().numpy(), pir.cpu().numpy())


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_solve_matches_mdp_solve_twice_in_a_row(mdp, prec):
    import torch
    p = mdp.MDP_FP32 if prec == "fp32" else mdp.MDP_FP64_CHECK
    envs = [inputs.tiny(r_term=5.0), inputs.energy(nx=30, ny=26, nt=6, N=300)]
    for env in envs:
        model = mdp.mdp_build(mdp.DeviceEnv(env, p), objs=env.objectives)
        Vr, pir, str_ = mdp.mdp_solve(model, 0, tol=0.0)
        dt = torch.float64 if p else torch.float32
        V = torch.full((env.nS + 1,), 7.0, dtype=dt, device="cuda")   # garbage in the output
        pi = torch.full((env.nS,), 9, dtype=torch.int16, device="cuda")
        for _ in range(2):    # the second call must not see the first call's scratch
            V, pi, st = mdp.mdp_solve_noalloc(model, 0, tol=0.0, V=V, policy=pi)
            assert st.sweeps == str_.sweeps and st.residual == str_.residual
            _check_same(V, pi, Vr, pir)
        # a tolerance that stops early, then an exact solve again
        _, _, st1 = mdp.mdp_solve_noalloc(model, 0, tol=1e3, V=V, policy=pi)
        assert st1.sweeps == 1
        V, pi, st = mdp.mdp_solve_noalloc(model, 0, tol=0.0, V=V, policy=pi)
        _check_same(V, pi, Vr, pir)


def test_noalloc_solve_rejects_sizes_beyond_its_scratch(mdp):
    env = inputs.tiny(nx=6, ny=6, nt=4, N=20)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32))
    with pytest.raises(mdp.MdpError) as ei:
        mdp.mdp_solve_noalloc(model, 0, max_sweeps=5000)
    assert ei.value.code == -1 and "4092" in str(ei.value)
    big = inputs.make_env(nx=220, ny=220, nt=45, K=1, N=2, L=5, sigma=(0.0,), seed=3,
                          amplitude=0.1, n_headings=4, n_speeds=1)
    assert big.nS > 2_097_151
    m2 = mdp.mdp_build(mdp.DeviceEnv(big, mdp.MDP_FP32))
    with pytest.raises(mdp.MdpError) as ei:
        mdp.mdp_solve_noalloc(m2, 0)
    assert ei.value.code == -1 and "states" in str(ei.value)


def _pool_and_free():
    """(used-memory high-water mark of the device's default memory pool after
    resetting it, a function reading (pool high-water mark, free device
    bytes)) through the CUDA driver API, which sees every stream-ordered
    allocation on the device whichever runtime made it."""
    import ctypes as C
    cu = C.CDLL("libcuda.so.1")
    dev = C.c_int()
    assert cu.cuCtxGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    USED_HIGH = 8   # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def reset():
        zero = C.c_uint64(0)   # resets the high-water mark to the current use
        assert cu.cuMemPoolSetAttribute(pool, USED_HIGH, C.byref(zero)) == 0

    def read():
        hi = C.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, USED_HIGH, C.byref(hi)) == 0
        free, total = C.c_size_t(), C.c_size_t()
        assert cu.cuMemGetInfo_v2(C.byref(free), C.byref(total)) == 0
        return hi.value, free.value
    return reset, read


def test_noalloc_solve_allocates_no_device_memory(mdp):
    """The promise itself: on a warmed model, a call leaves the device
    memory pool's used-memory high-water mark and the free device memory
    exactly where they were (mdp_solve on the same model, for contrast,
    allocates its scratch from that pool)."""
    import torch
    env = inputs.energy(nx=30, ny=26, nt=6, N=300)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=env.objectives)
    V = torch.zeros(env.nS + 1, dtype=torch.float32, device="cuda")
    pi = torch.zeros(env.nS, dtype=torch.int16, device="cuda")
    mdp.mdp_solve_noalloc(model, 0, V=V, policy=pi)     # warm: module loaded, scratch address known
    torch.cuda.synchronize()
    reset, read = _pool_and_free()
    reset()
    before = read()
    for _ in range(2):
        mdp.mdp_solve_noalloc(model, 0, V=V, policy=pi)
    torch.cuda.synchronize()
    assert read() == before
    reset()
    hi0, _ = read()
    mdp.mdp_solve(model, 0, tol=0.0, V=torch.zeros_like(V), policy=torch.zeros_like(pi))
    torch.cuda.synchronize()
    assert read()[0] > hi0   # the allocating solve does show up in the pool


def test_noalloc_full_sweeps_beyond_its_layer_flags(mdp):
    """A model with more time layers than the scratch has layer flags for
    runs full Jacobi sweeps: with an explicit max_sweeps it returns the same
    values, policy, sweep count and residual as mdp_solve; without one the
    default nt + 1 sweeps exceed the scratch and are refused."""
    env = inputs.make_env(nx=2, ny=3, nt=4100, K=1, N=8, L=7, sigma=(0.3,), seed=9,
                          amplitude=0.5, n_headings=4, n_speeds=1, r_term=2.0)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32))
    with pytest.raises(mdp.MdpError) as ei:
        mdp.mdp_solve_noalloc(model, 0)
    assert ei.value.code == -1 and "4092" in str(ei.value)
    for ms, tol in ((12, 0.0), (4092, 1e-3)):
        Vr, pir, sr = mdp.mdp_solve(model, 0, method=mdp.MDP_SOLVE_JACOBI_FULL, tol=tol, max_sweeps=ms)
        for _ in range(2):
            V, pi, st = mdp.mdp_solve_noalloc(model, 0, tol=tol, max_sweeps=ms)
            assert (st.sweeps, st.residual) == (sr.sweeps, sr.residual)
            _check_same(V, pi, Vr, pir)
