"""The 3-D grid build (mdp_build3d) through the C ABI.

Gates (as for 2-D): FP64 check mode -- counts and successor lists
bit-identical to the 3-D oracle, R within 1e-12 relative, values of the
solve within 1e-12; FP32 -- per-entry |d count| <= 2 against the oracle; a
one-layer grid without vertical motion gives the FP32 2-D build's counts
exactly."""
import numpy as np
import pytest

import oracle
from paper_2109_00857_gb300 import inputs
from test_oracle3d_pins import lift

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdp():
    import torch
    torch.cuda.set_device(0)
    from paper_2109_00857_gb300 import build_native, mdp as m
    build_native.build()
    m.load()
    return m


def export_np(mdp, model, obj=0):
    rp, col, cnt, R = mdp.mdp_export_csr(model, obj)
    return rp.cpu().numpy(), col.cpu().numpy(), cnt.cpu().numpy(), R.cpu().numpy()


def rows(rp, col, cnt):
    return [dict(zip(col[rp[r]:rp[r + 1]].tolist(), cnt[rp[r]:rp[r + 1]].tolist())) for r in range(len(rp) - 1)]


CASES = {
    "cube_small": lambda: inputs.cube(nx=10, ny=9, nz=4, nt=4, N=120, with_gbar=True,
                                      objectives=(0, 1, 2)),
    "cube_K1_A_odd": lambda: inputs.make_env3d(nx=7, ny=6, nz=5, nt=3, K=1, N=60, L=7, sigma=(0.3,), seed=9,
                                               amplitude=0.5, n_headings=5, elevations=(0.0, 1.0),
                                               speeds=(0.8,)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_check_mode_equals_the_3d_oracle(mdp, case):
    env = CASES[case]()
    objs = env.objectives if env.gbar is not None else (0,)
    ref = oracle.build3d(env, objs=objs)
    assert ref.overflow == 0
    model = mdp.mdp_build3d(mdp.DeviceEnv3D(env, mdp.MDP_FP64_CHECK), objs=objs)
    for o in range(len(objs)):
        rp, col, cnt, R = export_np(mdp, model, o)
        assert np.array_equal(rp, ref.rowptr) and np.array_equal(col, ref.col) and np.array_equal(cnt, ref.cnt)
        np.testing.assert_allclose(R, ref.R[o], rtol=1e-12, atol=1e-12)
    fx = oracle.fixed_mask3d(env)
    for o in range(len(objs)):
        V, pi, st = mdp.mdp_solve(model, o, tol=0.0)
        Vo, pio, sw, res = oracle.vi_jacobi(ref, ref.R[o], fx, tol=0.0, nt=env.nt)
        assert st.sweeps == sw
        np.testing.assert_allclose(V.cpu().numpy(), Vo, rtol=1e-12, atol=1e-12)
        assert np.array_equal(pi.cpu().numpy(), pio)


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp32_counts_within_2_of_the_oracle(mdp, case):
    env = CASES[case]()
    ref = oracle.build3d(env, objs=(0,))
    model = mdp.mdp_build3d(mdp.DeviceEnv3D(env, mdp.MDP_FP32), objs=(0,))
    rp, col, cnt, R = export_np(mdp, model, 0)
    A_ = rows(rp, col, cnt)
    B_ = rows(ref.rowptr, ref.col, ref.cnt)
    worst = 0
    for x, y in zip(A_, B_):
        for k in set(x) | set(y):
            worst = max(worst, abs(x.get(k, 0) - y.get(k, 0)))
    assert worst <= 2
    np.testing.assert_allclose(R, ref.R[0], rtol=0, atol=2.0 * abs(env.r_outbound) * 2 / env.N + 1e-4)


def test_single_layer_3d_build_equals_the_2d_build(mdp):
    env2 = inputs.energy(nx=16, ny=14, nt=5, N=300, L=11, amplitude=1.5, objectives=(0, 1, 2))
    d2 = mdp.DeviceEnv(env2, mdp.MDP_FP32)
    m2 = mdp.mdp_build(d2, objs=(0, 1, 2))
    m3 = mdp.mdp_build3d(mdp.DeviceEnv3D(lift(env2), mdp.MDP_FP32), objs=(0, 1, 2))
    for o in range(3):
        a2 = export_np(mdp, m2, o)
        a3 = export_np(mdp, m3, o)
        assert all(np.array_equal(x, y) for x, y in zip(a2[:3], a3[:3]))
        np.testing.assert_allclose(a3[3], a2[3], rtol=2e-6, atol=2e-5)


def test_3d_argument_errors(mdp):
    env = inputs.cube(nx=6, ny=6, nz=3, nt=2, N=20)
    d = mdp.DeviceEnv3D(env, mdp.MDP_FP32)
    for L in (4, 13, 0):
        with pytest.raises(mdp.MdpError) as ei:
            mdp.mdp_build3d(d, subgrid_L=L)
        assert ei.value.code == -1
    big = inputs.cube(nx=200, ny=200, nz=2, nt=2, N=4)
    with pytest.raises(mdp.MdpError) as ei:   # 16-bit successor offsets
        mdp.mdp_build3d(mdp.DeviceEnv3D(big, mdp.MDP_FP32), subgrid_L=3)
    assert ei.value.code == -1


RANK_CASES = {
    # one state per slice (24 actions), two (10 actions) and four (6 actions)
    "cube_spw1": lambda: inputs.cube(nx=12, ny=11, nz=5, nt=4, N=300, with_gbar=True, objectives=(0, 1, 2)),
    "spw2": lambda: inputs.make_env3d(nx=9, ny=8, nz=6, nt=4, K=2, N=200, L=9, sigma=(0.3, 0.2), seed=5,
                                      amplitude=0.6, n_headings=5, elevations=(0.0, 0.7), speeds=(0.9,)),
    "spw4": lambda: inputs.make_env3d(nx=10, ny=7, nz=4, nt=3, K=3, N=150, L=7, sigma=(0.3, 0.2, 0.1), seed=6,
                                      amplitude=0.7, n_headings=3, elevations=(-0.5, 0.5), speeds=(1.0,)),
    # wide velocity spreads and many step thresholds (20 actions: up to 8 per
    # axis): about 30 % of the slices' fine tables exceed the warp kernel's
    # memory and are built by the CTA kernel from its list
    "mixed_kernels": lambda: inputs.make_env3d(nx=10, ny=9, nz=5, nt=3, K=3, N=300, L=11, sigma=(0.4, 0.3, 0.25),
                                               seed=8, amplitude=0.2, n_headings=5,
                                               elevations=(-0.7, -0.3, 0.3, 0.7), speeds=(1.0,)),
}


@pytest.mark.parametrize("case", sorted(RANK_CASES))
def test_rank_counting_equals_per_action_counting(mdp, case):
    """FP32: counting each realization once at its fine coordinates (box sums
    of the prefix table; the warp-per-slice kernel, and the CTA kernel for the
    slices whose tables do not fit a warp) gives the same model as one
    increment per (realization, action) -- counts, successors and R bit for
    bit."""
    env = RANK_CASES[case]()
    objs = env.objectives if env.gbar is not None else (0,)
    d = mdp.DeviceEnv3D(env, mdp.MDP_FP32)
    fast = mdp.mdp_build3d(d, objs=objs)
    ref = mdp.mdp_build3d(d, objs=objs, per_action=True)
    assert fast.info().nnz == ref.info().nnz
    if case == "mixed_kernels":   # both rank-counting kernels contributed
        assert 0 < fast.info().wide_slices < env.nS
    for o in range(len(objs)):
        a = export_np(mdp, fast, o)
        b = export_np(mdp, ref, o)
        assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])), (case, o)
        assert np.array_equal(a[3].view(np.uint32), b[3].view(np.uint32)), (case, o)
