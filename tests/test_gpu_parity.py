"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Gates (written in each test):
  FP64 check mode  counts and successor lists bit-identical; R within 1e-12
                   relative; V within 1e-12 relative.
  FP32 production  per-entry |dP| <= 2/N (|d count| <= 2); R within the bound
                   implied by the count differences plus FP32 rounding.
  solver           on identical P/R (the GPU's exported model fed to the oracle's
                   value iteration): |dV| <= 1e-5 max(1, |V|); a policy differs
                   only where the oracle's Q of the two actions differ by
                   <= 1e-6 max(1, |Q|) (a tie).
"""
import numpy as np
import pytest

import oracle
from conftest import custom_env, policy_tie_check
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


def export_np(mdp, model, obj=0):
    rp, col, cnt, R = mdp.mdp_export_csr(model, obj)
    return rp.cpu().numpy(), col.cpu().numpy(), cnt.cpu().numpy(), R.cpu().numpy()


def row_dicts(rowptr, col, cnt):
    out = []
    for r in range(len(rowptr) - 1):
        out.append(dict(zip(col[rowptr[r]:rowptr[r + 1]].tolist(), cnt[rowptr[r]:rowptr[r + 1]].tolist())))
    return out


def max_count_diff(rp_a, col_a, cnt_a, rp_b, col_b, cnt_b):
    A = row_dicts(rp_a, col_a, cnt_a)
    B = row_dicts(rp_b, col_b, cnt_b)
    worst, l1 = 0, np.zeros(len(A))
    for r, (x, y) in enumerate(zip(A, B)):
        keys = set(x) | set(y)
        d = [abs(x.get(k, 0) - y.get(k, 0)) for k in keys]
        if d:
            worst = max(worst, max(d))
            l1[r] = sum(d)
    return worst, l1


# --------------------------------------------------------------- sampler ----
def test_sampler_fp64_bit_identical_and_fp32_is_rounded(mdp):
    sig = [0.3, 0.2, 0.15, 0.1, 0.05]
    Y64 = mdp.mdp_sample_coeffs(7, 301, 5, sig, seed=22, mdp_id=3,
                                precision=mdp.MDP_FP64_CHECK).cpu().numpy()
    ref = oracle.sample_coeffs(7, 301, 5, sig, seed=22, mdp_id=3)
    assert np.array_equal(Y64.view(np.uint64), ref.view(np.uint64))
    Y32 = mdp.mdp_sample_coeffs(7, 301, 5, sig, seed=22, mdp_id=3, precision=mdp.MDP_FP32).cpu().numpy()
    assert np.array_equal(Y32, ref.astype(np.float32))


# ---------------------------------------------------- FP64 check mode -----
CHECK_CASES = {
    "tiny": lambda: inputs.tiny(),
    "tiny_rterm": lambda: inputs.tiny(nx=13, ny=11, nt=6, N=77, r_term=4.0),
    "energy_small": lambda: inputs.energy(nx=24, ny=20, nt=5, N=50, L=15),
    "three_objectives": lambda: inputs.large(nx=18, ny=18, nt=4, N=40, L=15, square=5),
    "external_coeffs": lambda: inputs.tiny(nx=10, ny=10, nt=5, N=33, external_Y=True),
    "A12_ragged": lambda: inputs.make_env(nx=9, ny=7, nt=4, K=3, N=25, L=9, sigma=(0.3, 0.2, 0.1),
                                          seed=5, amplitude=0.8, n_headings=12, n_speeds=1,
                                          obstacle="squares", square=3),
    "A1": lambda: inputs.make_env(nx=6, ny=5, nt=4, K=1, N=20, L=7, sigma=(0.4,), seed=6,
                                  amplitude=0.5, n_headings=1, n_speeds=1),
    "A3_odd_cells": lambda: inputs.make_env(nx=5, ny=3, nt=3, K=2, N=9, L=7, sigma=(0.4, 0.3),
                                            seed=7, amplitude=0.5, n_headings=3, n_speeds=1),
}


@pytest.mark.parametrize("case", sorted(CHECK_CASES))
def test_check_mode_counts_bit_identical(mdp, case):
    env = CHECK_CASES[case]()
    objs = env.objectives
    ref = oracle.build(env, objs=objs)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP64_CHECK), objs=objs)
    for o in range(len(objs)):
        rp, col, cnt, R = export_np(mdp, model, o)
        assert np.array_equal(rp, ref.rowptr)
        assert np.array_equal(col, ref.col)
        assert np.array_equal(cnt, ref.cnt)
        np.testing.assert_allclose(R, ref.R[o], rtol=1e-12, atol=1e-12)
    # check-mode solve = oracle VI on the same model, to 1e-12
    fx = oracle.fixed_mask(env)
    for o in range(len(objs)):
        V, pi, st = mdp.mdp_solve(model, o, tol=0.0)
        Vo, pio, sw, res = oracle.vi_jacobi(ref, ref.R[o], fx, tol=0.0, nt=env.nt)
        assert st.sweeps == sw
        np.testing.assert_allclose(V.cpu().numpy(), Vo, rtol=1e-12, atol=1e-12)
        assert np.array_equal(pi.cpu().numpy(), pio)


def test_check_mode_edge_environments(mdp):
    """Obstacle cells that are also targets, nt = 1 (every row at the horizon),
    N = 1, a 1x1 grid, and no modes."""
    nt = 3
    obs = np.zeros((nt, 6, 6), np.uint8)
    obs[:, 2, 2] = 1
    obs[1, 3, 3] = 1
    tgt = np.zeros((6, 6), np.uint8)
    tgt[3, 3] = 1
    tgt[2, 2] = 1
    modes = np.zeros((nt, 1, 6, 6, 2))
    modes[..., 0] = 1.0
    cases = [
        custom_env(nx=6, ny=6, nt=nt, K=1, N=40, L=7, modes=modes, sigma=[0.5], obstacle=obs,
                   target=tgt, r_term=2.0, r_outbound=-30.0),
        custom_env(nx=4, ny=4, nt=1, K=1, N=5, L=5, r_outbound=-3.0),
        custom_env(nx=5, ny=5, nt=3, K=1, N=1, L=5, modes=modes[:, :, :5, :5], sigma=[0.7]),
        custom_env(nx=1, ny=1, nt=2, K=1, N=3, L=3),
        custom_env(nx=5, ny=4, nt=3, K=0, N=4, L=5, modes=np.zeros((3, 0, 4, 5, 2)), sigma=[]),
    ]
    for env in cases:
        ref = oracle.build(env)
        model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP64_CHECK))
        rp, col, cnt, R = export_np(mdp, model)
        assert np.array_equal(rp, ref.rowptr)
        assert np.array_equal(col, ref.col)
        assert np.array_equal(cnt, ref.cnt)
        np.testing.assert_allclose(R, ref.R[0], rtol=1e-12, atol=1e-12)


def test_subgrid_overflow_is_an_error_on_both_paths(mdp):
    vbar = np.zeros((3, 7, 7, 2))
    vbar[..., 0] = 2.2
    env = custom_env(nx=7, ny=7, nt=3, N=4, L=5, vbar=vbar)
    assert oracle.build(env).overflow > 0
    for prec in (mdp.MDP_FP64_CHECK, mdp.MDP_FP32):
        with pytest.raises(mdp.MdpError) as ei:
            mdp.mdp_build(mdp.DeviceEnv(env, prec))
        assert ei.value.code == -3
    env.L = 7
    for prec in (mdp.MDP_FP64_CHECK, mdp.MDP_FP32):
        mdp.mdp_build(mdp.DeviceEnv(env, prec))


def test_non_finite_velocities_are_a_subgrid_overflow(mdp):
    """An infinite or NaN mean velocity in one cell lands outside every
    sub-grid: the FP32 build reports MDP_ERR_SUBGRID_OVERFLOW (the warp kernel
    hands such a state to the full-window kernel, which counts it), and the
    same fields without it build."""
    for bad in (np.inf, -np.inf, np.nan):
        vbar = np.zeros((3, 7, 7, 2))
        vbar[0, 3, 2, 1] = bad
        env = custom_env(nx=7, ny=7, nt=3, N=8, L=5, vbar=vbar)
        with pytest.raises(mdp.MdpError) as ei:
            mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32))
        assert ei.value.code == -3, bad
    mdp.mdp_build(mdp.DeviceEnv(custom_env(nx=7, ny=7, nt=3, N=8, L=5), mdp.MDP_FP32))


def test_automatic_subgrid_holds_every_landing(mdp):
    env = inputs.energy(nx=20, ny=20, nt=4, N=60)
    m = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), subgrid_L=0, objs=(0,))
    L = m.info().L
    assert L % 2 == 1 and L <= 31
    env.L = L
    ref = oracle.build(env, objs=(0,))
    assert ref.overflow == 0


def test_invalid_arguments_are_rejected(mdp):
    env = inputs.tiny(nx=6, ny=6, nt=3, N=10)
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    for kw in (dict(N=0), dict(N=70000), dict(subgrid_L=4), dict(subgrid_L=257), dict(objs=(7,)),
               dict(objs=(2,))):
        with pytest.raises(mdp.MdpError) as ei:
            mdp.mdp_build(d, **kw)
        assert ei.value.code == -1


# ------------------------------------------------------- FP32 production ----
FP32_CASES = {
    "tiny": lambda: inputs.tiny(),
    "energy_small": lambda: inputs.energy(nx=30, ny=26, nt=6, N=400),
    "three_objectives": lambda: inputs.large(nx=22, ny=22, nt=5, N=300, L=15, square=5),
    "A12_ragged": lambda: inputs.make_env(nx=9, ny=7, nt=4, K=3, N=250, L=9, sigma=(0.3, 0.2, 0.1),
                                          seed=5, amplitude=0.8, n_headings=12, n_speeds=1,
                                          obstacle="squares", square=3),
    "wide_rows_pool_retry": lambda: custom_env(
        nx=9, ny=9, nt=3, K=2, N=3000, L=15, seed=12, sigma=[1.1, 1.0],
        modes=np.stack([np.stack([np.ones((3, 9, 9)), np.zeros((3, 9, 9))], -1),
                        np.stack([np.zeros((3, 9, 9)), np.ones((3, 9, 9))], -1)], 1)),
    "K7_runtime_modes": lambda: inputs.make_env(nx=12, ny=12, nt=4, K=7, N=300, L=15,
                                                sigma=tuple(0.2 for _ in range(7)), seed=8,
                                                amplitude=1.0, n_headings=16, n_speeds=2),
}


def check_fp32_against_oracle(mdp, env, objs, model=None, chunk=None):
    ref = oracle.build(env, objs=objs)
    if model is None:
        opts = None
        if chunk:
            opts = mdp.MdpBuildOpts()
            opts.chunk = chunk
        model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=objs, opts=opts)
    rmax = max(abs(env.r_outbound), 1.0 + abs(env.r_term) + 4.0)
    for o in range(len(objs)):
        rp, col, cnt, R = export_np(mdp, model, o)
        worst, l1 = max_count_diff(rp, col, cnt, ref.rowptr, ref.col, ref.cnt)
        assert worst <= 2, f"|d count| = {worst} > 2 (|dP| > 2/N)"
        tol = l1 / env.N * rmax + 1e-5 * np.maximum(1.0, np.abs(ref.R[o]))
        assert np.all(np.abs(R.astype(np.float64) - ref.R[o]) <= tol)
        # row sums: every non-terminal row holds exactly N realizations
        sums = np.add.reduceat(cnt, rp[:-1]) if len(cnt) else np.zeros(0)
        nonempty = np.diff(rp) > 0
        assert np.all(sums[nonempty] == env.N)
    return model, ref


@pytest.mark.parametrize("case", sorted(FP32_CASES))
def test_fp32_build_within_2_over_N(mdp, case):
    env = FP32_CASES[case]()
    check_fp32_against_oracle(mdp, env, env.objectives)


def test_fp32_chunked_realizations_match(mdp):
    """Realizations staged in several chunks give the same counts as one chunk."""
    env = inputs.energy(nx=16, ny=16, nt=4, N=700)
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    outs = []
    for ch in (700, 128, 33):
        o = mdp.MdpBuildOpts()
        o.chunk = ch
        outs.append(export_np(mdp, mdp.mdp_build(d, objs=(0,), opts=o)))
    for x in outs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(outs[0][:3], x[:3]))
        np.testing.assert_allclose(outs[0][3], x[3], rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("case", ["tiny", "energy_small", "three_objectives", "A12_ragged",
                                  "wide_rows_pool_retry"])
def test_warp_kernel_and_full_window_kernel_agree_bitwise(mdp, case):
    """The warp-per-slice kernel and the full-window CTA kernel (used for slices
    whose histogram does not fit) evaluate the same FP32 operations: forcing
    every slice through either one gives the same model bit for bit."""
    env = FP32_CASES[case]()
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    outs = []
    for cap in (0, 1, 24):
        o = mdp.MdpBuildOpts()
        o.hist_cap = cap
        m = mdp.mdp_build(d, objs=env.objectives, opts=o)
        info = m.info()
        if cap == 1:
            assert info.wide_slices > 0
        outs.append([export_np(mdp, m, k) for k in range(len(env.objectives))])
    for x in outs[1:]:
        for a_, b_ in zip(outs[0], x):
            assert all(np.array_equal(p, q) for p, q in zip(a_, b_))


def test_fp32_build_is_deterministic_across_block_shapes(mdp):
    env = inputs.tiny(nx=15, ny=15, nt=5, N=300)
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    outs = []
    for th in (64, 256, 512):
        o = mdp.MdpBuildOpts()
        o.threads = th
        outs.append(export_np(mdp, mdp.mdp_build(d, opts=o)))
    for x in outs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(outs[0], x))


# ------------------------------------------------------------ solver ----
def solver_parity(mdp, env, model, obj=0, method=0):
    V, pi, st = mdp.mdp_solve(model, obj, method=method, tol=0.0)
    V = V.cpu().numpy().astype(np.float64)
    pi = pi.cpu().numpy()
    rp, col, cnt, R = export_np(mdp, model, obj)
    om = oracle.model_from_csr(env.nS, env.A, env.N, rp, col, cnt)
    R64 = R.astype(np.float64)
    fx = oracle.fixed_mask(env)
    Vo, pio, sw, res = oracle.vi_jacobi(om, R64, fx, tol=0.0, nt=env.nt)
    scale = np.maximum(1.0, np.abs(Vo))
    assert np.all(np.abs(V - Vo) <= 1e-5 * scale), np.max(np.abs(V - Vo) / scale)
    Q = oracle.q_values(om, R64, Vo)
    policy_tie_check(pi, pio, Q)
    return V, pi, st


@pytest.mark.parametrize("case", ["tiny", "energy_small", "three_objectives"])
def test_solver_parity_on_identical_model(mdp, case):
    env = FP32_CASES[case]()
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=env.objectives)
    for o in range(len(env.objectives)):
        V, pi, st = solver_parity(mdp, env, model, o)
        assert st.sweeps <= env.nt + 1 and st.residual == 0.0


def test_layered_schedule_equals_jacobi_bitwise(mdp):
    for prec in (mdp.MDP_FP32, mdp.MDP_FP64_CHECK):
        env = inputs.energy(nx=20, ny=18, nt=7, N=200)
        model = mdp.mdp_build(mdp.DeviceEnv(env, prec))
        Vj, pij, stj = mdp.mdp_solve(model, 0, method=mdp.MDP_SOLVE_JACOBI, tol=0.0)
        Vl, pil, stl = mdp.mdp_solve(model, 0, method=mdp.MDP_SOLVE_LAYERED)
        assert np.array_equal(Vj.cpu().numpy(), Vl.cpu().numpy())
        assert np.array_equal(pij.cpu().numpy(), pil.cpu().numpy())


ACTIVE_CASES = {
    "three_objectives": lambda: inputs.large(nx=22, ny=22, nt=9, N=300, L=15, square=5),
    "A12_straddling_slices": lambda: inputs.make_env(nx=9, ny=7, nt=8, K=3, N=250, L=9,
                                                     sigma=(0.3, 0.2, 0.1), seed=5, amplitude=0.8,
                                                     n_headings=12, n_speeds=1, obstacle="squares",
                                                     square=3),
    "tiny_rterm": lambda: inputs.tiny(nx=13, ny=11, nt=12, N=77, r_term=4.0),
}


@pytest.mark.parametrize("case", sorted(ACTIVE_CASES))
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_active_layer_jacobi_equals_full_sweeps_bitwise(mdp, case, precision):
    # the active-layer schedule recomputes only layers whose inputs changed;
    # iterates, policy, sweep count and residual must equal full sweeps exactly
    env = ACTIVE_CASES[case]()
    prec = mdp.MDP_FP32 if precision == "fp32" else mdp.MDP_FP64_CHECK
    model = mdp.mdp_build(mdp.DeviceEnv(env, prec), objs=env.objectives)
    n = len(env.objectives)
    for tol, ms in ((0.0, 0), (0.0, 3), (1e-3, 0), (0.5, 0)):
        for o in range(n):
            Va, pa, sa = mdp.mdp_solve(model, o, method=mdp.MDP_SOLVE_JACOBI, tol=tol, max_sweeps=ms)
            Vf, pf, sf = mdp.mdp_solve(model, o, method=mdp.MDP_SOLVE_JACOBI_FULL, tol=tol, max_sweeps=ms)
            assert np.array_equal(Va.cpu().numpy().view(np.uint8), Vf.cpu().numpy().view(np.uint8))
            assert np.array_equal(pa.cpu().numpy(), pf.cpu().numpy())
            assert (sa.sweeps, sa.residual) == (sf.sweeps, sf.residual)
            assert sa.backups <= sf.backups
            if tol == 0.0 and ms == 0:   # later sweeps skip the layers that are final
                assert sa.backups < sf.backups
        if n > 1:
            objs = tuple(range(n))
            Vs, ps, ss = mdp.mdp_solve_multi(model, objs, method=mdp.MDP_SOLVE_JACOBI, tol=tol, max_sweeps=ms)
            Vg, pg, sg = mdp.mdp_solve_multi(model, objs, method=mdp.MDP_SOLVE_JACOBI_FULL, tol=tol,
                                             max_sweeps=ms)
            for o in range(n):
                assert np.array_equal(Vs[o].cpu().numpy().view(np.uint8), Vg[o].cpu().numpy().view(np.uint8))
                assert np.array_equal(ps[o].cpu().numpy(), pg[o].cpu().numpy())
                assert (ss[o].sweeps, ss[o].residual) == (sg[o].sweeps, sg[o].residual)


def test_solver_tolerance_stops_early_and_max_sweeps(mdp):
    env = inputs.tiny(nx=12, ny=12, nt=8, N=100, r_term=5.0)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP64_CHECK))
    ref = oracle.build(env)
    fx = oracle.fixed_mask(env)
    for tol, ms in ((0.0, 0), (1e3, 0), (0.0, 3), (1e-9, 0)):
        V, pi, st = mdp.mdp_solve(model, 0, tol=tol, max_sweeps=ms)
        Vo, pio, sw, res = oracle.vi_jacobi(ref, ref.R[0], fx, tol=tol,
                                            max_sweeps=ms if ms else env.nt + 1)
        assert st.sweeps == sw
        assert st.residual == pytest.approx(res, rel=1e-12, abs=1e-300)
        np.testing.assert_allclose(V.cpu().numpy(), Vo, rtol=1e-12, atol=1e-12)


def test_zero_flow_values_are_chebyshev_distance_on_gpu(mdp):
    nx = ny = 9
    nt = 7
    tgt = np.zeros((ny, nx), np.uint8)
    tgt[6:8, 4:6] = 1
    env = custom_env(nx=nx, ny=ny, nt=nt, N=4, L=5, target=tgt, r_term=3.0, r_outbound=-500.0)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32))
    V, pi, st = mdp.mdp_solve(model, 0, tol=0.0)
    V = V.cpu().numpy()
    tj, ti = np.nonzero(tgt)
    for t in range(nt):
        for j in range(ny):
            for i in range(nx):
                d = min(max(abs(i - a), abs(j - b)) for a, b in zip(ti, tj))
                if 0 < d <= nt - 1 - t:
                    assert V[t * nx * ny + j * nx + i] == pytest.approx(3.0 - d, abs=1e-5)


@pytest.mark.parametrize("scale,width", [(1.2, 12), (1.4, 14), (1.6, 16)])
def test_solvers_on_both_sides_of_the_grouped_sweep_width(mdp, scale, width):
    """32 actions with the widest slice at 12, 14 and 16 columns: the grouped
    sweep (four states per warp step, up to 13 columns) and the warp-per-slice
    sweep above it both return the oracle's values and policy in check mode,
    fused and single-objective, Jacobi and layered; FP32 passes the solver
    gate on its own exported model."""
    env = inputs.energy(nx=18, ny=16, nt=5, N=800, L=15, objectives=(0, 1, 2),
                        sigma=tuple(scale * x for x in (0.3, 0.2, 0.15, 0.1)))
    ref = oracle.build(env, objs=(0, 1, 2))
    fx = oracle.fixed_mask(env)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP64_CHECK), objs=(0, 1, 2))
    assert model.info().max_row_nnz == width
    for meth in (mdp.MDP_SOLVE_JACOBI, mdp.MDP_SOLVE_LAYERED):
        Vs, pis, sts = mdp.mdp_solve_multi(model, (0, 1, 2), method=meth, tol=0.0)
        for o in range(3):
            Vo, pio, sw, res = oracle.vi_jacobi(ref, ref.R[o], fx, tol=0.0, nt=env.nt)
            np.testing.assert_allclose(Vs[o].cpu().numpy(), Vo, rtol=1e-12, atol=1e-12)
            assert np.array_equal(pis[o].cpu().numpy(), pio)
            V1, pi1, st1 = mdp.mdp_solve(model, o, method=meth, tol=0.0)
            assert np.array_equal(V1.cpu().numpy().view(np.uint64), Vs[o].cpu().numpy().view(np.uint64))
            assert np.array_equal(pi1.cpu().numpy(), pis[o].cpu().numpy())
    m32 = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=(0, 1, 2))
    for o in range(3):
        solver_parity(mdp, env, m32, o)


def test_a_wait_that_runs_out_reports_timeout_and_the_context_stays_usable(mdp):
    """Failure detection without a GPU fault: every wait of the Bellman sweep is
    bounded.  A test hook makes the first round of the next solve expect bytes
    that are never copied (a completion that nothing delivers) and sets a short
    limit; the wait gives up, the kernel drains and returns, the call reports
    MDP_ERR_TIMEOUT, and the next solve on the same context gives the same
    values and policy as before."""
    env = inputs.energy(nx=20, ny=18, nt=5, N=200)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=env.objectives)
    V0, pi0, _ = mdp.mdp_solve(model, 0, tol=0.0)
    V0, pi0 = V0.cpu().numpy(), pi0.cpu().numpy()
    lib = mdp.load()
    assert lib.mdp_test_inject(7, 0) == -1 and lib.mdp_test_inject(1, 8) == -1
    assert lib.mdp_test_inject(2, 2_000_000) == 0    # about 1 ms at the GPU's clock
    assert lib.mdp_test_inject(1, 1024) == 0
    try:
        with pytest.raises(mdp.MdpError) as ei:
            mdp.mdp_solve(model, 0, tol=0.0)
        assert ei.value.code == -5 and "bounded" in str(ei.value)
    finally:
        lib.mdp_test_inject(2, 0)
    V1, pi1, st1 = mdp.mdp_solve(model, 0, tol=0.0)
    assert np.array_equal(V1.cpu().numpy(), V0) and np.array_equal(pi1.cpu().numpy(), pi0)
