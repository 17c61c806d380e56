"""Fused multi-objective value iteration (mdp_solve_multi) through the C ABI.

Gate: objective o of a fused solve equals mdp_solve on objective o alone bit
for bit (V, policy, sweeps, residual) for both schedules, both precisions and
every tolerance; in FP64 check mode it also equals the oracle's value
iteration (Sec. II-B) on the oracle's own model to 1e-12.
"""
import numpy as np
import pytest

import oracle
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


def three_obj_env(**kw):
    args = dict(nx=22, ny=21, nt=6, N=300, L=15, square=5)
    args.update(kw)
    return inputs.large(**args)


def assert_same(mdp, model, objs, method, tol=0.0, max_sweeps=0):
    Vs, pis, sts = mdp.mdp_solve_multi(model, objs, method=method, tol=tol, max_sweeps=max_sweeps)
    for o, slot in enumerate(objs):
        V1, pi1, st1 = mdp.mdp_solve(model, slot, method=method, tol=tol, max_sweeps=max_sweeps)
        a, b = Vs[o].cpu().numpy(), V1.cpu().numpy()
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), (slot, np.max(np.abs(a - b)))
        assert np.array_equal(pis[o].cpu().numpy(), pi1.cpu().numpy())
        assert sts[o].sweeps == st1.sweeps
        assert sts[o].residual == st1.residual
        assert sts[o].backups == st1.backups
    return Vs, pis, sts


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("method", ["jacobi", "layered"])
def test_fused_equals_separate_solves_bitwise(mdp, precision, method):
    prec = mdp.MDP_FP32 if precision == "fp32" else mdp.MDP_FP64_CHECK
    meth = mdp.MDP_SOLVE_JACOBI if method == "jacobi" else mdp.MDP_SOLVE_LAYERED
    env = three_obj_env(N=300 if precision == "fp32" else 60)
    model = mdp.mdp_build(mdp.DeviceEnv(env, prec), objs=env.objectives)
    for objs in ((0, 1, 2), (2, 0), (1,), (1, 1, 0)):
        assert_same(mdp, model, objs, meth)


def test_objectives_stop_on_their_own_tolerance(mdp):
    # each objective's residual history from its own solves; a tolerance
    # between two objectives' histories ends them at different sweeps, and
    # each must still return exactly its own solve's result
    env = three_obj_env(nt=9, N=200)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP64_CHECK), objs=env.objectives)
    hist = []
    for slot in range(3):
        hist.append([mdp.mdp_solve(model, slot, tol=0.0, max_sweeps=k)[2].residual
                     for k in range(1, env.nt + 2)])

    def stop(h, tol):
        return next((k + 1 for k, r in enumerate(h) if r <= tol), len(h))

    cands = sorted({r for h in hist for r in h if r > 0})
    split = [t for t in cands if len({stop(h, t) for h in hist}) > 1]
    assert split, hist
    for tol in split[:3] + [split[-1], 1e-9, 100.0]:
        _, _, sts = assert_same(mdp, model, (0, 1, 2), mdp.MDP_SOLVE_JACOBI, tol=tol)
        assert [s.sweeps for s in sts] == [stop(h, tol) for h in hist]
    for ms in (1, 2, 4):
        assert_same(mdp, model, (0, 1, 2), mdp.MDP_SOLVE_JACOBI, tol=0.0, max_sweeps=ms)


def test_fused_check_mode_matches_oracle_vi(mdp):
    env = three_obj_env(nx=16, ny=15, nt=5, N=40)
    ref = oracle.build(env, objs=env.objectives)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP64_CHECK), objs=env.objectives)
    Vs, pis, sts = mdp.mdp_solve_multi(model, (0, 1, 2), tol=0.0)
    fx = oracle.fixed_mask(env)
    for o in range(3):
        Vo, pio, sw, res = oracle.vi_jacobi(ref, ref.R[o], fx, tol=0.0, nt=env.nt)
        assert sts[o].sweeps == sw
        np.testing.assert_allclose(Vs[o].cpu().numpy(), Vo, rtol=1e-12, atol=1e-12)
        assert np.array_equal(pis[o].cpu().numpy(), pio)


def test_fused_solve_argument_errors(mdp):
    env = three_obj_env(nx=8, ny=8, nt=3, N=20, square=2)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=env.objectives)
    for objs in ((), (0, 1, 2, 0), (3,), (0, -1)):
        with pytest.raises(mdp.MdpError) as ei:
            mdp.mdp_solve_multi(model, objs)
        assert ei.value.code == -1
    with pytest.raises(mdp.MdpError) as ei:
        mdp.mdp_solve_multi(model, (0,), method=5)
    assert ei.value.code == -1
