"""Warm-started Jacobi (MDP_SOLVE_WARM: replanning from the previous plan's
values, Sec. V) through the C ABI.  On this time-layered MDP Jacobi reaches the
exact fixed point from any V_0 within nt + 1 sweeps, so with tol = 0 a warm
start returns the cold start's values and policy bit for bit; started at the
fixed point it stops after one sweep with residual 0; near it, a tolerance
stops it in fewer sweeps than the cold start."""
import numpy as np
import pytest

import oracle
from conftest import policy_tie_check
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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("method", ["jacobi", "jacobi_full"])
def test_warm_start_reaches_the_same_fixed_point(mdp, precision, method):
    import torch
    env = inputs.energy(nx=22, ny=18, nt=8, N=200 if precision == "fp32" else 60, L=15)
    prec = mdp.MDP_FP32 if precision == "fp32" else mdp.MDP_FP64_CHECK
    meth = mdp.MDP_SOLVE_JACOBI if method == "jacobi" else mdp.MDP_SOLVE_JACOBI_FULL
    model = mdp.mdp_build(mdp.DeviceEnv(env, prec), objs=env.objectives)
    Vc, pic, stc = mdp.mdp_solve(model, 0, method=meth, tol=0.0)
    # from the fixed point itself: one sweep, nothing changes
    V1 = Vc.clone()
    V1, pi1, st1 = mdp.mdp_solve(model, 0, method=meth, tol=0.0, V=V1, warm=True)
    assert st1.sweeps == 1 and st1.residual == 0.0
    assert torch.equal(V1, Vc) and torch.equal(pi1, pic)
    # from arbitrary values (the sink entry is reset): the same fixed point
    g = torch.Generator(device="cpu").manual_seed(3)
    V2 = (torch.randn(Vc.numel(), generator=g, dtype=torch.float64) * 50.0).to(Vc.device, Vc.dtype)
    V2, pi2, st2 = mdp.mdp_solve(model, 0, method=meth, tol=0.0, V=V2, warm=True)
    assert st2.sweeps <= env.nt + 1
    assert torch.equal(V2, Vc) and torch.equal(pi2, pic)
    assert V2[-1].item() == 0.0


def test_warm_start_near_the_fixed_point_needs_fewer_sweeps(mdp):
    import torch
    env = inputs.energy(nx=22, ny=18, nt=10, N=200, L=15)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=env.objectives)
    Vx, pix, stx = mdp.mdp_solve(model, 0, tol=0.0)
    tol = 1e-3
    Vc, pic, stc = mdp.mdp_solve(model, 0, tol=tol)
    V0 = Vx.clone()
    V0[:-1] += 1e-4 * torch.sign(torch.arange(V0.numel() - 1, device=V0.device, dtype=V0.dtype) % 3 - 1)
    Vw, piw, stw = mdp.mdp_solve(model, 0, tol=tol, V=V0, warm=True)
    assert stw.sweeps < stc.sweeps, (stw.sweeps, stc.sweeps)
    assert stw.residual <= tol
    assert float((Vw - Vx).abs().max()) <= 1e-3 * env.nt


def test_warm_start_argument_errors(mdp):
    env = inputs.tiny(nx=8, ny=8, nt=3, N=20)
    model = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32))
    V, pi, st = mdp.mdp_solve(model, 0, tol=0.0)
    with pytest.raises(ValueError):
        mdp.mdp_solve(model, 0, tol=0.0, warm=True)
    with pytest.raises(mdp.MdpError) as ei:   # the layered pass has no starting values
        mdp.mdp_solve(model, 0, method=mdp.MDP_SOLVE_LAYERED, V=V, warm=True)
    assert ei.value.code == -1
    with pytest.raises(mdp.MdpError) as ei:   # fused solves start cold
        mdp.mdp_solve_multi(model, (0, 0), method=mdp.MDP_SOLVE_JACOBI | mdp.MDP_SOLVE_WARM)
    assert ei.value.code == -1


def test_warm_start_iterates_equal_the_oracle_from_the_same_values(mdp):
    """Sweeps from a given v_0 (Sec. II-B update; replanning from a previous
    plan, Sec. V) against the oracle's value iteration from the same v_0.
    Check mode: after k = 1, 2, 3 sweeps and with a tolerance stop, V, policy,
    sweep count and residual equal the oracle's (V to 1e-12) on the oracle's
    own build.  FP32: on the GPU's exported P/R, |dV| <= 1e-5 max(1, |V|) and
    the policy equals the oracle's up to ties."""
    import torch
    env = inputs.energy(nx=14, ny=12, nt=6, N=60, L=15, objectives=(0, 1, 2))
    ref = oracle.build(env, objs=(0, 1, 2))
    fx = oracle.fixed_mask(env)
    m64 = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP64_CHECK), objs=(0, 1, 2))
    m32 = mdp.mdp_build(mdp.DeviceEnv(env, mdp.MDP_FP32), objs=(0, 1, 2))
    rng = np.random.default_rng(31)
    for o in range(3):
        V0 = rng.normal(0.0, 40.0, env.nS)
        for k, tol in ((1, 0.0), (2, 0.0), (3, 0.0), (0, 5.0)):
            V = torch.tensor(np.concatenate([V0, [99.0]]), dtype=torch.float64, device="cuda")
            V, pi, st = mdp.mdp_solve(m64, o, tol=tol, max_sweeps=k, V=V, warm=True)
            Vo, pio, sw, res = oracle.vi_jacobi(ref, ref.R[o], fx, tol=tol, max_sweeps=k or env.nt + 1,
                                                V0=V0)
            assert st.sweeps == sw and st.residual == pytest.approx(res, rel=1e-12, abs=1e-300)
            np.testing.assert_allclose(V.cpu().numpy(), Vo, rtol=1e-12, atol=1e-12)
            assert np.array_equal(pi.cpu().numpy(), pio)
        rp, col, cnt, R = (x.cpu().numpy() for x in mdp.mdp_export_csr(m32, o))
        om = oracle.model_from_csr(env.nS, env.A, env.N, rp, col, cnt)
        R64 = R.astype(np.float64)
        V0f = V0.astype(np.float32)
        for k in (1, 3):
            V = torch.tensor(np.concatenate([V0f, [0.0]]), dtype=torch.float32, device="cuda")
            V, pi, st = mdp.mdp_solve(m32, o, tol=0.0, max_sweeps=k, V=V, warm=True)
            Vo, pio, sw, res = oracle.vi_jacobi(om, R64, fx, tol=0.0, max_sweeps=k,
                                                V0=V0f.astype(np.float64))
            assert st.sweeps == sw
            Vg = V.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(Vg - Vo) <= 1e-5 * np.maximum(1.0, np.abs(Vo)))
            # the policy of sweep k is the argmax of the Q of the values before it
            Vprev, _, _, _ = oracle.vi_jacobi(om, R64, fx, tol=0.0, max_sweeps=k - 1,
                                              V0=V0f.astype(np.float64)) if k > 1 else \
                (np.concatenate([V0f.astype(np.float64), [0.0]]), None, 0, 0)
            policy_tie_check(pi.cpu().numpy(), pio, oracle.q_values(om, R64, Vprev))
