"""Batching: uneven MDPs built and solved in one persistent build launch and
batched Jacobi sweeps (CUDA graph, replayed) give, for every member, exactly
the model and values of building and solving it alone."""
import numpy as np
import pytest

from conftest import oracle_end_to_end
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


def members():
    envs = []
    for i in range(7):
        # keep the test small: shrink the member, keep its character
        side = 16 + 7 * i
        envs.append(inputs.batch_member(i, nx=side, ny=side - 2 * (i % 3), nt=5 + i, N=120 + 37 * i))
    envs.append(inputs.tiny(r_term=3.0))
    envs.append(inputs.energy(nx=22, ny=19, nt=6, N=200))
    return envs


def test_batch_equals_members_alone_and_replays(mdp):
    # tol = 0: the batch runs the layered pass; values and policies equal
    # each member's solo Jacobi solve and its solo layered pass bit for bit
    envs = members()
    assert len({e.A for e in envs}) > 1 and len({e.K for e in envs}) > 1
    assert len({e.nt for e in envs}) > 1
    denvs = [mdp.DeviceEnv(e, mdp.MDP_FP32) for e in envs]
    b = mdp.Batch(denvs, tol=0.0)
    for rep in range(2):   # the second run replays the captured graph
        sweeps, ms = b.run()
        assert ms > 0
        for i, (e, d) in enumerate(zip(envs, denvs)):
            m = mdp.mdp_build(d, objs=(e.objectives[0],))
            for method in (mdp.MDP_SOLVE_JACOBI, mdp.MDP_SOLVE_LAYERED):
                V, pi, st = mdp.mdp_solve(m, 0, method=method, tol=0.0)
                assert np.array_equal(b.V[i].cpu().numpy(), V.cpu().numpy()), (i, method)
                assert np.array_equal(b.policy[i].cpu().numpy(), pi.cpu().numpy()), (i, method)
            assert sweeps[i] == st.sweeps == 1, (i, sweeps[i], st.sweeps)
    b.close()


def test_batch_with_tolerance_stops_each_member_on_its_own(mdp):
    # members converge at different sweeps; the per-sweep plan must drop each
    # one as soon as its own residual meets tol and still match the solo solve
    envs = members()[:6]
    denvs = [mdp.DeviceEnv(e, mdp.MDP_FP32) for e in envs]
    for tol in (1e-3, 0.5):
        b = mdp.Batch(denvs, tol=tol)
        sweeps, ms = b.run()
        solo = []
        for i, (e, d) in enumerate(zip(envs, denvs)):
            m = mdp.mdp_build(d, objs=(e.objectives[0],))
            V, pi, st = mdp.mdp_solve(m, 0, tol=tol)
            solo.append(st.sweeps)
            assert sweeps[i] == st.sweeps, (tol, i, sweeps[i], st.sweeps)
            assert np.array_equal(b.V[i].cpu().numpy(), V.cpu().numpy()), (tol, i)
            assert np.array_equal(b.policy[i].cpu().numpy(), pi.cpu().numpy()), (tol, i)
        b.close()


def test_batch_rejects_fp64_items(mdp):
    e = inputs.tiny()
    with pytest.raises(mdp.MdpError):
        mdp.Batch([mdp.DeviceEnv(e, mdp.MDP_FP64_CHECK)])


def test_batch_members_match_the_oracle(mdp):
    """Members of a batch (16 and 32 actions, different mode counts, grids and
    horizons) against the oracle's build and value iteration of each member,
    end to end: |dV| <= 1e-5 max(1, |V|) plus the exact effect of the FP32
    build's count differences, policy equal up to ties within the same bound."""
    envs = [inputs.batch_member(i, nx=12 + 3 * i, ny=11 + 2 * i, nt=4 + i, N=50 + 10 * i)
            for i in range(3)]
    assert len({e.A for e in envs}) > 1
    b = mdp.Batch([mdp.DeviceEnv(e, mdp.MDP_FP32) for e in envs], tol=0.0)
    b.run()
    for i, e in enumerate(envs):
        oracle_end_to_end(mdp, e, e.objectives[0], b.V[i].cpu().numpy(), b.policy[i].cpu().numpy())
    b.close()
