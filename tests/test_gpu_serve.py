"""Serving: requests admitted under an HBM budget run concurrently on per-slot
streams; a request's result is the same alone and in a mix of concurrent
requests, and the same as a direct build + solve of the same parameters."""
import time

import numpy as np
import pytest

from conftest import device_pool_meter, oracle_end_to_end
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


def _env(seed=22):
    return inputs.energy(nx=40, ny=36, nt=12, N=300, seed=seed, L=15)


def _direct(mdp, env, target, sigma_scale, seed, N, obj):
    """The same request through mdp_build + mdp_solve."""
    e = inputs.Environment(**{**env.__dict__})
    e.target = inputs.target_block(env.nx, env.ny, target[0], target[1])
    e.sigma = env.sigma * sigma_scale
    e.seed, e.N, e.mdp_id = seed, N, 0
    m = mdp.mdp_build(mdp.DeviceEnv(e, mdp.MDP_FP32), objs=(obj,))
    V, pi, st = mdp.mdp_solve(m, 0, tol=0.0)
    return V.cpu().numpy(), pi.cpu().numpy()


def test_result_alone_equals_result_in_a_mix(mdp):
    env = _env()
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    probe = dict(start=(20, 7), target=(21, 28), sigma_scale=1.3, seed=77, N=300, objective=2)
    # alone: one slot, nothing else in flight
    s1 = mdp.Server(8 << 30, 1)
    eid = s1.register(d)
    t = s1.submit(eid, **probe)
    res, V_alone, pi_alone = s1.poll(t, timeout_ms=60000, env_id=eid, want_V=True)
    assert res.status == 0, mdp.load().mdp_last_error().decode()
    s1.close()
    # in a mix: 4 slots, 9 other requests submitted around it
    s4 = mdp.Server(8 << 30, 4)
    eid = s4.register(d)
    rng = np.random.default_rng(5)
    tickets = []
    for k in range(10):
        if k == 4:
            tickets.append(("probe", s4.submit(eid, **probe)))
        else:
            tickets.append(("other", s4.submit(
                eid, start=(int(rng.integers(0, 40)), int(rng.integers(0, 36))),
                target=(int(rng.integers(0, 38)), int(rng.integers(0, 34))),
                sigma_scale=float(rng.uniform(0.5, 1.5)), seed=int(rng.integers(1, 1000)),
                N=int(rng.integers(100, 400)), objective=int(rng.integers(0, 3)))))
    seen_overlap = 0
    for _ in range(200):
        inflight, queued, used = s4.stats()
        seen_overlap = max(seen_overlap, inflight)
        if queued == 0 and inflight == 0:
            break
        time.sleep(0.005)
    for kind, t in tickets:
        res, V, pi = s4.poll(t, timeout_ms=60000, env_id=eid, want_V=True)
        assert res.status == 0, mdp.load().mdp_last_error().decode()
        assert res.latency_ms >= res.queue_ms >= 0
        if kind == "probe":
            assert np.array_equal(V, V_alone) and np.array_equal(pi, pi_alone)
    s4.close()
    assert seen_overlap >= 2, "requests never overlapped"
    Vd, pid = _direct(mdp, env, probe["target"], probe["sigma_scale"], probe["seed"], probe["N"],
                      probe["objective"])
    assert np.array_equal(Vd, V_alone) and np.array_equal(pid, pi_alone)


def test_budget_admission_and_errors(mdp):
    env = _env()
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    probe = mdp.Server(8 << 30, 1)
    eid = probe.register(d)
    res, _, _ = probe.poll(probe.submit(eid, start=(1, 1), target=(20, 20), seed=99, N=300), timeout_ms=60000)
    probe.close()
    charge = res.device_bytes           # what one such request is charged
    budget = int(1.5 * charge)          # room for one such request at its admission charge
    s = mdp.Server(budget, 2)
    eid = s.register(d)
    with pytest.raises(mdp.MdpError) as ei:
        s.submit(eid + 5, start=(1, 1), target=(3, 3))
    assert ei.value.code == -9
    with pytest.raises(mdp.MdpError) as ei:
        s.submit(eid, start=(1, 1), target=(3, 3), N=0)
    assert ei.value.code == -1
    tk = [s.submit(eid, start=(1, 1), target=(20, 20), seed=i, N=300) for i in range(3)]
    peak = 0
    for _ in range(400):
        inflight, queued, used = s.stats()
        assert used <= budget
        peak = max(peak, inflight)
        if inflight == 0 and queued == 0:
            break
        time.sleep(0.002)
    for t in tk:
        res, _, _ = s.poll(t, timeout_ms=60000)
        assert res.status == 0, mdp.load().mdp_last_error().decode()
    s.close()
    big = mdp.Server(1 << 20, 1)    # 1 MiB: every request is larger than the whole budget
    eid = big.register(d)
    with pytest.raises(mdp.MdpError) as ei:
        big.submit(eid, start=(1, 1), target=(3, 3))
    assert ei.value.code == -7
    big.close()


def test_poll_pending_and_unknown_ticket(mdp):
    env = _env()
    s = mdp.Server(8 << 30, 1)
    eid = s.register(mdp.DeviceEnv(env, mdp.MDP_FP32))
    t = s.submit(eid, start=(2, 2), target=(30, 30), N=2000)
    r = s.poll(t, timeout_ms=0)
    assert r is None or r[0].status == 0
    res, _, _ = s.poll(t, timeout_ms=60000) if r is None else r
    assert res.status == 0
    with pytest.raises(mdp.MdpError) as ei:
        s.poll(t, timeout_ms=0)      # released after the first successful poll
    assert ei.value.code == -9
    s.close()


def test_replanning_from_a_later_time_step(mdp):
    """A request with start_t = t0 replans the remaining horizon on the
    resident fields: it equals a direct build + solve of the environment cut
    to layers t0..nt-1 with the same target, variance scale, seed and N."""
    env = _env()
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    srv = mdp.Server(8 << 30, 2)
    eid = srv.register(d)
    t0 = 5
    probe = dict(start=(9, 22), target=(30, 8), sigma_scale=0.8, seed=404, N=250, objective=1)
    t = srv.submit(eid, start_t=t0, **probe)
    res, V, pi = srv.poll(t, timeout_ms=60000, env_id=eid, want_V=True)
    assert res.status == 0, mdp.load().mdp_last_error().decode()
    srv.close()
    cut = inputs.Environment(**{**env.__dict__})
    cut.nt = env.nt - t0
    cut.vbar, cut.modes, cut.obstacle = env.vbar[t0:], env.modes[t0:], env.obstacle[t0:]
    cut.gbar = env.gbar[t0:] if env.gbar is not None else None
    Vd, pid = _direct(mdp, cut, probe["target"], probe["sigma_scale"], probe["seed"], probe["N"],
                      probe["objective"])
    assert V.shape == Vd.shape == (cut.nS + 1,)
    assert np.array_equal(V, Vd) and np.array_equal(pi, pid)
    s0 = probe["start"][1] * env.nx + probe["start"][0]
    assert res.V_start == V[s0] and res.pi_start == pi[s0]


def test_jacobi_request_warm_started_from_an_earlier_result(mdp):
    """Replanning warm (Sec. V): a Jacobi request started from the exact
    values of an earlier request with the same parameters stops after one
    sweep with those values bit for bit; started cold it needs more sweeps."""
    env = inputs.energy(nx=24, ny=20, nt=8, N=300, L=15)
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    srv = mdp.Server(8 << 30, 2)
    eid = srv.register(d)
    kw = dict(start=(3, 3), target=(15, 14), sigma_scale=0.9, seed=77, N=300)
    t0 = srv.submit(eid, **kw)                     # exact: the layered pass
    r0, V0, pi0 = srv.poll(t0, timeout_ms=120000, env_id=eid, want_V=True)
    assert r0.status == 0
    tw = srv.submit(eid, tol=1e-3, V0=V0, **kw)    # Jacobi from the exact values
    rw, Vw, piw = srv.poll(tw, timeout_ms=120000, env_id=eid, want_V=True)
    tc = srv.submit(eid, tol=1e-3, **kw)           # Jacobi from 0
    rc, Vc, pic = srv.poll(tc, timeout_ms=120000, env_id=eid, want_V=True)
    assert rw.status == 0 and rc.status == 0
    assert rw.sweeps == 1 and rc.sweeps > 1
    assert np.array_equal(Vw.view(np.uint32), V0.view(np.uint32))
    assert np.array_equal(piw, pi0)
    with pytest.raises(ValueError):
        srv.submit(eid, tol=1e-3, V0=V0[:-1], **kw)
    srv.close()


def _cut_request_env(env, t0, target, sigma_scale, seed, N):
    """The environment a request describes: layers t0..nt-1 of the resident
    fields, a 2x2 target block, sigma scaled, its own seed and N (mdp_id 0)."""
    e = inputs.Environment(**{**env.__dict__})
    e.nt = env.nt - t0
    e.vbar, e.modes, e.obstacle = env.vbar[t0:], env.modes[t0:], env.obstacle[t0:]
    e.gbar = env.gbar[t0:] if env.gbar is not None else None
    e.target = inputs.target_block(env.nx, env.ny, target[0], target[1])
    e.sigma = env.sigma * sigma_scale
    e.seed, e.N, e.mdp_id, e.Y = seed, N, 0, None
    return e


@pytest.mark.parametrize("t0,objective", [(0, 0), (2, 2)])
def test_served_request_matches_the_oracle(mdp, t0, objective):
    """A served request (t0 = 0) and a replanning request from a later step
    (t0 = 2: the remaining horizon on the resident fields with a fresh draw,
    Sec. V) against the oracle's build and value iteration of the horizon the
    request describes, end to end: |dV| <= 1e-5 max(1, |V|) plus the exact
    effect of the FP32 build's count differences, policy equal up to ties
    within the same bound."""
    env = inputs.energy(nx=16, ny=14, nt=7, N=60, L=15, seed=23)
    srv = mdp.Server(8 << 30, 2)
    eid = srv.register(mdp.DeviceEnv(env, mdp.MDP_FP32))
    probe = dict(start=(8, 3), target=(8, 10), sigma_scale=1.2, seed=41, N=60, objective=objective)
    t = srv.submit(eid, start_t=t0, **probe)
    res, V, pi = srv.poll(t, timeout_ms=60000, env_id=eid, want_V=True)
    assert res.status == 0, mdp.load().mdp_last_error().decode()
    srv.close()
    e = _cut_request_env(env, t0, probe["target"], probe["sigma_scale"], probe["seed"], probe["N"])
    assert V.shape == (e.nS + 1,)
    oracle_end_to_end(mdp, e, objective, V, pi)


def _wide_env():
    """Rows of 50+ successors (strong uniform modes): more entry-pool columns
    per slice than a first charge assumes."""
    nt = 3
    modes = np.stack([np.stack([np.ones((nt, 9, 9)), np.zeros((nt, 9, 9))], -1),
                      np.stack([np.zeros((nt, 9, 9)), np.ones((nt, 9, 9))], -1)], 1)
    from conftest import custom_env
    return custom_env(nx=9, ny=9, nt=nt, K=2, N=3000, L=15, seed=12, sigma=[1.1, 1.0], modes=modes)


def _charges(mdp, env, kw):
    """(charge of the largest possible pool, charge of the exact pool) of a
    request: the first from a server with room for it, the second from a
    server just too small for the first, where the request starts from the
    environment's narrower guess and is charged again for its exact need."""
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    big = mdp.Server(8 << 30, 1)
    eid = big.register(d)
    res, _, _ = big.poll(big.submit(eid, **kw), timeout_ms=60000)
    assert res.status == 0
    big.close()
    worst = res.device_bytes
    tight = mdp.Server(worst - 1, 1)
    eid = tight.register(d)
    res, _, _ = tight.poll(tight.submit(eid, **kw), timeout_ms=60000)
    assert res.status == 0, mdp.load().mdp_last_error().decode()
    tight.close()
    return worst, res.device_bytes


def test_a_request_never_holds_more_device_memory_than_it_was_charged(mdp):
    """The budget is a hard bound: measured by the device memory pool's
    high-water mark around each request (one slot, nothing else running), a
    request's peak stays within the largest charge it held -- with room for
    the largest pool its slices can need, and with a budget just below that,
    where it is first charged from narrower widths, for the wide environment
    stopped at that pool, charged again for the exact need and rerun -- and the
    result equals a direct build + solve."""
    import torch
    reset, read = device_pool_meter()
    for env, kw in ((_env(), dict(start=(3, 4), target=(20, 20), seed=5, N=300, objective=1)),
                    (_wide_env(), dict(start=(4, 4), target=(1, 1), seed=7, N=3000, objective=0))):
        worst, exact = _charges(mdp, env, kw)
        assert exact <= worst
        for budget in (8 << 30, worst - 1):
            srv = mdp.Server(budget, 1)
            eid = srv.register(mdp.DeviceEnv(env, mdp.MDP_FP32))
            for rep in range(2):   # the second request is priced from the first one's widths
                torch.cuda.synchronize()
                used0, _ = read()
                reset()
                res, V, pi = srv.poll(srv.submit(eid, **kw), timeout_ms=60000, env_id=eid, want_V=True)
                assert res.status == 0, mdp.load().mdp_last_error().decode()
                _, high = read()
                assert high - used0 <= res.device_bytes <= budget, (budget, rep, high - used0, res.device_bytes)
            srv.close()
        Vd, pid = _direct(mdp, env, kw["target"], 1.0, kw["seed"], kw["N"], kw.get("objective", 0))
        assert np.array_equal(V, Vd) and np.array_equal(pi, pid)


def test_a_request_that_outgrows_the_budget_is_refused(mdp):
    """Admitted under a charge from narrower widths, a request whose slices
    need a pool beyond the whole budget ends with MDP_ERR_BUDGET instead of
    allocating it, and leaves nothing held."""
    env = _wide_env()
    kw = dict(start=(4, 4), target=(1, 1), seed=7, N=3000)
    worst, exact = _charges(mdp, env, kw)
    small = mdp.Server(exact - 1, 1)       # admits the narrow first charge, not the exact one
    eid = small.register(mdp.DeviceEnv(env, mdp.MDP_FP32))
    res, _, _ = small.poll(small.submit(eid, **kw), timeout_ms=60000)
    assert res.status == -7
    inflight, queued, used = small.stats()
    assert inflight == 0 and queued == 0 and used == 0
    small.close()
