"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a library implementation of the same published definition, a closed
form the paper's definitions fix, an invariant, or brute force on tiny inputs.
No GPU is used here."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2109_00857_gb300 import inputs
from conftest import custom_env

M64 = (1 << 64) - 1


# ------------------------------------------------------------- sampler ----
def test_philox_matches_numpy_library():
    """Philox4x64-10 (Salmon et al. SC'11) against numpy.random.Philox, an
    independent implementation of the same published generator.  numpy bumps its
    256-bit counter before each block, so its first block uses counter + 1."""
    rng = np.random.default_rng(123)
    cases = [([0, 0, 0, 0], [0, 0]), ([M64] * 4, [M64, M64])]
    for _ in range(300):
        cases.append((list(rng.integers(0, M64, 4, dtype=np.uint64, endpoint=True)),
                       list(rng.integers(0, M64, 2, dtype=np.uint64, endpoint=True))))
    for t in range(3):      # the counters the sampler uses: (t, w, j, attempt)
        cases.append(([t, 17, 1, 0], [33, 0]))
    for ctr, key in cases:
        c = [int(x) for x in ctr]
        val = (c[0] | (c[1] << 64) | (c[2] << 128) | (c[3] << 192)) - 1
        val %= 1 << 256
        k = [int(x) for x in key]
        bg = np.random.Philox(counter=val, key=k[0] | (k[1] << 64))
        want = bg.random_raw(4)
        got = oracle.philox4x64_10(c, [int(k) for k in key])
        assert np.array_equal(got, want), (ctr, key)


def _ulp(x):
    return math.ulp(x)


def test_self_written_log_within_2ulp_of_libm():
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(0, 1, 100000), 10.0 ** rng.uniform(-300, 0, 20000),
                         np.array([1.0, 0.5, 0.25, 2.0 ** -1022, 0.7071067811865476,
                                   0.7071067811865475, 1 - 2 ** -53, 2 ** -53, 1e-300, 3.0])])
    xs = xs[xs > 0]
    worst = 0.0
    for x in xs:
        ref = math.log(float(x))
        got = oracle.ln(float(x))
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, abs(got - ref) / _ulp(ref))
    assert worst <= 2.0, worst


def test_polar_normals_moments_and_ks():
    """1e6 standard normals: mean, variance, skew and kurtosis within 5 standard
    errors, Kolmogorov-Smirnov p > 1e-3, and the attempt count ~ 4/pi."""
    Y = oracle.sample_coeffs(1, 500000, 2, [1.0, 1.0], seed=2024, mdp_id=0).reshape(-1)
    n = Y.size
    assert abs(Y.mean()) < 5 / math.sqrt(n)
    assert abs(Y.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(stats.skew(Y)) < 5 * math.sqrt(6 / n)
    assert abs(stats.kurtosis(Y)) < 5 * math.sqrt(24 / n)
    assert stats.kstest(Y, "norm").pvalue > 1e-3
    att = [oracle.polar_pair(7, 0, 0, w, 0)[2] for w in range(20000)]
    assert abs(np.mean(att) - 4 / math.pi) < 0.03


def test_coefficients_scale_with_sigma_and_are_keyed():
    a = oracle.sample_coeffs(3, 50, 3, [1.0, 2.0, 0.5], seed=9)
    b = oracle.sample_coeffs(3, 50, 3, [1.0, 1.0, 1.0], seed=9)
    assert np.array_equal(a[..., 0], b[..., 0])
    assert np.array_equal(a[..., 1], 2.0 * b[..., 1])
    assert np.array_equal(a[..., 2], 0.5 * b[..., 2])
    c = oracle.sample_coeffs(3, 50, 3, [1.0, 1.0, 1.0], seed=10)
    assert not np.array_equal(b, c)
    d = oracle.sample_coeffs(3, 50, 3, [1.0, 1.0, 1.0], seed=9, mdp_id=1)
    assert not np.array_equal(b, d)
    # the draw for (t, w) does not depend on how many realizations are drawn
    e = oracle.sample_coeffs(3, 80, 3, [1.0, 1.0, 1.0], seed=9)
    assert np.array_equal(b, e[:, :50])


# ---------------------------------------------------------- build pins ----
def _rows(m, a, s):
    r = a * m.nS + s
    return m.col[m.rowptr[r]:m.rowptr[r + 1]], m.cnt[m.rowptr[r]:m.rowptr[r + 1]]


def test_zero_flow_rows_are_one_hot_on_the_neighbour():
    """No flow and no uncertainty: every (s, a) lands in cell(x_s + a dt) with
    probability 1; with F = 1 and 16 headings that is always one of the 8
    neighbours, never the same cell (Sec. II-A kinematics, half-open cells)."""
    e = custom_env(nx=7, ny=7, nt=4, N=10, L=5)
    m = oracle.build(e)
    nS, Nc = e.nS, e.Nc
    for t in range(e.nt - 1):
        for j in range(e.ny):
            for i in range(e.nx):
                s = t * Nc + j * e.nx + i
                for a in range(e.A):
                    dxa, dya, _ = e.actions[a]
                    ip = math.floor(i + 0.5 + dxa)
                    jp = math.floor(j + 0.5 + dya)
                    assert (ip, jp) != (i, j)
                    assert max(abs(ip - i), abs(jp - j)) == 1
                    col, cnt = _rows(m, a, s)
                    assert len(col) == 1 and cnt[0] == e.N
                    if 0 <= ip < e.nx and 0 <= jp < e.ny:
                        assert col[0] == (t + 1) * Nc + jp * e.nx + ip
                    else:
                        assert col[0] == nS


def test_zero_flow_value_is_chebyshev_distance():
    """Time objective, zero flow, F = 1: V(s) = r_term - dt * d_inf(s, target)
    for every state that can reach the target within the horizon."""
    nx = ny = 9
    nt = 7
    tgt = np.zeros((ny, nx), np.uint8)
    tgt[6:8, 4:6] = 1
    e = custom_env(nx=nx, ny=ny, nt=nt, N=4, L=5, target=tgt, r_term=3.0, r_outbound=-500.0)
    m = oracle.build(e)
    V, pi, sw, res = oracle.vi_jacobi(m, m.R[0], oracle.fixed_mask(e), tol=0.0, nt=nt)
    assert res == 0.0 and sw <= nt + 1
    tj, ti = np.nonzero(tgt)
    checked = 0
    for t in range(nt):
        for j in range(ny):
            for i in range(nx):
                s = t * e.Nc + j * nx + i
                d = min(max(abs(i - a), abs(j - b)) for a, b in zip(ti, tj))
                if d == 0:
                    assert V[s] == 0.0 and pi[s] == -1
                elif d <= nt - 1 - t:
                    assert V[s] == pytest.approx(3.0 - 1.0 * d, abs=1e-12)
                    checked += 1
    assert checked > 100


def test_uniform_flow_without_modes_shifts_the_landing():
    """v = (c_x(t), c_y) constant in space: landing cell floor(i + 1/2 + c + d_a);
    c_x varies with t so a wrong time index in the mean field shows up."""
    nt = 4
    vbar = np.zeros((nt, 9, 9, 2))
    cx = [0.3, -1.7, 1.2, 0.0]
    for t in range(nt):
        vbar[t, :, :, 0] = cx[t]
        vbar[t, :, :, 1] = -0.45
    e = custom_env(nx=9, ny=9, nt=nt, N=8, L=7, vbar=vbar)
    m = oracle.build(e)
    for t in range(nt - 1):
        for (i, j) in [(4, 4), (2, 5), (6, 3)]:
            s = t * e.Nc + j * e.nx + i
            for a in range(e.A):
                ip = math.floor(i + 0.5 + (cx[t] + e.actions[a, 0]))
                jp = math.floor(j + 0.5 + (-0.45 + e.actions[a, 1]))
                col, cnt = _rows(m, a, s)
                assert len(col) == 1 and cnt[0] == e.N
                if 0 <= ip < e.nx and 0 <= jp < e.ny:
                    assert col[0] == (t + 1) * e.Nc + jp * e.nx + ip
                else:
                    assert col[0] == e.nS


def test_uniform_mode_gives_gaussian_drift_probabilities():
    """One spatially uniform mode phi = (1, 0) with coefficient sd sigma: the
    x-offset k has probability Phi((k+1/2-mu)/sigma) - Phi((k-1/2-mu)/sigma),
    mu = c_x + d_x; the y-offset is deterministic.  A second mode (0, 1) with
    sigma = 0 checks that modes are summed per component."""
    nt, N, sig = 3, 20000, 0.6
    vbar = np.zeros((nt, 7, 7, 2))
    vbar[..., 0] = 0.25
    modes = np.zeros((nt, 2, 7, 7, 2))
    modes[:, 0, :, :, 0] = 1.0
    modes[:, 1, :, :, 1] = 1.0
    acts = inputs.action_table(4, 1, 1.0)
    e = custom_env(nx=7, ny=7, nt=nt, K=2, N=N, L=7, vbar=vbar, modes=modes, sigma=[sig, 0.0],
                   actions=acts, seed=77)
    m = oracle.build(e)
    i = j = 3
    for t in range(nt - 1):
        s = t * e.Nc + j * 7 + i
        for a in range(e.A):
            mu = 0.25 + acts[a, 0]
            col, cnt = _rows(m, a, s)
            jp = math.floor(j + 0.5 + acts[a, 1])
            got = {}
            for cc, n in zip(col, cnt):
                if cc == e.nS:
                    got["sink"] = got.get("sink", 0) + n
                    continue
                loc = cc - (t + 1) * e.Nc
                assert loc // 7 == jp
                got[loc % 7 - i] = n
            for k in range(-3, 4):
                p = stats.norm.cdf((k + 0.5 - mu) / sig) - stats.norm.cdf((k - 0.5 - mu) / sig)
                if not (0 <= i + k < 7):
                    continue
                tol = 5 * math.sqrt(N * p * (1 - p)) + 1
                assert abs(got.get(k, 0) - N * p) <= tol, (t, a, k, got.get(k, 0), N * p)


def test_invariants_on_the_tiny_configuration():
    """Row sums = N, sink last and columns ascending, no mass on an obstacle at
    t+1, terminal rows empty, obstacle and horizon rows all-sink, and the
    expected reward from counts equals the paper's per-sample mean sum_R/N."""
    e = inputs.tiny()
    m = oracle.build(e, objs=(oracle.OBJ_TIME,))
    nS, Nc, A = e.nS, e.Nc, e.A
    assert m.overflow == 0
    tgt = np.broadcast_to(e.target[None], e.obstacle.shape).reshape(-1)
    obs = e.obstacle.reshape(-1)
    for r in range(A * nS):
        s = r % nS
        t = s // Nc
        col = m.col[m.rowptr[r]:m.rowptr[r + 1]]
        cnt = m.cnt[m.rowptr[r]:m.rowptr[r + 1]]
        if tgt[s]:
            assert len(col) == 0
            continue
        assert cnt.sum() == e.N
        assert np.all(np.diff(col) > 0)
        if obs[s] or t == e.nt - 1:
            assert list(col) == [nS]
            continue
        inner = col[col < nS]
        assert np.all(inner // Nc == t + 1)
        assert not np.any(obs[inner])
    np.testing.assert_allclose(m.R, m.R_lit, rtol=1e-12, atol=1e-12)
    sums = np.add.reduceat(m.prob, m.rowptr[:-1][np.diff(m.rowptr) > 0])
    np.testing.assert_allclose(sums, 1.0, atol=1e-12)


def test_obstacle_appearing_at_t_plus_1_sends_mass_to_the_sink():
    """The obstacle check uses the mask at the landing time t+1 (Alg. 2)."""
    nt = 3
    obs = np.zeros((nt, 7, 7), np.uint8)
    obs[1, 3, 4] = 1      # east neighbour of (3,3), present at t = 1 only
    e = custom_env(nx=7, ny=7, nt=nt, N=5, L=5, obstacle=obs, r_outbound=-50.0)
    m = oracle.build(e)
    s0 = 0 * e.Nc + 3 * 7 + 3            # (i, j) = (3, 3), t = 0
    col, cnt = _rows(m, 0, s0)           # heading 0 -> east
    assert list(col) == [e.nS]
    assert m.R[0, 0 * e.nS + s0] == -50.0
    s1 = 1 * e.Nc + 3 * 7 + 3            # same move from t = 1 lands at t = 2: free
    col, cnt = _rows(m, 0, s1)
    assert list(col) == [2 * e.Nc + 3 * 7 + 4]


def test_rewards_closed_forms_in_zero_flow():
    """Energy: -c_f F^2 dt; net energy: (-c_f F^2 + c_r (g(s)+g(s'))/2) dt;
    entering the target adds r_term; outside the domain gives r_outbound."""
    nt = 3
    g = np.random.default_rng(3).uniform(0, 2, (nt, 7, 7))
    tgt = np.zeros((7, 7), np.uint8)
    tgt[3, 4] = 1
    acts = inputs.action_table(4, 2, 1.0)    # speeds 0.5 and 1.0
    e = custom_env(nx=7, ny=7, nt=nt, N=6, L=5, gbar=g, target=tgt, actions=acts, c_f=0.7,
                   c_r=1.3, r_term=4.0, r_outbound=-9.0)
    e.dt = 0.5
    objs = (oracle.OBJ_TIME, oracle.OBJ_ENERGY, oracle.OBJ_NET_ENERGY)
    m = oracle.build(e, objs=objs)
    for t in range(nt - 1):
        for (i, j) in [(3, 3), (0, 0), (6, 2)]:
            s = t * e.Nc + j * 7 + i
            for a in range(e.A):
                dxa, dya, F = acts[a]
                ip = math.floor(((i + 0.5) * 1.0 + dxa * 0.5) / 1.0)
                jp = math.floor(((j + 0.5) * 1.0 + dya * 0.5) / 1.0)
                r = a * e.nS + s
                if not (0 <= ip < 7 and 0 <= jp < 7):
                    assert m.R[:, r].tolist() == [-9.0] * 3
                    continue
                bonus = 4.0 if tgt[jp, ip] else 0.0
                want = [-0.5 + bonus, -(0.7 * F * F) * 0.5 + bonus,
                        (-0.7 * F * F + 0.65 * g[t, j, i] + 0.65 * g[t + 1, jp, ip]) * 0.5 + bonus]
                np.testing.assert_allclose(m.R[:, r], want, rtol=1e-14, atol=1e-14)


def test_mean_scalar_field_theorem_by_sampling_the_scalar_field():
    """Sec. III-A: the expected net-energy reward over the joint distribution of
    (s', omega_g) equals the reward computed with the mean field alone.  Draw
    N_rg independent realizations g = gbar + noise for every velocity sample and
    average the per-sample rewards; compare with the oracle's R."""
    nt = 3
    rng = np.random.default_rng(11)
    gbar = rng.uniform(0.5, 1.5, (nt, 7, 7))
    modes = np.zeros((nt, 1, 7, 7, 2))
    modes[:, 0, :, :, 0] = 1.0
    e = custom_env(nx=7, ny=7, nt=nt, K=1, N=3000, L=7, modes=modes, sigma=[0.8], gbar=gbar,
                   actions=inputs.action_table(4, 1, 1.0), seed=5)
    m = oracle.build(e, objs=(oracle.OBJ_NET_ENERGY,))
    Y = oracle.coeffs_for(e)
    t, i, j, a = 0, 3, 3, 0
    s = t * e.Nc + j * 7 + i
    dxa, dya, F = e.actions[a]
    acc = []
    for w in range(e.N):
        ip = math.floor(i + 0.5 + (Y[t, w, 0] + dxa))
        jp = math.floor(j + 0.5 + dya)
        if not (0 <= ip < 7):
            acc.append(e.r_outbound)
            continue
        gs = gbar[t, j, i] + rng.normal(0, 0.5, 20)          # N_rg = 20 scalar realizations
        gsp = gbar[t + 1, jp, ip] + rng.normal(0, 0.5, 20)
        acc.append(np.mean(-F * F + 0.5 * (gs + gsp)))
    naive = np.mean(acc)
    se = 0.5 / math.sqrt(20 * e.N)
    assert abs(naive - m.R[0, a * e.nS + s]) < 6 * se


def test_subgrid_overflow_is_reported():
    vbar = np.zeros((3, 7, 7, 2))
    vbar[..., 0] = 2.2
    e = custom_env(nx=7, ny=7, nt=3, N=4, L=5, vbar=vbar)
    assert oracle.build(e).overflow > 0
    e.L = 7
    assert oracle.build(e).overflow == 0


# ---------------------------------------------------------- solver pins ----
def test_jacobi_fixed_point_equals_backward_induction_bitwise():
    e = inputs.tiny(nx=12, ny=12, nt=8, N=60)
    e.r_term = 5.0
    fx = oracle.fixed_mask(e)
    m = oracle.build(e, objs=(oracle.OBJ_TIME,))
    V, pi, sw, res = oracle.vi_jacobi(m, m.R[0], fx, tol=0.0, nt=e.nt)
    Vb, pib = oracle.vi_backward(m, m.R[0], fx, e.nt, e.Nc)
    assert sw <= e.nt + 1 and res == 0.0
    assert np.array_equal(V, Vb) and np.array_equal(pi, pib)


def test_dense_brute_force_value_iteration_5x5():
    """Dense brute force: P as a dense |S|x|S| matrix per action from the counts,
    r(s,a,s') recomputed per successor from the reward definitions, and
    v_{k+1}(s) = max_a sum_{s'} P(s'|s,a) [r(s,a,s') + v_k(s')] iterated to a
    fixed point -- the Bellman form itself rather than the oracle's R(s,a)."""
    nx = ny = 5
    nt = 6
    tgt = np.zeros((ny, nx), np.uint8)
    tgt[4, 2] = 1
    obs = np.zeros((nt, ny, nx), np.uint8)
    obs[:, 2, 1:3] = 1
    modes = np.zeros((nt, 2, ny, nx, 2))
    modes[:, 0, :, :, 0] = 1.0
    modes[:, 1, :, :, 1] = 1.0
    vbar = np.zeros((nt, ny, nx, 2))
    vbar[..., 0] = 0.2
    g = np.random.default_rng(8).uniform(0, 1, (nt, ny, nx))
    acts = inputs.action_table(8, 2, 1.0)
    e = custom_env(nx=nx, ny=ny, nt=nt, K=2, N=300, L=7, vbar=vbar, modes=modes,
                   sigma=[0.35, 0.2], gbar=g, target=tgt, obstacle=obs, actions=acts, seed=4,
                   r_term=2.0, r_outbound=-40.0, c_f=0.5, c_r=1.5)
    for obj in (oracle.OBJ_TIME, oracle.OBJ_ENERGY, oracle.OBJ_NET_ENERGY):
        m = oracle.build(e, objs=(obj,))
        nS, A, Nc = e.nS, e.A, e.Nc
        P = np.zeros((A, nS, nS + 1))
        for r in range(A * nS):
            a, s = divmod(r, nS)
            for cc, n in zip(m.col[m.rowptr[r]:m.rowptr[r + 1]], m.cnt[m.rowptr[r]:m.rowptr[r + 1]]):
                P[a, s, cc] = n / e.N
        rr = np.zeros((A, nS, nS + 1))
        for a in range(A):
            F = acts[a, 2]
            for s in range(nS):
                t, c = divmod(s, Nc)
                for sp in range(nS + 1):
                    if sp == nS or obs.reshape(-1)[s]:
                        rr[a, s, sp] = -40.0
                        continue
                    tp, cp = divmod(sp, Nc)
                    if obj == oracle.OBJ_TIME:
                        base = -1.0
                    elif obj == oracle.OBJ_ENERGY:
                        base = -0.5 * F * F
                    else:
                        base = -0.5 * F * F + 0.75 * (g.reshape(-1)[s] + g.reshape(-1)[sp])
                    rr[a, s, sp] = base + (2.0 if tgt.reshape(-1)[cp] else 0.0)
        V = np.zeros(nS + 1)
        for _ in range(200):
            Q = np.einsum("asp,asp->as", P, rr + V[None, None, :])
            Vn = np.concatenate([Q.max(axis=0), [0.0]])
            if np.array_equal(Vn, V):
                break
            V = Vn
        Vo, pio, sw, res = oracle.vi_jacobi(m, m.R[0], oracle.fixed_mask(e), tol=0.0, nt=nt)
        np.testing.assert_allclose(Vo, V, rtol=1e-12, atol=1e-12)
        fixed = oracle.fixed_mask(e)
        for s in range(nS):
            if fixed[s]:
                assert pio[s] == -1
                continue
            assert Q[pio[s], s] >= Q[:, s].max() - 1e-12


def _dense_P(m, nS, A, N):
    """Dense P[a][s][s'] (s' = nS is the sink) from the oracle's CSR counts."""
    P = np.zeros((A, nS, nS + 1))
    for r in range(A * nS):
        a, s = divmod(r, nS)
        lo, hi = m.rowptr[r], m.rowptr[r + 1]
        P[a, s, m.col[lo:hi]] += m.cnt[lo:hi] / N
    return P


def test_vi_from_given_values_one_sweep_is_the_bellman_operator():
    """One Jacobi sweep from an arbitrary v_0 (Sec. II-B update
    v_1(s) = max_a [R(s,a) + sum_s' P(s'|s,a) v_0(s')], V(sink) = 0), written
    out with a dense numpy matrix product, against the oracle started from
    the same v_0; also k sweeps = the dense operator applied k times."""
    e = inputs.energy(nx=6, ny=5, nt=4, N=90, L=11, objectives=(0, 1, 2))
    m = oracle.build(e, objs=(0, 1, 2))
    nS, A = e.nS, e.A
    P = _dense_P(m, nS, A, e.N)
    fx = oracle.fixed_mask(e)
    rng = np.random.default_rng(17)
    for o in range(3):
        V0 = rng.normal(0.0, 30.0, nS)
        V = np.concatenate([V0, [0.0]])
        for k in (1, 2, 3):
            Q = m.R[o].reshape(A, nS) + P @ V
            V = np.concatenate([Q.max(axis=0), [0.0]])
            Vo, pio, sw, res = oracle.vi_jacobi(m, m.R[o], fx, tol=-1.0, max_sweeps=k, V0=V0)
            assert sw == k and Vo[nS] == 0.0
            np.testing.assert_allclose(Vo, V, rtol=1e-12, atol=1e-9)
            best = Q.max(axis=0)
            for s in range(nS):
                if fx[s]:
                    assert pio[s] == -1
                else:
                    assert Q[pio[s], s] >= best[s] - 1e-9 * max(1.0, abs(best[s]))


def test_vi_from_any_values_reaches_the_cold_fixed_point_in_nt_plus_1_sweeps():
    """Transitions go from layer t to t+1 or the sink (Sec. II-A, t' = t + dt),
    so after k sweeps layers t >= nt - k no longer depend on v_0: from any v_0
    the iteration is at the cold start's fixed point after nt sweeps (bit for
    bit: the same operations on the same operands) and sweep nt + 1 changes
    nothing."""
    e = inputs.tiny(nx=9, ny=8, nt=6, N=70, r_term=3.0)
    m = oracle.build(e)
    fx = oracle.fixed_mask(e)
    Vc, pic, swc, resc = oracle.vi_jacobi(m, m.R[0], fx, tol=0.0, nt=e.nt)
    rng = np.random.default_rng(5)
    for scale in (1.0, 1e3):
        V0 = rng.normal(0.0, scale, e.nS)
        Vw, piw, sww, resw = oracle.vi_jacobi(m, m.R[0], fx, tol=0.0, nt=e.nt, V0=V0)
        assert sww <= e.nt + 1 and resw == 0.0
        assert np.array_equal(Vw, Vc) and np.array_equal(piw, pic)
    # V0 = 0 given explicitly is the cold start
    Vz, piz, swz, resz = oracle.vi_jacobi(m, m.R[0], fx, tol=0.0, nt=e.nt, V0=np.zeros(e.nS))
    assert np.array_equal(Vz, Vc) and swz == swc
