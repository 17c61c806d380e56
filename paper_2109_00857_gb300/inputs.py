"""Seeded synthetic environments (inputs only; none of the method's arithmetic).

The paper's experiments run on a DO-QG stochastic double gyre in a 1000 km
basin (Sec. IV) whose solution is not available, so these generators stand in
for it with the same shapes: a square grid in nondimensional cell units
(dx = dt = 1), 16 headings x 1-2 speeds, up to N = 5000 realizations, a
21x21 neighbouring sub-grid, square obstacles that enter from the west and
move east, a westward-drifting scalar (solar) field, start and target at 0.2
and 0.8 of the domain height.

  mean flow  : the analytic time-periodic double gyre (Shadden, Lekien & Marsden
               2005), psi = A sin(pi f(x,t)) sin(pi y),
               f = eps sin(wt) x^2 + (1 - 2 eps sin(wt)) x on [0,2]x[0,1],
               rescaled so that max |vbar| over grid and time = amplitude
  DO modes   : velocities of psi_mn = sin(m pi x - 0.1 pi t/Nt) sin(n pi y)
               on the unit square, Gram-Schmidt orthonormalised per time step
               under <a,b> = mean over cells of (a_u b_u + a_v b_v)
  sigma      : per-mode standard deviations of the DO coefficients
  gbar       : three unit Gaussian blobs (std 0.1 Nx) drifting west 1 cell/step
  obstacles  : squares entering from the west, moving east 1 cell per 2 steps
  actions    : theta_h = 2 pi h / Nh, F_f = Fmax (f+1)/NF, a = f*Nh + h,
               table (F cos theta, F sin theta, F) computed here in FP64

Both the CUDA library and the oracle consume these arrays; this module holds
no part of the MDP build or the value iteration.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

OBJ_TIME, OBJ_ENERGY, OBJ_NET_ENERGY = 0, 1, 2


@dataclasses.dataclass
class Environment:
    nx: int
    ny: int
    nt: int
    K: int
    N: int
    L: int
    vbar: np.ndarray          # [nt][ny][nx][2] float64
    modes: np.ndarray         # [nt][K][ny][nx][2] float64
    sigma: np.ndarray         # [K] float64
    seed: int
    obstacle: np.ndarray      # [nt][ny][nx] uint8
    target: np.ndarray        # [ny][nx] uint8
    actions: np.ndarray       # [A][3] float64 (dx_a, dy_a, F_a)
    gbar: Optional[np.ndarray] = None   # [nt][ny][nx] float64
    Y: Optional[np.ndarray] = None      # [nt][N][K] external coefficient table, or None
    mdp_id: int = 0
    dx: float = 1.0
    dt: float = 1.0
    c_f: float = 1.0
    c_r: float = 1.0
    r_term: float = 0.0
    r_outbound: float = 0.0
    start: tuple = (0, 0)
    objectives: tuple = (OBJ_TIME,)
    name: str = ""

    @property
    def A(self) -> int:
        return int(self.actions.shape[0])

    @property
    def Nc(self) -> int:
        return self.nx * self.ny

    @property
    def nS(self) -> int:
        return self.nt * self.nx * self.ny

    def samples(self) -> int:
        """Landing evaluations of one full build, N*A per (t, cell)."""
        return self.N * self.A * self.nS


# ------------------------------------------------------------------ pieces --
def action_table(n_headings: int, n_speeds: int, f_max: float) -> np.ndarray:
    """(F cos theta, F sin theta, F) for a = f*Nh + h (Sec. II-A action space)."""
    a = np.zeros((n_headings * n_speeds, 3), dtype=np.float64)
    for f in range(n_speeds):
        F = f_max * (f + 1) / n_speeds
        for h in range(n_headings):
            th = 2.0 * math.pi * h / n_headings
            a[f * n_headings + h] = (F * math.cos(th), F * math.sin(th), F)
    return a


def double_gyre(nx: int, ny: int, nt: int, amplitude: float, eps: float = 0.25,
                phase: float = 0.0) -> np.ndarray:
    """Mean flow [nt][ny][nx][2] in cells per step, max speed = amplitude."""
    xh = (np.arange(nx) + 0.5) / nx * 2.0
    yh = (np.arange(ny) + 0.5) / ny
    X, Yg = np.meshgrid(xh, yh)            # [ny][nx]
    out = np.zeros((nt, ny, nx, 2), dtype=np.float64)
    om = 2.0 * math.pi / max(nt, 1)
    for t in range(nt):
        st = eps * math.sin(om * t + phase)
        f = st * X ** 2 + (1.0 - 2.0 * st) * X
        dfdx = 2.0 * st * X + (1.0 - 2.0 * st)
        u = -math.pi * np.sin(math.pi * f) * np.cos(math.pi * Yg)
        v = math.pi * np.cos(math.pi * f) * np.sin(math.pi * Yg) * dfdx
        out[t, :, :, 0] = u * (nx / 2.0)   # unit-square coordinates -> cells
        out[t, :, :, 1] = v * ny
    sp = np.sqrt(out[..., 0] ** 2 + out[..., 1] ** 2).max()
    if sp > 0:
        out *= amplitude / sp
    return out


_MODE_ORDER = [(1, 1), (2, 1), (1, 2), (2, 2), (3, 1), (1, 3), (3, 2), (2, 3)]


def do_modes(nx: int, ny: int, nt: int, K: int) -> np.ndarray:
    """Orthonormal sinusoidal modes [nt][K][ny][nx][2] (unit RMS speed each)."""
    assert K <= len(_MODE_ORDER)
    xt = (np.arange(nx) + 0.5) / nx
    yt = (np.arange(ny) + 0.5) / ny
    X, Yg = np.meshgrid(xt, yt)
    out = np.zeros((nt, K, ny, nx, 2), dtype=np.float64)
    for t in range(nt):
        ph = 0.1 * math.pi * t / max(nt, 1)
        basis = []
        for k in range(K):
            m, n = _MODE_ORDER[k]
            u = -n * math.pi * np.sin(m * math.pi * X - ph) * np.cos(n * math.pi * Yg)
            v = m * math.pi * np.cos(m * math.pi * X - ph) * np.sin(n * math.pi * Yg)
            vec = np.stack([u, v], axis=-1)
            for b in basis:
                vec = vec - np.mean(np.sum(vec * b, axis=-1)) * b
            nrm = math.sqrt(np.mean(np.sum(vec * vec, axis=-1)))
            vec = vec / nrm
            basis.append(vec)
            out[t, k] = vec
    return out


def solar_field(nx: int, ny: int, nt: int, rng: np.random.Generator) -> np.ndarray:
    """Three unit Gaussian blobs (std 0.1 Nx) drifting west 1 cell/step, periodic in x."""
    cx0 = rng.uniform(0, nx, size=3)
    cy = rng.uniform(0.2 * ny, 0.8 * ny, size=3)
    sd = 0.1 * nx
    xi = np.arange(nx) + 0.5
    yj = np.arange(ny) + 0.5
    out = np.zeros((nt, ny, nx), dtype=np.float64)
    for t in range(nt):
        for b in range(3):
            cx = (cx0[b] - t) % nx
            dxp = np.minimum(np.abs(xi - cx), nx - np.abs(xi - cx))
            out[t] += np.exp(-0.5 * (dxp[None, :] ** 2 + (yj[:, None] - cy[b]) ** 2) / sd ** 2)
    return out


def moving_squares(nx: int, ny: int, nt: int, side: int, rows=(0.35, 0.65),
                   starts=None) -> np.ndarray:
    """Squares entering from the west and moving east 1 cell per 2 steps."""
    m = np.zeros((nt, ny, nx), dtype=np.uint8)
    if starts is None:
        starts = [-side, -side - nx // 4]
    for t in range(nt):
        for r, x0 in zip(rows, starts):
            xl = x0 + t // 2
            yc = int(round(r * ny))
            y0 = yc - side // 2
            xs, xe = max(xl, 0), min(xl + side, nx)
            ys, ye = max(y0, 0), min(y0 + side, ny)
            if xs < xe and ys < ye:
                m[t, ys:ye, xs:xe] = 1
    return m


def target_block(nx: int, ny: int, i0: int, j0: int, size: int = 2) -> np.ndarray:
    tg = np.zeros((ny, nx), dtype=np.uint8)
    tg[j0:j0 + size, i0:i0 + size] = 1
    return tg


def external_coefficients(nt: int, N: int, K: int, sigma: Sequence[float], seed: int) -> np.ndarray:
    """An externally supplied coefficient table Y[t][w][k] (e.g. the output of a
    DO solver, the paper's Alg. 1 input mu_i) drawn with numpy's own generator."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nt, N, K)) * np.asarray(sigma, dtype=np.float64)[None, None, :]


# ----------------------------------------------------------------- configs --
def make_env(nx, ny, nt, K, N, L, sigma, seed, amplitude, n_headings, n_speeds, f_max=1.0,
             obstacle="none", square=10, with_gbar=False, objectives=(OBJ_TIME,), name="",
             r_term=0.0, r_outbound=None, c_f=1.0, c_r=1.0, mdp_id=0, eps=0.25, phase=0.0,
             external_Y=False) -> Environment:
    rng = np.random.default_rng(seed)
    vbar = double_gyre(nx, ny, nt, amplitude, eps=eps, phase=phase)
    modes = do_modes(nx, ny, nt, K)
    if obstacle == "none":
        obs = np.zeros((nt, ny, nx), dtype=np.uint8)
    elif obstacle == "static_rect_20":
        obs = np.zeros((nt, ny, nx), dtype=np.uint8)
        obs[:, 6:14, 8:12] = 1
    elif obstacle == "squares":
        obs = moving_squares(nx, ny, nt, square)
    else:
        raise ValueError(obstacle)
    i0, j0 = nx // 2, int(round(0.8 * ny))
    tgt = target_block(nx, ny, i0, min(j0, ny - 2))
    start = (nx // 2, int(round(0.2 * ny)))
    gbar = solar_field(nx, ny, nt, rng) if with_gbar else None
    sig = np.asarray(sigma, dtype=np.float64)
    if r_outbound is None:
        r_outbound = -10.0 * nt * 1.0
    Y = external_coefficients(nt, N, K, sig, seed + 7919) if external_Y else None
    return Environment(nx=nx, ny=ny, nt=nt, K=K, N=N, L=L, vbar=vbar, modes=modes, sigma=sig,
                       seed=seed, obstacle=obs, target=tgt,
                       actions=action_table(n_headings, n_speeds, f_max), gbar=gbar, Y=Y,
                       mdp_id=mdp_id, c_f=c_f, c_r=c_r, r_term=r_term, r_outbound=r_outbound,
                       start=start, objectives=tuple(objectives), name=name)


def tiny(**kw) -> Environment:
    """Plain method, tiny: 20x20, nt=10, K=2 sigma=(0.2,0.1), N=200, 16 headings at F=1,
    one static rectangle, time objective, 7x7 sub-grid, mean flow amplitude 0.5."""
    args = dict(nx=20, ny=20, nt=10, K=2, N=200, L=7, sigma=(0.2, 0.1), seed=11,
                amplitude=0.5, n_headings=16, n_speeds=1, obstacle="static_rect_20",
                objectives=(OBJ_TIME,), name="tiny-20x20x10-N200-A16")
    args.update(kw)
    return make_env(**args)


def energy(**kw) -> Environment:
    """Energy harvesting: 100x100, nt=60, K=4, N=1000, 32 actions (16 x {0.5,1}), solar
    mean field, two moving 10x10 squares, net-energy objective, 15x15 sub-grid."""
    args = dict(nx=100, ny=100, nt=60, K=4, N=1000, L=15, sigma=(0.3, 0.2, 0.15, 0.1), seed=22,
                amplitude=2.5, n_headings=16, n_speeds=2, obstacle="squares", square=10,
                with_gbar=True, objectives=(OBJ_NET_ENERGY,),
                name="energy-100x100x60-N1000-A32")
    args.update(kw)
    return make_env(**args)


def large(**kw) -> Environment:
    """Large single instance: 200x200, nt=120, K=8 sigma_k=0.3*2^(-k/2), N=5000, 32 actions,
    all three objectives from one build, 21x21 sub-grid, two moving 20x20 squares."""
    args = dict(nx=200, ny=200, nt=120, K=8, N=5000, L=21,
                sigma=tuple(0.3 * 2.0 ** (-k / 2.0) for k in range(8)), seed=33,
                amplitude=2.5, n_headings=16, n_speeds=2, obstacle="squares", square=20,
                with_gbar=True, objectives=(OBJ_TIME, OBJ_ENERGY, OBJ_NET_ENERGY),
                name="large-200x200x120-N5000-A32")
    args.update(kw)
    return make_env(**args)


def batch_member(i: int, **kw) -> Environment:
    """One of the 64 uneven MDPs: side ~U{40..160}, nt ~U{20..80}, K ~U{2..6},
    N ~U{500..2000}, A in {16, 32}, own seed, eps, phase and obstacles."""
    rng = np.random.default_rng(4400 + i)
    side = int(rng.integers(40, 161))
    nt = int(rng.integers(20, 81))
    K = int(rng.integers(2, 7))
    N = int(rng.integers(500, 2001))
    nspd = int(rng.integers(1, 3))
    sig = tuple(0.3 * 2.0 ** (-k / 2.0) for k in range(K))
    args = dict(nx=side, ny=side, nt=nt, K=K, N=N, L=21, sigma=sig, seed=4400 + i,
                amplitude=2.0, n_headings=16, n_speeds=nspd, obstacle="squares",
                square=max(4, side // 10), with_gbar=True, objectives=(OBJ_TIME,),
                eps=float(rng.uniform(0.1, 0.3)), phase=float(rng.uniform(0, 2 * math.pi)),
                mdp_id=i, name=f"batch-{i}")
    args.update(kw)
    return make_env(**args)


# ------------------------------------------------------------------ 3-D grid --
@dataclasses.dataclass
class Environment3D:
    """A 3-D environment (Sec. II-A with n = 3): cube cells, three velocity
    components, actions with a vertical component."""
    nx: int
    ny: int
    nz: int
    nt: int
    K: int
    N: int
    L: int
    vbar: np.ndarray          # [nt][nz][ny][nx][3] float64
    modes: np.ndarray         # [nt][K][nz][ny][nx][3] float64
    sigma: np.ndarray         # [K] float64
    seed: int
    obstacle: np.ndarray      # [nt][nz][ny][nx] uint8
    target: np.ndarray        # [nz][ny][nx] uint8
    actions: np.ndarray       # [A][4] float64 (dx_a, dy_a, dz_a, F_a)
    gbar: Optional[np.ndarray] = None   # [nt][nz][ny][nx] float64
    Y: Optional[np.ndarray] = None      # [nt][N][K] or None
    mdp_id: int = 0
    dx: float = 1.0
    dt: float = 1.0
    c_f: float = 1.0
    c_r: float = 1.0
    r_term: float = 0.0
    r_outbound: float = 0.0
    objectives: tuple = (OBJ_TIME,)
    name: str = ""

    @property
    def A(self) -> int:
        return int(self.actions.shape[0])

    @property
    def Nc(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nS(self) -> int:
        return self.nt * self.Nc

    def samples(self) -> int:
        return self.N * self.A * self.nS


def action_table3d(n_headings: int, elevations: Sequence[float], speeds: Sequence[float]) -> np.ndarray:
    """(F cos e cos theta, F cos e sin theta, F sin e, F) for every speed F,
    elevation angle e and heading theta_h = 2 pi h / Nh (a = (f*Ne + e)*Nh + h);
    straight up/down (|e| = pi/2) is listed once per speed."""
    rows = []
    for F in speeds:
        for e in elevations:
            hs = [0] if abs(abs(e) - math.pi / 2) < 1e-12 else range(n_headings)
            for h in hs:
                th = 2.0 * math.pi * h / n_headings
                rows.append((F * math.cos(e) * math.cos(th), F * math.cos(e) * math.sin(th), F * math.sin(e), F))
    return np.asarray(rows, dtype=np.float64)


def make_env3d(nx, ny, nz, nt, K, N, L, sigma, seed, amplitude, w_amplitude=0.3, n_headings=8,
               elevations=(-math.pi / 4, 0.0, math.pi / 4), speeds=(1.0,), obstacle_boxes=1,
               with_gbar=False, objectives=(OBJ_TIME,), r_term=0.0, r_outbound=None, name="",
               mdp_id=0) -> Environment3D:
    """Layers of the 2-D double gyre (amplitude decaying with depth), a weak
    vertical velocity cos(pi z) sin(2 pi x), modes = the 2-D modes with a
    vertical component sin(pi z) (orthonormalised per step), boxes drifting
    east, target block near the top, solar field on every layer."""
    rng = np.random.default_rng(seed)
    g2 = double_gyre(nx, ny, nt, amplitude)
    zt = (np.arange(nz) + 0.5) / nz
    xt = (np.arange(nx) + 0.5) / nx
    vbar = np.zeros((nt, nz, ny, nx, 3))
    for k in range(nz):
        vbar[:, k, :, :, :2] = g2 * (1.0 - 0.5 * zt[k])
        vbar[:, k, :, :, 2] = w_amplitude * math.cos(math.pi * zt[k]) * np.sin(2 * math.pi * xt)[None, None, :]
    m2 = do_modes(nx, ny, nt, K)
    modes = np.zeros((nt, K, nz, ny, nx, 3))
    for t in range(nt):
        basis = []
        for q in range(K):
            vec = np.zeros((nz, ny, nx, 3))
            vec[..., :2] = m2[t, q][None] * np.cos(0.5 * math.pi * zt)[:, None, None, None]
            vec[..., 2] = 0.5 * m2[t, q][None, ..., 0] * np.sin(math.pi * zt)[:, None, None]
            for b in basis:
                vec = vec - np.mean(np.sum(vec * b, axis=-1)) * b
            vec = vec / math.sqrt(np.mean(np.sum(vec * vec, axis=-1)))
            basis.append(vec)
            modes[t, q] = vec
    obs = np.zeros((nt, nz, ny, nx), dtype=np.uint8)
    for bx in range(obstacle_boxes):
        y0 = int(rng.integers(ny // 4, max(ny // 4 + 1, 3 * ny // 4 - 2)))
        z0 = int(rng.integers(0, max(1, nz - 2)))
        side = max(2, nx // 6)
        for t in range(nt):
            x0 = -side + t // 2 + bx * nx // 3
            xs, xe = max(x0, 0), min(x0 + side, nx)
            if xs < xe:
                obs[t, z0:z0 + max(2, nz // 3), y0:y0 + side, xs:xe] = 1
    tgt = np.zeros((nz, ny, nx), dtype=np.uint8)
    tgt[nz - 2:nz, int(0.8 * ny):int(0.8 * ny) + 2, nx // 2:nx // 2 + 2] = 1
    gbar = None
    if with_gbar:
        s2 = solar_field(nx, ny, nt, rng)
        gbar = np.repeat(s2[:, None], nz, axis=1) * (0.5 + 0.5 * zt)[None, :, None, None]
    if r_outbound is None:
        r_outbound = -10.0 * nt
    return Environment3D(nx=nx, ny=ny, nz=nz, nt=nt, K=K, N=N, L=L, vbar=vbar, modes=modes,
                         sigma=np.asarray(sigma, dtype=np.float64), seed=seed, obstacle=obs, target=tgt,
                         actions=action_table3d(n_headings, elevations, speeds), gbar=gbar,
                         mdp_id=mdp_id, r_term=r_term, r_outbound=r_outbound,
                         objectives=tuple(objectives), name=name)


def cube(**kw) -> Environment3D:
    """3-D instance: 64x64x16 cells, nt = 40, K = 4, N = 1000, 8 headings at
    elevations -45, 0 and +45 degrees (24 actions), 7x7x7 sub-grid."""
    args = dict(nx=64, ny=64, nz=16, nt=40, K=4, N=1000, L=7,
                sigma=tuple(0.15 * 2.0 ** (-q / 2.0) for q in range(4)), seed=61, amplitude=0.8,
                objectives=(OBJ_TIME,), name="cube-64x64x16x40-N1000-A24")
    args.update(kw)
    return make_env3d(**args)
