"""Benchmark: one step = the whole hot path on one synthetic workload.

Default workload (N=1): the large single instance -- 200x200 grid, nt = 120,
K = 8 DO modes, N = 5000 realizations, 32 actions, 21x21 sub-grid, all three
objectives from one build -- i.e. one MDP build (coefficient sampling, fused
transition counting and emit) followed by one Jacobi value iteration per
objective, through the C ABI with every input resident in HBM.

value = transitions sampled per second over the whole step (samples / step
time); bellman_updates_per_s = (s, a) backups per second of the solve phase.
With torchrun (N > 1) every rank builds and solves its own independent
instance (different Philox key), no collective on the data path (weak scaling);
the step time is the max over ranks.

--impl reference times the FP64 CPU oracle (the baseline arm: there is no
reference implementation to install) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "transitions sampled/s & Bellman updates/s (% HBM roofline); replan p50/p99 ms"
UNIT = "transitions/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def workload(name, rank=0, nt=None):
    from paper_2109_00857_gb300 import inputs
    kw = {"mdp_id": rank}
    if nt:
        kw["nt"] = nt
    env = getattr(inputs, name)(**kw)
    return env


def source_digest(paths):
    """sha256 of the code of C/CUDA sources with comments and whitespace
    removed (a comment edit keeps the digest; any code edit changes it)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for src in paths:
        with open(os.path.join(ROOT, src)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def kernel_counters(kernel, workload_name):
    """ncu per-unit counters of a kernel (profiles/counters.json), or None when
    the kernel's code changed since the capture or the workload differs."""
    try:
        with open(os.path.join(ROOT, "profiles", "counters.json")) as f:
            c = json.load(f)[kernel]
        if source_digest(c["sources"]) != c["code_sha256"] or \
                not workload_name.startswith(c.get("workload", "large")):
            return None
        return c
    except Exception:
        return None


def bellman_bytes_per_sweep(info, nS, n_obj=1):
    """Algorithmic bytes of one Jacobi sweep solving n_obj objectives on one
    P: 4 B per in-domain successor (offset, count), read once for all
    objectives; per objective 4 B of R per row and, per state, the old V
    read, the V and policy writes and one read of V(s') of the next layer
    (the gathers are served from L1/L2); the cell class once per state.
    Sink entries need no bytes (V = 0); the sliced-ELL padding the layout
    carries is not counted."""
    return 4 * info.nnz_domain + n_obj * (4 * info.rows + nS * (4 + 4 + 2 + 4)) + nS * 1


class ClockSampler:
    def __init__(self, idx):
        self.idx = idx
        self.f = tempfile.NamedTemporaryFile(prefix="clk", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_baseline(env, seconds=12.0):
    """The oracle as it stands, single thread, on a bounded sample of units
    of the same workload (coefficients drawn first, not timed)."""
    import oracle
    Y = oracle.coeffs_for(env)
    env_o = env
    env_o.Y = Y
    t_mid = env.nt // 2
    u0 = t_mid * env.Nc + env.Nc // 3
    per_unit = env.N * env.A
    # calibrate on a few units, then size the sample to ~seconds
    t0 = time.perf_counter()
    oracle.build_units(env_o, env.objectives, u0, u0 + 4, with_literal=False)
    dt = max(time.perf_counter() - t0, 1e-6)
    n = max(4, min(env.Nc, int(4 * seconds / dt)))
    t0 = time.perf_counter()
    out = oracle.build_units(env_o, env.objectives, u0, u0 + n, with_literal=False)
    dt = time.perf_counter() - t0
    env.Y = None
    assert out["status"] == 0
    return {"value": n * per_unit / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} (t, cell) units of layer t={t_mid} x {env.A} actions x N={env.N} "
                      f"({n * per_unit:.3e} landings, {dt:.1f} s, FP64 oracle, 1 thread)",
            "seconds": dt}


def layer_slice(env, t):
    """Layers t and t+1 of `env` as a two-layer environment with those layers'
    coefficients attached: its layer 0 builds exactly env's layer t (the
    moves land in layer 1, which is not the last), so workers need only a
    few MB instead of the whole field."""
    import dataclasses
    import oracle
    Y = env.Y if env.Y is not None else oracle.coeffs_for(env)
    sl = slice(t, t + 2)
    return dataclasses.replace(env, nt=2, vbar=np.ascontiguousarray(env.vbar[sl]),
                               modes=np.ascontiguousarray(env.modes[sl]),
                               obstacle=np.ascontiguousarray(env.obstacle[sl]),
                               gbar=None if env.gbar is None else np.ascontiguousarray(env.gbar[sl]),
                               Y=np.ascontiguousarray(Y[sl]))


_W_ENV = None


def _w_init(env):
    global _W_ENV
    _W_ENV = env
    import oracle
    oracle.lib()


def _w_cells(job):
    objs, u0, u1 = job
    import oracle
    return oracle.build_units(_W_ENV, objs, u0, u1, with_literal=False)["status"]


def cpu_baseline_all_cores(env, seconds=8.0, workers=0):
    """The oracle as it stands on every host core: one spawned process per
    core builds a share of the cells of layer nt/2 (a two-layer slice of the
    environment), wall time from the first to the last cell."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle
    workers = workers or os.cpu_count() or 1
    t_mid = env.nt // 2
    es = layer_slice(env, t_mid)
    per_unit = env.N * env.A
    t0 = time.perf_counter()     # single-thread calibration on a few cells
    oracle.build_units(es, env.objectives, 0, 4, with_literal=False)
    per_cell = max(time.perf_counter() - t0, 1e-6) / 4
    n = int(max(workers, min(env.Nc, seconds * workers / per_cell)))
    chunk = max(1, -(-n // (4 * workers)))
    jobs = [(env.objectives, u, min(n, u + chunk)) for u in range(0, n, chunk)]
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx, initializer=_w_init,
                                initargs=(es,)) as pool:
        list(pool.map(_w_cells, [(env.objectives, 0, 1)] * workers))   # load the library everywhere
        t0 = time.perf_counter()
        status = list(pool.map(_w_cells, jobs))
        dt = time.perf_counter() - t0
    assert all(st == 0 for st in status)
    return {"value": n * per_unit / dt, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{n} cells of layer t={t_mid} x {env.A} actions x N={env.N} "
                      f"({n * per_unit:.3e} landings, {dt:.1f} s, FP64 oracle, {workers} processes)",
            "seconds": dt}


def run_reference(args):
    """Baseline arm: the FP64 oracle on the host cores, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    if args.config == "cube":
        from paper_2109_00857_gb300 import inputs
        env = inputs.cube(with_gbar=True, objectives=(0, 1, 2), name="cube-64x64x16x40-N1000-A24-3obj")
        build = lambda a, b: oracle.build3d_units(env, env.objectives, a, b)
    else:
        env = workload(args.config)
        build = lambda a, b: oracle.build_units(env, env.objectives, a, b, with_literal=False)
    Y = oracle.coeffs_for(env)
    env.Y = Y
    t_mid = env.nt // 2
    u0 = t_mid * env.Nc
    per_unit = env.N * env.A
    t0 = time.perf_counter()
    build(u0, u0 + 2)
    per = (time.perf_counter() - t0) / 2
    n = max(2, int(args.ref_step_seconds / max(per, 1e-6)))
    for w in range(args.warmup):
        build(u0, u0 + n)
    times = []
    for k in range(args.steps):
        a = u0 + (k * n) % max(1, env.Nc - n)
        t0 = time.perf_counter()
        build(a, a + n)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    val = args.steps * n * per_unit / T
    sample = (f"{n} (t, cell) units of layer t={t_mid} per step x {env.A} actions x N={env.N}; "
              f"FP64 oracle build, 1 thread")
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": env.name, "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate(t_ms, samples, backups, world, device):
    """Whole-job numbers over ranks: the step time is the slowest rank's, the
    work is the sum of every rank's (independent instances, weak scaling)."""
    if world <= 1:
        return float(t_ms), float(samples), float(backups)
    import torch
    import torch.distributed as dist
    tmax = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = torch.tensor([float(samples), float(backups)], dtype=torch.float64, device=device)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0]), float(tsum[1])


def batch_compare(steps, warmup):
    """64 uneven MDPs solved exactly (tol = 0): one batched run (persistent
    build launches + the batched layered pass, CUDA graph) against the same 64
    built and solved one after another with the plain calls -- the plain
    method (Jacobi sweeps to tol = 0, the same values bit for bit) and, to
    separate the batching gain from the schedule, the plain layered pass.
    Returns the result line (dict)."""
    import torch
    from paper_2109_00857_gb300 import inputs, mdp
    envs = [inputs.batch_member(i) for i in range(64)]
    denvs = [mdp.DeviceEnv(e, mdp.MDP_FP32) for e in envs]
    b = mdp.Batch(denvs, tol=0.0)
    for _ in range(warmup):
        b.run()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        sweeps, ms = b.run()
        times.append(time.perf_counter() - t0)
    batch_s = statistics.median(times)
    samples = sum(e.samples() - e.N * e.A * e.Nc for e in envs)   # the last layer needs no sampling

    # the plain path: build + solve each member in turn
    def plain(method):
        for d, e in zip(denvs, envs):
            m = mdp.mdp_build(d, objs=(e.objectives[0],))
            mdp.mdp_solve(m, 0, method=method, tol=0.0)
            m.free()

    def timed(method):
        plain(method)
        torch.cuda.synchronize()
        pt = []
        for _ in range(max(1, steps // 2)):
            t0 = time.perf_counter()
            plain(method)
            torch.cuda.synchronize()
            pt.append(time.perf_counter() - t0)
        return statistics.median(pt)
    plain_s = timed(mdp.MDP_SOLVE_JACOBI)
    layered_s = timed(mdp.MDP_SOLVE_LAYERED)
    clocks = clk.stop()
    b.close()
    return {"metric": "batched build+solve to the exact fixed point, solves/s (64 uneven MDPs)",
            "value": 64 / batch_s,
            "unit": "solves/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": batch_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 batch members: side U{40..160}, nt U{20..80}, K U{2..6}, "
                                   "N U{500..2000}, A in {16, 32}", "states": sum(e.nS for e in envs)},
            "transitions_per_s": samples / batch_s, "graph_ms_device": ms,
            "solve": "batched layered pass (tol = 0)",
            "sequential_plain": {"solves_per_s": 64 / plain_s, "ms": plain_s * 1e3,
                                 "solve": "mdp_solve Jacobi, tol = 0"},
            "sequential_layered": {"solves_per_s": 64 / layered_s, "ms": layered_s * 1e3,
                                   "solve": "mdp_solve layered"},
            "speedup_vs_sequential": plain_s / batch_s,
            "speedup_vs_sequential_layered": layered_s / batch_s, "clocks": clocks}


def run_batch(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2109_00857_gb300 import mdp
    mdp.load()
    print(json.dumps(batch_compare(args.steps, args.warmup)), flush=True)


def run_cube(args):
    """The 3-D grid (Sec. II-A with n = 3): one step = the 3-D build of all
    three objectives + one fused Jacobi solve, inputs resident in HBM."""
    import torch
    torch.cuda.set_device(0)
    from paper_2109_00857_gb300 import inputs, mdp
    mdp.load()
    kw = {"nt": args.nt} if args.nt else {}
    env = inputs.cube(with_gbar=True, objectives=(0, 1, 2), name="cube-64x64x16x40-N1000-A24-3obj", **kw)
    objs = env.objectives
    denv = mdp.DeviceEnv3D(env, mdp.MDP_FP32)
    stream = torch.cuda.Stream()
    Vbuf = [torch.empty(env.nS + 1, dtype=torch.float32, device="cuda") for _ in objs]
    Pbuf = [torch.empty(env.nS, dtype=torch.int16, device="cuda") for _ in objs]
    rec = {}

    def step():
        m = mdp.mdp_build3d(denv, objs=objs, stream=stream)
        info = m.info()
        _, _, sts = mdp.mdp_solve_multi(m, tuple(range(len(objs))), tol=0.0, V=Vbuf, policy=Pbuf,
                                        stream=stream)
        rec["info"], rec["stats"] = info, sts
        m.free()
        return info, sts

    for _ in range(args.warmup):
        step()
    clk = ClockSampler(0)
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern_ms, build_ms, solve_ms, samples, backups, launches, full_equiv = [], [], [], 0, 0, 0, 0.0
    e0.record(stream)
    for _ in range(args.steps):
        info, sts = step()
        kern_ms.append(info.kernel_ms)
        build_ms.append(info.build_ms)
        solve_ms.append(sts[0].solve_ms)
        samples += info.samples
        backups += sum(s.backups for s in sts)
        full_equiv += max(s.backups / (env.nS * env.A) for s in sts)
        launches += info.launches + (env.nt + 1) + len(sts)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_ms = e0.elapsed_time(e1)
    info = rec["info"]
    hbm, sm_mhz, peak_kind = peaks()
    bpsw = bellman_bytes_per_sweep(info, env.nS, len(objs))
    sweep_ms = sum(solve_ms) / max(full_equiv, 1e-9)
    bell = bpsw / (sweep_ms / 1e3) / 1e9
    # 3-D build kernel against the issue-slot roofline (as the 2-D build)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    issue_peak = sms * 4 * sm_mhz * 1e6 / 1e12
    kmean = statistics.mean(kern_ms)
    cb = kernel_counters("build3d_warp_kernel", env.name)
    b_ach = cb["warp_inst_per_unit"] * env.nS / (kmean / 1e3) / 1e12 if cb else None
    roof_build = {"kernel": "build3d_warp_kernel (+ build3d_kernel on the slices it leaves)", "bound": "alu",
                  "achieved": b_ach, "peak": issue_peak,
                  "unit": "T warp-inst/s", "frac": b_ach / issue_peak if cb else None,
                  "traffic": cb["dram_bytes_per_unit"] * env.nS if cb else None,
                  "units_per_launch": env.nS, "ms_per_launch": kmean,
                  "counters": cb["summary"] if cb else "stale or absent",
                  "peak_basis": f"{sms} SMs x 4 issue slots x {sm_mhz:.0f} MHz (sm_max_mhz, {peak_kind})"}
    line = {"metric": METRIC, "value": samples / (t_ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": env.name, "grid": [env.nx, env.ny, env.nz, env.nt], "K": env.K,
                       "N": env.N, "A": env.A, "subgrid": f"{env.L}^3", "objectives": list(objs),
                       "solve": "jacobi (fused objectives)", "tol": 0.0, "l2": "inputs_gt_l2"},
            "build_transitions_per_s": info.samples / (statistics.mean(build_ms) / 1e3),
            "bellman_updates_per_s": backups / (sum(solve_ms) / 1e3),
            "phase_ms": {"build": statistics.mean(build_ms), "build_kernel": statistics.mean(kern_ms),
                         "solve": statistics.mean(solve_ms)},
            "sweeps": [s.sweeps for s in rec["stats"]],
            "roofline": roof_build, "roofline_build": roof_build,
            "roofline_bellman": {"kernel": "bellman_kernel_ws" if env.A > 16 else "bellman_kernel", "bound": "hbm", "achieved": bell, "peak": hbm,
                                 "unit": "GB/s", "frac": bell / hbm, "bytes_per_sweep": bpsw,
                                 "ms_per_sweep": sweep_ms, "peak_basis": f"hbm_gbs ({peak_kind})"},
            "gpu_launches": launches, "clocks": clocks, "tuning": None,
            "model": {"nnz": info.nnz, "rows": info.rows, "max_row_nnz": info.max_row_nnz,
                      "device_bytes": info.device_bytes}}
    if not args.no_cpu_baseline:
        import oracle
        env.Y = oracle.coeffs_for(env)
        s0 = (env.nt // 2) * env.Nc + env.Nc // 3
        t0 = time.perf_counter()
        oracle.build3d_units(env, objs, s0, s0 + 2)
        per = max(time.perf_counter() - t0, 1e-6) / 2
        n = max(2, min(env.Nc, int(args.cpu_seconds / per)))
        t0 = time.perf_counter()
        out = oracle.build3d_units(env, objs, s0, s0 + n)
        dt = time.perf_counter() - t0
        assert out["status"] == 0
        line["cpu_baseline"] = {"value": n * env.N * env.A / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{n} start states of layer t={env.nt // 2} x {env.A} actions x "
                                          f"N={env.N}, FP64 3-D oracle build, 1 thread, {dt:.1f} s"}
    print(json.dumps(line), flush=True)


def serve_compare(rates, seconds, n_envs=24):
    """Poisson replanning requests (Sec. V) against the server -- 8 slots and
    1 slot, 120 GB budget -- and against one-at-a-time plain calls (build +
    solve + V and policy to the host, in arrival order) with the plain Jacobi
    schedule and with the plain layered pass; the same request stream for all
    four.  Requests draw one of n_envs resident environments (sides U{30..120},
    nt U{20..60}, K U{1..6}), a start and 2x2 target, sigma x U[0.5, 1.5], a
    seed, N U{500..2000} and an objective.  Returns the result line (dict)."""
    import copy
    import dataclasses
    import torch
    from paper_2109_00857_gb300 import inputs, mdp
    rng = np.random.default_rng(5500)
    envs = []
    for k in range(n_envs):
        side = int(rng.integers(30, 121))
        nt = int(rng.integers(20, 61))
        K = int(rng.integers(1, 7))
        envs.append(inputs.make_env(nx=side, ny=side, nt=nt, K=K, N=1000, L=21,
                                    sigma=tuple(0.3 * 2.0 ** (-q / 2.0) for q in range(K)), seed=5501 + k,
                                    amplitude=2.0, n_headings=16, n_speeds=1 + (k % 2), obstacle="squares",
                                    square=max(4, side // 10), with_gbar=True))
    denvs = [mdp.DeviceEnv(e, mdp.MDP_FP32) for e in envs]

    def requests(rate, seed):
        r = np.random.default_rng(seed)
        t, out = 0.0, []
        while True:
            t += r.exponential(1.0 / rate)
            if t > seconds:
                return out
            k = int(r.integers(0, len(envs)))
            side = envs[k].nx
            out.append((t, k, dict(start=(int(r.integers(0, side)), int(r.integers(0, side))),
                                   target=(int(r.integers(0, side - 2)), int(r.integers(0, side - 2))),
                                   sigma_scale=float(r.uniform(0.5, 1.5)), seed=int(r.integers(1, 1 << 30)),
                                   N=int(r.integers(500, 2001)), objective=int(r.integers(0, 3)))))

    def summary(lat, wall):
        lat = np.asarray(lat)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "solves_per_s": len(lat) / wall, "requests": len(lat), "wall_s": wall}

    def served(slots, reqs):
        srv = mdp.Server(120 << 30, slots)
        ids = [srv.register(d) for d in denvs]
        for i in ids[:4]:   # warm-up
            srv.poll(srv.submit(i, start=(1, 1), target=(5, 5), N=200), timeout_ms=120000)
        t0 = time.perf_counter()
        tickets = []
        for (ta, k, kw) in reqs:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            tickets.append(srv.submit(ids[k], **kw))
        lat = []
        for t in tickets:
            res, _, _ = srv.poll(t, timeout_ms=600000)
            if res.status != 0:
                raise RuntimeError(f"request failed with status {res.status}")
            lat.append(res.latency_ms)
        wall = time.perf_counter() - t0
        srv.close()
        return summary(lat, wall)

    def plain(reqs, method):
        """The plain calls one request at a time, in arrival order;
        latency = completion - arrival."""
        stream = torch.cuda.Stream()
        t0 = time.perf_counter()
        lat = []
        for (ta, k, kw) in reqs:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            e = envs[k]
            d = copy.copy(denvs[k])
            d.env = dataclasses.replace(e, seed=kw["seed"], mdp_id=0, N=kw["N"])
            d.sigma = denvs[k].sigma * kw["sigma_scale"]
            tgt = torch.zeros((e.ny, e.nx), dtype=torch.uint8, device="cuda")
            ti, tj = kw["target"]
            tgt[tj:tj + 2, ti:ti + 2] = 1
            d.target = tgt
            m = mdp.mdp_build(d, objs=(kw["objective"],), stream=stream)
            V, pi, st = mdp.mdp_solve(m, 0, method=method, tol=0.0, stream=stream)
            V.cpu(), pi.cpu()
            m.free()
            lat.append(time.perf_counter() - t0 - ta)
        wall = time.perf_counter() - t0
        return summary(np.array(lat) * 1e3, wall)

    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    rows = []
    for rate in rates:
        reqs = requests(rate, int(rate) + 1)
        s8 = served(8, reqs)
        s1 = served(1, reqs)
        pj = plain(reqs, mdp.MDP_SOLVE_JACOBI)
        pl = plain(reqs, mdp.MDP_SOLVE_LAYERED)
        rows.append({"rate_per_s": rate, "served_8_slots": s8, "server_1_slot": s1,
                     "plain_jacobi": pj, "plain_layered": pl,
                     "served_beats_plain": bool(s8["p99_ms"] < min(pj["p99_ms"], pl["p99_ms"]) and
                                                s8["solves_per_s"] >= 0.99 * max(pj["solves_per_s"],
                                                                                 pl["solves_per_s"]))})
    clocks = clk.stop()
    top = rows[-1]["served_8_slots"]
    return {"metric": "replan p50/p99 ms", "value": top["p99_ms"], "unit": "ms (p99 at the highest rate)",
            "n_gpus": 1, "steps": len(rows), "warmup": 1, "ms_per_step": None, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Poisson replanning requests, {seconds:.0f} s per rate and arm, "
                                   f"{n_envs} resident environments: sides U{{30..120}}, nt U{{20..60}}, "
                                   "K U{1..6}; N U{500..2000}, sigma x U[0.5, 1.5], 120 GB budget",
                       "baseline": "plain mdp_build + mdp_solve one request at a time (Jacobi and layered)"},
            "rates": rows, "clocks": clocks}


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2109_00857_gb300 import mdp
    mdp.load()
    rates = [float(x) for x in args.serve_rates.split(",")]
    print(json.dumps(serve_compare(rates, args.serve_seconds)), flush=True)


def plain_workload(name, steps, warmup):
    """Build + fused Jacobi solve of one configuration (tiny, energy), inputs
    resident in HBM: transitions/s with its own clock record."""
    import torch
    from paper_2109_00857_gb300 import mdp
    env = workload(name)
    objs = env.objectives
    denv = mdp.DeviceEnv(env, mdp.MDP_FP32)
    stream = torch.cuda.Stream()
    Vb = [torch.empty(env.nS + 1, device="cuda") for _ in objs]
    Pb = [torch.empty(env.nS, dtype=torch.int16, device="cuda") for _ in objs]

    def step():
        m = mdp.mdp_build(denv, objs=objs, stream=stream)
        info = m.info()
        _, _, sts = mdp.mdp_solve_multi(m, tuple(range(len(objs))), tol=0.0, V=Vb, policy=Pb, stream=stream)
        m.free()
        return info, sts
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    samples, bms, sms = 0, [], []
    e0.record(stream)
    for _ in range(steps):
        info, sts = step()
        samples += info.samples
        bms.append(info.build_ms)
        sms.append(sts[0].solve_ms)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_ms = e0.elapsed_time(e1)
    return {"workload": env.name, "value": samples / (t_ms / 1e3), "unit": UNIT, "steps": steps,
            "ms_per_step": t_ms / steps, "phase_ms": {"build": statistics.mean(bms), "solve": statistics.mean(sms)},
            "objectives": list(objs), "solve": "jacobi (fused objectives), tol = 0", "clocks": clocks}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", default="large", choices=["tiny", "energy", "large", "batch", "serve", "cube"])
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-rates", default="20,100,200,400")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the tiny / energy / batch / serving measurements of the default line")
    ap.add_argument("--solve", default="jacobi", choices=["jacobi", "jacobi_full", "layered"])
    ap.add_argument("--separate", action="store_true",
                    help="solve the objectives one after another instead of one fused solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-rollout", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--nt", type=int, default=0, help="override nt (small profiling cases only)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == "batch":
        run_batch(args)
        return
    if args.config == "serve":
        run_serve(args)
        return
    if args.config == "cube":
        run_cube(args)
        return

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2109_00857_gb300 import mdp
    mdp.load()

    env = workload(args.config, rank, args.nt)
    objs = env.objectives
    method = {"jacobi": mdp.MDP_SOLVE_JACOBI, "jacobi_full": mdp.MDP_SOLVE_JACOBI_FULL,
              "layered": mdp.MDP_SOLVE_LAYERED}[args.solve]
    denv = mdp.DeviceEnv(env, mdp.MDP_FP32)
    stream = torch.cuda.Stream()
    Vbuf = [torch.empty(env.nS + 1, dtype=torch.float32, device="cuda") for _ in objs]
    Pbuf = [torch.empty(env.nS, dtype=torch.int16, device="cuda") for _ in objs]
    opts = mdp.MdpBuildOpts()
    opts.threads, opts.chunk = args.threads, args.chunk
    rec = {}
    # launch shapes for this workload class, timed on a calibration cut
    # (outside the timed region); the timed builds and solves use them
    tuning = None if args.no_autotune else mdp.mdp_autotune(denv, objs=objs, stream=stream).as_dict()

    def step(d=denv):
        m = mdp.mdp_build(d, objs=objs, opts=opts, stream=stream)
        info = m.info()
        if args.separate:
            sts = []
            for o in range(len(objs)):
                _, _, st = mdp.mdp_solve(m, o, method=method, tol=0.0, V=Vbuf[o], policy=Pbuf[o],
                                         stream=stream)
                sts.append(st)
        else:
            _, _, sts = mdp.mdp_solve_multi(m, tuple(range(len(objs))), method=method, tol=0.0,
                                            V=Vbuf, policy=Pbuf, stream=stream)
        rec["info"], rec["stats"] = info, sts
        m.free()
        return info, sts

    for _ in range(args.warmup):
        step()
    clk = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kern_ms, solve_ms, build_ms, samples, backups, launches, sweeps = [], [], [], 0, 0, 0, []
    full_equiv = 0.0   # solve work in units of one full sweep over every state
    e0.record(stream)
    for _ in range(args.steps):
        info, sts = step()
        kern_ms.append(info.kernel_ms)
        build_ms.append(info.build_ms)
        solve_ms.append(sum(s.solve_ms for s in sts) if args.separate else sts[0].solve_ms)
        samples += info.samples
        backups += sum(s.backups for s in sts)
        sweeps.append([s.sweeps for s in sts])
        per_obj = [s.backups / (env.nS * env.A) for s in sts]
        full_equiv += sum(per_obj) if args.separate else max(per_obj)
        # Jacobi: nt + 1 sweep launches (those after convergence exit at once) + one
        # finalize per objective; layered: one launch per time layer
        n_solves = len(sts) if args.separate else 1
        jac = method != mdp.MDP_SOLVE_LAYERED
        launches += info.launches + n_solves * ((env.nt + 1) if jac else env.nt)
        launches += len(sts) if jac else (0 if args.separate or len(sts) == 1 else 1)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    t_ms = e0.elapsed_time(e1)
    t_ms, samples, backups = aggregate(t_ms, samples, backups, world, "cuda")
    value = samples / (t_ms / 1e3)
    info = rec["info"]
    hbm, sm_mhz, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    # build kernel against the issue-slot roofline: ncu warp instructions per
    # slice x slices per launch / launch time, against one warp instruction
    # per SM sub-partition per cycle (SMs x 4 x sm_max_mhz)
    kmean = statistics.mean(kern_ms)
    n_slices = -(-env.nS // (32 // max(1, 1 << (env.A - 1).bit_length())))
    cb = kernel_counters("build_warp_kernel", env.name)
    issue_peak = sms * 4 * sm_mhz * 1e6 / 1e12                      # T warp-inst/s
    build_achieved = cb["warp_inst_per_unit"] * n_slices / (kmean / 1e3) / 1e12 if cb else None
    # Bellman sweep against HBM
    n_fused = 1 if args.separate else len(objs)
    bpsw = bellman_bytes_per_sweep(info, env.nS, n_fused)
    # device time per full-sweep equivalent of work (Jacobi: the layers the
    # sweeps recomputed; layered: one pass = one sweep's work)
    sweep_ms = sum(solve_ms) / max(full_equiv, 1e-9)
    bell_achieved = bpsw / (sweep_ms / 1e3) / 1e9
    cs = kernel_counters("bellman_kernel_fused3", env.name) if n_fused == 3 else None
    roof_build = {"kernel": "build_warp_kernel (+ build_fp32_kernel on wide slices)", "bound": "alu",
                  "achieved": build_achieved, "peak": issue_peak, "unit": "T warp-inst/s",
                  "frac": build_achieved / issue_peak if cb else None,
                  "traffic": cb["dram_bytes_per_unit"] * n_slices if cb else None,
                  "units_per_launch": n_slices,
                  "warp_inst_per_unit": cb["warp_inst_per_unit"] if cb else None,
                  # HBM is not this kernel's bound (about 0.01 B per landing); reported as asked
                  "dram_gbs": cb["dram_bytes_per_unit"] * n_slices / (kmean / 1e3) / 1e9 if cb else None,
                  "dram_frac_of_hbm": cb["dram_bytes_per_unit"] * n_slices / (kmean / 1e3) / 1e9 / hbm if cb else None,
                  "shared_atom_wavefronts_per_s": (cb.get("shared_atom_wavefronts_per_unit", 0) * n_slices /
                                                   (kmean / 1e3)) if cb else None,
                  "counters": cb["summary"] if cb else "stale or absent: kernel changed since the capture",
                  "ms_per_launch": kmean,
                  "peak_basis": f"{sms} SMs x 4 issue slots x {sm_mhz:.0f} MHz (sm_max_mhz, {peak_kind})"}
    # the warp-specialized sweep serves one-state slices (A_pad = 32)
    bell_name = "bellman_kernel_ws" if env.A > 16 else "bellman_kernel"
    roof_bell = {"kernel": bell_name, "objectives_per_sweep": n_fused, "bound": "hbm",
                 "achieved": bell_achieved, "peak": hbm, "unit": "GB/s", "frac": bell_achieved / hbm,
                 "traffic": cs["dram_bytes_per_unit"] * n_slices if cs else None,
                 "bytes_per_sweep": bpsw, "ms_per_sweep": sweep_ms,
                 "full_sweep_equivalents_per_solve": full_equiv / args.steps,
                 "counters": cs["summary"] if cs else "stale or absent",
                 "peak_basis": f"hbm_gbs ({peak_kind})"}
    build_share = sum(kern_ms) / t_ms
    solve_share = sum(solve_ms) / t_ms
    dominant = roof_build if build_share >= solve_share else roof_bell

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": env.name, "objectives": list(objs), "solve": args.solve,
                       "objective_solves": "separate" if args.separate else "fused",
                       "tol": 0.0, "subgrid": env.L, "l2": "inputs_gt_l2 (model 7 GB, modes 307 MB)",
                       "parallelism": f"replicas x{world}"},
            "bellman_updates_per_s": backups / (sum(solve_ms) / 1e3) / max(1, 1),
            "build_transitions_per_s": info.samples / (statistics.mean(build_ms) / 1e3),
            "phase_ms": {"build": statistics.mean(build_ms), "build_kernel": kmean,
                         "solve": statistics.mean(solve_ms)},
            "sweeps": sweeps[-1],
            "roofline": dominant, "roofline_build": roof_build, "roofline_bellman": roof_bell,
            "gpu_launches": launches, "clocks": clocks, "tuning": tuning,
            "model": {"nnz": info.nnz, "rows": info.rows, "max_row_nnz": info.max_row_nnz,
                      "device_bytes": info.device_bytes}}
    if world > 1:
        line["bellman_updates_per_s"] = backups / (t_ms / 1e3)

    # policy rollouts (Sec. IV) from a grid of starts with the last solve's
    # time-optimal policy, all N realizations each; outside the timed step
    if not args.no_rollout:
        starts = [(i, j) for j in range(env.ny // 16, env.ny, env.ny // 8) for i in range(env.nx // 16, env.nx, env.nx // 8)]
        n_obj = len(objs)
        for _ in range(2):
            rr = mdp.mdp_rollout(denv, Pbuf[0], starts, objs=objs, stream=stream)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        ret_t, steps_t, status_t, summ = mdp.mdp_rollout(denv, Pbuf[0], starts, objs=objs, stream=stream)
        r1.record(stream)
        torch.cuda.synchronize()
        r_ms = r0.elapsed_time(r1)
        n_paths = len(starts) * env.N
        n_steps = int(steps_t.to(torch.int64).sum().item())
        line["rollout"] = {"starts": len(starts), "paths": n_paths, "steps": n_steps, "ms": r_ms,
                           "paths_per_s": n_paths / (r_ms / 1e3), "steps_per_s": n_steps / (r_ms / 1e3),
                           "policy": f"objective {objs[0]}",
                           "p_target_mean": float(np.mean([q.p_target for q in summ])),
                           "note": "includes the coefficient draw and the per-start summaries"}

    # end to end through the C ABI from pinned host buffers
    if not args.no_e2e:
        host = {k: getattr(denv, k).cpu().pin_memory() for k in ("vbar", "modes", "gbar", "obstacle", "target")
                if getattr(denv, k) is not None}
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        Vh = [torch.empty_like(v, device="cpu").pin_memory() for v in Vbuf]
        Ph = [torch.empty_like(p, device="cpu").pin_memory() for p in Pbuf]
        d2h = sum(v.numel() * 4 for v in Vh) + sum(p.numel() * 2 for p in Ph)
        for _ in range(max(1, args.warmup)):
            with torch.cuda.stream(stream):
                for k, t in host.items():
                    getattr(denv, k).copy_(t, non_blocking=True)
            step()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                for k, t in host.items():
                    getattr(denv, k).copy_(t, non_blocking=True)
            step()
            with torch.cuda.stream(stream):
                for v, vh in zip(Vbuf, Vh):
                    vh.copy_(v, non_blocking=True)
                for p, ph in zip(Pbuf, Ph):
                    ph.copy_(p, non_blocking=True)
        f1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = f0.elapsed_time(f1)
        if world > 1:
            tm = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(tm, op=dist.ReduceOp.MAX)
            e2e_ms = float(tm[0])
        line["e2e"] = {"value": samples / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps,
                       "wall_s": time.perf_counter() - t0}

    # the same model solved by the layered pass (backward induction over the
    # time layers, the Jacobi fixed point bit for bit), outside the timed step
    m = mdp.mdp_build(denv, objs=objs, opts=opts, stream=stream)
    lay = []
    for _ in range(3):
        _, _, sts = mdp.mdp_solve_multi(m, tuple(range(len(objs))), method=mdp.MDP_SOLVE_LAYERED, V=Vbuf,
                                        policy=Pbuf, stream=stream)
        lay.append(sts[0].solve_ms)
    m.free()
    line["layered_solve"] = {"ms": min(lay), "objectives": len(objs),
                             "bellman_updates_per_s": env.nS * env.A * len(objs) / (min(lay) / 1e3),
                             "achieved_gbs": bellman_bytes_per_sweep(info, env.nS, len(objs)) / (min(lay) / 1e3) / 1e9,
                             "note": "one pass over P (nt launches): the same values and policy as the Jacobi solve"}

    # the other workloads of the metric, each with its own clock record
    if world == 1 and not args.no_extras and args.config == "large":
        rates = [float(x) for x in args.serve_rates.split(",")]
        line["tiny"] = plain_workload("tiny", 20, 5)
        line["energy"] = plain_workload("energy", 5, 2)
        line["batch"] = batch_compare(5, 2)
        line["serve"] = serve_compare(rates, args.serve_seconds)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(env, args.cpu_seconds)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(env, args.cpu_seconds * 0.7)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
