"""The all-cores CPU baseline builds a two-layer slice of the environment:
its layer 0 must give exactly the full environment's layer t (same counts,
successors shifted by t*Nc, same rewards), and the spawned-process run must
finish with every chunk's status 0."""
import numpy as np

import bench
import oracle
from paper_2109_00857_gb300 import inputs


def test_layer_slice_builds_the_same_layer():
    env = inputs.energy(nx=18, ny=15, nt=7, N=150, L=15)
    env.Y = oracle.coeffs_for(env)
    t = 3
    full = oracle.build_units(env, env.objectives, t * env.Nc, (t + 1) * env.Nc)
    sl = oracle.build_units(bench.layer_slice(env, t), env.objectives, 0, env.Nc)
    assert full["status"] == 0 and sl["status"] == 0
    assert np.array_equal(full["nnz"], sl["nnz"])
    assert np.array_equal(full["cnt"], sl["cnt"])
    inner = sl["col"] < 2 * env.Nc                      # in-domain successors of the slice
    shifted = np.where(inner, sl["col"] + t * env.Nc, env.nS)   # sink of the full model
    mask = np.arange(full["col"].shape[1])[None, :] < full["nnz"][:, None]
    assert np.array_equal(np.where(mask, full["col"], 0), np.where(mask, shifted, 0))
    assert np.array_equal(full["R"], sl["R"])


def test_all_cores_baseline_runs_on_two_processes():
    env = inputs.tiny(nx=12, ny=10, nt=4, N=40)
    out = bench.cpu_baseline_all_cores(env, seconds=0.2, workers=2)
    assert out["cores"] == 2 and out["value"] > 0 and out["kind"] == "oracle"


def test_counter_digest_ignores_comments_but_not_code(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// header\n__global__ void k(int *x) {\n  x[0] = 1;  /* one */\n}\n")
    b.write_text("/* another\n   header */\n__global__ void k(int *x) {   // a kernel\n      x[0] = 1;\n}\n")
    c.write_text("// header\n__global__ void k(int *x) {\n  x[0] = 2;  /* one */\n}\n")
    assert bench.source_digest([str(a)]) == bench.source_digest([str(b)])
    assert bench.source_digest([str(a)]) != bench.source_digest([str(c)])
