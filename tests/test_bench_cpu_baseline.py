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
