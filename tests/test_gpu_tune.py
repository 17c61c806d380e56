"""The autotuner (launch shapes per workload class; the paper's authors tuned
threads per block by hand per GPU, Sec. IV-D): it times its candidates,
records the fastest for the class in the process table and a JSON file, and
later builds and solves of that class use them -- with the same model, values
and policy bit for bit as the default shapes, which is what makes tuning safe.
A table loaded from a file applies the same way; a malformed file is refused."""
import json
import os

import numpy as np
import pytest

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


def _run(mdp, d, objs):
    m = mdp.mdp_build(d, objs=objs)
    info = m.info()
    ex = [[x.cpu().numpy() for x in mdp.mdp_export_csr(m, o)] for o in range(len(objs))]
    Vs, ps, sts = mdp.mdp_solve_multi(m, tuple(range(len(objs))), tol=0.0)
    return info, ex, [v.cpu().numpy() for v in Vs], [p.cpu().numpy() for p in ps], [s.sweeps for s in sts]


def _same(a, b):
    assert all(np.array_equal(x, y) for ex_a, ex_b in zip(a[1], b[1]) for x, y in zip(ex_a, ex_b))
    assert all(np.array_equal(x.view(np.uint32), y.view(np.uint32)) for x, y in zip(a[2], b[2]))
    assert all(np.array_equal(x, y) for x, y in zip(a[3], b[3]))
    assert a[4] == b[4]


def test_tuned_shapes_give_the_default_results_bit_for_bit(mdp, tmp_path):
    env = inputs.large(nx=40, ny=36, nt=7, N=900, L=15, square=6)   # a class no other test tunes
    d = mdp.DeviceEnv(env, mdp.MDP_FP32)
    before = _run(mdp, d, env.objectives)                           # default shapes
    path = str(tmp_path / "tuning.json")
    t = mdp.mdp_autotune(d, objs=env.objectives, json_path=path)
    assert t.candidates >= 9 and t.build_warps in (4, 8) and t.sweep_smem_kb in (132, 160, 190)
    assert 1536 <= t.hist_cap <= 4096 and t.build_kernel_ms > 0 and t.sweep_ms > 0
    table = json.load(open(path))
    assert table[t.key.decode()]["hist_cap"] == t.hist_cap
    _same(before, _run(mdp, d, env.objectives))                     # the tuned shapes
    # shapes forced through a loaded file: the other extremes of the candidates
    other = {"build_warps": 12 - t.build_warps, "hist_cap": 1536 if t.hist_cap != 1536 else 4096,
             "threads": 512, "chunk": 333, "sweep_smem_kb": 132 if t.sweep_smem_kb != 132 else 190}
    table[t.key.decode()] = other
    p2 = str(tmp_path / "forced.json")
    json.dump(table, open(p2, "w"))
    mdp.mdp_tuning_load(p2)
    _same(before, _run(mdp, d, env.objectives))
    mdp.mdp_tuning_load(path)                                       # back to the tuned entry


def test_malformed_or_missing_tuning_files_are_refused(mdp, tmp_path):
    bad = tmp_path / "bad.json"
    bad.write_text('{"A32_K1": {"build_warps": 8,, }')
    for p in (str(bad), str(tmp_path / "missing.json")):
        with pytest.raises(mdp.MdpError) as ei:
            mdp.mdp_tuning_load(p)
        assert ei.value.code == -1
