"""Golden fixtures: the paper's printed numbers (tests/golden/paper_numbers.json,
each with its citation) and the oracle's stored outputs on small seeded cases
(tests/golden/oracle_small.json, written by make_oracle_golden.py from the
oracle only) -- a guard against unintended changes to the oracle."""
import json
import math
import os

import sys

import numpy as np

from paper_2109_00857_gb300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def test_paper_storage_example():
    """Sec. III-A: storing every realization of a 100^3 grid with 1000
    realizations as floats takes 8 GB; the DO form (mean, 10 modes and a
    10 x 1000 x 100 coefficient matrix, per velocity component) takes 96 MB."""
    g = json.load(open(os.path.join(HERE, "paper_numbers.json")))["storage_example"]
    nx, ny, nt = g["grid"]
    Ng, Nr, Nm, b = nx * ny * nt, g["realizations"], g["modes"], g["bytes_per_value"]
    full = Ng * Nr * 2 * b
    assert full == g["full_ensemble_GB"] * 1e9
    per_component = (Ng + Nm * Ng + Nm * Nr * nt) * b
    assert 2 * per_component == g["do_form_MB"] * 1e6
    # this library's layout stores the (scalar) DO coefficients once for both
    # components: mean [nt][ny][nx][2] + modes [nt][K][ny][nx][2] + Y [nt][N][K]
    ours = (Ng * 2 + Nm * Ng * 2 + nt * Nr * Nm) * b
    assert ours == 92e6


def test_paper_application_action_space():
    """Sec. IV: 16 headings x 2 speeds = 32 actions, speeds in (0, F_max]."""
    g = json.load(open(os.path.join(HERE, "paper_numbers.json")))["application_setup"]
    acts = inputs.action_table(g["headings"], g["speeds"], 1.0)
    assert acts.shape[0] == g["actions"]
    assert sorted(set(np.round(acts[:, 2], 12))) == [0.5, 1.0]
    env = inputs.large()
    assert (env.start, env.L) == (tuple(g["start"]), g["subgrid"][0])
    tj, ti = np.nonzero(env.target)
    assert (int(ti.min()), int(tj.min())) == tuple(g["target"])
    for a in range(acts.shape[0]):
        assert math.isclose(math.hypot(acts[a, 0], acts[a, 1]), acts[a, 2], rel_tol=1e-15)


def test_oracle_matches_its_stored_outputs():
    import platform

    import pytest
    import make_oracle_golden as mk
    stored = json.load(open(os.path.join(HERE, "oracle_small.json")))
    machine = stored.pop("_machine")
    if platform.machine() != machine:
        pytest.skip(f"digests were made on {machine}; input generation may round differently here")
    assert mk.compute() == stored
