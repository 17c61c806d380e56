"""Writes tests/golden/oracle_small.json: digests and a few values of the FP64
oracle on small seeded environments.  Calls only oracle/ (and the seeded input
generator); rerun it only when a change to the oracle's arithmetic is justified
by the paper, and say which passage in the commit message."""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2109_00857_gb300 import inputs  # noqa: E402


def cases():
    return {
        "tiny_12x12x6": inputs.tiny(nx=12, ny=12, nt=6, N=64, r_term=5.0),
        "energy_16x14x5": inputs.energy(nx=16, ny=14, nt=5, N=80),
    }


def digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def compute():
    out = {}
    for name, env in cases().items():
        m = oracle.build(env, objs=env.objectives)
        V, pi, sw, res = oracle.vi_jacobi(m, m.R[0], oracle.fixed_mask(env), tol=0.0, nt=env.nt)
        s0 = env.start[1] * env.nx + env.start[0]
        out[name] = {"rows": int(len(m.rowptr) - 1), "nnz": int(m.rowptr[-1]),
                     "counts_sha256": digest(m.rowptr, m.col, m.cnt),
                     "R_sha256": digest(m.R), "V_sha256": digest(V, pi),
                     "sweeps": int(sw), "V_start_t0": float(V[s0]), "R_sum": float(m.R.sum())}
    return out


if __name__ == "__main__":
    import platform
    data = compute()
    # the seeded inputs use numpy's transcendental functions, whose last bits
    # may differ between CPU architectures: record where the digests were made
    data["_machine"] = platform.machine()
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")
