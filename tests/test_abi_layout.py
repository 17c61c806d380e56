"""The ctypes structures of the binding have the C header's layout: a small C
program compiled against include/mdp.h prints sizeof and offsetof of every
field, which must equal the ctypes classes' sizes and field offsets (a field
added on one side only fails here, on the CPU)."""
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2109_00857_gb300 import mdp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C type name -> ctypes class
PAIRS = {
    "mdp_grid": mdp.MdpGrid,
    "mdp_actions": mdp.MdpActions,
    "mdp_env": mdp.MdpEnv,
    "mdp_build_opts": mdp.MdpBuildOpts,
    "mdp_model_info_t": mdp.MdpModelInfo,
    "mdp_solve_stats": mdp.MdpSolveStats,
    "mdp_grid3d": mdp.MdpGrid3D,
    "mdp_env3d": mdp.MdpEnv3D,
    "mdp_actions3d": mdp.MdpActions3D,
    "mdp_build3d_opts": mdp.MdpBuild3DOpts,
    "mdp_rollout_summary": mdp.MdpRolloutSummary,
    "mdp_batch_item": mdp.MdpBatchItem,
    "mdp_request": mdp.MdpRequest,
    "mdp_result": mdp.MdpResult,
    "mdp_tuning": mdp.MdpTuning,
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_struct_layouts_match_the_header():
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mdp.h"', "int main(void) {"]
    for cname, cls in PAIRS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field in cls._fields_:
            f = field[0]
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            name, field, val = ln.split()
            got[(name, field)] = int(val)
    for cname, cls in PAIRS.items():
        assert got[(cname, "size")] == __import__("ctypes").sizeof(cls), cname
        for field in cls._fields_:
            f = field[0]
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
