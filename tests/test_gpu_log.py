"""HQ_LOG: one JSON line per hq_step call (step counter, steps taken, the
gradient norm the call returns, inner PCG solves and iterations, wall time),
and the NVTX-instrumented public calls running under it.  Run in a child
process, since the library reads the switch once per process."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
from paper_2605_25149_gb300 import hq, inputs
m, N = 12, 4
s = hq.Solver(m, N, tau=0.4, cg_rtol=1e-10, precision="fp64")
s.set_potential(inputs.wells(m, 2))
s.set_initial(inputs.initial_block(m, N, 102))
gs = [s.step(2) for _ in range(3)]
print(json.dumps({"g": gs, "stats": list(s.pcg_stats())}))
"""


def test_step_log_records_every_call(tmp_path):
    log = tmp_path / "steps.jsonl"
    env = dict(os.environ, HQ_LOG=str(log))
    out = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    lines = [json.loads(l) for l in log.read_text().splitlines()]
    assert len(lines) == 3
    assert [l["step"] for l in lines] == [2, 4, 6]
    assert all(l["nsteps"] == 2 and l["status"] == 0 and l["ms"] > 0 for l in lines)
    assert [l["g"] for l in lines] == res["g"]
    # at least one inner solve per step; the calls' counts add up to the context's
    assert all(l["pcg_solves"] >= 2 for l in lines)
    assert sum(l["pcg_solves"] for l in lines) == res["stats"][0]
    assert sum(l["pcg_iterations"] for l in lines) == res["stats"][1]
    assert all(l["pcg_iterations"] > 0 for l in lines)
