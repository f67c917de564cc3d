"""Failure detection on the GPU without a fault: the x-forward pass's bulk copy
completes on an mbarrier whose wait is bounded.  With APM_FAULT_INJECT=wait the
copy is told to expect 16 bytes more than it moves, so the wait runs out; the
kernel sets the status word's timeout bit and returns, apm_sync_status reports
APM_E_TIMEOUT, and the same context then solves normally."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import os, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1410_0010_gb300.solver import Particles, Solver
from paper_1410_0010_gb300._lib import ApmError

dev = torch.device("cuda", 0)
rng = np.random.default_rng(3)
n = 500
pos = 0.2 + 0.6 * rng.random((3, n))
parts = dict(x=pos[0], y=pos[1], z=pos[2], vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n),
             m=np.full(n, 1.0 / n))
P = Particles({k: torch.as_tensor(np.ascontiguousarray(v), device=dev) for k, v in parts.items()})
s = Solver([(0, -1, (0, 0, 0), (16, 16, 16))], periodic=False, precision="fp32", device=0)
bufs = s.alloc_all()
pacc = torch.zeros((3, n), dtype=torch.float32, device=dev)

os.environ["APM_FAULT_INJECT"] = "wait"
s.step(P, 0.0, bufs, pacc)
try:
    s.sync_status()
    print("NO-TIMEOUT")
except ApmError as e:
    print("TIMEOUT" if e.code == 7 else f"OTHER {e.code}")

os.environ.pop("APM_FAULT_INJECT")
pacc.zero_()
s.step(P, 0.0, bufs, pacc)
s.sync_status()
ok = bool(torch.isfinite(pacc).all()) and float(pacc.abs().sum()) > 0
print("RECOVERED" if ok else "BROKEN")
s.close()
"""


def test_bounded_wait_runs_out_and_context_survives():
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.split()
    assert "TIMEOUT" in lines, r.stdout
    assert "RECOVERED" in lines, r.stdout
