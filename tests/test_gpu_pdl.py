"""Programmatic dependent launches (the level-0 well rows, level 0's
pipelined colour kernels, the V-cycle below level 0 and its transfers, the
ILU(0) forward sweep's well rows) change when a kernel may start, never
what it computes: two timesteps of a field in the bench's options (report
mode, FP32 preconditioner, the pipelined level-0 kernel) end in the same
state bit for bit with every class of them (DPSIM_PDL=31, the default),
with none (0), with the early trigger off (27) and with the ILU(0) forward
wells in the colour launch's last CTA instead (15).  DPSIM_PDL is read once
per process, so each setting runs in a child process of its own."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import dp_inputs as di
from paper_1808_04338_gb300 import dpsim
prob = di.field8m(120, 100, 14)
sim = dpsim.Sim(prob, dpsim.options("report", precision=1, cluster_rows=0))
rc, st = sim.advance(prob.dt)            # builds the hierarchy and level 0's colour copy
assert rc == 0 and st.converged, rc
sim.set_l0_kernel(-1)                    # the pipelined bulk-copy colour kernels
rc, st = sim.advance(prob.dt)
assert rc == 0 and st.converged, rc
nlev = len(sim.amg_level_sizes())
p, sw, bhp = sim.get_state()
np.savez(sys.argv[2], p=p, sw=sw, bhp=bhp, nlev=nlev, its=st.linear_iters)
"""


def run_child(mode, out):
    env = dict(os.environ, DPSIM_PDL=str(mode))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, out], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


def test_dependent_launches_change_no_result(tmp_path):
    res = {m: run_child(m, str(tmp_path / f"pdl{m}.npz")) for m in (31, 0, 27, 15)}
    assert int(res[31]["nlev"]) >= 3   # coarse levels below level 0 exist
    for m in (0, 27, 15):
        for k in ("p", "sw", "bhp"):
            assert np.array_equal(res[m][k], res[31][k]), (m, k)
        assert int(res[m]["its"]) == int(res[31]["its"])
