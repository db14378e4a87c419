"""Writes layered_100x100x10_run.npz: the oracle's run of the 100x100x10
layered five-spot problem (200k cells, 400k unknowns), thirty 5-day
timesteps of the FP64 method (fixed forcing term 1e-10, Newton tolerance
1e-9: the round-off floor of this grid's residual lies near 1e-10), with
the state after every step sampled at 1024 fixed cells and all wells.

Calls only the oracle; run from the repository root:
    python tests/golden/make_layered_run.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import dp_inputs as di  # noqa: E402
import oracle as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "layered_100x100x10_run.npz")
NSAMPLE = 1024
OPTS = dict(newton_tol=1e-9)


def sample_cells(n_cells):
    """1024 cells spread over the grid: every location class, both continua."""
    return np.unique(np.linspace(0, n_cells - 1, NSAMPLE).astype(np.int64))


def main():
    prob = di.layered()
    s = O.OracleSim(prob, O.options("parity", **OPTS))
    cells = sample_cells(prob.n_cells)
    P, S, B, newton, linear = [], [], [], [], []
    for step in range(prob.nsteps):
        t = time.time()
        rc, st = s.advance(prob.dt)
        assert rc == 0, (step, rc)
        p, sw, bhp = s.get_state()
        P.append(p[cells]); S.append(sw[cells]); B.append(bhp)
        newton.append(st.newton_iters); linear.append(st.linear_iters)
        print(step, st.newton_iters, st.linear_iters, f"{time.time() - t:.1f}s", flush=True)
    np.savez_compressed(OUT, cells=cells, p=np.array(P), sw=np.array(S), bhp=np.array(B),
                        newton=np.array(newton), linear=np.array(linear),
                        newton_tol=OPTS["newton_tol"])


if __name__ == "__main__":
    main()
