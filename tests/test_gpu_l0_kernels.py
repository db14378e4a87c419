"""Level 0's Gauss-Seidel colour and residual kernels (sim_set_l0_kernel)
on a 201x199x21 field (1.68M cells, about 840k rows per colour, colour
starts off the 16-byte grid): from the same state and hierarchy, one
timestep with each kernel.

* a thread per row (1), the CTA-staged rows (0), the three pipelined
  bulk-copy kernels (-1: every tile's entries fit its stage; -2: three
  stages; -3: no tile fits, so the entries come from global memory) and the
  whole sweep as one cooperative persistent launch with grid barriers (-4)
  sum every row in the same order: the timesteps end in the same state bit
  for bit, in FP32 and in FP64;
* with several tiles per CTA, the pipelined kernels reuse their stages, and
  none of their bounded waits gives up (the timestep returns DP_OK);
* the lanes-per-row kernels (2, 4, 8) converge to the same state within the
  Newton tolerance.
"""
import numpy as np
import pytest

import dp_inputs as di

pytestmark = pytest.mark.gpu

SAME = (1, 0, -1, -2, -3, -4)


def gpu():
    from paper_1808_04338_gb300 import dpsim
    return dpsim


@pytest.fixture(scope="module")
def prob():
    return di.field8m(201, 199, 21)


@pytest.mark.parametrize("precision", [1, 0])
def test_level0_kernels_agree(prob, precision):
    d = gpu()
    g = d.Sim(prob, d.options("report", precision=precision, cluster_rows=0))
    rc, _ = g.advance(prob.dt)   # builds the hierarchy and level 0's colour copy
    assert rc == 0
    start = g.get_state()
    colour, nc = g.colours()
    counts = np.bincount(colour, minlength=nc)
    assert nc >= 2 and counts[0] > 4 * 256 * 152 and counts[0] % 4 != 0
    states, launches = {}, {}
    for v in SAME + (2, 4, 8):
        g.set_state(*start)
        g.set_l0_kernel(v)
        g.time_kernel("_tma" if v > -4 else "_sweep")
        g.kernel_timing(reset=True)
        rc, st = g.advance(prob.dt)
        _, launches[v] = g.kernel_timing(reset=True)
        g.time_kernel(None)
        assert rc == 0 and st.converged, (v, rc)
        states[v] = g.get_state()
    for v in SAME:
        assert (launches[v] > 0) == (v < 0), (v, launches[v])
        for a, b in zip(states[v], states[1]):
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), v
    p1, s1, b1 = states[1]
    for v in (2, 4, 8):
        p, s, b = states[v]
        assert np.abs(p - p1).max() <= 1e-5 * np.abs(p1).max(), v
        assert np.abs(s - s1).max() <= 1e-5, v
    with pytest.raises(RuntimeError):
        g.set_l0_kernel(3)
    g.close()
