"""Batched timesteps of uneven-size realisations (sim_advance_many): each
realisation's result in the mix equals its result alone, bit for bit, and
the FP64 path still matches the oracle."""
import numpy as np
import pytest

import dp_inputs as di
from oracle import OracleSim, options as oracle_options

pytestmark = pytest.mark.gpu


def gpu():
    from paper_1808_04338_gb300 import dpsim
    return dpsim


def run_alone(members, mode, precision):
    import torch
    out = []
    for prob in members:
        s = gpu().Sim(prob, gpu().options(mode, precision=precision), stream=torch.cuda.Stream())
        rc, st = s.advance(prob.dt)
        out.append((rc, st.newton_iters, st.linear_iters, s.get_state()))
        s.close()
    return out


def run_mix(members, mode, precision, threads):
    import torch
    sims = [gpu().Sim(p, gpu().options(mode, precision=precision), stream=torch.cuda.Stream())
            for p in members]
    rc, stats, status = gpu().advance_many(sims, [p.dt for p in members], threads=threads)
    out = [(status[k], stats[k].newton_iters, stats[k].linear_iters, s.get_state())
           for k, s in enumerate(sims)]
    return rc, out, sims


@pytest.mark.parametrize("mode,precision,threads", [("parity", 0, 3), ("report", 1, 8)])
def test_mix_equals_alone(mode, precision, threads):
    members = [di.ensemble_member(r) for r in (0, 7, 14, 21, 28, 3, 10, 17)]
    alone = run_alone(members, mode, precision)
    rc, mix, sims = run_mix(members, mode, precision, threads)
    assert rc == 0
    for k, (a, m) in enumerate(zip(alone, mix)):
        assert a[0] == m[0] == 0, k
        assert a[1:3] == m[1:3], (k, a[1:3], m[1:3])
        for x, y in zip(a[3], m[3]):
            np.testing.assert_array_equal(x, y)
    if mode == "parity":
        # the smallest member in the mix against the oracle
        prob = members[0]
        o = OracleSim(prob, oracle_options("parity"))
        assert o.advance(prob.dt)[0] == 0
        p, sw, bhp = mix[0][3]
        po, swo, bo = o.get_state()
        assert np.max(np.abs(p - po) / np.abs(po)) < 1e-8
        assert np.max(np.abs(sw - swo)) < 1e-8
        assert np.max(np.abs(bhp - bo) / np.abs(bo)) < 1e-8
    for s in sims:
        s.close()


def test_shared_streams_serialise_and_duplicates_are_rejected():
    """Sims on one stream are served one after another with the same results;
    a sim listed twice is an error."""
    import torch
    st = torch.cuda.Stream()
    members = [di.ensemble_member(r) for r in (0, 5)]
    alone = run_alone(members, "report", 0)
    sims = [gpu().Sim(p, gpu().options("report"), stream=st) for p in members]
    rc, stats, status = gpu().advance_many(sims, [p.dt for p in members], threads=2)
    assert rc == 0
    for k, s in enumerate(sims):
        for x, y in zip(alone[k][3], s.get_state()):
            np.testing.assert_array_equal(x, y)
    rc, _, _ = gpu().advance_many([sims[0], sims[0]], [1.0, 1.0])
    assert rc == gpu().DP_EINVAL
    for s in sims:
        s.close()


def test_owned_streams_are_distinct():
    ss = [gpu().OwnedStream() for _ in range(40)]
    assert len({s.h.value for s in ss}) == 40
    for s in ss:
        s.close()
