"""The request server (srv_*): concurrent requests of uneven-size
realisations give each realisation the result it has alone (bit for bit
while resident, within the parity tolerance across evictions), admission
respects the device-memory budget, and an oversized realisation is refused."""
import numpy as np
import pytest

import dp_inputs as di

pytestmark = pytest.mark.gpu


def gpu():
    from paper_1808_04338_gb300 import dpsim
    return dpsim


MEMBERS = (0, 9, 18, 27, 4)
DTS = (2.0, 5.0, 3.0)   # days, per request of each realisation


def alone(mode):
    import torch
    out, peaks = [], []
    for r in MEMBERS:
        prob = di.ensemble_member(r)
        s = gpu().Sim(prob, gpu().options(mode), stream=torch.cuda.Stream())
        its = []
        for d in DTS:
            rc, st = s.advance(d * di.DAY)
            assert rc == 0
            its.append((st.newton_iters, st.linear_iters))
        out.append((its, s.get_state()))
        peaks.append(s.footprint()[1])
        s.close()
    return out, peaks


def serve(mode, workers, budget):
    srv = gpu().Server(workers, budget, gpu().options(mode))
    ids = [srv.add(di.ensemble_member(r)) for r in MEMBERS]
    tickets = [[] for _ in ids]
    for d in DTS:                      # interleaved arrivals
        for k, rid in enumerate(ids):
            tickets[k].append(srv.submit(rid, d * di.DAY))
    res = [[srv.wait(t) for t in tk] for tk in tickets]
    states = [srv.state(rid) for rid in ids]
    info = srv.info()
    srv.close()
    return res, states, info


def test_resident_requests_equal_alone():
    ref, peaks = alone("report")
    res, states, info = serve("report", 3, 64 << 30)
    assert info.evictions == 0 and info.loads == len(MEMBERS)
    for k in range(len(MEMBERS)):
        assert [r.status for r in res[k]] == [0] * len(DTS)
        assert [(r.stats.newton_iters, r.stats.linear_iters) for r in res[k]] == ref[k][0]
        for x, y in zip(ref[k][1], states[k]):
            np.testing.assert_array_equal(x, y)
        # one realisation's requests ran in submission order
        t = [(r.t_start_ms, r.t_done_ms) for r in res[k]]
        assert all(t[i][1] <= t[i + 1][0] for i in range(len(t) - 1))
    assert info.resident_bytes <= 64 << 30


def test_evictions_stay_within_budget_and_tolerance():
    ref, peaks = alone("parity")
    budget = int(1.5 * max(peaks))     # the largest realisation and a small one at most
    res, states, info = serve("parity", 3, budget)
    detail = (peaks, budget, info.evictions, info.loads, info.peak_resident_bytes,
              info.bytes_per_row)
    assert info.evictions > 0, detail
    assert info.peak_resident_bytes <= budget, detail
    for k in range(len(MEMBERS)):
        assert [r.status for r in res[k]] == [0] * len(DTS)
        p, sw, bhp = states[k]
        pr, swr, bhpr = ref[k][1]
        assert np.max(np.abs(p - pr) / np.abs(pr)) < 1e-8
        assert np.max(np.abs(sw - swr)) < 1e-8
        assert np.max(np.abs(bhp - bhpr) / np.abs(bhpr)) < 1e-8


def test_oversized_realisation_is_refused():
    """Once a realisation has been measured, one whose estimated footprint
    exceeds the budget gets DP_ENOMEM without being loaded."""
    import torch
    small = di.ensemble_member(0)
    s = gpu().Sim(small, gpu().options("report"), stream=torch.cuda.Stream())
    s.advance(small.dt)
    peak = s.footprint()[1]
    s.close()
    srv = gpu().Server(2, int(1.5 * peak), gpu().options("report"))
    a = srv.add(small)
    b = srv.add(di.ensemble_member(40))   # about 30 times the rows
    assert srv.wait(srv.submit(a, di.DAY)).status == 0
    r = srv.wait(srv.submit(b, di.DAY))
    assert r.status == gpu().DP_ENOMEM and r.loaded == 0
    info = srv.info()
    assert info.resident == 1 and info.loads == 1
    srv.close()
