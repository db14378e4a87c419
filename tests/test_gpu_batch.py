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


def _batch_run(members, opts, steps, owned=True):
    """Each member advanced `steps` timesteps by one lockstep batch; returns
    per step [(status, newton, linear, state)] and the batch's launch count.
    owned: the batch on a stream of its own, where its Arnoldi steps are
    captured into CUDA graphs and replayed (else torch's current stream,
    the legacy default stream, where they are launched directly)."""
    import torch
    sims = [gpu().Sim(p, opts, stream=torch.cuda.Stream()) for p in members]
    bst = gpu().OwnedStream() if owned else None
    b = gpu().Batch(sims, stream=bst.torch if owned else None)
    out = []
    for _ in range(steps):   # (j, mask) keys recur across Newton rounds: graphs replayed
        rc, stats, status = b.advance([p.dt for p in members])
        out.append([(status[k], stats[k].newton_iters, stats[k].linear_iters, s.get_state())
                    for k, s in enumerate(sims)])
    n = b.launch_count()
    b.close()
    if bst:
        bst.close()
    for s in sims:
        s.close()
    return out, n


def _alone_run(members, opts, steps):
    import torch
    out = [[] for _ in range(steps)]
    for prob in members:
        s = gpu().Sim(prob, opts, stream=torch.cuda.Stream())
        for t in range(steps):
            rc, st = s.advance(prob.dt)
            out[t].append((rc, st.newton_iters, st.linear_iters, s.get_state()))
        s.close()
    return out


@pytest.mark.parametrize("precision", [1, 2])
def test_batch_equals_alone_bit_for_bit(precision):
    """The lockstep batch (one launch per phase over all members' tiles)
    gives every member exactly what sim_advance gives it alone: the same
    codes, Newton and FGMRES counts and states, bit for bit, over two
    timesteps (the second reuses the AMG hierarchy), with its Arnoldi steps
    replayed from CUDA graphs (its own stream) or launched directly (the
    legacy default stream); a batch of one gives the same too."""
    members = [di.ensemble_member(r) for r in (0, 7, 14, 21, 28, 3, 10, 17)]
    opts = gpu().options("report", precision=precision, cluster_rows=-1)
    alone = _alone_run(members, opts, 2)
    mix, launches = _batch_run(members, opts, 2)
    direct, _ = _batch_run(members, opts, 2, owned=False)
    single, _ = _batch_run(members[3:4], opts, 2)
    for t in range(2):
        for k, (a, m, d) in enumerate(zip(alone[t], mix[t], direct[t])):
            assert a[0] == m[0] == d[0] == 0, (t, k)
            assert a[1:3] == m[1:3] == d[1:3], (t, k, a[1:3], m[1:3])
            for x, y, z in zip(a[3], m[3], d[3]):
                np.testing.assert_array_equal(x, y)
                np.testing.assert_array_equal(x, z)
        for x, y in zip(single[t][0][3], mix[t][3][3]):
            np.testing.assert_array_equal(x, y)
    assert launches > 0


def test_batch_fp_states_match_the_oracle():
    """The batched members in parity mode's tolerances against the FP64
    oracle after one timestep (FP32 preconditioner, fixed forcing term)."""
    members = [di.ensemble_member(r) for r in (0, 5)]
    opts = gpu().options("parity", precision=1, amg_gs_levels=1, cluster_rows=-1)
    mix, _ = _batch_run(members, opts, 1)
    for k, prob in enumerate(members):
        o = OracleSim(prob, oracle_options("parity", amg_gs_levels=1))
        assert o.advance(prob.dt)[0] == 0
        po, so, bo = o.get_state()
        pg, sg, bg = mix[0][k][3]
        assert np.abs(pg - po).max() <= 1e-8 * np.abs(po).max()
        assert np.abs(sg - so).max() <= 1e-8
        assert np.abs(bg - bo).max() <= 1e-8 * np.abs(bo).max()


def test_batch_rejects_unsupported_members():
    """FP64 preconditioner, Gauss-Seidel below level 0, ILU(0) alone or the
    cluster kernel allowed: not batched."""
    import ctypes as C
    prob = di.ensemble_member(0)
    L = gpu().load()
    for kw in (dict(precision=0), dict(precision=1, amg_gs_levels=30), dict(precision=1, precond=1),
               dict(precision=1)):   # the last: the default cluster_rows
        s = gpu().Sim(prob, gpu().options("report", **kw))
        H = (C.c_void_p * 1)(s.h.value)
        h = C.c_void_p()
        assert L.batch_create(C.cast(H, C.c_void_p), 1, None, C.byref(h)) == gpu().DP_EINVAL, kw
        s.close()
