"""Failures made on the host, on the GPU path (nothing faults the device):

* a device allocator that returns NULL on its k-th call: the call that
  needed the memory returns DP_ENOMEM, later calls refuse work, and
  sim_destroy hands every block it obtained back to the allocator;
* a linear solve that cannot reach its forcing term (one FGMRES iteration
  allowed at eta = 1e-14): sim_solve_step returns DP_ELINEAR and leaves the
  state as it was, sim_advance returns DP_ELINEAR with the old time level
  restored, as the oracle does.
"""
import ctypes as C

import numpy as np
import pytest

import dp_inputs as di
import oracle as O

pytestmark = pytest.mark.gpu


def gpu():
    from paper_1808_04338_gb300 import dpsim
    return dpsim


class CountingAllocator:
    """dp_allocator over torch's caching allocator that counts calls, fails
    the `fail_at`-th one (1-based; 0: never) and keeps a ledger of the blocks
    handed out and not yet returned."""

    def __init__(self, fail_at=0):
        import torch
        d = gpu()
        self.calls, self.fail_at, self.live, self.failed = 0, fail_at, {}, False

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                self.failed = True
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                   stream)
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, nbytes, stream, ctx):
            assert ptr in self.live and self.live[ptr] == nbytes
            del self.live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

        self._a, self._f = d.ALLOC_FN(_alloc), d.FREE_FN(_free)
        self.struct = d.dp_allocator(self._a, self._f, None)


def _run_with_failure(prob, opts, k):
    """Create and advance one timestep with the k-th allocation failing;
    returns (where it failed, rc) and checks the ledger after destroy."""
    L = gpu().load()
    a = CountingAllocator(k)
    try:
        s = gpu().Sim(prob, opts, allocator=a)
    except RuntimeError as e:
        assert a.failed and f"({gpu().DP_ENOMEM})" in str(e), str(e)
        assert not a.live, "blocks left after a failed sim_create"
        return "create", gpu().DP_ENOMEM
    st = gpu().dp_stats()
    rc = L.sim_advance(s.h, float(prob.dt), C.byref(st))
    if a.failed:
        assert rc == gpu().DP_ENOMEM
        # every later call refuses work
        assert L.sim_assemble(s.h, float(prob.dt)) == gpu().DP_ENOMEM
        assert L.sim_advance(s.h, float(prob.dt), C.byref(st)) == gpu().DP_ENOMEM
        cur, peak = s.footprint()
        assert cur == sum(a.live.values()) and peak >= cur
    s.close()
    assert not a.live, "blocks left after sim_destroy"
    return ("solve" if a.failed else "none"), rc


def test_allocator_failure_at_every_stage():
    """The tiny problem with the CPR-FPF preconditioner, FP32 and FP64: count
    the allocations of a whole timestep, then fail each of a spread of them
    (every one of sim_create's first 40, then every fifth) and check the
    code, the refusal of later work and the returned blocks."""
    import torch
    torch.cuda.set_device(0)
    prob = di.tiny()
    for precision in (0, 1):
        opts = gpu().options("report", precision=precision)
        a = CountingAllocator(0)
        s = gpu().Sim(prob, opts, allocator=a)
        n_create = a.calls
        rc, _ = s.advance(prob.dt)
        assert rc == 0
        n_total = a.calls
        s.close()
        assert not a.live and n_total > n_create > 10
        ks = sorted(set(list(range(1, min(n_create, 40) + 1)) + list(range(1, n_total + 1, 5)) +
                    [n_create, n_create + 1, n_total]))
        seen = set()
        for k in ks:
            where, rc = _run_with_failure(prob, opts, k)
            seen.add(where)
            assert where != "none", k
        assert seen == {"create", "solve"}


def test_failed_linear_solve_leaves_the_state():
    """One FGMRES iteration at eta = 1e-14 cannot converge: the solve
    returns DP_ELINEAR without an update, the timestep returns DP_ELINEAR
    with x^n restored; the oracle returns the same codes and also keeps its
    state."""
    prob = di.tiny()
    kw = dict(eta_fixed=1e-14, gmres_maxit=1)
    g = gpu().Sim(prob, gpu().options("parity", **kw))
    o = O.OracleSim(prob, O.options("parity", **kw))
    rng = np.random.default_rng(5)
    state = (prob.p0 + rng.uniform(-1e5, 1e5, prob.n_cells), rng.uniform(0.25, 0.6, prob.n_cells),
             prob.bhp0 + rng.uniform(-1e5, 1e5, prob.n_wells))
    for s in (g, o):
        s.set_state(*state)
        s.assemble(prob.dt)
        n0 = s.norms()
        rc, st = s.solve_step()
        assert rc == gpu().DP_ELINEAR and st.linear_iters == 1 and not st.converged
        for a, b in zip(s.get_state(), state):
            np.testing.assert_array_equal(a, b)
        rc, st = s.advance(prob.dt)
        assert rc == gpu().DP_ELINEAR
        for a, b in zip(s.get_state(), state):
            np.testing.assert_array_equal(a, b)
        # still usable: the same state assembles to the same residual
        s.assemble(prob.dt)
        np.testing.assert_array_equal(s.norms(), n0)
