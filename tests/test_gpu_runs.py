"""Longer GPU runs against the oracle:

* the three forcing terms of Section 3.1 (tiny grid, ten timesteps): every
  Newton iteration's eta and FGMRES count of the first timestep equal the
  oracle's, and the states of all ten steps match;
* the 100x100x10 layered five-spot (200k cells, 400k unknowns), all thirty
  5-day timesteps of the FP64 method, against the oracle's run stored by
  tests/golden/make_layered_run.py (the state after every step, sampled at
  1024 cells and every well);
* the bench's own options (report mode, FP32 preconditioner) over 100 days
  of Example 1's physics on a 20x20x10 grid: after every timestep the GPU's
  state satisfies the oracle's residual equations to the Newton tolerance
  with the mass balance closed, and sim_run over the same period ends in
  the same state.
"""
import os

import numpy as np
import pytest

import dp_inputs as di
import oracle as O

pytestmark = pytest.mark.gpu

P_REL, S_ABS = 1e-8, 1e-8
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "layered_100x100x10_run.npz")


def gpu():
    from paper_1808_04338_gb300 import dpsim
    return dpsim


def state_close(a, b):
    pa, sa, ba = a
    pb, sb, bb = b
    assert np.abs(pa - pb).max() <= P_REL * np.abs(pb).max()
    assert np.abs(sa - sb).max() <= S_ABS
    if len(bb):
        assert np.abs(ba - bb).max() <= P_REL * np.abs(bb).max()


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_forcing_terms_tiny_steps(mode):
    prob = di.tiny()
    kw = dict(eta_mode=mode, eta_min=1e-4, eta_max=0.1)
    g = gpu().Sim(prob, gpu().options("parity", **kw))
    o = O.OracleSim(prob, O.options("parity", **kw))
    opts = O.options("parity")
    # the first timestep Newton iteration by iteration
    res0, etas = None, []
    for l in range(opts.newton_max):
        g.assemble(prob.dt)
        o.assemble(prob.dt)
        ng, no = g.norms(), o.norms()
        res0 = no[0] if l == 0 else res0
        # the same state at l = 0; after that the two updates differ at the
        # rounding of their FGMRES runs, and near convergence the residuals
        # reach the rounding floor of the assembly (about 1e-9 of res0 here)
        np.testing.assert_allclose(ng[:2], no[:2], rtol=1e-12 if l == 0 else 1e-6,
                                   atol=0.0 if l == 0 else 1e-9 * res0)
        if no[0] <= opts.newton_tol * res0 or no[1] <= opts.newton_atol:
            break
        rcg, stg = g.solve_step()
        rco, sto = o.solve_step()
        assert rcg == rco == 0, l
        if no[0] > 1e-7 * res0:   # above the floor: the same eta and FGMRES count
            assert stg.eta == pytest.approx(sto.eta, rel=1e-6), (l, stg.eta, sto.eta)
            assert abs(stg.linear_iters - sto.linear_iters) <= 1, l
            etas.append(sto.eta)
    assert len(etas) >= 3 and len(set(etas)) >= 2
    state_close(g.get_state(), o.get_state())
    # the other nine timesteps
    for step in range(1, prob.nsteps):
        rcg, stg = g.advance(prob.dt)
        rco, sto = o.advance(prob.dt)
        assert rcg == rco == 0, step
        assert abs(stg.newton_iters - sto.newton_iters) <= 1, step
        state_close(g.get_state(), o.get_state())


def test_layered_thirty_steps_against_the_stored_oracle_run():
    ref = np.load(GOLDEN)
    prob = di.layered()
    g = gpu().Sim(prob, gpu().options("parity", newton_tol=float(ref["newton_tol"])))
    cells = ref["cells"]
    assert prob.nsteps == len(ref["p"]) == 30
    for step in range(prob.nsteps):
        rc, st = g.advance(prob.dt)
        assert rc == 0, step
        assert abs(st.newton_iters - int(ref["newton"][step])) <= 1, step
        p, sw, bhp = g.get_state()
        state_close((p[cells], sw[cells], bhp), (ref["p"][step], ref["sw"][step], ref["bhp"][step]))


def _schedule(t_end, dt0, dt_max):
    t, dt, out = 0.0, dt0, []
    while t_end - t > 1e-9 * t_end:
        h = min(dt, t_end - t)
        out.append(h)
        t += h
        dt = min(2.0 * h, dt_max)
    return out


def test_report_mode_run_satisfies_the_oracle_residual_every_step():
    day = di.DAY
    prob = di.paper_example(1, grid=(20, 20, 10))
    gopts = gpu().options("report", precision=1)
    g = gpu().Sim(prob, gopts)
    o = O.OracleSim(prob, O.options("report"))
    tol, atol = gopts.newton_tol, gopts.newton_atol
    kinds0 = [w.kind for w in prob.wells]
    steps = _schedule(100 * day, 1 * day, 20 * day)
    for k, h in enumerate(steps):
        prev = g.get_state()
        rc, st = g.advance(h)
        assert rc == 0 and st.converged, k
        kind, _ = g.well_controls()
        assert list(kind) == kinds0, k          # no control switch in these 100 days
        new = g.get_state()
        o.set_state(*prev)                      # x^n = the GPU's previous state
        o.assemble(h)
        r0 = o.norms()
        o.set_iterate(*new)
        o.assemble(h)
        r = o.norms()
        assert r[0] <= tol * r0[0] * (1 + 1e-6) or r[1] <= atol, (k, r[0] / r0[0])
        for a in range(2):                      # mass change = h x well inflow
            dm, w = r[4 + a], r[6 + a] * h
            assert abs(dm - w) <= 1e-3 * max(abs(dm), abs(w)), (k, a)
    # sim_run over the same period takes the same steps to the same state
    g2 = gpu().Sim(prob, gopts)
    rc, rs = g2.run(100 * day, 1 * day, 20 * day, 0.001 * day)
    assert rc == 0 and rs.steps == len(steps) and rs.cuts == 0
    for a, b in zip(g2.get_state(), g.get_state()):
        np.testing.assert_array_equal(a, b)
