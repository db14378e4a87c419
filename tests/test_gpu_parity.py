"""GPU (C ABI) against the CPU oracle on the same seeded inputs.

Bit-exact: Jacobian, residual, decoupled matrix, colourings, AMG aggregates
and level operators (integer setup and the values it is computed from).
Floating point: Newton updates and states, pressure within rel 1e-8 and
saturation within abs 1e-8 (FP64 path).
"""
import math

import numpy as np
import pytest

import dp_inputs as di
import oracle as O

pytestmark = pytest.mark.gpu

P_REL, S_ABS = 1e-8, 1e-8


def gpu():
    from paper_1808_04338_gb300 import dpsim
    return dpsim


def small(nx, ny, nz, seed=1, wells="two", g=0.0):
    n = nx * ny * nz
    kf = np.exp(math.log(100.0) + di.normals(seed, 0, n))
    if wells == "two":
        W = [di.Well(di.WELL_RATE_INJ, 0, 0, 0, nz - 1, 100.0 * di.BBL_DAY),
             di.Well(di.WELL_BHP, nx - 1, ny - 1, 0, nz - 1, 2500.0 * di.PSI)]
    elif wells == "bhp":
        W = [di.Well(di.WELL_BHP, 0, 0, 0, nz - 1, 2500.0 * di.PSI)]
    else:
        W = []
    return di._base(f"s{nx}x{ny}x{nz}", nx, ny, nz, kf, np.full(n, 0.1), 0.01, 0.2, 0.08, W,
                    seed, dt_days=1.0, nsteps=2, g=g)


# capillary pressure curves (s_w, p_cow in Pa): weak in the fracture, strong
# in the matrix
PC_F = np.array([[0.2, 2.0e4], [0.5, 5.0e3], [0.8, 0.0]])
PC_M = np.array([[0.2, 5.0e5], [0.35, 2.0e5], [0.5, 8.0e4], [0.65, 2.0e4], [0.8, 0.0]])


def with_pc(prob, pc_f=PC_F, pc_m=PC_M):
    prob.pc_f, prob.pc_m = pc_f, pc_m
    return prob


def pair(prob, mode="parity", **kw):
    return gpu().Sim(prob, gpu().options(mode, **kw)), O.OracleSim(prob, O.options(mode, **kw))


def state_close(g, o, prob):
    pg, sg, bg = g.get_state()
    po, so, bo = o.get_state()
    assert np.abs(pg - po).max() <= P_REL * np.abs(po).max()
    assert np.abs(sg - so).max() <= S_ABS
    if len(bo):
        assert np.abs(bg - bo).max() <= P_REL * np.abs(bo).max()


def update_close(yg, yo, nc):
    assert np.abs(yg[0:2 * nc:2] - yo[0:2 * nc:2]).max() <= P_REL * 3e7
    assert np.abs(yg[1:2 * nc:2] - yo[1:2 * nc:2]).max() <= S_ABS
    assert np.abs(yg[2 * nc::2] - yo[2 * nc::2]).max(initial=0.0) <= P_REL * 3e7


def interior(prob, seed=7):
    rng = np.random.default_rng(seed)
    nc = prob.n_cells
    return (prob.p0 + rng.uniform(-3e5, 3e5, nc), rng.uniform(0.25, 0.75, nc),
            prob.bhp0 + rng.uniform(-1e5, 1e5, prob.n_wells))


@pytest.mark.parametrize("make", [di.tiny, lambda: small(7, 5, 3), lambda: small(1, 1, 1, wells="bhp"),
                                  lambda: small(9, 1, 1), lambda: small(4, 3, 2, wells="none"),
                                  lambda: small(3, 4, 5, g=9.80665),
                                  lambda: di.paper_example(1), lambda: di.paper_example(2),
                                  lambda: with_pc(small(7, 5, 3)),
                                  lambda: with_pc(small(3, 4, 5, g=9.80665)),
                                  lambda: with_pc(small(3, 4, 5, g=9.80665), pc_f=None)])
def test_jacobian_residual_bit_exact(make):
    prob = make()
    g, o = pair(prob)
    for state in (None, interior(prob)):
        if state is not None:
            g.set_iterate(*state)
            o.set_iterate(*state)
        g.assemble(prob.dt)
        o.assemble(prob.dt)
        rg, cg, vg, resg = g.jacobian()
        ro, co, vo, reso = o.jacobian()
        np.testing.assert_array_equal(rg, ro)
        np.testing.assert_array_equal(cg, co)
        assert np.array_equal(vg.view(np.uint64), vo.view(np.uint64))
        assert np.array_equal(resg.view(np.uint64), reso.view(np.uint64))
        ng, no = g.norms(), o.norms()
        np.testing.assert_allclose(ng, no, rtol=1e-12, atol=1e-12 * np.abs(no).max())
    np.testing.assert_array_equal(g.well_index(), o.well_index())


@pytest.mark.parametrize("decouple,schur", [(0, 0), (1, 0), (2, 0), (0, 1), (2, 1)])
def test_decoupling_colours_and_amg_setup_bit_exact(decouple, schur):
    """The decoupled system (the paper's step, ABF, True-IMPES; the full
    system or the fracture-and-well system left by eliminating the matrix
    cells), the colouring and the AMG set-up built on its pressure block,
    bit for bit."""
    prob = di.tiny()
    g, o = pair(prob, decouple=decouple, schur=schur)
    assert (g.snb, g.snnzb) == (o.snb, o.snnzb)
    g.assemble(prob.dt)
    o.assemble(prob.dt)
    g.solve_step()
    o.solve_step()
    vg, bg = g.decoupled()
    vo, bo = o.decoupled()
    assert np.array_equal(vg.view(np.uint64), vo.view(np.uint64))
    assert np.array_equal(bg.view(np.uint64), bo.view(np.uint64))
    cg, ncg = g.colours()
    co, nco = o.colours()
    assert ncg == nco
    np.testing.assert_array_equal(cg, co)
    Lg, Lo = g.amg_levels(), o.amg_levels()
    assert len(Lg) == len(Lo) >= 2
    for a, b in zip(Lg, Lo):
        assert (a["n"], a["nnz"], a["nagg"]) == (b["n"], b["nnz"], b["nagg"])
        for k in ("rowptr", "col", "agg", "colour"):
            np.testing.assert_array_equal(a[k], b[k])
        assert np.array_equal(a["val"].view(np.uint64), b["val"].view(np.uint64))


def dense_from_bsr(rowptr, col, val):
    n = len(rowptr) - 1
    A = np.zeros((2 * n, 2 * n))
    for i in range(n):
        for e in range(rowptr[i], rowptr[i + 1]):
            A[2 * i:2 * i + 2, 2 * col[e]:2 * col[e] + 2] = val[e]
    return A


@pytest.mark.parametrize("precond,gs_levels,decouple,schur", [(1, 30, 0, 0), (2, 30, 0, 0),
                                                               (2, 0, 0, 0), (2, 30, 1, 0),
                                                               (2, 30, 2, 0), (2, 30, 0, 1),
                                                               (1, 30, 0, 1)])
def test_newton_update_parity(precond, gs_levels, decouple, schur):
    """One linear solve at eta = 1e-12 on both sides: the GPU update's true
    residual (dense J from the oracle) is at the tolerance, it agrees with
    the oracle's update as closely as the conditioning of J (~1e12) allows,
    and both take (nearly) the same number of FGMRES iterations."""
    prob = di.tiny()
    g, o = pair(prob, precond=precond, eta_fixed=1e-12, gmres_maxit=1000,
                amg_gs_levels=gs_levels, decouple=decouple, schur=schur)
    st = interior(prob, 3)
    for s in (g, o):
        s.set_iterate(*st)
        s.assemble(prob.dt)
    rowptr, col, val, res = o.jacobian()
    rcg, stg = g.solve_step()
    rco, sto = o.solve_step()
    assert rcg == 0 and rco == 0
    yg, yo = g.update(), o.update()
    J = dense_from_bsr(rowptr, col, val)
    assert np.linalg.norm(J @ yg + res) <= 20 * 1e-12 * np.linalg.norm(res)
    nc = prob.n_cells
    assert np.abs(yg[0:2 * nc:2] - yo[0:2 * nc:2]).max() <= 1e-6 * np.abs(yo[0:2 * nc:2]).max()
    assert np.abs(yg[1:2 * nc:2] - yo[1:2 * nc:2]).max() <= 1e-6
    assert abs(stg.linear_iters - sto.linear_iters) <= 2


@pytest.mark.parametrize("gs_levels,graphs,cluster_rows",
                         [(30, 1, 0), (30, 0, 0), (1, 1, 0), (1, 0, 0), (0, 1, 0),
                          (1, 1, 20000), (0, 1, 20000), (30, 1, -1)])
def test_preconditioner_residual_after_five_iterations(gs_levels, graphs, cluster_rows):
    """The CPR-FPF preconditioner itself, on the 200k-cell layered problem
    (five AMG levels; with graphs and a cluster threshold the coarse ones run
    in the cluster kernel): five FGMRES iterations from zero on both sides
    leave the same relative residual, whichever smoother each level uses
    (Gauss-Seidel on all levels, l1-Jacobi below the finest, l1-Jacobi
    everywhere) and wherever the coarse levels run."""
    prob = di.layered()
    g, o = pair(prob, "parity", eta_fixed=1e-14, gmres_maxit=5, amg_gs_levels=gs_levels)
    g.close()
    g = gpu().Sim(prob, gpu().options("parity", eta_fixed=1e-14, gmres_maxit=5,
                                      amg_gs_levels=gs_levels, use_graphs=graphs,
                                      cluster_rows=cluster_rows))
    for s in (g, o):
        s.assemble(prob.dt)
    rcg, stg = g.solve_step()
    rco, sto = o.solve_step()
    assert stg.linear_iters == sto.linear_iters == 5
    assert 0 < sto.lin_relres < 0.5
    assert abs(stg.lin_relres - sto.lin_relres) <= 1e-6 * sto.lin_relres


def test_unpreconditioned_gmres_single_location():
    """No preconditioner on a one-location problem (6 unknowns): FGMRES
    reduces to GMRES and must reach the dense solution."""
    prob = small(1, 1, 1, wells="bhp")
    g, o = pair(prob, precond=0, eta_fixed=1e-13)
    for s in (g, o):
        s.set_iterate(*interior(prob, 2))
        s.assemble(prob.dt)
    rowptr, col, val, res = o.jacobian()
    rcg, stg = g.solve_step()
    assert rcg == 0 and stg.linear_iters <= 6
    y = np.linalg.solve(dense_from_bsr(rowptr, col, val), -res)
    np.testing.assert_allclose(g.update(), y, rtol=1e-8, atol=1e-8 * np.abs(y).max())


@pytest.mark.parametrize("graphs", [0, 1])
def test_ten_steps_tiny_state_parity(graphs):
    prob = di.tiny()
    g = gpu().Sim(prob, gpu().options("parity", use_graphs=graphs))
    o = O.OracleSim(prob, O.options("parity"))
    for step in range(prob.nsteps):
        rcg, stg = g.advance(prob.dt)
        rco, sto = o.advance(prob.dt)
        assert rcg == 0 and rco == 0, step
        state_close(g, o, prob)


@pytest.mark.parametrize("make", [lambda: small(7, 5, 3), lambda: small(1, 1, 1, wells="bhp"),
                                  lambda: small(9, 1, 1), lambda: small(4, 3, 2, wells="none"),
                                  lambda: small(3, 4, 5, g=9.80665)])
def test_edge_case_steps(make):
    prob = make()
    g, o = pair(prob)
    for step in range(prob.nsteps):
        rcg, _ = g.advance(prob.dt)
        rco, _ = o.advance(prob.dt)
        assert rcg == rco == 0
        state_close(g, o, prob)


@pytest.mark.parametrize("example,days,nsteps", [(1, 5.0, 8), (2, 5.0, 6)])
def test_paper_example_timesteps_and_well_switching(example, days, nsteps):
    """The setups of the paper's two examples (oil-rate producers with a
    minimum BHP, an injector with a given well index and a maximum BHP,
    three layers under gravity in the second): every timestep's state and
    the controls it ended on match the oracle; in the second example both
    producers reach their minimum BHP and go on BHP control."""
    prob = di.paper_example(example, days=days)
    g, o = pair(prob)
    switched = False
    for step in range(nsteps):
        rcg, stg = g.advance(prob.dt)
        rco, sto = o.advance(prob.dt)
        assert rcg == rco == 0, step
        assert stg.newton_iters == sto.newton_iters, step
        state_close(g, o, prob)
        kg, tg = g.well_controls()
        ko, to = o.well_controls()
        np.testing.assert_array_equal(kg, ko)
        np.testing.assert_array_equal(tg, to)
        switched = switched or bool((kg == di.WELL_BHP).any())
    assert switched == (example == 2)


def schedule(total_days, dt_max_days):
    """Timesteps of 1, 2, 4, ... days up to dt_max, the last one ending the period."""
    t, dt, out = 0.0, 1.0, []
    while t < total_days - 1e-9:
        h = min(dt, total_days - t)
        out.append(h)
        t += h
        dt = min(2.0 * dt, dt_max_days)
    return out


@pytest.mark.parametrize("example,total_days", [(1, 800.0), (2, 1600.0)])
def test_paper_example_full_period(example, total_days):
    """The paper's simulation periods (800 and 1600 days) in 20-day steps:
    after every timestep the controls are equal, the states match, and the
    per-well oil and water rates match the oracle's; every producer ends on
    BHP control at its minimum, having produced its target before."""
    prob = di.paper_example(example)
    g, o = pair(prob)
    seen_rate = np.zeros(len(prob.wells), bool)
    for step, days in enumerate(schedule(total_days, 20.0)):
        rcg, _ = g.advance(days * di.DAY)
        rco, _ = o.advance(days * di.DAY)
        assert rcg == rco == 0, step
        state_close(g, o, prob)
        kg, tg = g.well_controls()
        ko, to = o.well_controls()
        np.testing.assert_array_equal(kg, ko)
        np.testing.assert_array_equal(tg, to)
        qg, qo = np.concatenate(g.well_rates()), np.concatenate(o.well_rates())
        assert np.abs(qg - qo).max() <= 1e-6 * np.abs(qo).max(), step
        seen_rate |= kg == di.WELL_OIL_RATE
    assert (kg[1:] == di.WELL_BHP).all() and seen_rate[1:].all()


def test_well_rates_bit_exact_at_the_same_state():
    prob = di.paper_example(2)
    g, o = pair(prob)
    for state in (None, interior(prob, seed=3)):
        if state is not None:
            g.set_state(*state)
            o.set_state(*state)
        for a, b in zip(g.well_rates(), o.well_rates()):
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_layered_200k_first_step_parity():
    """100x100x10 (200k cells): bit-exact assembly and AMG setup, then one
    timestep of Newton in report mode on both sides."""
    prob = di.layered()
    g, o = pair(prob, "report")
    g.assemble(prob.dt)
    o.assemble(prob.dt)
    _, _, vg, rg = g.jacobian()
    _, _, vo, ro = o.jacobian()
    assert np.array_equal(vg.view(np.uint64), vo.view(np.uint64))
    assert np.array_equal(rg.view(np.uint64), ro.view(np.uint64))
    g.solve_step()
    o.solve_step()
    Lg, Lo = g.amg_levels(), o.amg_levels()
    assert len(Lg) == len(Lo)
    for lev, (a, b) in enumerate(zip(Lg, Lo)):
        np.testing.assert_array_equal(a["agg"], b["agg"])
        if lev == 0:   # report options: Gauss-Seidel on level 0 only
            np.testing.assert_array_equal(a["colour"], b["colour"])
        else:          # l1-Jacobi levels get no colouring
            assert (a["colour"] == -1).all(), lev
        assert np.array_equal(a["val"].view(np.uint64), b["val"].view(np.uint64))


@pytest.mark.parametrize("amg_refresh,schur", [(0, 0), (1, 0), (0, 1)])
def test_layered_200k_timestep_parity(amg_refresh, schur):
    """One 5-day timestep of the 200k-cell grid; with amg_refresh = 1 both
    sides keep the coarse AMG values of the timestep's first Newton
    iteration for the later ones."""
    prob = di.layered()
    g, o = pair(prob, "parity", amg_refresh=amg_refresh, schur=schur)
    rcg, stg = g.advance(prob.dt)
    rco, sto = o.advance(prob.dt)
    assert rcg == rco == 0
    assert stg.newton_iters == sto.newton_iters > 1
    state_close(g, o, prob)


@pytest.mark.parametrize("schur", [0, 1])
def test_capillary_pressure_tiny_steps(schur):
    """Ten timesteps with capillary pressure curves in both continua (the
    matrix imbibes water from the fracture): states match the oracle's."""
    prob = with_pc(di.tiny())
    g, o = pair(prob, schur=schur)
    for step in range(prob.nsteps):
        rcg, _ = g.advance(prob.dt)
        rco, _ = o.advance(prob.dt)
        assert rcg == rco == 0, step
        state_close(g, o, prob)


@pytest.mark.parametrize("kw", [dict(amg_refresh=1), dict(decouple=1), dict(decouple=2),
                                dict(schur=1), dict(schur=1, precision=1), dict(reorth=0.0),
                                dict(reorth=1.0)])
def test_tiny_steps_option_variants(kw):
    """Ten tiny timesteps against the FP64 oracle with the coarse AMG values
    kept for a timestep, with the ABF and True-IMPES decouplings, with the
    matrix cells eliminated (FP64 and FP32 preconditioner), and with one or
    always two Gram-Schmidt passes."""
    prob = di.tiny()
    okw = {k: v for k, v in kw.items() if k != "precision"}
    g = gpu().Sim(prob, gpu().options("parity", **kw))
    o = O.OracleSim(prob, O.options("parity", **okw))
    for step in range(prob.nsteps):
        rcg, _ = g.advance(prob.dt)
        rco, _ = o.advance(prob.dt)
        assert rcg == rco == 0, step
        state_close(g, o, prob)


@pytest.mark.parametrize("precond,precision", [(1, 1), (2, 1), (2, 2)])
def test_mixed_precision_preconditioner_tiny_steps(precond, precision):
    """FP32 ILU(0) and AMG inside FP64 FGMRES (precision 2: the coarse AMG
    levels stored in BF16): the Newton states still match the FP64 oracle to
    the parity tolerance (FGMRES wins the accuracy back)."""
    prob = di.tiny()
    g = gpu().Sim(prob, gpu().options("parity", precision=precision, precond=precond,
                                      gmres_maxit=600))
    o = O.OracleSim(prob, O.options("parity", precond=precond, gmres_maxit=600))
    for step in range(4):
        rcg, stg = g.advance(prob.dt)
        rco, sto = o.advance(prob.dt)
        assert rcg == rco == 0, step
        state_close(g, o, prob)


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_layered_timestep(precision):
    prob = di.layered()
    g = gpu().Sim(prob, gpu().options("parity", precision=precision))
    o = O.OracleSim(prob, O.options("parity"))
    rcg, stg = g.advance(prob.dt)
    rco, sto = o.advance(prob.dt)
    assert rcg == rco == 0
    state_close(g, o, prob)
    assert stg.linear_iters <= 2 * sto.linear_iters


def test_autotune_keeps_parity():
    """The autotuner changes launch shapes only: after it, the next timestep
    still matches the oracle; before any hierarchy exists it refuses."""
    prob = di.layered()
    g, o = pair(prob, "parity", newton_tol=1e-9)   # the second step stalls near 1e-10 on both sides
    with pytest.raises(RuntimeError):
        g.autotune(2)
    assert g.advance(prob.dt)[0] == 0 and o.advance(prob.dt)[0] == 0
    rep = g.autotune(3)
    assert "level 0" in rep and "prolongation" in rep and "restriction" in rep
    rcg, _ = g.advance(di.DAY)
    rco, _ = o.advance(di.DAY)
    assert rcg == 0 and rco == 0
    state_close(g, o, prob)


def test_run_matches_the_oracle_over_example_1():
    """sim_run over Example 1's 800 days (steps doubling from 1 day up to 20)
    against oracle_run: the same accepted steps and cuts, the same end time,
    the final state within the parity tolerances."""
    prob = di.paper_example(1)
    g, o = pair(prob)
    args = (800 * di.DAY, 1 * di.DAY, 20 * di.DAY, 0.01 * di.DAY)
    rcg, sg = g.run(*args)
    rco, so = o.run(*args)
    assert rcg == rco == 0
    assert (sg.steps, sg.cuts) == (so.steps, so.cuts) and sg.t == so.t
    assert abs(sg.newton_iters - so.newton_iters) <= 0.02 * so.newton_iters
    state_close(g, o, prob)


def _gpu_python_run(s, t_end, dt0, dt_max, dt_min):
    t, dt, steps, cuts = 0.0, dt0, 0, 0
    while t_end - t > 1e-9 * t_end:
        h = min(dt, t_end - t)
        rc, st = s.advance(h)
        if rc in (gpu().DP_ENEWTON, gpu().DP_ELINEAR):
            cuts += 1
            dt = 0.5 * h
            if dt < dt_min:
                return rc, t, steps, cuts
            continue
        assert rc == 0
        t += h
        steps += 1
        dt = min(2.0 * h, dt_max)
    return 0, t, steps, cuts


def test_run_cuts_follow_the_rule_on_the_gpu():
    """With at most four Newton iterations per step some of Example 2's steps
    fail and are halved; sim_run reaches the same counts and the same state as
    the rule restated with sim_advance calls (the GPU path is deterministic)."""
    day = di.DAY
    res = []
    for how in ("run", "python"):
        prob = di.paper_example(2)
        s = gpu().Sim(prob, gpu().options("report", newton_max=4))
        if how == "run":
            rc, st = s.run(200 * day, 10 * day, 80 * day, 0.01 * day)
            res.append(((rc, st.t, st.steps, st.cuts), s.get_state()))
        else:
            res.append((_gpu_python_run(s, 200 * day, 10 * day, 80 * day, 0.01 * day),
                        s.get_state()))
    (ca, sa), (cb, sb) = res
    assert ca == cb and ca[0] == 0 and ca[3] > 0
    for a, b in zip(sa, sb):
        np.testing.assert_array_equal(a, b)


def test_run_matches_the_oracle_on_a_layered_example():
    """Example 1's physics on a 20x20x10 grid (Example 3's recipe at a small
    size) for 100 days: sim_run and oracle_run take the same steps (a Newton
    count may differ by one where a residual sits at the tolerance) and end in
    the same state."""
    prob = di.paper_example(1, grid=(20, 20, 10))
    g, o = pair(prob)
    args = (100 * di.DAY, 1 * di.DAY, 20 * di.DAY, 0.001 * di.DAY)
    rcg, sg = g.run(*args)
    rco, so = o.run(*args)
    assert rcg == rco == 0
    assert (sg.steps, sg.cuts) == (so.steps, so.cuts) and sg.t == so.t
    assert abs(sg.newton_iters - so.newton_iters) <= 2
    state_close(g, o, prob)
