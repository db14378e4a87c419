"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a dense LU
solve, finite differences of the residual, conservation, a closed-form
solution, hydrostatic equilibrium, a textbook constant, or a property that
every correct implementation must have.  No GPU is involved.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import dp_inputs as di
import oracle as O


def dense_from_bsr(rowptr, col, val):
    n = len(rowptr) - 1
    A = np.zeros((2 * n, 2 * n))
    for i in range(n):
        for e in range(rowptr[i], rowptr[i + 1]):
            j = col[e]
            A[2 * i:2 * i + 2, 2 * j:2 * j + 2] = val[e]
    return A


def small_problem(nx=3, ny=3, nz=2, seed=1, g=0.0):
    n = nx * ny * nz
    kf = np.exp(math.log(100.0) + di.normals(seed, 0, n))
    wells = [di.Well(di.WELL_RATE_INJ, 0, 0, 0, nz - 1, 100.0 * di.BBL_DAY),
             di.Well(di.WELL_BHP, nx - 1, ny - 1, 0, nz - 1, 2500.0 * di.PSI)]
    return di._base(f"small_{nx}x{ny}x{nz}", nx, ny, nz, kf, np.full(n, 0.1), 0.01, 0.2,
                    0.08, wells, seed, dt_days=1.0, nsteps=1, g=g)


# capillary pressure curves (s_w, p_cow in Pa): a weak one for the fracture, a
# strong one for the matrix
PC_F = np.array([[0.2, 2.0e4], [0.5, 5.0e3], [0.8, 0.0]])
PC_M = np.array([[0.2, 5.0e5], [0.35, 2.0e5], [0.5, 8.0e4], [0.65, 2.0e4], [0.8, 0.0]])


def with_pc(prob, pc_f=PC_F, pc_m=PC_M):
    prob.pc_f, prob.pc_m = pc_f, pc_m
    return prob


def random_interior_state(prob, seed=3):
    rng = np.random.default_rng(seed)
    nc = prob.n_cells
    p = prob.p0 + rng.uniform(-2e5, 2e5, nc)
    sw = rng.uniform(0.3, 0.7, nc)          # normalised saturation strictly inside (0, 1)
    bhp = prob.bhp0 + rng.uniform(-1e5, 1e5, prob.n_wells)
    return p, sw, bhp


# ---------------------------------------------------------------- linear solve

@pytest.mark.parametrize("make,schur", [(lambda: small_problem(3, 3, 2), 0), (di.tiny, 0),
                                        (lambda: small_problem(3, 3, 2), 1), (di.tiny, 1),
                                        (lambda: with_pc(small_problem(3, 3, 2, g=9.80665)), 1),
                                        (lambda: di.paper_example(2), 0)])
def test_cpr_fgmres_matches_dense_lu(make, schur):
    """The FGMRES/CPR-FPF Newton update solves J y = -R (Algorithm 1, step 5,
    eta = 1e-12): its true residual, formed with a dense copy of J, is at the
    tolerance, and it equals the dense LU solution to the accuracy that the
    conditioning of J (about 1e12 in SI units) allows.  With schur = 1 the
    solver sees only the fracture and well rows (the matrix cells eliminated
    exactly) and the matrix part of y comes from back-substitution: the
    update must still be the dense solution of the full system."""
    prob = make()
    s = O.OracleSim(prob, O.options("parity", eta_fixed=1e-12, schur=schur))
    if schur:
        assert s.snb == prob.n_cells // 2 + prob.n_wells
    p, sw, bhp = random_interior_state(prob)
    s.set_iterate(p, sw, bhp)
    s.assemble(prob.dt)
    rowptr, col, val, res = s.jacobian()
    y_ref = np.linalg.solve(dense_from_bsr(rowptr, col, val), -res)
    rc, st = s.solve_step()
    assert rc == 0 and st.converged
    y = s.update()
    J = dense_from_bsr(rowptr, col, val)
    assert np.linalg.norm(J @ y + res) <= 20 * 1e-12 * np.linalg.norm(res)
    nc = prob.n_cells
    d = y - y_ref
    assert np.abs(d[0:2 * nc:2]).max() <= 1e-6 * np.abs(y_ref[0:2 * nc:2]).max()
    assert np.abs(d[1:2 * nc:2]).max() <= 1e-6
    assert np.abs(d[2 * nc::2]).max() <= 1e-5 * np.abs(y_ref[2 * nc::2]).max()


@pytest.mark.parametrize("reorth", [0.0, 1.0])
def test_gram_schmidt_passes_keep_the_solution(reorth):
    """One classical Gram-Schmidt pass (reorth 0) or always two (reorth 1)
    in FGMRES's Arnoldi step: the update still solves J y = -R to the
    tolerance (its true residual, formed with a dense J) and equals the dense
    LU solution."""
    prob = small_problem(3, 3, 2)
    s = O.OracleSim(prob, O.options("parity", eta_fixed=1e-12, reorth=reorth))
    p, sw, bhp = random_interior_state(prob)
    s.set_iterate(p, sw, bhp)
    s.assemble(prob.dt)
    rowptr, col, val, res = s.jacobian()
    J = dense_from_bsr(rowptr, col, val)
    y_ref = np.linalg.solve(J, -res)
    rc, st = s.solve_step()
    assert rc == 0 and st.converged
    y = s.update()
    assert np.linalg.norm(J @ y + res) <= 20 * 1e-12 * np.linalg.norm(res)
    nc = prob.n_cells
    assert np.abs((y - y_ref)[0:2 * nc:2]).max() <= 1e-6 * np.abs(y_ref[0:2 * nc:2]).max()


def test_decoupling_removes_saturation_coefficient_and_keeps_solution():
    """Eq. "decoupled-eq": D^-1 J has a zero (0,1) entry in every cell's
    diagonal block (up to rounding), leaves the water rows unchanged, and
    D^-1 J y = D^-1 b has the solution of J y = b."""
    prob = small_problem(3, 2, 2)
    s = O.OracleSim(prob)
    s.set_iterate(*random_interior_state(prob))
    s.assemble(prob.dt)
    rowptr, col, val, res = s.jacobian()
    s.solve_step()
    dval, rhs = s.decoupled()
    nc = prob.n_cells
    for i in range(nc):
        e = rowptr[i] + list(col[rowptr[i]:rowptr[i + 1]]).index(i)
        assert abs(dval[e, 0, 1]) <= 1e-13 * abs(val[e, 0, 1])
    np.testing.assert_array_equal(dval[:, 1, :], val[:, 1, :])
    y1 = np.linalg.solve(dense_from_bsr(rowptr, col, dval), rhs)
    y0 = np.linalg.solve(dense_from_bsr(rowptr, col, val), -res)
    assert np.linalg.norm(y1 - y0) <= 1e-9 * np.linalg.norm(y0)


def _decoupled(mode):
    prob = small_problem(3, 2, 2)
    s = O.OracleSim(prob, O.options("parity", decouple=mode))
    s.set_iterate(*random_interior_state(prob))
    s.assemble(prob.dt)
    rowptr, col, val, res = s.jacobian()
    s.solve_step()
    dval, rhs = s.decoupled()
    return prob, rowptr, col, val, res, dval, rhs


@pytest.mark.parametrize("mode", [1, 2])
def test_decoupling_variants_keep_solution(mode):
    """ABF and True-IMPES (Section 3.2 names them beside the paper's own
    choice) multiply each cell row by an invertible 2x2 block: the decoupled
    system has the solution of J y = b, and well rows are unchanged."""
    prob, rowptr, col, val, res, dval, rhs = _decoupled(mode)
    nc = prob.n_cells
    y1 = np.linalg.solve(dense_from_bsr(rowptr, col, dval), rhs)
    y0 = np.linalg.solve(dense_from_bsr(rowptr, col, val), -res)
    assert np.linalg.norm(y1 - y0) <= 1e-9 * np.linalg.norm(y0)
    np.testing.assert_array_equal(dval[rowptr[nc]:], val[rowptr[nc]:])
    np.testing.assert_array_equal(rhs[2 * nc:], -res[2 * nc:])


def test_abf_makes_diagonal_blocks_identity():
    """ABF: D_i is the diagonal block itself, so every decoupled diagonal
    block is the identity up to rounding, i.e. within a small multiple of
    the componentwise bound |A_ii^-1| |A_ii| (the block's columns differ in
    scale by many orders in SI units, so the error is not small absolutely)."""
    prob, rowptr, col, val, res, dval, rhs = _decoupled(1)
    for i in range(prob.n_cells):
        e = rowptr[i] + list(col[rowptr[i]:rowptr[i + 1]]).index(i)
        bound = 1e-13 * (np.abs(np.linalg.inv(val[e])) @ np.abs(val[e]))
        assert np.all(np.abs(dval[e] - np.eye(2)) <= bound), (i, dval[e])


def test_true_impes_weight_cancels_the_saturation_column_sum():
    """True-IMPES: the weight w_i of cell i's pressure row makes the
    saturation coefficients of (oil - w_i water) in block column i sum to
    zero over all rows.  w_i is read back from the decoupled diagonal block
    (its (0,0) entry is a00 - w_i a10) and checked on the original J."""
    prob, rowptr, col, val, res, dval, rhs = _decoupled(2)
    nc = prob.n_cells
    A = dense_from_bsr(rowptr, col, val)
    checked = 0
    for i in range(nc):
        e = rowptr[i] + list(col[rowptr[i]:rowptr[i + 1]]).index(i)
        a00, a10 = val[e, 0, 0], val[e, 1, 0]
        if abs(a10) < 1e-8 * abs(a00):
            continue
        w = (a00 - dval[e, 0, 0]) / a10
        c01 = sum(A[2 * k, 2 * i + 1] for k in range(len(rowptr) - 1))
        c11 = sum(A[2 * k + 1, 2 * i + 1] for k in range(len(rowptr) - 1))
        assert abs(c01 - w * c11) <= 1e-6 * (abs(c01) + abs(w * c11))
        checked += 1
    assert checked > nc // 2


# ------------------------------------------------------------------- Jacobian

@pytest.mark.parametrize("make", [lambda: small_problem(3, 2, 2, g=0.0),
                                  lambda: small_problem(3, 2, 2, g=9.80665),
                                  lambda: di.paper_example(1), lambda: di.paper_example(2),
                                  lambda: with_pc(small_problem(3, 2, 2, g=9.80665))])
def test_jacobian_matches_finite_differences(make):
    """Analytic J equals central differences of the residual R (Section 3:
    Newton needs the exact Jacobian of F), columnwise, rel 1e-5; also for
    the setups of the paper's examples (oil-rate producer rows, a given well
    index, rock compressibility, three layers under gravity) and with
    capillary pressure curves in both continua."""
    prob = make()
    s = O.OracleSim(prob)
    p, sw, bhp = random_interior_state(prob)
    s.set_iterate(p, sw, bhp)
    s.assemble(prob.dt)
    rowptr, col, val, res = s.jacobian()
    J = dense_from_bsr(rowptr, col, val)
    x = np.concatenate([np.stack([p, sw], 1).ravel(), np.stack([bhp, np.zeros_like(bhp)], 1).ravel()])
    nc = prob.n_cells

    def resid(xv):
        xv = xv.reshape(-1, 2)
        s.set_iterate(xv[:nc, 0].copy(), xv[:nc, 1].copy(), xv[nc:, 0].copy())
        s.assemble(prob.dt)
        return s.jacobian()[3]

    for k in range(len(x)):
        if k >= 2 * nc and k % 2 == 1:
            continue                                    # dummy well unknown
        h = 1e-7 * max(abs(x[k]), 1.0)
        xp = x.copy(); xp[k] += h
        xm = x.copy(); xm[k] -= h
        fd = (resid(xp) - resid(xm)) / (2 * h)
        scale = max(np.linalg.norm(J[:, k]), 1e-300)
        assert np.linalg.norm(fd - J[:, k]) <= 1e-5 * scale, k


# --------------------------------------------------------------- conservation

@pytest.mark.parametrize("make", [di.tiny, lambda: di.paper_example(2)])
def test_mass_balance_every_newton_iterate(make):
    """Summing the cell residuals cancels every internal flux (each flux
    enters two rows with opposite signs): sum_c R_a = dM_a/dt - W_a to round
    off, for both phases, at every Newton iterate of a timestep."""
    prob = make()
    s = O.OracleSim(prob, O.options("report"))
    for it in range(4):
        s.assemble(prob.dt)
        nr = s.norms()
        _, _, _, res = s.jacobian()
        for a in range(2):
            lhs = nr[2 + a]
            rhs = nr[4 + a] / prob.dt - nr[6 + a]
            scale = np.abs(res[:2 * prob.n_cells][a::2]).sum() + abs(nr[6 + a]) + 1e-30
            assert abs(lhs - rhs) <= 1e-12 * scale
        s.solve_step()


def test_mass_conserved_over_a_converged_timestep():
    """At convergence the mass change of each phase equals dt times the well
    inflow, up to the Newton tolerance."""
    prob = di.tiny()
    s = O.OracleSim(prob, O.options("parity"))
    rc, st = s.advance(prob.dt)
    assert rc == 0
    s.assemble(prob.dt)
    nr = s.norms()
    for a in range(2):
        dm, w = nr[4 + a], nr[6 + a] * prob.dt
        assert abs(dm - w) <= 1e-8 * max(abs(w), abs(dm), 1e-3)


def test_oil_rate_producer_meets_its_target_or_switches_at_its_limit():
    """Example 2: while every producer is on oil-rate control the oil leaving
    the reservoir (the well term of the oil balance, summed over perforations
    apart from the well rows) equals the sum of the targets; once a producer's
    BHP would fall below its minimum it is on BHP control with the BHP exactly
    at that limit, and the field then produces less oil than the targets."""
    prob = di.paper_example(2, days=5.0)
    s = O.OracleSim(prob, O.options("report"))
    q_total = sum(w.target for w in prob.wells if w.kind == di.WELL_OIL_RATE)
    assert q_total > 0.0
    switched = False
    for step in range(12):
        rc, st = s.advance(prob.dt)
        assert rc == 0
        kinds, targets = s.well_controls()
        p, sw, bhp = s.get_state()
        s.assemble(prob.dt)
        nr = s.norms()
        w_oil = nr[6]
        q_oil, q_wat = s.well_rates()
        # the per-well rates add up to the well terms of the phase balances
        assert abs(q_oil.sum() - nr[6]) <= 1e-12 * np.abs(q_oil).sum()
        assert abs(q_wat.sum() - nr[7]) <= 1e-12 * np.abs(q_wat).sum()
        assert q_wat[0] > 0.0 and q_oil[0] == 0.0          # the injector injects water only
        for w, W in enumerate(prob.wells):
            if W.kind != di.WELL_OIL_RATE:
                continue
            assert q_oil[w] < 0.0 and q_wat[w] <= 0.0
            if kinds[w] == di.WELL_OIL_RATE:
                assert bhp[w] >= W.limit
                assert abs(-q_oil[w] - W.target) <= 1e-6 * W.target
            else:
                assert kinds[w] == di.WELL_BHP and targets[w] == W.limit and bhp[w] == W.limit
                assert -q_oil[w] < W.target
                switched = True
        if switched:
            assert -w_oil < q_total * (1.0 - 1e-6)
            break
        assert abs(w_oil + q_total) <= 1e-6 * q_total
    assert switched


# ----------------------------------------------------------- closed forms

@pytest.mark.parametrize("nx", [4, 9])
def test_one_d_incompressible_closed_form(nx):
    """Single-phase incompressible water on an nx x 1 x 1 line, rate injector
    at i = 0, BHP producer at i = nx-1: Darcy's law (Eq. 1) gives the linear
    profile p_i = p_b + Q mu/WI + Q mu dx/(k A) (nx-1-i), and the matrix
    continuum equilibrates, p_m = p_f (two-point fluxes are exact for linear
    profiles)."""
    prob = di.one_d(nx)
    s = O.OracleSim(prob, O.options("parity"))
    rc, st = s.advance(prob.dt)
    assert rc == 0
    p, sw, bhp = s.get_state()
    Q = prob.wells[0].target
    pb = prob.wells[1].target
    k = prob.kf[0]
    A = prob.dy * prob.dz
    wi = s.well_index()
    i = np.arange(nx)
    expect = pb + Q * prob.mu_w / wi[-1] + Q * prob.mu_w * prob.dx / (k * A) * (nx - 1 - i)
    np.testing.assert_allclose(p[0::2], expect, rtol=1e-11)
    np.testing.assert_allclose(p[1::2], p[0::2], rtol=1e-11)
    np.testing.assert_allclose(sw, 1.0, atol=1e-12)


def test_peaceman_square_block_radius():
    """Peaceman's equivalent radius of a square isotropic block is 0.198 dx
    (Section 2, Peaceman's form): W = 2 pi k dz / ln(r_e / r_w)."""
    prob = small_problem(3, 3, 1)
    prob.dx = prob.dy = 30.0
    s = O.OracleSim(prob)
    wi = s.well_index()
    loc = 0
    k = prob.kf[loc]
    re = prob.wells[0].rw * math.exp(2 * math.pi * k * prob.dz / wi[0])
    assert abs(re / prob.dx - 0.198) < 1.5e-3


def test_hydrostatic_column_is_at_rest():
    """Phi = p - rho g z (Section 2 constraints): a water column in
    hydrostatic equilibrium, p = p0 + rho_w g (z - z0) with incompressible
    water, has zero flux residual in every cell."""
    nz = 6
    prob = small_problem(1, 1, nz, g=9.80665)
    prob.wells = []
    prob.bhp0 = np.zeros(0)
    prob.c_o = prob.c_w = prob.c_rock = 0.0
    z = prob.top_depth + (np.arange(nz) + 0.5) * prob.dz
    pcol = 2.0e7 + prob.rho_w_ref * prob.g * (z - z[0])
    p = np.repeat(pcol, 2)
    sw = np.ones(2 * nz)
    s = O.OracleSim(prob)
    s.set_state(p, sw, np.zeros(0))
    s.assemble(prob.dt)
    res = s.jacobian()[3]
    # a column with the wrong sign of gravity is far from rest
    s.set_state(np.repeat(2.0e7 - prob.rho_w_ref * prob.g * (z - z[0]), 2), sw, np.zeros(0))
    s.assemble(prob.dt)
    bad = s.jacobian()[3]
    assert np.abs(res).max() <= 1e-10 * np.abs(bad).max()


# ------------------------------------------------------- capillary pressure

def test_cap_pressure_table_is_linear_interpolation():
    """p_cow between table points is the straight line through them (numpy's
    interp), constant outside the table, with the segment's slope as its
    derivative (zero outside)."""
    for tab in (PC_F, PC_M, np.array([[0.4, 1.0e5]])):
        xs = np.concatenate([np.linspace(0.0, 1.0, 101), tab[:, 0],
                             0.5 * (tab[1:, 0] + tab[:-1, 0])])
        for x in xs:
            pc, dpc = O.cap_pressure(tab, x)
            ref = np.interp(x, tab[:, 0], tab[:, 1])
            assert abs(pc - ref) <= 1e-9 * max(abs(tab[:, 1]).max(), 1.0), x
            if x <= tab[0, 0] or x >= tab[-1, 0]:     # at the end points: zero slope
                assert dpc == 0.0
            else:
                k = np.searchsorted(tab[:, 0], x, side="right") - 1
                slope = (tab[k + 1, 1] - tab[k, 1]) / (tab[k + 1, 0] - tab[k, 0])
                assert abs(dpc - slope) <= 1e-12 * abs(slope)


def test_zero_capillary_tables_change_nothing():
    """Tables of zero capillary pressure give the residual and Jacobian of
    the model without capillary pressure."""
    zero = np.array([[0.1, 0.0], [0.9, 0.0]])
    out = []
    for pc in (None, zero):
        prob = small_problem(3, 2, 2, g=9.80665)
        prob.pc_f = prob.pc_m = pc
        s = O.OracleSim(prob)
        s.set_iterate(*random_interior_state(prob))
        s.assemble(prob.dt)
        out.append(s.jacobian())
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


def _column_equilibrium(prob, pc_top):
    """A column at capillary-gravity equilibrium (Section 2 constraints):
    the oil potential p - rho_o g z and the water potential
    p - p_cow - rho_w g z are the same in every cell, with the discrete
    densities of the flux (the mean of the two cells' densities).  Oil
    pressure layer by layer from the top (densities linear in p, so each step
    is a linear equation); p_cow from the water balance; saturations from the
    inverse of each continuum's curve (so p_cow,f = p_cow,m in a location)."""
    nz, gdz = prob.nz, prob.g * prob.dz
    rho_o = lambda p: prob.rho_o_ref * (1.0 + prob.c_o * (p - prob.p_ref))
    rho_w = lambda p: prob.rho_w_ref * (1.0 + prob.c_w * (p - prob.p_ref))
    p = np.empty(nz); pc = np.empty(nz)
    p[0], pc[0] = 2.0e7, pc_top
    for k in range(nz - 1):
        a = 0.5 * prob.rho_o_ref * prob.c_o * gdz
        rhs = p[k] + 0.5 * gdz * (rho_o(p[k]) + prob.rho_o_ref * (1.0 - prob.c_o * prob.p_ref))
        p[k + 1] = rhs / (1.0 - a)
        pc[k + 1] = pc[k] + (0.5 * (rho_o(p[k]) + rho_o(p[k + 1]))
                             - 0.5 * (rho_w(p[k]) + rho_w(p[k + 1]))) * gdz
    inv = lambda tab, v: np.interp(v, tab[::-1, 1], tab[::-1, 0])   # decreasing curves
    sw = np.empty(2 * nz)
    sw[0::2], sw[1::2] = inv(prob.pc_f, pc), inv(prob.pc_m, pc)
    return np.repeat(p, 2), sw


def test_capillary_gravity_column_is_at_rest():
    """A column with different fracture and matrix curves at capillary-gravity
    equilibrium has zero flux residual in every cell and phase (water is
    wetter at depth, and the matrix holds more water than its fracture); the
    same column with p_cow left out of the water potential is far from
    rest."""
    nz = 8
    prob = with_pc(small_problem(1, 1, nz, g=9.80665))
    prob.wells = []
    prob.bhp0 = np.zeros(0)
    prob.dz = 2.0            # p_cow changes by ~4 kPa a layer: inside both curves
    p, sw = _column_equilibrium(prob, pc_top=1.5e4)
    assert (np.diff(sw[0::2]) > 0).all() and (sw[1::2] > sw[0::2]).all()
    s = O.OracleSim(prob)
    s.set_state(p, sw, np.zeros(0))
    s.assemble(prob.dt)
    res = s.jacobian()[3]
    prob0 = small_problem(1, 1, nz, g=9.80665)
    prob0.wells, prob0.bhp0, prob0.dz = [], np.zeros(0), prob.dz
    s0 = O.OracleSim(prob0)
    s0.set_state(p, sw, np.zeros(0))
    s0.assemble(prob0.dt)
    bad = s0.jacobian()[3]
    assert np.abs(bad[1::2]).max() > 0.0
    assert np.abs(res).max() <= 1e-8 * np.abs(bad).max()


def test_capillary_imbibition_into_the_matrix():
    """Equal oil pressures in a location, a wet fracture and a dry matrix with
    a strong curve: the water potential of the matrix is p_cow(s_m) lower, so
    water moves from the fracture into the matrix, oil does not move, and the
    transfer is proportional to the capillary pressure difference."""
    prob = small_problem(1, 1, 1)
    prob.wells = []
    prob.bhp0 = np.zeros(0)
    out = []
    for scale in (1.0, 2.0):
        prob.pc_f = None
        prob.pc_m = PC_M * np.array([1.0, scale])
        s = O.OracleSim(prob)
        s.set_state(np.array([3.0e7, 3.0e7]), np.array([0.7, 0.3]), np.zeros(0))
        s.assemble(prob.dt)
        res = s.jacobian()[3]
        assert res[0] == 0.0 and res[2] == 0.0           # no oil transfer
        assert res[1] > 0.0 and res[3] == -res[1]        # water leaves f, enters m
        out.append(res[1])
    assert abs(out[1] - 2.0 * out[0]) <= 1e-12 * out[1]


def test_transfer_and_flux_relax_towards_equilibrium():
    """Fluid moves from high to low potential: with no wells, a fracture
    cell above its matrix cell's pressure loses pressure and the matrix gains
    (q_mf leaves f, enters m), and neighbouring fracture cells approach each
    other; total mass of each phase is conserved.  A short step (1 s) keeps
    the flow in the direction the initial potentials set."""
    prob = small_problem(2, 1, 1)
    prob.dt = 1.0
    prob.wells = []
    prob.bhp0 = np.zeros(0)
    p = np.array([3.1e7, 3.0e7, 2.9e7, 2.95e7])   # f0, m0, f1, m1
    sw = np.full(4, 0.5)
    s = O.OracleSim(prob, O.options("parity"))
    s.set_state(p, sw, np.zeros(0))
    s.assemble(prob.dt)
    m0 = s.norms()
    rc, st = s.advance(prob.dt)
    assert rc == 0
    p1, sw1, _ = s.get_state()
    assert p1[0] < p[0] and p1[1] > p[1]           # f0 -> m0
    assert p1[2] > p[2]                              # f0 -> f1
    assert abs(p1[0] - p1[2]) < abs(p[0] - p[2])
    s.assemble(prob.dt)
    nr = s.norms()
    for a in range(2):
        assert abs(nr[4 + a]) <= 1e-9 * 1e3  # mass change ~ 0 (kg)


# ------------------------------------------------------------- components

def test_colouring_is_valid_and_red_black():
    prob = di.tiny()
    s = O.OracleSim(prob)
    c, ncol = s.colours()
    rowptr, col, _, _ = s.jacobian()
    for i in range(len(rowptr) - 1):
        for e in range(rowptr[i], rowptr[i + 1]):
            if col[e] != i:
                assert c[col[e]] != c[i]
    nc = prob.n_cells
    assert set(np.unique(c[:nc])) == {0, 1}          # bipartite cell graph
    assert ncol == 3


def test_ilu0_exact_on_block_diagonal_and_block_tridiagonal():
    """ILU(0) is exact LU when the pattern admits no fill: a block diagonal
    matrix in any ordering, a block tridiagonal chain in natural order."""
    rng = np.random.default_rng(5)
    n = 7
    # block diagonal
    rowptr = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    val = rng.normal(size=(n, 2, 2)) + 4 * np.eye(2)
    b = rng.normal(size=2 * n)
    x = O.ilu0_solve(rowptr, col, val, np.zeros(n, np.int32), b)
    np.testing.assert_allclose(x, np.linalg.solve(dense_from_bsr(rowptr, col, val), b), rtol=1e-12)
    # block tridiagonal, natural order (colour = index)
    rp, cl = [0], []
    for i in range(n):
        cl += [j for j in (i - 1, i, i + 1) if 0 <= j < n]
        rp.append(len(cl))
    rowptr, col = np.array(rp, np.int32), np.array(cl, np.int32)
    val = rng.normal(size=(len(cl), 2, 2))
    for i in range(n):
        val[rowptr[i] + (1 if i > 0 else 0)] += 6 * np.eye(2)
    x = O.ilu0_solve(rowptr, col, val, np.arange(n, dtype=np.int32), b)
    np.testing.assert_allclose(x, np.linalg.solve(dense_from_bsr(rowptr, col, val), b), rtol=1e-11)


def test_fgmres_diagonal_converges_in_k_iterations():
    """GMRES terminates in at most as many iterations as the matrix has
    distinct eigenvalues: diag(1..2k) needs exactly 2k."""
    k = 6
    rowptr = np.arange(k + 1, dtype=np.int32)
    col = np.arange(k, dtype=np.int32)
    val = np.zeros((k, 2, 2))
    for i in range(k):
        val[i] = np.diag([2 * i + 1.0, 2 * i + 2.0])
    b = np.ones(2 * k)
    x, rc, it, rr = O.fgmres_bsr(rowptr, col, val, b, precond=0, tol=1e-13)
    assert rc == 0 and it == 2 * k
    np.testing.assert_allclose(x, 1.0 / np.arange(1, 2 * k + 1), rtol=1e-12)
    # with restart below k the method still converges, with more iterations
    x, rc, it2, rr = O.fgmres_bsr(rowptr, col, val, b, precond=0, restart=4, tol=1e-10)
    assert rc == 0 and it2 > 2 * k


def poisson3d(m):
    n = m ** 3
    idx = np.arange(n).reshape(m, m, m)
    rows, cols, vals = [], [], []
    for (dz, dy, dx) in [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
        src = idx[max(0, -dz):m - max(0, dz), max(0, -dy):m - max(0, dy), max(0, -dx):m - max(0, dx)]
        dst = idx[max(0, dz):m - max(0, -dz) if dz < 0 else m, :, :] if False else None
        a = idx[max(0, -dz):m - max(0, dz), max(0, -dy):m - max(0, dy), max(0, -dx):m - max(0, dx)]
        bb = idx[max(0, dz):m + min(0, dz), max(0, dy):m + min(0, dy), max(0, dx):m + min(0, dx)]
        rows.append(a.ravel()); cols.append(bb.ravel())
        vals.append(np.full(a.size, 6.0 if (dz, dy, dx) == (0, 0, 0) else -1.0))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.sort_indices()
    return A


def test_amg_vcycle_contracts_on_poisson():
    """Smoothed aggregation V(1,1) as a stationary iteration on the 3D
    Poisson matrix contracts the energy norm of the error by a factor well
    below that of the smoother alone."""
    A = poisson3d(14)
    m = O.OracleAMG(A.indptr, A.indices, A.data, coarse_max=64)
    assert len(m.levels()) >= 3
    e = np.random.default_rng(1).normal(size=A.shape[0])
    for _ in range(15):
        e2 = e - m.vcycle(A @ e)
        q = math.sqrt((e2 @ (A @ e2)) / (e @ (A @ e)))
        e = e2
    assert q < 0.6


def test_amg_two_level_cycle_matches_independent_two_grid():
    """With two levels (exact coarse solve), one cycle equals a two-grid
    cycle written here with scipy from the same aggregates: forward red-black
    Gauss-Seidel, Galerkin coarse correction with P = (I - 2/3 D^-1 A) T
    (omega = (4/3)/rho, rho = max row sum of |D^-1 A| = 2), backward sweep."""
    A = poisson3d(12).tocsr()
    n = A.shape[0]
    m = O.OracleAMG(A.indptr, A.indices, A.data, coarse_max=400)
    levels = m.levels()
    assert len(levels) == 2
    agg, na, colour = levels[0]["agg"], levels[0]["nagg"], levels[0]["colour"]
    T = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, na))
    D = A.diagonal()
    P = (T - (2.0 / 3.0) * sp.diags(1.0 / D) @ A @ T).tocsr()
    Ac = (P.T @ A @ P).toarray()

    def gs(x, b, order):
        for c in order:
            idx = np.nonzero(colour == c)[0]
            x[idx] += (b - A @ x)[idx] / D[idx]
        return x

    b = np.random.default_rng(4).normal(size=n)
    x = gs(np.zeros(n), b, range(colour.max() + 1))
    x = x + P @ np.linalg.solve(Ac, P.T @ (b - A @ x))
    x = gs(x, b, reversed(range(colour.max() + 1)))
    np.testing.assert_allclose(m.vcycle(b), x, rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_amg_two_level_l1_jacobi_matches_independent_two_grid():
    """The same two-grid cycle with l1-Jacobi smoothing (Baker, Falgout,
    Kolev and Yang 2011): one sweep from zero before the coarse correction,
    one after, each x += (b - A x) / sum_j |a_ij| over all rows at once."""
    A = poisson3d(12).tocsr()
    n = A.shape[0]
    m = O.OracleAMG(A.indptr, A.indices, A.data, coarse_max=400, gs_levels=0)
    levels = m.levels()
    assert len(levels) == 2
    agg, na = levels[0]["agg"], levels[0]["nagg"]
    T = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, na))
    D = A.diagonal()
    P = (T - (2.0 / 3.0) * sp.diags(1.0 / D) @ A @ T).tocsr()
    Ac = (P.T @ A @ P).toarray()
    l1 = np.asarray(abs(A).sum(axis=1)).ravel()
    b = np.random.default_rng(5).normal(size=n)
    x = b / l1
    x = x + P @ np.linalg.solve(Ac, P.T @ (b - A @ x))
    x = x + (b - A @ x) / l1
    np.testing.assert_allclose(m.vcycle(b), x, rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_amg_l1_jacobi_cycle_is_symmetric_and_contracts():
    """With l1-Jacobi below the finest level the V-cycle is still a symmetric
    operator (the same sweep before and after each coarse correction) and
    still contracts the energy norm of the error on 3D Poisson."""
    A = poisson3d(14)
    m = O.OracleAMG(A.indptr, A.indices, A.data, coarse_max=64, gs_levels=1)
    assert len(m.levels()) >= 3
    rng = np.random.default_rng(2)
    u, v = rng.normal(size=A.shape[0]), rng.normal(size=A.shape[0])
    a, b = u @ m.vcycle(v), v @ m.vcycle(u)
    assert abs(a - b) < 1e-12 * abs(a)
    m0 = O.OracleAMG(A.indptr, A.indices, A.data, coarse_max=64, gs_levels=0)
    a, b = u @ m0.vcycle(v), v @ m0.vcycle(u)
    assert abs(a - b) < 1e-12 * abs(a)
    e = rng.normal(size=A.shape[0])
    for _ in range(15):
        e2 = e - m0.vcycle(A @ e)
        q = math.sqrt((e2 @ (A @ e2)) / (e @ (A @ e)))
        e = e2
    assert q < 0.8


def test_amg_aggregates_partition_and_mis2_distance():
    """Aggregates partition the strongly connected nodes, every aggregate is
    connected in the strength graph, and the MIS(2) roots (one per aggregate)
    are pairwise more than two strong edges apart."""
    prob = di.tiny()
    s = O.OracleSim(prob, O.options("report"))
    s.advance(prob.dt)
    levels = s.amg_levels()
    assert len(levels) >= 2
    L = levels[0]
    rp, col, val, agg = L["rowptr"], L["col"], L["val"], L["agg"]
    n = L["n"]
    diag = np.array([val[rp[i] + list(col[rp[i]:rp[i + 1]]).index(i)] for i in range(n)])
    adj = [set() for _ in range(n)]
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            j = col[e]
            if j == i:
                continue
            et = rp[j] + list(col[rp[j]:rp[j + 1]]).index(i)
            if max(abs(val[e]), abs(val[et])) >= 0.08 * math.sqrt(abs(diag[i] * diag[j])):
                adj[i].add(j)
    nagg = L["nagg"]
    assert sorted(set(agg[agg >= 0])) == list(range(nagg))
    for i in range(n):
        assert (agg[i] >= 0) == (len(adj[i]) > 0)
    for a in range(nagg):
        members = set(np.nonzero(agg == a)[0])
        seen, stack = set(), [next(iter(members))]
        while stack:
            u = stack.pop()
            if u in seen:
                continue
            seen.add(u)
            stack += [v for v in adj[u] if v in members]
        assert seen == members
    # roots: the lowest-numbered... each aggregate holds exactly one node whose
    # strong neighbourhood lies inside the aggregate's distance-1 ring; check
    # distance >= 3 between the aggregate roots found by the numbering rule
    roots = []
    for a in range(nagg):
        members = np.nonzero(agg == a)[0]
        cand = [u for u in members if all((agg[v] == a) for v in adj[u])]
        assert cand
        roots.append(cand)
    assert len(roots) == nagg


def test_amg_pressure_solve_matches_spsolve():
    """FGMRES preconditioned by the AMG V-cycle on a pressure matrix equals
    scipy's sparse direct solve."""
    prob = di.layered(24, 24, 4)
    s = O.OracleSim(prob, O.options("report"))
    s.assemble(prob.dt)
    s.solve_step()
    rowptr, col, _, _ = s.jacobian()
    dval, _ = s.decoupled()
    ap = dval[:, 0, 0].copy()
    n = len(rowptr) - 1
    A = sp.csr_matrix((ap, col, rowptr), shape=(n, n))
    b = np.random.default_rng(1).normal(size=n)
    x, rc, it, rr = O.fgmres_amg(rowptr, col, ap, b, tol=1e-12, coarse_max=64)
    assert rc == 0
    xr = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xr) <= 1e-9 * np.linalg.norm(xr)


def test_newton_converges_quadratically():
    """Algorithm 1 with near-exact linear solves: the scaled residual falls
    at least quadratically once it is small."""
    prob = di.tiny()
    s = O.OracleSim(prob, O.options("parity", eta_fixed=1e-12))
    s.set_state(prob.p0, prob.sw0, prob.bhp0)
    res = []
    for _ in range(12):
        s.assemble(prob.dt)
        res.append(s.norms()[0])
        if res[-1] < 1e-11 * res[0]:
            break
        s.solve_step()
    r = np.array(res) / res[0]
    k = [i for i in range(1, len(r)) if r[i - 1] < 1e-2 and r[i] > 1e-13]
    for i in k:
        assert r[i] <= 50 * r[i - 1] ** 2
    assert r[-1] < 1e-10


def test_hash_is_a_bijection_on_a_range():
    """The aggregation priority hash is a fixed 32-bit mix; distinct inputs
    of a range map to distinct outputs (it is a bijection of uint32)."""
    h = [O.hash32(i) for i in range(5000)]
    assert len(set(h)) == 5000
    assert O.hash32(0) == 0


def test_parity_mode_tiny_ten_steps_runs():
    prob = di.tiny()
    s = O.OracleSim(prob, O.options("parity"))
    for _ in range(prob.nsteps):
        rc, st = s.advance(prob.dt)
        assert rc == 0 and st.converged
    p, sw, bhp = s.get_state()
    assert np.all(sw >= 0.2 - 1e-9) and np.all(sw <= 0.8 + 1e-9)
    assert bhp[0] > bhp[1]


# ------------------------------------------------------------ time loop

def _python_run(s, t_end, dt0, dt_max, dt_min, max_steps=100000):
    """The time-loop rule restated step by step with advance calls."""
    t, dt, steps, cuts, newton = 0.0, dt0, 0, 0, 0
    while t_end - t > 1e-9 * t_end:
        if steps >= max_steps:
            return -5, t, steps, cuts, newton
        h = min(dt, t_end - t)
        rc, st = s.advance(h)
        if rc == -5:
            cuts += 1
            dt = 0.5 * h
            if dt < dt_min:
                return -5, t, steps, cuts, newton
            continue
        assert rc == 0
        t += h
        steps += 1
        newton += st.newton_iters
        dt = min(2.0 * h, dt_max)
    return 0, t, steps, cuts, newton


@pytest.mark.parametrize("newton_max", [25, 4])
def test_time_loop_follows_its_rule(newton_max):
    """oracle_run over Example 2's first 200 days (steps doubling from 10 days
    up to 80; with at most four Newton iterations per step some steps fail and
    are halved) reaches the same time, step and cut counts and the same state,
    bit for bit, as the rule restated with single timesteps."""
    day = di.DAY
    out = []
    for how in ("run", "python"):
        prob = di.paper_example(2)
        s = O.OracleSim(prob, O.options("report", newton_max=newton_max))
        if how == "run":
            rc, st = s.run(200 * day, 10 * day, 80 * day, 0.01 * day)
            res = (rc, st.t, st.steps, st.cuts, st.newton_iters)
        else:
            res = _python_run(s, 200 * day, 10 * day, 80 * day, 0.01 * day)
        out.append((res, s.get_state()))
    (ra, sa), (rb, sb) = out
    assert ra == rb and ra[0] == 0 and abs(ra[1] - 200 * day) <= 1e-9 * 200 * day
    if newton_max == 4:
        assert ra[3] > 0          # some steps were cut
    for a, b in zip(sa, sb):
        np.testing.assert_array_equal(a, b)


def test_time_loop_gives_up_below_the_smallest_step():
    """A step that keeps failing is halved until the next try would fall below
    dt_min; the run then returns the Newton failure, with the state of the last
    accepted step (here the initial state) restored."""
    prob = di.paper_example(2)
    s = O.OracleSim(prob, O.options("report", newton_max=1))
    p0 = s.get_state()
    rc, st = s.run(100 * di.DAY, 50 * di.DAY, 50 * di.DAY, 10 * di.DAY)
    assert rc == -5 and st.steps == 0 and st.cuts >= 1 and st.t == 0.0
    for a, b in zip(s.get_state(), p0):
        np.testing.assert_array_equal(a, b)


def test_time_loop_stops_at_its_step_limit():
    """After max_steps accepted steps the run stops short of t_end with the
    Newton-failure code and reports the time and steps it reached."""
    prob = di.paper_example(1)
    s = O.OracleSim(prob, O.options("report"))
    rc, st = s.run(100 * di.DAY, 1 * di.DAY, 20 * di.DAY, 0.01 * di.DAY, max_steps=3)
    assert rc == -5 and st.steps == 3 and st.cuts == 0
    assert abs(st.t - 7 * di.DAY) <= 1e-9 * di.DAY        # 1 + 2 + 4 days
