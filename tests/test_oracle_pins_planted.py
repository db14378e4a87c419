"""Pins of four oracle parts that no other test fixes, each run against the
oracle and against copies of it with a mistake planted in the source (the
pin must catch every planted mistake):

* the scaled residual norm of Algorithm 1 (cell rows times dt / (rho_ref
  phi_ref V), well rows divided by the well's target), computed here by hand
  on one location with a well of each kind;
* the three forcing terms of Section 3.1, recomputed here from the paper's
  formulas with the linear residual r = b - J y formed from the oracle's
  assembled Jacobian, residual and update;
* MIS(2) of the AMG set-up: roots pairwise more than two strong edges apart,
  every strongly connected node within two edges of a root, and the
  aggregates numbered by their roots;
* the smoothed prolongator built from the filtered operator (weak entries
  lumped into the diagonal), on an anisotropic Laplacian whose vertical
  couplings are weak, against a two-grid cycle written here with scipy.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import dp_inputs as di
import oracle as O

# ------------------------------------------------------------ planted mistakes


def _plant(src: str, func: str, old: str, new: str) -> str:
    """Replace `old` by `new` inside the body of the C function whose
    definition starts with `func` (exactly one occurrence there)."""
    a = src.index(func)
    b = src.index("\n}\n", a)
    body = src[a:b]
    assert body.count(old) == 1, (func, old)
    return src[:a] + body.replace(old, new) + src[b:]


PLANTS = {
    # scaled norm: matrix cells scaled with the fracture porosity
    "norm_phi": ("static void norms(og_sim *s)",
                 "(c % 2 == 0) ? s->phi_f[loc] : s->phi_m[loc]", "s->phi_f[loc]"),
    # scaled norm: the step length left out of the cell rows
    "norm_dt": ("static void norms(og_sim *s)",
                "double v = (s->R[2 * c + al] * s->dt) / ((rref * phi_ref) * V);",
                "double v = s->R[2 * c + al] / ((rref * phi_ref) * V);"),
    # scaled norm: well rows not divided by their target
    "norm_well": ("static void norms(og_sim *s)", "double v = s->R[row] / sc;",
                  "double v = s->R[row];"),
    # forcing term 2: ||r^{l-1}|| added instead of subtracted
    "eta2_sign": ("static double forcing(og_sim *s, double res)",
                  "eta = (res - s->lin_norms[0]) / s->prev_res",
                  "eta = (res + s->lin_norms[0]) / s->prev_res"),
    # forcing terms: ||b(x^{l-1})|| taken from the first iterate, not the previous one
    "eta_prev_iterate": ("int oracle_solve_step(void *h, og_stats *st)",
                         "s->prev_res = s->norms[0];",
                         "if (s->prev_res <= 0.0) s->prev_res = s->norms[0];"),
    # forcing term 1 in norm form instead of the norm of the vector difference
    "eta1_norm_form": ("static double forcing(og_sim *s, double res)",
                       "eta = s->lin_norms[1] / s->prev_res",
                       "eta = fabs(res - s->lin_norms[0]) / s->prev_res"),
    # forcing terms: the linear residual formed as J y - R (R's sign flipped)
    "eta_linres_sign": ("static void linear_residual(og_sim *s)",
                        "double a0 = s->R[2 * i], a1 = s->R[2 * i + 1];",
                        "double a0 = -s->R[2 * i], a1 = -s->R[2 * i + 1];"),
    # MIS(2) with one propagation pass: an MIS(1)
    "mis1": ("static void mis2(const og_csr *A, const unsigned char *s, int *state)",
             "for (int pass = 0; pass < 2; ++pass)", "for (int pass = 0; pass < 1; ++pass)"),
    # filtered operator: weak entries subtracted from the diagonal
    "lump_sign": ("static void smoothed_prolongator(", "d = d + A->val[e];", "d = d - A->val[e];"),
    # filtered operator: weak entries dropped without lumping
    "lump_none": ("static void smoothed_prolongator(", "d = d + A->val[e];", "d = d;"),
}


@pytest.fixture(scope="module")
def planted(tmp_path_factory):
    """Library path of the oracle with each planted mistake, built on demand."""
    d = tmp_path_factory.mktemp("planted")
    src = O.source()
    cache = {}

    def get(name):
        if name not in cache:
            func, old, new = PLANTS[name]
            cache[name] = O.build_variant(_plant(src, func, old, new), str(d), name)
        return cache[name]
    return get


# ------------------------------------------------------------ the scaled norm

def _one_location_three_wells():
    """One location (fracture and matrix cell) with a water-rate injector, a
    BHP well and an oil-rate producer on it; porosities 0.01 / 0.2 and
    densities 929 / 999.6 kg/m^3 differ, so every weight of the norm is
    distinct."""
    wells = [di.Well(di.WELL_RATE_INJ, 0, 0, 0, 0, 50.0 * di.BBL_DAY),
             di.Well(di.WELL_BHP, 0, 0, 0, 0, 2800.0 * di.PSI),
             di.Well(di.WELL_OIL_RATE, 0, 0, 0, 0, 0.02)]
    prob = di._base("one_location", 1, 1, 1, np.array([100.0]), np.array([0.1]), 0.01, 0.2,
                    0.08, wells, 0, dt_days=2.0)
    prob.bhp0 = np.array([3100.0, 2750.0, 2900.0]) * di.PSI   # the BHP well off its target
    return prob


def check_scaled_norm():
    prob = _one_location_three_wells()
    o = O.OracleSim(prob, O.options("report"))
    o.set_iterate(np.array([3050.0, 2990.0]) * di.PSI, np.array([0.45, 0.3]), prob.bhp0)
    dt = prob.dt
    o.assemble(dt)
    _, _, _, R = o.jacobian()
    out = o.norms()
    V = prob.dx * prob.dy * prob.dz
    phi = [prob.phi_f[0], prob.phi_m[0]]
    rho = [prob.rho_o_ref, prob.rho_w_ref]
    v = []
    for c in range(2):                      # fracture cell, matrix cell
        for al in range(2):                 # oil, water equation
            v.append(R[2 * c + al] * dt / (rho[al] * phi[c] * V))
    for w, W in enumerate(prob.wells):      # the well equations (their dummy rows are 0)
        scale = max(W.target, 1e-12) if W.kind == di.WELL_RATE_INJ else W.target
        v.append(R[2 * (2 + w)] / scale)
    v = np.array(v)
    assert np.all(v != 0.0)
    assert out[0] == pytest.approx(math.sqrt(np.sum(v * v)), rel=1e-14)
    assert out[1] == pytest.approx(np.abs(v).max(), rel=1e-14)


def test_scaled_norm_by_hand():
    check_scaled_norm()


@pytest.mark.parametrize("name", ["norm_phi", "norm_dt", "norm_well"])
def test_scaled_norm_catches_planted(planted, name):
    with O.use_library(planted(name)):
        with pytest.raises(AssertionError):
            check_scaled_norm()


# ------------------------------------------------------------ forcing terms

def _weights(prob, dt, nb):
    """Per residual row, the factor of the scaled norm (dummy rows 0)."""
    V = prob.dx * prob.dy * prob.dz
    w = np.zeros(2 * nb)
    nc = prob.n_cells
    phi = np.empty(nc)
    phi[0::2], phi[1::2] = prob.phi_f, prob.phi_m
    w[0:2 * nc:2] = dt / (prob.rho_o_ref * phi * V)
    w[1:2 * nc:2] = dt / (prob.rho_w_ref * phi * V)
    for q, W in enumerate(prob.wells):
        w[2 * (nc + q)] = 1.0 / (max(W.target, 1e-12) if W.kind == di.WELL_RATE_INJ else W.target)
    return w


def _bsr_matvec(rowptr, col, val, x):
    n = len(rowptr) - 1
    A = sp.bsr_matrix((val, col, rowptr), shape=(2 * n, 2 * n))
    return A @ x


def check_forcing(mode):
    """Run Newton iterations of one timestep; at each l >= 1 the oracle's
    eta_l equals the paper's formula evaluated here."""
    prob = di.tiny()
    gamma, beta, eta_min, eta_max = 0.9, 2.0, 1e-12, 0.5
    opts = O.options("report", eta_mode=mode, eta_gamma=gamma, eta_beta=beta,
                     eta_min=eta_min, eta_max=eta_max)
    o = O.OracleSim(prob, opts)
    o.set_state(prob.p0, prob.sw0, prob.bhp0)
    w = _weights(prob, prob.dt, o.nb)
    hist = []
    checked = 0
    for l in range(6):
        o.assemble(prob.dt)
        res = o.norms()[0]
        rowptr, col, J, R = o.jacobian()
        if l > 0 and res < 1e-12 * hist[0]["res"]:
            break
        rc, st = o.solve_step()
        assert rc == 0
        if l == 0:
            assert st.eta == eta_max
        else:
            prev = hist[-1]
            q = prev["R"] + _bsr_matvec(prev["rowptr"], prev["col"], prev["J"], prev["y"])
            if mode == 1:
                e = np.linalg.norm(w * (R - q)) / prev["res"]
                tol = 1e-10 * e
            elif mode == 2:
                nq = np.linalg.norm(w * q)
                e = (res - nq) / prev["res"]
                tol = 1e-10 * (res + nq) / prev["res"]
            else:
                e = gamma * (res / prev["res"]) ** beta
                tol = 1e-12 * e
            if eta_min < e < eta_max:
                checked += 1
            e = min(max(e, eta_min), eta_max)
            assert abs(st.eta - e) <= tol + 1e-300, (l, st.eta, e)
        hist.append(dict(res=res, R=R, J=J, rowptr=rowptr, col=col, y=o.update()))
    assert checked >= 2


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_forcing_terms_follow_section_3_1(mode):
    check_forcing(mode)


@pytest.mark.parametrize("name,mode", [("eta2_sign", 2), ("eta_prev_iterate", 2),
                                       ("eta_prev_iterate", 3), ("eta1_norm_form", 1),
                                       ("eta_linres_sign", 1), ("eta_linres_sign", 2)])
def test_forcing_terms_catch_planted(planted, name, mode):
    with O.use_library(planted(name)):
        with pytest.raises(AssertionError):
            check_forcing(mode)


# ------------------------------------------------------------ MIS(2)

def _strong_graph(A, theta):
    """Adjacency sets of the strength graph: i ~ j when
    max(|a_ij|, |a_ji|) >= theta sqrt(|a_ii a_jj|), written from the
    definition."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    d = A.diagonal()
    At = A.T.tocsr()
    adj = [set() for _ in range(n)]
    for M in (A, At):
        coo = M.tocoo()
        for i, j, v in zip(coo.row, coo.col, coo.data):
            if i != j and abs(v) >= theta * math.sqrt(abs(d[i] * d[j])):
                adj[i].add(j)
                adj[j].add(i)
    return adj


def _within2(adj, i):
    ring1 = adj[i]
    out = set(ring1)
    for j in ring1:
        out |= adj[j]
    out.discard(i)
    return out


def laplacian3d(m, eps_z=1.0, jitter=0.0, seed=0):
    """7-point Laplacian on an m^3 grid with vertical coupling eps_z; with
    jitter the off-diagonal magnitudes vary by a factor up to 1 + jitter
    (symmetric)."""
    n = m ** 3
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    idx = np.arange(n).reshape(m, m, m)          # [z, y, x]
    for axis, eps in ((2, 1.0), (1, 1.0), (0, eps_z)):
        a = np.take(idx, range(m - 1), axis=axis).ravel()
        b = np.take(idx, range(1, m), axis=axis).ravel()
        v = -eps * (1.0 + jitter * rng.random(a.size))
        rows += [a, b]
        cols += [b, a]
        vals += [v, v]
    r, c, v = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    A = sp.csr_matrix((v, (r, c)), shape=(n, n))
    A = A + sp.diags(-np.asarray(A.sum(axis=1)).ravel() + 0.01)
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A


def _tiny_pressure_block():
    prob = di.tiny()
    o = O.OracleSim(prob, O.options("report"))
    o.assemble(prob.dt)
    o.solve_step()
    rowptr, col, _, _ = o.jacobian()
    dval, _ = o.decoupled()
    n = len(rowptr) - 1
    A = sp.csr_matrix((dval[:, 0, 0].copy(), col, rowptr), shape=(n, n))
    A.sort_indices()
    return A


def check_mis2():
    theta = 0.08
    cases = [laplacian3d(9), laplacian3d(9, eps_z=0.01), laplacian3d(8, jitter=30.0, seed=3),
             _tiny_pressure_block()]
    for A in cases:
        st, nroots = O.mis2(A.indptr, A.indices, A.data, theta)
        adj = _strong_graph(A, theta)
        roots = np.nonzero(st == 2)[0]
        assert nroots == len(roots) > 1
        assert set(np.unique(st)) <= {0, 2}
        rootset = set(roots.tolist())
        for r in roots:                       # independence at distance 2
            assert not (_within2(adj, r) & rootset), r
        for i in range(A.shape[0]):           # maximality; isolated nodes stay out
            if not adj[i]:
                assert st[i] == 0
            elif st[i] != 2:
                assert _within2(adj, i) & rootset, i
        # the aggregates of the AMG set-up are numbered by these roots
        m = O.OracleAMG(A.indptr, A.indices, A.data, theta=theta, coarse_max=8)
        L0 = m.levels()[0]
        assert L0["nagg"] == nroots
        np.testing.assert_array_equal(L0["agg"][roots], np.arange(nroots))


def test_mis2_distance_and_maximality():
    check_mis2()


def test_mis2_catches_planted(planted):
    with O.use_library(planted("mis1")):
        with pytest.raises(AssertionError):
            check_mis2()


# ------------------------------------------------------------ filtered prolongator

def check_filtered_prolongator():
    """Two levels (exact coarse solve) on a Laplacian whose vertical
    couplings are weak at theta = 0.08: the oracle's cycle equals a two-grid
    cycle built here from the same aggregates with P = (I - omega D_F^-1 A_F)
    T, A_F the strong off-diagonal entries of A with every weak entry of a
    row added to its diagonal, omega = (4/3) / max_i sum_j |aF_ij| / |dF_i|,
    the Galerkin operator P^T A P of the unfiltered A, forward multicolour
    Gauss-Seidel before and backward after."""
    A = laplacian3d(10, eps_z=0.01)
    n = A.shape[0]
    theta = 0.08
    adj = _strong_graph(A, theta)
    m = O.OracleAMG(A.indptr, A.indices, A.data, theta=theta, coarse_max=400)
    levels = m.levels()
    assert len(levels) == 2
    agg, na, colour = levels[0]["agg"], levels[0]["nagg"], levels[0]["colour"]
    assert (agg >= 0).all()
    coo = A.tocoo()
    off = coo.row != coo.col
    strong = np.array([j in adj[i] for i, j in zip(coo.row, coo.col)])
    assert (off & ~strong).sum() > 0 and (off & strong).sum() > 0
    weak_sum = np.zeros(n)
    np.add.at(weak_sum, coo.row[off & ~strong], coo.data[off & ~strong])
    dF = A.diagonal() + weak_sum
    keep = off & strong
    AF = sp.csr_matrix((coo.data[keep], (coo.row[keep], coo.col[keep])), shape=(n, n)) + sp.diags(dF)
    rho = np.max(np.asarray(abs(AF).sum(axis=1)).ravel() / np.abs(dF))
    omega = (4.0 / 3.0) / rho
    T = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, na))
    P = (T - omega * sp.diags(1.0 / dF) @ AF @ T).tocsr()
    Ac = (P.T @ A @ P).toarray()
    D = A.diagonal()

    def gs(x, b, order):
        for c in order:
            idx = np.nonzero(colour == c)[0]
            x[idx] += (b - A @ x)[idx] / D[idx]
        return x

    b = np.random.default_rng(11).normal(size=n)
    x = gs(np.zeros(n), b, range(colour.max() + 1))
    x = x + P @ np.linalg.solve(Ac, P.T @ (b - A @ x))
    x = gs(x, b, reversed(range(colour.max() + 1)))
    np.testing.assert_allclose(m.vcycle(b), x, rtol=1e-10, atol=1e-12 * np.abs(x).max())


def test_filtered_prolongator_two_grid():
    check_filtered_prolongator()


@pytest.mark.parametrize("name", ["lump_sign", "lump_none"])
def test_filtered_prolongator_catches_planted(planted, name):
    with O.use_library(planted(name)):
        with pytest.raises(AssertionError):
            check_filtered_prolongator()
