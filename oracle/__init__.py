"""ctypes wrapper of the CPU FP64 oracle (``dpsim_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA library never imports or
links it, and it imports nothing from the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpsim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OG_OK, OG_EINVAL, OG_ENOMEM, OG_ELINEAR, OG_ENEWTON = 0, -1, -2, -4, -5


def _compile(src: str, out: str) -> None:
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
           "-fno-fast-math", "-fPIC", "-shared", "-I", _HERE, src, "-o", out + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(out + ".tmp", out)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, IEEE double)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "dpsim_oracle.h"))):
        _compile(_SRC, _LIB)
    return _LIB


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def build_variant(text: str, directory: str, name: str = "variant") -> str:
    """Compile a modified copy of the oracle's source (tests that plant a
    mistake and check that a pin catches it) into `directory`; returns the
    library path.  The oracle itself is not touched."""
    src = os.path.join(directory, name + ".c")
    with open(src, "w") as f:
        f.write(text)
    out = os.path.join(directory, "lib" + name + ".so")
    _compile(src, out)
    return out


class og_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("top_depth", C.c_double)]


class og_rock(C.Structure):
    _fields_ = [("kf", C.c_void_p), ("km", C.c_void_p), ("phi_f", C.c_void_p),
                ("phi_m", C.c_void_p), ("sigma", C.c_double),
                ("c_rock", C.c_double), ("p_ref", C.c_double)]


class og_fluid(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("mu_o", "mu_w", "c_o", "c_w", "rho_o_ref", "rho_w_ref", "p_ref",
                 "swc", "sor", "g")] + [("pc_n", C.c_int32 * 2), ("pc_table", C.c_void_p * 2)]


class og_well(C.Structure):
    _fields_ = [("kind", C.c_int32), ("i", C.c_int32), ("j", C.c_int32),
                ("k_top", C.c_int32), ("k_bot", C.c_int32),
                ("target", C.c_double), ("rw", C.c_double), ("skin", C.c_double),
                ("limit", C.c_double), ("wi", C.c_double)]


class og_options(C.Structure):
    _fields_ = [("newton_tol", C.c_double), ("newton_atol", C.c_double),
                ("newton_max", C.c_int32), ("eta_mode", C.c_int32),
                ("eta_fixed", C.c_double), ("eta_gamma", C.c_double),
                ("eta_beta", C.c_double), ("eta_min", C.c_double),
                ("eta_max", C.c_double), ("gmres_restart", C.c_int32),
                ("gmres_maxit", C.c_int32), ("amg_theta", C.c_double),
                ("amg_coarse_max", C.c_int32), ("amg_max_levels", C.c_int32),
                ("precond", C.c_int32), ("ds_max", C.c_double),
                ("amg_gs_levels", C.c_int32), ("amg_refresh", C.c_int32),
                ("decouple", C.c_int32), ("schur", C.c_int32), ("reorth", C.c_double)]


class og_run_stats(C.Structure):
    _fields_ = [("steps", C.c_int32), ("cuts", C.c_int32), ("newton_iters", C.c_int32),
                ("linear_iters", C.c_int32), ("t", C.c_double)]


class og_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("linear_iters", C.c_int32),
                ("converged", C.c_int32), ("amg_levels", C.c_int32),
                ("res0", C.c_double), ("res", C.c_double),
                ("lin_relres", C.c_double), ("eta", C.c_double)]


def options(mode: str = "parity", **kw) -> og_options:
    """Solver options.  'parity': fixed eta 1e-10 and Newton tolerance 1e-10
    so that two correct implementations agree far inside 1e-8.  'report':
    the second forcing term of Section 3.1 clipped to [1e-4, 0.1], Newton
    tolerance 1e-6, l1-Jacobi instead of multicolour Gauss-Seidel on the AMG
    levels below the finest, the coarse AMG values refreshed once per
    timestep, and a second Gram-Schmidt pass only after near-total
    cancellation (reorth 1e-10; parity mode 0.5)."""
    o = og_options()
    o.newton_max = 25
    o.newton_atol = 1e-13
    o.gmres_restart = 30
    o.gmres_maxit = 300
    o.amg_theta = 0.08
    o.amg_coarse_max = 128
    o.amg_max_levels = 20
    o.precond = 2
    o.ds_max = 0.2
    o.amg_gs_levels = 30
    o.reorth = 0.5
    o.eta_gamma, o.eta_beta, o.eta_min, o.eta_max = 0.9, 2.0, 1e-4, 0.1
    if mode == "parity":
        o.eta_mode, o.eta_fixed, o.newton_tol = 0, 1e-10, 1e-10
    else:
        o.eta_mode, o.eta_fixed, o.newton_tol = 2, 1e-4, 1e-6
        o.amg_gs_levels = 1
        o.amg_refresh = 1
        o.reorth = 1e-10
    for k, v in kw.items():
        setattr(o, k, v)
    return o


_lib = None
_override = None


def lib():
    """The oracle library in use: the built oracle, or a variant installed by
    ``use_library``."""
    global _lib
    if _override is not None:
        return _override
    if _lib is None:
        _lib = load_library(build())
    return _lib


class use_library:
    """Context manager: objects created inside it use the library at `path`
    (a variant from ``build_variant``)."""

    def __init__(self, path: str):
        self.L = load_library(path)

    def __enter__(self):
        global _override
        self._prev, _override = _override, self.L
        return self.L

    def __exit__(self, *exc):
        global _override
        _override = self._prev
        return False


def load_library(path: str):
    """The library at `path` with the argument types of every entry point."""
    L = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int32, C.c_double
    L.oracle_create.argtypes = [C.POINTER(og_grid), C.POINTER(og_rock), C.POINTER(og_fluid),
                                C.POINTER(og_well), I, C.POINTER(og_options), C.POINTER(P)]
    L.oracle_destroy.argtypes = [P]
    L.oracle_destroy.restype = None
    for name in ("oracle_set_state", "oracle_set_iterate", "oracle_get_state"):
        getattr(L, name).argtypes = [P, P, P, P]
    L.oracle_sizes.argtypes = [P, P, P]
    L.oracle_solver_sizes.argtypes = [P, P, P]
    L.oracle_well_controls.argtypes = [P, P, P]
    L.oracle_well_rates.argtypes = [P, P, P]
    L.oracle_cap_pressure.argtypes = [C.c_int32, P, C.c_double, P, P]
    L.oracle_cap_pressure.restype = None
    L.oracle_run.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                             C.POINTER(og_run_stats)]
    L.oracle_assemble.argtypes = [P, D]
    L.oracle_get_jacobian.argtypes = [P, P, P, P, P]
    L.oracle_get_norms.argtypes = [P, P]
    L.oracle_solve_step.argtypes = [P, C.POINTER(og_stats)]
    L.oracle_advance.argtypes = [P, D, C.POINTER(og_stats)]
    L.oracle_get_update.argtypes = [P, P]
    L.oracle_get_decoupled.argtypes = [P, P, P]
    L.oracle_get_colours.argtypes = [P, P]
    L.oracle_amg_level_info.argtypes = [P, I, P, P, P]
    L.oracle_amg_level_arrays.argtypes = [P, I, P, P, P, P, P]
    L.oracle_well_index.argtypes = [P, P]
    L.oracle_greedy_colour.argtypes = [I, P, P, P]
    L.oracle_ilu0_solve.argtypes = [I, P, P, P, P, P, P]
    L.oracle_amg_create.argtypes = [I, P, P, P, D, I, I, C.POINTER(P)]
    L.oracle_amg_vcycle.argtypes = [P, P, P]
    L.oracle_amg_set_smoother.argtypes = [P, I]
    L.oracle_amg_info.argtypes = [P, I, P, P, P]
    L.oracle_amg_arrays.argtypes = [P, I, P, P, P, P, P]
    L.oracle_amg_destroy.argtypes = [P]
    L.oracle_amg_destroy.restype = None
    L.oracle_fgmres_bsr.argtypes = [I, P, P, P, P, P, I, I, I, D, P, P]
    L.oracle_fgmres_amg.argtypes = [I, P, P, P, P, P, D, I, I, I, D, P, P]
    L.oracle_hash32.argtypes = [C.c_uint32]
    L.oracle_hash32.restype = C.c_uint32
    L.oracle_mis2.argtypes = [I, P, P, P, D, P]
    return L


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleSim:
    """One realisation in the oracle.  ``prob`` is a ``dp_inputs.Problem``."""

    def __init__(self, prob, opts: og_options | None = None):
        L = self._L = lib()
        self.prob = prob
        self.opts = opts if opts is not None else options("parity")
        g = og_grid(prob.nx, prob.ny, prob.nz, prob.dx, prob.dy, prob.dz, prob.top_depth)
        self._keep = [_f64(prob.kf), _f64(prob.km), _f64(prob.phi_f), _f64(prob.phi_m)]
        r = og_rock(*[a.ctypes.data for a in self._keep], prob.sigma, prob.c_rock,
                    prob.p_ref_rock)
        f = og_fluid(prob.mu_o, prob.mu_w, prob.c_o, prob.c_w, prob.rho_o_ref,
                     prob.rho_w_ref, prob.p_ref, prob.swc, prob.sor, prob.g)
        for k, (n, tab) in enumerate(prob.pc_tables()):
            self._keep.append(tab)
            f.pc_n[k] = n
            f.pc_table[k] = tab.ctypes.data
        nw = len(prob.wells)
        W = (og_well * max(nw, 1))()
        for q, w in enumerate(prob.wells):
            W[q] = og_well(w.kind, w.i, w.j, w.k_top, w.k_bot, w.target, w.rw, w.skin,
                           w.limit, w.wi)
        h = C.c_void_p()
        rc = L.oracle_create(C.byref(g), C.byref(r), C.byref(f), W, nw,
                             C.byref(self.opts), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle_create failed ({rc})")
        self.h = h
        nb, nnz = C.c_int32(), C.c_int32()
        L.oracle_sizes(h, C.byref(nb), C.byref(nnz))
        self.nb, self.nnzb = nb.value, nnz.value
        L.oracle_solver_sizes(h, C.byref(nb), C.byref(nnz))
        self.snb, self.snnzb = nb.value, nnz.value      # the system the solver sees
        self.nc = prob.n_cells
        self.nw = nw
        self.set_state(prob.p0, prob.sw0, prob.bhp0)

    def __del__(self):
        if getattr(self, "h", None):
            self._L.oracle_destroy(self.h)
            self.h = None

    def set_state(self, p, sw, bhp):
        p, sw, bhp = _f64(p), _f64(sw), _f64(bhp if len(bhp) else np.zeros(1))
        self._L.oracle_set_state(self.h, _p(p), _p(sw), _p(bhp))

    def set_iterate(self, p, sw, bhp):
        p, sw, bhp = _f64(p), _f64(sw), _f64(bhp if len(bhp) else np.zeros(1))
        self._L.oracle_set_iterate(self.h, _p(p), _p(sw), _p(bhp))

    def get_state(self):
        p = np.zeros(self.nc); sw = np.zeros(self.nc); bhp = np.zeros(max(self.nw, 1))
        self._L.oracle_get_state(self.h, _p(p), _p(sw), _p(bhp))
        return p, sw, bhp[:self.nw]

    def assemble(self, dt):
        rc = self._L.oracle_assemble(self.h, float(dt))
        if rc:
            raise ValueError(f"oracle_assemble failed ({rc})")

    def jacobian(self):
        rowptr = np.zeros(self.nb + 1, np.int32); col = np.zeros(self.nnzb, np.int32)
        val = np.zeros((self.nnzb, 2, 2)); res = np.zeros(2 * self.nb)
        self._L.oracle_get_jacobian(self.h, _p(rowptr), _p(col), _p(val), _p(res))
        return rowptr, col, val, res

    def norms(self):
        out = np.zeros(8)
        self._L.oracle_get_norms(self.h, _p(out))
        return out

    def solve_step(self):
        st = og_stats()
        rc = self._L.oracle_solve_step(self.h, C.byref(st))
        return rc, st

    def advance(self, dt):
        st = og_stats()
        rc = self._L.oracle_advance(self.h, float(dt), C.byref(st))
        return rc, st

    def run(self, t_end, dt0, dt_max, dt_min, max_steps=100000):
        """oracle_run: (rc, og_run_stats) of the period [0, t_end] (seconds)."""
        st = og_run_stats()
        rc = self._L.oracle_run(self.h, float(t_end), float(dt0), float(dt_max), float(dt_min),
                              int(max_steps), C.byref(st))
        return rc, st

    def update(self):
        y = np.zeros(2 * self.nb)
        self._L.oracle_get_update(self.h, _p(y))
        return y

    def decoupled(self):
        val = np.zeros((self.snnzb, 2, 2)); rhs = np.zeros(2 * self.snb)
        self._L.oracle_get_decoupled(self.h, _p(val), _p(rhs))
        return val, rhs

    def well_controls(self):
        k = np.zeros(max(self.nw, 1), np.int32); t = np.zeros(max(self.nw, 1))
        self._L.oracle_well_controls(self.h, _p(k), _p(t))
        return k[:self.nw], t[:self.nw]

    def well_rates(self):
        """Per well (oil, water) mass rates, kg/s, positive into the reservoir."""
        qo = np.zeros(max(self.nw, 1)); qw = np.zeros(max(self.nw, 1))
        self._L.oracle_well_rates(self.h, _p(qo), _p(qw))
        return qo[:self.nw], qw[:self.nw]

    def colours(self):
        c = np.zeros(self.snb, np.int32)
        ncol = self._L.oracle_get_colours(self.h, _p(c))
        return c, ncol

    def well_index(self):
        wi = np.zeros(sum(w.k_bot - w.k_top + 1 for w in self.prob.wells) + 1)
        n = self._L.oracle_well_index(self.h, _p(wi))
        return wi[:n]

    def amg_levels(self):
        """Per level: dict(n, nnz, nagg, rowptr, col, val, agg, colour)."""
        L = self._L
        out = []
        lev = 0
        while True:
            n, nnz, nagg = C.c_int32(), C.c_int32(), C.c_int32()
            nl = L.oracle_amg_level_info(self.h, lev, C.byref(n), C.byref(nnz), C.byref(nagg))
            if nl < 0:
                break
            d = dict(n=n.value, nnz=nnz.value, nagg=nagg.value,
                     rowptr=np.zeros(n.value + 1, np.int32), col=np.zeros(nnz.value, np.int32),
                     val=np.zeros(nnz.value), agg=np.zeros(n.value, np.int32),
                     colour=np.zeros(n.value, np.int32))
            L.oracle_amg_level_arrays(self.h, lev, _p(d["rowptr"]), _p(d["col"]), _p(d["val"]),
                                      _p(d["agg"]), _p(d["colour"]))
            out.append(d)
            lev += 1
            if lev >= nl:
                break
        return out


class OracleAMG:
    """Smoothed-aggregation AMG of the oracle on a scalar CSR matrix."""

    def __init__(self, rowptr, col, val, theta=0.08, coarse_max=128, max_levels=20,
                 gs_levels=30):
        self._a = (_i32(rowptr), _i32(col), _f64(val))
        self.n = len(rowptr) - 1
        self._L = lib()
        h = C.c_void_p()
        self._L.oracle_amg_create(self.n, *[_p(a) for a in self._a], float(theta),
                                int(coarse_max), int(max_levels), C.byref(h))
        self.h = h
        self._L.oracle_amg_set_smoother(self.h, int(gs_levels))

    def __del__(self):
        if getattr(self, "h", None):
            self._L.oracle_amg_destroy(self.h)
            self.h = None

    def vcycle(self, b):
        b = _f64(b); x = np.zeros(self.n)
        self._L.oracle_amg_vcycle(self.h, _p(b), _p(x))
        return x

    def levels(self):
        out = []
        lev = 0
        while True:
            n, nnz, nagg = C.c_int32(), C.c_int32(), C.c_int32()
            nl = self._L.oracle_amg_info(self.h, lev, C.byref(n), C.byref(nnz), C.byref(nagg))
            if nl < 0:
                break
            d = dict(n=n.value, nnz=nnz.value, nagg=nagg.value,
                     rowptr=np.zeros(n.value + 1, np.int32), col=np.zeros(nnz.value, np.int32),
                     val=np.zeros(nnz.value), agg=np.zeros(n.value, np.int32),
                     colour=np.zeros(n.value, np.int32))
            self._L.oracle_amg_arrays(self.h, lev, _p(d["rowptr"]), _p(d["col"]), _p(d["val"]),
                                    _p(d["agg"]), _p(d["colour"]))
            out.append(d)
            lev += 1
            if lev >= nl:
                break
        return out


def cap_pressure(table, sw):
    """p_cow(s_w) and its slope from an (n, 2) table of (s_w, p_cow) points."""
    t = np.ascontiguousarray(np.asarray(table, np.float64).reshape(-1, 2))
    pc, dpc = C.c_double(), C.c_double()
    lib().oracle_cap_pressure(t.shape[0], _p(t), float(sw), C.byref(pc), C.byref(dpc))
    return pc.value, dpc.value


def greedy_colour(rowptr, col):
    rowptr, col = _i32(rowptr), _i32(col)
    n = len(rowptr) - 1
    c = np.zeros(n, np.int32)
    ncol = lib().oracle_greedy_colour(n, _p(rowptr), _p(col), _p(c))
    return c, ncol


def ilu0_solve(rowptr, col, val, colour, b):
    rowptr, col, val, colour, b = _i32(rowptr), _i32(col), _f64(val), _i32(colour), _f64(b)
    n = len(rowptr) - 1
    x = np.zeros(2 * n)
    lib().oracle_ilu0_solve(n, _p(rowptr), _p(col), _p(val), _p(colour), _p(b), _p(x))
    return x


def fgmres_bsr(rowptr, col, val, b, precond=0, restart=30, maxit=300, tol=1e-10):
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = len(rowptr) - 1
    x = np.zeros(2 * n)
    it, rr = C.c_int32(), C.c_double()
    rc = lib().oracle_fgmres_bsr(n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), precond,
                                 restart, maxit, tol, C.byref(it), C.byref(rr))
    return x, rc, it.value, rr.value


def fgmres_amg(rowptr, col, val, b, theta=0.08, coarse_max=128, restart=30, maxit=300,
               tol=1e-10):
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    n = len(rowptr) - 1
    x = np.zeros(n)
    it, rr = C.c_int32(), C.c_double()
    rc = lib().oracle_fgmres_amg(n, _p(rowptr), _p(col), _p(val), _p(b), _p(x), theta,
                                 coarse_max, restart, maxit, tol, C.byref(it), C.byref(rr))
    return x, rc, it.value, rr.value


def hash32(i: int) -> int:
    return lib().oracle_hash32(i)


def mis2(rowptr, col, val, theta=0.08):
    """MIS(2) of the strength graph of a scalar CSR matrix: (state, roots),
    state 2 for a root and 0 otherwise."""
    rowptr, col, val = _i32(rowptr), _i32(col), _f64(val)
    n = len(rowptr) - 1
    st = np.zeros(n, np.int32)
    roots = lib().oracle_mis2(n, _p(rowptr), _p(col), _p(val), float(theta), _p(st))
    return st, roots
