"""Python binding of the dpsim C ABI (include/dpsim.h).

Argument marshalling only: every numerical step runs in the CUDA kernels of
``libdpsim.so``.  PyTorch supplies the CUDA stream and, through the
allocator callbacks, the device memory (its caching allocator).  There is no
CPU fallback: without the built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdpsim.so")

DP_OK, DP_EINVAL, DP_ENOMEM, DP_ECUDA, DP_ELINEAR, DP_ENEWTON, DP_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
WELL_RATE_INJ, WELL_BHP, WELL_OIL_RATE = 0, 1, 2


class dp_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("top_depth", C.c_double)]


class dp_rock(C.Structure):
    _fields_ = [("kf", C.c_void_p), ("km", C.c_void_p), ("phi_f", C.c_void_p),
                ("phi_m", C.c_void_p), ("sigma", C.c_double), ("c_rock", C.c_double),
                ("p_ref", C.c_double)]


class dp_fluid(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("mu_o", "mu_w", "c_o", "c_w", "rho_o_ref", "rho_w_ref", "p_ref", "swc",
                 "sor", "g")] + [("pc_n", C.c_int32 * 2), ("pc_table", C.c_void_p * 2)]


def _fluid(prob, keep):
    """dp_fluid of a Problem; its capillary tables are appended to keep."""
    f = dp_fluid(prob.mu_o, prob.mu_w, prob.c_o, prob.c_w, prob.rho_o_ref, prob.rho_w_ref,
                 prob.p_ref, prob.swc, prob.sor, prob.g)
    for k, (n, tab) in enumerate(prob.pc_tables()):
        keep.append(tab)
        f.pc_n[k] = n
        f.pc_table[k] = tab.ctypes.data
    return f


class dp_well(C.Structure):
    _fields_ = [("kind", C.c_int32), ("i", C.c_int32), ("j", C.c_int32),
                ("k_top", C.c_int32), ("k_bot", C.c_int32), ("target", C.c_double),
                ("rw", C.c_double), ("skin", C.c_double), ("limit", C.c_double),
                ("wi", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class dp_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class dp_options(C.Structure):
    _fields_ = [("newton_tol", C.c_double), ("newton_atol", C.c_double),
                ("newton_max", C.c_int32), ("eta_mode", C.c_int32),
                ("eta_fixed", C.c_double), ("eta_gamma", C.c_double),
                ("eta_beta", C.c_double), ("eta_min", C.c_double), ("eta_max", C.c_double),
                ("gmres_restart", C.c_int32), ("gmres_maxit", C.c_int32),
                ("amg_theta", C.c_double), ("amg_coarse_max", C.c_int32),
                ("amg_max_levels", C.c_int32), ("precond", C.c_int32),
                ("ds_max", C.c_double), ("precision", C.c_int32), ("use_graphs", C.c_int32),
                ("amg_gs_levels", C.c_int32), ("cluster_rows", C.c_int32),
                ("amg_refresh", C.c_int32), ("decouple", C.c_int32), ("schur", C.c_int32),
                ("reorth", C.c_double)]


class dp_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("linear_iters", C.c_int32),
                ("converged", C.c_int32), ("amg_levels", C.c_int32), ("res0", C.c_double),
                ("res", C.c_double), ("lin_relres", C.c_double), ("eta", C.c_double),
                ("ms_setup", C.c_double), ("ms_solve", C.c_double)]


def options(mode: str = "parity", **kw) -> dp_options:
    """'parity': fixed eta 1e-10, Newton tolerance 1e-10 (agreement with an
    independent FP64 evaluation far inside 1e-8); 'report': the second
    forcing term of Section 3.1 clipped to [1e-4, 0.1], Newton tolerance
    1e-6, l1-Jacobi instead of multicolour Gauss-Seidel on the AMG levels
    below the finest, the coarse AMG values refreshed once per timestep, and a
    second Gram-Schmidt pass only after near-total cancellation (reorth 1e-10;
    parity mode: 0.5)."""
    o = dp_options()
    o.newton_max = 25
    o.newton_atol = 1e-13
    o.gmres_restart = 30
    o.gmres_maxit = 300
    o.amg_theta = 0.08
    o.amg_coarse_max = 128
    o.amg_max_levels = 20
    o.precond = 2
    o.ds_max = 0.2
    o.precision = 0
    o.use_graphs = 1
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


def load():
    """Load libdpsim.so (built by ``paper_1808_04338_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    L = C.CDLL(LIB_PATH)
    P, I, D = C.c_void_p, C.c_int32, C.c_double
    L.sim_create.argtypes = [C.POINTER(dp_grid), C.POINTER(dp_rock), C.POINTER(dp_fluid),
                             C.POINTER(dp_well), I, C.POINTER(dp_options),
                             C.POINTER(dp_allocator), P, C.POINTER(P)]
    L.sim_destroy.argtypes = [P]
    L.sim_destroy.restype = None
    L.sim_sizes.argtypes = [P, P, P, P, P]
    for n in ("sim_set_state", "sim_set_iterate", "sim_set_state_device", "sim_get_state"):
        getattr(L, n).argtypes = [P, P, P, P]
    L.sim_assemble.argtypes = [P, D]
    L.sim_get_jacobian.argtypes = [P, P, P, P, P]
    L.sim_get_norms.argtypes = [P, P]
    L.sim_solve_step.argtypes = [P, C.POINTER(dp_stats)]
    L.sim_advance.argtypes = [P, D, C.POINTER(dp_stats)]
    L.sim_run.argtypes = [P, D, D, D, D, I, C.POINTER(dp_run_stats)]
    L.sim_get_update.argtypes = [P, P]
    L.sim_get_decoupled.argtypes = [P, P, P]
    L.sim_get_colours.argtypes = [P, P]
    L.sim_well_index.argtypes = [P, P]
    L.sim_well_controls.argtypes = [P, P, P]
    L.sim_well_rates.argtypes = [P, P, P]
    L.sim_amg_level_info.argtypes = [P, I, P, P, P]
    L.sim_amg_level_arrays.argtypes = [P, I, P, P, P, P, P]
    L.sim_amg_transfer_info.argtypes = [P, I, P, P]
    L.sim_time_kernel.argtypes = [P, C.c_char_p]
    L.sim_kernel_timing.argtypes = [P, P, P, I]
    L.sim_launch_count.argtypes = [P]
    L.sim_launch_count.restype = C.c_int64
    L.sim_last_error.argtypes = [P]
    L.sim_last_error.restype = C.c_char_p
    L.sim_advance_many.argtypes = [P, I, P, I, P, P]
    L.sim_footprint.argtypes = [P, P, P]
    L.sim_autotune.argtypes = [P, I, C.c_char_p, I]
    L.sim_set_l0_kernel.argtypes = [P, I]
    L.sim_solver_sizes.argtypes = [P, P, P]
    L.dp_stream_create.argtypes = [P]
    L.dp_stream_destroy.argtypes = [P]
    L.srv_create.argtypes = [I, C.c_uint64, P, P]
    L.srv_add.argtypes = [P, P, P, P, P, I, P, P, P, P]
    L.srv_submit.argtypes = [P, I, C.c_double, P]
    L.srv_wait.argtypes = [P, C.c_int64, P]
    L.srv_get_state.argtypes = [P, I, P, P, P]
    L.srv_info.argtypes = [P, P]
    L.srv_destroy.argtypes = [P]
    L.batch_create.argtypes = [P, I, P, P]
    L.batch_advance.argtypes = [P, P, P, P]
    L.batch_destroy.argtypes = [P]
    L.batch_destroy.restype = None
    L.batch_last_error.argtypes = [P]
    L.batch_last_error.restype = C.c_char_p
    L.batch_launch_count.argtypes = [P]
    L.batch_launch_count.restype = C.c_int64
    L.batch_profile.argtypes = [P, P, P]
    L.dp_residual_norms_noalloc.argtypes = [C.POINTER(dp_grid), C.POINTER(dp_fluid), P, P, I, P,
                                            P, P, D, P, P, C.c_char_p, C.c_size_t]
    _lib = L
    return L


def _p(a):
    return C.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def residual_norms_noalloc(prob, phi_f, phi_m, well_kind, well_target, res, dt, out2,
                           stream=0):
    """Scaled residual 2-norm and max-norm into out2 (device tensors in, no
    allocation by the library); returns (rc, message)."""
    g = dp_grid(prob.nx, prob.ny, prob.nz, prob.dx, prob.dy, prob.dz, prob.top_depth)
    keep = []
    f = _fluid(prob, keep)
    buf = C.create_string_buffer(256)

    def ptr(t):
        return C.c_void_p(t.data_ptr()) if t is not None else None

    rc = load().dp_residual_norms_noalloc(C.byref(g), C.byref(f), ptr(phi_f), ptr(phi_m),
                                          len(prob.wells), ptr(well_kind), ptr(well_target),
                                          ptr(res), float(dt), ptr(out2), C.c_void_p(stream),
                                          buf, 256)
    return rc, buf.value.decode()


class OwnedStream:
    """A distinct non-blocking stream made by the library (torch's pool
    hands out at most 32 distinct streams); ``.torch`` wraps it for torch."""

    def __init__(self):
        import torch
        h = C.c_void_p()
        rc = load().dp_stream_create(C.byref(h))
        if rc != 0:
            raise RuntimeError(f"dp_stream_create failed ({rc})")
        self.h = h
        self.torch = torch.cuda.ExternalStream(h.value)

    def close(self):
        if getattr(self, "h", None):
            import torch
            torch.cuda.synchronize()
            load().dp_stream_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def advance_many(sims, dts, threads=0):
    """One timestep of every realisation in `sims` (each with its own stream),
    concurrently; returns (rc, stats list, status list)."""
    n = len(sims)
    H = (C.c_void_p * max(n, 1))(*[s.h.value for s in sims])
    D = (C.c_double * max(n, 1))(*[float(d) for d in dts])
    st = (dp_stats * max(n, 1))()
    rs = (C.c_int32 * max(n, 1))()
    rc = load().sim_advance_many(C.cast(H, C.c_void_p), n, C.cast(D, C.c_void_p), int(threads),
                                 C.cast(st, C.c_void_p), C.cast(rs, C.c_void_p))
    return rc, [st[k] for k in range(n)], [rs[k] for k in range(n)]


class Batch:
    """Realisations advanced in lockstep by one batched engine (batch_* in
    include/dpsim.h): one launch per phase of each FGMRES iteration over all
    of them.  The realisations must outlive the batch."""

    def __init__(self, sims, stream=None):
        import torch
        self.sims = list(sims)
        n = len(self.sims)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        H = (C.c_void_p * max(n, 1))(*[s.h.value for s in self.sims])
        h = C.c_void_p()
        rc = load().batch_create(C.cast(H, C.c_void_p), n, C.c_void_p(self.stream.cuda_stream),
                                 C.byref(h))
        if rc != 0:
            raise RuntimeError(f"batch_create failed ({rc})")
        self.h = h
        for s in self.sims:        # a member closed first closes the batch first
            s._batches.append(self)

    def advance(self, dts):
        """One timestep of every realisation; returns (rc, stats, status)."""
        n = len(self.sims)
        D = (C.c_double * max(n, 1))(*[float(d) for d in dts])
        st = (dp_stats * max(n, 1))()
        rs = (C.c_int32 * max(n, 1))()
        rc = load().batch_advance(self.h, C.cast(D, C.c_void_p), C.cast(st, C.c_void_p),
                                  C.cast(rs, C.c_void_p))
        if rc < 0 and rc not in (DP_ENEWTON, DP_ELINEAR):
            msg = load().batch_last_error(self.h)
            raise RuntimeError(f"batch_advance failed ({rc}): {msg.decode() if msg else ''}")
        return rc, [st[k] for k in range(n)], [rs[k] for k in range(n)]

    def launch_count(self):
        return load().batch_launch_count(self.h)

    def profile(self):
        """(ms of set-up, batched FGMRES, updates; Newton rounds, cycles, Arnoldi steps)"""
        ms = (C.c_double * 3)()
        n = (C.c_int64 * 3)()
        load().batch_profile(self.h, C.cast(ms, C.c_void_p), C.cast(n, C.c_void_p))
        return list(ms), list(n)

    def close(self):
        if getattr(self, "h", None):
            load().batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class dp_run_stats(C.Structure):
    _fields_ = [("steps", C.c_int32), ("cuts", C.c_int32), ("newton_iters", C.c_int32),
                ("linear_iters", C.c_int32), ("t", C.c_double)]


class dp_srv_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("realisation", C.c_int32), ("loaded", C.c_int32),
                ("evicted", C.c_int32), ("t_submit_ms", C.c_double), ("t_start_ms", C.c_double),
                ("t_done_ms", C.c_double), ("stats", dp_stats)]


class dp_srv_info(C.Structure):
    _fields_ = [("registered", C.c_int32), ("resident", C.c_int32), ("queued", C.c_int32),
                ("running", C.c_int32), ("served", C.c_int64), ("loads", C.c_int64),
                ("evictions", C.c_int64), ("launches", C.c_int64), ("resident_bytes", C.c_uint64),
                ("peak_resident_bytes", C.c_uint64), ("budget_bytes", C.c_uint64),
                ("bytes_per_row", C.c_double)]


def _inputs(prob):
    """ctypes views of a Problem's grid, rock, fluid and wells (the arrays
    they point to are returned too and must outlive the call)."""
    g = dp_grid(prob.nx, prob.ny, prob.nz, prob.dx, prob.dy, prob.dz, prob.top_depth)
    keep = [_f64(prob.kf), _f64(prob.km), _f64(prob.phi_f), _f64(prob.phi_m)]
    r = dp_rock(*[a.ctypes.data for a in keep], prob.sigma, prob.c_rock, prob.p_ref_rock)
    f = _fluid(prob, keep)
    nw = len(prob.wells)
    W = (dp_well * max(nw, 1))()
    for q, w in enumerate(prob.wells):
        W[q] = dp_well(w.kind, w.i, w.j, w.k_top, w.k_bot, w.target, w.rw, w.skin, w.limit,
                       w.wi)
    return g, r, f, W, nw, keep


class Server:
    """Request server over resident realisations (srv_* in include/dpsim.h)."""

    def __init__(self, workers: int, hbm_budget: int, opts: dp_options | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("dpsim needs a CUDA device")
        self.opts = opts if opts is not None else options("report")
        h = C.c_void_p()
        rc = load().srv_create(int(workers), int(hbm_budget), C.byref(self.opts), C.byref(h))
        if rc != 0:
            raise RuntimeError(f"srv_create failed ({rc})")
        self.h = h
        self.sizes = []

    def add(self, prob) -> int:
        g, r, f, W, nw, keep = _inputs(prob)
        p, sw = _f64(prob.p0), _f64(prob.sw0)
        bhp = _f64(prob.bhp0 if len(prob.bhp0) else np.zeros(1))
        rid = C.c_int32()
        rc = load().srv_add(self.h, C.byref(g), C.byref(r), C.byref(f), W, nw, _p(p), _p(sw),
                            _p(bhp), C.byref(rid))
        if rc != 0:
            raise RuntimeError(f"srv_add failed ({rc})")
        self.sizes.append((prob.n_cells, nw))
        return rid.value

    def submit(self, rid: int, dt: float) -> int:
        t = C.c_int64()
        rc = load().srv_submit(self.h, int(rid), float(dt), C.byref(t))
        if rc != 0:
            raise RuntimeError(f"srv_submit failed ({rc})")
        return t.value

    def wait(self, ticket: int) -> dp_srv_result:
        out = dp_srv_result()
        rc = load().srv_wait(self.h, int(ticket), C.byref(out))
        if rc != 0:
            raise RuntimeError(f"srv_wait failed ({rc})")
        return out

    def state(self, rid: int):
        nc, nw = self.sizes[rid]
        p = np.zeros(nc); sw = np.zeros(nc); bhp = np.zeros(max(nw, 1))
        rc = load().srv_get_state(self.h, int(rid), _p(p), _p(sw), _p(bhp))
        if rc != 0:
            raise RuntimeError(f"srv_get_state failed ({rc})")
        return p, sw, bhp[:nw]

    def info(self) -> dp_srv_info:
        out = dp_srv_info()
        load().srv_info(self.h, C.byref(out))
        return out

    def close(self):
        if getattr(self, "h", None):
            load().srv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TorchAllocator:
    """dp_allocator backed by PyTorch's CUDA caching allocator."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream)
            except Exception:
                return None

        def _free(ptr, nbytes, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = dp_allocator(self._a, self._f, None)


class Sim:
    """One realisation on the GPU.  ``prob`` is a ``dp_inputs.Problem``."""

    def __init__(self, prob, opts: dp_options | None = None, stream=None, use_torch_alloc=True,
                 allocator=None):
        """allocator: an object with a ``struct`` dp_allocator (default: torch's
        caching allocator; None with use_torch_alloc False: the library's own).
        A failed sim_create raises RuntimeError with the code in ``self.create_rc``."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("dpsim needs a CUDA device")
        L = load()
        self.prob = prob
        self.opts = opts if opts is not None else options("parity")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g, r, f, W, nw, keep = _inputs(prob)
        if allocator is not None:
            self._alloc = allocator
        else:
            self._alloc = TorchAllocator(torch.cuda.current_device()) if use_torch_alloc else None
        self._batches = []
        h = C.c_void_p()
        rc = L.sim_create(C.byref(g), C.byref(r), C.byref(f), W, nw, C.byref(self.opts),
                          C.byref(self._alloc.struct) if self._alloc else None,
                          C.c_void_p(self.stream.cuda_stream), C.byref(h))
        self.create_rc = rc
        if rc != 0:
            raise RuntimeError(f"sim_create failed ({rc})")
        self.h = h
        nb, nnz, nc, nwl = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        L.sim_sizes(h, C.byref(nb), C.byref(nnz), C.byref(nc), C.byref(nwl))
        self.nb, self.nnzb, self.nc, self.nw = nb.value, nnz.value, nc.value, nwl.value
        L.sim_solver_sizes(h, C.byref(nb), C.byref(nnz))
        self.snb, self.snnzb = nb.value, nnz.value     # the system the solver sees
        if prob.p0 is not None:
            self.set_state(prob.p0, prob.sw0, prob.bhp0)

    def close(self):
        if getattr(self, "h", None):
            for b in getattr(self, "_batches", []):
                b.close()
            load().sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc < 0:
            msg = load().sim_last_error(self.h)
            raise RuntimeError(f"{what} failed ({rc}): {msg.decode() if msg else ''}")
        return rc

    def set_state(self, p, sw, bhp):
        p, sw, bhp = _f64(p), _f64(sw), _f64(bhp if len(bhp) else np.zeros(1))
        self._check(load().sim_set_state(self.h, _p(p), _p(sw), _p(bhp)), "sim_set_state")

    def set_state_device(self, p, sw, bhp):
        """Device tensors (float64, on this GPU)."""
        self._check(load().sim_set_state_device(self.h, C.c_void_p(p.data_ptr()),
                                                C.c_void_p(sw.data_ptr()),
                                                C.c_void_p(bhp.data_ptr())), "sim_set_state_device")

    def set_state_ptr(self, p, sw, bhp):
        """Raw pointers (host pinned or device), stream-ordered copy."""
        self._check(load().sim_set_state(self.h, C.c_void_p(p), C.c_void_p(sw), C.c_void_p(bhp)),
                    "sim_set_state")

    def set_iterate(self, p, sw, bhp):
        p, sw, bhp = _f64(p), _f64(sw), _f64(bhp if len(bhp) else np.zeros(1))
        self._check(load().sim_set_iterate(self.h, _p(p), _p(sw), _p(bhp)), "sim_set_iterate")

    def get_state(self):
        p = np.zeros(self.nc); sw = np.zeros(self.nc); bhp = np.zeros(max(self.nw, 1))
        self._check(load().sim_get_state(self.h, _p(p), _p(sw), _p(bhp)), "sim_get_state")
        return p, sw, bhp[:self.nw]

    def get_state_ptr(self, p, sw, bhp):
        self._check(load().sim_get_state(self.h, C.c_void_p(p), C.c_void_p(sw), C.c_void_p(bhp)),
                    "sim_get_state")

    def assemble(self, dt):
        self._check(load().sim_assemble(self.h, float(dt)), "sim_assemble")

    def jacobian(self):
        rowptr = np.zeros(self.nb + 1, np.int32); col = np.zeros(self.nnzb, np.int32)
        val = np.zeros((self.nnzb, 2, 2)); res = np.zeros(2 * self.nb)
        self._check(load().sim_get_jacobian(self.h, _p(rowptr), _p(col), _p(val), _p(res)),
                    "sim_get_jacobian")
        return rowptr, col, val, res

    def norms(self):
        out = np.zeros(8)
        self._check(load().sim_get_norms(self.h, _p(out)), "sim_get_norms")
        return out

    def solve_step(self):
        st = dp_stats()
        rc = load().sim_solve_step(self.h, C.byref(st))
        if rc < 0 and rc != DP_ELINEAR:
            self._check(rc, "sim_solve_step")
        return rc, st

    def advance(self, dt):
        st = dp_stats()
        rc = load().sim_advance(self.h, float(dt), C.byref(st))
        if rc < 0 and rc not in (DP_ENEWTON, DP_ELINEAR):
            self._check(rc, "sim_advance")
        return rc, st

    def run(self, t_end, dt0, dt_max, dt_min, max_steps=100000):
        """sim_run: (rc, dp_run_stats) of the period [0, t_end] (seconds)."""
        st = dp_run_stats()
        rc = load().sim_run(self.h, float(t_end), float(dt0), float(dt_max), float(dt_min),
                            int(max_steps), C.byref(st))
        if rc < 0 and rc != DP_ENEWTON:
            self._check(rc, "sim_run")
        return rc, st

    def update(self):
        y = np.zeros(2 * self.nb)
        self._check(load().sim_get_update(self.h, _p(y)), "sim_get_update")
        return y

    def decoupled(self):
        val = np.zeros((self.snnzb, 2, 2)); rhs = np.zeros(2 * self.snb)
        self._check(load().sim_get_decoupled(self.h, _p(val), _p(rhs)), "sim_get_decoupled")
        return val, rhs

    def colours(self):
        c = np.zeros(self.snb, np.int32)
        n = self._check(load().sim_get_colours(self.h, _p(c)), "sim_get_colours")
        return c, n

    def set_l0_kernel(self, variant: int):
        """The kernel of level 0's Gauss-Seidel colours and residual (1: a
        thread per row, 0: rows staged in shared memory, -1/-2/-3: the
        pipelined bulk-copy kernels, 2/4/8: lanes per row)."""
        self._check(load().sim_set_l0_kernel(self.h, int(variant)), "sim_set_l0_kernel")

    def autotune(self, reps: int = 20) -> str:
        """Time the AMG level kernels' launch shapes and keep the fastest;
        returns the decisions as text."""
        buf = C.create_string_buffer(16384)
        self._check(load().sim_autotune(self.h, int(reps), buf, len(buf)), "sim_autotune")
        return buf.value.decode()

    def footprint(self):
        cur, peak = C.c_uint64(), C.c_uint64()
        self._check(load().sim_footprint(self.h, C.byref(cur), C.byref(peak)), "sim_footprint")
        return cur.value, peak.value

    def well_index(self):
        wi = np.zeros(sum(w.k_bot - w.k_top + 1 for w in self.prob.wells) + 1)
        n = self._check(load().sim_well_index(self.h, _p(wi)), "sim_well_index")
        return wi[:n]

    def well_controls(self):
        """The wells' current (kind, target), as sim_well_controls."""
        k = np.zeros(max(self.nw, 1), np.int32); t = np.zeros(max(self.nw, 1))
        self._check(load().sim_well_controls(self.h, _p(k), _p(t)), "sim_well_controls")
        return k[:self.nw], t[:self.nw]

    def well_rates(self):
        """Per well (oil, water) mass rates, kg/s, positive into the reservoir
        (sim_well_rates)."""
        qo = np.zeros(max(self.nw, 1)); qw = np.zeros(max(self.nw, 1))
        self._check(load().sim_well_rates(self.h, _p(qo), _p(qw)), "sim_well_rates")
        return qo[:self.nw], qw[:self.nw]

    def amg_levels(self):
        L = load()
        out = []
        lev = 0
        while True:
            n, nnz, nagg = C.c_int32(), C.c_int32(), C.c_int32()
            nl = L.sim_amg_level_info(self.h, lev, C.byref(n), C.byref(nnz), C.byref(nagg))
            if nl < 0:
                break
            d = dict(n=n.value, nnz=nnz.value, nagg=nagg.value,
                     rowptr=np.zeros(n.value + 1, np.int32), col=np.zeros(nnz.value, np.int32),
                     val=np.zeros(nnz.value), agg=np.zeros(n.value, np.int32),
                     colour=np.zeros(n.value, np.int32))
            self._check(L.sim_amg_level_arrays(self.h, lev, _p(d["rowptr"]), _p(d["col"]),
                                               _p(d["val"]), _p(d["agg"]), _p(d["colour"])),
                        "sim_amg_level_arrays")
            out.append(d)
            lev += 1
            if lev >= nl:
                break
        return out

    def amg_level_sizes(self):
        """Per AMG level: dict(n, nnz, nagg, p_nnz, smoother) without the
        arrays (sim_amg_level_info, sim_amg_transfer_info; smoother 0
        Gauss-Seidel, 1 l1-Jacobi, 2 direct solve)."""
        L = load()
        out = []
        lev = 0
        while True:
            n, nnz, nagg = C.c_int32(), C.c_int32(), C.c_int32()
            pn, sm = C.c_int32(), C.c_int32()
            nl = L.sim_amg_level_info(self.h, lev, C.byref(n), C.byref(nnz), C.byref(nagg))
            if nl < 0:
                break
            self._check(L.sim_amg_transfer_info(self.h, lev, C.byref(pn), C.byref(sm)),
                        "sim_amg_transfer_info")
            out.append(dict(n=n.value, nnz=nnz.value, nagg=nagg.value, p_nnz=pn.value,
                            smoother=sm.value))
            lev += 1
            if lev >= nl:
                break
        return out

    def time_kernel(self, name: str | None):
        self._check(load().sim_time_kernel(self.h, name.encode() if name else None),
                    "sim_time_kernel")

    def kernel_timing(self, reset=True):
        ms, n = C.c_double(), C.c_int64()
        self._check(load().sim_kernel_timing(self.h, C.byref(ms), C.byref(n), int(reset)),
                    "sim_kernel_timing")
        return ms.value, n.value

    def launch_count(self):
        return load().sim_launch_count(self.h)
