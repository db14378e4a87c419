"""The C ABI library builds, loads without a GPU and exports every entry
point that include/*.h declares; the binding declares each of them."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(sim_\w+|dp_\w+|srv_\w+|batch_\w+)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1808_04338_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared()
    for n in ("sim_create", "sim_assemble", "sim_solve_step", "sim_advance", "sim_set_state",
              "sim_get_state", "sim_get_jacobian", "sim_destroy", "sim_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in sorted(declared()):
        assert hasattr(lib, n), n


def test_binding_declares_every_symbol(lib):
    from paper_1808_04338_gb300 import dpsim
    L = dpsim.load()
    for n in sorted(declared()):
        assert getattr(L, n).argtypes is not None, n


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    """Argument checks happen before any CUDA call."""
    from paper_1808_04338_gb300 import dpsim
    L = dpsim.load()
    out = ctypes.c_void_p()
    assert L.sim_create(None, None, None, None, 0, None, None, None, ctypes.byref(out)) == dpsim.DP_EINVAL
    g = dpsim.dp_grid(0, 1, 1, 1.0, 1.0, 1.0, 0.0)
    o = dpsim.options()
    assert L.sim_create(ctypes.byref(g), None, None, None, 0, ctypes.byref(o), None, None,
                        ctypes.byref(out)) == dpsim.DP_EINVAL
    assert L.sim_assemble(None, 1.0) == dpsim.DP_EINVAL
    assert L.sim_solve_step(None, None) == dpsim.DP_EINVAL
    srv = ctypes.c_void_p()
    assert L.srv_create(0, 1 << 30, ctypes.byref(o), ctypes.byref(srv)) == dpsim.DP_EINVAL
    assert L.srv_create(2, 0, ctypes.byref(o), ctypes.byref(srv)) == dpsim.DP_EINVAL
    assert L.srv_submit(None, 0, 1.0, None) == dpsim.DP_EINVAL
    assert L.sim_advance_many(None, 2, None, 0, None, None) == dpsim.DP_EINVAL
    assert L.sim_well_controls(None, None, None) == dpsim.DP_EINVAL
    assert L.sim_well_rates(None, None, None) == dpsim.DP_EINVAL
    assert L.sim_run(None, 1.0, 1.0, 1.0, 0.1, 10, None) == dpsim.DP_EINVAL
    assert L.sim_autotune(None, 1, None, 0) == dpsim.DP_EINVAL
    assert L.sim_set_l0_kernel(None, 1) == dpsim.DP_EINVAL
    assert L.sim_amg_level_info(None, 0, None, None, None) == dpsim.DP_EINVAL
    assert L.sim_amg_transfer_info(None, 0, None, None) == dpsim.DP_EINVAL
    assert L.sim_time_kernel(None, b"sweep.gs") == dpsim.DP_EINVAL
    bat = ctypes.c_void_p()
    assert L.batch_create(None, 0, None, ctypes.byref(bat)) == dpsim.DP_EINVAL
    assert L.batch_advance(None, None, None, None) == dpsim.DP_EINVAL
    # wells: unknown control kind, negative limit, negative well index
    import dataclasses
    import dp_inputs as di
    prob = di.paper_example(2)
    for bad in (dict(kind=3), dict(limit=-1.0), dict(wi=-1.0), dict(limit=float("nan"))):
        wells = [dataclasses.replace(prob.wells[0], **bad)] + list(prob.wells[1:])
        g, r, f, W, nw, keep = dpsim._inputs(dataclasses.replace(prob, wells=wells))
        assert L.sim_create(ctypes.byref(g), ctypes.byref(r), ctypes.byref(f), W, nw,
                            ctypes.byref(o), None, None, ctypes.byref(out)) == dpsim.DP_EINVAL, bad
    # capillary tables: s_w not strictly ascending, a NaN, too many points, no array
    import numpy as np
    for tab in (np.array([[0.2, 1e5], [0.2, 0.0]]), np.array([[0.2, np.nan], [0.5, 0.0]]),
                np.column_stack([np.linspace(0, 1, 257), np.zeros(257)])):
        g, r, f, W, nw, keep = dpsim._inputs(dataclasses.replace(prob, pc_m=tab))
        assert L.sim_create(ctypes.byref(g), ctypes.byref(r), ctypes.byref(f), W, nw,
                            ctypes.byref(o), None, None, ctypes.byref(out)) == dpsim.DP_EINVAL
    g, r, f, W, nw, keep = dpsim._inputs(prob)
    f.pc_n[0] = 3
    assert L.sim_create(ctypes.byref(g), ctypes.byref(r), ctypes.byref(f), W, nw,
                        ctypes.byref(o), None, None, ctypes.byref(out)) == dpsim.DP_EINVAL


def test_oracle_is_not_linked_into_the_library(lib):
    from paper_1808_04338_gb300 import build
    import subprocess
    out = subprocess.run(["nm", "-D", build.LIB], capture_output=True, text=True).stdout
    assert "oracle_" not in out
