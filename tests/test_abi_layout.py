"""The ctypes mirrors of the C ABI's structs (paper_1808_04338_gb300/dpsim.py)
and of the oracle's (oracle/__init__.py) have the layout the C compiler gives
the headers: same size, every field at the same offset.  A small C program
built with the host compiler prints sizeof and offsetof; no GPU involved."""
import ctypes as C
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "paper_1808_04338_gb300", "_build")


def _layouts(header, structs):
    """{name: (size, {field: offset})} from the C compiler."""
    lines = ["#include <stdio.h>", "#include <stddef.h>",
             f'#include "{os.path.basename(header)}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("S {name} %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'  printf("F {name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    os.makedirs(OUT, exist_ok=True)
    stem = os.path.join(OUT, "layout_" + os.path.basename(header).split(".")[0])
    with open(stem + ".c", "w") as fh:
        fh.write("\n".join(lines) + "\n")
    inc = os.path.dirname(header)
    subprocess.run(["gcc", "-I", inc, stem + ".c", "-o", stem], check=True, capture_output=True)
    out = subprocess.run([stem], check=True, capture_output=True, text=True).stdout
    res = {}
    for ln in out.splitlines():
        kind, name, *rest = ln.split()
        if kind == "S":
            res.setdefault(name, [0, {}])[0] = int(rest[0])
        else:
            res.setdefault(name, [0, {}])[1][rest[0]] = int(rest[1])
    return res


def _check(header, structs):
    got = _layouts(header, structs)
    for name, cls in structs.items():
        size, offs = got[name]
        assert C.sizeof(cls) == size, (name, C.sizeof(cls), size)
        for f in cls._fields_:
            assert getattr(cls, f[0]).offset == offs[f[0]], (name, f[0])


def test_library_structs_match_the_header():
    from paper_1808_04338_gb300 import dpsim as d
    _check(os.path.join(ROOT, "include", "dpsim.h"),
           {"dp_grid": d.dp_grid, "dp_rock": d.dp_rock, "dp_fluid": d.dp_fluid,
            "dp_well": d.dp_well, "dp_allocator": d.dp_allocator, "dp_options": d.dp_options,
            "dp_stats": d.dp_stats, "dp_run_stats": d.dp_run_stats,
            "dp_srv_result": d.dp_srv_result, "dp_srv_info": d.dp_srv_info})


def test_oracle_structs_match_its_header():
    import oracle as O
    _check(os.path.join(ROOT, "oracle", "dpsim_oracle.h"),
           {"og_grid": O.og_grid, "og_rock": O.og_rock, "og_fluid": O.og_fluid,
            "og_well": O.og_well, "og_options": O.og_options, "og_stats": O.og_stats,
            "og_run_stats": O.og_run_stats})
