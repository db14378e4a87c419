"""Every kernel of the library's solo path starts with DP_KERNEL_BEGIN.

The solo path launches its kernels with programmatic dependent launch: a
kernel may be scheduled while the previous one on the stream still runs, and
only its first instruction (griddepcontrol.wait) keeps its memory accesses
after the previous kernel's.  A kernel without it could read data the
previous kernel has not written yet, so this checks, in the sources, that the
body of every __global__ function opens with it."""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1808_04338_gb300", "csrc")
FILES = ["dp_la.cu", "dp_phys.cu", "dp_amg.cu", "dp_cycle.cu"]


def kernels(text):
    """(name, first statement of the body) of every __global__ function
    outside comments."""
    out = []
    code = re.sub(r"//[^\n]*", "", text)
    code = re.sub(r"/\*.*?\*/", "", code, flags=re.S)
    for m in re.finditer(r"__global__", code):
        brace = code.index("{", m.end())
        sig = code[m.end():brace]
        name = re.findall(r"(\w+)\s*\(", sig)
        name = [n for n in name if n != "__launch_bounds__"]
        body = code[brace + 1:brace + 200].lstrip()
        out.append((name[0] if name else "?", body.split(";")[0].strip()))
    return out


@pytest.mark.parametrize("fname", FILES)
def test_every_kernel_begins_with_the_dependency_wait(fname):
    with open(os.path.join(CSRC, fname)) as f:
        ks = kernels(f.read())
    assert ks, fname
    bad = [n for n, first in ks if first != "DP_KERNEL_BEGIN()"]
    assert not bad, (fname, bad)


def test_the_launch_macro_uses_the_checked_launcher():
    with open(os.path.join(CSRC, "dp_internal.h")) as f:
        text = f.read()
    macro = text[text.index("#define DP_LAUNCH"):text.index("while (0)", text.index("#define DP_LAUNCH"))]
    assert "launch_kernel" in macro and "<<<" not in macro
    assert "griddepcontrol.wait" in text
    # no kernel of these files is launched around the macro with <<< >>>
    for fname in FILES:
        with open(os.path.join(CSRC, fname)) as f:
            assert "<<<" not in re.sub(r"//[^\n]*", "", f.read()), fname
