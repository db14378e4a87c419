"""A kernel launched as a programmatic dependent (DP_LAUNCH_PDL) may start
while the kernel before it is still running, so it must execute
griddep_wait() before it reads anything that kernel writes.  This checks the
sources: every kernel launched that way calls griddep_wait, in its own body
or in a device function its body calls, and writes through no pointer before
that call (no store precedes the wait in the kernel's own body)."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1808_04338_gb300", "csrc")


def sources():
    text = ""
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name)) as f:
                text += f.read() + "\n"
    return text


def body_of(text, name, kind):
    """The body of the first `kind` (__global__ or __device__) function
    called `name`, or None."""
    for m in re.finditer(r"\b" + re.escape(name) + r"\s*\(", text):
        head = text[max(0, m.start() - 400):m.start()]
        if kind not in head.split(";")[-1].split("}")[-1]:
            continue
        i = text.find("{", m.end())
        semi = text.find(";", m.end())
        if i < 0 or (0 <= semi < i):
            continue   # a declaration or a call, not a definition
        depth, j = 0, i
        while j < len(text):
            if text[j] == "{":
                depth += 1
            elif text[j] == "}":
                depth -= 1
                if depth == 0:
                    return text[i + 1:j]
            j += 1
    return None


def pdl_kernels(text):
    names = set()
    for m in re.finditer(r"DP_LAUNCH_PDL\(\s*\w+\s*,\s*\w+\s*,\s*\(?\s*(\w+)", text):
        line = text[text.rfind("\n", 0, m.start()) + 1:m.start()]
        if "#define" not in line:   # the macro itself
            names.add(m.group(1))
    return names


def violations(text):
    """The kernels launched by DP_LAUNCH_PDL in `text` that reach no
    griddep_wait (in their body or a device function it calls) or store
    before it."""
    bad = []
    for k in sorted(pdl_kernels(text)):
        body = body_of(text, k, "__global__")
        if body is None:
            bad.append((k, "no definition"))
            continue
        if "griddep_wait()" not in body:   # the wait in a device function the kernel calls
            for callee in re.findall(r"\b(\w+)\s*(?:<[^;()]*>)?\s*\(", body):
                cb = body_of(text, callee, "__device__")
                if cb and "griddep_wait()" in cb:
                    body = cb
                    break
        if "griddep_wait()" not in body:
            bad.append((k, "no wait"))
            continue
        st = stores(body[:body.index("griddep_wait()")])
        if st:
            bad.append((k, st))
    return bad


def test_every_dependent_kernel_waits_before_it_writes():
    text = sources()
    assert {"k_gs_c_wp", "k_resid_c_wp", "k_csr_mv_p", "k_jacobi_pre_p", "k_jacobi_sweep_p",
            "k_dense_mv_p", "k_gs_c_tma", "k_resid_c_tma", "k_ilu_fwd_wp"} <= pdl_kernels(text)
    assert violations(text) == []


def test_the_check_catches_planted_mistakes():
    src = """
__device__ __forceinline__ void helper(float *x) { x[0] = 1.f; griddep_wait(); }
__global__ void k_store_first(float *x) { helper(x); }
__global__ void k_no_wait(float *x) { x[1] = 2.f; }
__global__ void k_fine(const float *y, float *x) { float a = y[0]; griddep_wait(); x[0] = a; }
void launch(Sim *s, float *x) {
  DP_LAUNCH_PDL(s, kPdlWells, k_store_first, 1, 32, 0, x);
  DP_LAUNCH_PDL(s, kPdlWells, (k_no_wait), 1, 32, 0, x);
  DP_LAUNCH_PDL(s, kPdlWells, k_fine, 1, 32, 0, x, x);
}
"""
    assert [k for k, _ in violations(src)] == ["k_no_wait", "k_store_first"]


DECL = re.compile(r"^(?:const\s+)?(?:using|unsigned|int|bool|float|double|size_t|uint\w*|auto|"
                  r"T2?|TR|R2|TV)\b")


def stores(code):
    """Statements of `code` that store through an array element or a
    dereferenced pointer, or call an atomic (declarations with initialisers,
    `T a[4] = {...}` or `const T *p = ...`, are not stores)."""
    out = []
    for st in re.split(r"[;{}]", code):
        st = st.strip()
        if not st or DECL.match(st):
            continue
        if re.search(r"\w\s*\[[^\]]*\]\s*=[^=]|^\*\s*\w+\s*=[^=]|atomic\w*\(", st):
            out.append(st)
    return out


def test_the_store_check_sees_stores():
    assert stores("x[i] = 1") and stores("*p = 2") and stores("atomicAdd(c, 1)")
    assert not stores("T a[4] = {T(0)}; const T *p = q + 1; int e = rowptr[i]; v = x[c] == 0")
