"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/lp.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lp_create", "lp_solve", "lp_solve_batch", "lp_grad", "lp_destroy",
              "lp_status_string", "lp_opts_default"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2508_16806_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lp_[a-z_0-9]+)", out))
    assert set(declared_functions()) <= exported


def test_host_only_calls_without_gpu():
    """lp_opts_default, lp_status_string and lp_abi_version make no CUDA call."""
    from paper_2508_16806_gb300 import lp as L
    o = L.lp_opts_default()
    assert o.tol == 1e-4 and o.check_every == 64 and o.eta_scale == 0.9
    assert o.beta_sufficient == 0.2 and o.beta_necessary == 0.8 and o.beta_artificial == 0.36
    assert o.infeas_detect == 1 and o.infeas_tol == 1e-6 and o.autotune == 0
    assert o.halpern == 0 and o.halpern_reflect == 1.0
    assert L.lp_status_string(1) == "LP_OPTIMAL"
    assert L.lp_status_string(-1) == "LP_INVALID_ARGUMENT"
    assert L.load().lp_abi_version() == 5


def test_binding_mirrors_struct_sizes():
    """The ctypes structs have the C layout: compile a probe against lp.h."""
    import tempfile
    from paper_2508_16806_gb300 import lp as L
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "lp.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lp_desc), sizeof(lp_opts),
         sizeof(lp_result), sizeof(lp_trace_rec), offsetof(lp_result, x), offsetof(lp_opts, x0),
         offsetof(lp_opts, halpern_reflect), offsetof(lp_opts, pc_alpha),
         offsetof(lp_result, pc_alpha_used));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        open(c, "w").write(probe)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(t) for t in subprocess.check_output([exe]).split()]
    want = [ctypes.sizeof(L.LpDesc), ctypes.sizeof(L.LpOpts), ctypes.sizeof(L.LpResult),
            ctypes.sizeof(L.LpTraceRec), L.LpResult.x.offset, L.LpOpts.x0.offset,
            L.LpOpts.halpern_reflect.offset, L.LpOpts.pc_alpha.offset,
            L.LpResult.pc_alpha_used.offset]
    assert got == want
