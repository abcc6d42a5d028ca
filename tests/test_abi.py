"""The C-ABI library loads and exports every function that include/*.h
declares; host-only entry points answer without a GPU.  CPU only."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][A-Za-z0-9_]*[\s*]+)+([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_06938_gb300 import _build
    _build.build()
    from paper_2507_06938_gb300 import bta
    return bta.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["bta_create", "bta_assemble", "bta_factor", "bta_logdet", "bta_solve",
                     "bta_selinv", "fobj_eval", "bta_model_create", "bta_sync"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(lib._name)
    for name in _declared_functions():
        assert hasattr(raw, name), name


def test_binding_matches_header():
    from paper_2507_06938_gb300 import bta
    assert sorted(bta.exported_symbols()) == _declared_functions()


def test_binding_constants_match_header():
    """Every integer #define of the header has the same value in the binding."""
    from paper_2507_06938_gb300 import bta
    text = open(os.path.join(ROOT, "include", "bta.h")).read()
    defs = dict(re.findall(r"^#define\s+(BTA_[A-Z0-9_]+)\s+(-?\d+)\b", text, flags=re.M))
    assert "BTA_PHASES" in defs and "BTA_MIXED_HI" in defs
    for name, value in defs.items():
        if hasattr(bta, name):
            assert getattr(bta, name) == int(value), name
    assert len(bta.PHASE_NAMES) == bta.BTA_PHASES


def test_host_only_entry_points(lib):
    assert lib.bta_strerror(0) == b"ok"
    assert b"positive definite" in lib.bta_strerror(3)
    # nominal flop model: n b^3/3 + (n-1) 2 b^3 + n (a b^2 + a^2 b) + (n-1) 2 a b^2 + a^3/3
    n, b, a = 64, 1024, 4
    expect = n * b ** 3 / 3 + (n - 1) * 2 * b ** 3 + n * (a * b * b + a * a * b) + (n - 1) * 2 * a * b * b + a ** 3 / 3
    assert abs(lib.bta_flops_factor(n, b, a) - expect) < 1e-6 * expect
    # argument validation happens on the host, before any device work
    h = ctypes.c_void_p()
    assert lib.bta_create(0, 10, 2, 0, None, ctypes.byref(h)) == 1
    assert lib.bta_create(4, 10, 2, 7, None, ctypes.byref(h)) == 1
    assert lib.bta_model_create(None, ctypes.byref(h)) == 1
    # the multi-problem entry rejects an empty or incomplete request before launching anything
    P = ctypes.c_void_p
    one = (ctypes.c_int * 1)(1)
    null = (P * 1)(None)
    assert lib.bta_fobj_eval_multi(0, null, null, null, one, null, None, None, None) == 1
    assert lib.bta_fobj_eval_multi(1, null, null, null, one, null, None, None, None) == 1
    assert lib.bta_fobj_eval_multi(1, None, None, None, None, None, None, None, None) == 1
    # the creation flags, the layout switches and the read-outs check their arguments first
    assert lib.bta_create_ex(4, 10, 2, 0, 1, 2, None, ctypes.byref(h)) == 1
    assert lib.bta_create_ex(4, 10, 2, 0, 0, 1, None, ctypes.byref(h)) == 1
    assert lib.bta_set_low_memory(None, 1) == 1
    assert lib.bta_set_time_partitions(None, 2) == 1
    ms = (ctypes.c_double * 5)()
    assert lib.bta_profile_phases(None, ms, 5) == 1


C_PROGRAM = r"""
#include "bta.h"
#include <stdio.h>
#include <string.h>

int main(void) {
    bta_ctx_t ctx = NULL;
    bta_model_t model = NULL;
    const bta_ctx_t ctxs[1] = {NULL};
    const bta_model_t models[1] = {NULL};
    const double* thetas[1] = {NULL};
    double* fs[1] = {NULL};
    const int n_theta[1] = {1};
    const char* ok = bta_strerror(BTA_OK);
    double f = bta_flops_factor(64, 1024, 4) + bta_flops_selinv(64, 1024, 4);
    if (strcmp(ok, "ok") != 0 || !(f > 0.0)) return 10;
    if (bta_create(0, 10, 2, BTA_FP64, NULL, &ctx) != BTA_ERR_ARG) return 11;
    if (bta_create_batched(4, 10, 2, BTA_MIXED, 0, NULL, &ctx) != BTA_ERR_ARG) return 12;
    if (bta_model_create(NULL, &model) != BTA_ERR_ARG) return 13;
    if (bta_fobj_eval_multi(0, ctxs, models, thetas, n_theta, fs, NULL, NULL, NULL) != BTA_ERR_ARG) return 14;
    if (bta_fobj_eval_multi(1, ctxs, models, thetas, n_theta, fs, NULL, NULL, NULL) != BTA_ERR_ARG) return 15;
    if (bta_chol_inv_noalloc(NULL, 4, 4, NULL, 4, NULL, NULL) != BTA_ERR_ARG) return 16;
    if (bta_create_ex(4, 10, 2, BTA_MIXED_HI, 0, BTA_CREATE_LOW_MEMORY, NULL, &ctx) != BTA_ERR_ARG) return 17;
    if (bta_set_low_memory(NULL, 1) != BTA_ERR_ARG) return 18;
    printf("%s|%s\n", bta_strerror(BTA_ERR_ARG), bta_strerror(BTA_ERR_STATE));
    return 0;
}
"""


def test_header_compiles_as_c_and_links(lib, tmp_path):
    """include/bta.h is self-contained C99: a C program that includes only it
    compiles with -Wall -Werror, links libbta.so and gets the host-side
    answers (no GPU needed)."""
    import shutil
    import subprocess
    cc = shutil.which("cc") or shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_bta.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_bta"
    libdir = os.path.dirname(lib._name)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                        "-L", libdir, "-lbta", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    env = dict(os.environ)
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    env["LD_LIBRARY_PATH"] = cuda_lib + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    r = subprocess.run([str(exe)], capture_output=True, text=True, env=env)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == "invalid argument|call out of order"
