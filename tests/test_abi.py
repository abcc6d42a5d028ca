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
