"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/*.h declares; host-side argument validation (no GPU work) rejects bad input."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            if not src[m.start():m.end()].lstrip().startswith(("typedef", "return", "#")):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2010_10199_gb300 import build, gft
    build.build()
    return gft.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("anova_plan_create", "anova_plan_destroy", "grouped_trafo", "grouped_adjoint",
                     "lsqr_solve", "fista_solve", "anova_num_coeffs", "anova_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(os.path.join(ROOT, "paper_2010_10199_gb300", "libanova_gft.so"))
    missing = [n for n in _declared_functions() if not hasattr(raw, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings(lib):
    from paper_2010_10199_gb300 import gft
    assert gft.anova_status_string(0) == "ok"
    assert "invalid" in gft.anova_status_string(-1)
    assert "sm_103a" in gft.anova_version()


@pytest.mark.parametrize("case", ["d0", "odd_bandwidth", "coord_out_of_range", "unsorted", "gap", "no_terms"])
def test_plan_rejects_bad_arguments_before_any_device_work(lib, case):
    from paper_2010_10199_gb300 import gft
    terms, bw, d = [(), (0,), (0, 1)], [0, 8, 4], 3
    if case == "d0":
        d = 0
    elif case == "odd_bandwidth":
        bw = [0, 7, 4]
    elif case == "coord_out_of_range":
        terms = [(), (3,)]
        bw = [0, 8]
    elif case == "unsorted":
        terms = [(1, 0)]
        bw = [4]
    elif case == "no_terms":
        terms, bw = [], []
    if case == "gap":
        n = 1
        td = (ctypes.c_int32 * 3)(0, -1, 1)
        b = (ctypes.c_int32 * 1)(4)
        h = ctypes.c_void_p()
        rc = lib.anova_plan_create(ctypes.byref(h), 3, 0, None, n, td, b, None, None)
        assert rc == -1
        return
    with pytest.raises(gft.AnovaError) as e:
        gft.anova_plan_create(d, 0, 0, terms, bw)
    assert e.value.status == -1
