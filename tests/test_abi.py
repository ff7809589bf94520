"""The C-ABI library builds for sm_103a, loads, and exports every function
include/ttc.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ttc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(ttc_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2501_13385_gb300 import build
    path = build.build()
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ttc_create", "ttc_set_observations", "ttc_step", "ttc_solve", "ttc_get_cores",
                     "ttc_set_cores", "ttc_destroy", "ttc_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_exports(built_lib):
    from paper_2501_13385_gb300 import ttc
    L = ttc.lib()
    assert set(declared_functions()) <= set(ttc.EXPORTS) | {"ttc_default_options"}
    assert L.ttc_strerror(-4) == b"duplicate index in Omega"
    assert L.ttc_strerror(0) == b"ok"


def test_default_options_from_library(built_lib):
    from paper_2501_13385_gb300 import ttc
    o = ttc.default_options()
    assert o.precision == ttc.PREC_MIXED and o.eps_rel == 1.0 and o.alpha_scale == 1.5
    assert o.max_iter == 500 and o.use_graph == 1
    assert o.step_fallback == 1 and o.dense_mode == ttc.DENSE_AUTO and o.polish_factor == 10.0


@pytest.mark.parametrize("n,r", [
    ([12, 10, 11, 9], [1, 12, 17, 11, 1]),    # r_3 = 11 > n_4 = 9
    ([3, 40, 40], [1, 4, 2, 1]),              # r_1 = 4 > n_1 = 3
    ([2, 2, 2, 2], [1, 2, 5, 2, 1]),          # r_2 = 5 > n_1 n_2 = 4
])
def test_infeasible_tt_ranks_are_rejected_before_any_device_work(built_lib, n, r):
    # a TT-rank above either dimension of its unfolding is no tensor's rank;
    # ttc_create refuses it before it touches the GPU (so this runs here)
    from paper_2501_13385_gb300 import ttc
    import numpy as np
    L = ttc.lib()
    h = ctypes.c_void_p()
    na = np.asarray(n, dtype=np.int64)
    ra = np.asarray(r, dtype=np.int32)
    st = L.ttc_create(ctypes.byref(h), len(n), na.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                      ra.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, None)
    assert st == -1 and not h.value


def test_compiled_for_sm_103a_only():
    from paper_2501_13385_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
