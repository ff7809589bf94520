"""The allocation-free distance call (ttc_tt_dist2_static) against the
context-based relative error (ttc_relerr), through the C ABI, on two calls in
a row.  Collected last on purpose.  GPU only.

It serves callers that may not allocate device memory themselves (a fixed
memory budget, or a framework that owns all device allocations): the test
allocates the inputs and the output with PyTorch on the caller's behalf and
the call itself allocates nothing, using a fixed device array for its
partial sums.
"""
import ctypes as C
import math

import numpy as np
import pytest

import oracle as o
from paper_2501_13385_gb300 import ttc
from paper_2501_13385_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def _static_dist2(n, ra, a_cores, rb, b_cores, torch):
    """Calls the C ABI with device copies of the cores; returns (||A-B||^2, ||B||^2).
    PyTorch's allocator holds the same bytes before and after the call (the
    call takes no memory from it)."""
    dev = torch.device("cuda:0")
    a_t = [torch.from_numpy(np.ascontiguousarray(c)).to(dev) for c in a_cores]
    b_t = [torch.from_numpy(np.ascontiguousarray(c)).to(dev) for c in b_cores]
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated(dev)
    d = len(n)
    n_a = np.asarray(n, dtype=np.int64)
    ra_a = np.asarray(ra, dtype=np.int32)
    rb_a = np.asarray(rb, dtype=np.int32)
    ap = (C.c_void_p * d)(*[t.data_ptr() for t in a_t])
    bp = (C.c_void_p * d)(*[t.data_ptr() for t in b_t])
    stream = torch.cuda.current_stream(dev)
    st = ttc.lib().ttc_tt_dist2_static(d, n_a.ctypes.data_as(C.POINTER(C.c_int64)),
                                       ra_a.ctypes.data_as(C.POINTER(C.c_int32)), ap,
                                       rb_a.ctypes.data_as(C.POINTER(C.c_int32)), bp,
                                       C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == 0, ttc.lib().ttc_strerror(st)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(dev) == held
    res = out.cpu().numpy()
    return float(res[0]), float(res[1])


def test_static_scratch_distance_matches_relerr_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2501_13385_gb300 import build
    build.build()
    P = w.planted_small(0)
    with ttc.Context(P.n, P.r, precision=ttc.PREC_FP64) as c:
        c.set_observations(P.idx, P.y)
        c.set_cores(P.init)
        c.set_truth(P.truth)
        for call in range(2):
            rel = c.relerr()
            cur = c.get_cores()
            d2, b2 = _static_dist2(P.n, P.r, cur, [1, 2, 2, 2, 1], P.truth, torch)
            assert math.sqrt(d2 / b2) == pytest.approx(rel, rel=1e-12)
            assert math.sqrt(d2) == pytest.approx(o.tt_dist(cur, P.truth), rel=1e-10)
            c.step()      # the second call sees a different iterate


def test_static_scratch_rejects_shapes_beyond_its_limits():
    pytest.importorskip("torch")
    from paper_2501_13385_gb300 import build
    build.build()
    L = ttc.lib()
    d = 3
    n = np.asarray([2048, 2048, 2048], dtype=np.int64)     # d* = 2^33 > 2^32
    r = np.asarray([1, 1, 1, 1], dtype=np.int32)
    ptrs = (C.c_void_p * d)(*[1, 1, 1])                     # never dereferenced: rejected first
    st = L.ttc_tt_dist2_static(d, n.ctypes.data_as(C.POINTER(C.c_int64)), r.ctypes.data_as(C.POINTER(C.c_int32)),
                               ptrs, r.ctypes.data_as(C.POINTER(C.c_int32)), ptrs, C.c_void_p(1), None)
    assert st == -10
    r_big = np.asarray([1, 33, 1, 1], dtype=np.int32)
    n_small = np.asarray([4, 4, 4], dtype=np.int64)
    st = L.ttc_tt_dist2_static(d, n_small.ctypes.data_as(C.POINTER(C.c_int64)),
                               r_big.ctypes.data_as(C.POINTER(C.c_int32)), ptrs,
                               r.ctypes.data_as(C.POINTER(C.c_int32)), ptrs, C.c_void_p(1), None)
    assert st == -10


def test_static_scratch_grid_stride_shape_then_a_smaller_one():
    """d* = 64 * 64 * 96 = 393 216 entries: more than 1024 blocks' worth, so
    every block strides over the entries and the finish sums 1024 partials;
    then a smaller shape (fewer blocks) whose call must not read the first
    call's extra slots.  Against the oracle's distance and norm to 1e-10."""
    torch = pytest.importorskip("torch")
    from paper_2501_13385_gb300 import build
    build.build()
    for (n, ra, rb, seed) in (([64, 64, 96], [1, 8, 8, 1], [1, 3, 5, 1], 31), ([6, 7, 5], [1, 2, 3, 1], [1, 3, 2, 1], 32)):
        A = w.random_problem(seed, n, ra, 10, init_rel=0.0).truth
        B = w.random_problem(seed + 100, n, rb, 10, init_rel=0.0).truth
        d2, b2 = _static_dist2(n, ra, A, rb, B, torch)
        assert math.sqrt(d2) == pytest.approx(o.tt_dist(A, B), rel=1e-10)
        assert math.sqrt(b2) == pytest.approx(o.tt_norm(B), rel=1e-10)


def test_static_scratch_rejects_work_beyond_its_budget():
    """d* = 4^16 = 2^32 entries of rank-32 trains: far more than 2^34 FMAs."""
    pytest.importorskip("torch")
    from paper_2501_13385_gb300 import build
    build.build()
    L = ttc.lib()
    d = 16
    n = np.asarray([4] * d, dtype=np.int64)
    r = np.asarray([1] + [32] * (d - 1) + [1], dtype=np.int32)
    ptrs = (C.c_void_p * d)(*([1] * d))                   # never dereferenced: rejected first
    st = L.ttc_tt_dist2_static(d, n.ctypes.data_as(C.POINTER(C.c_int64)), r.ctypes.data_as(C.POINTER(C.c_int32)),
                               ptrs, r.ctypes.data_as(C.POINTER(C.c_int32)), ptrs, C.c_void_p(1), None)
    assert st == -10
