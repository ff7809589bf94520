"""Why the FP32 sampled pass keeps FP32 core storage: cores rounded to BF16
(8-bit mantissa, round to nearest even) put the sampled entries of the
workloads far outside the stated FP32 tolerance (1e-5 of max(|v|, rms v)),
while FP32 cores stay inside it.  Plain CPU arithmetic on the oracle's chain
evaluation (Eq. (TT Core)); no GPU."""
import numpy as np
import pytest

import oracle as o
from paper_2501_13385_gb300 import workloads as w


def to_bf16(x):
    """Round to the nearest BF16 value (ties to even) and return it as FP64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32)
    r = ((a + np.uint32(0x7FFF) + ((a >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def test_bf16_rounding_is_round_to_nearest_even():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1.0)
    assert to_bf16(1.0 + 2.0 ** -8)[()] == 1.0
    assert to_bf16(1.0 + 3 * 2.0 ** -8)[()] == 1.0 + 2.0 ** -6
    assert to_bf16(-3.0)[()] == -3.0


@pytest.mark.parametrize("maker", ["orthogonal_cubic", "tomography_like"])
def test_bf16_cores_break_the_fp32_tolerance(maker):
    P = getattr(w, maker)(0)
    sel = np.random.default_rng(0).choice(P.N, 5000, replace=False)
    v64 = o.tt_eval(P.init, P.idx[sel])
    floor = np.maximum(np.abs(v64), np.sqrt(np.mean(v64 ** 2)))
    v_bf16 = o.tt_eval([to_bf16(c) for c in P.init], P.idx[sel])
    v_f32 = o.tt_eval([np.asarray(c, dtype=np.float32).astype(np.float64) for c in P.init], P.idx[sel])
    assert np.max(np.abs(v_f32 - v64) / floor) <= 1e-5
    assert np.max(np.abs(v_bf16 - v64) / floor) >= 100 * 1e-5
