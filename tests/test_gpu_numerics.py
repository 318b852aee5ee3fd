"""The FP32 reciprocal and reciprocal square root of the Landau frame (a
hardware estimate refined by one Newton step) against exact FP64 values:
within 1.5 units in the last place everywhere the frame uses them, about
half a unit on average (a correctly rounded result has at most 0.5)."""
import json
import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


def test_frame_reciprocals_are_within_one_and_a_half_ulp():
    src = os.path.join(HERE, "numerics", "frame_math_check.cu")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "frame_math_check")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "--expt-relaxed-constexpr", "-o", exe, src], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    r = json.loads(out.strip().splitlines()[-1])
    assert r["recip_max_ulp"] <= 1.5 and r["rsqrt_max_ulp"] <= 1.5, r
    assert r["recip_mean_ulp"] < 0.6 and r["rsqrt_mean_ulp"] < 0.6, r
