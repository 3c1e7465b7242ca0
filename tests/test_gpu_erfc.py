"""The FP32 erfc of the real-space kernel (A&S 7.1.26) against CUDA's FP64 erfc -- GPU.

The approximation's own bound is 1.5e-7 absolute.  Evaluating it in FP32 adds
rounding:
  - the Horner polynomial has coefficients of magnitude up to 1.45 with
    alternating signs, worth a few ulp of 1.2e-7 near x = 0, where erfc is
    close to 1;
  - the approximate reciprocal and exponential (__fdividef, __expf) add at most
    2 ulp each.
So the test allows 1e-6 absolute over [0, 14].  The relative error at the
workload cutoff (alpha r_c = 2.72) stays within 3e-3, because there the
absolute bound dominates.
"""

import numpy as np
import pytest

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_erfc32_within_bound():
    qg = cuda_or_skip()
    x = torch.linspace(0.0, 14.0, 2_000_001, dtype=torch.float32, device="cuda")
    out = torch.empty_like(x)
    qg._lib.qeq_selftest_erfc32(x, out)
    ref = torch.special.erfc(x.double())
    err = (out.double() - ref).abs()
    assert err.max().item() < 1e-6
    # beyond x = 1 the approximation's own bound dominates
    tail = x >= 1.0
    assert err[tail].max().item() < 2.5e-7
    i = int(2.72 / 14.0 * 2_000_000)
    assert abs(out[i].item() / ref[i].item() - 1.0) < 3e-3
