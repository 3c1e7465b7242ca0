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


def test_erfc64_piecewise_against_fp64_erfc():
    """The FP64 piecewise erfc and its derivative against CUDA's FP64 erfc and exp.

    Below x = 6.5 the relative error must stay under 1e-13 (the construction
    gives about 1e-14).  Beyond 6.5 the table returns 0, and the true values
    are below 4e-20.
    """
    import math

    qg = cuda_or_skip()
    sysm = qg.System(qg.make_params(10, (20.0, 20.0, 20.0), mesh=(8, 8, 8)))
    x = torch.linspace(0.0, 7.0, 1_400_001, dtype=torch.float64, device="cuda")
    out = torch.empty_like(x)
    dout = torch.empty_like(x)
    qg._lib.qeq_selftest_erfc64(sysm.ctx, x, out, dout)
    ref = torch.special.erfc(x)
    dref = -2.0 / math.sqrt(math.pi) * torch.exp(-x * x)
    inside = x < 6.5
    assert ((out - ref).abs() / ref)[inside].max().item() < 1e-13
    assert ((dout - dref).abs() / dref.abs())[inside].max().item() < 1e-13
    assert out[~inside].abs().max().item() == 0.0 and ref[~inside].max().item() < 4e-20
    sysm.close()
