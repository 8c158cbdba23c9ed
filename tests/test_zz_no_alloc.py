"""rp_fit_noalloc (static device scratch, no allocation) against rp_fit with a
caller workspace: identical results, on two calls in a row."""
import pytest
import torch

import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import dev, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,degrees", [("fp32", (2, 3)), ("tf32", (2, 3)), ("fp64", (2, 3)),
                                               ("fp32", (2, 4))])
def test_fit_noalloc_matches_rp_fit(precision, degrees):
    """Degrees (2, 4): the batch runs as a degree-3 and a degree-4 launch
    (and, for fits the FP32 solve passes on, FP64 launches), all sharing
    the static counters, each reset before its launch."""
    need_gpu()
    inst = W.batched_instance(48, seed=71, degree_choices=degrees, m_range=(64, 1024))
    x, y, off, deg = (dev(inst[k]) for k in ("x", "y", "fit_off", "degree"))
    dmax = max(degrees)
    ref = rp.rp_fit(x, y, off, dmax, precision=precision, degrees=deg)
    for _ in range(2):
        got = rp.rp_fit_noalloc(x, y, off, dmax, precision=precision, degrees=deg)
        torch.cuda.synchronize()
        for k in ("coef", "coef32", "box", "status", "rank"):
            assert torch.equal(got[k], ref[k]), (precision, k)
