"""Launch-shape autotuning and the dynamic fit schedule: neither changes a
result (each fit is solved by one CTA, each query by one thread, whatever
the grid or the order in which CTAs claim work)."""
import numpy as np
import pytest
import torch

import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import dev, need_gpu, program_to_device

pytestmark = pytest.mark.gpu


def test_fit_schedules_and_tuning_agree():
    need_gpu()
    inst = W.batched_instance(64, seed=61, degree_choices=(2, 3), m_range=(64, 2048))
    x, y, off, deg = (dev(inst[k]) for k in ("x", "y", "fit_off", "degree"))
    for prec in ("fp32", "tf32", "fp64"):
        a = rp.rp_fit(x, y, off, 3, precision=prec, degrees=deg, schedule="static")
        b = rp.rp_fit(x, y, off, 3, precision=prec, degrees=deg, schedule="dynamic")
        cap = rp.rp_tune_fit(x, y, off, 3, precision=prec, degrees=deg)
        assert 1 <= cap <= 16
        c = rp.rp_fit(x, y, off, 3, precision=prec, degrees=deg)
        torch.cuda.synchronize()
        for k in ("coef", "coef32", "box", "status", "rank"):
            assert torch.equal(a[k], b[k]), (prec, k)
            assert torch.equal(a[k], c[k]), (prec, k)


def test_search_tuning_agrees():
    need_gpu()
    K, d = 64, 3
    prog = W.synthetic_program(K, d, seed=62)
    buf = program_to_device(prog)
    q = dev(W.queries(300_000, K, seed=63))
    before = rp.rp_eval_search(buf, K, d, q)
    t, c = rp.rp_tune_search(buf, K, d, q)
    assert t in (64, 128, 256) and 2 <= c <= 32
    after = rp.rp_eval_search(buf, K, d, q)
    torch.cuda.synchronize()
    for k in before:
        assert torch.equal(before[k], after[k]), k
