"""The generated rational program on the GPU (Sec. 3.3 Step 3 / Sec. 4.3.1):
one kernel's program written out as source with its coefficients as
constants, compiled at run time (NVRTC) and run on that kernel's queries,
gives the table-driven search's results bit for bit (the same per-
configuration arithmetic); queries naming another kernel are RP_Q_BAD."""
import numpy as np
import pytest
import torch

import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import dev, host, need_gpu, program_to_device
from test_codegen_cpu import host_program

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d", [2, 3, 4])
def test_generated_program_equals_table_search(d):
    need_gpu()
    K = 4
    prog = W.synthetic_program(K, d, seed=70 + d)
    kid = 1
    try:
        gen = rp.GeneratedProgram(rp.rp_codegen_source(host_program(prog), K, d, kid))
    except rp.RPError as e:
        if "not supported" in str(e) or "(-2)" in str(e):
            pytest.skip(str(e))
        raise
    q = W.queries(50000, K, seed=80 + d)
    q[:, W.Q_KID] = np.array([kid], np.int32).view(np.float32)[0]
    q[:7, W.Q_KID] = np.array([3], np.int32).view(np.float32)[0]     # another kernel's queries
    q[7, W.Q_N] = np.nan                                                # a bad query
    g = {k: host(v) for k, v in gen.search(dev(q)).items()}
    t = {k: host(v) for k, v in rp.rp_eval_search(program_to_device(prog), K, d, dev(q[7:])).items()}
    for k in ("argmin", "best", "second", "status"):
        np.testing.assert_array_equal(g[k][7:], t[k], err_msg=k)
    assert (g["status"][:7] & rp.RP_Q_BAD).all() and (g["argmin"][:7] == -1).all()
