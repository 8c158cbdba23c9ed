"""A stream of steps on two CUDA streams -- the fit of step k+1 on a
high-priority stream while the pack and search of step k run on a second
one, three buffer sets (the schedule bench.py times) -- gives every step the
results of the same step run alone on one stream, bit for bit: the library's
calls are stream-ordered and keep no state between calls."""
import numpy as np
import pytest
import torch

import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import dev, need_gpu

pytestmark = pytest.mark.gpu


def test_pipelined_steps_equal_serial_steps():
    need_gpu()
    K, Q, D = 96, 50_000, 3
    inst = W.batched_instance(K, seed=141, m=512, d=D)
    xp, poff = W.shared_points(inst)
    x, y, off, deg = dev(xp), dev(inst["y"]), dev(inst["fit_off"]), dev(inst["degree"])
    fk = dict(point_off=dev(poff), fits_per_point_set=W.N_METRICS)
    mm = dev(inst["metric_map"])
    gd = torch.full((K,), 2, dtype=torch.int32, device="cuda")
    q = dev(W.queries(Q, K, seed=142, n_log2=(6, 20)))
    fit_kw = dict(precision="fp32", tol=1e-8, max_refine=16, degrees=deg, **fk)

    def step(fo, prog, so, s_fit, s_eval):
        rp.rp_fit(x, y, off, D, out=fo, stream=s_fit, **fit_kw)
        done = torch.cuda.Event()
        done.record(s_fit)
        s_eval.wait_event(done)
        rp.rp_program_pack(fo["coef"], fo["box"], deg, mm, gd, D, program=prog, stream=s_eval)
        rp.rp_eval_search(prog, K, D, q, out=so, stream=s_eval)

    # reference: one step alone on one stream
    ref_fit = rp.rp_fit(x, y, off, D, **fit_kw)
    ref_prog = rp.rp_program_pack(ref_fit["coef"], ref_fit["box"], deg, mm, gd, D)
    ref = rp.rp_eval_search(ref_prog, K, D, q)
    torch.cuda.synchronize()

    NB = 3
    fos = [{k: torch.empty_like(v) for k, v in ref_fit.items()} for _ in range(NB)]
    progs = [torch.empty_like(ref_prog) for _ in range(NB)]
    sos = [{k: torch.empty_like(v) for k, v in ref.items()} for _ in range(NB)]
    s_fit, s_eval = torch.cuda.Stream(priority=-1), torch.cuda.Stream()
    pack_done = [None] * NB
    results = []
    for k in range(7):
        b = k % NB
        if pack_done[b] is not None:            # step k - NB's pack has read fit set b
            s_fit.wait_event(pack_done[b])
        step(fos[b], progs[b], sos[b], s_fit, s_eval)
        pack_done[b] = torch.cuda.Event()
        pack_done[b].record(s_eval)
        if k >= NB - 1:                          # read back step k - NB + 1's results
            b0 = (k - NB + 1) % NB
            s_eval.synchronize()
            results.append(({n: v.clone() for n, v in fos[b0].items() if n != "workspace"},
                            {n: v.clone() for n, v in sos[b0].items() if n != "workspace"}))
            torch.cuda.synchronize()             # the copies are done before set b0 is reused
    torch.cuda.synchronize()
    assert len(results) == 5
    for fit_out, srch in results:
        for n in ("coef", "coef32", "box", "status", "rank"):
            assert torch.equal(fit_out[n], ref_fit[n]), n
        for n in ("argmin", "best", "second", "status"):
            assert torch.equal(srch[n], ref[n]), n
