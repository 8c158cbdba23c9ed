"""The path's stated workloads beyond the benchmarked one, as parity cases.

* Plain FP64 tiny case: 4 integer-coefficient rational metrics of degree 2,
  64 noise-free lattice samples each; GPU FP64 predictions on the whole
  462-point lattice against the oracle's fit of the same FP32 samples, then
  one query over the 66 configurations.
* Differentiation: 4096 degree-3 fits of 512 samples, initialised from the
  GPU's linearised fit, 20 Adam steps on the mean squared relative error;
  the backward kernel against the oracle's gradient on sampled fits.
* Uneven batch: 8192 fits with 64..4096 samples (log-uniform) and degree
  2..4, fit -> pack -> search over 1e7 queries captured in one CUDA graph;
  replay equals the eager launches bit for bit; sampled fits against the
  oracle; the graph's argmin against the oracle's own program where both
  are decisive.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import HW, dev, eval_coef_at, host, need_gpu
from test_gpu_fit import compare

pytestmark = pytest.mark.gpu


def test_tiny_plain_fp64_lattice_and_query():
    need_gpu()
    inst = W.tiny_instance()
    x, y, off, deg = inst["x"], inst["y"], inst["fit_off"], inst["degree"]
    g = rp.rp_fit(dev(x), dev(y), dev(off), 2, precision="fp64", degrees=dev(deg))
    g = {k: host(v) for k, v in g.items()}
    ref = oracle.fit(x, y, off, deg)          # the same FP32 samples
    lat = inst["lattice"].astype(np.float64)
    for f in range(len(off) - 1):
        pg = eval_coef_at(g["coef"][f], g["box"][f], 2, lat)
        po = eval_coef_at(ref["coef"][f], ref["box"][f], 2, lat)
        assert np.max(np.abs(pg - po) / np.abs(po)) < 1e-8, f
    # one query (N = 2^12, hardware at the middle of its ranges), 66 configs
    mm = np.full((1, 8), -1, np.int32)
    mm[0, :4] = np.arange(4)
    gd = np.array([2], np.int32)
    buf = rp.rp_program_pack(dev(g["coef"]), dev(g["box"]), dev(deg), dev(mm), dev(gd), 2)
    q = np.zeros((1, 8), np.float32)
    q[0, W.Q_N], q[0, W.Q_NSM], q[0, W.Q_FGHZ] = 4096, 120, 1.6
    q[0, W.Q_MEMLD], q[0, W.Q_BW], q[0, W.Q_DDC], q[0, W.Q_DDU] = 600, 4500, 10.5, 10.5
    q[0, W.Q_KID] = np.array([0], np.int32).view(np.float32)[0]
    out = {k: host(v) for k, v in rp.rp_eval_search(buf, 1, 2, dev(q)).items()}
    prog = oracle.pack(ref["coef"], ref["box"], ref["degree"], mm, 2)
    prog["grid_dims"] = gd
    s = oracle.search(prog, HW, q)
    ev = oracle.evaluate(prog, HW, q)
    gap = (s["second"][0] - s["best"][0]) / s["best"][0]
    if gap > 1e-5 and ev["margin"][0].min() >= 1e-5:
        assert out["argmin"][0] == s["argmin"][0]
    assert abs(out["best"][0] - s["best"][0]) <= 1e-4 * s["best"][0]


def test_differentiation_4096_fits():
    need_gpu()
    inst = W.batched_instance(512, seed=20190604, m=512, d=3)
    x, y, off, deg = (dev(inst[k]) for k in ("x", "y", "fit_off", "degree"))
    F = len(inst["fit_off"]) - 1
    assert F == 4096
    fit = rp.rp_fit(x, y, off, 3, precision="fp32", degrees=deg)
    box = fit["box"]
    c = fit["coef"].clone()
    # the backward kernel against the oracle's gradient (itself pinned to
    # central finite differences) on sampled fits, at the linearised fit
    loss = host(rp.rp_relmse_fwd(x, y, off, deg, c, box))
    grad = host(rp.rp_relmse_bwd(x, y, off, deg, c, box, torch.ones(F, device="cuda")))
    pick = np.sort(np.random.default_rng(3).choice(F, 32, replace=False))
    xs, ys, offs = [], [], [0]
    for f in pick:
        a, b = inst["fit_off"][f], inst["fit_off"][f + 1]
        xs.append(inst["x"][:, a:b]); ys.append(inst["y"][a:b]); offs.append(offs[-1] + b - a)
    sub_off = np.array(offs, np.int64)
    lo, go = oracle.relmse(np.ascontiguousarray(np.concatenate(xs, 1)), np.concatenate(ys), sub_off,
                           inst["degree"][pick], host(c)[pick], host(box)[pick])
    np.testing.assert_allclose(loss[pick], lo, rtol=1e-4)
    scale = np.abs(go).max(axis=1, keepdims=True)
    assert np.max(np.abs(grad[pick] - go) / scale) < 1e-4
    # 20 Adam steps (default step) from the linearised fit
    l0, l1 = rp.refine_relmse(c, x, y, off, deg, box, steps=20)
    l0, l1 = host(l0), host(l1)
    assert np.isfinite(l1).all()
    assert (l1 <= l0 * (1 + 1e-6)).mean() > 0.9, (l1 > l0).sum()


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_uneven_batch_graph_captured(precision):
    need_gpu()
    K = 1024
    inst = W.batched_instance(K, seed=20190605, degree_choices=(2, 3, 4), m_range=(64, 4096))
    F = len(inst["fit_off"]) - 1
    x, y, off, deg = (dev(inst[k]) for k in ("x", "y", "fit_off", "degree"))
    mm = dev(inst["metric_map"])
    gd = torch.full((K,), 2, dtype=torch.int32, device="cuda")
    q = dev(W.queries(10_000_000, K, seed=20190606, n_log2=(6, 12)))
    Q = q.shape[0]
    fit_out = dict(coef=torch.empty((F, 70), dtype=torch.float64, device="cuda"),
                   coef32=torch.empty((F, 70), dtype=torch.float32, device="cuda"),
                   box=torch.empty((F, 6), dtype=torch.float64, device="cuda"),
                   status=torch.empty(F, dtype=torch.int32, device="cuda"),
                   rank=torch.empty(F, dtype=torch.int32, device="cuda"))
    prog = torch.empty(rp.rp_program_size(K, 4), dtype=torch.uint8, device="cuda")
    s_out = dict(argmin=torch.empty(Q, dtype=torch.int32, device="cuda"),
                 best=torch.empty(Q, dtype=torch.float32, device="cuda"),
                 second=torch.empty(Q, dtype=torch.float32, device="cuda"),
                 status=torch.empty(Q, dtype=torch.int32, device="cuda"),
                 workspace=torch.empty(rp.rp_search_workspace_size(K, Q), dtype=torch.uint8,
                                       device="cuda"))

    def step(stream):
        rp.rp_fit(x, y, off, 4, precision=precision, degrees=deg, out=fit_out, stream=stream,
                  max_refine=16 if precision == "bf16" else 8)
        rp.rp_program_pack(fit_out["coef"], fit_out["box"], deg, mm, gd, 4, program=prog,
                           stream=stream)
        rp.rp_eval_search(prog, K, 4, q, out=s_out, stream=stream)

    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        step(s)                       # eager (also the first-call set-up)
    torch.cuda.synchronize()
    # the workspaces are scratch (the fit's holds the dynamic schedule's
    # counters and the basis cache), not results
    outs = {**{"fit_" + k: v for k, v in fit_out.items() if k != "workspace"},
            **{"search_" + k: v for k, v in s_out.items() if k != "workspace"}}
    eager = {k: v.clone() for k, v in outs.items()}
    for v in outs.values():
        v.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        step(s)
    graph.replay()
    torch.cuda.synchronize()
    for k, v in outs.items():
        assert torch.equal(v, eager[k]), k
    # sampled fits against the oracle (objective, predictions as in the
    # batched fit tests)
    st = host(fit_out["status"])
    assert not (st & rp.RP_FIT_TIMEOUT).any()
    pick = np.sort(np.random.default_rng(7).choice(F, 24, replace=False))
    xs, ys, offs = [], [], [0]
    for f in pick:
        a, b = inst["fit_off"][f], inst["fit_off"][f + 1]
        xs.append(inst["x"][:, a:b]); ys.append(inst["y"][a:b]); offs.append(offs[-1] + b - a)
    sub = dict(x=np.ascontiguousarray(np.concatenate(xs, 1)), y=np.concatenate(ys),
               fit_off=np.array(offs, np.int64), degree=inst["degree"][pick])
    ref = oracle.fit(sub["x"], sub["y"], sub["fit_off"], sub["degree"])
    gsub = {k: host(v)[pick] for k, v in fit_out.items() if k != "workspace"}
    compare(sub, gsub, ref)
    # the argmin of the graph's search against the oracle's own program
    # (oracle fits of sampled kernels), where both are decisive.  Only
    # kernels with >= 1024 samples: with fewer, a degree-4 fit (69 unknowns)
    # is (nearly) under-determined and its values between the samples are
    # not fixed by the data (GPU and oracle agree on the samples only)
    counts = np.diff(inst["fit_off"])[::8]
    big = np.where(counts >= 1024)[0]
    kern = np.sort(np.random.default_rng(9).choice(big, 6, replace=False))
    fits = np.concatenate([np.arange(8 * k, 8 * k + 8) for k in kern])
    xs, ys, offs = [], [], [0]
    for f in fits:
        a, b = inst["fit_off"][f], inst["fit_off"][f + 1]
        xs.append(inst["x"][:, a:b]); ys.append(inst["y"][a:b]); offs.append(offs[-1] + b - a)
    ref2 = oracle.fit(np.ascontiguousarray(np.concatenate(xs, 1)), np.concatenate(ys),
                      np.array(offs, np.int64), inst["degree"][fits])
    mm2 = np.arange(8 * len(kern), dtype=np.int32).reshape(len(kern), 8)
    prog_o = oracle.pack(ref2["coef"], ref2["box"], ref2["degree"], mm2, 4)
    prog_o["grid_dims"] = np.full(len(kern), 2, np.int32)
    qh = host(q)
    kid = W.query_kernel_ids(qh)
    sel = np.where(np.isin(kid, kern))[0]
    sel = sel[np.random.default_rng(8).choice(len(sel), min(3000, len(sel)), replace=False)]
    qs = qh[sel].copy()
    remap = {int(k): i for i, k in enumerate(kern)}
    qs[:, W.Q_KID] = np.array([remap[int(k)] for k in kid[sel]], np.int32).view(np.float32)
    so = oracle.search(prog_o, HW, qs)
    ga = host(s_out["argmin"])[sel]
    gb = host(s_out["best"])[sel]
    gap_o = (so["second"] - so["best"]) / so["best"]
    gap_g = (host(s_out["second"])[sel] - gb) / gb
    # the graph's program comes from the GPU's fits, which agree with the
    # oracle's to 1e-4: identical argmins wherever the oracle's top-two gap
    # is decisive at 1e-3, and on all but a few queries at 1e-5
    # (queries whose best or second configuration is FP32-ill-conditioned or
    # within 1e-5 of a case boundary excluded, as in the search tests)
    ev = oracle.evaluate(prog_o, HW, qs)
    rows = np.arange(len(qs))
    sec = np.argsort(ev["exec"], axis=1)[:, 1]
    ill = ((ev["margin"][rows, so["argmin"]] < 1e-5) | (ev["cond"][rows, so["argmin"]] > 30) |
           (ev["margin"][rows, sec] < 1e-5) | (ev["cond"][rows, sec] > 30))
    d3, d5 = (gap_o > 1e-3) & ~ill, (gap_o > 1e-5) & ~ill
    assert d3.sum() > 500
    assert (ga[d3] == so["argmin"][d3]).all()
    assert (ga[d5] == so["argmin"][d5]).mean() > 0.999
