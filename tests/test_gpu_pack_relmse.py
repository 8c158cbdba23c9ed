"""GPU program packing and relative-MSE forward/backward against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import HW, dev, host, need_gpu, program_to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fitted():
    inst = W.batched_instance(6, seed=51, m=256, d=3)
    ref = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    return inst, ref


def test_pack_parity(fitted):
    need_gpu()
    inst, ref = fitted
    K = inst["metric_map"].shape[0]
    gd = (np.arange(K) % 2 + 1).astype(np.int32)
    o = oracle.pack(ref["coef"], ref["box"], ref["degree"], inst["metric_map"], 3)
    buf = rp.rp_program_pack(dev(ref["coef"]), dev(ref["box"]), dev(inst["degree"]),
                             dev(inst["metric_map"]), dev(gd), 3)
    aN, bN, g_gd, tab = (host(t) for t in rp.program_views(buf, K, 3))
    np.testing.assert_array_equal(aN, o["aN"])
    np.testing.assert_array_equal(bN, o["bN"])
    np.testing.assert_array_equal(g_gd, gd)
    # FP64 sums in a possibly different order, each rounded to float: equal
    # up to one float rounding of the larger terms
    scale = np.maximum(np.abs(o["table"]), 1e-30)
    assert np.max(np.abs(tab - o["table"]) / scale) < 1e-6 or np.allclose(tab, o["table"], rtol=1e-6, atol=1e-9)


def test_pack_absent_metric_and_degree_mix():
    need_gpu()
    inst = W.batched_instance(2, seed=52, m=128, degree_choices=(1, 2, 3))
    ref = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    mm = inst["metric_map"].copy()
    mm[1, 4] = -1
    gd = np.array([2, 1], np.int32)
    o = oracle.pack(ref["coef"], ref["box"], ref["degree"], mm, 3)
    buf = rp.rp_program_pack(dev(ref["coef"]), dev(ref["box"]), dev(inst["degree"]), dev(mm),
                             dev(gd), 3)
    _, _, _, tab = (host(t) for t in rp.program_views(buf, 2, 3))
    assert (tab[1, :, 4, 0] == 0).all() and (tab[1, :, 4, 1, 0] == 1).all()
    np.testing.assert_allclose(tab, o["table"], rtol=1e-6, atol=1e-9)


def test_pipeline_fit_pack_search():
    """GPU fit -> GPU pack -> GPU search, checked two ways.
    1. The search on the same input as the oracle: the GPU evaluates the
       oracle's own program (oracle fits, oracle pack); argmin identical
       wherever the oracle's top-two gap exceeds 1e-5 relative, except
       queries whose best or second configuration is FP32-ill-conditioned
       or within 1e-5 of a case boundary (the exclusions of the search
       tests, counted).
    2. End to end: the GPU's program (from the GPU's fits) against the
       oracle's; the fits agree to 1e-4, so the argmins agree wherever the
       oracle's gap is decisive at 1e-3, and on all but a few queries at
       1e-5."""
    need_gpu()
    inst = W.batched_instance(8, seed=53, m=512, d=3)
    K = 8
    g = rp.rp_fit(dev(inst["x"]), dev(inst["y"]), dev(inst["fit_off"]), 3, precision="fp32",
                  degrees=dev(inst["degree"]), tol=1e-8)
    gd = torch.full((K,), 2, dtype=torch.int32, device="cuda")
    buf = rp.rp_program_pack(g["coef"], g["box"], dev(inst["degree"]), dev(inst["metric_map"]), gd, 3)
    q = W.queries(4000, K, seed=54, n_log2=(6, 12))      # inside the fitted range of N
    out = rp.rp_eval_search(buf, K, 3, dev(q))
    ref = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    prog = oracle.pack(ref["coef"], ref["box"], ref["degree"], inst["metric_map"], 3)
    prog["grid_dims"] = np.full(K, 2, np.int32)
    s = oracle.search(prog, HW, q)
    gap = (s["second"] - s["best"]) / s["best"]
    # 1. same program on both sides
    same = rp.rp_eval_search(program_to_device(prog), K, 3, dev(q))
    ev = oracle.evaluate(prog, HW, q)
    rows = np.arange(len(q))
    second = np.argsort(ev["exec"], axis=1)[:, 1]
    ill = ((ev["margin"][rows, s["argmin"]] < 1e-5) | (ev["cond"][rows, s["argmin"]] > 30) |
           (ev["margin"][rows, second] < 1e-5) | (ev["cond"][rows, second] > 30))
    dec = (gap > 1e-5) & ~ill
    assert dec.sum() > 2000, (dec.sum(), ill.sum())
    assert (host(same["argmin"])[dec] == s["argmin"][dec]).all()
    # 2. end to end (same exclusions)
    ga = host(out["argmin"])
    d3 = (gap > 1e-3) & ~ill
    assert (ga[d3] == s["argmin"][d3]).all()
    assert (ga[dec] == s["argmin"][dec]).mean() > 0.999


def test_relmse_forward_backward(fitted):
    """Loss within 1e-4 relative and gradient within 1e-4 of its largest
    entry, against the oracle's FP64 loss and closed-form gradient (the
    oracle's gradient is itself pinned to central finite differences)."""
    need_gpu()
    inst, ref = fitted
    x, y, off, deg = inst["x"], inst["y"], inst["fit_off"], inst["degree"]
    rng = np.random.default_rng(0)
    c = ref["coef"] * (1 + 1e-3 * rng.standard_normal(ref["coef"].shape))
    loss_o, grad_o = oracle.relmse(x, y, off, deg, c, ref["box"])
    loss_g = host(rp.rp_relmse_fwd(dev(x), dev(y), dev(off), dev(deg), dev(c), dev(ref["box"])))
    np.testing.assert_allclose(loss_g, loss_o, rtol=1e-4)
    gl = np.linspace(0.5, 2.0, len(off) - 1).astype(np.float32)
    grad_g = host(rp.rp_relmse_bwd(dev(x), dev(y), dev(off), dev(deg), dev(c), dev(ref["box"]), dev(gl)))
    ref_g = grad_o * gl[:, None]
    scale = np.abs(ref_g).max(axis=1, keepdims=True)
    assert np.max(np.abs(grad_g - ref_g) / scale) < 1e-4
    assert (grad_g[:, 35] == 0).all()


def test_relmse_autograd_and_adam(fitted):
    need_gpu()
    inst, ref = fitted
    x, y, off, deg = (dev(inst[k]) for k in ("x", "y", "fit_off", "degree"))
    box = dev(ref["box"])
    c0 = ref["coef"] * (1 + 1e-3 * np.random.default_rng(1).standard_normal(ref["coef"].shape))
    c = dev(c0).requires_grad_(True)
    loss = rp.RelMSE.apply(c, x, y, off, deg, box)
    loss.sum().backward()
    g2 = rp.rp_relmse_bwd(x, y, off, deg, dev(c0), box, torch.ones_like(loss))
    torch.testing.assert_close(c.grad, g2.double())
    # one Adam step equals the closed form
    p = dev(c0)
    m = torch.zeros(p.shape, dtype=torch.float32, device=p.device)
    v = torch.zeros(p.shape, dtype=torch.float32, device=p.device)
    mask = rp.refine_mask(deg)
    rp.rp_adam_step(p, g2, m, v, 1, lr=1e-3, mask=mask)
    gh, ph = host(g2).astype(np.float64), c0
    mh = 0.1 * gh
    vh = 0.001 * gh * gh
    expect = ph - 1e-3 * (mh / 0.1) / (np.sqrt(vh / 0.001) + 1e-8)
    mk = host(mask).astype(bool)
    np.testing.assert_allclose(host(p)[mk], expect[mk], rtol=1e-6, atol=1e-9)
    np.testing.assert_array_equal(host(p)[~mk], c0[~mk])
    # 20 refinement steps (default step) reduce the relative error of
    # perturbed fits
    p = dev(c0)
    l0, l1 = rp.refine_relmse(p, x, y, off, deg, box, steps=20)
    assert (host(l1) <= host(l0)).mean() > 0.9
