"""More GPU fit cases against the oracle: sample counts around the
shared-memory sample cache (512) and far beyond it, unweighted rows
(RP_FIT_UNWEIGHTED), and batches of a single degree 1 or 4."""
import numpy as np
import pytest

import oracle
import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import dev, host, lin_objective, need_gpu, per_fit_max, predictions
from test_gpu_fit import compare, gpu_fit

pytestmark = pytest.mark.gpu


def concat(insts):
    x = np.ascontiguousarray(np.concatenate([i["x"] for i in insts], 1))
    y = np.concatenate([i["y"] for i in insts])
    offs = [0]
    for i in insts:
        offs.extend(offs[-1] + np.diff(i["fit_off"]))
    deg = np.concatenate([i["degree"] for i in insts])
    return dict(x=x, y=y, fit_off=np.array(offs, np.int64), degree=deg)


@pytest.mark.parametrize("precision", ["fp32", "tf32", "fp64"])
def test_fit_sample_counts_around_and_beyond_the_cache(precision):
    need_gpu()
    insts = [W.batched_instance(1, seed=80 + k, m=mk, d=3, n_metrics=2)
             for k, mk in enumerate([26, 511, 512, 513, 2048, 20000])]
    inst = concat(insts)
    g = gpu_fit(inst, precision, degree=3)
    assert not (g["status"] & rp.RP_FIT_TIMEOUT).any()
    compare(inst, g, all_fits=(precision == "fp64"))


@pytest.mark.parametrize("d", [1, 4])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fit_single_degree_batches(d, precision):
    need_gpu()
    inst = W.batched_instance(6, seed=90 + d, m=512, d=d)
    g = gpu_fit(inst, precision, degree=d)
    compare(inst, g, all_fits=(precision == "fp64"))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fit_unweighted_rows(precision):
    """w_i = 1 (RP_FIT_UNWEIGHTED): the absolute linearised residual."""
    need_gpu()
    inst = W.batched_instance(6, seed=95, m=384, d=3)
    x, y, off, deg = inst["x"], inst["y"], inst["fit_off"], inst["degree"]
    out = rp.rp_fit(dev(x), dev(y), dev(off), 3, precision=precision, degrees=dev(deg),
                    weighted=False)
    g = {k: host(v) for k, v in out.items()}
    ref = oracle.fit(x, y, off, deg, weighted=False)
    sens = oracle.fit_sensitivity(x, y, off, deg, base=ref, weighted=False)
    np.testing.assert_array_equal(g["box"], ref["box"])
    for f in range(len(off) - 1):
        a, b = off[f], off[f + 1]
        pts = x[:, a:b].T.astype(np.float64)
        yy = y[a:b].astype(np.float64)
        og = lin_objective(g["coef"][f], g["box"][f], 3, pts, yy, weighted=False)
        oo = lin_objective(ref["coef"][f], ref["box"][f], 3, pts, yy, weighted=False)
        slack = 1e-10 + (0.0 if precision == "fp64" else (30.0 * sens[f]) ** 2)
        # unweighted residuals carry y's scale: the slack scales with mean y^2
        assert og <= oo * (1 + 1e-4) + slack * np.sum(yy ** 2), (f, og, oo, float(sens[f]))
    p_o = oracle.predict_samples(ref, x, off)
    p_g = predictions(g["coef"], g["box"], deg, x, off)
    err = per_fit_max(np.abs(p_g - p_o) / np.abs(p_o), off)
    gate = np.full(len(err), 1e-4) if precision == "fp64" else np.maximum(1e-4, 30.0 * sens)
    checked = np.ones(len(err), bool) if precision == "fp64" else sens < 1e-2
    assert (err[checked] <= gate[checked]).all(), (err, sens)
