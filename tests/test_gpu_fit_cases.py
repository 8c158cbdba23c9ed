"""More GPU fit cases against the oracle: sample counts around the
shared-memory sample cache (512) and far beyond it, unweighted rows
(RP_FIT_UNWEIGHTED), and batches of a single degree 1 or 4."""
import numpy as np
import pytest

import oracle
import paper_1906_00142_gb300 as rp
import workloads as W
from gpu_util import dev, host, need_gpu
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
    compare(inst, g)


@pytest.mark.parametrize("d", [1, 4])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fit_single_degree_batches(d, precision):
    need_gpu()
    inst = W.batched_instance(6, seed=90 + d, m=512, d=d)
    g = gpu_fit(inst, precision, degree=d)
    compare(inst, g)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fit_unweighted_rows(precision):
    """w_i = 1 (RP_FIT_UNWEIGHTED): the absolute linearised residual."""
    need_gpu()
    inst = W.batched_instance(6, seed=95, m=384, d=3)
    x, y, off, deg = inst["x"], inst["y"], inst["fit_off"], inst["degree"]
    out = rp.rp_fit(dev(x), dev(y), dev(off), 3, precision=precision, degrees=dev(deg),
                    weighted=False)
    g = {k: host(v) for k, v in out.items()}
    compare(inst, g, weighted=False)


@pytest.mark.parametrize("precision,degrees", [("fp32", None), ("tf32", None), ("fp64", None),
                                               ("fp32", (2, 3, 4))])
def test_fit_shared_point_sets(precision, degrees):
    """The metrics of a kernel share their sample points (x stored once per
    kernel, point_off): the box, marginal polynomials and whitening are
    computed once per set, at the set's largest degree; every fit against
    the oracle, boxes equal to the per-fit layout's."""
    need_gpu()
    if degrees is None:
        inst = W.batched_instance(6, seed=97, m=512, d=3)
    else:
        inst = W.batched_instance(6, seed=98, degree_choices=degrees, m_range=(64, 1500))
    xp, poff = W.shared_points(inst)
    d = int(inst["degree"].max())
    out = rp.rp_fit(dev(xp), dev(inst["y"]), dev(inst["fit_off"]), d, precision=precision,
                    degrees=dev(inst["degree"]), point_off=dev(poff), fits_per_point_set=8)
    g = {k: host(v) for k, v in out.items()}
    assert not (g["status"] & rp.RP_FIT_TIMEOUT).any()
    compare(inst, g)
    # a fit whose value count differs from its set's point count: empty
    out2 = rp.rp_fit(dev(xp[:, :-1].copy()), dev(inst["y"]), dev(inst["fit_off"]), d, precision=precision,
                     degrees=dev(inst["degree"]), point_off=dev(np.minimum(poff, xp.shape[1] - 1)),
                     fits_per_point_set=8)
    st = host(out2["status"])
    assert (st[-8:] & rp.RP_FIT_EMPTY).all()
