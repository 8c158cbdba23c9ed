"""More GPU fit cases against the oracle: sample counts around the
shared-memory sample cache (512) and far beyond it, unweighted rows
(RP_FIT_UNWEIGHTED), and batches of a single degree 1 or 4."""
import numpy as np
import pytest
import torch

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
    g = {k: host(v) for k, v in out.items() if k != "workspace"}
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
    g = {k: host(v) for k, v in out.items() if k != "workspace"}
    assert not (g["status"] & rp.RP_FIT_TIMEOUT).any()
    compare(inst, g)
    # a fit whose value count differs from its set's point count: empty
    out2 = rp.rp_fit(dev(xp[:, :-1].copy()), dev(inst["y"]), dev(inst["fit_off"]), d, precision=precision,
                     degrees=dev(inst["degree"]), point_off=dev(np.minimum(poff, xp.shape[1] - 1)),
                     fits_per_point_set=8)
    st = host(out2["status"])
    assert (st[-8:] & rp.RP_FIT_EMPTY).all()


@pytest.mark.parametrize("precision,degrees", [("fp32", None), ("tf32", None), ("fp32", (2, 3))])
def test_basis_cache_leaves_results_unchanged(precision, degrees):
    """The accurate passes' basis cache (a workspace of
    rp_fit_cache_workspace_size bytes) changes no output bit: the same fits
    with the cache (dynamic schedule) and without any workspace (static
    schedule, no cache), on shared point sets whose fits reuse the slab, and
    on sets whose fits have different degrees (the slab holds the set's
    degree-D basis, a lower-degree fit uses its leading part)."""
    need_gpu()
    if degrees is None:
        inst = W.batched_instance(24, seed=131, m=512, d=3)
    else:
        inst = W.batched_instance(24, seed=132, degree_choices=degrees, m_range=(64, 512))
    xp, poff = W.shared_points(inst)
    d = int(inst["degree"].max())
    args = (dev(xp), dev(inst["y"]), dev(inst["fit_off"]), d)
    kw = dict(precision=precision, degrees=dev(inst["degree"]), point_off=dev(poff), fits_per_point_set=8)
    cached = rp.rp_fit(*args, **kw)
    ws = cached["workspace"]
    assert ws.numel() >= 256 and ws.numel() == rp.rp_fit_cache_workspace_size(
        rp.FitDesc(len(inst["fit_off"]) - 1, len(inst["y"]), d, rp.PREC[precision], 8, 0, 1e-8, None))
    plain = rp.rp_fit(*args, schedule="static", **kw)
    for k in ("coef", "coef32", "box", "status", "rank"):
        assert torch.equal(cached[k], plain[k]), k
    acc = (host(cached["status"]) >> 16) & 255
    assert acc.max() >= 2          # later accurate passes of a claim read the slab


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fit_svd_solver(precision):
    """RP_FIT_SOLVER_SVD (the paper's solver, Sec. 4.2): Jacobi SVD of the
    equilibrated design with truncation, as first solution and
    preconditioner.  Every fit against the oracle as in the other fit tests,
    including rank-deficient lattice fits (fewer samples than unknowns; a
    constant thread-block dimension), which are compared on the objective
    (their least-squares solution is not unique); the ranks of those fits
    equal the oracle's."""
    need_gpu()
    base = W.batched_instance(3, seed=99, m=512, d=3)
    rng = np.random.default_rng(100)
    lat = W.lattice()
    pts = [lat[rng.choice(462, 24, replace=False)], lat[rng.choice(462, 200, replace=False)]]
    pts[1] = pts[1].copy()
    pts[1][:, 2] = 1.0                                  # B1 constant
    ys = [np.exp(rng.uniform(0, 2, len(p))) for p in pts]
    x = np.concatenate([base["x"]] + [p.T.astype(np.float32) for p in pts], 1)
    y = np.concatenate([base["y"]] + [v.astype(np.float32) for v in ys])
    off = np.concatenate([base["fit_off"], base["fit_off"][-1] + np.cumsum([len(v) for v in ys])])
    inst = dict(x=np.ascontiguousarray(x), y=y, fit_off=off.astype(np.int64),
                degree=np.concatenate([base["degree"], np.full(2, 3, np.int8)]))
    out = rp.rp_fit(dev(inst["x"]), dev(inst["y"]), dev(inst["fit_off"]), 3, precision=precision,
                    degrees=dev(inst["degree"]), solver="svd")
    g = {k: host(v) for k, v in out.items() if k != "workspace"}
    ref = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    compare(inst, g, ref)
    rd = (ref["status"] & oracle.FS_RANK_DEFICIENT) != 0
    assert rd[-2:].all()
    assert (g["rank"][rd] == ref["rank"][rd]).all(), (g["rank"][rd], ref["rank"][rd])
    assert ((g["status"][rd] & rp.RP_FIT_RANK_DEFICIENT) != 0).all()
