"""Pins for the FP64 oracle's fit, pack and relative-MSE gradient.

Each check ties the oracle to something other than itself: exact recovery of
known rational functions from noise-free samples (Sec. 3.3 Step 2: exact
data determine g_i by interpolation), numpy's SVD / least squares on the
same matrices (a library routine, not the oracle's Jacobi code), brute
facts (permutation and scale invariance), finite differences, and the
paper's Table 3 rows for the Error % formula.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _truth_at_samples(inst):
    off = inst["fit_off"]
    return np.concatenate([t(inst["x"][:, off[f]:off[f + 1]].T.astype(float))
                           for f, t in enumerate(inst["truths"])])


def test_exact_recovery_tiny_lattice():
    """Integer-coefficient deg-2 rationals, 64 noise-free samples: the fit
    reproduces the true function at all 462 lattice points."""
    inst = W.tiny_instance()
    r = oracle.fit(inst["x"], inst["y64"], inst["fit_off"], inst["degree"])
    assert (r["status"] == 0).all() and (r["rank"] == 19).all()
    lat = inst["lattice"]
    for f, t in enumerate(inst["truths"]):
        p = oracle.predict(r["coef"][f], r["box"][f], 2, lat)
        assert np.max(np.abs(p - t(lat)) / np.abs(t(lat))) < 1e-9


@pytest.mark.parametrize("d", [2, 3])
def test_exact_recovery_positive_truths(d):
    inst = W.batched_instance(2, seed=11 + d, d=d, noise=0.0, m=256)
    r = oracle.fit(inst["x"], inst["y64"], inst["fit_off"], inst["degree"])
    pred = oracle.predict_samples(r, inst["x"], inst["fit_off"])
    tv = _truth_at_samples(inst)
    assert np.max(np.abs(pred - tv) / tv) < 1e-7
    # off-sample: the whole training lattice
    lat = W.lattice()
    for f, t in enumerate(inst["truths"]):
        p = oracle.predict(r["coef"][f], r["box"][f], d, lat)
        assert np.max(np.abs(p - t(lat)) / t(lat)) < 1e-5


def test_jacobi_svd_matches_numpy():
    rng = np.random.default_rng(0)
    for (m, n) in [(30, 7), (64, 19), (10, 12)]:
        A = rng.standard_normal((m, n)) * np.logspace(0, -6, n)[None, :]
        sv, sweeps = oracle.svd_values(A)
        ref = np.linalg.svd(A, compute_uv=False)
        k = min(m, n)
        assert sweeps > 0
        np.testing.assert_allclose(sv[:k], ref, rtol=1e-10, atol=1e-13 * ref[0])


def test_lstsq_min_norm_rank_deficient_matches_pinv():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 5)) @ rng.standard_normal((5, 9))   # rank 5
    b = rng.standard_normal(40)
    x, r = oracle.lstsq_svd(A, b, rcond=1e-10)
    assert r == 5
    np.testing.assert_allclose(x, np.linalg.pinv(A, rcond=1e-10) @ b, rtol=1e-9, atol=1e-11)


def test_lstsq_qr_matches_numpy_full_rank():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((50, 8))
    b = rng.standard_normal(50)
    np.testing.assert_allclose(oracle.lstsq_qr(A, b), np.linalg.lstsq(A, b, rcond=None)[0],
                               rtol=1e-11, atol=1e-12)


def test_weighted_polynomial_special_case_matches_numpy_lstsq():
    """When the data are a polynomial and the denominator part is removed
    the linearised problem is weighted polynomial least squares; here the
    rational fit of polynomial data must give exactly that polynomial
    (exact recovery through numpy's lstsq on a library Vandermonde)."""
    rng = np.random.default_rng(3)
    pts = W.lattice()[rng.choice(462, 120, replace=False)]
    lo, hi = pts.min(0), pts.max(0)
    xn = 2 * (pts - lo) / (hi - lo) - 1
    V = np.polynomial.polynomial.polyvander3d(xn[:, 0], xn[:, 1], xn[:, 2], [2, 2, 2])
    c = np.zeros(27)
    c[[0, 1, 3, 9]] = [3.0, 0.5, 0.25, 0.125]      # 3 + 0.5 B1' + 0.25 B0' + 0.125 N'
    y = V @ c + 0.3 * xn[:, 0] ** 2
    x = np.ascontiguousarray(pts.T)
    r = oracle.fit(x, y, np.array([0, len(y)]), [2])
    p = oracle.predict(r["coef"][0], r["box"][0], 2, pts)
    np.testing.assert_allclose(p, y, rtol=1e-10)
    # same numbers from numpy lstsq of the polynomial part alone
    keep = [0, 1, 3, 9, 18]  # 1, B1', B0', N', N'^2 in polyvander3d order
    sol = np.linalg.lstsq(V[:, keep] / y[:, None], np.ones_like(y), rcond=None)[0]
    np.testing.assert_allclose(V[:, keep] @ sol, y, rtol=1e-10)


def test_svd_and_qr_fits_agree_noisy():
    inst = W.batched_instance(2, seed=5)
    a = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    b = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"], method="qr")
    pa = oracle.predict_samples(a, inst["x"], inst["fit_off"])
    pb = oracle.predict_samples(b, inst["x"], inst["fit_off"])
    assert np.max(np.abs(pa - pb) / np.abs(pa)) < 1e-8


def test_noisy_fit_tracks_truth():
    inst = W.batched_instance(2, seed=6, noise=0.01)
    r = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    pred = oracle.predict_samples(r, inst["x"], inst["fit_off"])
    tv = _truth_at_samples(inst)
    assert np.median(np.abs(pred - tv) / tv) < 0.01
    assert (r["status"] & oracle.FS_POLE == 0).all()


def test_permutation_and_scale_invariance():
    inst = W.batched_instance(1, seed=7, n_metrics=2)
    x, y, off = inst["x"].astype(np.float64), inst["y"].astype(np.float64), inst["fit_off"]
    r0 = oracle.fit(x, y, off, inst["degree"])
    p0 = oracle.predict_samples(r0, x, off)
    perm = np.concatenate([off[f] + np.random.default_rng(f).permutation(off[f + 1] - off[f])
                           for f in range(len(off) - 1)])
    r1 = oracle.fit(x[:, perm], y[perm], off, inst["degree"])
    p1 = oracle.predict_samples(r1, x[:, perm], off)
    np.testing.assert_allclose(p1, p0[perm], rtol=1e-8)
    r2 = oracle.fit(x, 8.0 * y, off, inst["degree"])
    np.testing.assert_allclose(oracle.predict_samples(r2, x, off), 8.0 * p0, rtol=1e-8)


def test_mean_normalisation_of_denominator():
    """The homogeneous system is normalised by mean(q) = 1 over the fit's
    samples."""
    inst = W.batched_instance(1, seed=8, n_metrics=3)
    r = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    e = oracle.exponents(3)
    for f in range(3):
        a, b = inst["fit_off"][f], inst["fit_off"][f + 1]
        pts = inst["x"][:, a:b].T.astype(float)
        lo, hi = r["box"][f, 0::2], r["box"][f, 1::2]
        xn = 2 * (pts - lo) / (hi - lo) - 1
        phi = np.prod(xn[:, None, :] ** e[None], axis=2)
        q = phi @ r["coef"][f, 35:35 + len(e)]
        assert abs(q.mean() - 1.0) < 1e-10


def test_status_codes():
    x = np.array([[64.0, 128, 256], [1, 2, 4], [1, 1, 1]])
    y = np.array([1.0, -2.0, 3.0])
    r = oracle.fit(x, y, np.array([0, 3, 3]), [1, 1])
    assert r["status"][0] & oracle.FS_NONPOS_Y
    assert r["status"][1] & oracle.FS_EMPTY
    y2 = np.array([1.0, np.nan, 3.0])
    assert oracle.fit(x, y2, np.array([0, 3]), [1])["status"][0] & oracle.FS_NONFINITE


def test_pack_reproduces_trivariate_fit():
    """The B-specialised univariate table evaluated at t = aN*N + bN equals
    the fitted p/q at (N, B0, B1) for every configuration."""
    inst = W.batched_instance(2, seed=9)
    r = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    prog = oracle.pack(r["coef"], r["box"], r["degree"], inst["metric_map"], 3)
    Ns = np.array([64.0, 1000.0, 4096.0])
    for k in range(2):
        for mt in range(8):
            fi = inst["metric_map"][k, mt]
            for c, (b0, b1) in enumerate(W.CONFIGS):
                pts = np.stack([Ns, np.full(3, b0, float), np.full(3, b1, float)], 1)
                ref = oracle.predict(r["coef"][fi], r["box"][fi], 3, pts)
                t = prog["aN"][k, mt].astype(float) * Ns + prog["bN"][k, mt].astype(float)
                num = np.polynomial.polynomial.polyval(t, prog["table"][k, c, mt, 0].astype(float))
                den = np.polynomial.polynomial.polyval(t, prog["table"][k, c, mt, 1].astype(float))
                np.testing.assert_allclose(num / den, ref, rtol=2e-4)


def test_relmse_loss_and_gradient():
    inst = W.batched_instance(1, seed=10, n_metrics=2, m=128)
    x, y, off, deg = inst["x"], inst["y"], inst["fit_off"], inst["degree"]
    r = oracle.fit(x, y, off, deg)
    coef = r["coef"] * (1.0 + 0.01 * np.random.default_rng(0).standard_normal(r["coef"].shape))
    res = dict(r, coef=coef)
    loss, grad = oracle.relmse(x, y, off, deg, coef, r["box"])
    pred = oracle.predict_samples(res, x, off)
    for f in range(2):
        a, b = off[f], off[f + 1]
        ref = np.mean(((pred[a:b] - y[a:b]) / y[a:b]) ** 2)
        assert abs(loss[f] - ref) <= 1e-12 * ref
    # central differences, relative step 1e-6
    f = 0
    for j in [0, 3, 19, 36, 50]:
        h = 1e-6 * max(abs(coef[f, j]), 1e-3)
        cp, cm = coef.copy(), coef.copy()
        cp[f, j] += h
        cm[f, j] -= h
        lp, _ = oracle.relmse(x, y, off, deg, cp, r["box"])
        lm, _ = oracle.relmse(x, y, off, deg, cm, r["box"])
        fd = (lp[f] - lm[f]) / (2 * h)
        assert abs(fd - grad[f, j]) <= 1e-5 * max(abs(fd), 1e-8 * loss[f]), (j, fd, grad[f, j])
    assert grad[f, 35] == 0.0   # beta_0 frozen


def test_error_pct_table3_rows():
    g = json.load(open(os.path.join(GOLD, "error_pct_table3.json")))
    for row in g["rows"]:
        # the printed runtimes are rounded: propagate half a unit of the
        # last printed digit through the formula
        def ulp(v):
            s = f"{v}"
            dec = len(s.split(".")[1]) if "." in s else 0
            return 0.5 * 10.0 ** (-dec)
        c, bt, wt = row["C_rt"], row["B_t"], row["W_t"]
        vals = [oracle.error_pct(c + sc * ulp(c), bt + sb * ulp(bt), wt + sw * ulp(wt))
                for sc in (-1, 1) for sb in (-1, 1) for sw in (-1, 1)]
        mid = oracle.error_pct(c, bt, wt)
        lo, hi = min(vals + [mid]), max(vals + [mid])
        assert lo - 0.01 <= row["error_pct"] <= hi + 0.01, row
