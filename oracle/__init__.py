"""FP64 CPU oracle for the rational-program fit and MWP-CWP search.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg are the only users.  The product path (the CUDA
library and its binding) never imports this package.

The arithmetic lives in ``rp_oracle.c`` (plain C, FP64, one fit or query per
loop iteration, OpenMP only across independent fits/queries).  This module
builds it with gcc on first use and marshals numpy arrays.

Parity status per function (see the C header comment for the citations):
  fit / predict / pack / relmse -- pinned (exact recovery, library
      least-squares special cases, SVD vs QR, brute-force, finite
      differences).
  eval / search -- MWP-CWP formulas are not printed in the paper; pinned
      only by hand-worked examples, invariants and brute force
      ("parity unpinned" for the model constants and case details).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rp_oracle.c")
_SO = os.path.join(_HERE, "_rp_oracle.so")
_lock = threading.Lock()
_lib = None

COEF_STRIDE = 70          # alpha at [0, 35), beta at [35, 70)
NCFG, NMET = 66, 8

FS_RANK_DEFICIENT, FS_NOT_CONVERGED, FS_POLE = 1, 2, 4
FS_NONFINITE, FS_NONPOS_Y, FS_EMPTY = 8, 16, 32
QS_NO_VALID, QS_POLE, QS_BAD = 1, 2, 4
EV_INVALID, EV_POLE, EV_BADQ = -1, -2, -3


def build(force: bool = False) -> str:
    """Compile rp_oracle.c into _rp_oracle.so (gcc, -O2, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                                   _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_SO)
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        lib.rpo_fit.argtypes = [i64, P, P, P, i64, P, i32, dbl, i64, P, P, P, P]
        lib.rpo_fit_qr.argtypes = [i64, P, P, P, i64, P, i32, i64, P, P, P, P]
        lib.rpo_predict.argtypes = [i64, P, i32, P, i64, P, P]
        lib.rpo_relmse.argtypes = [i64, P, P, P, i64, P, P, i64, P, P, P]
        lib.rpo_pack.argtypes = [i64, i32, P, i64, P, P, P, P, P, P]
        lib.rpo_eval.argtypes = [i64, i32, P, P, P, P, P, i64, P, P, P, P, P, P]
        lib.rpo_search.argtypes = [i64, i32, P, P, P, P, P, i64, P, P, P, P, P]
        lib.rpo_svd_values.argtypes = [i32, i32, P, P]
        lib.rpo_lstsq_svd.argtypes = [i32, i32, P, P, dbl, P, C.POINTER(C.c_int)]
        lib.rpo_lstsq_qr.argtypes = [i32, i32, P, P, P]
        lib.rpo_exponents.argtypes = [i32, P]
        lib.rpo_set_threads.argtypes = [i32]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def set_threads(n: int) -> None:
    _load().rpo_set_threads(int(n))


def get_threads() -> int:
    return _load().rpo_get_threads()


def exponents(d: int) -> np.ndarray:
    nm = (d + 1) * (d + 2) * (d + 3) // 6
    e = np.zeros((nm, 3), np.int32)
    _load().rpo_exponents(d, _p(e))
    return e


def _fit_args(x, y, fit_off, degree):
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    off = np.ascontiguousarray(fit_off, np.int64)
    F = len(off) - 1
    deg = np.ascontiguousarray(np.broadcast_to(np.asarray(degree, np.int8), (F,)))
    return x, y, off, deg, F


def fit(x, y, fit_off, degree, weighted=True, rcond=1e-12, method="svd"):
    """Least-squares rational fits.  Returns dict(coef[F][70], box[F][6],
    rank[F], status[F]) in the normalised monomial basis."""
    lib = _load()
    x, y, off, deg, F = _fit_args(x, y, fit_off, degree)
    S = y.shape[0]
    coef = np.zeros((F, COEF_STRIDE))
    box = np.zeros((F, 6))
    rank = np.zeros(F, np.int32)
    status = np.zeros(F, np.int32)
    if method == "svd":
        rc = lib.rpo_fit(F, _p(off), _p(x), _p(y), S, _p(deg), int(weighted), float(rcond),
                         COEF_STRIDE, _p(coef), _p(box), _p(rank), _p(status))
    else:
        rc = lib.rpo_fit_qr(F, _p(off), _p(x), _p(y), S, _p(deg), int(weighted),
                            COEF_STRIDE, _p(coef), _p(box), _p(rank), _p(status))
    if rc != 0:
        raise ValueError("oracle fit: bad degree")
    return dict(coef=coef, box=box, rank=rank, status=status, degree=deg)


def predict(coef_row, box_row, d, pts):
    """Evaluate one fitted rational at raw points pts[P][3]."""
    pts = np.ascontiguousarray(pts, np.float64)
    out = np.zeros(len(pts))
    cr = np.ascontiguousarray(coef_row, np.float64)
    br = np.ascontiguousarray(box_row, np.float64)
    _load().rpo_predict(len(pts), _p(pts), int(d), _p(cr), COEF_STRIDE, _p(br), _p(out))
    return out


def predict_samples(res, x, fit_off):
    """Predictions of every fit at its own samples (concatenated)."""
    x = np.asarray(x, np.float64)
    out = np.zeros(x.shape[1])
    for f in range(len(fit_off) - 1):
        a, b = fit_off[f], fit_off[f + 1]
        if b > a:
            out[a:b] = predict(res["coef"][f], res["box"][f], res["degree"][f], x[:, a:b].T)
    return out


def relmse(x, y, fit_off, degree, coef, box):
    """Per-fit relative MSE and its gradient (beta_0 held fixed)."""
    lib = _load()
    x, y, off, deg, F = _fit_args(x, y, fit_off, degree)
    coef = np.ascontiguousarray(coef, np.float64)
    box = np.ascontiguousarray(box, np.float64)
    loss = np.zeros(F)
    grad = np.zeros((F, COEF_STRIDE))
    lib.rpo_relmse(F, _p(off), _p(x), _p(y), y.shape[0], _p(deg), _p(coef), COEF_STRIDE,
                   _p(box), _p(loss), _p(grad))
    return loss, grad


def pack(coef, box, degree, metric_map, d):
    """Program table from fitted coefficients: aN[K][8], bN[K][8],
    table[K][66][8][2][d+1] (FP32)."""
    lib = _load()
    mm = np.ascontiguousarray(metric_map, np.int32)
    K = mm.shape[0]
    coef = np.ascontiguousarray(coef, np.float64)
    box = np.ascontiguousarray(box, np.float64)
    deg = np.ascontiguousarray(degree, np.int8)
    aN = np.zeros((K, NMET), np.float32)
    bN = np.zeros((K, NMET), np.float32)
    table = np.zeros((K, NCFG, NMET, 2, d + 1), np.float32)
    rc = lib.rpo_pack(K, int(d), _p(coef), COEF_STRIDE, _p(box), _p(deg), _p(mm), _p(aN),
                      _p(bN), _p(table))
    if rc != 0:
        raise ValueError("oracle pack: fit degree exceeds table degree")
    return dict(aN=aN, bN=bN, table=table, d=d)


def _hw(hw):
    return np.array([hw["warp_size"], hw["t_max"], hw["b_max"], hw["w_max"], hw["r_sm"],
                     hw["z_sm"], hw["issue_cycles"]], np.float64)


def _prog_args(prog):
    aN = np.ascontiguousarray(prog["aN"], np.float32)
    bN = np.ascontiguousarray(prog["bN"], np.float32)
    tab = np.ascontiguousarray(prog["table"], np.float32)
    gd = np.ascontiguousarray(prog["grid_dims"], np.int32)
    return aN, bN, tab, gd, aN.shape[0], int(prog["d"])


def evaluate(prog, hw, queries):
    """Per (query, configuration): exec cycles (inf if invalid), case id,
    decision margin, Horner condition number, and the model's MWP, CWP,
    active-warp count Nw and active-block count B_active (NaN where not
    computed; B_active 0 where the block cannot be resident)."""
    lib = _load()
    aN, bN, tab, gd, K, d = _prog_args(prog)
    q = np.ascontiguousarray(queries, np.float32)
    Q = q.shape[0]
    ex = np.zeros((Q, NCFG))
    cs = np.zeros((Q, NCFG), np.int32)
    mg = np.zeros((Q, NCFG))
    cd = np.zeros((Q, NCFG))
    dg = np.zeros((Q, NCFG, 4))
    h = _hw(hw)
    lib.rpo_eval(K, d, _p(aN), _p(bN), _p(tab), _p(gd), _p(h), Q, _p(q), _p(ex), _p(cs),
                 _p(mg), _p(cd), _p(dg))
    return dict(exec=ex, case=cs, margin=mg, cond=cd, mwp=dg[..., 0], cwp=dg[..., 1],
                nw=dg[..., 2], bact=dg[..., 3])


def search(prog, hw, queries):
    """Exhaustive argmin per query: argmin (-1 if none valid), best and
    second-best exec cycles, status bits."""
    lib = _load()
    aN, bN, tab, gd, K, d = _prog_args(prog)
    q = np.ascontiguousarray(queries, np.float32)
    Q = q.shape[0]
    am = np.zeros(Q, np.int32)
    b1 = np.zeros(Q)
    b2 = np.zeros(Q)
    st = np.zeros(Q, np.int32)
    h = _hw(hw)
    lib.rpo_search(K, d, _p(aN), _p(bN), _p(tab), _p(gd), _p(h), Q, _p(q), _p(am), _p(b1),
                   _p(b2), _p(st))
    return dict(argmin=am, best=b1, second=b2, status=st)


def svd_values(A):
    A = np.ascontiguousarray(A, np.float64)
    m, n = A.shape
    sv = np.zeros(n)
    sw = _load().rpo_svd_values(m, n, _p(A), _p(sv))
    return sv, sw


def lstsq_svd(A, b, rcond=1e-12):
    A = np.ascontiguousarray(A, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    m, n = A.shape
    x = np.zeros(n)
    r = C.c_int(0)
    _load().rpo_lstsq_svd(m, n, _p(A), _p(b), float(rcond), _p(x), C.byref(r))
    return x, r.value


def lstsq_qr(A, b):
    A = np.ascontiguousarray(A, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    m, n = A.shape
    x = np.zeros(n)
    _load().rpo_lstsq_qr(m, n, _p(A), _p(b), _p(x))
    return x


def error_pct(c_rt, best_t, worst_t):
    """Error % of a chosen configuration (Sec. 5):
    (C_rt - Best_time) / (Worst_time - Best_time) * 100."""
    return (c_rt - best_t) / (worst_t - best_t) * 100.0


def search_tiebreak(prog, hw, queries, tie_rel):
    """Step 5 with a second metric (Sec. 3.3): the configurations whose exec
    cycles are at most (1 + tie_rel) times the smallest are optimal; of them
    the one with the most active warps per SM (W_active), lowest index among
    equals.  Returns argmin per query (-1 if none valid) and the oracle's
    evaluation (for exclusions near the threshold)."""
    ev = evaluate(prog, hw, queries)
    ex = ev["exec"]
    Q = ex.shape[0]
    arg = np.full(Q, -1, np.int32)
    for i in range(Q):
        best = np.min(ex[i])
        if not np.isfinite(best):
            continue
        opt = np.where(ex[i] <= best * (1.0 + tie_rel))[0]
        nw = ev["nw"][i, opt]
        arg[i] = opt[np.argmax(nw)]        # first maximum: lowest index among equals
    return arg, ev


def error_pct_table(runtimes, choice):
    """Error % (Sec. 5) of the chosen configuration of every query: with B and
    W the smallest and largest finite runtime of the query, (t[choice] - B) /
    (W - B) * 100, 0 when W == B; NaN when the query has no finite runtime or
    the choice is out of range or has none.  FP64, one query per step."""
    rt = np.asarray(runtimes, np.float64)
    ch = np.asarray(choice)
    out = np.full(len(ch), np.nan)
    for i in range(len(ch)):
        fin = rt[i][np.isfinite(rt[i])]
        c = int(ch[i])
        if len(fin) == 0 or c < 0 or c >= rt.shape[1] or not np.isfinite(rt[i, c]):
            continue
        b, w = fin.min(), fin.max()
        out[i] = error_pct(rt[i, c], b, w) if w > b else 0.0
    return out
