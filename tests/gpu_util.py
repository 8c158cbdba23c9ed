"""Helpers shared by the GPU parity tests (test code only)."""
import numpy as np
import pytest
import torch

import workloads as W

HW = W.HW_FIXED_DEFAULT


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_00142_gb300 import build
    build.build()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def eval_coef_at(coef_row, box_row, d, pts):
    """Evaluate p/q from coefficients in the normalised monomial basis at
    raw points (FP64, used to look at GPU outputs)."""
    e = W.exponents(d)
    lo, hi = box_row[0::2], box_row[1::2]
    span = np.where(hi > lo, hi - lo, 1.0)
    xn = np.where(hi > lo, 2.0 * (pts - lo) / span - 1.0, 0.0)
    phi = np.prod(xn[:, None, :] ** e[None, :, :], axis=2)
    nm = len(e)
    return (phi @ coef_row[:nm]) / (phi @ coef_row[35:35 + nm])


def predictions(coef, box, degree, x, fit_off):
    out = np.zeros(x.shape[1])
    for f in range(len(fit_off) - 1):
        a, b = fit_off[f], fit_off[f + 1]
        if b > a:
            out[a:b] = eval_coef_at(coef[f], box[f], int(degree[f]), x[:, a:b].T.astype(np.float64))
    return out


def per_fit_max(rel, fit_off):
    return np.array([rel[fit_off[f]:fit_off[f + 1]].max() if fit_off[f + 1] > fit_off[f] else 0.0
                     for f in range(len(fit_off) - 1)])


def program_to_device(prog):
    """Lay a program dict (aN, bN, grid_dims, table) out in the packed format."""
    import paper_1906_00142_gb300 as rp
    K = prog["aN"].shape[0]
    d = int(prog["d"])
    buf = torch.zeros(rp.rp_program_size(K, d), dtype=torch.uint8, device="cuda")
    aN, bN, gd, tab = rp.program_views(buf, K, d)
    aN.copy_(torch.from_numpy(prog["aN"]))
    bN.copy_(torch.from_numpy(prog["bN"]))
    gd.copy_(torch.from_numpy(prog["grid_dims"].astype(np.int32)))
    tab.copy_(torch.from_numpy(prog["table"].astype(np.float32)))
    return buf


def lin_objective(coef_row, box_row, d, pts, y, weighted=True):
    """Linearised least-squares objective sum_i w_i^2 (p_i - y_i q_i)^2 with
    (p, q) rescaled so that q averages to 1 over the samples (FP64)."""
    e = W.exponents(d)
    lo, hi = box_row[0::2], box_row[1::2]
    span = np.where(hi > lo, hi - lo, 1.0)
    xn = np.where(hi > lo, 2.0 * (pts - lo) / span - 1.0, 0.0)
    phi = np.prod(xn[:, None, :] ** e[None, :, :], axis=2)
    nm = len(e)
    p = phi @ coef_row[:nm]
    q = phi @ coef_row[35:35 + nm]
    s = q.mean()
    p, q = p / s, q / s
    w = 1.0 / np.abs(y) if weighted else 1.0
    return float(np.sum((w * (p - y * q)) ** 2))
