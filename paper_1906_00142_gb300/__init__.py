"""GB300 rational-program library: Python binding of the C ABI in include/rp.h.

Argument marshalling only: every step of the fit, pack, search and
refinement runs in the CUDA kernels of ``librp.so`` (built in-tree for
sm_103a by ``paper_1906_00142_gb300.build``).  PyTorch provides device
memory and streams.  There is no CPU fallback: if the library or a CUDA
device is missing, calls raise.

Entry points (same names as the C ABI):
    rp_fit, rp_fit_workspace_size, rp_program_size, rp_program_pack,
    rp_eval_search, rp_search_workspace_size, rp_relmse_fwd, rp_relmse_bwd,
    rp_adam_step, rp_tune_fit, rp_tune_search, rp_fit_noalloc,
    rp_eval_search_tiebreak, rp_eval_occupancy, rp_error_pct, rp_codegen_source,
    rp_codegen_compile / rp_codegen_search / rp_codegen_free (GeneratedProgram),
    rp_strerror, rp_version
plus ``RelMSE`` (a torch.autograd.Function over rp_relmse_fwd/bwd) and
``refine_relmse`` (Adam steps with the hand-written backward).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librp.so")

RP_COEF_STRIDE = 70
RP_NUM_CONFIGS = 66
RP_NUM_METRICS = 8
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "tf32x3": 3, "bf16": 4, "bf16x3": 5}
RP_FIT_RANK_DEFICIENT, RP_FIT_NOT_CONVERGED, RP_FIT_POLE = 1, 2, 4
RP_FIT_NONFINITE, RP_FIT_NONPOS_Y, RP_FIT_EMPTY, RP_FIT_TIMEOUT, RP_FIT_ESCALATED = 8, 16, 32, 64, 128
RP_FIT_ITER_SHIFT, RP_FIT_ITER_MASK = 8, 0xFF00
RP_FIT_ACC_SHIFT, RP_FIT_ACC_MASK = 16, 0xFF0000
RP_FIT_FP64_PASS = 1 << 24
RP_Q_NO_VALID, RP_Q_POLE, RP_Q_BAD = 1, 2, 4
RP_EP_NO_RUNTIME, RP_EP_BAD_CHOICE = 1, 2
RP_FIT_UNWEIGHTED, RP_FIT_SOLVER_SVD = 1, 2


class RPError(RuntimeError):
    pass


class FitDesc(C.Structure):
    _fields_ = [("num_fits", C.c_int64), ("num_samples", C.c_int64), ("degree", C.c_int32),
                ("precision", C.c_int32), ("max_refine", C.c_int32), ("flags", C.c_int32),
                ("tol", C.c_double), ("degrees", C.c_void_p), ("point_off", C.c_void_p),
                ("num_points", C.c_int64), ("fits_per_point_set", C.c_int32),
                ("reserved", C.c_int32)]


class HwFixed(C.Structure):
    _fields_ = [("warp_size", C.c_int32), ("t_max", C.c_int32), ("b_max", C.c_int32),
                ("w_max", C.c_int32), ("r_sm", C.c_int32), ("z_sm", C.c_int32),
                ("issue_cycles", C.c_float), ("reserved", C.c_int32)]


HW_DEFAULT = dict(warp_size=32, t_max=1024, b_max=32, w_max=64, r_sm=65536, z_sm=58368,
                  issue_cycles=1.0)

_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load librp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RPError(f"{path} not built; run python -m paper_1906_00142_gb300.build")
            lib = C.CDLL(path)
            P, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
            lib.rp_fit_workspace_size.argtypes = [C.POINTER(FitDesc), C.POINTER(C.c_size_t)]
            lib.rp_fit_cache_workspace_size.argtypes = [C.POINTER(FitDesc), C.POINTER(C.c_size_t)]
            lib.rp_fit.argtypes = [C.POINTER(FitDesc), P, P, P, P, P, P, P, P, P, C.c_size_t, P]
            lib.rp_program_size.argtypes = [i64, i32]
            lib.rp_program_size.restype = C.c_size_t
            lib.rp_program_pack.argtypes = [i64, i32, P, P, P, P, P, P, C.c_size_t, P]
            lib.rp_eval_search.argtypes = [P, i64, i32, C.POINTER(HwFixed), P, i64, P, P, P, P, P,
                                           C.c_size_t, P]
            lib.rp_search_workspace_size.argtypes = [i64, i64, C.POINTER(C.c_size_t)]
            lib.rp_eval_search_tiebreak.argtypes = [P, i64, i32, C.POINTER(HwFixed), P, i64,
                                                    C.c_float, P, P, P, P, P, C.c_size_t, P]
            lib.rp_eval_occupancy.argtypes = [P, i64, i32, C.POINTER(HwFixed), P, i64, P, P, P, P]
            lib.rp_error_pct.argtypes = [P, P, i64, P, P, P]
            lib.rp_codegen_source.argtypes = [P, i64, i32, i64, C.POINTER(HwFixed), P,
                                              C.POINTER(C.c_size_t)]
            lib.rp_codegen_compile.argtypes = [C.c_char_p, C.POINTER(C.c_void_p), P, C.c_size_t]
            lib.rp_codegen_search.argtypes = [P, P, i64, P, P, P, P, P]
            lib.rp_codegen_free.argtypes = [P]
            lib.rp_relmse_fwd.argtypes = [i64, i64, P, P, P, P, P, P, P, P]
            lib.rp_relmse_bwd.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P]
            lib.rp_adam_step.argtypes = [i64, P, P, P, P, P, i32, C.c_float, C.c_float, C.c_float,
                                         C.c_float, P]
            lib.rp_fit_noalloc.argtypes = [C.POINTER(FitDesc), P, P, P, P, P, P, P, P, P]
            lib.rp_tune_search.argtypes = [P, i64, i32, C.POINTER(HwFixed), P, i64, P, P, P, P, P,
                                           C.c_size_t, P, C.POINTER(i32), C.POINTER(i32)]
            lib.rp_tune_fit.argtypes = [C.POINTER(FitDesc), P, P, P, P, P, P, P, P, P, C.c_size_t, P,
                                        C.POINTER(i32)]
            lib.rp_strerror.argtypes = [C.c_int]
            lib.rp_strerror.restype = C.c_char_p
            lib.rp_version.restype = C.c_int
            _lib = lib
    return _lib


def rp_version() -> int:
    return load_library().rp_version()


def rp_strerror(code: int) -> str:
    return load_library().rp_strerror(int(code)).decode()


def _check(rc: int, what: str):
    if rc != 0:
        raise RPError(f"{what}: {rp_strerror(rc)} ({rc})")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise RPError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise RPError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise RPError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _ptr_or_null(t, dtype, name):
    return C.c_void_p(0) if t is None else _dev(t, dtype, name)


def rp_fit_workspace_size(desc: FitDesc) -> int:
    b = C.c_size_t(0)
    _check(load_library().rp_fit_workspace_size(C.byref(desc), C.byref(b)), "rp_fit_workspace_size")
    return b.value


def rp_fit_cache_workspace_size(desc: FitDesc) -> int:
    b = C.c_size_t(0)
    _check(load_library().rp_fit_cache_workspace_size(C.byref(desc), C.byref(b)),
           "rp_fit_cache_workspace_size")
    return b.value


def _fit_args(x, y, fit_off, degree, precision, max_refine, tol, degrees, weighted, out,
              stream, schedule, point_off=None, fits_per_point_set=1, solver="sweep"):
    if solver not in ("sweep", "svd"):
        raise RPError(f"unknown solver {solver!r}")
    F = fit_off.numel() - 1
    S = y.numel()
    dev = y.device
    if out is None:
        out = dict(coef=torch.empty((F, RP_COEF_STRIDE), dtype=torch.float64, device=dev),
                   coef32=torch.empty((F, RP_COEF_STRIDE), dtype=torch.float32, device=dev),
                   box=torch.empty((F, 6), dtype=torch.float64, device=dev),
                   status=torch.empty(F, dtype=torch.int32, device=dev),
                   rank=torch.empty(F, dtype=torch.int32, device=dev))
    desc = FitDesc(F, S, int(degree), PREC[precision], int(max_refine),
                   (0 if weighted else RP_FIT_UNWEIGHTED) | (RP_FIT_SOLVER_SVD if solver == "svd" else 0),
                   float(tol),
                   _ptr_or_null(degrees, torch.int8, "degrees").value,
                   _ptr_or_null(point_off, torch.int64, "point_off").value,
                   x.shape[1] if point_off is not None else 0,
                   int(fits_per_point_set) if point_off is not None else 0, 0)
    st = torch.cuda.current_stream() if stream is None else stream
    ws_bytes = rp_fit_workspace_size(desc)
    ws = None
    if schedule == "dynamic" and ws_bytes:
        # the workspace with the basis cache (out["workspace"], kept there
        # for the next call with the same out)
        ws_bytes = rp_fit_cache_workspace_size(desc)
        ws = out.get("workspace")
        if ws is None or ws.numel() < ws_bytes:
            with torch.cuda.stream(st):        # stream-ordered reuse of the buffer
                ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
            out["workspace"] = ws
    elif schedule not in ("dynamic", "static"):
        raise RPError(f"unknown schedule {schedule!r}")
    args = (C.byref(desc), _dev(x, torch.float32, "x"), _dev(y, torch.float32, "y"),
            _dev(fit_off, torch.int64, "fit_off"), _dev(out["coef"], torch.float64, "coef"),
            _ptr_or_null(out.get("coef32"), torch.float32, "coef32"),
            _dev(out["box"], torch.float64, "box"), _dev(out["status"], torch.int32, "status"),
            _dev(out["rank"], torch.int32, "rank"),
            C.c_void_p(0 if ws is None else ws.data_ptr()),
            C.c_size_t(0 if ws is None else ws.numel()), C.c_void_p(st.cuda_stream))
    return out, args, ws


def rp_fit(x: torch.Tensor, y: torch.Tensor, fit_off: torch.Tensor, degree: int,
           precision: str = "fp32", max_refine: int = 8, tol: float = 1e-8,
           degrees: torch.Tensor | None = None, weighted: bool = True, out=None, stream=None,
           schedule: str = "dynamic", point_off: torch.Tensor | None = None,
           fits_per_point_set: int = 1, solver: str = "sweep"):
    """Batched rational least-squares fits (see rp_fit in include/rp.h).
    x: float32 [3, S], y: float32 [S], fit_off: int64 [F+1] (all CUDA); with
    point_off (int64 [P+1]) x is float32 [3, num_points] and each run of
    fits_per_point_set consecutive fits shares one point set.
    schedule "dynamic" (CTAs claim point sets from a counter in the 32-byte
    workspace, out["workspace"] or allocated here) or "static".  solver
    "sweep" (sweep operator with pivot dropping) or "svd" (Jacobi SVD of the
    design, truncated pseudo-inverse: RP_FIT_SOLVER_SVD).
    Returns dict(coef float64 [F,70], coef32 float32 [F,70], box float64 [F,6],
    status int32 [F], rank int32 [F])."""
    out, args, _ws = _fit_args(x, y, fit_off, degree, precision, max_refine, tol, degrees,
                               weighted, out, stream, schedule, point_off, fits_per_point_set,
                               solver)
    _check(load_library().rp_fit(*args), "rp_fit")
    return out


def rp_fit_noalloc(x, y, fit_off, degree: int, precision: str = "fp32", max_refine: int = 8,
                   tol: float = 1e-8, degrees=None, weighted: bool = True, out=None,
                   stream=None, point_off=None, fits_per_point_set: int = 1, solver="sweep"):
    """rp_fit with the library's static scratch instead of a workspace (see
    rp_fit_noalloc in include/rp.h); outputs as rp_fit."""
    out, args, _ws = _fit_args(x, y, fit_off, degree, precision, max_refine, tol, degrees,
                               weighted, out, stream, "static", point_off, fits_per_point_set,
                               solver)
    _check(load_library().rp_fit_noalloc(*args[:9], args[11]), "rp_fit_noalloc")
    return out


def rp_tune_fit(x, y, fit_off, degree: int, precision: str = "fp32", max_refine: int = 8,
                tol: float = 1e-8, degrees=None, weighted: bool = True, out=None, stream=None,
                schedule: str = "dynamic", point_off=None, fits_per_point_set: int = 1) -> int:
    """Time the fit kernel's grid sizes on these fits (see rp_tune_fit in
    include/rp.h); returns the CTAs per SM now used for this precision and
    degree.  Synchronises; call before any graph capture."""
    out, args, _ws = _fit_args(x, y, fit_off, degree, precision, max_refine, tol, degrees,
                               weighted, out, stream, schedule, point_off, fits_per_point_set)
    c = C.c_int32(0)
    _check(load_library().rp_tune_fit(*args, C.byref(c)), "rp_tune_fit")
    return c.value


def rp_program_size(num_kernels: int, degree: int) -> int:
    return load_library().rp_program_size(int(num_kernels), int(degree))


def rp_program_pack(coef, box, degrees, metric_map, grid_dims, degree: int, program=None,
                    stream=None):
    """Pack fitted metrics into the rational program's table (uint8 buffer)."""
    lib = load_library()
    K = metric_map.shape[0]
    nbytes = rp_program_size(K, degree)
    if program is None:
        program = torch.empty(nbytes, dtype=torch.uint8, device=coef.device)
    rc = lib.rp_program_pack(K, int(degree), _dev(coef, torch.float64, "coef"),
                             _dev(box, torch.float64, "box"), _dev(degrees, torch.int8, "degrees"),
                             _dev(metric_map, torch.int32, "metric_map"),
                             _dev(grid_dims, torch.int32, "grid_dims"),
                             _dev(program, torch.uint8, "program"), C.c_size_t(program.numel()),
                             _stream(stream))
    _check(rc, "rp_program_pack")
    return program


def program_views(program: torch.Tensor, num_kernels: int, degree: int):
    """(aN, bN, grid_dims, table) tensor views of a packed program buffer."""
    K = num_kernels

    def a16(v):
        return (v + 15) & ~15
    o1 = a16(4 * K * 8)
    o2 = o1 + a16(4 * K * 8)
    o3 = o2 + a16(4 * K)
    aN = program[0:4 * K * 8].view(torch.float32).view(K, 8)
    bN = program[o1:o1 + 4 * K * 8].view(torch.float32).view(K, 8)
    gd = program[o2:o2 + 4 * K].view(torch.int32)
    n = K * RP_NUM_CONFIGS * RP_NUM_METRICS * 2 * (degree + 1)
    tab = program[o3:o3 + 4 * n].view(torch.float32).view(K, RP_NUM_CONFIGS, RP_NUM_METRICS, 2,
                                                          degree + 1)
    return aN, bN, gd, tab


def hw_struct(hw=None) -> HwFixed:
    h = dict(HW_DEFAULT)
    if hw:
        h.update(hw)
    return HwFixed(h["warp_size"], h["t_max"], h["b_max"], h["w_max"], h["r_sm"], h["z_sm"],
                   float(h["issue_cycles"]), 0)


def rp_search_workspace_size(num_kernels: int, num_queries: int) -> int:
    """Bytes of rp_eval_search's optional workspace (0: the search runs
    unbucketed for these sizes)."""
    b = C.c_size_t(0)
    _check(load_library().rp_search_workspace_size(int(num_kernels), int(num_queries), C.byref(b)),
           "rp_search_workspace_size")
    return b.value


def _search_args(program, num_kernels, degree, queries, hw, out, stream, grouped):
    Q = queries.shape[0]
    dev = queries.device
    if out is None:
        out = dict(argmin=torch.empty(Q, dtype=torch.int32, device=dev),
                   best=torch.empty(Q, dtype=torch.float32, device=dev),
                   second=torch.empty(Q, dtype=torch.float32, device=dev),
                   status=torch.empty(Q, dtype=torch.int32, device=dev))
    st = torch.cuda.current_stream() if stream is None else stream
    ws = None
    ws_bytes = rp_search_workspace_size(num_kernels, Q) if grouped else 0
    if ws_bytes:
        ws = out.get("workspace")
        if ws is None or ws.numel() < ws_bytes:
            with torch.cuda.stream(st):        # stream-ordered reuse of the buffer
                ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    h = hw_struct(hw)
    args = (_dev(program, torch.uint8, "program"), int(num_kernels), int(degree), C.byref(h),
            _dev(queries, torch.float32, "queries"), Q, _dev(out["argmin"], torch.int32, "argmin"),
            _dev(out["best"], torch.float32, "best"), _dev(out["second"], torch.float32, "second"),
            _dev(out["status"], torch.int32, "status"),
            C.c_void_p(0 if ws is None else ws.data_ptr()),
            C.c_size_t(0 if ws is None else ws.numel()), C.c_void_p(st.cuda_stream))
    return out, args, (h, ws)


def rp_eval_search(program, num_kernels: int, degree: int, queries: torch.Tensor, hw=None,
                   out=None, stream=None, grouped: bool = True):
    """Evaluate-and-argmin for queries float32 [Q, 8] (CUDA).  grouped: bucket
    the queries by kernel first (workspace out["workspace"] or allocated
    here; used where rp_search_workspace_size is non-zero); False: each
    query reads its kernel's table from global memory.  Returns dict(argmin
    int32 [Q], best float32 [Q], second float32 [Q], status int32 [Q])."""
    out, args, _keep = _search_args(program, num_kernels, degree, queries, hw, out, stream, grouped)
    _check(load_library().rp_eval_search(*args), "rp_eval_search")
    return out


def rp_eval_search_tiebreak(program, num_kernels: int, degree: int, queries: torch.Tensor,
                            tie_rel: float, hw=None, out=None, stream=None, grouped: bool = True):
    """rp_eval_search with Step 5's second metric (see rp_eval_search_tiebreak
    in include/rp.h): among configurations within (1 + tie_rel) of the best,
    the one with the most active warps per SM."""
    out, args, _keep = _search_args(program, num_kernels, degree, queries, hw, out, stream, grouped)
    args = args[:6] + (C.c_float(tie_rel),) + args[6:]
    _check(load_library().rp_eval_search_tiebreak(*args), "rp_eval_search_tiebreak")
    return out


def rp_eval_occupancy(program, num_kernels: int, degree: int, queries: torch.Tensor, hw=None,
                      out=None, stream=None):
    """B_active and W_active of every configuration of every query (see
    rp_eval_occupancy in include/rp.h).  Returns dict(b_active int32 [Q, 66],
    w_active int32 [Q, 66], status int32 [Q])."""
    Q = queries.shape[0]
    dev = queries.device
    if out is None:
        out = dict(b_active=torch.empty((Q, RP_NUM_CONFIGS), dtype=torch.int32, device=dev),
                   w_active=torch.empty((Q, RP_NUM_CONFIGS), dtype=torch.int32, device=dev),
                   status=torch.empty(Q, dtype=torch.int32, device=dev))
    h = hw_struct(hw)
    _check(load_library().rp_eval_occupancy(
        _dev(program, torch.uint8, "program"), int(num_kernels), int(degree), C.byref(h),
        _dev(queries, torch.float32, "queries"), Q, _dev(out["b_active"], torch.int32, "b_active"),
        _dev(out["w_active"], torch.int32, "w_active"), _dev(out["status"], torch.int32, "status"),
        _stream(stream)), "rp_eval_occupancy")
    return out


def rp_error_pct(runtimes: torch.Tensor, choice: torch.Tensor, out=None, stream=None):
    """Error % (Sec. 5) of the chosen configuration of every query from
    measured runtimes float32 [Q, 66] and choices int32 [Q] (see rp_error_pct
    in include/rp.h).  Returns dict(err_pct float32 [Q], status int32 [Q])."""
    Q = choice.numel()
    dev = choice.device
    if out is None:
        out = dict(err_pct=torch.empty(Q, dtype=torch.float32, device=dev),
                   status=torch.empty(Q, dtype=torch.int32, device=dev))
    _check(load_library().rp_error_pct(
        _dev(runtimes, torch.float32, "runtimes"), _dev(choice, torch.int32, "choice"), Q,
        _dev(out["err_pct"], torch.float32, "err_pct"), _dev(out["status"], torch.int32, "status"),
        _stream(stream)), "rp_error_pct")
    return out


def rp_codegen_source(program_host, num_kernels: int, degree: int, kernel_id: int, hw=None) -> str:
    """CUDA source of one kernel's rational program with its coefficients
    written in (see rp_codegen_source in include/rp.h).  program_host: the
    packed program as a host buffer (numpy uint8 array or CPU uint8 tensor)."""
    import numpy as np
    buf = np.ascontiguousarray(program_host.numpy() if isinstance(program_host, torch.Tensor)
                               else program_host, dtype=np.uint8)
    h = hw_struct(hw)
    n = C.c_size_t(0)
    lib = load_library()
    ptr = C.c_void_p(buf.ctypes.data)
    _check(lib.rp_codegen_source(ptr, int(num_kernels), int(degree), int(kernel_id), C.byref(h),
                                 None, C.byref(n)), "rp_codegen_source")
    out = C.create_string_buffer(n.value)
    _check(lib.rp_codegen_source(ptr, int(num_kernels), int(degree), int(kernel_id), C.byref(h),
                                 out, C.byref(n)), "rp_codegen_source")
    return out.value.decode()


class GeneratedProgram:
    """A generated rational program compiled at run time (rp_codegen_compile);
    search() runs it on queries of its kernel (rp_codegen_search)."""

    def __init__(self, source: str):
        lib = load_library()
        self._h = C.c_void_p(0)
        log = C.create_string_buffer(1 << 16)
        rc = lib.rp_codegen_compile(source.encode(), C.byref(self._h), log, len(log))
        if rc != 0:
            raise RPError(f"rp_codegen_compile: {rp_strerror(rc)} ({rc}): {log.value.decode()[:2000]}")

    def search(self, queries: torch.Tensor, out=None, stream=None):
        Q = queries.shape[0]
        dev = queries.device
        if out is None:
            out = dict(argmin=torch.empty(Q, dtype=torch.int32, device=dev),
                       best=torch.empty(Q, dtype=torch.float32, device=dev),
                       second=torch.empty(Q, dtype=torch.float32, device=dev),
                       status=torch.empty(Q, dtype=torch.int32, device=dev))
        _check(load_library().rp_codegen_search(
            self._h, _dev(queries, torch.float32, "queries"), Q, _dev(out["argmin"], torch.int32, "argmin"),
            _dev(out["best"], torch.float32, "best"), _dev(out["second"], torch.float32, "second"),
            _dev(out["status"], torch.int32, "status"), _stream(stream)), "rp_codegen_search")
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rp_codegen_free(self._h)
            self._h = None


def rp_tune_search(program, num_kernels: int, degree: int, queries: torch.Tensor, hw=None,
                   out=None, stream=None, grouped: bool = True):
    """Time the search kernel's launch shapes on these queries (see
    rp_tune_search in include/rp.h); returns (threads per CTA, CTAs per SM)
    now used for this degree.  Synchronises; call before any graph capture."""
    out, args, _keep = _search_args(program, num_kernels, degree, queries, hw, out, stream, grouped)
    t, c = C.c_int32(0), C.c_int32(0)
    _check(load_library().rp_tune_search(*args, C.byref(t), C.byref(c)), "rp_tune_search")
    return t.value, c.value


def rp_relmse_fwd(x, y, fit_off, degrees, coef, box, loss=None, stream=None):
    lib = load_library()
    F = fit_off.numel() - 1
    if loss is None:
        loss = torch.empty(F, dtype=torch.float32, device=y.device)
    rc = lib.rp_relmse_fwd(F, y.numel(), _dev(x, torch.float32, "x"), _dev(y, torch.float32, "y"),
                           _dev(fit_off, torch.int64, "fit_off"), _dev(degrees, torch.int8, "degrees"),
                           _dev(coef, torch.float64, "coef"), _dev(box, torch.float64, "box"),
                           _dev(loss, torch.float32, "loss"), _stream(stream))
    _check(rc, "rp_relmse_fwd")
    return loss


def rp_relmse_bwd(x, y, fit_off, degrees, coef, box, grad_loss, grad=None, stream=None):
    lib = load_library()
    F = fit_off.numel() - 1
    if grad is None:
        grad = torch.empty((F, RP_COEF_STRIDE), dtype=torch.float32, device=y.device)
    rc = lib.rp_relmse_bwd(F, y.numel(), _dev(x, torch.float32, "x"), _dev(y, torch.float32, "y"),
                           _dev(fit_off, torch.int64, "fit_off"), _dev(degrees, torch.int8, "degrees"),
                           _dev(coef, torch.float64, "coef"), _dev(box, torch.float64, "box"),
                           _dev(grad_loss, torch.float32, "grad_loss"),
                           _dev(grad, torch.float32, "grad"), _stream(stream))
    _check(rc, "rp_relmse_bwd")
    return grad


def rp_adam_step(param, grad, m, v, t: int, lr=1e-6, beta1=0.9, beta2=0.999, eps=1e-8, mask=None,
                 stream=None):
    lib = load_library()
    rc = lib.rp_adam_step(param.numel(), _dev(param, torch.float64, "param"),
                          _dev(grad, torch.float32, "grad"), _dev(m, torch.float32, "m"),
                          _dev(v, torch.float32, "v"), _ptr_or_null(mask, torch.uint8, "mask"),
                          int(t), float(lr), float(beta1), float(beta2), float(eps), _stream(stream))
    _check(rc, "rp_adam_step")


class RelMSE(torch.autograd.Function):
    """Per-fit mean squared relative error of the FP64 coefficients coef
    [F, 70] with a hand-written CUDA backward (rp_relmse_fwd /
    rp_relmse_bwd); the gradient is computed in FP32 and returned as FP64."""

    @staticmethod
    def forward(ctx, coef, x, y, fit_off, degrees, box):
        ctx.save_for_backward(coef, x, y, fit_off, degrees, box)
        return rp_relmse_fwd(x, y, fit_off, degrees, coef.contiguous(), box)

    @staticmethod
    def backward(ctx, grad_loss):
        coef, x, y, fit_off, degrees, box = ctx.saved_tensors
        g = rp_relmse_bwd(x, y, fit_off, degrees, coef.contiguous(), box,
                          grad_loss.contiguous().float())
        return g.double(), None, None, None, None, None


def refine_mask(degrees: torch.Tensor) -> torch.Tensor:
    """uint8 [F, 70] mask of trainable coefficients: all alpha_j and beta_j
    (j >= 1) of each fit's degree; beta_0 frozen."""
    F = degrees.numel()
    nm = ((degrees.long() + 1) * (degrees.long() + 2) * (degrees.long() + 3) // 6).view(F, 1)
    j = torch.arange(35, device=degrees.device).view(1, 35)
    num = (j < nm)
    den = (j < nm) & (j >= 1)
    return torch.cat([num, den], 1).to(torch.uint8).contiguous()


def refine_relmse(coef, x, y, fit_off, degrees, box, steps=20, lr=1e-6, beta1=0.9,
                  beta2=0.999, eps=1e-8, stream=None):
    """Adam on the mean squared relative error, using the CUDA forward and
    backward kernels and the CUDA Adam update.  Updates the FP64 coefficients
    coef [F, 70] in place and returns the per-fit losses before and after.
    The default step suits the fitted monomial coefficients, which cancel
    heavily: Adam moves every coefficient by ~lr per step."""
    F = fit_off.numel() - 1
    dev = coef.device
    m = torch.zeros(coef.shape, dtype=torch.float32, device=dev)
    v = torch.zeros(coef.shape, dtype=torch.float32, device=dev)
    mask = refine_mask(degrees)
    ones = torch.ones(F, dtype=torch.float32, device=dev)
    grad = torch.empty(coef.shape, dtype=torch.float32, device=dev)
    loss0 = rp_relmse_fwd(x, y, fit_off, degrees, coef, box, stream=stream).clone()
    for t in range(1, steps + 1):
        rp_relmse_bwd(x, y, fit_off, degrees, coef, box, ones, grad=grad, stream=stream)
        rp_adam_step(coef, grad, m, v, t, lr, beta1, beta2, eps, mask=mask, stream=stream)
    loss1 = rp_relmse_fwd(x, y, fit_off, degrees, coef, box, stream=stream)
    return loss0, loss1
