"""Benchmark: the rational-program hot path on GB300.

One step = the whole path over one batch of synthetic input:
  rp_fit          8192 fits (1024 kernels x 8 metrics), 512 samples each,
                  total degree <= 3 (20 + 20 monomials), lognormal noise 1%
  rp_program_pack the 1024 kernels' programs (66 configurations x 8 metrics)
  rp_eval_search  1e6 queries x 66 configurations, per-query argmin
Metric: rational fits/s of the whole step (the step's queries/s is reported
beside it), timed over a stream of steps: step k+1's fit runs on a
high-priority stream while step k's pack and search run on a second one
(three buffer sets; the serial step time is reported beside it).  Inputs are
resident in HBM before timing; L2 is flushed (160 MiB write, inside the
timed region) before each step's fit.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rational fits/s and MWP-CWP evals/s (argmin queries/s), batched vs plain, at stated tol"
N_KERNELS, N_METRICS, M_SAMPLES, DEGREE = 1024, 8, 512, 3
N_QUERIES = 1_000_000
SEED = 20190602
# rp_fit settings of the timed step (the full-size parity test runs the same)
BENCH_TOL, BENCH_MAX_REFINE = 1e-8, 16
WORKLOAD = ("batched fit 1024 kernels x 8 metrics (the metrics of a kernel share its 512 sample "
            "points), deg<=3, then MWP-CWP search 1e6 queries x 66 configs")


# DRAM bytes per fit of the fit kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of fit_kernel<float, 3, 0>,
# 2048 fits of 512 samples in the shared-point layout; traffic scales with
# the fit count), valid only for the kernel sources they were taken on
# (SHA-256 of the files below) and that layout.
FIT_TRAFFIC = {"sources_sha256": "9acbc2561a56b06c2fb9041ae7b1e02fb4b25b0537a0dbc0ca92fe0f700b006c",
               "bytes_per_fit": (6259968 + 2311680) / 2048, "layout": "shared point sets"}
FIT_SOURCES = ("paper_1906_00142_gb300/csrc/rp_fit_kernel.cuh", "paper_1906_00142_gb300/csrc/rp_fit.cuh",
               "paper_1906_00142_gb300/csrc/rp_fit_f32.cu", "paper_1906_00142_gb300/csrc/rp_tc.cuh")


def fit_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in FIT_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak_tflops(sm_count, sm_mhz):
    # 128 FP32 lanes per SM, an FMA counts 2 flops
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12


def search_flops_per_query(d):
    # per (query, configuration): 8 metrics x (2 Horner polynomials of degree d
    # in FMA = 4d flops, 1 division) + 36 flops of MWP-CWP arithmetic;
    # per query: 8 affine maps of N (16 flops)
    return 66 * (8 * (4 * d + 1) + 36) + 16


def fit_flops_per_fit(m, d):
    # the augmented Gram product, symmetric: m * n_aug * (n_aug + 1) flops
    nm = (d + 1) * (d + 2) * (d + 3) // 6
    naug = 2 * nm
    return m * naug * (naug + 1)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.idx = gpu_index

    def start(self):
        try:
            self.path = f"/tmp/rp_clocks_{os.getpid()}.csv"
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), active=parts[4],
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (read-only queries)
    every 2 ms from a background thread during a region; None if NVML is not
    available (the nvidia-smi sampler is used instead)."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, gpu_index):
        import ctypes
        import threading
        self.ok = False
        self.rows = []
        self._stop = threading.Event()
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(self.h)) != 0:
                return
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
            mx = ctypes.c_uint(0)
            lib.nvmlDeviceGetMaxClockInfo(self.h, ctypes.c_int(1), ctypes.byref(mx))
            self.max_mhz = float(mx.value)
            self.lib, self.ct = lib, ctypes
            self.ok = True
        except Exception:
            self.ok = False

    def _run(self):
        ct = self.ct
        mhz, rs = ct.c_uint(0), ct.c_ulonglong(0)
        while not self._stop.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, ct.c_int(1), ct.byref(mhz)) == 0 and \
                    self.reasons_fn(self.h, ct.byref(rs)) == 0:
                self.rows.append((float(mhz.value), int(rs.value)))
            time.sleep(0.002)

    def start(self):
        import threading
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()

    def stop(self):
        self._stop.set()
        self.t.join()
        if not self.rows:
            return None
        reasons = sorted({name for _, r in self.rows for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(m for m, _ in self.rows), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(self.rows), "source": "nvml, 2 ms"}


def dist_setup(ngpus):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def rank_seed(rank):
    """Each rank draws its own fits and queries (weak scaling: the per-rank
    workload is the same size at every N)."""
    return SEED + 1000 * rank


def max_over_ranks(value, ws, device):
    """The largest of the ranks' values (torch.distributed all-reduce MAX)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, units_per_rank, ms_per_step):
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return ws * units_per_rank / (ms_per_step / 1e3)


def workload_config(precision, tol=BENCH_TOL, max_refine=BENCH_MAX_REFINE):
    return {"workload": WORKLOAD, "fits": N_KERNELS * N_METRICS, "samples_per_fit": M_SAMPLES,
            "degree": DEGREE, "queries": N_QUERIES, "configs": 66, "precision": precision,
            "tol": tol, "max_refine": max_refine,
            "l2": "flushed (160 MiB write, inside the timed region) before each step's fit"}


def make_inputs(seed):
    import workloads as W
    inst = W.batched_instance(N_KERNELS, seed=seed, m=M_SAMPLES, d=DEGREE)
    q = W.queries(N_QUERIES, N_KERNELS, seed=seed + 1)
    gd = (np.arange(N_KERNELS) % 2 + 1).astype(np.int32)
    return inst, q, gd


# --------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)

def oracle_rates(inst, q, gd, budget_s=20.0):
    """Time the oracle on bounded samples of the workload; returns per-unit
    seconds for fit, pack (per kernel) and search, plus what was sampled."""
    import oracle
    import workloads as W
    ncores = os.cpu_count() or 1
    oracle.set_threads(ncores)
    off = inst["fit_off"]
    # fits: whole kernels (8 fits) at a time until ~budget/2
    t0 = time.perf_counter()
    nk = 0
    res = []
    while time.perf_counter() - t0 < budget_s * 0.45 and nk < N_KERNELS:
        k1 = min(N_KERNELS, nk + max(1, ncores // 2))
        a, b = off[nk * N_METRICS], off[k1 * N_METRICS]
        sub_off = off[nk * N_METRICS:k1 * N_METRICS + 1] - a
        r = oracle.fit(inst["x"][:, a:b], inst["y"][a:b], sub_off, inst["degree"][nk * N_METRICS:k1 * N_METRICS])
        res.append(r)
        nk = k1
    t_fit = time.perf_counter() - t0
    coef = np.concatenate([r["coef"] for r in res])
    box = np.concatenate([r["box"] for r in res])
    deg = np.concatenate([r["degree"] for r in res])
    mm = np.arange(nk * N_METRICS, dtype=np.int32).reshape(nk, N_METRICS)
    t0 = time.perf_counter()
    prog = oracle.pack(coef, box, deg, mm, DEGREE)
    t_pack = time.perf_counter() - t0
    prog["grid_dims"] = gd[:nk]
    # queries: those of the sampled kernels, until ~budget/2
    kid = W.query_kernel_ids(q)
    qs = q[kid < nk]
    t0 = time.perf_counter()
    nq = 0
    chunk = 20000
    while time.perf_counter() - t0 < budget_s * 0.45 and nq < len(qs):
        oracle.search(prog, W.HW_FIXED_DEFAULT, qs[nq:nq + chunk])
        nq += min(chunk, len(qs) - nq)
    t_search = time.perf_counter() - t0
    nf = nk * N_METRICS
    step_s = (t_fit / nf) * N_KERNELS * N_METRICS + (t_pack / nk) * N_KERNELS + \
        (t_search / max(nq, 1)) * N_QUERIES
    full = nf == N_KERNELS * N_METRICS and nq == N_QUERIES
    sample = (f"{nf} fits ({nk} kernels), pack of {nk} kernels, {nq} queries; " +
              ("the whole step" if full else
               f"scaled to {N_KERNELS * N_METRICS} fits + {N_QUERIES} queries per step"))
    return dict(step_s=step_s, cores=oracle.get_threads(), sample=sample,
                wall_s=t_fit + t_pack + t_search, scaled=not full,
                fit_s=t_fit / nf, search_s=t_search / max(nq, 1),
                fits=dict(coef=coef, box=box, degree=deg, n=nf), queries_idx=np.where(kid < nk)[0][:nq],
                search=oracle.search(prog, W.HW_FIXED_DEFAULT, qs[:min(nq, 20000)]))


def _pq(coef_row, box_row, d, pts):
    """p(x)/q(x) of coefficients in the box-normalised monomial basis at raw
    points (FP64; to compare the GPU's fits with the oracle's)."""
    import workloads as W
    e = W.exponents(d)
    lo, hi = box_row[0::2], box_row[1::2]
    span = np.where(hi > lo, hi - lo, 1.0)
    xn = np.where(hi > lo, 2.0 * (pts - lo) / span - 1.0, 0.0)
    phi = np.prod(xn[:, None, :] ** e[None, :, :], axis=2)
    return (phi @ coef_row[:len(e)]), (phi @ coef_row[35:35 + len(e)])


def fit_errors(inst, coef, box, ref):
    """Per fit: the largest relative difference between the GPU's and the
    oracle's predictions p/q at the fit's own samples, and the GPU's
    linearised objective (q normalised to mean 1) relative to the oracle's
    optimum minus 1 (FP64; fits of one degree and sample count in chunks)."""
    import workloads as W
    off = inst["fit_off"]
    F = len(off) - 1
    err, excess = np.zeros(F), np.zeros(F)
    deg = inst["degree"]
    counts = np.diff(off)
    uniform = (deg == deg[0]).all() and (counts == counts[0]).all()
    step = 256 if uniform else 1
    for f0 in range(0, F, step):
        f1 = min(F, f0 + step)
        d, m = int(deg[f0]), int(counts[f0])
        e = W.exponents(d)
        nm = len(e)
        pts = inst["x"][:, off[f0]:off[f1]].astype(np.float64).reshape(3, f1 - f0, m).transpose(1, 2, 0)
        y = inst["y"][off[f0]:off[f1]].astype(np.float64).reshape(f1 - f0, m)
        out = {}
        for name, c, b in (("g", coef[f0:f1], box[f0:f1]), ("o", ref["coef"][f0:f1], ref["box"][f0:f1])):
            lo, hi = b[:, None, 0::2], b[:, None, 1::2]
            span = np.where(hi > lo, hi - lo, 1.0)
            xn = np.where(hi > lo, 2.0 * (pts - lo) / span - 1.0, 0.0)
            phi = np.prod(xn[:, :, None, :] ** e[None, None, :, :], axis=3)
            pv = np.einsum("fij,fj->fi", phi, c[:, :nm])
            qv = np.einsum("fij,fj->fi", phi, c[:, 35:35 + nm])
            sc = qv.mean(axis=1, keepdims=True)
            out[name] = (pv / qv, np.sum(((pv - y * qv) / sc / y) ** 2, axis=1))
        err[f0:f1] = np.max(np.abs(out["g"][0] - out["o"][0]) / np.abs(out["o"][0]), axis=1)
        excess[f0:f1] = out["g"][1] / out["o"][1] - 1.0
    return err, excess


def parity_against_oracle(inst, q, r, g, ref):
    """The timed steps' GPU results against the oracle: every fit (predictions
    and least-squares objective, pole flags), and the argmin of the queries of
    the cpu_baseline sample (GPU program from the GPU's fits against the
    oracle's program from the oracle's fits)."""
    err, excess = fit_errors(inst, g["coef"], g["box"], ref)
    pole_g = (g["status"] & 4) != 0
    pole_o = (ref["status"] & 4) != 0
    s = r["search"]
    idx = r["queries_idx"][:len(s["argmin"])]
    with np.errstate(invalid="ignore", divide="ignore"):   # +inf second (one valid config)
        gap_o = (s["second"] - s["best"]) / s["best"]
    ga = g["argmin"][idx]
    out = {"fits": int(len(err)), "pred_rel_err_median": float(np.median(err)),
           "pred_rel_err_p99": float(np.percentile(err, 99)), "pred_rel_err_max": float(err.max()),
           "fits_within_1e-4": float((err <= 1e-4).mean()),
           "objective_excess_max": float(excess.max()),
           "pole_flags_equal": bool((pole_g == pole_o).all()), "oracle_pole_fits": int(pole_o.sum()),
           "queries": int(len(idx))}
    for gap in (1e-5, 1e-3):
        dec = gap_o > gap
        out[f"argmin_agree_gap_{gap:g}"] = float((ga[dec] == s["argmin"][dec]).mean()) if dec.any() else None
        out[f"decisive_gap_{gap:g}"] = int(dec.sum())
    out["note"] = ("all fits of the timed step against the oracle's fits of the same inputs; argmin: "
                   "GPU program from GPU fits vs oracle program from oracle fits, where the "
                   "oracle's top-two gap exceeds the stated relative gap")
    return out


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    inst, q, gd = make_inputs(SEED)
    per_step = max(5.0, 150.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rates(inst, q, gd, budget_s=min(per_step, 5.0))
    times, walls, scaled = [], [], False
    last = None
    for _ in range(args.steps):
        last = oracle_rates(inst, q, gd, budget_s=per_step)
        times.append(last["step_s"])
        walls.append(last["wall_s"])
        scaled = scaled or last["scaled"]
    step_s = statistics.mean(times)
    value = N_KERNELS * N_METRICS / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "fits/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.precision, args.tol, args.max_refine),
            "queries_per_s": N_QUERIES / step_s,
            "cpu_baseline": {"value": value, "unit": "fits/s", "cores": last["cores"],
                             "kind": "oracle", "sample": last["sample"],
                             "scaled_to_full_step": scaled},
            # ms_per_step is the time of one whole step at the rates each
            # step's sample measured (scaled up when the sample is smaller
            # than the step); the wall time each step actually took:
            "sample_wall_s_per_step": statistics.mean(walls),
            "e2e": {"value": value, "unit": "fits/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------

def _timed(fn, reps, flush, stream):
    """Mean device time (ms) of fn() over reps calls, L2 flushed before each."""
    import torch
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.mean(ts)


def extra_measurements(rp, args, inst, x, x_full, FK, y, off, deg, mm, gd, q, fit_out, prog, s_out, flush,
                       stream, step, fit_ms, search_ms, step_ms):
    """Fit-only rates per precision; the plain form (FP64 fits and single
    queries, one per launch, no tensor cores) on a sample, and the batched
    form's speedup over it; the step replayed from a CUDA graph."""
    import torch
    F = N_KERNELS * N_METRICS
    out = {}
    rates, escal = {}, {}
    for prec in ("fp32", "tf32", "tf32x3", "bf16", "bf16x3", "fp64"):
        mr = 16 if prec == "bf16" else 8
        fn = lambda: rp.rp_fit(x, y, off, DEGREE, precision=prec, max_refine=mr, tol=args.tol,
                               degrees=deg, out=fit_out, stream=stream, **FK)
        fn()
        rates[prec] = F / (_timed(fn, 3, flush, stream) / 1e3)
        st = fit_out["status"].cpu().numpy()
        escal[prec] = float(((st & rp.RP_FIT_ESCALATED) != 0).mean())
    out["fit_only_fits_per_s"] = rates
    out["fit_escalated_frac"] = escal
    # the whole step with the TF32 tensor-core design Gram (BASELINE config 2's
    # precision): timed like the FP32 step; its fits are kept for the parity
    # check against the oracle
    tf32_out = {k: torch.empty_like(v) for k, v in fit_out.items()}

    def step_tf32():
        rp.rp_fit(x, y, off, DEGREE, precision="tf32", max_refine=args.max_refine, tol=args.tol,
                  degrees=deg, out=tf32_out, stream=stream, **FK)
        rp.rp_program_pack(tf32_out["coef"], tf32_out["box"], deg, mm, gd, DEGREE, program=prog,
                           stream=stream)
        rp.rp_eval_search(prog, N_KERNELS, DEGREE, q, out=s_out, stream=stream)
    step_tf32()
    t_tf32 = _timed(step_tf32, 3, flush, stream)
    out["tf32_step"] = {"ms_per_step": t_tf32, "fits_per_s": F / (t_tf32 / 1e3),
                        "queries_per_s": N_QUERIES / (t_tf32 / 1e3),
                        "escalated_frac": float(((tf32_out["status"].cpu().numpy() &
                                                  rp.RP_FIT_ESCALATED) != 0).mean())}
    out["_tf32_fits"] = {k: tf32_out[k].cpu().numpy() for k in ("coef", "box", "status")}
    # the SVD route (RP_FIT_SOLVER_SVD: Jacobi SVD of the design instead of
    # the sweep operator) on the same fits, FP32 design: fit-only rate; its
    # fits are kept for the parity check
    svd_out = {k: torch.empty_like(v) for k, v in fit_out.items()}
    fn_svd = lambda: rp.rp_fit(x, y, off, DEGREE, precision=args.precision, max_refine=args.max_refine,
                               tol=args.tol, degrees=deg, out=svd_out, stream=stream, solver="svd", **FK)
    fn_svd()
    t_svd = _timed(fn_svd, 3, flush, stream)
    out["svd_solver"] = {"fit_ms": t_svd, "fit_only_fits_per_s": F / (t_svd / 1e3),
                         "fp64_pass_frac": float(((svd_out["status"].cpu().numpy() >> 24) & 1).mean())}
    out["_svd_fits"] = {k: svd_out[k].cpu().numpy() for k in ("coef", "box", "status")}
    # the generated rational program (Sec. 3.3 Step 3): kernel 0's program
    # written out with its coefficients as constants, compiled at run time,
    # against the table-driven search on 1e6 queries of that kernel
    try:
        t0 = time.perf_counter()
        gen = rp.GeneratedProgram(rp.rp_codegen_source(prog.cpu(), N_KERNELS, DEGREE, 0))
        t_compile = time.perf_counter() - t0
        q0 = q.clone()
        q0[:, 7] = torch.zeros(1, dtype=torch.int32, device=q.device).view(torch.float32)
        g_out = gen.search(q0)
        t_out = rp.rp_eval_search(prog, N_KERNELS, DEGREE, q0)
        t_gen = _timed(lambda: gen.search(q0, out=g_out), 3, flush, stream)
        t_tab = _timed(lambda: rp.rp_eval_search(prog, N_KERNELS, DEGREE, q0, out=t_out), 3, flush, stream)
        out["codegen"] = {"kernel": 0, "queries": int(q0.shape[0]), "compile_s": t_compile,
                          "generated_ms": t_gen, "table_ms": t_tab,
                          "results_equal": bool(all(torch.equal(g_out[k], t_out[k])
                                                    for k in ("argmin", "best", "second", "status")))}
        del gen
    except Exception as e:   # reported, never silently replaced
        out["codegen"] = {"error": str(e).splitlines()[0][:300]}
    # restore the FP32 step's program and search results for what follows
    step()
    torch.cuda.synchronize()
    # plain form: one FP64 fit per launch over 64 fits, one query per launch
    # over 2000 queries (launch-bound; rates scale to any count)
    n_pf, n_pq = 64, 2000
    offs = torch.stack([off[:-1], off[1:]], 1).contiguous()
    pf_out = {k: v for k, v in fit_out.items()}

    def plain_fits():
        for f in range(n_pf):
            rp.rp_fit(x_full, y, offs[f], DEGREE, precision="fp64", max_refine=args.max_refine, tol=args.tol,
                      degrees=deg[f:f + 1], stream=stream, schedule="static",
                      out={k: v[f:f + 1] for k, v in pf_out.items() if k != "workspace"})

    def plain_queries():
        for i in range(n_pq):
            rp.rp_eval_search(prog, N_KERNELS, DEGREE, q[i:i + 1], stream=stream,
                              out={k: v[i:i + 1] for k, v in s_out.items()})
    plain_fits()
    plain_queries()
    t_pf = _timed(plain_fits, 2, flush, stream)
    t_pq = _timed(plain_queries, 2, flush, stream)
    plain = {"fits_per_s": n_pf / (t_pf / 1e3), "queries_per_s": n_pq / (t_pq / 1e3),
             "sample": f"{n_pf} FP64 fits and {n_pq} queries, one per launch"}
    out["plain"] = plain
    out["speedup_vs_plain"] = {"fit": rates["fp32"] / plain["fits_per_s"],
                               "search": (N_QUERIES / (search_ms / 1e3)) / plain["queries_per_s"]}
    # the whole step captured in one CUDA graph
    try:
        s2 = torch.cuda.Stream()
        s2.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s2):
            step(st=s2)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s2):
            step(st=s2)
        g.replay()
        torch.cuda.synchronize()
        out["graph_ms_per_step"] = _timed(lambda: g.replay(), 5, flush, torch.cuda.current_stream())
    except Exception as e:   # reported, never silently replaced
        out["graph_ms_per_step"] = None
        out["graph_error"] = str(e).splitlines()[0]
    return out


def _timed_plain(fn, reps, stream):
    """Mean device time (ms) of fn() over reps back-to-back calls (one
    untimed call first)."""
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def workload_tiny(rp, dev, stream):
    """The plain FP64 tiny case: 4 fits of 64 noise-free lattice samples
    (degree 2), pack, one query over the 66 configurations; latency per call
    and parity against the oracle (predictions on the 462-point lattice,
    argmin of the query)."""
    import torch
    import oracle
    import workloads as W
    inst = W.tiny_instance()
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, y, off, deg = (td(inst[k]) for k in ("x", "y", "fit_off", "degree"))
    mm_np = np.full((1, 8), -1, np.int32)
    mm_np[0, :4] = np.arange(4)
    mm, gd = td(mm_np), torch.tensor([2], dtype=torch.int32, device=dev)
    q_np = np.zeros((1, 8), np.float32)
    q_np[0, W.Q_N], q_np[0, W.Q_NSM], q_np[0, W.Q_FGHZ], q_np[0, W.Q_MEMLD] = 4096, 120, 1.6, 600
    q_np[0, W.Q_BW], q_np[0, W.Q_DDC], q_np[0, W.Q_DDU] = 4500, 10.5, 10.5
    q = td(q_np)
    out = rp.rp_fit(x, y, off, 2, precision="fp64", degrees=deg, stream=stream)
    prog = rp.rp_program_pack(out["coef"], out["box"], deg, mm, gd, 2, stream=stream)
    s_out = rp.rp_eval_search(prog, 1, 2, q, stream=stream)

    def call():
        rp.rp_fit(x, y, off, 2, precision="fp64", degrees=deg, out=out, stream=stream)
        rp.rp_program_pack(out["coef"], out["box"], deg, mm, gd, 2, program=prog, stream=stream)
        rp.rp_eval_search(prog, 1, 2, q, out=s_out, stream=stream)
    ms = _timed_plain(call, 50, stream)
    ref = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
    coef, box = out["coef"].cpu().numpy(), out["box"].cpu().numpy()
    lat = inst["lattice"].astype(np.float64)
    err = 0.0
    for f in range(4):
        pg, qg = _pq(coef[f], box[f], 2, lat)
        po, qo = _pq(ref["coef"][f], ref["box"][f], 2, lat)
        err = max(err, float(np.max(np.abs(pg / qg - po / qo) / np.abs(po / qo))))
    prog_o = oracle.pack(ref["coef"], ref["box"], ref["degree"], mm_np, 2)
    prog_o["grid_dims"] = np.array([2], np.int32)
    so = oracle.search(prog_o, W.HW_FIXED_DEFAULT, q_np)
    return {"workload": "tiny FP64: 4 fits x 64 samples (deg 2), pack, 1 query x 66 configs",
            "us_per_call": ms * 1e3, "launches_per_call": 3,
            "parity": {"lattice_pred_rel_err_max": err,
                       "argmin_equal": bool(int(s_out["argmin"].item()) == int(so["argmin"][0])),
                       "oracle_top_two_gap": float((so["second"][0] - so["best"][0]) / so["best"][0])}}


def workload_diff(rp, dev, stream):
    """4096 degree-3 fits of 512 samples: 20 Adam steps on the mean squared
    relative error (forward, hand-written backward, Adam); fit-steps/s, and
    the gradient at the linearised optimum against the oracle's on 16 fits."""
    import torch
    import oracle
    import workloads as W
    inst = W.batched_instance(512, seed=20190604, m=512, d=3)
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, y, off, deg = (td(inst[k]) for k in ("x", "y", "fit_off", "degree"))
    fit = rp.rp_fit(x, y, off, 3, precision="fp32", degrees=deg, tol=BENCH_TOL, stream=stream)
    c0 = fit["coef"].clone()
    F = len(inst["fit_off"]) - 1
    loss0 = rp.rp_relmse_fwd(x, y, off, deg, c0, fit["box"]).cpu().numpy()
    c = c0.clone()
    ms = _timed_plain(lambda: (c.copy_(c0), rp.refine_relmse(c, x, y, off, deg, fit["box"], steps=20)),
                      3, stream)
    loss1 = rp.rp_relmse_fwd(x, y, off, deg, c, fit["box"]).cpu().numpy()
    grad = rp.rp_relmse_bwd(x, y, off, deg, c0, fit["box"], torch.ones(F, device=dev)).cpu().numpy()
    pick = np.arange(0, F, F // 16)
    sub_off = np.concatenate([[0], np.cumsum(np.diff(inst["fit_off"])[pick])])
    xs = np.concatenate([inst["x"][:, inst["fit_off"][f]:inst["fit_off"][f + 1]] for f in pick], 1)
    ys = np.concatenate([inst["y"][inst["fit_off"][f]:inst["fit_off"][f + 1]] for f in pick])
    _, g_o = oracle.relmse(xs, ys, sub_off, inst["degree"][pick], c0.cpu().numpy()[pick],
                           fit["box"].cpu().numpy()[pick])
    gerr = float(max(np.max(np.abs(grad[f] - g_o[i])) / np.max(np.abs(g_o[i])) for i, f in enumerate(pick)))
    return {"workload": "4096 fits x 512 samples (deg 3), 20 Adam steps on the relative MSE "
                        "(forward, hand-written backward, Adam) + 2 loss evaluations",
            "ms_per_20_steps": ms, "fit_steps_per_s": F * 20 / (ms / 1e3),
            "parity": {"loss_lowered_frac": float((loss1 < loss0).mean()),
                       "grad_rel_err_max_vs_oracle": gerr, "grad_fits_checked": int(len(pick))}}


def workload_uneven(rp, dev, stream, precision="fp32"):
    """8192 fits of 64..4096 samples (log-uniform) and degree 2..4; pack;
    1e7 queries; fit -> pack -> search replayed from one CUDA graph; parity of
    64 sampled fits against the oracle."""
    import torch
    import oracle
    import workloads as W
    K = 1024
    inst = W.batched_instance(K, seed=20190605, degree_choices=(2, 3, 4), m_range=(64, 4096))
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x, y, off, deg = (td(inst[k]) for k in ("x", "y", "fit_off", "degree"))
    mm = td(inst["metric_map"])
    gd = torch.full((K,), 2, dtype=torch.int32, device=dev)
    qn = 10_000_000
    q = td(W.queries(qn, K, seed=20190606))
    F = len(inst["fit_off"]) - 1
    mr = 16 if precision.startswith("bf16") else BENCH_MAX_REFINE
    out = rp.rp_fit(x, y, off, 4, precision=precision, degrees=deg, max_refine=mr, tol=BENCH_TOL,
                    stream=stream)
    prog = rp.rp_program_pack(out["coef"], out["box"], deg, mm, gd, 4, stream=stream)
    s_out = rp.rp_eval_search(prog, K, 4, q, stream=stream)
    s_out["workspace"] = torch.empty(rp.rp_search_workspace_size(K, qn), dtype=torch.uint8, device=dev)
    s2 = torch.cuda.Stream()

    def step(st):
        rp.rp_fit(x, y, off, 4, precision=precision, degrees=deg, out=out, stream=st, max_refine=mr,
                  tol=BENCH_TOL)
        rp.rp_program_pack(out["coef"], out["box"], deg, mm, gd, 4, program=prog, stream=st)
        rp.rp_eval_search(prog, K, 4, q, out=s_out, stream=st)
    s2.wait_stream(stream)
    with torch.cuda.stream(s2):
        step(s2)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s2):
        step(s2)
    ms = _timed_plain(lambda: g.replay(), 5, stream)
    fit_ms = _timed_plain(lambda: rp.rp_fit(x, y, off, 4, precision=precision, degrees=deg, out=out,
                                            max_refine=mr, tol=BENCH_TOL, stream=stream), 3, stream)
    search_ms = _timed_plain(lambda: rp.rp_eval_search(prog, K, 4, q, out=s_out, stream=stream), 3,
                             stream)
    st = out["status"].cpu().numpy()
    pick = np.sort(np.random.default_rng(7).choice(F, 64, replace=False))
    sub = {"x": np.ascontiguousarray(np.concatenate(
               [inst["x"][:, inst["fit_off"][f]:inst["fit_off"][f + 1]] for f in pick], 1)),
           "y": np.concatenate([inst["y"][inst["fit_off"][f]:inst["fit_off"][f + 1]] for f in pick]),
           "fit_off": np.concatenate([[0], np.cumsum(np.diff(inst["fit_off"])[pick])]).astype(np.int64),
           "degree": inst["degree"][pick]}
    ref = oracle.fit(sub["x"], sub["y"], sub["fit_off"], sub["degree"])
    err, excess = fit_errors(sub, out["coef"].cpu().numpy()[pick], out["box"].cpu().numpy()[pick], ref)
    # fits the oracle reports rank deficient (e.g. degree 4 with fewer samples
    # than its 69 unknowns) have no unique p/q: compared on the objective only
    rd = (ref["status"] & 1) != 0
    return {"workload": f"{F} fits, 64..4096 samples (log-uniform, {len(inst['y'])} in all), deg 2..4; "
                        "pack; 1e7 queries x 66 configs; one CUDA graph",
            "precision": precision, "graph_ms": ms, "fits_per_s": F / (ms / 1e3),
            "queries_per_s": qn / (ms / 1e3), "fit_ms": fit_ms, "search_ms": search_ms,
            "escalated_frac": float(((st & rp.RP_FIT_ESCALATED) != 0).mean()),
            "fp64_pass_frac": float(((st >> 24) & 1).mean()),
            "parity": {"fits_checked": int(len(pick)), "oracle_rank_deficient": int(rd.sum()),
                       "pred_rel_err_max": float(err[~rd].max()),
                       "fits_within_1e-4": float((err[~rd] <= 1e-4).mean()),
                       "objective_excess_max": float(excess.max())}}


def run_secondary(args):
    """--workload tiny|diff|uneven: one of the path's other stated workloads
    on its own (the default run reports all three under "workloads")."""
    import torch
    import paper_1906_00142_gb300 as rp
    from paper_1906_00142_gb300 import build as rpbuild
    rpbuild.build()
    rp.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    fn = {"tiny": workload_tiny, "diff": workload_diff, "uneven": workload_uneven}[args.workload]
    print(json.dumps(fn(rp, dev, stream)))


def main():
    global N_KERNELS, N_QUERIES
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tol", type=float, default=BENCH_TOL)
    ap.add_argument("--max-refine", type=int, default=BENCH_MAX_REFINE)
    ap.add_argument("--kernels", type=int, default=N_KERNELS,
                    help="smaller workloads for profiling captures only")
    ap.add_argument("--queries", type=int, default=N_QUERIES)
    ap.add_argument("--only", default="all", choices=["all", "fit", "search"],
                    help="profiling captures: launch only one phase per step")
    ap.add_argument("--no-tune", action="store_true", help="built-in launch shapes")
    ap.add_argument("--workload", default="step", choices=["step", "tiny", "diff", "uneven"],
                    help="step: the benchmarked fit + pack + search step; the others measure the "
                         "path's other stated workloads")
    ap.add_argument("--per-fit-points", action="store_true",
                    help="x carries every fit's points (no shared point sets)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the per-precision, plain-form and graph measurements")
    args = ap.parse_args()
    if args.workload != "step":
        run_secondary(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    N_KERNELS, N_QUERIES = args.kernels, args.queries
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import workloads as W
    ws, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1906_00142_gb300 import build as rpbuild
    if rank == 0:
        rpbuild.build()
    if ws > 1:
        torch.distributed.barrier()
    import paper_1906_00142_gb300 as rp
    rp.load_library()

    inst, q_np, gd_np = make_inputs(rank_seed(rank))
    F = N_KERNELS * N_METRICS
    td = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    # the metrics of a kernel share its sample points: x holds each kernel's
    # points once (point_off), unless --per-fit-points
    if args.per_fit_points:
        x_np, poff_np = inst["x"], None
    else:
        x_np, poff_np = W.shared_points(inst)
    x, y, off, deg = td(x_np), td(inst["y"]), td(inst["fit_off"]), td(inst["degree"])
    x_full = td(inst["x"]) if poff_np is not None else x
    FK = {} if poff_np is None else {"point_off": td(poff_np), "fits_per_point_set": N_METRICS}
    mm, gd, q = td(inst["metric_map"]), td(gd_np), td(q_np)
    fit_out = dict(coef=torch.empty((F, 70), dtype=torch.float64, device=dev),
                   coef32=torch.empty((F, 70), dtype=torch.float32, device=dev),
                   box=torch.empty((F, 6), dtype=torch.float64, device=dev),
                   status=torch.empty(F, dtype=torch.int32, device=dev),
                   rank=torch.empty(F, dtype=torch.int32, device=dev),
                   workspace=torch.zeros(32, dtype=torch.uint8, device=dev))
    # the fit's workspace with the basis cache of the accurate passes (the
    # binding sizes it with rp_fit_cache_workspace_size on the first call,
    # outside the timed region, and keeps it in fit_out)
    prog = torch.empty(rp.rp_program_size(N_KERNELS, DEGREE), dtype=torch.uint8, device=dev)
    s_ws = rp.rp_search_workspace_size(N_KERNELS, N_QUERIES)   # queries bucketed by kernel
    s_out = dict(argmin=torch.empty(N_QUERIES, dtype=torch.int32, device=dev),
                 best=torch.empty(N_QUERIES, dtype=torch.float32, device=dev),
                 second=torch.empty(N_QUERIES, dtype=torch.float32, device=dev),
                 status=torch.empty(N_QUERIES, dtype=torch.int32, device=dev),
                 workspace=torch.empty(s_ws, dtype=torch.uint8, device=dev))
    # kernels per step: fit, pack; search: bucket count, scan, scatter and
    # the grouped kernel (one kernel when the sizes select the direct path)
    search_launches = 4 if s_ws > 0 else 1
    # L2 flush: a 160 MiB write (the L2 holds 126.5 MiB) before each step's fit
    flush = torch.empty(160 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None, st=None):
        st = stream if st is None else st
        if ev:
            ev[0].record(st)
        if args.only in ("all", "fit"):
            rp.rp_fit(x, y, off, DEGREE, precision=args.precision, max_refine=args.max_refine, tol=args.tol,
                      degrees=deg, out=fit_out, stream=st, **FK)
        if ev:
            ev[1].record(st)
        if args.only in ("all", "fit"):
            rp.rp_program_pack(fit_out["coef"], fit_out["box"], deg, mm, gd, DEGREE, program=prog,
                               stream=st)
        if ev:
            ev[2].record(st)
        if args.only in ("all", "search"):
            rp.rp_eval_search(prog, N_KERNELS, DEGREE, q, out=s_out, stream=st)
        if ev:
            ev[3].record(st)

    if args.only == "search":   # program from one fit + pack, outside the timed steps
        rp.rp_fit(x, y, off, DEGREE, precision=args.precision, max_refine=args.max_refine, tol=args.tol,
                  degrees=deg, out=fit_out, stream=stream, **FK)
        rp.rp_program_pack(fit_out["coef"], fit_out["box"], deg, mm, gd, DEGREE, program=prog,
                           stream=stream)

    # launch shapes chosen by the library's autotuner on this workload
    # (outside the timed region; the tuned shapes are what the steps use)
    tuned = {}
    if not args.no_tune:
        if args.only in ("all", "fit"):
            tuned["fit_ctas_per_sm"] = rp.rp_tune_fit(x, y, off, DEGREE, precision=args.precision,
                                                      max_refine=args.max_refine, tol=args.tol, degrees=deg,
                                                      out=fit_out, stream=stream, **FK)
        rp.rp_program_pack(fit_out["coef"], fit_out["box"], deg, mm, gd, DEGREE, program=prog,
                           stream=stream)
        if args.only in ("all", "search"):
            t, c = rp.rp_tune_search(prog, N_KERNELS, DEGREE, q, out=s_out, stream=stream)
            tuned["search_threads"], tuned["search_ctas_per_sm"] = t, c

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = NvmlSampler(torch.cuda.current_device())
    if not clocks.ok:
        clocks = ClockSampler(torch.cuda.current_device())
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    fit_ms = [e[0].elapsed_time(e[1]) for e in evs]
    pack_ms = [e[1].elapsed_time(e[2]) for e in evs]
    search_ms = [e[2].elapsed_time(e[3]) for e in evs]
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    serial_ms_per_step = max_over_ranks(sum(step_ms), ws, dev) / args.steps

    # The headline: the same steps as a stream of batches on two compute
    # streams.  Step k's fit runs on the fit stream; its pack and search run
    # on the evaluation stream once the fit is done, while step k+1's fit
    # starts on the fit stream (three sets of fit outputs, programs and search
    # outputs).  The search of step k then fills the SMs that step k+1's fit
    # has not yet taken and those the FP64 launch of a step leaves idle.
    # Every step does all of its work; L2 is flushed before each fit (the
    # flush is inside the timed region).  With copies=True every step also
    # copies its inputs in (pinned host buffers, a copy stream, ahead of its
    # fit) and its results out (a second copy stream) inside the timed region.
    NB = 3   # three buffer sets: a step's copy-in need not wait for the search two steps back
    p_fit = [fit_out] + [{k: torch.empty_like(v) for k, v in fit_out.items()} for _ in range(NB - 1)]
    p_srch = [s_out] + [{k: torch.empty_like(v) for k, v in s_out.items()} for _ in range(NB - 1)]
    p_prog = [prog] + [torch.empty_like(prog) for _ in range(NB - 1)]
    # the fit stream has the higher priority: its CTAs are dispatched first,
    # so each step's fit -> FP64-launch chain runs at full speed and the
    # evaluation stream's CTAs fill the SMs it leaves free
    s_fit, s_eval = torch.cuda.Stream(priority=-1), torch.cuda.Stream()
    copy_in, copy_out = torch.cuda.Stream(), torch.cuda.Stream()
    pipe_io = {}

    def pipelined(nsteps, copies=False):
        pack_done, eval_done, out_done = [None] * NB, [None] * NB, [None] * NB
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_fit.wait_stream(stream)
        start.record(s_fit)
        for s_ in (s_eval, copy_in, copy_out):
            s_.wait_event(start)
        for k in range(nsteps):
            b = k % NB
            fo, so, pg = p_fit[b], p_srch[b], p_prog[b]
            if copies:
                di, ho, h = pipe_io["in"][b], pipe_io["out"][b], pipe_io["h"]
                if eval_done[b] is not None:      # step k - NB has read input set b
                    copy_in.wait_event(eval_done[b])
                with torch.cuda.stream(copy_in):
                    for key in h:
                        di[key].copy_(h[key], non_blocking=True)
                in_done = torch.cuda.Event()
                in_done.record(copy_in)
                s_fit.wait_event(in_done)
                ix, iy, ioff, ideg, imm, igd, iq = (di[k2] for k2 in ("x", "y", "off", "deg", "mm", "gd", "q"))
                ifk = pipe_io["fk"](di)
            else:
                ix, iy, ioff, ideg, imm, igd, iq, ifk = x, y, off, deg, mm, gd, q, FK
            if pack_done[b] is not None:          # step k - NB's pack has read fit set b
                s_fit.wait_event(pack_done[b])
            if out_done[b] is not None:           # and its status was read back
                s_fit.wait_event(out_done[b])
            with torch.cuda.stream(s_fit):
                flush.zero_()
            rp.rp_fit(ix, iy, ioff, DEGREE, precision=args.precision, max_refine=args.max_refine,
                      tol=args.tol, degrees=ideg, out=fo, stream=s_fit, **ifk)
            fit_done = torch.cuda.Event()
            fit_done.record(s_fit)
            s_eval.wait_event(fit_done)
            if out_done[b] is not None:           # step k - NB's search results read back
                s_eval.wait_event(out_done[b])
            rp.rp_program_pack(fo["coef"], fo["box"], ideg, imm, igd, DEGREE, program=pg, stream=s_eval)
            pack_done[b] = torch.cuda.Event()
            pack_done[b].record(s_eval)
            rp.rp_eval_search(pg, N_KERNELS, DEGREE, iq, out=so, stream=s_eval)
            eval_done[b] = torch.cuda.Event()
            eval_done[b].record(s_eval)
            if copies:
                copy_out.wait_event(eval_done[b])
                with torch.cuda.stream(copy_out):
                    ho["status"].copy_(fo["status"], non_blocking=True)
                    ho["argmin"].copy_(so["argmin"], non_blocking=True)
                    ho["best"].copy_(so["best"], non_blocking=True)
                out_done[b] = torch.cuda.Event()
                out_done[b].record(copy_out)
        for ev in eval_done + out_done:
            if ev is not None:
                s_fit.wait_event(ev)
        end.record(s_fit)
        stream.wait_stream(s_fit)
        torch.cuda.synchronize()
        return start.elapsed_time(end) / nsteps

    if args.only == "all":
        pipelined(NB + 1)                         # warm-up of the two-stream schedule
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        pipe_ms = pipelined(args.steps)
    else:                                         # profiling captures of one phase: serial steps
        pipe_ms = serial_ms_per_step
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    ms_per_step = max_over_ranks(pipe_ms, ws, dev)
    value = job_rate(ws, F, ms_per_step)
    # the pipelined steps reproduce the serial steps' results
    if args.only == "all":
        assert all(torch.equal(p_srch[b]["argmin"], p_srch[0]["argmin"]) for b in range(NB)), \
            "pipelined argmin mismatch"

    # the timed steps' results, kept for the comparison with the oracle
    g_res = {"coef": fit_out["coef"].cpu().numpy(), "box": fit_out["box"].cpu().numpy(),
             "status": fit_out["status"].cpu().numpy(),
             "argmin": s_out["argmin"].cpu().numpy(), "best": s_out["best"].cpu().numpy(),
             "second": s_out["second"].cpu().numpy()}

    # fit status summary (informational)
    st = fit_out["status"].cpu().numpy()
    fit_ok = float(((st & (rp.RP_FIT_POLE | rp.RP_FIT_EMPTY | rp.RP_FIT_NONFINITE)) == 0).mean())

    # end to end through the public API with pinned host buffers
    h = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
         for k, v in dict(x=x_np, y=inst["y"], off=inst["fit_off"], deg=inst["degree"],
                          mm=inst["metric_map"], gd=gd_np, q=q_np,
                          **({} if poff_np is None else {"poff": poff_np})).items()}
    fk_dev = lambda d: {} if poff_np is None else {"point_off": d["poff"],
                                                    "fits_per_point_set": N_METRICS}
    h_out = dict(argmin=torch.empty(N_QUERIES, dtype=torch.int32).pin_memory(),
                 best=torch.empty(N_QUERIES, dtype=torch.float32).pin_memory(),
                 status=torch.empty(F, dtype=torch.int32).pin_memory())
    d_in = {k: torch.empty_like(v, device=dev) for k, v in h.items()}
    h2d = sum(v.numel() * v.element_size() for v in h.values())
    d2h = sum(v.numel() * v.element_size() for v in h_out.values())

    side = torch.cuda.Stream()

    def e2e_step():
        # the queries travel on a second stream while the fit runs, and the
        # fit status returns while pack and search run; every copy lies
        # between the step's start and end on the main stream
        start = torch.cuda.Event()
        start.record(stream)
        side.wait_event(start)
        with torch.cuda.stream(side):
            d_in["q"].copy_(h["q"], non_blocking=True)
        q_ready = torch.cuda.Event()
        q_ready.record(side)
        for k in h:
            if k != "q":
                d_in[k].copy_(h[k], non_blocking=True)
        rp.rp_fit(d_in["x"], d_in["y"], d_in["off"], DEGREE, precision=args.precision,
                  max_refine=args.max_refine, tol=args.tol, degrees=d_in["deg"], out=fit_out, stream=stream,
                  **fk_dev(d_in))
        fit_done = torch.cuda.Event()
        fit_done.record(stream)
        side.wait_event(fit_done)
        with torch.cuda.stream(side):
            h_out["status"].copy_(fit_out["status"], non_blocking=True)
        rp.rp_program_pack(fit_out["coef"], fit_out["box"], d_in["deg"], d_in["mm"], d_in["gd"],
                           DEGREE, program=prog, stream=stream)
        stream.wait_event(q_ready)
        rp.rp_eval_search(prog, N_KERNELS, DEGREE, d_in["q"], out=s_out, stream=stream)
        h_out["argmin"].copy_(s_out["argmin"], non_blocking=True)
        h_out["best"].copy_(s_out["best"], non_blocking=True)
        side_done = torch.cuda.Event()
        side_done.record(side)
        stream.wait_event(side_done)

    e2e_step()
    torch.cuda.synchronize()
    e_ms = []
    for _ in range(args.e2e_steps if args.only == "all" else 0):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e_ms.append(a.elapsed_time(b))
    e2e_serial_ms = max_over_ranks(statistics.mean(e_ms) if e_ms else float("nan"), ws, dev)

    # end to end as a stream of batches: the two-stream schedule above with
    # every step's inputs copied in and results copied out (three buffer sets)
    pipe_io["h"] = h
    pipe_io["in"] = [d_in] + [{k: torch.empty_like(v) for k, v in d_in.items()} for _ in range(NB - 1)]
    pipe_io["out"] = [h_out] + [{k: torch.empty_like(v).pin_memory() for k, v in h_out.items()}
                                for _ in range(NB - 1)]
    pipe_io["fk"] = fk_dev

    e2e_ms = float("nan")
    if args.only == "all" and args.e2e_steps > 0:
        n_pipe = max(args.steps, args.e2e_steps, NB + 1)
        pipelined(NB + 1, copies=True)             # warm-up (allocator, first-use paths)
        e2e_ms = max_over_ranks(pipelined(n_pipe, copies=True), ws, dev)
        # the last step's results match the device-timed steps' (same inputs)
        last = (n_pipe - 1) % NB
        assert torch.equal(pipe_io["out"][last]["argmin"], s_out["argmin"].cpu()), "e2e argmin mismatch"

    extra = {}
    if args.only == "all" and not args.no_extras:
        extra = extra_measurements(rp, args, inst, x, x_full, FK, y, off, deg, mm, gd, q, fit_out, prog, s_out,
                                   flush, stream, step, statistics.mean(fit_ms),
                                   statistics.mean(search_ms), ms_per_step)

    if rank == 0:
        pk, src = peaks()
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        fit_avg, search_avg = statistics.mean(fit_ms), statistics.mean(search_ms)
        alu_peak = fp32_peak_tflops(sm_count, pk.get("sm_max_mhz", 2070.0))
        # the fit's dense contraction (the augmented design Gram) against the
        # tensor-core roofline: TF32 dense peak = the measured BF16 burst peak
        # x 1/2 (nominal dense TF32 : BF16 = 1.1 : 2.25 PFLOP/s on GB300)
        tf32_peak = pk.get("bf16_tflops", 1900.0) * 0.5
        fit_flops = F * fit_flops_per_fit(M_SAMPLES, DEGREE)
        # per fit: its values, its share of its set's points (or its own
        # points), its outputs
        fit_bytes = F * (4 * M_SAMPLES + (12 * M_SAMPLES // N_METRICS if FK else 12 * M_SAMPLES) + 896)
        traffic = None
        if (FIT_TRAFFIC["bytes_per_fit"] is not None and args.precision == "fp32" and FK
                and FIT_TRAFFIC["sources_sha256"] == fit_sources_sha256()):
            traffic = FIT_TRAFFIC["bytes_per_fit"] * F
        if fit_avg >= search_avg:
            ach = fit_flops / (fit_avg / 1e3) / 1e12
            roof = {"kernel": "rp_fit (fit_kernel)", "bound": "tensor", "achieved": ach,
                    "peak": tf32_peak, "unit": "TFLOP/s", "frac": ach / tf32_peak, "traffic": traffic,
                    "peak_source": f"{src} bf16_tflops {pk.get('bf16_tflops')} x 1/2 (dense TF32 : "
                                   "BF16 = 1.1 : 2.25), burst (the fit is timed alone per step)",
                    "algorithmic": f"{fit_flops_per_fit(M_SAMPLES, DEGREE)} flop per fit (augmented "
                                   f"Gram m n_aug (n_aug + 1), m = {M_SAMPLES}, n_aug = 40) x {F} fits",
                    "hbm": {"achieved_gbs": fit_bytes / (fit_avg / 1e3) / 1e9,
                            "peak_gbs": pk.get("hbm_gbs"),
                            "frac": fit_bytes / (fit_avg / 1e3) / 1e9 / pk.get("hbm_gbs", 6800.0),
                            "algorithmic_bytes": fit_bytes},
                    "alu": {"achieved_tflops": ach, "peak_tflops": alu_peak, "frac": ach / alu_peak,
                            "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {src} sm_max_mhz"}}
        else:
            ach = N_QUERIES * search_flops_per_query(DEGREE) / (search_avg / 1e3) / 1e12
            roof = {"kernel": "rp_eval_search", "bound": "alu", "achieved": ach, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": ach / alu_peak, "traffic": None,
                    "peak_source": f"FP32 lanes x SM clock ({src} sm_max_mhz)"}
        line = {"metric": METRIC, "value": value, "unit": "fits/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.precision, args.tol, args.max_refine),
                "queries_per_s": ws * N_QUERIES / (ms_per_step / 1e3),
                "phase_ms": {"fit": fit_avg, "pack": statistics.mean(pack_ms), "search": search_avg},
                "fit_ok_frac": fit_ok,
                "roofline": roof,
                "e2e": {"value": job_rate(ws, F, e2e_ms), "unit": "fits/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                        "pipelined": "the two-stream schedule of the headline with each step's "
                                     "copy-in on a copy stream ahead of its fit and its copy-out on a "
                                     "second copy stream (three buffer sets); L2 flushed before each fit",
                        "serial_ms_per_step": e2e_serial_ms},
                "schedule": {"pipelined": "fit of step k+1 on a high-priority stream while pack + search "
                                          "of step k run on a second (three buffer sets); L2 flushed before "
                                          "each fit, inside the timed region",
                             "serial_ms_per_step": serial_ms_per_step},
                "gpu_launches": {"all": 3 + search_launches, "fit": 2,
                                 "search": search_launches}[args.only] * args.steps,
                "clocks": clk, "tuned": tuned}
        line.update(extra)
        if ws == 1 and not args.no_cpu_baseline and args.only == "all":
            r = oracle_rates(inst, q_np, gd_np, budget_s=20.0)
            line["cpu_baseline"] = {"value": F / r["step_s"], "unit": "fits/s", "cores": r["cores"],
                                    "kind": "oracle", "sample": r["sample"],
                                    "scaled_to_full_step": r["scaled"], "wall_s": r["wall_s"]}
            import oracle
            oracle.set_threads(os.cpu_count() or 1)
            ref = oracle.fit(inst["x"], inst["y"], inst["fit_off"], inst["degree"])
            line["parity_vs_oracle"] = parity_against_oracle(inst, q_np, r, g_res, ref)
            tf = line.pop("_tf32_fits", None)
            if tf is not None and "tf32_step" in line:
                err, excess = fit_errors(inst, tf["coef"], tf["box"], ref)
                line["tf32_step"]["parity"] = {
                    "fits": int(len(err)), "pred_rel_err_max": float(err.max()),
                    "pred_rel_err_median": float(np.median(err)),
                    "fits_within_1e-4": float((err <= 1e-4).mean()),
                    "objective_excess_max": float(excess.max()),
                    "pole_flags_equal": bool((((tf["status"] & 4) != 0) ==
                                              ((ref["status"] & 4) != 0)).all())}
            sv = line.pop("_svd_fits", None)
            if sv is not None and "svd_solver" in line:
                err, excess = fit_errors(inst, sv["coef"], sv["box"], ref)
                line["svd_solver"]["parity"] = {
                    "fits": int(len(err)), "pred_rel_err_max": float(err.max()),
                    "pred_rel_err_median": float(np.median(err)),
                    "fits_within_1e-4": float((err <= 1e-4).mean()),
                    "objective_excess_max": float(excess.max())}
        line.pop("_tf32_fits", None)
        line.pop("_svd_fits", None)
        if ws == 1 and not args.no_extras and args.only == "all":
            # the path's other stated workloads (tiny FP64 latency,
            # differentiation, uneven batch with one CUDA graph), each with its
            # own parity summary
            line["workloads"] = {"tiny_fp64": workload_tiny(rp, dev, stream),
                                 "diff": workload_diff(rp, dev, stream),
                                 "uneven_graph_fp32": workload_uneven(rp, dev, stream, "fp32"),
                                 "uneven_graph_bf16": workload_uneven(rp, dev, stream, "bf16")}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
