/*
 * rp.h -- C ABI of the GB300 rational-program library.
 *
 * The library implements the data-parallel hot path of the rational-program
 * technique for choosing GPU launch parameters (Brandt, Mohajerani, Moreno
 * Maza, Paudel, Wang, "A Technique for Finding Optimal Program Launch
 * Parameters Targeting Manycore Accelerators", arXiv:1906.00142):
 *
 *   rp_fit           Step 2 of Sec. 3.3 / Sec. 4.2: least-squares estimation of
 *                    rational functions p/q in the data and program parameters
 *                    (N, B0, B1) from sampled low-level metrics.
 *   rp_program_pack  Step 3 of Sec. 3.3 / Sec. 4.3.1: turn the fitted metrics
 *                    of each kernel into the rational program's coefficient
 *                    table (no source generation).
 *   rp_eval_search   Steps 4-5 of Sec. 3.3 / Sec. 4.3.2: evaluate the
 *                    MWP-CWP rational program (Sec. 2, Example 2; occupancy,
 *                    Example 1) at every admissible thread-block format and
 *                    take the argmin, for many (data, hardware) queries.
 *   rp_relmse_fwd/bwd, rp_adam_step
 *                    nonlinear refinement of fitted coefficients on the mean
 *                    squared relative error (no counterpart in the paper).
 *
 * Conventions for every entry point:
 *  - Arrays are caller-owned DEVICE memory unless stated otherwise; the
 *    library allocates nothing and keeps no pointer after returning.
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t, 0 = legacy
 *    default stream); nothing synchronises the host.
 *  - The return value is RP_OK (0) or a negative rp_status; arguments are
 *    checked before anything is launched, so an error return launches
 *    nothing.  Per-item outcomes are reported in status arrays.
 *  - Results are deterministic for fixed inputs (no floating-point atomics).
 */
#ifndef RP_H_
#define RP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RP_VERSION 3
#define RP_MAX_DEGREE 4          /* total degree bound d <= 4 */
#define RP_COEF_STRIDE 70        /* alpha_j at [0, 35), beta_j at [35, 70) */
#define RP_NUM_CONFIGS 66        /* (2^a, 2^b), a + b <= 10 */
#define RP_NUM_METRICS 8

/* Return codes (negative = nothing was launched). */
typedef enum rp_status {
  RP_OK = 0,
  RP_ERR_INVALID_ARG = -1,
  RP_ERR_UNSUPPORTED = -2,
  RP_ERR_WORKSPACE = -3,
  RP_ERR_CUDA = -4,
  RP_ERR_ALIGNMENT = -5,
  RP_ERR_NO_DEVICE = -6
} rp_status;

/* Per-fit status bits (rp_fit). */
#define RP_FIT_RANK_DEFICIENT 1   /* columns dropped by the factorisation */
#define RP_FIT_NOT_CONVERGED 2    /* refinement ended (max_refine steps, or steps that kept raising
                                     the objective) before its stop test was met; on the FP32 and
                                     tensor-core precisions such a fit is solved again with FP64
                                     arithmetic (RP_FIT_FP64_PASS) */
#define RP_FIT_POLE 4             /* fitted q <= 0 at one of the fit's samples */
#define RP_FIT_NONFINITE 8        /* NaN/Inf in the fit's samples: no fit */
#define RP_FIT_NONPOS_Y 16        /* y <= 0 with relative weighting: no fit */
#define RP_FIT_EMPTY 32           /* no samples: no fit */
#define RP_FIT_TIMEOUT 64         /* a bounded wait of the tensor-core path ran out: no fit */
#define RP_FIT_ESCALATED 128      /* tensor-core precisions: refinement from the low-precision
                                     Gram stopped short of tol (or dropped pivots), so the fit
                                     was solved again from the FP32 Gram on CUDA cores */
#define RP_FIT_ITER_SHIFT 8       /* bits 8..15: refinement iterations performed */
#define RP_FIT_ITER_MASK 0xFF00
#define RP_FIT_ACC_SHIFT 16       /* bits 16..23: of those, accurate (double-float residual)
                                     passes on the FP32 and tensor-core precisions */
#define RP_FIT_ACC_MASK 0xFF0000
#define RP_FIT_FP64_PASS (1 << 24) /* FP32 and tensor-core precisions: the fit's own solve dropped
                                     pivots at its drop tolerance or stopped short of tol, so the
                                     fit was solved again with RP_PREC_FP64 arithmetic (its basis
                                     and design Grams summed in double-float arithmetic from FP64
                                     rows, ~1e-14 relative; the other bits then describe that
                                     solve) */

/* Per-query status bits (rp_eval_search). */
#define RP_Q_NO_VALID 1           /* no configuration valid: argmin = -1 */
#define RP_Q_POLE 2               /* some configuration hit q <= 0 (excluded) */
#define RP_Q_BAD 4                /* non-finite query field, N < 1, bad kernel id */

/* Arithmetic used by rp_fit for the Gram product of the design matrix. */
typedef enum rp_precision {
  RP_PREC_FP64 = 0,    /* plain form: FP64 design, Gram, factor and residuals on CUDA cores */
  RP_PREC_FP32 = 1,    /* FP32 design, Gram products and factor on CUDA cores */
  RP_PREC_TF32 = 2,    /* FP32 design; design Gram in one TF32 tensor-core pass (tcgen05),
                          basis Gram in split TF32; FP32 factor; residuals from the samples */
  RP_PREC_TF32X3 = 3,  /* as TF32 with both Grams in split TF32 (hi*hi + hi*lo + lo*hi) */
  RP_PREC_BF16 = 4,    /* FP32 design rounded to BF16 for a one-pass tensor-core design Gram
                          (tcgen05 kind::f16, FP32 accumulation); as TF32 otherwise */
  RP_PREC_BF16X3 = 5   /* as BF16 with split BF16 operands (hi*hi + hi*lo + lo*hi) */
} rp_precision;

/* rp_fit flags */
#define RP_FIT_UNWEIGHTED 1       /* rows not weighted by 1/|y| */
#define RP_FIT_SOLVER_SVD 2       /* solve through the singular value decomposition of the
                                     (equilibrated, whitened) design, the paper's solver
                                     (Sec. 4.2): cyclic Jacobi rotations of its normal matrix
                                     give the right singular vectors and squared singular
                                     values; directions below drop tolerance are truncated (the
                                     rank) and the truncated pseudo-inverse is the first
                                     solution and the refinement's preconditioner (instead of
                                     the sweep operator with pivot dropping) */

typedef struct rp_fit_desc {
  int64_t num_fits;        /* F >= 0 */
  int64_t num_samples;     /* S: length of y and of each of the 3 rows of x */
  int32_t degree;          /* total degree bound 1..4 used when degrees == NULL */
  int32_t precision;       /* rp_precision */
  int32_t max_refine;      /* refinement iterations after the first solve, 0..64 */
  int32_t flags;           /* RP_FIT_* flags */
  double tol;              /* refinement stops once an accurate step (FP64 on the FP64 path,
                              double-float on the others) leaves an estimated relative error
                              c * ||dx|| / ||x|| <= tol, c = the contraction per step estimated
                              from the steps (at least 1e-3); e.g. 1e-8, or 1e-12 to refine to
                              the arithmetic's floor */
  const int8_t *degrees;   /* optional device array [F] of per-fit degrees 1..4 */
  /* Shared sample points (Sec. 3.3 Step 1 measures all metrics of a kernel
     at the same points).  point_off NULL: fit f's points are the columns
     fit_off[f] .. fit_off[f+1] of x, a float[3][num_samples] array.
     Otherwise each run of fits_per_point_set consecutive fits shares one
     point set: fit f uses set p = f / fits_per_point_set, the columns
     point_off[p] .. point_off[p+1] of x (a float[3][num_points] array), and
     its values y[fit_off[f] .. fit_off[f+1]), one per point (a fit whose
     value count differs from its set's point count gets RP_FIT_EMPTY).  The
     box, marginal polynomials and basis whitening are then computed once
     per set.  point_off: device int64 [ceil(F / fits_per_point_set) + 1]. */
  const int64_t *point_off;
  int64_t num_points;      /* columns of x when point_off is given */
  int32_t fits_per_point_set;   /* >= 1 when point_off is given */
  int32_t reserved;        /* must be 0 */
} rp_fit_desc;

/*
 * rp_fit_workspace_size -- bytes of the optional device workspace of rp_fit
 * for `desc`, written to *bytes: 32 for a non-empty batch (two 64-bit
 * counters 16 bytes apart: the dynamic fit schedule's claims and the number
 * of fits passed on to the FP64 path, RP_FIT_FP64_PASS), 0 otherwise.
 * Host-only, launches nothing.
 */
int rp_fit_workspace_size(const rp_fit_desc *desc, size_t *bytes);

/*
 * rp_fit_cache_workspace_size -- bytes of a workspace that also holds the
 * basis cache of rp_fit's accurate refinement passes (Sec. 4.2's
 * least-squares solve as refined here), written to *bytes.  The basis
 * values of a point set's samples depend only on the samples, not on the
 * metric fitted: with a workspace of at least this size, the first
 * accurate pass of each claim of fits writes them (as pairs of FP32
 * numbers) to a slab of the CTA that fits them and the claim's later passes
 * read them back instead of recomputing them.  Results are identical with
 * and without the cache.  Size: 256 bytes (the counters of
 * rp_fit_workspace_size, padded), then per resident CTA of the largest
 * launch the batch makes a slab of 512 samples x ceil(NM / 2) x 16 bytes
 * (NM = (d+1)(d+2)(d+3)/6); about 50 MB for degree 3 on a 152-SM GB300.
 * FP64 precision and the FP32 degree-4 launch (no sample cache) use no
 * slab.  Queries the device (SM count, residency); launches nothing.
 * Errors: RP_ERR_INVALID_ARG (null pointers, degree or precision out of
 * range).
 */
int rp_fit_cache_workspace_size(const rp_fit_desc *desc, size_t *bytes);

/*
 * rp_fit -- batched least-squares fit of rational functions (Sec. 4.2).
 *
 * For fit f with samples i in [fit_off[f], fit_off[f+1]):
 *   raw variables (N, B0, B1) = (x[i], x[S+i], x[2S+i]), value y[i];
 *   each variable is mapped affinely to [-1, 1] over the fit's own samples
 *   (box[f] = lo_N, hi_N, lo_B0, hi_B0, lo_B1, hi_B1; a constant variable
 *   maps to 0); p and q are polynomials of total degree <= d in the mapped
 *   variables; the linearised residual w_i (p(x_i) - y_i q(x_i)) with
 *   w_i = 1/|y_i| is minimised in the 2-norm (the "linear in the
 *   coefficients" system A x = b of Sec. 4.2) under the normalisation that
 *   q averages to 1 over the fit's samples (the system is homogeneous,
 *   footnote of Sec. 4.2).
 * Outputs, in the graded-lex monomial basis of the mapped variables
 * (degree ascending, then exponent of N descending, then of B0 descending):
 *   coef[f*70 + j] = alpha_j (numerator), coef[f*70 + 35 + j] = beta_j
 *   (denominator), unused entries 0; coef32 (optional, may be NULL) the same
 *   rounded to float; box[f*6 + ...] as above; rank[f] = columns kept by the
 *   factorisation; status[f] = RP_FIT_* bits.
 * Inputs: x float[3][S], y float[S], fit_off int64[F+1] non-decreasing with
 * fit_off[0] = 0 and fit_off[F] <= S (checked on the device: a fit with a
 * bad range gets RP_FIT_EMPTY).  workspace: NULL, or device memory of at
 * least rp_fit_workspace_size bytes, 16-byte aligned, owned by the caller
 * and used by one call at a time: with it, CTAs claim fits dynamically from
 * a counter kept there (reset on the stream with cudaMemsetAsync before the
 * launch), so CTAs that draw large fits take fewer; with NULL each CTA takes
 * every (grid size)-th fit.  With at least rp_fit_cache_workspace_size
 * bytes the workspace also holds the basis cache (see there).  Results do
 * not depend on the schedule or the cache.
 * Errors: RP_ERR_INVALID_ARG for null pointers, F < 0, degree or precision
 * out of range; RP_ERR_WORKSPACE / RP_ERR_ALIGNMENT for a workspace that is
 * too small or misaligned; RP_ERR_CUDA if a launch fails.
 */
int rp_fit(const rp_fit_desc *desc, const float *x, const float *y, const int64_t *fit_off,
           double *coef, float *coef32, double *box, int32_t *status, int32_t *rank,
           void *workspace, size_t workspace_bytes, void *stream);

/*
 * rp_fit_noalloc -- rp_fit (same arguments, results and errors) for callers
 * that cannot provide device memory, e.g. a host thread on a latency path
 * where cudaMalloc's implicit device synchronisation is not acceptable.  It
 * allocates nothing: its scratch (the two 64-bit counters that make up
 * rp_fit_workspace_size) is a statically allocated 32-byte device array of
 * the library, reset with cudaMemsetAsync on `stream` before use.  The
 * paper has no counterpart (it describes no GPU fitting).
 * Limit: scratch of 32 bytes, which covers any batch size; a larger need
 * returns RP_ERR_WORKSPACE.  The first call on each device resolves the
 * array's address (cudaGetSymbolAddress) with that device current: make it
 * before capturing any stream.  Calls that overlap in time (any streams,
 * any threads) share the counters and race: serialise them.
 */
int rp_fit_noalloc(const rp_fit_desc *desc, const float *x, const float *y,
                   const int64_t *fit_off, double *coef, float *coef32, double *box,
                   int32_t *status, int32_t *rank, void *stream);

/*
 * rp_program_size -- bytes of the packed program for K kernels whose fitted
 * metrics have degree <= d.  Layout (all little-endian, 16-byte aligned
 * sections): aN float[K][8], bN float[K][8], grid_dims int32[K] (padded),
 * table float[K][66][8][2][d+1].
 */
size_t rp_program_size(int64_t num_kernels, int32_t degree);

/*
 * rp_program_pack -- the coefficient table of the rational program
 * (Sec. 3.3 Step 3; Sec. 4.3.1 builds C source, here a table).
 * For kernel k, configuration c = (B0, B1) and metric m (order: comp insts,
 * coalesced mem insts, uncoalesced mem insts, transactions per uncoalesced
 * warp access, synch insts, load bytes per warp, registers per thread,
 * shared-memory words per block -- the metrics of Sec. 4.1), with
 * f = metric_map[k*8 + m] (-1 = metric absent, evaluates to 0):
 *   aN, bN map N to the fit's normalised variable t = aN*N + bN;
 *   table holds, for numerator and denominator, the coefficients of t^0..t^d
 *   obtained by fixing the normalised B0, B1 at configuration c (FP64
 *   arithmetic, stored as float).
 * Inputs (device): coef double[F][70], box double[F][6], degrees int8[F]
 * (per-fit degree, each <= degree), metric_map int32[K][8], grid_dims
 * int32[K] (1 = one-dimensional grid of ceil(N/T) blocks, 2 = ceil(N/B0) *
 * ceil(N/B1) blocks).  program: device buffer of rp_program_size bytes,
 * 16-byte aligned.  Errors: RP_ERR_INVALID_ARG, RP_ERR_ALIGNMENT,
 * RP_ERR_CUDA.
 */
int rp_program_pack(int64_t num_kernels, int32_t degree, const double *coef, const double *box,
                    const int8_t *degrees, const int32_t *metric_map, const int32_t *grid_dims,
                    void *program, size_t program_bytes, void *stream);

/* Fixed architecture constants of the MWP-CWP/occupancy model (host struct). */
typedef struct rp_hw_fixed {
  int32_t warp_size;       /* 32 */
  int32_t t_max;           /* max threads per block, 1024 */
  int32_t b_max;           /* max resident blocks per SM */
  int32_t w_max;           /* max resident warps per SM */
  int32_t r_sm;            /* registers per SM */
  int32_t z_sm;            /* shared-memory words per SM */
  float issue_cycles;      /* cycles per issued instruction */
  int32_t reserved;        /* must be 0 */
} rp_hw_fixed;

/*
 * rp_eval_search -- exhaustive evaluate-and-argmin (Sec. 3.3 Steps 4-5).
 * For every query q (device float[Q][8]: N, number of SMs, SM clock in GHz,
 * memory latency in cycles, memory bandwidth in GB/s, coalesced and
 * uncoalesced departure delay in cycles, kernel id as int32 bits) the
 * MWP-CWP execution time in cycles is evaluated in FP32 at all 66
 * configurations from the packed program; argmin[q] receives the index of
 * the smallest (ties: lowest index; -1 if none valid), best[q] and
 * second[q] the smallest and second-smallest cycle counts (+inf if absent),
 * status[q] RP_Q_* bits.  Configuration index c enumerates (2^a, 2^b) with
 * a ascending then b ascending (c = 11a - a(a-1)/2 + b).
 * Model: occupancy (Example 1, W_active = min(floor(B_active T/32), W_max)),
 * MWP-CWP as in Hong & Kim 2009 (the paper cites it and does not print
 * it); see the library's design notes for the exact statement.
 * hw: host pointer.  workspace: NULL, or device memory of at least
 * rp_search_workspace_size bytes, 16-byte aligned, owned by the caller and
 * used by one call at a time.  With it (and a non-zero size for this K and
 * Q) the queries are first bucketed by kernel id on the device and each
 * block of threads evaluates queries of one kernel from a copy of that
 * kernel's table in shared memory; with NULL each query gathers its table
 * rows from global memory.  Results do not depend on the path.
 * Errors: RP_ERR_INVALID_ARG, RP_ERR_WORKSPACE (workspace too small),
 * RP_ERR_ALIGNMENT, RP_ERR_CUDA.
 */
int rp_eval_search(const void *program, int64_t num_kernels, int32_t degree,
                   const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                   int32_t *argmin, float *best, float *second, int32_t *status,
                   void *workspace, size_t workspace_bytes, void *stream);

/*
 * rp_eval_search_tiebreak -- rp_eval_search with Step 5's choice among
 * several optimal configurations made by a second metric (Sec. 3.3 Step 5
 * suggests one): the configurations whose cycles are at most
 * (1 + tie_rel) times the smallest count as optimal, and argmin[q] is the
 * one of them with the most active warps per SM (W_active, Sec. 2 Example
 * 1); among equal W_active the lowest index.  best[q] and second[q] are the
 * smallest and second-smallest cycle counts as in rp_eval_search (argmin's
 * own count may exceed best by up to the factor).  Each query's
 * configurations are evaluated twice (FP32, identically).  tie_rel in
 * [0, 1) (0: only exact ties).  Other arguments, errors and workspace as
 * rp_eval_search.
 */
int rp_eval_search_tiebreak(const void *program, int64_t num_kernels, int32_t degree,
                            const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                            float tie_rel, int32_t *argmin, float *best, float *second,
                            int32_t *status, void *workspace, size_t workspace_bytes,
                            void *stream);

/*
 * rp_eval_occupancy -- the occupancy rational program on its own (Sec. 2,
 * Example 1): for every query and configuration c, from the program's
 * fitted registers per thread R and shared-memory words per block Z
 * (metrics 7 and 8, rounded to the nearest integer) at the query's N,
 *   B_active = min(b_max, floor(w_max / wpb), floor(r_sm / (R wpb warp)) [R > 0],
 *              floor(z_sm / Z) [Z > 0]), 0 if T > t_max, R T > r_sm or Z > z_sm,
 *   W_active = min(B_active wpb, w_max), wpb = ceil(T / warp), T = B0 B1;
 * written to b_active[q*66 + c] and w_active[q*66 + c] (device int32
 * [Q][66]); both 0 where the configuration cannot be resident or a metric's
 * denominator is <= 0 at N (status RP_Q_POLE), and for a bad query
 * (RP_Q_BAD, as rp_eval_search).  program, hw, queries as rp_eval_search.
 * Errors: RP_ERR_INVALID_ARG, RP_ERR_ALIGNMENT, RP_ERR_CUDA.
 */
int rp_eval_occupancy(const void *program, int64_t num_kernels, int32_t degree,
                      const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                      int32_t *b_active, int32_t *w_active, int32_t *status, void *stream);

/* Per-query status bits (rp_error_pct). */
#define RP_EP_NO_RUNTIME 1        /* no finite runtime for the query: err = NaN */
#define RP_EP_BAD_CHOICE 2        /* choice outside 0..65 or its runtime not finite: err = NaN */

/*
 * rp_error_pct -- Error % of chosen configurations (Sec. 5): with measured
 * runtimes t[q][0..65] (device float [Q][66], +inf or NaN for a
 * configuration not run) and the configuration chosen for each query
 * (device int32 [Q], e.g. rp_eval_search's argmin),
 *   B = min and W = max of the query's finite runtimes,
 *   err_pct[q] = (t[q][choice[q]] - B) / (W - B) * 100   (0 when W == B),
 * in FP32; status[q] RP_EP_* bits.  Errors: RP_ERR_INVALID_ARG, RP_ERR_CUDA.
 */
int rp_error_pct(const float *runtimes, const int32_t *choice, int64_t num_queries,
                 float *err_pct, int32_t *status, void *stream);

/*
 * The rational program as generated code (Sec. 3.3 Step 3; Sec. 4.3.1
 * generates the program's source with the fitted functions written in).
 *
 * rp_codegen_source -- CUDA C++ source of the rational program of kernel
 * kernel_id of a packed program: its 66 x 8 numerator and denominator
 * coefficient rows, its data-parameter maps, grid dimensionality and the
 * architecture constants hw written in as constants (exact hexadecimal
 * floats), and a kernel `rp_generated_search` that evaluates and takes the
 * argmin of queries of that kernel with the same arithmetic as
 * rp_eval_search (queries naming another kernel get RP_Q_BAD).
 * program_host: a HOST copy of the packed program (rp_program_size bytes).
 * src: host buffer of *len bytes, or NULL to ask for the size; *len
 * receives the bytes needed including the terminating NUL.  Host-only.
 * Errors: RP_ERR_INVALID_ARG; RP_ERR_WORKSPACE if *len is too small.
 */
int rp_codegen_source(const void *program_host, int64_t num_kernels, int32_t degree,
                      int64_t kernel_id, const rp_hw_fixed *hw, char *src, size_t *len);

/*
 * rp_codegen_compile -- compiles generated source at run time (NVRTC, for
 * the current device's architecture) and loads it; *handle (opaque) is
 * valid on that device until rp_codegen_free.  log (may be NULL): host
 * buffer of log_len bytes for the compiler's messages.  Synchronous; not
 * capturable.  Errors: RP_ERR_UNSUPPORTED (NVRTC not found), RP_ERR_NO_DEVICE,
 * RP_ERR_INVALID_ARG (the source does not compile), RP_ERR_CUDA.
 */
int rp_codegen_compile(const char *src, void **handle, char *log, size_t log_len);

/*
 * rp_codegen_search -- runs a compiled generated program on num_queries
 * queries (device float [Q][8], as rp_eval_search) on `stream`; outputs as
 * rp_eval_search.  Errors: RP_ERR_INVALID_ARG, RP_ERR_ALIGNMENT, RP_ERR_CUDA.
 */
int rp_codegen_search(void *handle, const float *queries, int64_t num_queries, int32_t *argmin,
                      float *best, float *second, int32_t *status, void *stream);

/* rp_codegen_free -- unloads a compiled generated program (NULL: no-op). */
int rp_codegen_free(void *handle);

/*
 * rp_search_workspace_size -- bytes of the optional device workspace of
 * rp_eval_search for num_kernels kernels and num_queries queries, written
 * to *bytes: the bucket offsets and cursors (4 (2K + 3) bytes) and the
 * bucketed query indices (4 Q bytes), each rounded up to 16 bytes.  0 when
 * the search runs unbucketed for these sizes: fewer than 32 queries per
 * kernel on average, Q >= 2^31 - 1 or K >= 2^30.  Host-only, launches
 * nothing.  Errors: RP_ERR_INVALID_ARG (null bytes, negative sizes).
 */
int rp_search_workspace_size(int64_t num_kernels, int64_t num_queries, size_t *bytes);

/*
 * rp_relmse_fwd -- per-fit mean squared relative error
 *   L_f = (1/m) sum_i ((p(x_i)/q(x_i) - y_i) / y_i)^2
 * of the coefficients coef double[F][70] (layout and precision of rp_fit's
 * output) with the fits' boxes (double[F][6]) on the fits' samples (x, y,
 * fit_off as rp_fit), written to loss float[F].  p and q are evaluated in
 * FP64 (fitted monomial coefficients cancel by up to ~1e9); residuals and
 * sums in FP32.  degrees: int8[F] device.
 */
int rp_relmse_fwd(int64_t num_fits, int64_t num_samples, const float *x, const float *y,
                  const int64_t *fit_off, const int8_t *degrees, const double *coef,
                  const double *box, float *loss, void *stream);

/*
 * rp_relmse_bwd -- gradient of sum_f g_f L_f with respect to coef, given
 * g = grad_loss float[F]; written to grad float[F][70]:
 *   dL/dalpha_j = (2/m) sum r_i phi_j(x_i) / (y_i q_i)
 *   dL/dbeta_j  = -(2/m) sum r_i p_i phi_j(x_i) / (y_i q_i^2)   (j >= 1)
 * with beta_0 held fixed (its gradient is written as 0).
 */
int rp_relmse_bwd(int64_t num_fits, int64_t num_samples, const float *x, const float *y,
                  const int64_t *fit_off, const int8_t *degrees, const double *coef,
                  const double *box, const float *grad_loss, float *grad, void *stream);

/*
 * rp_adam_step -- one Adam update (Kingma & Ba 2015) of n parameters in
 * place: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  Entries with
 * mask[i] == 0 are left unchanged.  param double[n] (the fitted
 * coefficients; an FP32 copy could not hold steps below its rounding),
 * grad, m, v float[n], mask uint8[n] (may be NULL = all), all on the device.
 * t >= 1.
 */
int rp_adam_step(int64_t n, double *param, const float *grad, float *m, float *v,
                 const uint8_t *mask, int32_t t, float lr, float beta1, float beta2, float eps,
                 void *stream);

/*
 * Launch-shape autotuning (no counterpart in the paper; the paper's search is
 * the evaluation itself).  Each call runs its kernel several times on the
 * caller's buffers (the outputs end holding a valid result of the call),
 * synchronises the host with the stream, and records the fastest shape for
 * the current device; later launches of that kind use it.  Results never
 * depend on the shape.  Not capturable into a CUDA graph: call before
 * capturing.  Not thread-safe against concurrent launches of the same kind.
 *
 * rp_tune_search -- arguments as rp_eval_search; times persistent grids of
 * {256, 128, 64} threads per CTA and 2..32 CTAs per SM for `degree` on the
 * path the workspace selects (the shape is shared by both paths) and writes
 * the chosen threads per CTA and CTAs per SM.
 */
int rp_tune_search(const void *program, int64_t num_kernels, int32_t degree,
                   const rp_hw_fixed *hw, const float *queries, int64_t num_queries,
                   int32_t *argmin, float *best, float *second, int32_t *status,
                   void *workspace, size_t workspace_bytes, void *stream, int32_t *threads,
                   int32_t *ctas_per_sm);

/*
 * rp_tune_fit -- arguments as rp_fit; times persistent grids of 1 .. (the
 * residency limit of the variant desc selects) CTAs per SM for desc's
 * precision and degree and writes the chosen CTAs per SM.
 */
int rp_tune_fit(const rp_fit_desc *desc, const float *x, const float *y, const int64_t *fit_off,
                double *coef, float *coef32, double *box, int32_t *status, int32_t *rank,
                void *workspace, size_t workspace_bytes, void *stream, int32_t *ctas_per_sm);

/* Message for an rp_status code (static string). */
const char *rp_strerror(int code);

/* RP_VERSION of the loaded library. */
int rp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RP_H_ */
