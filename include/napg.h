/*
 * napg.h -- C ABI of the GB300 library for all-pairs statistical tests with
 * pairwise deletion (NApy, arXiv 2505.00448).
 *
 * Problem statement (Sec. 3.2-3.4): a data matrix X of F variables x S samples;
 * a missing-value sentinel m; variables are continuous or categorical
 * (categorical labels are integers 0..c-1 stored as floating-point values).
 * For a pair of variables (g, h) only the samples where both are observed are
 * used: I(g,h) = {(g_i, h_i) : g_i != m and h_i != m} (Sec. 3.2). For every pair
 * the library returns the test statistic, its p-value and n = |I(g,h)|.
 *
 * Tests (Sec. 3.5):
 *   NAPG_PEARSON   continuous x continuous, r, p from the Beta CDF   (Sec. 3.5.2)
 *   NAPG_SPEARMAN  continuous x continuous, rho on tie-averaged ranks (Sec. 3.5.3)
 *   NAPG_CHI2      categorical x categorical, chi-squared           (Sec. 3.5.4)
 *   NAPG_ANOVA     categorical x continuous, one-way F               (Sec. 3.5.7)
 *   NAPG_TTEST     dichotomous x continuous, Welch (or Student) t   (Sec. 3.5.5)
 *   NAPG_MWU       dichotomous x continuous, Mann-Whitney U          (Sec. 3.5.6)
 *   NAPG_KRUSKAL   categorical x continuous, Kruskal-Wallis H        (Sec. 3.5.8)
 *
 * Conventions for every entry point:
 *   - Errors are returned as a napg_status; nothing aborts. A statistically
 *     undefined result is not an error: stat/p are NaN (n is still written).
 *     napg_last_error() returns a message for the last failing call on a context.
 *   - The caller owns every buffer it passes. The context owns the device copy
 *     of the cohort and its work memory until napg_destroy.
 *   - Work is ordered on the context's CUDA stream. A call whose outputs are in
 *     host memory returns after they are written; a call whose outputs are all
 *     in device memory returns once the work is queued (synchronize the stream,
 *     or call napg_sync, before reading them).
 *   - Host or device pointers are told apart with cudaPointerGetAttributes.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef NAPG_H
#define NAPG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct napg_ctx napg_ctx;

typedef enum {
    NAPG_OK = 0,
    NAPG_E_ARG = 1,          /* invalid argument (shape, variable type, level count, NULL) */
    NAPG_E_OOM = 2,          /* device memory allocation failed */
    NAPG_E_CUDA = 3,         /* a CUDA runtime call failed (message in napg_last_error) */
    NAPG_E_LABEL = 4,        /* a categorical value is not an integer in [0, c) */
    NAPG_E_NONFINITE = 5,    /* a non-missing value is +-inf or NaN */
    NAPG_E_TIMEOUT = 6,      /* a bounded device wait gave up */
    NAPG_E_UNSUPPORTED = 7,  /* valid request outside the library's limits */
    NAPG_E_BUSY = 8          /* serving queue full / no free slot */
} napg_status;

typedef enum {
    NAPG_PEARSON = 0, NAPG_SPEARMAN = 1, NAPG_CHI2 = 2, NAPG_ANOVA = 3,
    NAPG_TTEST = 4, NAPG_MWU = 5, NAPG_KRUSKAL = 6
} napg_test;

/* Arithmetic of the moment contractions (Pearson, ANOVA, t-test):
 *   NAPG_FP64_PLAIN  every sum in FP64 on the CUDA cores;
 *   NAPG_MIXED       column-shifted values, scaled by a power of two per
 *                    variable and split into FP16 hi/lo parts, contracted on the
 *                    tensor cores (tcgen05) with FP32 accumulation drained into
 *                    float-float sums in short chunks; finalize and p-values in
 *                    FP64; ill-conditioned pairs recomputed exactly in FP64.
 * Counts, contingency tables and rank sums are exact integers in both forms. */
typedef enum { NAPG_FP64_PLAIN = 0, NAPG_MIXED = 1 } napg_precision;

typedef enum { NAPG_F32 = 0, NAPG_F64 = 1 } napg_dtype;

/* Maximum levels of a categorical variable the library accepts. */
#define NAPG_MAX_LEVELS 64

typedef struct {
    int32_t precision;       /* napg_precision; default NAPG_FP64_PLAIN */
    int32_t welch;           /* 1: Welch t (default), 0: Student t (Sec. 3.5.5) */
    int32_t yates_2x2;       /* 1: Yates continuity correction on 2x2 tables; default 0 */
    int32_t mwu_mode;        /* 0 auto (default), 1 exact, 2 asymptotic (Sec. 3.5.6). Auto takes
                                the exact null distribution when there are no ties and
                                min(n0, n1) < 8. Forced exact (1) counts arrangements in exact
                                128-bit integers: a pair with min(n0, n1) > 64, C(n, n0) >= 2^126
                                or min(U0, U1) above max(3.5 n_samples, 65,534) gets p = NaN, and the call
                                returns NAPG_E_UNSUPPORTED once all its outputs are written
                                (napg_sync for asynchronous calls; a serving request's status) */
    int32_t mwu_continuity;  /* 1: 0.5 continuity correction in asymptotic mode (default) */
    int32_t debug_checks;    /* 1: extra device-side argument checks */
    int32_t async_host_outputs; /* 1: napg_run / napg_run_ex return once the work and the
                                   copies of host outputs are queued (outputs valid after
                                   napg_sync; one call's copies overlap the next call's
                                   kernels; pinned host buffers let them run asynchronously);
                                   0 (default): those calls return with host outputs written */
} napg_options;

/* Fills *opt with the defaults above. */
void napg_default_options(napg_options *opt);

/* Creates a context on CUDA device `device`. `cuda_stream` is a cudaStream_t to
 * order all work on, or NULL for a stream owned by the context.
 * Errors: NAPG_E_ARG (out NULL), NAPG_E_CUDA. */
napg_status napg_create(napg_ctx **out, int device, void *cuda_stream);

/* Frees the context, its device cohort and its work memory. NULL is a no-op. */
void napg_destroy(napg_ctx *ctx);

/* Message describing the last failure on ctx (never NULL; "" after success). */
const char *napg_last_error(const napg_ctx *ctx);

/* Blocks until all work queued on the context's stream is done. */
napg_status napg_sync(napg_ctx *ctx);

/* Copies the cohort to the device and checks it (Sec. 3.2, 3.3).
 *   X            n_vars x n_samples values of type `dtype` (napg_dtype), row-major
 *                with one row per variable; with samples_major != 0 the matrix is
 *                n_samples x n_vars (one row per sample: the paper's `axis`
 *                choice) and is transposed on the device. Host or device memory.
 *   missing      the sentinel m; NaN means "a value is missing iff it is NaN".
 *                For F32 data a value is missing iff (double)x == missing.
 *   var_type     n_vars bytes, host: 0 continuous, 1 categorical.
 *   n_levels     n_vars int32, host: level count c (1..NAPG_MAX_LEVELS) of each
 *                categorical variable (ignored for continuous ones).
 * Replaces any cohort loaded before. Synchronous.
 * Errors: NAPG_E_ARG, NAPG_E_OOM, NAPG_E_LABEL (categorical value not an integer
 * in [0,c)), NAPG_E_NONFINITE (non-missing +-inf or NaN), NAPG_E_UNSUPPORTED
 * (n_levels above NAPG_MAX_LEVELS, n_samples >= 2^24), NAPG_E_CUDA. */
napg_status napg_load_cohort(napg_ctx *ctx, const void *X, int32_t dtype, int64_t n_vars,
                             int64_t n_samples, int32_t samples_major, double missing,
                             const uint8_t *var_type, const int32_t *n_levels);

/* Marks the context's derived data stale: the FP16 planes kept from the last
 * run without a sample context (reused by the next run on the same continuous
 * variables) and the presort of the continuous variables (Sec. 3.5.3: sorted once
 * per feature). The next run rebuilds what it needs; buffers are kept for reuse.
 * Errors: NAPG_E_ARG (NULL context). */
napg_status napg_release_cache(napg_ctx *ctx);

/* Runs one test over all pairs vars_a x vars_b of the loaded cohort.
 *   test         napg_test.
 *   opt          options, or NULL for the defaults.
 *   sample_mask  n_samples bytes (host or device), nonzero = sample in the
 *                context; NULL = all samples. A context is treated as its own
 *                sub-cohort: a categorical level never observed in it is not a
 *                category of the call.
 *   vars_a/n_a   host int32 indices into the cohort. For the categorical x
 *                continuous tests A holds the categorical variables (Sec. 3.4:
 *                an F_C x F_Q output) and must be NAPG_TTEST/NAPG_MWU: c == 2,
 *                NAPG_ANOVA/NAPG_KRUSKAL: c >= 2.
 *   vars_b/n_b   host int32 indices; NULL makes the call symmetric (A x A) for
 *                PEARSON, SPEARMAN and CHI2; required for the mixed tests.
 *   stat, pval   n_a x n_b doubles, row-major, host or device; may be NULL.
 *   n            n_a x n_b int32 co-observed counts; may be NULL.
 * Symmetric calls fill both triangles. Statistic reported: r (PEARSON), rho
 * (SPEARMAN), chi2, F, t (level 0 minus level 1), U of level 0, H.
 * Errors: NAPG_E_ARG (bad index, wrong variable type or level count, no
 * cohort), NAPG_E_OOM, NAPG_E_CUDA, NAPG_E_UNSUPPORTED. */
napg_status napg_run(napg_ctx *ctx, int32_t test, const napg_options *opt,
                     const uint8_t *sample_mask, const int32_t *vars_a, int32_t n_a,
                     const int32_t *vars_b, int32_t n_b, double *stat, double *pval,
                     int32_t *n);

/* napg_run with the effect sizes of Table 2 as two more outputs (n_a x n_b
 * doubles, row-major, host or device; either may be NULL):
 *   effect   PEARSON r^2; SPEARMAN rho; CHI2 phi = sqrt(chi2 / n); TTEST Cohen's d
 *            (mean_0 - mean_1 over the pooled SD for Student, over
 *            sqrt((v_0 + v_1) / 2) for Welch); MWU Pearson's r = |z| / sqrt(n)
 *            (z tie-corrected, no continuity correction); ANOVA partial eta^2 =
 *            SSB / (SSB + SSW); KRUSKAL eta^2 = (H - k + 1) / (n - k).
 *   effect2  CHI2 Cramer's V = sqrt(chi2 / (n (min(k_a, k_b) - 1))) over the levels
 *            present in the context; TTEST the degrees of freedom of the t
 *            distribution its p-value is taken from (Welch-Satterthwaite nu for
 *            Welch, n - 2 for Student; NaN where t is NaN or infinite); NaN for the
 *            other tests.
 * Each is NaN where the statistic is NaN, and where the paper makes it
 * undefined (Sec. 3.5.4, 3.5.5, 3.5.8): V with a single level, Welch's d when
 * both groups are constant, Kruskal-Wallis eta^2 when n <= k.
 * Errors: as napg_run. */
napg_status napg_run_ex(napg_ctx *ctx, int32_t test, const napg_options *opt,
                        const uint8_t *sample_mask, const int32_t *vars_a, int32_t n_a,
                        const int32_t *vars_b, int32_t n_b, double *stat, double *pval,
                        int32_t *n, double *effect, double *effect2);

/* One part of a call split over n_parts processes, one per GPU (Sec. 3.5.1: the
 * pairs are independent, so the output splits without any exchange during the
 * computation). Arguments as napg_run, plus:
 *   part, n_parts  0 <= part < n_parts; n_parts == 1 is napg_run.
 * The output rows (the rows of vars_a) go in blocks of NAPG_PART_ROWS
 * consecutive rows, dealt to the parts back and forth: block b belongs to
 * part b mod n_parts in even rounds r = b / n_parts and to part
 * n_parts - 1 - (b mod n_parts) in odd rounds, so a triangle's long and short
 * rows pair up. A symmetric call (vars_b == NULL) computes the pairs (i, j),
 * i <= j, whose row i is owned, and writes both (i, j) and (j, i); an A x B
 * call computes the owned rows of A. Every output entry is written by exactly
 * one part (entry (i, j) of a symmetric call by the owner of min(i, j)), with
 * the same value as the unsplit call; entries of other parts are left as they
 * were, so the union of the parts' writes is the whole matrix. Synchronous.
 * Errors: as napg_run; NAPG_E_ARG for part outside [0, n_parts). */
#define NAPG_PART_ROWS 256
napg_status napg_run_part(napg_ctx *ctx, int32_t test, const napg_options *opt,
                          const uint8_t *sample_mask, const int32_t *vars_a, int32_t n_a,
                          const int32_t *vars_b, int32_t n_b, int32_t part, int32_t n_parts,
                          double *stat, double *pval, int32_t *n);

/* Effect sizes are returned by napg_run_ex only; the batch and serving entry
 * points return stat, p and n. */

/* Multiple-testing correction (Sec. 3.4). */
typedef enum { NAPG_ADJ_BONFERRONI = 0, NAPG_ADJ_BH = 1, NAPG_ADJ_BY = 2 } napg_adjust_method;

/* Adjusts a rows x cols p-value matrix (row-major doubles, host or device) into
 * out (same shape, host or device; may equal p only when both are on the
 * device). The tests are the entries with a p-value (not NaN); with symmetric != 0
 * (rows == cols, one variable set against itself) each unordered pair i < j is
 * one test, both triangles of out get its adjusted value and the diagonal is
 * NaN (a variable against itself is no test). With m tests and ascending
 * p_(1) <= ... <= p_(m):
 *   NAPG_ADJ_BONFERRONI  min(1, m p)
 *   NAPG_ADJ_BH          Benjamini-Hochberg: min over k >= i of p_(k) m / k, capped at 1
 *   NAPG_ADJ_BY          Benjamini-Yekutieli: as BH with m c(m), c(m) = sum_{k <= m} 1/k
 * Entries without a p-value stay NaN. Runs on the context's stream; synchronous.
 * Errors: NAPG_E_ARG (unknown method, rows != cols for symmetric, NULL pointer),
 * NAPG_E_OOM, NAPG_E_CUDA. */
napg_status napg_adjust(napg_ctx *ctx, int32_t method, const double *p, int64_t rows, int64_t cols,
                        int32_t symmetric, double *out);

/* Runs one test for n_ctx sample contexts with the same variable sets
 * (Sec. 1: per-context association networks). sample_masks[k] is a context mask
 * as in napg_run (host or device); stat[k], pval[k], n[k] are n_a x n_b outputs
 * (each may be NULL). The contexts are processed from one captured CUDA graph
 * per batch shape; results equal n_ctx separate napg_run calls. With host
 * outputs the graph writes every context's outputs to one device region
 * (n_ctx x the outputs' bytes, kept by the context for reuse until
 * napg_destroy), which is then copied back; if that region cannot be allocated
 * the contexts run one napg_run at a time instead. The A x B form of Pearson and
 * chi-squared also runs one context at a time. Synchronous with host outputs.
 * Errors: as napg_run. */
napg_status napg_run_batch(napg_ctx *ctx, int32_t test, const napg_options *opt,
                           int32_t n_ctx, const uint8_t *const *sample_masks,
                           const int32_t *vars_a, int32_t n_a, const int32_t *vars_b,
                           int32_t n_b, double *const *stat, double *const *pval,
                           int32_t *const *n);

/* The library's device p-value functions applied to caller-supplied values,
 * for checking them on their own (Sec. 3.5: Beta CDF for r and t, F, chi-squared
 * and normal survival functions). s, a, b, p: count doubles each, host or device
 * (b read only for kinds 2 and 5, a not read for kinds 4, 7 and 8):
 *   0: p of a correlation s with n = a observations, I_{1-s^2}((a-2)/2, 1/2)
 *   1: two-sided p of Student t = s with a degrees of freedom
 *   2: F survival function at s with (a, b) degrees of freedom
 *   3: chi-squared survival function at s with a degrees of freedom
 *   4: standard normal survival function at s
 *   5: regularized incomplete beta I_s(a, b)
 *   6: regularized upper incomplete gamma Q(a, s)
 *   7: erfcx(sqrt s) = exp(s) erfc(sqrt s), s >= 0, by the library's own
 *      approximation (the one the p-value expansions use)
 *   8: the same through CUDA's erfcx, for comparison
 * Synchronous. Errors: NAPG_E_ARG (unknown kind, NULL array), NAPG_E_OOM, NAPG_E_CUDA. */
napg_status napg_debug_pvalues(napg_ctx *ctx, int32_t kind, const double *s, const double *a,
                               const double *b, int64_t count, double *p);

/* Exact integer quantities of one pair (a, b) for bit-exact checks, computed by
 * the device kernels of the test (host output):
 *   NAPG_CHI2:      out[g*c_b + h] = contingency count O_gh over all c_a x c_b levels.
 *   NAPG_SPEARMAN:  {n, sum 2Rx*2Ry, sum (2Rx)^2, sum (2Ry)^2} (doubled ranks
 *                   2R = 2L + t + 1, L = co-observed values strictly below, t =
 *                   co-observed size of the tie group).
 *   NAPG_MWU/NAPG_KRUSKAL: {n, T, n_0, S_0, n_1, S_1, ...}: T = sum (t^3 - t) over
 *                   co-observed tie groups, S_g = sum of doubled ranks of level g.
 *   NAPG_ANOVA/NAPG_TTEST: {n, n_0, n_1, ...}.  NAPG_PEARSON: {n}.
 * *written receives the count. Errors: NAPG_E_ARG (cap too small, bad pair). */
napg_status napg_debug_integers(napg_ctx *ctx, int32_t test, const uint8_t *sample_mask,
                                int32_t a, int32_t b, int64_t *out, int64_t cap,
                                int64_t *written);

/* ---------------------------------------------------------------- serving --
 * A request loop over the resident cohort (Sec. 1: on-the-fly, real-time
 * analyses). Requests are admitted while a slot and device memory are free;
 * admitted requests run concurrently on per-slot streams. */
typedef struct {
    int32_t test;                 /* napg_test */
    napg_options opt;
    const uint8_t *sample_mask;   /* host, n_samples bytes, or NULL; copied at submit */
    const int32_t *vars_a;        /* host; copied at submit */
    int32_t n_a;
    const int32_t *vars_b;        /* host or NULL; copied at submit */
    int32_t n_b;
    double *stat;                 /* host outputs n_a x n_b (may be NULL) */
    double *pval;
    int32_t *n;
} napg_request;

/* Starts the serving loop: `slots` concurrent requests (1..64) within
 * `mem_budget` bytes of work memory (0 = 80% of the free device memory). Builds
 * the presort of the continuous variables first (shared by the slots). While
 * serving, napg_load_cohort and napg_release_cache return NAPG_E_BUSY.
 * Errors: NAPG_E_ARG, NAPG_E_BUSY (already started), NAPG_E_OOM, NAPG_E_CUDA. */
napg_status napg_serve_start(napg_ctx *ctx, size_t mem_budget, int32_t slots);

/* Queues a request; *ticket identifies it. The request's host buffers must stay
 * valid until napg_serve_poll reports it done. Errors: NAPG_E_ARG,
 * NAPG_E_BUSY (queue full), NAPG_E_UNSUPPORTED (request larger than the budget). */
napg_status napg_serve_submit(napg_ctx *ctx, const napg_request *req, uint64_t *ticket);

/* *done = 1 once the request's outputs are written; *latency_ms = submit-to-done
 * wall time. *status_out (may be NULL) receives the request's own status. */
napg_status napg_serve_poll(napg_ctx *ctx, uint64_t ticket, int32_t *done, double *latency_ms,
                            int32_t *status_out);

/* Drains the queue, waits for running requests and stops the loop. */
napg_status napg_serve_stop(napg_ctx *ctx);

/* The admission policy of the serving loop on its own (host only, no GPU):
 * queued requests in arrival order with device-memory estimates est[q] and
 * waiting times age_ms[q]; slots holding slot_mem[k] bytes, busy if
 * slot_busy[k]. Each idle slot takes the first queued request whose estimate
 * fits next to the memory of the other slots (a slot keeps what it holds);
 * a request waiting 200 ms or more is not overtaken. assign[k] receives the
 * queue index given to slot k, or -1. Errors: NAPG_E_ARG. */
napg_status napg_serve_plan(const uint64_t *est, const double *age_ms, int32_t nq, const uint64_t *slot_mem,
                            const int32_t *slot_busy, int32_t nslots, uint64_t budget, int32_t *assign);

/* ----------------------------------------------------------------- tracing --
 * With tracing on, every stage of a run (bitmasks, contraction, finalize, ...)
 * is bracketed by CUDA events on the stream it runs on. napg_trace_read waits
 * for the recorded stages, then writes a JSON object
 *   {"stages": {"<name>": {"launches": L, "ms": T}, ...}, "kernel_launches": K}
 * (T = summed device time) into buf (NUL-terminated, truncated to cap) and
 * clears the record. Errors: NAPG_E_ARG, NAPG_E_CUDA. */
napg_status napg_trace_enable(napg_ctx *ctx, int32_t on);
napg_status napg_trace_read(napg_ctx *ctx, char *buf, size_t cap);

/* Autotuner (on by default): the first run of a problem shape times each
 * launch-shape candidate of its tunable kernels once (the B-tile width of the
 * stacked tensor contractions, the samples per pipeline stage of the Sxy
 * contraction, threads per pair of the rank kernels) and keeps the fastest for
 * the context; candidates give identical results. Runs being captured into a
 * CUDA graph use the choice recorded for the nearest shape.
 * napg_tune_read writes the records as JSON
 *   [{"kind": K, "rows_a": A, "rows_b": B, "k": L, "choice": C, "ms": [...]}, ...]
 * napg_tune_pin fixes the candidate of one kind for every later run of the
 * context, without timing; choice -1 unpins. Kinds and their candidates:
 * "stacked_mask", "stacked_onehot", "stacked_onehot_counts_sums",
 * "stacked_observed_squares" (0-3: B-tile width, then 1 or 2 K-blocks per
 * pipeline stage), "sxy_stage_samples", "spearman_threads",
 * "rank_groups_threads" (0-1).
 * Errors: NAPG_E_ARG (NULL context, buffer too small, unknown kind, choice
 * outside [-1, 3]; a choice past the kind's candidates fails at the next run
 * that launches it). */
napg_status napg_tune_enable(napg_ctx *ctx, int32_t on);
napg_status napg_tune_read(napg_ctx *ctx, char *buf, size_t cap);
napg_status napg_tune_pin(napg_ctx *ctx, const char *kind, int32_t choice);

/* Number of kernels this process has launched through the library so far. */
uint64_t napg_kernel_launches(void);

/* ------------------------------------------------------- allocation-free --
 * All-pairs Pearson r, p and n in the plain FP64 form for a small matrix that is
 * already on the GPU, without allocating any memory. (The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, such as code
 * running inside a framework whose own allocator owns the device memory, a
 * process with a hard device-memory cap, or a latency-critical path that must
 * not block in the allocator.)
 *   X          device, n_vars x n_samples doubles, row-major (one row per variable)
 *   missing    the sentinel; NaN means "missing iff NaN"
 *   r, p       device, n_vars x n_vars doubles, row-major (either may be NULL)
 *   n          device, n_vars x n_vars int32 co-observed counts (may be NULL)
 *   stream     cudaStream_t to run on (NULL: the default stream)
 * Work space is one fixed 24 MiB array inside the library, held by every GPU
 * that loads the library until the process exits; the call allocates nothing.
 * Limits: 1 <= n_vars <= 256 and 1 <= n_samples <= 8192; larger requests return
 * NAPG_E_UNSUPPORTED without touching the GPU.
 * The first call on each device looks up the array's device address; make that
 * first call before capturing any stream. Do not use this entry point after
 * resetting the device (cudaDeviceReset) in the same process: the address
 * looked up before the reset may no longer be the array's. All calls share the
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and give wrong results; serialize them. The call returns after its results are written
 * (it reads a status word back), with NAPG_E_NONFINITE if a non-missing value is
 * +-inf or NaN, NAPG_E_ARG for bad arguments and NAPG_E_CUDA on a CUDA error. */
napg_status napg_pearson_fp64_noalloc(const double *X, int32_t n_vars, int32_t n_samples, double missing,
                                      double *r, double *p, int32_t *n, void *stream);

/* Library version string. */
const char *napg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NAPG_H */
