// Internal declarations of the napg library (CUDA, sm_103a). Not installed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/napg.h"

namespace napg {

constexpr int kMaxLevels = NAPG_MAX_LEVELS;
constexpr uint8_t kMissingLabel = 0xFF;
constexpr int64_t kMaxSamples = (int64_t)1 << 24;      // counts stay exact in FP32 sums
constexpr int64_t kMaxRankSamples = 163840;  // per-pair rank state fits shared memory

// Error flags raised by device-side checks (bitwise OR into a device word).
enum : uint32_t { kErrLabel = 1u, kErrNonfinite = 2u, kErrTimeout = 4u, kErrIndex = 8u, kErrExactLimit = 16u };

// A pair whose centred sum falls to rel_tol x its raw sum (about the column's
// in-context mean) is recomputed exactly by the two-pass rescue: for the FP64
// form only true degeneracy (a constant column/group) reaches 1e-9; for the
// mixed form the sums carry ~1e-7 relative error, so the statistic keeps
// |dr| <= 1e-6 only while raw/centred stays small. Every entry point that
// finalizes moments uses these two values, so all of them rescue the same pairs.
constexpr double kPlainRelTol = 1e-9;
constexpr double kMixedRelTol = 0.25;

// Device-resident cohort (Sec. 3.2): one row per variable.
struct Cohort {
    int64_t F = 0, S = 0, W = 0;         // variables, samples, 32-bit words per bit row
    int32_t dtype = NAPG_F64;
    double missing = 0.0;
    bool loaded = false;
    uint64_t gen = 0;                    // unique per load (keys derived data)
    void *X = nullptr;                   // F x S values (input dtype)
    uint32_t *obs = nullptr;             // F x W observed bits (no context applied)
    uint8_t *lab = nullptr;              // n_cat x S labels (kMissingLabel = missing)
    std::vector<uint8_t> vtype;          // host copies
    std::vector<int32_t> nlev;
    std::vector<int32_t> cat_index;      // var -> categorical row (or -1)
    std::vector<int32_t> cont_index;     // var -> continuous row (or -1)
    int64_t n_cat = 0, n_cont = 0;
    // presort of every continuous variable (built on first rank test, kept):
    bool sorted = false;
    int32_t *perm = nullptr;             // n_cont x S: sample ids in value order (observed only)
    int32_t *pos = nullptr;              // n_cont x S: position of each sample in that order (-1 if missing)
    int32_t *nobs = nullptr;             // n_cont observed counts
    uint32_t *tie = nullptr;             // n_cont x W: bit p set when position p starts a tie group
    int32_t *gsw = nullptr;              // n_cont x W: start of the group open at word w's first position
    int32_t *gew = nullptr;              // n_cont x W: first group start after word w (or nobs)
    int64_t presort_cap = 0;             // samples the presort arrays hold (per variable)
    int32_t *cont_vars_dev = nullptr;    // the continuous variable ids (device), for the presort
    bool owns = true;                    // false: arrays borrowed (freed by their owner)
    size_t x_bytes = 0, obs_bytes = 0, lab_bytes = 0;   // allocated sizes (napg_load_cohort reuses them)
};

// Grow-only named device buffers; a run asks for capacity and gets a pointer.
struct Workspace {
    enum Slot {
        kCtxBits, kObsA, kObsB, kShiftA, kShiftB, kXsA, kXsB, kVarA, kLevBits, kLevCnt,
        kLevPresent, kMomA, kMomB, kMomC, kMomD, kMomE, kMomF, kIntA, kIntB, kIntC, kFlagList,
        kCounter, kOutStat, kOutP, kOutN, kMask, kVarsDev, kTmpA, kTmpB, kTmpC, kTmpD, kTmpE,
        kTmpF, kTmpG, kVsq, kUnionS, kUnionP, kUnionN, kExp, kPjJobs, kPjSorted, kPjMeta, kPlShift, kPlVsq,
        kPresortTmp, kBgrat, kUnionE1, kUnionE2, kOutE1, kOutE2, kAdjKeys, kAdjVals, kAdjTmp,
        kOutStatB, kOutPB, kOutNB, kOutE1B, kOutE2B, kLargeA, kPartS, kPartP, kPartN, kPartOwn, kNumSlots
    };
    void *ptr[kNumSlots] = {};
    size_t cap[kNumSlots] = {};
    // The FP16 planes in kTmpA..kTmpE (with kExp, kPlShift, kPlVsq) describe the
    // variables `vars` of cohort generation `gen` without a sample context; a
    // later run on the same list reuses them. Cleared when a slot is reallocated.
    struct PlaneKey {
        bool valid = false;
        uint64_t gen = 0;
        std::vector<int32_t> vars;
    } plane_key;
    bool bgrat_ready = false;   // kBgrat holds the p-value expansion coefficients
    // kLargeA holds the sf::LargeATab entries for 2a <= lat_n2a, 2b <= lat_rows
    bool lat_ready = false;
    int32_t lat_n2a = 0, lat_rows = 0;
    static bool plane_slot(int s) { return (s >= kTmpA && s <= kTmpE) || s == kExp || s == kPlShift || s == kPlVsq; }
    size_t total() const {
        size_t t = 0;
        for (int i = 0; i < kNumSlots; ++i) t += cap[i];
        return t;
    }
};

// ---- autotuner (tune.cu)
enum TuneKind : int { kTuneStackMask = 1, kTuneStackOneHot = 2, kTuneSpearman = 3, kTuneRankGroups = 4,
                      kTuneStackOneHotNS1 = 5, kTuneStackSquares = 6, kTuneSxy = 7, kTuneKindMax = 7 };
struct TuneKey {
    int kind;
    int64_t a, b, c;    // rows of A, rows of B, K length (shape of the problem)
    bool operator<(const TuneKey &o) const {
        if (kind != o.kind) return kind < o.kind;
        if (a != o.a) return a < o.a;
        if (b != o.b) return b < o.b;
        return c < o.c;
    }
};
struct TuneRec { int choice; std::vector<float> ms; };
struct Tuner {
    std::mutex mu;
    bool on = true;
    std::map<TuneKey, TuneRec> best;
    std::map<int, int> pinned;      // kind -> candidate fixed by napg_tune_pin
};

struct ServeState;   // serving loop (serve.cu)
struct BatchState;   // batched contexts (batch.cu)

// Stage timing with CUDA events (napg_trace_*).
struct Tracer {
    bool on = false;
    struct Rec { std::string name; cudaEvent_t a, b; uint64_t launches; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    struct Agg { uint64_t launches = 0; double ms = 0.0; };
    std::vector<std::pair<std::string, Agg>> agg;
    std::mutex mu;
};

// counts every kernel launch made by the library
void count_launch(uint64_t k = 1);
uint64_t launches_so_far();
void uncount_launches(uint64_t k);

// RAII: records an event pair around a stage when tracing is on
struct Stage {
    Tracer *tr; cudaStream_t st; std::string name; cudaEvent_t a = nullptr; uint64_t l0 = 0;
    Stage(Tracer &t, cudaStream_t s, const char *n);
    void end();          // records the end now (the destructor then does nothing)
    ~Stage() { end(); }
};

}  // namespace napg

struct napg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    napg::Cohort coh;
    napg::Workspace ws;
    std::string err;
    uint32_t *dev_err = nullptr;       // device error word for checks
    uint32_t *host_err = nullptr;      // pinned mirror
    napg::ServeState *serve = nullptr;
    napg::BatchState *batch = nullptr;
    napg::Tracer trace;
    napg::Tuner tune;
    std::mutex mu;                     // guards cohort/workspace use from the serving threads
    // asynchronous host outputs: two staging sets (kOut* and kOut*B), copied to
    // the host on copy_stream; ev_copy[k] marks set k's last copy done
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_run[2] = {nullptr, nullptr}, ev_copy[2] = {nullptr, nullptr};
    bool copy_used[2] = {false, false};
    int stage_set = 0;
};

namespace napg {

napg_status fail(napg_ctx *ctx, napg_status code, const std::string &msg);
napg_status cuda_fail(napg_ctx *ctx, cudaError_t e, const char *what);
void *ws_get(napg_ctx *ctx, Workspace &ws, int slot, size_t bytes, napg_status *st);
bool is_device_ptr(const void *p);

// One test over vars_a x vars_b on a given stream and workspace (shared by
// napg_run, napg_run_batch and the serving slots).
struct RunArgs {
    int32_t test;
    napg_options opt;
    Cohort *coh;              // cohort to run on (NULL: the context's)
    bool no_plane_cache;      // never reuse FP16 planes across runs
    // variable lists already on the device, as run_on_stream would stage them
    // ([va | vb | crow_a | crow_b | catrow | nlev | levoff]); NULL: stage them
    const int32_t *dints;
    const size_t *dints_off;
    const uint8_t *mask;      // host or device (mask_on_device tells)
    bool mask_on_device;
    const int32_t *va;        // host
    int32_t na;
    const int32_t *vb;        // host or NULL
    int32_t nb;
    double *stat, *pval;      // device buffers (n_a x n_b) or NULL
    int32_t *n;
    double *es1, *es2;        // effect sizes (device, n_a x n_b) or NULL: Table 2's effect size, and
                              // Cramer's V for chi-squared (NaN for the other tests)
    // symmetric calls split by napg_run_part (NULL: every row): own[i] != 0 for
    // the output rows i this part computes (pairs i <= j of the upper triangle)
    const uint8_t *own;
};

// Split of a call's output rows over parts (napg_run_part): rows go in blocks
// of kPartRows, dealt to the parts back and forth (0, 1, ..., n-1, n-1, ..., 1,
// 0, 0, 1, ...) so that the blocks of a triangle's long and short rows pair up.
constexpr int kPartRows = NAPG_PART_ROWS;
__host__ __device__ inline int part_of_row(int64_t row, int nparts) {
    const int64_t b = row / kPartRows, r = b / nparts, k = b - r * nparts;
    return (int)((r & 1) ? nparts - 1 - k : k);
}
// a tile of rows [r0, r0 + len) of a split call takes part in it when any row is owned
__host__ __device__ inline bool rows_owned(const uint8_t *own, int64_t r0, int64_t len, int64_t rows) {
    if (!own) return true;
    const int64_t r1 = r0 + len < rows ? r0 + len : rows;
    for (int64_t r = r0; r < r1; ++r)
        if (own[r]) return true;
    return false;
}
napg_status run_on_stream(napg_ctx *ctx, Workspace &ws, cudaStream_t st, const RunArgs &a);
void free_cohort(Cohort &c);
uint64_t next_cohort_gen();
napg_status run_with_outputs(napg_ctx *ctx, Workspace &ws, cudaStream_t st, RunArgs a, bool symmetric_shape);
// orders the context stream after every pending host-output copy (device-side wait)
napg_status wait_pending_copies(napg_ctx *ctx);
// runs run(choice) with the launch shape the autotuner picks for `key`
napg_status tuned_launch(napg_ctx *ctx, const TuneKey &key, int ncand, const std::function<napg_status(int)> &run,
                         cudaStream_t st);
napg_status run_batch(napg_ctx *ctx, const RunArgs &a0, int32_t n_ctx, const uint8_t *const *masks,
                      double *const *stat, double *const *pval, int32_t *const *n);
void free_batch(napg_ctx *ctx);
napg_status check_run_vars(napg_ctx *ctx, const RunArgs &a, bool *symmetric);
void var_lists(const Cohort &c, const RunArgs &a, bool symmetric, std::vector<int32_t> &va,
               std::vector<int32_t> &vb, std::vector<int32_t> &catrow, std::vector<int32_t> &nlev,
               std::vector<int32_t> &levoff, int32_t &R, int32_t &maxlev, std::vector<int32_t> &all,
               std::vector<size_t> &off);
napg_status ensure_presort(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st);

// ---- kernel launchers (defined in the .cu files) ---------------------------
}  // namespace napg
#include "pjobs.cuh"
namespace napg {
void launch_pjobs_eval(const PJobQueue &q, PJob *sorted, int32_t *offs, int32_t *cursor, double *pval,
                       cudaStream_t st, int sm_count);
void launch_bgrat_table(double *tab, cudaStream_t st);
void launch_large_a_table(double2 *v, int32_t n2a, int32_t rows, cudaStream_t st);
void launch_debug_pvalues(int32_t kind, const double *s, const double *a, const double *b, int64_t count, double *p,
                          const double *bgrat, cudaStream_t st);
// prep
void launch_validate_obs(const void *X, int32_t dtype, int64_t F, int64_t S, int64_t W, double missing,
                         const uint8_t *vtype_dev, const int32_t *nlev_dev, const int32_t *catrow_dev,
                         uint32_t *obs, uint8_t *lab, uint32_t *err, cudaStream_t st, void *copy_to = nullptr);
void launch_transpose(const void *in, void *out, int32_t dtype, int64_t rows, int64_t cols, cudaStream_t st);
void launch_ctx_bits(const uint8_t *mask, int64_t S, int64_t W, uint32_t *ctxw, cudaStream_t st);
void launch_gather_obs(const uint32_t *obs, const int32_t *vars_dev, int32_t nv, const uint32_t *ctxw,
                       int64_t W, uint32_t *out, cudaStream_t st);
void launch_shift_values(const void *X, int32_t dtype, int64_t S, int64_t S_pad, const int32_t *vars_dev,
                         int32_t nv, const uint32_t *obsv, int64_t W, double *shift, double *xs,
                         cudaStream_t st);
void launch_level_bits(const uint8_t *lab, int64_t S, int64_t W, const int32_t *catrow_dev,
                       const int32_t *levoff_dev, const int32_t *nlev_dev, int32_t nv,
                       const uint32_t *obsv, uint32_t *levbits, int32_t *levcnt, cudaStream_t st);
// plain FP64 moments
void launch_pearson_fp64(const double *xs, int64_t S_pad, const uint32_t *obsv, int64_t W, int32_t nv,
                         double *Sxy, double *Sx, double *Sxx, int32_t *nn, cudaStream_t st,
                         const uint8_t *own = nullptr);
void launch_groupsum_fp64(const uint8_t *lab, int64_t S, const int32_t *catrow_dev, int32_t na,
                          const int32_t *levoff_dev, const int32_t *nlev_dev, const double *xs,
                          int64_t S_pad, const uint32_t *obsb, int64_t W, int32_t nb,
                          int32_t *gn, double *g1, double *g2, int32_t max_levels, cudaStream_t st);
// contingency tables
void launch_contingency(const uint32_t *levbits, int64_t W, int32_t R, int32_t *T, const uint8_t *own_lev,
                        cudaStream_t st);
// own_lev[levoff[a] + g] = own[a] for the levels g of every variable a
void launch_level_ownership(const uint8_t *own, const int32_t *levoff, const int32_t *nlev, int32_t na,
                            uint8_t *own_lev, cudaStream_t st);
// finalize (p-values included)
struct PearsonFin {
    const double *Sxy, *Sx, *Sxx; const int32_t *nn; const double *shift; int32_t nv;
    double rel_tol;      // ill-conditioned when a centred sum <= rel_tol x its raw sum
    const double *vsq;   // mixed form: Sxx holds sum (x~^2 - v) m; add v n back (NULL: plain)
    PJobQueue q;         // p-value jobs (q.jobs NULL: no p-values wanted)
    const int32_t *vars; // variable ids of the rows (NULL: rows are distinct variables)
    const uint8_t *own;  // split calls: rows computed (NULL: all)
};
void launch_finalize_pearson(const PearsonFin &f, double *stat, double *pval, int32_t *nout,
                             int32_t *flag_list, int32_t *flag_count, cudaStream_t st);
struct GroupFin {
    const int32_t *gn; const double *g1, *g2; int32_t total_rows;
    const int32_t *levoff, *nlev, *present; int32_t na, nb; int32_t test; int32_t welch;
    double rel_tol;
    const double *vsq;   // mixed form: g2 holds sum (x~^2 - v); add v n_g back (NULL: plain)
    PJobQueue q;
    const double *g2tot; // ANOVA, mixed form: [na][nb] sum (x~^2 - v) over all co-observed samples
                         // (then g2 is not read); NULL: per-level g2
    double *es;          // t-test: Cohen's d per pair (NULL: not asked)
    double *es2;         // t-test: degrees of freedom of the t distribution per pair (NULL: not asked)
};
void launch_finalize_groups(const GroupFin &f, double *stat, double *pval, int32_t *nout,
                            int32_t *flag_list, int32_t *flag_count, cudaStream_t st);
struct Chi2Fin {
    const int32_t *T; int32_t R; const int32_t *levoff_a, *nlev_a, *levoff_b, *nlev_b;
    const int32_t *present; int32_t na, nb; int32_t symmetric; int32_t yates;
    PJobQueue q;
    int32_t maxc;        // most levels of any variable in the call
    const uint8_t *own;  // split symmetric calls: rows (variables of A) computed (NULL: all)
};
void launch_finalize_chi2(const Chi2Fin &f, double *stat, double *pval, int32_t *nout, cudaStream_t st);
// exact rescue of pairs whose moments are degenerate (constant columns/groups)
struct RescueArgs {
    const void *X; int32_t dtype; int64_t S; int64_t W; const uint32_t *ctxw; const uint32_t *obs;
    const uint8_t *lab; const int32_t *catrow; const int32_t *va, *vb; int32_t na, nb; int32_t test;
    int32_t welch; const int32_t *nlev_a; const int32_t *present; const int32_t *levoff;
    double *es;          // t-test: Cohen's d of the rescued pairs (NULL: not asked)
    double *es2;         // t-test: degrees of freedom of the rescued pairs (NULL: not asked)
    PJobQueue q;         // the call's p-value jobs (q.jobs NULL: the rescue forms p itself)
};
void launch_rescue(const RescueArgs &r, const int32_t *flag_list, const int32_t *flag_count, int32_t max_flags,
                   double *stat, double *pval, int32_t *nout, int32_t symmetric, int32_t max_levels,
                   cudaStream_t st);
void launch_rescue_serial(const RescueArgs &r, const int32_t *flag_list, const int32_t *flag_count, int32_t max_flags,
                          double *stat, double *pval, int32_t *nout, int32_t symmetric, cudaStream_t st);
// effect sizes from the final statistics (the t-test's Cohen's d comes from the
// group finalize and the rescue)
struct EffectArgs {
    int32_t test, na, nb, symmetric;
    const double *stat; const int32_t *n;
    const int32_t *levcnt, *levoff, *nlev;   // in-context level counts, per categorical of vars_a
    const int32_t *rcnt; const int64_t *tie; // Mann-Whitney: per-level counts [R][nb], tie terms [na][nb]
    double *es1, *es2;
};
void launch_effects(const EffectArgs &e, cudaStream_t st);
// multiple-testing correction of a p-value matrix (device buffers)
napg_status adjust_pvalues(napg_ctx *ctx, Workspace &ws, cudaStream_t st, int32_t method, const double *p,
                           int64_t rows, int64_t cols, int32_t symmetric, double *out);
// ranks
void launch_presort(const void *X, int32_t dtype, int64_t S, int64_t W, const int32_t *contvars_dev,
                    int32_t ncont, const uint32_t *obs, int32_t *perm, int32_t *pos, int32_t *nobs,
                    uint32_t *tie, int32_t *gsw, int32_t *gew, void *tmp, size_t tmp_bytes, cudaStream_t st);
size_t presort_tmp_bytes(int64_t S, int32_t ncont);
struct RankData {
    const int32_t *perm, *pos, *nobs; const uint32_t *tie; const int32_t *gsw, *gew;
    int64_t S, W;
};
void launch_spearman_pairs(const RankData &rd, const int32_t *crow_a, const int32_t *crow_b,
                           const uint32_t *obs_a, const uint32_t *obs_b, int32_t na, int32_t nb,
                           int32_t symmetric, int64_t *out4, cudaStream_t st, int threads = 0,
                           const uint8_t *own = nullptr);
int rank_threads_default(int64_t W, bool groups);
void launch_rank_groups(const RankData &rd, const uint8_t *lab, const int32_t *catrow_a,
                        const int32_t *nlev_a, const int32_t *levoff_a, int32_t na, const int32_t *crow_b,
                        const uint32_t *obs_a, const uint32_t *obs_b, int32_t nb, int32_t max_levels,
                        int64_t *rsum, int32_t *rcnt, int64_t *tie_term, cudaStream_t st, int threads = 0);
struct SpearmanFin {
    const int64_t *q; int32_t na, nb; int32_t symmetric; PJobQueue pq;
    const uint8_t *own;  // split symmetric calls: rows computed (NULL: all)
};
void launch_finalize_spearman(const SpearmanFin &f, double *stat, double *pval, int32_t *nout, cudaStream_t st);
struct RankGroupFin {
    const int64_t *rsum; const int32_t *rcnt; const int64_t *tie_term; int32_t total_rows;
    const int32_t *levoff, *nlev, *present; int32_t na, nb; int32_t test; int32_t mwu_mode; int32_t mwu_cc;
    PJobQueue q;
};
void launch_finalize_rankgroups(const RankGroupFin &f, double *stat, double *pval, int32_t *nout,
                                int32_t *flag_list, int32_t *flag_count, cudaStream_t st);
void launch_mwu_exact(const double *stat, const int32_t *rcnt, const int32_t *levoff, int32_t total_rows,
                      int32_t nb, const int32_t *flag_list, const int32_t *flag_count, int32_t max_flags,
                      double *pval, void *scratch, size_t scratch_bytes, uint32_t *err, cudaStream_t st);
// the status a finished call reports for the device error word `bits` (timeouts
// first, then forced exact Mann-Whitney p-values beyond the exact range)
napg_status device_error_status(napg_ctx *ctx, uint32_t bits);
size_t mwu_exact_scratch_bytes(int64_t S, bool forced);
void launch_fill_nan(double *p, int64_t count, cudaStream_t st);

// mixed precision (tcgen05) path
struct MixedPlan;
// cache_vars: host copy of the variable list when the run has no sample context
// (the planes may then be reused by the next run on the same list), else NULL
napg_status mixed_pearson(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st, const int32_t *vars_dev, int32_t nv,
                          const uint32_t *obsv, double *Sxy, double *Sx, double *Sxx, int32_t *nn,
                          double *shift_out, double *vsq_out, const std::vector<int32_t> *cache_vars,
                          const uint8_t *own = nullptr);
napg_status mixed_groupsum(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st, const uint32_t *levbits, int32_t R,
                           const int32_t *vars_b_dev, int32_t nb, const uint32_t *obsb, int32_t *gn,
                           double *g1, double *g2, double *shift_out, double *vsq_out,
                           const std::vector<int32_t> *cache_vars,
                           const uint32_t *obsa = nullptr, int32_t na = 0, double *g2tot = nullptr);
napg_status mixed_contingency(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st, const uint32_t *levbits,
                              int32_t R, int32_t *T, const uint8_t *own_lev = nullptr);

}  // namespace napg

#define NAPG_CU(ctx, call)                                           \
    do {                                                             \
        cudaError_t e__ = (call);                                    \
        if (e__ != cudaSuccess) return napg::cuda_fail((ctx), e__, #call); \
    } while (0)

#define NAPG_ST(expr)                                                \
    do {                                                             \
        napg_status s__ = (expr);                                    \
        if (s__ != NAPG_OK) return s__;                              \
    } while (0)
