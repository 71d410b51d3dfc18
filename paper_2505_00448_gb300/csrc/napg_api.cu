// C ABI of the napg library: contexts, cohort upload and validation, and the
// per-test pipelines (bitmasks -> contraction or rank kernel -> finalize ->
// exact rescue), all ordered on one CUDA stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>

#include "napg_internal.cuh"

namespace napg {

uint64_t next_cohort_gen() {
    static std::atomic<uint64_t> g{0};
    return ++g;
}

napg_status fail(napg_ctx *ctx, napg_status code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

napg_status cuda_fail(napg_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? NAPG_E_OOM : NAPG_E_CUDA, m);
}

void *ws_get(napg_ctx *ctx, Workspace &ws, int slot, size_t bytes, napg_status *st) {
    bytes = ((std::max<size_t>(bytes, 16) + 255) / 256) * 256;
    if (ws.cap[slot] >= bytes) return ws.ptr[slot];
    if (Workspace::plane_slot(slot)) ws.plane_key.valid = false;
    if (slot == Workspace::kBgrat) ws.bgrat_ready = false;
    if (slot == Workspace::kLargeA) ws.lat_ready = false;
    if (ws.ptr[slot]) {
        cudaFree(ws.ptr[slot]);
        ws.ptr[slot] = nullptr;
        ws.cap[slot] = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        *st = cuda_fail(ctx, e, "cudaMalloc(workspace)");
        return nullptr;
    }
    ws.ptr[slot] = p;
    ws.cap[slot] = bytes;
    return p;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void free_cohort(Cohort &c) {
    void *ptrs[] = {c.X, c.obs, c.lab, c.perm, c.pos, c.nobs, c.tie, c.gsw, c.gew, c.cont_vars_dev};
    if (c.owns) {
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
    c = Cohort();
}

static void free_ws(Workspace &ws) {
    for (int i = 0; i < Workspace::kNumSlots; ++i)
        if (ws.ptr[i]) cudaFree(ws.ptr[i]);
    ws = Workspace();
}

// ---------------------------------------------------------------- helpers --

#define WS(slot, type, count)                                                         \
    ([&]() -> type * {                                                                \
        napg_status s_ = NAPG_OK;                                                     \
        type *p_ = (type *)ws_get(ctx, ws, Workspace::slot, sizeof(type) * (size_t)(count), &s_); \
        if (!p_) st_ = s_;                                                            \
        return p_;                                                                    \
    }())

struct HostLists {
    std::vector<int32_t> va, vb, crow_a, crow_b, catrow, nlev, levoff;
    int32_t R = 0, maxlev = 0;
};

napg_status check_run_vars(napg_ctx *ctx, const RunArgs &a, bool *symmetric) {
    const Cohort &c = a.coh ? *a.coh : ctx->coh;
    const int t = a.test;
    if (t < NAPG_PEARSON || t > NAPG_KRUSKAL) return fail(ctx, NAPG_E_ARG, "unknown test");
    if (a.na < 0 || a.nb < 0 || (a.na > 0 && !a.va)) return fail(ctx, NAPG_E_ARG, "bad variable list");
    const bool homo = (t == NAPG_PEARSON || t == NAPG_SPEARMAN || t == NAPG_CHI2);
    *symmetric = (a.vb == nullptr);
    if (!homo && *symmetric) return fail(ctx, NAPG_E_ARG, "categorical x continuous tests need vars_b");
    const int want_a = (t == NAPG_PEARSON || t == NAPG_SPEARMAN) ? 0 : 1;
    const int want_b = (t == NAPG_CHI2) ? 1 : 0;
    for (int i = 0; i < a.na; ++i) {
        const int v = a.va[i];
        if (v < 0 || v >= c.F) return fail(ctx, NAPG_E_ARG, "vars_a index out of range");
        if (c.vtype[v] != want_a) return fail(ctx, NAPG_E_ARG, "vars_a has a variable of the wrong type");
        if ((t == NAPG_TTEST || t == NAPG_MWU) && c.nlev[v] != 2)
            return fail(ctx, NAPG_E_ARG, "t-test / Mann-Whitney need 2 levels in vars_a");
        if ((t == NAPG_ANOVA || t == NAPG_KRUSKAL) && c.nlev[v] < 2)
            return fail(ctx, NAPG_E_ARG, "ANOVA / Kruskal-Wallis need >= 2 levels in vars_a");
    }
    if (!*symmetric) {
        for (int i = 0; i < a.nb; ++i) {
            const int v = a.vb[i];
            if (v < 0 || v >= c.F) return fail(ctx, NAPG_E_ARG, "vars_b index out of range");
            if (c.vtype[v] != want_b) return fail(ctx, NAPG_E_ARG, "vars_b has a variable of the wrong type");
        }
    }
    if ((t == NAPG_SPEARMAN || t == NAPG_MWU || t == NAPG_KRUSKAL) && c.S > kMaxRankSamples)
        return fail(ctx, NAPG_E_UNSUPPORTED, "rank tests support at most 163840 samples");
    return NAPG_OK;
}

static void level_lists(const Cohort &c, const std::vector<int32_t> &vars, std::vector<int32_t> &catrow,
                        std::vector<int32_t> &nlev, std::vector<int32_t> &levoff, int32_t &R, int32_t &maxlev) {
    catrow.resize(vars.size());
    nlev.resize(vars.size());
    levoff.resize(vars.size());
    R = 0;
    maxlev = 0;
    for (size_t i = 0; i < vars.size(); ++i) {
        catrow[i] = c.cat_index[vars[i]];
        nlev[i] = c.nlev[vars[i]];
        levoff[i] = R;
        R += nlev[i];
        maxlev = std::max(maxlev, nlev[i]);
    }
}

// upload a host int32 vector into a slice of one workspace slot
struct DevInts {
    std::vector<int32_t> all;
    std::vector<size_t> off;
    size_t add(const std::vector<int32_t> &v) {
        off.push_back(all.size());
        all.insert(all.end(), v.begin(), v.end());
        return off.size() - 1;
    }
};

__global__ void k_gather_block(const double *sstat, const double *sp, const int32_t *sn, int32_t nu,
                               const int32_t *ia, const int32_t *ib, int32_t na, int32_t nb, double *stat, double *p,
                               int32_t *n) {
    const int64_t total = (int64_t)na * nb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / nb), b = (int)(t - (int64_t)a * nb);
        const int64_t src = (int64_t)ia[a] * nu + ib[b];
        if (stat) stat[t] = sstat[src];
        if (p) p[t] = sp[src];
        if (n) n[t] = sn[src];
    }
}

// ------------------------------------------------------------ run pipeline --

// Presort of every continuous variable of `c`: stream-ordered, no host
// synchronisation; the arrays are allocated (or grown) only when too small, so a
// run whose sizes were seen before makes no allocation (graph capture relies on it).
napg_status ensure_presort(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st) {
    if (c.sorted || c.n_cont == 0) {
        c.sorted = true;
        return NAPG_OK;
    }
    const int64_t nc = c.n_cont, S = c.S, W = c.W;
    if (c.presort_cap < S) {
        if (!c.owns) return fail(ctx, NAPG_E_ARG, "presort arrays of a borrowed cohort are too small");
        void *old[] = {c.perm, c.pos, c.nobs, c.tie, c.gsw, c.gew};
        for (void *p : old)
            if (p) cudaFree(p);
        const int64_t Wc = (S + 31) / 32;
        NAPG_CU(ctx, cudaMalloc(&c.perm, sizeof(int32_t) * nc * S));
        NAPG_CU(ctx, cudaMalloc(&c.pos, sizeof(int32_t) * nc * S));
        NAPG_CU(ctx, cudaMalloc(&c.nobs, sizeof(int32_t) * nc));
        NAPG_CU(ctx, cudaMalloc(&c.tie, sizeof(uint32_t) * nc * Wc));
        NAPG_CU(ctx, cudaMalloc(&c.gsw, sizeof(int32_t) * nc * Wc));
        NAPG_CU(ctx, cudaMalloc(&c.gew, sizeof(int32_t) * nc * Wc));
        c.presort_cap = S;
    }
    const size_t tb = presort_tmp_bytes(S, (int32_t)nc);
    napg_status st_ = NAPG_OK;
    void *tmp = ws_get(ctx, ws, Workspace::kPresortTmp, tb, &st_);
    if (st_) return st_;
    { Stage s_(ctx->trace, st, "presort"); launch_presort(c.X, c.dtype, S, W, c.cont_vars_dev, (int32_t)nc, c.obs, c.perm, c.pos, c.nobs, c.tie, c.gsw, c.gew, tmp, tb, st); }
    NAPG_CU(ctx, cudaGetLastError());
    c.sorted = true;
    return NAPG_OK;
}

// P-value job queue of one run (see pjobs.cuh)
struct PJobBufs {
    PJobQueue q{};
    PJob *sorted = nullptr;
    int32_t *offs = nullptr, *cursor = nullptr;
};

constexpr size_t kLargeATabMaxBytes = (size_t)128 << 20;

static napg_status pjobs_setup(napg_ctx *ctx, Workspace &ws, cudaStream_t st, int64_t capacity, bool want,
                               PJobBufs &b) {
    b = PJobBufs();
    if (!want || capacity <= 0) return NAPG_OK;
    if (capacity > INT32_MAX - 1) return fail(ctx, NAPG_E_UNSUPPORTED, "too many pairs in one call");
    napg_status st_ = NAPG_OK;
    b.q.jobs = (PJob *)ws_get(ctx, ws, Workspace::kPjJobs, sizeof(PJob) * (size_t)capacity, &st_);
    b.sorted = (PJob *)ws_get(ctx, ws, Workspace::kPjSorted, sizeof(PJob) * (size_t)capacity, &st_);
    int32_t *meta = (int32_t *)ws_get(ctx, ws, Workspace::kPjMeta, sizeof(int32_t) * (1 + 3 * kPjBins), &st_);
    if (st_) return st_;
    b.q.count = meta;
    b.q.hist = meta + 1;
    b.offs = meta + 1 + kPjBins;
    b.cursor = meta + 1 + 2 * kPjBins;
    b.q.capacity = (int32_t)capacity;
    NAPG_CU(ctx, cudaMemsetAsync(meta, 0, sizeof(int32_t) * (1 + kPjBins), st));
    // expansion coefficients of the large-parameter incomplete beta, once per workspace
    double *tab = (double *)ws_get(ctx, ws, Workspace::kBgrat, sizeof(double) * sf::kBgratRows * sf::kBgratTerms, &st_);
    if (st_) return st_;
    if (!ws.bgrat_ready) {
        launch_bgrat_table(tab, st);
        NAPG_CU(ctx, cudaGetLastError());
        ws.bgrat_ready = true;
    }
    b.q.bgrat = tab;
    // (log M, 1/T^2) of the large-a expansion for every degrees-of-freedom value
    // the cohort's tests can produce (2a <= S, 2b <= levels - 1), once per
    // workspace. Not while a graph is captured: a replay must not hold a pointer
    // that a later, larger table frees (the jobs then form the values themselves).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NAPG_CU(ctx, cudaStreamIsCapturing(st, &cap));
    if (cap == cudaStreamCaptureStatusNone) {
        int32_t maxlev = 0;
        for (size_t v = 0; v < ctx->coh.nlev.size(); ++v)
            if (ctx->coh.vtype[v] == 1) maxlev = std::max(maxlev, ctx->coh.nlev[v]);
        const int32_t rows = std::min(64, std::max(1, maxlev - 1));
        const int64_t n2a = ctx->coh.S;
        const size_t bytes = sizeof(double2) * (size_t)rows * (size_t)(n2a + 1);
        if (n2a > 0 && bytes <= kLargeATabMaxBytes) {
            double2 *lt = (double2 *)ws_get(ctx, ws, Workspace::kLargeA, bytes, &st_);
            if (st_) return st_;
            if (!ws.lat_ready || ws.lat_n2a < n2a || ws.lat_rows < rows) {
                launch_large_a_table(lt, (int32_t)n2a, rows, st);
                NAPG_CU(ctx, cudaGetLastError());
                ws.lat_ready = true;
                ws.lat_n2a = (int32_t)n2a;
                ws.lat_rows = rows;
            }
            b.q.lat = sf::LargeATab{lt, ws.lat_n2a, ws.lat_rows};
        }
    }
    return NAPG_OK;
}

static void pjobs_run(napg_ctx *ctx, const PJobBufs &b, double *pval, cudaStream_t st) {
    if (!b.q.jobs || !pval) return;
    Stage s_(ctx->trace, st, "pvalues");
    launch_pjobs_eval(b.q, b.sorted, b.offs, b.cursor, pval, st, ctx->sm_count);
}

// Host lists of one run, concatenated as they are staged on the device:
// [va | vb | crow_a | crow_b | catrow | nlev | levoff] with their offsets.
void var_lists(const Cohort &c, const RunArgs &a, bool symmetric, std::vector<int32_t> &va,
               std::vector<int32_t> &vb, std::vector<int32_t> &catrow, std::vector<int32_t> &nlev,
               std::vector<int32_t> &levoff, int32_t &R, int32_t &maxlev, std::vector<int32_t> &all,
               std::vector<size_t> &off) {
    const int t = a.test;
    const int32_t na = a.na, nb = symmetric ? a.na : a.nb;
    va.assign(a.va, a.va + a.na);
    if (!symmetric) vb.assign(a.vb, a.vb + a.nb);
    else vb = va;
    std::vector<int32_t> crow_a(na), crow_b(nb);
    for (int i = 0; i < na; ++i) crow_a[i] = c.cont_index[va[i]];
    for (int i = 0; i < nb; ++i) crow_b[i] = c.cont_index[vb[i]];
    R = 0;
    maxlev = 0;
    catrow.clear();
    nlev.clear();
    levoff.clear();
    if (t != NAPG_PEARSON && t != NAPG_SPEARMAN) level_lists(c, va, catrow, nlev, levoff, R, maxlev);
    DevInts di;
    di.add(va);
    di.add(vb);
    di.add(crow_a);
    di.add(crow_b);
    di.add(catrow);
    di.add(nlev);
    di.add(levoff);
    all = di.all;
    off = di.off;
}

napg_status run_on_stream(napg_ctx *ctx, Workspace &ws, cudaStream_t st, const RunArgs &a) {
    Cohort &c = a.coh ? *a.coh : ctx->coh;
    if (!c.loaded) return fail(ctx, NAPG_E_ARG, "no cohort loaded");
    bool symmetric = false;
    NAPG_ST(check_run_vars(ctx, a, &symmetric));
    const int t = a.test;
    const int64_t S = c.S, W = c.W, S_pad = ((S + 31) / 32) * 32;
    const bool mixed = a.opt.precision == NAPG_MIXED;
    const int32_t na = a.na, nb = symmetric ? a.na : a.nb;
    if (na == 0 || nb == 0) return NAPG_OK;
    napg_status st_ = NAPG_OK;

    // Pearson / chi-squared on A x B: run the symmetric problem on the union of
    // the two lists and gather the block.
    if (!symmetric && (t == NAPG_PEARSON || t == NAPG_CHI2)) {
        std::vector<int32_t> u(a.va, a.va + a.na);
        u.insert(u.end(), a.vb, a.vb + a.nb);
        std::vector<int32_t> uniq = u;
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        const int32_t nu = (int32_t)uniq.size();
        std::vector<int32_t> ia(a.na), ib(a.nb);
        for (int i = 0; i < a.na; ++i) ia[i] = (int32_t)(std::lower_bound(uniq.begin(), uniq.end(), a.va[i]) - uniq.begin());
        for (int i = 0; i < a.nb; ++i) ib[i] = (int32_t)(std::lower_bound(uniq.begin(), uniq.end(), a.vb[i]) - uniq.begin());
        double *ts = WS(kUnionS, double, (int64_t)nu * nu);
        double *tp = WS(kUnionP, double, (int64_t)nu * nu);
        int32_t *tn = WS(kUnionN, int32_t, (int64_t)nu * nu + 2 * (nu + a.na + a.nb));
        if (st_) return st_;
        double *te1 = a.es1 ? WS(kUnionE1, double, (int64_t)nu * nu) : nullptr;
        double *te2 = a.es2 ? WS(kUnionE2, double, (int64_t)nu * nu) : nullptr;
        if (st_) return st_;
        RunArgs b = a;
        b.va = uniq.data();
        b.na = nu;
        b.vb = nullptr;
        b.nb = 0;
        b.stat = ts;
        b.pval = tp;
        b.n = tn;
        b.es1 = te1;
        b.es2 = te2;
        NAPG_ST(run_on_stream(ctx, ws, st, b));
        int32_t *dia = tn + (int64_t)nu * nu, *dib = dia + a.na;
        NAPG_CU(ctx, cudaMemcpyAsync(dia, ia.data(), sizeof(int32_t) * a.na, cudaMemcpyHostToDevice, st));
        NAPG_CU(ctx, cudaMemcpyAsync(dib, ib.data(), sizeof(int32_t) * a.nb, cudaMemcpyHostToDevice, st));
        const int64_t tot = (int64_t)a.na * a.nb;
        count_launch();
        k_gather_block<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, st>>>(
            ts, tp, tn, nu, dia, dib, a.na, a.nb, a.stat, a.pval, a.n);
        NAPG_CU(ctx, cudaGetLastError());
        if (a.es1 || a.es2) {
            count_launch();
            k_gather_block<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, st>>>(
                te1, te2, nullptr, nu, dia, dib, a.na, a.nb, a.es1, a.es2, nullptr);
            NAPG_CU(ctx, cudaGetLastError());
        }
        NAPG_CU(ctx, cudaStreamSynchronize(st));   // host vectors ia/ib and uniq go out of scope
        return NAPG_OK;
    }

    // context bits
    uint32_t *ctxw = WS(kCtxBits, uint32_t, W);
    const uint8_t *mask_dev = nullptr;
    if (a.mask) {
        if (a.mask_on_device) {
            mask_dev = a.mask;
        } else {
            uint8_t *m = WS(kMask, uint8_t, S);
            if (st_) return st_;
            NAPG_CU(ctx, cudaMemcpyAsync(m, a.mask, S, cudaMemcpyHostToDevice, st));
            mask_dev = m;
        }
    }
    if (st_) return st_;
    Stage prep_stage(ctx->trace, st, "prep");
    launch_ctx_bits(mask_dev, S, W, ctxw, st);

    // variable lists on the device: [va | vb | crow_a | crow_b | catrow | nlev | levoff]
    std::vector<int32_t> va, vb, catrow, nlev, levoff;
    int32_t R = 0, maxlev = 0;
    std::vector<int32_t> all_ints;
    std::vector<size_t> off;
    var_lists(c, a, symmetric, va, vb, catrow, nlev, levoff, R, maxlev, all_ints, off);
    enum { i_va, i_vb, i_ca, i_cb, i_cat, i_nl, i_lo };
    const int32_t *dints = a.dints;
    const size_t *doff = a.dints ? a.dints_off : off.data();
    if (!dints) {
        int32_t *d = WS(kVarsDev, int32_t, all_ints.size() + 1);
        if (st_) return st_;
        NAPG_CU(ctx, cudaMemcpyAsync(d, all_ints.data(), sizeof(int32_t) * all_ints.size(), cudaMemcpyHostToDevice, st));
        dints = d;
    }
    const int32_t *d_va = dints + doff[i_va], *d_vb = dints + doff[i_vb];
    const int32_t *d_ca = dints + doff[i_ca], *d_cb = dints + doff[i_cb];
    const int32_t *d_cat = dints + doff[i_cat], *d_nl = dints + doff[i_nl], *d_lo = dints + doff[i_lo];

    // effective observed bits (observed AND in context)
    uint32_t *obsA = WS(kObsA, uint32_t, (int64_t)na * W);
    uint32_t *obsB = symmetric ? obsA : WS(kObsB, uint32_t, (int64_t)nb * W);
    if (st_) return st_;
    launch_gather_obs(c.obs, d_va, na, ctxw, W, obsA, st);
    if (!symmetric) launch_gather_obs(c.obs, d_vb, nb, ctxw, W, obsB, st);

    int32_t *counter = WS(kCounter, int32_t, 4);
    if (st_) return st_;
    NAPG_CU(ctx, cudaMemsetAsync(counter, 0, sizeof(int32_t) * 4, st));

    // level bitmasks and in-context level counts of the categorical variables
    uint32_t *levbits = nullptr;
    int32_t *levcnt = nullptr;
    if (R > 0) {
        levbits = WS(kLevBits, uint32_t, (int64_t)R * W);
        levcnt = WS(kLevCnt, int32_t, R);
        if (st_) return st_;
        NAPG_CU(ctx, cudaMemsetAsync(levcnt, 0, sizeof(int32_t) * R, st));
        launch_level_bits(c.lab, S, W, d_cat, d_lo, d_nl, na, obsA, levbits, levcnt, st);
    }
    prep_stage.end();

    RescueArgs rsc{c.X, c.dtype, S, W, ctxw, c.obs, c.lab, d_cat, d_va, symmetric ? nullptr : d_vb, na, nb, t,
                   a.opt.welch, d_nl, levcnt, d_lo, t == NAPG_TTEST ? a.es1 : nullptr,
                   t == NAPG_TTEST ? a.es2 : nullptr};
    // Mann-Whitney's per-level counts and tie terms, for its effect size
    const int32_t *eff_rcnt = nullptr;
    const int64_t *eff_tie = nullptr;

    if (t == NAPG_PEARSON) {
        const int64_t nn2 = (int64_t)na * na;
        double *Sxy = WS(kMomA, double, nn2), *Sx = WS(kMomB, double, nn2), *Sxx = WS(kMomC, double, nn2);
        int32_t *nn = WS(kIntA, int32_t, nn2);
        int32_t *flags = WS(kFlagList, int32_t, nn2 / 2 + na + 1);
        double *shift = WS(kShiftA, double, na);
        double *vsq = mixed ? WS(kVsq, double, na) : nullptr;
        if (st_) return st_;
        if (mixed) {
            NAPG_ST(mixed_pearson(ctx, c, ws, st, d_va, na, obsA, Sxy, Sx, Sxx, nn, shift, vsq, (a.mask || a.no_plane_cache) ? nullptr : &va, a.own));
        } else {
            double *xs = WS(kXsA, double, (int64_t)na * S_pad);
            if (st_) return st_;
            { Stage s_(ctx->trace, st, "shift_fp64"); launch_shift_values(c.X, c.dtype, S, S_pad, d_va, na, obsA, W, shift, xs, st); }
            { Stage s_(ctx->trace, st, "pearson_moments_fp64"); launch_pearson_fp64(xs, S_pad, obsA, W, na, Sxy, Sx, Sxx, nn, st, a.own); }
        }
        PJobBufs pj;
        NAPG_ST(pjobs_setup(ctx, ws, st, (int64_t)na * (na + 1) / 2, a.pval != nullptr, pj));
        PearsonFin f{Sxy, Sx, Sxx, nn, shift, na, mixed ? kMixedRelTol : kPlainRelTol, vsq, pj.q, d_va, a.own};
        { Stage s_(ctx->trace, st, "finalize_pearson"); launch_finalize_pearson(f, a.stat, a.pval, a.n, flags, counter, st); }
        // the rescued pairs queue their p-values with the others, before the evaluation
        rsc.q = pj.q;
        { Stage s_(ctx->trace, st, "rescue"); launch_rescue(rsc, flags, counter, (int32_t)(nn2 / 2 + na + 1), a.stat, a.pval, a.n, 1, 0, st); }
        pjobs_run(ctx, pj, a.pval, st);
    } else if (t == NAPG_ANOVA || t == NAPG_TTEST) {
        const int64_t rb = (int64_t)R * nb;
        int32_t *gn = WS(kIntA, int32_t, rb);
        double *g1 = WS(kMomA, double, rb), *g2 = WS(kMomB, double, rb);
        int32_t *flags = WS(kFlagList, int32_t, (int64_t)na * nb + 1);
        double *shift = WS(kShiftB, double, nb);
        double *vsq = mixed ? WS(kVsq, double, nb) : nullptr;
        if (st_) return st_;
        // mixed-form ANOVA: the centred squares summed per (a, j) over all levels
        double *g2tot = (mixed && t == NAPG_ANOVA) ? WS(kMomC, double, (int64_t)na * nb) : nullptr;
        if (st_) return st_;
        if (mixed) {
            NAPG_ST(mixed_groupsum(ctx, c, ws, st, levbits, R, d_vb, nb, obsB, gn, g1, g2, shift, vsq,
                                   (a.mask || a.no_plane_cache) ? nullptr : &vb, obsA, na, g2tot));
        } else {
            double *xs = WS(kXsB, double, (int64_t)nb * S_pad);
            if (st_) return st_;
            { Stage s_(ctx->trace, st, "shift_fp64"); launch_shift_values(c.X, c.dtype, S, S_pad, d_vb, nb, obsB, W, shift, xs, st); }
            { Stage s_(ctx->trace, st, "groupsum_fp64"); launch_groupsum_fp64(c.lab, S, d_cat, na, d_lo, d_nl, xs, S_pad, obsB, W, nb, gn, g1, g2, maxlev, st); }
        }
        PJobBufs pj;
        NAPG_ST(pjobs_setup(ctx, ws, st, (int64_t)na * nb, a.pval != nullptr, pj));
        GroupFin f{gn, g1, g2, R, d_lo, d_nl, levcnt, na, nb, t, a.opt.welch, mixed ? kMixedRelTol : kPlainRelTol,
                   vsq, pj.q, g2tot, t == NAPG_TTEST ? a.es1 : nullptr, t == NAPG_TTEST ? a.es2 : nullptr};
        { Stage s_(ctx->trace, st, "finalize_groups"); launch_finalize_groups(f, a.stat, a.pval, a.n, flags, counter, st); }
        rsc.q = pj.q;
        { Stage s_(ctx->trace, st, "rescue"); launch_rescue(rsc, flags, counter, (int32_t)((int64_t)na * nb + 1), a.stat, a.pval, a.n, 0, maxlev, st); }
        pjobs_run(ctx, pj, a.pval, st);
    } else if (t == NAPG_CHI2) {
        int32_t *T = WS(kIntA, int32_t, (int64_t)R * R);
        if (st_) return st_;
        // a split call: the level rows of the part's variables
        uint8_t *own_lev = nullptr;
        if (a.own) {
            own_lev = WS(kTmpE, uint8_t, R);
            if (st_) return st_;
            launch_level_ownership(a.own, d_lo, d_nl, na, own_lev, st);
        }
        if (mixed) NAPG_ST(mixed_contingency(ctx, c, ws, st, levbits, R, T, own_lev));
        else { Stage s_(ctx->trace, st, "contingency_popc"); launch_contingency(levbits, W, R, T, own_lev, st); }
        PJobBufs pj;
        NAPG_ST(pjobs_setup(ctx, ws, st, (int64_t)na * (na + 1) / 2, a.pval != nullptr, pj));
        Chi2Fin f{T, R, d_lo, d_nl, d_lo, d_nl, levcnt, na, na, 1, a.opt.yates_2x2, pj.q, maxlev, a.own};
        { Stage s_(ctx->trace, st, "finalize_chi2"); launch_finalize_chi2(f, a.stat, a.pval, a.n, st); }
        pjobs_run(ctx, pj, a.pval, st);
    } else if (t == NAPG_SPEARMAN) {
        NAPG_ST(ensure_presort(ctx, c, ws, st));
        int64_t *q = WS(kMomA, int64_t, (int64_t)na * nb * 4);
        if (st_) return st_;
        RankData rd{c.perm, c.pos, c.nobs, c.tie, c.gsw, c.gew, S, W};
        {
            Stage s_(ctx->trace, st, "spearman_rank");
            const int t0 = rank_threads_default(W, false), cand[2] = {t0, t0 == 256 ? 1024 : 256};
            auto run = [&](int c) -> napg_status {
                launch_spearman_pairs(rd, d_ca, d_cb, obsA, obsB, na, nb, symmetric ? 1 : 0, q, st, cand[c],
                                      symmetric ? a.own : nullptr);
                NAPG_CU(ctx, cudaGetLastError());
                return NAPG_OK;
            };
            NAPG_ST(tuned_launch(ctx, TuneKey{kTuneSpearman, na, nb, W}, 2, run, st));
        }
        PJobBufs pj;
        NAPG_ST(pjobs_setup(ctx, ws, st, (int64_t)na * nb, a.pval != nullptr, pj));
        SpearmanFin f{q, na, nb, symmetric ? 1 : 0, pj.q, symmetric ? a.own : nullptr};
        { Stage s_(ctx->trace, st, "finalize_spearman"); launch_finalize_spearman(f, a.stat, a.pval, a.n, st); }
        pjobs_run(ctx, pj, a.pval, st);
    } else {  // MWU / KRUSKAL
        NAPG_ST(ensure_presort(ctx, c, ws, st));
        const int64_t rb = (int64_t)R * nb;
        int64_t *rsum = WS(kMomA, int64_t, rb);
        int32_t *rcnt = WS(kIntA, int32_t, rb);
        int64_t *tie = WS(kMomB, int64_t, (int64_t)na * nb);
        int32_t *flags = WS(kFlagList, int32_t, (int64_t)na * nb + 1);
        if (st_) return st_;
        RankData rd{c.perm, c.pos, c.nobs, c.tie, c.gsw, c.gew, S, W};
        {
            Stage s_(ctx->trace, st, "rank_groups");
            const int t0 = rank_threads_default(W, true), cand[2] = {t0, t0 == 256 ? 1024 : 256};
            auto run = [&](int cc) -> napg_status {
                launch_rank_groups(rd, c.lab, d_cat, d_nl, d_lo, na, d_cb, obsA, obsB, nb, maxlev, rsum, rcnt, tie, st,
                                   cand[cc]);
                NAPG_CU(ctx, cudaGetLastError());
                return NAPG_OK;
            };
            NAPG_ST(tuned_launch(ctx, TuneKey{kTuneRankGroups, na, nb, W}, 2, run, st));
        }
        PJobBufs pj;
        NAPG_ST(pjobs_setup(ctx, ws, st, (int64_t)na * nb, a.pval != nullptr && t == NAPG_KRUSKAL, pj));
        RankGroupFin f{rsum, rcnt, tie, R, d_lo, d_nl, levcnt, na, nb, t, a.opt.mwu_mode, a.opt.mwu_continuity, pj.q};
        eff_rcnt = rcnt;
        eff_tie = tie;
        { Stage s_(ctx->trace, st, "finalize_rankgroups"); launch_finalize_rankgroups(f, a.stat, a.pval, a.n, flags, counter, st); }
        pjobs_run(ctx, pj, a.pval, st);
        if (t == NAPG_MWU && a.pval) {
            const size_t sb = mwu_exact_scratch_bytes(S, a.opt.mwu_mode == 1);
            void *scratch = ws_get(ctx, ws, Workspace::kTmpG, sb, &st_);
            if (st_) return st_;
            if (!a.stat) return fail(ctx, NAPG_E_ARG, "exact Mann-Whitney p needs the stat buffer");
            Stage s_(ctx->trace, st, "mwu_exact");
            launch_mwu_exact(a.stat, rcnt, d_lo, R, nb, flags, counter, (int32_t)((int64_t)na * nb + 1), a.pval,
                             scratch, sb, ctx->dev_err, st);
        }
    }
    if (a.es1 || a.es2) {
        Stage s_(ctx->trace, st, "effect_sizes");
        EffectArgs e{t, na, nb, symmetric ? 1 : 0, a.stat, a.n, levcnt, d_lo, d_nl, eff_rcnt, eff_tie, a.es1, a.es2};
        launch_effects(e, st);
    }
    NAPG_CU(ctx, cudaGetLastError());
    return NAPG_OK;
}

napg_status device_error_status(napg_ctx *ctx, uint32_t bits) {
    if (bits & kErrTimeout) return fail(ctx, NAPG_E_TIMEOUT, "a device wait timed out");
    if (bits & kErrExactLimit)
        return fail(ctx, NAPG_E_UNSUPPORTED,
                    "forced exact Mann-Whitney p beyond the exact range (min(n0, n1) > 64, C(n, n0) >= 2^126, or "
                    "min(U0, U1) above max(3.5 x samples, 65,534)): those p-values are NaN");
    return NAPG_OK;
}

// Outputs: device pointers are written in place; host ones through workspace
// buffers copied back before returning.
napg_status wait_pending_copies(napg_ctx *ctx) {
    for (int k = 0; k < 2; ++k)
        if (ctx->copy_used[k]) NAPG_CU(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_copy[k], 0));
    return NAPG_OK;
}

// Host outputs are staged in device buffers and copied back. Synchronous by
// default; with opt.async_host_outputs (the context's own stream and workspace
// only) the copies go on copy_stream after the run and the call returns: the
// staging set alternates between calls, and a call first waits (on the device)
// for the last copy out of the set it is about to overwrite, so one call's
// copies overlap the next call's kernels.
napg_status run_with_outputs(napg_ctx *ctx, Workspace &ws, cudaStream_t st, RunArgs a, bool symmetric_shape) {
    const int64_t cnt = (int64_t)a.na * (symmetric_shape ? a.na : a.nb);
    const bool async = a.opt.async_host_outputs && &ws == &ctx->ws && st == ctx->stream;
    const int set = async ? ctx->stage_set : 0;
    const int sl_stat = set ? Workspace::kOutStatB : Workspace::kOutStat, sl_p = set ? Workspace::kOutPB : Workspace::kOutP,
              sl_n = set ? Workspace::kOutNB : Workspace::kOutN, sl_e1 = set ? Workspace::kOutE1B : Workspace::kOutE1,
              sl_e2 = set ? Workspace::kOutE2B : Workspace::kOutE2;
    if (&ws == &ctx->ws) {
        // staging set `set` may still be read by an earlier asynchronous copy
        if (async) {
            if (ctx->copy_used[set]) NAPG_CU(ctx, cudaStreamWaitEvent(st, ctx->ev_copy[set], 0));
        } else {
            NAPG_ST(wait_pending_copies(ctx));
        }
    }
    double *hs = a.stat, *hp = a.pval;
    int32_t *hn = a.n;
    const bool ds = !hs || is_device_ptr(hs), dp = !hp || is_device_ptr(hp), dn = !hn || is_device_ptr(hn);
    double *he1 = a.es1, *he2 = a.es2;
    const bool de1 = !he1 || is_device_ptr(he1), de2 = !he2 || is_device_ptr(he2);
    napg_status st_ = NAPG_OK;
    if (!ds) a.stat = (double *)ws_get(ctx, ws, sl_stat, sizeof(double) * cnt, &st_);
    if (!dp) a.pval = (double *)ws_get(ctx, ws, sl_p, sizeof(double) * cnt, &st_);
    if (!dn) a.n = (int32_t *)ws_get(ctx, ws, sl_n, sizeof(int32_t) * cnt, &st_);
    if (!de1) a.es1 = (double *)ws_get(ctx, ws, sl_e1, sizeof(double) * cnt, &st_);
    if (!de2) a.es2 = (double *)ws_get(ctx, ws, sl_e2, sizeof(double) * cnt, &st_);
    if (st_) return st_;
    // the effect sizes are formed from the statistic and n
    if (a.es1 || a.es2) {
        if (!a.stat) { a.stat = (double *)ws_get(ctx, ws, sl_stat, sizeof(double) * cnt, &st_); hs = nullptr; }
        if (!a.n) { a.n = (int32_t *)ws_get(ctx, ws, sl_n, sizeof(int32_t) * cnt, &st_); hn = nullptr; }
        if (st_) return st_;
    }
    // exact Mann-Whitney p reads the statistic back: give it a buffer if none
    if (a.test == NAPG_MWU && a.pval && !a.stat) {
        a.stat = (double *)ws_get(ctx, ws, sl_stat, sizeof(double) * cnt, &st_);
        if (st_) return st_;
        hs = nullptr;
    }
    // an asynchronous call leaves the error word to napg_sync (earlier queued
    // calls may have set it)
    if (!async) NAPG_CU(ctx, cudaMemsetAsync(ctx->dev_err, 0, sizeof(uint32_t), st));
    NAPG_ST(run_on_stream(ctx, ws, st, a));
    const bool host_out = !ds || !dp || !dn || !de1 || !de2;
    if (async && host_out) {
        if (!ctx->copy_stream) {
            NAPG_CU(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
            for (int k = 0; k < 2; ++k) {
                NAPG_CU(ctx, cudaEventCreateWithFlags(&ctx->ev_run[k], cudaEventDisableTiming));
                NAPG_CU(ctx, cudaEventCreateWithFlags(&ctx->ev_copy[k], cudaEventDisableTiming));
            }
        }
        cudaStream_t cs = ctx->copy_stream;
        NAPG_CU(ctx, cudaEventRecord(ctx->ev_run[set], st));
        NAPG_CU(ctx, cudaStreamWaitEvent(cs, ctx->ev_run[set], 0));
        if (!ds) NAPG_CU(ctx, cudaMemcpyAsync(hs, a.stat, sizeof(double) * cnt, cudaMemcpyDeviceToHost, cs));
        if (!dp) NAPG_CU(ctx, cudaMemcpyAsync(hp, a.pval, sizeof(double) * cnt, cudaMemcpyDeviceToHost, cs));
        if (!dn) NAPG_CU(ctx, cudaMemcpyAsync(hn, a.n, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, cs));
        if (!de1) NAPG_CU(ctx, cudaMemcpyAsync(he1, a.es1, sizeof(double) * cnt, cudaMemcpyDeviceToHost, cs));
        if (!de2) NAPG_CU(ctx, cudaMemcpyAsync(he2, a.es2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, cs));
        NAPG_CU(ctx, cudaEventRecord(ctx->ev_copy[set], cs));
        ctx->copy_used[set] = true;
        ctx->stage_set = 1 - set;
        return NAPG_OK;
    }
    if (!ds) NAPG_CU(ctx, cudaMemcpyAsync(hs, a.stat, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    if (!dp) NAPG_CU(ctx, cudaMemcpyAsync(hp, a.pval, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    if (!dn) NAPG_CU(ctx, cudaMemcpyAsync(hn, a.n, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, st));
    if (!de1) NAPG_CU(ctx, cudaMemcpyAsync(he1, a.es1, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    if (!de2) NAPG_CU(ctx, cudaMemcpyAsync(he2, a.es2, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
    if (host_out) {
        NAPG_CU(ctx, cudaMemcpyAsync(ctx->host_err, ctx->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        NAPG_CU(ctx, cudaStreamSynchronize(st));
        if (*ctx->host_err) return device_error_status(ctx, *ctx->host_err);
    }
    return NAPG_OK;
}

}  // namespace napg

using namespace napg;

// ================================================================ C ABI ==

extern "C" {

void napg_default_options(napg_options *o) {
    if (!o) return;
    o->precision = NAPG_FP64_PLAIN;
    o->welch = 1;
    o->yates_2x2 = 0;
    o->mwu_mode = 0;
    o->mwu_continuity = 1;
    o->debug_checks = 0;
    o->async_host_outputs = 0;
}

const char *napg_version(void) { return "napg 0.1 (sm_103a)"; }

napg_status napg_create(napg_ctx **out, int device, void *cuda_stream) {
    if (!out) return NAPG_E_ARG;
    *out = nullptr;
    napg_ctx *ctx = new (std::nothrow) napg_ctx();
    if (!ctx) return NAPG_E_OOM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete ctx;
        return NAPG_E_CUDA;
    }
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            return NAPG_E_CUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaMalloc(&ctx->dev_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->host_err, sizeof(uint32_t)) != cudaSuccess) {
        if (ctx->dev_err) cudaFree(ctx->dev_err);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return NAPG_E_OOM;
    }
    *out = ctx;
    return NAPG_OK;
}

void napg_destroy(napg_ctx *ctx) {
    if (!ctx) return;
    if (ctx->serve) napg_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
        for (int k = 0; k < 2; ++k) {
            cudaEventDestroy(ctx->ev_run[k]);
            cudaEventDestroy(ctx->ev_copy[k]);
        }
    }
    free_batch(ctx);
    free_cohort(ctx->coh);
    free_ws(ctx->ws);
    if (ctx->dev_err) cudaFree(ctx->dev_err);
    if (ctx->host_err) cudaFreeHost(ctx->host_err);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *napg_last_error(const napg_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

napg_status napg_sync(napg_ctx *ctx) {
    if (!ctx) return NAPG_E_ARG;
    NAPG_CU(ctx, cudaMemcpyAsync(ctx->host_err, ctx->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    NAPG_CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->copy_stream) NAPG_CU(ctx, cudaStreamSynchronize(ctx->copy_stream));
    if (*ctx->host_err & (kErrTimeout | kErrExactLimit)) {
        const uint32_t bits = *ctx->host_err;
        NAPG_CU(ctx, cudaMemset(ctx->dev_err, 0, sizeof(uint32_t)));
        return device_error_status(ctx, bits);
    }
    return NAPG_OK;
}

napg_status napg_release_cache(napg_ctx *ctx) {
    if (!ctx) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serve) return fail(ctx, NAPG_E_BUSY, "the serving loop reads the presort");
    ctx->ws.plane_key.valid = false;
    ctx->coh.sorted = false;
    return NAPG_OK;
}

napg_status napg_load_cohort(napg_ctx *ctx, const void *X, int32_t dtype, int64_t n_vars, int64_t n_samples,
                             int32_t samples_major, double missing, const uint8_t *var_type, const int32_t *n_levels) {
    if (!ctx) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->serve) return fail(ctx, NAPG_E_BUSY, "stop the serving loop before loading a cohort");
    ctx->err.clear();
    if (!X || !var_type || !n_levels || n_vars <= 0 || n_samples <= 0 || (dtype != NAPG_F32 && dtype != NAPG_F64))
        return fail(ctx, NAPG_E_ARG, "bad cohort arguments");
    if (n_samples >= kMaxSamples) return fail(ctx, NAPG_E_UNSUPPORTED, "n_samples must be below 2^24");
    if (n_vars > INT32_MAX / 2) return fail(ctx, NAPG_E_UNSUPPORTED, "too many variables");
    for (int64_t v = 0; v < n_vars; ++v) {
        if (var_type[v] > 1) return fail(ctx, NAPG_E_ARG, "var_type must be 0 or 1");
        if (var_type[v] == 1 && (n_levels[v] < 1 || n_levels[v] > kMaxLevels))
            return fail(ctx, n_levels[v] > kMaxLevels ? NAPG_E_UNSUPPORTED : NAPG_E_ARG, "bad level count");
    }
    NAPG_CU(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    NAPG_CU(ctx, cudaStreamSynchronize(st));
    // the previous cohort's value, bit and label buffers are kept for this one
    // when large enough (no free and allocation per load); nothing uses them now
    struct Kept { void *p = nullptr; size_t cap = 0; } kx, kobs, klab;
    if (ctx->coh.owns) {
        kx = {ctx->coh.X, ctx->coh.x_bytes};
        kobs = {ctx->coh.obs, ctx->coh.obs_bytes};
        klab = {ctx->coh.lab, ctx->coh.lab_bytes};
        ctx->coh.X = nullptr; ctx->coh.obs = nullptr; ctx->coh.lab = nullptr;
    }
    free_cohort(ctx->coh);
    auto take = [](Kept &k, size_t need, void **out, size_t *cap) -> cudaError_t {
        if (k.p && k.cap >= need) {
            *out = k.p;
            *cap = k.cap;
            k.p = nullptr;
            return cudaSuccess;
        }
        *cap = need;
        return cudaMalloc(out, need);
    };
    auto drop_kept = [&]() {
        for (Kept *k : {&kx, &kobs, &klab})
            if (k->p) { cudaFree(k->p); k->p = nullptr; }
    };
    Cohort &c = ctx->coh;
    c.F = n_vars;
    c.S = n_samples;
    c.W = (n_samples + 31) / 32;
    c.dtype = dtype;
    c.missing = missing;
    c.vtype.assign(var_type, var_type + n_vars);
    c.nlev.assign(n_vars, 0);
    c.cat_index.assign(n_vars, -1);
    c.cont_index.assign(n_vars, -1);
    for (int64_t v = 0; v < n_vars; ++v) {
        if (var_type[v] == 1) {
            c.nlev[v] = n_levels[v];
            c.cat_index[v] = (int32_t)c.n_cat++;
        } else {
            c.cont_index[v] = (int32_t)c.n_cont++;
        }
    }
    const size_t esz = dtype == NAPG_F32 ? 4 : 8;
    const size_t xbytes = esz * (size_t)n_vars * (size_t)n_samples;
    {
        const size_t obs_need = sizeof(uint32_t) * (size_t)n_vars * c.W;
        const size_t lab_need = std::max<size_t>(1, (size_t)c.n_cat * (size_t)n_samples);
        cudaError_t e1 = take(kx, xbytes, &c.X, &c.x_bytes);
        cudaError_t e2 = e1 == cudaSuccess ? take(kobs, obs_need, (void **)&c.obs, &c.obs_bytes) : e1;
        cudaError_t e3 = e2 == cudaSuccess ? take(klab, lab_need, (void **)&c.lab, &c.lab_bytes) : e2;
        drop_kept();
        if (e3 != cudaSuccess) {
            free_cohort(ctx->coh);
            return cuda_fail(ctx, e3, "cohort allocation");
        }
    }
    const bool on_dev = is_device_ptr(X);
    // page-locked host memory mapped for the device: the validation kernel reads
    // it over the host link and writes the device copy as it checks each value
    // (one pass instead of a copy and a pass)
    const void *mapped = nullptr;
    if (!on_dev && !samples_major) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, X) == cudaSuccess) {
            if (at.type == cudaMemoryTypeHost && at.devicePointer) mapped = at.devicePointer;
        } else {
            (void)cudaGetLastError();
        }
    }
    if (!samples_major) {
        if (!mapped)
            NAPG_CU(ctx, cudaMemcpyAsync(c.X, X, xbytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
        void *tmp = nullptr;
        NAPG_CU(ctx, cudaMalloc(&tmp, xbytes));
        NAPG_CU(ctx, cudaMemcpyAsync(tmp, X, xbytes, on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        launch_transpose(tmp, c.X, dtype, n_samples, n_vars, st);
        NAPG_CU(ctx, cudaGetLastError());
        NAPG_CU(ctx, cudaStreamSynchronize(st));
        cudaFree(tmp);
    }
    // per-variable tables for the validation kernel
    std::vector<int32_t> tab(2 * n_vars);
    for (int64_t v = 0; v < n_vars; ++v) { tab[v] = c.nlev[v]; tab[n_vars + v] = c.cat_index[v]; }
    int32_t *dtab = nullptr;
    uint8_t *dvt = nullptr;
    NAPG_CU(ctx, cudaMalloc(&dtab, sizeof(int32_t) * tab.size()));
    NAPG_CU(ctx, cudaMalloc(&dvt, (size_t)n_vars));
    NAPG_CU(ctx, cudaMemcpyAsync(dtab, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice, st));
    NAPG_CU(ctx, cudaMemcpyAsync(dvt, var_type, (size_t)n_vars, cudaMemcpyHostToDevice, st));
    NAPG_CU(ctx, cudaMemsetAsync(ctx->dev_err, 0, sizeof(uint32_t), st));
    launch_validate_obs(mapped ? mapped : c.X, dtype, n_vars, n_samples, c.W, missing, dvt, dtab, dtab + n_vars,
                        c.obs, c.lab, ctx->dev_err, st, mapped ? c.X : nullptr);
    NAPG_CU(ctx, cudaGetLastError());
    NAPG_CU(ctx, cudaMemcpyAsync(ctx->host_err, ctx->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    NAPG_CU(ctx, cudaStreamSynchronize(st));
    cudaFree(dtab);
    cudaFree(dvt);
    const uint32_t e = *ctx->host_err;
    if (e & kErrNonfinite) {
        free_cohort(ctx->coh);
        return fail(ctx, NAPG_E_NONFINITE, "a non-missing value is not finite");
    }
    if (e & kErrLabel) {
        free_cohort(ctx->coh);
        return fail(ctx, NAPG_E_LABEL, "a categorical value is not an integer in [0, c)");
    }
    if (c.n_cont > 0) {
        std::vector<int32_t> cv;
        for (int64_t v = 0; v < c.F; ++v)
            if (c.vtype[v] == 0) cv.push_back((int32_t)v);
        NAPG_CU(ctx, cudaMalloc(&c.cont_vars_dev, sizeof(int32_t) * cv.size()));
        NAPG_CU(ctx, cudaMemcpy(c.cont_vars_dev, cv.data(), sizeof(int32_t) * cv.size(), cudaMemcpyHostToDevice));
    }
    c.gen = next_cohort_gen();
    c.loaded = true;
    return NAPG_OK;
}

napg_status napg_run(napg_ctx *ctx, int32_t test, const napg_options *opt, const uint8_t *sample_mask,
                     const int32_t *vars_a, int32_t n_a, const int32_t *vars_b, int32_t n_b, double *stat,
                     double *pval, int32_t *n) {
    return napg_run_ex(ctx, test, opt, sample_mask, vars_a, n_a, vars_b, n_b, stat, pval, n, nullptr, nullptr);
}

napg_status napg_run_ex(napg_ctx *ctx, int32_t test, const napg_options *opt, const uint8_t *sample_mask,
                        const int32_t *vars_a, int32_t n_a, const int32_t *vars_b, int32_t n_b, double *stat,
                        double *pval, int32_t *n, double *effect, double *effect2) {
    if (!ctx) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    NAPG_CU(ctx, cudaSetDevice(ctx->device));
    RunArgs a{};
    a.test = test;
    if (opt) a.opt = *opt;
    else napg_default_options(&a.opt);
    a.mask = sample_mask;
    a.mask_on_device = is_device_ptr(sample_mask);
    a.va = vars_a;
    a.na = n_a;
    a.vb = vars_b;
    a.nb = vars_b ? n_b : n_a;
    a.stat = stat;
    a.pval = pval;
    a.n = n;
    a.es1 = effect;
    a.es2 = effect2;
    return run_with_outputs(ctx, ctx->ws, ctx->stream, a, vars_b == nullptr);
}

// One part of a call split over n_parts (Sec. 3.5.1: the pairs are independent).
// Output rows go in blocks of kPartRows dealt back and forth to the parts.
// Symmetric calls compute the pairs (i, j), i <= j, of the owned rows i and
// write (i, j) and (j, i); A x B calls compute the owned rows of A. Entries of
// other parts are left as they were (host outputs are staged on the device
// from the caller's arrays, so the copy back keeps them).
napg_status napg_run_part(napg_ctx *ctx, int32_t test, const napg_options *opt, const uint8_t *sample_mask,
                          const int32_t *vars_a, int32_t n_a, const int32_t *vars_b, int32_t n_b, int32_t part,
                          int32_t n_parts, double *stat, double *pval, int32_t *n) {
    if (!ctx) return NAPG_E_ARG;
    if (n_parts < 1 || part < 0 || part >= n_parts) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        return fail(ctx, NAPG_E_ARG, "part must be in [0, n_parts) with n_parts >= 1");
    }
    if (n_parts == 1) return napg_run(ctx, test, opt, sample_mask, vars_a, n_a, vars_b, n_b, stat, pval, n);
    if (n_a < 0 || (vars_b && n_b < 0) || (n_a > 0 && !vars_a)) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        return fail(ctx, NAPG_E_ARG, "bad variable lists");
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    NAPG_CU(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    NAPG_ST(wait_pending_copies(ctx));
    RunArgs a{};
    a.test = test;
    if (opt) a.opt = *opt;
    else napg_default_options(&a.opt);
    a.opt.async_host_outputs = 0;
    a.mask = sample_mask;
    a.mask_on_device = is_device_ptr(sample_mask);
    const bool symmetric = vars_b == nullptr;
    const int32_t nb = symmetric ? n_a : n_b;
    std::vector<int32_t> rows;
    for (int32_t i = 0; i < n_a; ++i)
        if (part_of_row(i, n_parts) == part) rows.push_back(i);
    napg_status st_ = NAPG_OK;
    double *outs_d[2] = {stat, pval};
    const int sl_d[2] = {Workspace::kPartS, Workspace::kPartP};
    if (symmetric) {
        const int64_t cnt = (int64_t)n_a * n_a;
        std::vector<uint8_t> own(std::max<int32_t>(n_a, 1), 0);
        for (int32_t i : rows) own[i] = 1;
        uint8_t *own_d = (uint8_t *)ws_get(ctx, ctx->ws, Workspace::kPartOwn, own.size(), &st_);
        if (st_) return st_;
        NAPG_CU(ctx, cudaMemcpyAsync(own_d, own.data(), own.size(), cudaMemcpyHostToDevice, st));
        // host outputs: staged on the device from the caller's arrays
        double *dd[2] = {stat, pval};
        int32_t *dn = n;
        for (int k = 0; k < 2; ++k)
            if (outs_d[k] && !is_device_ptr(outs_d[k])) {
                dd[k] = (double *)ws_get(ctx, ctx->ws, sl_d[k], sizeof(double) * cnt, &st_);
                if (st_) return st_;
                NAPG_CU(ctx, cudaMemcpyAsync(dd[k], outs_d[k], sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
            }
        if (n && !is_device_ptr(n)) {
            dn = (int32_t *)ws_get(ctx, ctx->ws, Workspace::kPartN, sizeof(int32_t) * cnt, &st_);
            if (st_) return st_;
            NAPG_CU(ctx, cudaMemcpyAsync(dn, n, sizeof(int32_t) * cnt, cudaMemcpyHostToDevice, st));
        }
        a.va = vars_a;
        a.na = n_a;
        a.nb = n_a;
        a.stat = dd[0];
        a.pval = dd[1];
        a.n = dn;
        a.own = own_d;
        NAPG_CU(ctx, cudaMemsetAsync(ctx->dev_err, 0, sizeof(uint32_t), st));
        if (!rows.empty()) NAPG_ST(run_with_outputs(ctx, ctx->ws, st, a, true));
        for (int k = 0; k < 2; ++k)
            if (dd[k] != outs_d[k])
                NAPG_CU(ctx, cudaMemcpyAsync(outs_d[k], dd[k], sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
        if (dn != n) NAPG_CU(ctx, cudaMemcpyAsync(n, dn, sizeof(int32_t) * cnt, cudaMemcpyDeviceToHost, st));
    } else {
        // A x B: the owned rows of A into device buffers, then row blocks copied to the outputs
        if (rows.empty()) return NAPG_OK;
        const int32_t np = (int32_t)rows.size();
        std::vector<int32_t> va(np);
        for (int32_t r = 0; r < np; ++r) va[r] = vars_a[rows[r]];
        const int64_t cnt = (int64_t)np * nb;
        double *td[2] = {nullptr, nullptr};
        for (int k = 0; k < 2; ++k)
            if (outs_d[k]) {
                td[k] = (double *)ws_get(ctx, ctx->ws, sl_d[k], sizeof(double) * cnt, &st_);
                if (st_) return st_;
            }
        int32_t *tn = nullptr;
        if (n) {
            tn = (int32_t *)ws_get(ctx, ctx->ws, Workspace::kPartN, sizeof(int32_t) * cnt, &st_);
            if (st_) return st_;
        }
        a.va = va.data();
        a.na = np;
        a.vb = vars_b;
        a.nb = n_b;
        a.stat = td[0];
        a.pval = td[1];
        a.n = tn;
        NAPG_CU(ctx, cudaMemsetAsync(ctx->dev_err, 0, sizeof(uint32_t), st));
        NAPG_ST(run_with_outputs(ctx, ctx->ws, st, a, false));
        // runs of consecutive owned rows are one copy each
        for (int32_t r0 = 0; r0 < np;) {
            int32_t r1 = r0 + 1;
            while (r1 < np && rows[r1] == rows[r1 - 1] + 1) ++r1;
            const size_t len = (size_t)(r1 - r0) * (size_t)nb;
            const int64_t src = (int64_t)r0 * nb, dst = (int64_t)rows[r0] * nb;
            for (int k = 0; k < 2; ++k)
                if (outs_d[k])
                    NAPG_CU(ctx, cudaMemcpyAsync(outs_d[k] + dst, td[k] + src, sizeof(double) * len, cudaMemcpyDefault, st));
            if (n) NAPG_CU(ctx, cudaMemcpyAsync(n + dst, tn + src, sizeof(int32_t) * len, cudaMemcpyDefault, st));
            r0 = r1;
        }
    }
    // synchronous: the row lists above live on the host
    NAPG_CU(ctx, cudaMemcpyAsync(ctx->host_err, ctx->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    NAPG_CU(ctx, cudaStreamSynchronize(st));
    if (*ctx->host_err) return device_error_status(ctx, *ctx->host_err);
    return NAPG_OK;
}

napg_status napg_adjust(napg_ctx *ctx, int32_t method, const double *p, int64_t rows, int64_t cols,
                        int32_t symmetric, double *out) {
    if (!ctx) return NAPG_E_ARG;
    if (!p || !out || rows < 0 || cols < 0) return fail(ctx, NAPG_E_ARG, "bad correction arguments");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    NAPG_CU(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t bytes = sizeof(double) * (size_t)rows * (size_t)cols;
    if (bytes == 0) return NAPG_OK;
    NAPG_ST(wait_pending_copies(ctx));
    napg_status st_ = NAPG_OK;
    const bool dp = is_device_ptr(p), dout = is_device_ptr(out);
    const double *pd = p;
    double *od = out;
    if (!dp) {
        double *b = (double *)ws_get(ctx, ctx->ws, Workspace::kOutP, bytes, &st_);
        if (st_) return st_;
        NAPG_CU(ctx, cudaMemcpyAsync(b, p, bytes, cudaMemcpyHostToDevice, st));
        pd = b;
    }
    if (!dout) {
        od = (double *)ws_get(ctx, ctx->ws, Workspace::kOutE1, bytes, &st_);
        if (st_) return st_;
    }
    NAPG_ST(adjust_pvalues(ctx, ctx->ws, st, method, pd, rows, cols, symmetric, od));
    if (!dout) NAPG_CU(ctx, cudaMemcpyAsync(out, od, bytes, cudaMemcpyDeviceToHost, st));
    NAPG_CU(ctx, cudaStreamSynchronize(st));
    return NAPG_OK;
}

napg_status napg_run_batch(napg_ctx *ctx, int32_t test, const napg_options *opt, int32_t n_ctx,
                           const uint8_t *const *sample_masks, const int32_t *vars_a, int32_t n_a,
                           const int32_t *vars_b, int32_t n_b, double *const *stat, double *const *pval,
                           int32_t *const *n) {
    if (!ctx || n_ctx < 0) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->err.clear();
    NAPG_CU(ctx, cudaSetDevice(ctx->device));
    RunArgs a{};
    a.test = test;
    if (opt) a.opt = *opt;
    else napg_default_options(&a.opt);
    a.opt.async_host_outputs = 0;               // the batch call returns with its outputs written
    a.va = vars_a;
    a.na = n_a;
    a.vb = vars_b;
    a.nb = vars_b ? n_b : n_a;
    NAPG_ST(wait_pending_copies(ctx));
    return run_batch(ctx, a, n_ctx, sample_masks, stat, pval, n);
}

napg_status napg_debug_pvalues(napg_ctx *ctx, int32_t kind, const double *s, const double *a, const double *b,
                               int64_t count, double *p) {
    if (!ctx || count < 0 || kind < 0 || kind > 8) return NAPG_E_ARG;
    if (count == 0) return NAPG_OK;
    if (!s || !p || (kind != 4 && kind < 7 && !a) || ((kind == 2 || kind == 5) && !b)) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    NAPG_ST(wait_pending_copies(ctx));
    ctx->err.clear();
    NAPG_CU(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;
    const size_t bytes = sizeof(double) * (size_t)count;
    double *d = nullptr;
    const size_t tab = sizeof(double) * sf::kBgratRows * sf::kBgratTerms;
    NAPG_CU(ctx, cudaMalloc(&d, 4 * bytes + tab));
    double *ds = d, *da = d + count, *db = d + 2 * count, *dp = d + 3 * count, *dt = d + 4 * count;
    launch_bgrat_table(dt, st);
    cudaError_t e = cudaMemcpyAsync(ds, s, bytes, cudaMemcpyDefault, st);
    if (e == cudaSuccess && a) e = cudaMemcpyAsync(da, a, bytes, cudaMemcpyDefault, st);
    if (e == cudaSuccess && b) e = cudaMemcpyAsync(db, b, bytes, cudaMemcpyDefault, st);
    if (e == cudaSuccess) {
        launch_debug_pvalues(kind, ds, a ? da : ds, b ? db : ds, count, dp, dt, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, dp, bytes, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "napg_debug_pvalues");
    return NAPG_OK;
}

napg_status napg_debug_integers(napg_ctx *ctx, int32_t test, const uint8_t *sample_mask, int32_t a, int32_t b,
                                int64_t *out, int64_t cap, int64_t *written) {
    if (!ctx || !out || !written) return NAPG_E_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    NAPG_ST(wait_pending_copies(ctx));
    ctx->err.clear();
    NAPG_CU(ctx, cudaSetDevice(ctx->device));
    Cohort &c = ctx->coh;
    if (!c.loaded) return fail(ctx, NAPG_E_ARG, "no cohort loaded");
    if (a < 0 || a >= c.F || b < 0 || b >= c.F) return fail(ctx, NAPG_E_ARG, "pair index out of range");
    Workspace &ws = ctx->ws;
    cudaStream_t st = ctx->stream;
    RunArgs r{};
    r.test = test;
    napg_default_options(&r.opt);
    r.opt.mwu_mode = 2;
    r.mask = sample_mask;
    r.mask_on_device = is_device_ptr(sample_mask);
    int32_t va = a, vb = b;
    r.va = &va;
    r.na = 1;
    r.vb = &vb;
    r.nb = 1;
    napg_status st_ = NAPG_OK;
    double *ds = (double *)ws_get(ctx, ws, Workspace::kOutStat, 16, &st_);
    double *dp = (double *)ws_get(ctx, ws, Workspace::kOutP, 16, &st_);
    int32_t *dn = (int32_t *)ws_get(ctx, ws, Workspace::kOutN, 16, &st_);
    if (st_) return st_;
    r.stat = ds;
    r.pval = dp;
    r.n = dn;
    if (test == NAPG_SPEARMAN && a == b) r.vb = nullptr;
    if (test != NAPG_CHI2) {
        NAPG_ST(run_on_stream(ctx, ws, st, r));
        NAPG_CU(ctx, cudaStreamSynchronize(st));
    }
    std::vector<int64_t> res;
    if (test == NAPG_CHI2) {
        // recompute the pair's table from the level bitmasks of a (and b)
        std::vector<int32_t> vars = {a};
        if (b != a) vars.push_back(b);
        RunArgs s = r;
        s.va = vars.data();
        s.na = (int32_t)vars.size();
        s.vb = nullptr;
        NAPG_ST(run_on_stream(ctx, ws, st, s));
        NAPG_CU(ctx, cudaStreamSynchronize(st));
        const int ca = c.nlev[a], cb = c.nlev[b];
        const int R = (b != a) ? ca + cb : ca;
        std::vector<int32_t> T((size_t)R * R);
        NAPG_CU(ctx, cudaMemcpy(T.data(), ws.ptr[Workspace::kIntA], sizeof(int32_t) * T.size(), cudaMemcpyDeviceToHost));
        const int ob = (b != a) ? ca : 0;
        for (int g = 0; g < ca; ++g)
            for (int h = 0; h < cb; ++h) res.push_back(T[(size_t)g * R + ob + h]);
    } else if (test == NAPG_SPEARMAN) {
        int64_t q[4];
        NAPG_CU(ctx, cudaMemcpy(q, ws.ptr[Workspace::kMomA], sizeof(q), cudaMemcpyDeviceToHost));
        res.assign(q, q + 4);
    } else if (test == NAPG_MWU || test == NAPG_KRUSKAL) {
        const int L = c.nlev[a];
        std::vector<int64_t> rs(L);
        std::vector<int32_t> rc(L);
        int64_t T = 0;
        NAPG_CU(ctx, cudaMemcpy(rs.data(), ws.ptr[Workspace::kMomA], sizeof(int64_t) * L, cudaMemcpyDeviceToHost));
        NAPG_CU(ctx, cudaMemcpy(rc.data(), ws.ptr[Workspace::kIntA], sizeof(int32_t) * L, cudaMemcpyDeviceToHost));
        NAPG_CU(ctx, cudaMemcpy(&T, ws.ptr[Workspace::kMomB], sizeof(int64_t), cudaMemcpyDeviceToHost));
        int64_t n = 0;
        for (int g = 0; g < L; ++g) n += rc[g];
        res.push_back(n);
        res.push_back(T);
        for (int g = 0; g < L; ++g) { res.push_back(rc[g]); res.push_back(rs[g]); }
    } else if (test == NAPG_ANOVA || test == NAPG_TTEST) {
        const int L = c.nlev[a];
        std::vector<int32_t> gn(L);
        NAPG_CU(ctx, cudaMemcpy(gn.data(), ws.ptr[Workspace::kIntA], sizeof(int32_t) * L, cudaMemcpyDeviceToHost));
        int64_t n = 0;
        for (int g = 0; g < L; ++g) n += gn[g];
        res.push_back(n);
        for (int g = 0; g < L; ++g) res.push_back(gn[g]);
    } else {
        int32_t nn = 0;
        NAPG_CU(ctx, cudaMemcpy(&nn, dn, sizeof(int32_t), cudaMemcpyDeviceToHost));
        res.push_back(nn);
    }
    if ((int64_t)res.size() > cap) return fail(ctx, NAPG_E_ARG, "cap too small");
    std::copy(res.begin(), res.end(), out);
    *written = (int64_t)res.size();
    return NAPG_OK;
}

}  // extern "C"
