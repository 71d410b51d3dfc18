// Many sample contexts in one call (Sec. 1: per-context association networks
// in interactive tools; Sec. 3.3: a sample context is a submatrix call).
//
// Each context k is compacted to its own N_k samples: a gather kernel writes the
// selected variables' values, observed bits and labels for the context's
// samples into a dense sub-cohort, and the ordinary pipeline runs on it with
// no mask. Tensor and rank work then scale with N_k instead of the cohort's S.
// The contexts are dealt to kBatchBranches branches (largest first, onto the
// least-loaded branch), each with its own sub-cohort, workspace and stream, so
// that the kernels of small contexts run side by side. The whole batch
// (compaction of every mask, then the branches forked from it, gather +
// pipeline per context, joined at the end) is captured once into a CUDA graph
// and replayed by a single graph launch; the
// executable graph is kept for the next call with the same shape (test,
// options, variable lists, context sizes, output buffers). Only the mask
// contents change between such calls: they are copied into a staging buffer
// the graph reads.
#include <algorithm>
#include <numeric>

#include "napg_internal.cuh"

namespace napg {

// ------------------------------------------------------------------ kernels --

// one block per context: its number of selected samples
__global__ void k_ctx_count(const uint8_t *__restrict__ masks, int64_t S, int32_t *counts) {
    const uint8_t *m = masks + (int64_t)blockIdx.x * S;
    int c = 0;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) c += m[s] != 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    __shared__ int red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        counts[blockIdx.x] = t;
    }
}

// one block (1024 threads) per context: idx[k][j] = the j-th selected sample
__global__ void __launch_bounds__(1024) k_ctx_compact(const uint8_t *__restrict__ masks, int64_t S,
                                                      int32_t *__restrict__ idx, int64_t idx_stride) {
    const uint8_t *m = masks + (int64_t)blockIdx.x * S;
    int32_t *out = idx + (int64_t)blockIdx.x * idx_stride;
    __shared__ int warp_tot[32];
    __shared__ int base_s;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t s0 = 0; s0 < S; s0 += blockDim.x) {
        const int64_t s = s0 + threadIdx.x;
        const bool sel = s < S && m[s] != 0;
        const unsigned b = __ballot_sync(0xffffffffu, sel);
        if (lane == 0) warp_tot[wid] = __popc(b);
        __syncthreads();
        int before = base_s;
        for (int w = 0; w < wid; ++w) before += warp_tot[w];
        if (sel) out[before + __popc(b & ((1u << lane) - 1u))] = (int32_t)s;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += warp_tot[w];
            base_s += t;
        }
        __syncthreads();
    }
}

// dense sub-cohort of context k: row r takes parent variable vars[r]; values,
// observed bits (32 compact samples per word) and labels of the selected samples
template <typename T>
__global__ void k_ctx_gather(const T *__restrict__ X, const uint32_t *__restrict__ obs,
                             const uint8_t *__restrict__ lab, int64_t S, int64_t W, const int32_t *__restrict__ vars,
                             const int32_t *__restrict__ cat_row, const int32_t *__restrict__ idx, int64_t Nk,
                             int64_t Wk, T *__restrict__ Xs, uint32_t *__restrict__ obss, uint8_t *__restrict__ labs) {
    const int r = blockIdx.y;
    const int v = vars[r];
    const int cr = cat_row[r];          // row among the sub-cohort's categoricals, or -1
    const int lane = threadIdx.x & 31;
    for (int64_t j0 = (int64_t)blockIdx.x * blockDim.x; j0 < Wk * 32; j0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = j0 + threadIdx.x;
        bool o = false;
        if (j < Nk) {
            const int64_t s = idx[j];
            Xs[(int64_t)r * Nk + j] = X[(int64_t)v * S + s];
            o = (obs[(int64_t)v * W + (s >> 5)] >> (s & 31)) & 1u;
            if (cr >= 0) labs[(int64_t)cr * Nk + j] = lab[(int64_t)cat_row[gridDim.y + r] * S + s];
        }
        const unsigned b = __ballot_sync(0xffffffffu, o);
        if (lane == 0 && (j >> 5) < Wk) obss[(int64_t)r * Wk + (j >> 5)] = b;
    }
}

// ------------------------------------------------------------- batch state --

// Contexts run on this many concurrent branches of the captured graph, each with
// its own dense sub-cohort, workspace and stream: a small context leaves most
// SMs idle, and the other branches' contexts fill them.
constexpr int kBatchBranches = 4;

struct BatchBranch {
    Cohort sub;                          // dense sub-cohort, arrays sized for the branch's largest context
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    size_t sub_x_cap = 0, sub_obs_cap = 0, sub_lab_cap = 0;
    std::vector<int32_t> ctxs;           // contexts of this branch, in launch order
};

struct BatchState {
    // shape of the captured graph
    bool valid = false;
    uint64_t parent_gen = 0;
    int32_t test = -1;
    napg_options opt{};
    std::vector<int32_t> va, vb;
    bool symmetric = true;
    std::vector<int64_t> nk;
    std::vector<void *> outs;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // buffers
    BatchBranch br[kBatchBranches];
    uint8_t *masks = nullptr;            // [n_ctx][S] staged masks
    size_t masks_cap = 0;
    int32_t *idx = nullptr;              // [n_ctx][idx_stride] selected sample ids
    size_t idx_cap = 0;
    int32_t *counts = nullptr;           // [n_ctx]
    size_t counts_cap = 0;
    int32_t *rows = nullptr;             // [3 F_sub]: parent ids, categorical row in the sub-cohort (or -1), in the parent
    int32_t *dints = nullptr;            // staged variable lists of the sub-cohort run
    std::vector<size_t> doff;
    int32_t *host_counts = nullptr;      // pinned
    void *stage = nullptr;               // device outputs of every context when the caller's are on the host
    size_t stage_cap = 0;
};

void free_batch(napg_ctx *ctx) {
    BatchState *b = ctx->batch;
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (BatchBranch &r : b->br) {
        free_cohort(r.sub);
        for (int i = 0; i < Workspace::kNumSlots; ++i)
            if (r.ws.ptr[i]) cudaFree(r.ws.ptr[i]);
        if (r.done) cudaEventDestroy(r.done);
        if (r.stream) cudaStreamDestroy(r.stream);
    }
    void *p[] = {b->masks, b->idx, b->counts, b->rows, b->dints, b->stage};
    for (void *q : p)
        if (q) cudaFree(q);
    if (b->host_counts) cudaFreeHost(b->host_counts);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    ctx->batch = nullptr;
}

static napg_status grow(napg_ctx *ctx, void **p, size_t *cap, size_t bytes) {
    if (*cap >= bytes) return NAPG_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    NAPG_CU(ctx, cudaMalloc(p, std::max<size_t>(bytes, 256)));
    *cap = std::max<size_t>(bytes, 256);
    return NAPG_OK;
}

static bool same_opt(const napg_options &a, const napg_options &b) {
    return a.precision == b.precision && a.welch == b.welch && a.yates_2x2 == b.yates_2x2 &&
           a.mwu_mode == b.mwu_mode && a.mwu_continuity == b.mwu_continuity && a.debug_checks == b.debug_checks;
}

// gather + pipeline of context k (stream-ordered, capture-safe once sized)
static napg_status run_context(napg_ctx *ctx, BatchState &b, BatchBranch &br, cudaStream_t st, int k,
                               int64_t idx_stride,
                               const int32_t *sub_va, const int32_t *sub_vb, int32_t na, int32_t nb,
                               double *stat, double *pval, int32_t *n) {
    const Cohort &P = ctx->coh;
    Cohort &c = br.sub;
    const int64_t Nk = b.nk[k];
    c.S = Nk;
    c.W = (Nk + 31) / 32;
    c.sorted = false;
    c.gen = next_cohort_gen();
    const int F = (int)c.F;
    if (Nk > 0 && F > 0) {
        const int64_t words = c.W;
        const unsigned gx = (unsigned)std::min<int64_t>((words * 32 + 255) / 256, 64);
        count_launch();
        if (P.dtype == NAPG_F32)
            k_ctx_gather<float><<<dim3(gx, (unsigned)F), 256, 0, st>>>(
                (const float *)P.X, P.obs, P.lab, P.S, P.W, b.rows, b.rows + F, b.idx + (int64_t)k * idx_stride, Nk,
                words, (float *)c.X, c.obs, c.lab);
        else
            k_ctx_gather<double><<<dim3(gx, (unsigned)F), 256, 0, st>>>(
                (const double *)P.X, P.obs, P.lab, P.S, P.W, b.rows, b.rows + F, b.idx + (int64_t)k * idx_stride, Nk,
                words, (double *)c.X, c.obs, c.lab);
        NAPG_CU(ctx, cudaGetLastError());
    }
    RunArgs a{};
    a.test = b.test;
    a.opt = b.opt;
    a.coh = &c;
    a.no_plane_cache = true;
    a.dints = b.dints;
    a.dints_off = b.doff.data();
    a.va = sub_va;
    a.na = na;
    a.vb = b.symmetric ? nullptr : sub_vb;
    a.nb = nb;
    a.stat = stat;
    a.pval = pval;
    a.n = n;
    if (Nk == 0) {
        // an empty context: every pair undefined, n = 0
        const int64_t cnt = (int64_t)na * (b.symmetric ? na : nb);
        if (stat) launch_fill_nan(stat, cnt, st);
        if (pval) launch_fill_nan(pval, cnt, st);
        if (n) NAPG_CU(ctx, cudaMemsetAsync(n, 0, sizeof(int32_t) * cnt, st));
        return NAPG_OK;
    }
    return run_on_stream(ctx, br.ws, st, a);
}

// loop over the contexts through napg_run's path (host outputs, or shapes the
// graph path does not take)

static napg_status batch_loop(napg_ctx *ctx, const RunArgs &a0, int32_t n_ctx, const uint8_t *const *masks,
                              double *const *stat, double *const *pval, int32_t *const *n) {
    for (int32_t k = 0; k < n_ctx; ++k) {
        RunArgs a = a0;
        a.mask = masks[k];
        a.mask_on_device = is_device_ptr(masks[k]);
        a.stat = stat ? stat[k] : nullptr;
        a.pval = pval ? pval[k] : nullptr;
        a.n = n ? n[k] : nullptr;
        NAPG_ST(run_with_outputs(ctx, ctx->ws, ctx->stream, a, a0.vb == nullptr));
    }
    return NAPG_OK;
}

// Host outputs: the batch runs on the graph path into device buffers (one region
// for every context's outputs), then each context's outputs are copied back.
// If the region cannot be allocated, the contexts go through the loop instead.
static napg_status batch_host_outputs(napg_ctx *ctx, const RunArgs &a0, int32_t n_ctx, const uint8_t *const *masks,
                                      double *const *stat, double *const *pval, int32_t *const *n, bool symmetric) {
    if (!ctx->batch) ctx->batch = new BatchState();
    BatchState &b = *ctx->batch;
    const int64_t cnt = (int64_t)a0.na * (symmetric ? a0.na : a0.nb);
    const size_t dbl = sizeof(double) * (size_t)cnt, i32 = sizeof(int32_t) * (size_t)cnt;
    const size_t per = (stat ? dbl : 0) + (pval ? dbl : 0) + (n ? ((i32 + 255) / 256) * 256 : 0);
    const size_t need = per * (size_t)n_ctx;
    if (b.stage_cap < need) {
        if (b.stage) cudaFree(b.stage);
        b.stage = nullptr;
        b.stage_cap = 0;
        if (cudaMalloc(&b.stage, need) != cudaSuccess) {
            (void)cudaGetLastError();
            b.stage = nullptr;
            return batch_loop(ctx, a0, n_ctx, masks, stat, pval, n);
        }
        b.stage_cap = need;
    }
    std::vector<double *> ds(n_ctx, nullptr), dp(n_ctx, nullptr);
    std::vector<int32_t *> dn(n_ctx, nullptr);
    unsigned char *cur = (unsigned char *)b.stage;
    for (int32_t k = 0; k < n_ctx; ++k) {
        if (stat) { ds[k] = (double *)cur; cur += dbl; }
        if (pval) { dp[k] = (double *)cur; cur += dbl; }
        if (n) { dn[k] = (int32_t *)cur; cur += ((i32 + 255) / 256) * 256; }
    }
    NAPG_ST(run_batch(ctx, a0, n_ctx, masks, stat ? ds.data() : nullptr, pval ? dp.data() : nullptr,
                      n ? dn.data() : nullptr));
    cudaStream_t st = ctx->stream;
    for (int32_t k = 0; k < n_ctx; ++k) {
        if (stat && stat[k]) NAPG_CU(ctx, cudaMemcpyAsync(stat[k], ds[k], dbl, cudaMemcpyDefault, st));
        if (pval && pval[k]) NAPG_CU(ctx, cudaMemcpyAsync(pval[k], dp[k], dbl, cudaMemcpyDefault, st));
        if (n && n[k]) NAPG_CU(ctx, cudaMemcpyAsync(n[k], dn[k], i32, cudaMemcpyDefault, st));
    }
    NAPG_CU(ctx, cudaMemcpyAsync(ctx->host_err, ctx->dev_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    NAPG_CU(ctx, cudaStreamSynchronize(st));
    if (*ctx->host_err) return device_error_status(ctx, *ctx->host_err);
    return NAPG_OK;
}

napg_status run_batch(napg_ctx *ctx, const RunArgs &a0, int32_t n_ctx, const uint8_t *const *masks,
                      double *const *stat, double *const *pval, int32_t *const *n) {
    Cohort &P = ctx->coh;
    if (!P.loaded) return fail(ctx, NAPG_E_ARG, "no cohort loaded");
    bool symmetric = false;
    NAPG_ST(check_run_vars(ctx, a0, &symmetric));
    if (n_ctx == 0 || a0.na == 0 || (!symmetric && a0.nb == 0)) return NAPG_OK;
    // Graph path: device outputs, and no A x B form of Pearson / chi-squared
    // (those run on the union of the lists and gather a block with a host sync).
    bool graphable = symmetric || !(a0.test == NAPG_PEARSON || a0.test == NAPG_CHI2);
    if (a0.test == NAPG_MWU && a0.pval && !a0.stat) graphable = false;   // exact U reads the statistic back
    bool host_out = false;
    for (int32_t k = 0; k < n_ctx && graphable; ++k) {
        const void *o[3] = {stat ? stat[k] : nullptr, pval ? pval[k] : nullptr, n ? n[k] : nullptr};
        for (const void *q : o)
            if (q && !is_device_ptr(q)) host_out = true;
        if (a0.test == NAPG_MWU && pval && pval[k] && !(stat && stat[k])) graphable = false;
    }
    if (!graphable) return batch_loop(ctx, a0, n_ctx, masks, stat, pval, n);
    if (host_out) return batch_host_outputs(ctx, a0, n_ctx, masks, stat, pval, n, symmetric);

    if (!ctx->batch) ctx->batch = new BatchState();
    BatchState &b = *ctx->batch;
    cudaStream_t st = ctx->stream;
    if (!b.stream) {
        NAPG_CU(ctx, cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking));
        NAPG_CU(ctx, cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming));
        NAPG_CU(ctx, cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming));
    }
    const int64_t S = P.S;
    const int32_t na = a0.na, nb = symmetric ? a0.na : a0.nb;

    // stage the masks (NULL = every sample) and count each context
    NAPG_ST(grow(ctx, (void **)&b.masks, &b.masks_cap, (size_t)n_ctx * (size_t)S));
    NAPG_ST(grow(ctx, (void **)&b.counts, &b.counts_cap, sizeof(int32_t) * (size_t)n_ctx));
    for (int32_t k = 0; k < n_ctx; ++k) {
        uint8_t *dst = b.masks + (int64_t)k * S;
        if (!masks || !masks[k]) NAPG_CU(ctx, cudaMemsetAsync(dst, 1, (size_t)S, st));
        else NAPG_CU(ctx, cudaMemcpyAsync(dst, masks[k], (size_t)S, cudaMemcpyDefault, st));
    }
    if (!b.host_counts) NAPG_CU(ctx, cudaMallocHost(&b.host_counts, sizeof(int32_t) * 4096));
    std::vector<int64_t> nk(n_ctx);
    for (int32_t k0 = 0; k0 < n_ctx; k0 += 4096) {
        const int32_t m = std::min<int32_t>(4096, n_ctx - k0);
        count_launch();
        k_ctx_count<<<m, 256, 0, st>>>(b.masks + (int64_t)k0 * S, S, b.counts + k0);
        NAPG_CU(ctx, cudaGetLastError());
        NAPG_CU(ctx, cudaMemcpyAsync(b.host_counts, b.counts + k0, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, st));
        NAPG_CU(ctx, cudaStreamSynchronize(st));
        for (int32_t j = 0; j < m; ++j) nk[k0 + j] = b.host_counts[j];
    }

    std::vector<int32_t> va(a0.va, a0.va + a0.na), vb;
    if (!symmetric) vb.assign(a0.vb, a0.vb + a0.nb);
    std::vector<void *> outs;
    for (int32_t k = 0; k < n_ctx; ++k) {
        outs.push_back(stat ? stat[k] : nullptr);
        outs.push_back(pval ? pval[k] : nullptr);
        outs.push_back(n ? n[k] : nullptr);
    }
    const bool same = b.valid && b.exec && b.parent_gen == P.gen && b.test == a0.test && same_opt(b.opt, a0.opt) &&
                      b.va == va && b.vb == vb && b.symmetric == symmetric && b.nk == nk && b.outs == outs;
    const int64_t nmax = n_ctx ? *std::max_element(nk.begin(), nk.end()) : 0;
    const int64_t idx_stride = std::max<int64_t>(nmax, 1);
    if (!same) {
        b.valid = false;
        if (b.exec) {
            cudaGraphExecDestroy(b.exec);
            b.exec = nullptr;
        }
        b.parent_gen = P.gen;
        b.test = a0.test;
        b.opt = a0.opt;
        b.va = va;
        b.vb = vb;
        b.symmetric = symmetric;
        b.nk = nk;
        b.outs = outs;
        // sub-cohort: rows 0..na-1 = vars_a, then vars_b (mixed-type tests)
        std::vector<int32_t> parent = va;
        if (!symmetric) parent.insert(parent.end(), vb.begin(), vb.end());
        const int F = (int)parent.size();
        Cohort &c = b.br[0].sub;
        c.F = F;
        c.dtype = P.dtype;
        c.missing = P.missing;
        c.loaded = true;
        c.vtype.assign(F, 0);
        c.nlev.assign(F, 0);
        c.cat_index.assign(F, -1);
        c.cont_index.assign(F, -1);
        c.n_cat = c.n_cont = 0;
        std::vector<int32_t> rows(2 * F + F, -1), cont_ids;
        for (int r = 0; r < F; ++r) {
            const int v = parent[r];
            rows[r] = v;
            c.vtype[r] = P.vtype[v];
            if (P.vtype[v] == 1) {
                c.nlev[r] = P.nlev[v];
                c.cat_index[r] = (int32_t)c.n_cat;
                rows[F + r] = (int32_t)c.n_cat;
                rows[2 * F + r] = P.cat_index[v];     // parent label row (read as cat_row[gridDim.y + r])
                ++c.n_cat;
            } else {
                c.cont_index[r] = (int32_t)c.n_cont++;
                cont_ids.push_back(r);
            }
        }
        // k_ctx_gather reads cat_row[r] (sub row) and cat_row[F + r] (parent row)
        std::vector<int32_t> rows_dev(3 * F);
        for (int r = 0; r < F; ++r) {
            rows_dev[r] = rows[r];
            rows_dev[F + r] = rows[F + r];
            rows_dev[2 * F + r] = rows[2 * F + r];
        }
        if (b.rows) cudaFree(b.rows);
        b.rows = nullptr;
        NAPG_CU(ctx, cudaMalloc(&b.rows, sizeof(int32_t) * rows_dev.size()));
        NAPG_CU(ctx, cudaMemcpy(b.rows, rows_dev.data(), sizeof(int32_t) * rows_dev.size(), cudaMemcpyHostToDevice));
        // contexts to branches, largest first onto the least-loaded branch
        std::vector<int32_t> order(n_ctx);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return nk[x] > nk[y]; });
        int64_t load[kBatchBranches] = {};
        for (BatchBranch &r : b.br) r.ctxs.clear();
        for (int32_t k : order) {
            int jb = 0;
            for (int j = 1; j < kBatchBranches; ++j)
                if (load[j] < load[jb]) jb = j;
            load[jb] += std::max<int64_t>(nk[k], 1);
            b.br[jb].ctxs.push_back(k);
        }
        const size_t esz = P.dtype == NAPG_F32 ? 4 : 8;
        for (int j = 0; j < kBatchBranches; ++j) {
            BatchBranch &r = b.br[j];
            std::sort(r.ctxs.begin(), r.ctxs.end());
            Cohort &cj = r.sub;
            if (j > 0) {
                cj.F = c.F; cj.dtype = c.dtype; cj.missing = c.missing; cj.loaded = true;
                cj.vtype = c.vtype; cj.nlev = c.nlev; cj.cat_index = c.cat_index; cj.cont_index = c.cont_index;
                cj.n_cat = c.n_cat; cj.n_cont = c.n_cont;
            }
            if (!r.stream) {
                NAPG_CU(ctx, cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking));
                NAPG_CU(ctx, cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming));
            }
            if (cj.cont_vars_dev) cudaFree(cj.cont_vars_dev);
            cj.cont_vars_dev = nullptr;
            if (!cont_ids.empty()) {
                NAPG_CU(ctx, cudaMalloc(&cj.cont_vars_dev, sizeof(int32_t) * cont_ids.size()));
                NAPG_CU(ctx, cudaMemcpy(cj.cont_vars_dev, cont_ids.data(), sizeof(int32_t) * cont_ids.size(),
                                        cudaMemcpyHostToDevice));
            }
            int64_t nj = 1;
            for (int32_t k : r.ctxs) nj = std::max<int64_t>(nj, nk[k]);
            const int64_t wj = (nj + 31) / 32;
            NAPG_ST(grow(ctx, &cj.X, &r.sub_x_cap, esz * (size_t)F * (size_t)nj));
            NAPG_ST(grow(ctx, (void **)&cj.obs, &r.sub_obs_cap, sizeof(uint32_t) * (size_t)F * (size_t)wj));
            NAPG_ST(grow(ctx, (void **)&cj.lab, &r.sub_lab_cap, (size_t)std::max<int64_t>(c.n_cat, 1) * (size_t)nj));
        }
        NAPG_ST(grow(ctx, (void **)&b.idx, &b.idx_cap, sizeof(int32_t) * (size_t)n_ctx * (size_t)idx_stride));
        // variable lists of the sub-cohort run, staged once
        std::vector<int32_t> sva(na), svb(symmetric ? 0 : nb);
        std::iota(sva.begin(), sva.end(), 0);
        std::iota(svb.begin(), svb.end(), na);
        RunArgs la{};
        la.test = a0.test;
        la.va = sva.data();
        la.na = na;
        la.vb = symmetric ? nullptr : svb.data();
        la.nb = nb;
        std::vector<int32_t> l_va, l_vb, l_cat, l_nl, l_lo, all;
        int32_t R = 0, maxlev = 0;
        var_lists(c, la, symmetric, l_va, l_vb, l_cat, l_nl, l_lo, R, maxlev, all, b.doff);
        if (b.dints) cudaFree(b.dints);
        b.dints = nullptr;
        NAPG_CU(ctx, cudaMalloc(&b.dints, sizeof(int32_t) * (all.size() + 1)));
        NAPG_CU(ctx, cudaMemcpy(b.dints, all.data(), sizeof(int32_t) * all.size(), cudaMemcpyHostToDevice));

        // size every branch with its largest context, uncaptured
        const bool trace_on = ctx->trace.on;
        ctx->trace.on = false;
        NAPG_CU(ctx, cudaEventRecord(b.fork, st));
        NAPG_CU(ctx, cudaStreamWaitEvent(b.stream, b.fork, 0));
        count_launch();
        k_ctx_compact<<<n_ctx, 1024, 0, b.stream>>>(b.masks, S, b.idx, idx_stride);
        NAPG_CU(ctx, cudaGetLastError());
        NAPG_CU(ctx, cudaEventRecord(b.join, b.stream));
        napg_status r0 = NAPG_OK;
        for (BatchBranch &r : b.br) {
            if (r.ctxs.empty() || r0 != NAPG_OK) continue;
            int32_t kmax = r.ctxs[0];
            for (int32_t k : r.ctxs)
                if (nk[k] > nk[kmax]) kmax = k;
            NAPG_CU(ctx, cudaStreamWaitEvent(r.stream, b.join, 0));
            r0 = run_context(ctx, b, r, r.stream, kmax, idx_stride, sva.data(), svb.data(), na, nb,
                             stat ? stat[kmax] : nullptr, pval ? pval[kmax] : nullptr, n ? n[kmax] : nullptr);
        }
        cudaError_t e0 = cudaSuccess;
        for (BatchBranch &r : b.br) {
            const cudaError_t e = cudaStreamSynchronize(r.stream);
            if (e0 == cudaSuccess) e0 = e;
        }
        if (r0 != NAPG_OK) { ctx->trace.on = trace_on; return r0; }
        if (e0 != cudaSuccess) { ctx->trace.on = trace_on; return cuda_fail(ctx, e0, "batch sizing run"); }

        // capture the whole batch: compaction, then the branches forked from it and joined at the end
        cudaGraph_t g = nullptr;
        NAPG_CU(ctx, cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeRelaxed));
        const uint64_t l0 = launches_so_far();
        k_ctx_compact<<<n_ctx, 1024, 0, b.stream>>>(b.masks, S, b.idx, idx_stride);
        napg_status rc = NAPG_OK;
        cudaError_t ef = cudaEventRecord(b.fork, b.stream);
        for (BatchBranch &r : b.br) {
            if (r.ctxs.empty() || rc != NAPG_OK || ef != cudaSuccess) continue;
            ef = cudaStreamWaitEvent(r.stream, b.fork, 0);
            for (size_t q = 0; q < r.ctxs.size() && rc == NAPG_OK && ef == cudaSuccess; ++q) {
                const int32_t k = r.ctxs[q];
                rc = run_context(ctx, b, r, r.stream, k, idx_stride, sva.data(), svb.data(), na, nb,
                                 stat ? stat[k] : nullptr, pval ? pval[k] : nullptr, n ? n[k] : nullptr);
            }
            if (ef == cudaSuccess) ef = cudaEventRecord(r.done, r.stream);
            if (ef == cudaSuccess) ef = cudaStreamWaitEvent(b.stream, r.done, 0);
        }
        const cudaError_t ec = cudaStreamEndCapture(b.stream, &g);
        ctx->trace.on = trace_on;
        if (rc == NAPG_OK && ef != cudaSuccess) rc = cuda_fail(ctx, ef, "batch graph branches");
        if (rc != NAPG_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return cuda_fail(ctx, ec, "batch graph capture");
        // kernels in the graph (the capture counted them as launches: take them back)
        size_t nn = 0;
        NAPG_CU(ctx, cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        NAPG_CU(ctx, cudaGraphGetNodes(g, nodes.data(), &nn));
        uint64_t kern = 0;
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kern;
        }
        uncount_launches(launches_so_far() - l0);
        b.kernels = kern;
        const cudaError_t ei = cudaGraphInstantiate(&b.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            b.exec = nullptr;
            return cuda_fail(ctx, ei, "batch graph instantiate");
        }
        b.valid = true;
    }
    // one graph launch for the batch, ordered after the staging copies
    NAPG_CU(ctx, cudaMemsetAsync(ctx->dev_err, 0, sizeof(uint32_t), st));
    NAPG_CU(ctx, cudaEventRecord(b.fork, st));
    NAPG_CU(ctx, cudaStreamWaitEvent(b.stream, b.fork, 0));
    NAPG_CU(ctx, cudaGraphLaunch(b.exec, b.stream));
    count_launch(b.kernels);
    NAPG_CU(ctx, cudaEventRecord(b.join, b.stream));
    NAPG_CU(ctx, cudaStreamWaitEvent(st, b.join, 0));
    return NAPG_OK;
}

}  // namespace napg
