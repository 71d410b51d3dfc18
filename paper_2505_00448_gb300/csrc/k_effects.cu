// Effect sizes (Table 2) from the final statistics, and multiple-testing
// correction of a p-value matrix (Sec. 3.4: Bonferroni, Benjamini-Hochberg,
// Benjamini-Yekutieli).
//
// Effect sizes, NaN wherever the statistic is NaN: Pearson r^2; Spearman rho;
// chi-squared phi = sqrt(chi2 / n) and Cramer's V = sqrt(chi2 / (n (min(k_a, k_b)
// - 1))) over the levels present in the context (V NaN with a single level);
// ANOVA partial eta^2 = F d1 / (F d1 + d2) (= SSB / (SSB + SSW); 1 when F is
// infinite); Mann-Whitney r = |U_0 - n_0 n_1 / 2| / sigma / sqrt(n) with the
// tie-corrected sigma, no continuity correction; Kruskal-Wallis eta^2 =
// (H - k + 1) / (n - k), NaN when n <= k. The t-test's Cohen's d and its
// degrees of freedom are formed by the group finalize and the rescue, which
// hold the group variances.
//
// Correction: the tests are the entries with a p-value (the upper triangle
// i < j of a symmetric matrix, whose diagonal is no test and becomes NaN). The
// m valid p-values are compacted (prefix sum of flags), sorted ascending
// (radix sort), and p_adj_(i) = min over k >= i of (p_(k) scale) / k with
// scale = m (Benjamini-Hochberg) or m c(m), c(m) = sum_{k <= m} 1/k
// (Benjamini-Yekutieli): a minimum scan over the reversed sequence. Bonferroni
// is min(1, m p) elementwise. Results are capped at 1 and scattered back
// (mirrored for a symmetric matrix); entries without a p-value stay NaN.
#include "napg_internal.cuh"

#include <cub/cub.cuh>

namespace napg {

__device__ __forceinline__ double enan() { return __longlong_as_double(0x7ff8000000000000LL); }

// levels of categorical i of vars_a present in the context
__device__ __forceinline__ int present_levels(const EffectArgs &e, int i) {
    const int c = e.nlev[i], off = e.levoff[i];
    int k = 0;
    for (int g = 0; g < c; ++g) k += e.levcnt[off + g] > 0;
    return k;
}

__global__ void k_effects(EffectArgs e) {
    const int64_t total = (int64_t)e.na * e.nb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / e.nb), j = (int)(t - (int64_t)a * e.nb);
        const double s = e.stat[t], n = (double)e.n[t];
        double x1 = enan(), x2 = enan();
        if (!isnan(s)) {
            switch (e.test) {
                case NAPG_PEARSON: x1 = s * s; break;
                case NAPG_SPEARMAN: x1 = s; break;
                case NAPG_CHI2: {
                    x1 = sqrt(s / n);
                    const int m = min(present_levels(e, a), present_levels(e, j)) - 1;
                    if (m >= 1) x2 = sqrt(s / (n * (double)m));
                    break;
                }
                case NAPG_ANOVA: {
                    const int k = present_levels(e, a);
                    if (isinf(s)) {
                        x1 = 1.0;
                    } else {
                        const double d1 = (double)(k - 1), d2 = n - (double)k;
                        x1 = s * d1 / (s * d1 + d2);
                    }
                    break;
                }
                case NAPG_MWU: {
                    const int off = e.levoff[a];
                    const double n0 = (double)e.rcnt[(int64_t)off * e.nb + j];
                    const double n1 = (double)e.rcnt[(int64_t)(off + 1) * e.nb + j];
                    const double T = (double)e.tie[t];
                    const double var = n0 * n1 / 12.0 * ((n + 1.0) - T / (n * (n - 1.0)));
                    if (var > 0.0) x1 = fabs(s - 0.5 * n0 * n1) / sqrt(var) / sqrt(n);
                    break;
                }
                case NAPG_KRUSKAL: {
                    const int k = present_levels(e, a);
                    if (n > (double)k) x1 = (s - (double)k + 1.0) / (n - (double)k);
                    break;
                }
                default: break;
            }
        }
        // the t-test's two outputs (Cohen's d, degrees of freedom) come from the
        // group finalize and the rescue
        if (e.es1 && e.test != NAPG_TTEST) e.es1[t] = x1;
        if (e.es2 && e.test != NAPG_TTEST) e.es2[t] = x2;
    }
}

void launch_effects(const EffectArgs &e, cudaStream_t st) {
    const int64_t total = (int64_t)e.na * e.nb;
    if (total == 0 || (!e.es1 && !e.es2)) return;
    count_launch();
    k_effects<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, st>>>(e);
}

// ------------------------------------------------------------- correction --

// flag[q] = 1 for the entries that are tests (a p-value, above the diagonal of a
// symmetric matrix); the adjusted matrix starts as NaN
__global__ void k_adj_flags(const double *p, int64_t rows, int64_t cols, int32_t symmetric, int64_t *flag,
                            double *out) {
    const int64_t total = rows * cols;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / cols, j = q - i * cols;
        flag[q] = (!symmetric || i < j) && !isnan(p[q]) ? 1 : 0;
        out[q] = enan();
    }
}

// compact the tests' p-values and their matrix positions (pos = exclusive
// prefix sum of the flags: the order of the matrix is kept)
__global__ void k_adj_compact(const double *p, int64_t total, const int64_t *flag, const int64_t *pos, double *keys,
                              int64_t *idx) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
        if (flag[q]) { keys[pos[q]] = p[q]; idx[pos[q]] = q; }
}

__global__ void k_adj_bonferroni(const double *keys, const int64_t *idx, int64_t m, int64_t cols, int32_t symmetric,
                                 double *out) {
    const double md = (double)m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = fmin(1.0, keys[i] * md);
        const int64_t q = idx[i];
        out[q] = v;
        if (symmetric) out[(q % cols) * cols + q / cols] = v;
    }
}

// terms (p_(i) scale) / i in reversed order, for the minimum scan
__global__ void k_adj_terms(const double *sorted, int64_t m, double scale, double *rev) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        rev[m - 1 - i] = (sorted[i] * scale) / (double)(i + 1);
}

__global__ void k_adj_scatter(const double *revmin, const int64_t *sidx, int64_t m, int64_t cols, int32_t symmetric,
                              double *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = fmin(1.0, revmin[m - 1 - i]);
        const int64_t q = sidx[i];
        out[q] = v;
        if (symmetric) out[(q % cols) * cols + q / cols] = v;
    }
}

struct MinOp {
    __device__ __forceinline__ double operator()(double a, double b) const { return b < a ? b : a; }
};

static unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

napg_status adjust_pvalues(napg_ctx *ctx, Workspace &ws, cudaStream_t st, int32_t method, const double *p,
                           int64_t rows, int64_t cols, int32_t symmetric, double *out) {
    if (method != NAPG_ADJ_BONFERRONI && method != NAPG_ADJ_BH && method != NAPG_ADJ_BY)
        return fail(ctx, NAPG_E_ARG, "unknown correction method");
    if (rows < 0 || cols < 0 || (symmetric && rows != cols)) return fail(ctx, NAPG_E_ARG, "bad matrix shape");
    const int64_t total = rows * cols;
    if (total == 0) return NAPG_OK;
    // scratch: flags and positions, keys in/out, indices in/out, CUB temporary
    size_t tmp_scan = 0, tmp_sort = 0, tmp_min = 0;
    NAPG_CU(ctx, cub::DeviceScan::ExclusiveSum(nullptr, tmp_scan, (const int64_t *)nullptr, (int64_t *)nullptr, total));
    NAPG_CU(ctx, cub::DeviceRadixSort::SortPairs(nullptr, tmp_sort, (const double *)nullptr, (double *)nullptr,
                                                 (const int64_t *)nullptr, (int64_t *)nullptr, total));
    NAPG_CU(ctx, cub::DeviceScan::InclusiveScan(nullptr, tmp_min, (const double *)nullptr, (double *)nullptr, MinOp(),
                                                total));
    const size_t tmp_bytes = std::max(tmp_scan, std::max(tmp_sort, tmp_min));
    napg_status st_ = NAPG_OK;
    int64_t *fl = (int64_t *)ws_get(ctx, ws, Workspace::kAdjTmp, sizeof(int64_t) * 2 * (size_t)total + tmp_bytes + 256,
                                    &st_);
    double *keys = (double *)ws_get(ctx, ws, Workspace::kAdjKeys, sizeof(double) * 2 * (size_t)total, &st_);
    int64_t *idx = (int64_t *)ws_get(ctx, ws, Workspace::kAdjVals, sizeof(int64_t) * 2 * (size_t)total, &st_);
    if (st_) return st_;
    int64_t *pos = fl + total;
    void *tmp = (void *)(((uintptr_t)(pos + total) + 255) & ~(uintptr_t)255);
    double *keys2 = keys + total;
    int64_t *idx2 = idx + total;
    count_launch();
    k_adj_flags<<<grid_for(total), 256, 0, st>>>(p, rows, cols, symmetric, fl, out);
    NAPG_CU(ctx, cudaGetLastError());
    size_t tb = tmp_bytes;
    NAPG_CU(ctx, cub::DeviceScan::ExclusiveSum(tmp, tb, fl, pos, total, st));
    count_launch();
    k_adj_compact<<<grid_for(total), 256, 0, st>>>(p, total, fl, pos, keys, idx);
    NAPG_CU(ctx, cudaGetLastError());
    // m = last position + last flag
    int64_t tail[2] = {0, 0};
    NAPG_CU(ctx, cudaMemcpyAsync(&tail[0], pos + total - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    NAPG_CU(ctx, cudaMemcpyAsync(&tail[1], fl + total - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    NAPG_CU(ctx, cudaStreamSynchronize(st));
    const int64_t m = tail[0] + tail[1];
    if (m == 0) return NAPG_OK;
    if (method == NAPG_ADJ_BONFERRONI) {
        count_launch();
        k_adj_bonferroni<<<grid_for(m), 256, 0, st>>>(keys, idx, m, cols, symmetric, out);
        NAPG_CU(ctx, cudaGetLastError());
        return NAPG_OK;
    }
    tb = tmp_bytes;
    NAPG_CU(ctx, cub::DeviceRadixSort::SortPairs(tmp, tb, keys, keys2, idx, idx2, m, 0, 64, st));
    double scale = (double)m;
    if (method == NAPG_ADJ_BY) {
        double cm = 0.0;                         // c(m), summed in increasing k
        for (int64_t k = 1; k <= m; ++k) cm += 1.0 / (double)k;
        scale = (double)m * cm;
    }
    count_launch();
    k_adj_terms<<<grid_for(m), 256, 0, st>>>(keys2, m, scale, keys);
    NAPG_CU(ctx, cudaGetLastError());
    tb = tmp_bytes;   // the sorted keys are spent: their buffer takes the scan
    NAPG_CU(ctx, cub::DeviceScan::InclusiveScan(tmp, tb, keys, keys2, MinOp(), m, st));
    count_launch();
    k_adj_scatter<<<grid_for(m), 256, 0, st>>>(keys2, idx2, m, cols, symmetric, out);
    NAPG_CU(ctx, cudaGetLastError());
    return NAPG_OK;
}

}  // namespace napg
