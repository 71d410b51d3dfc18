// P-value evaluation of queued jobs (pjobs.cuh): counting sort by key, then one
// thread per job in key order, so that neighbouring lanes take the same branch
// of the special function with continued fractions of similar length.
#include <algorithm>

#include "napg_internal.cuh"
#include "pjobs.cuh"
#include "specfun.cuh"

namespace napg {

// exclusive scan of the per-key histogram; cursors zeroed
__global__ void k_pj_scan(const int32_t *hist, int32_t *offs, int32_t *cursor) {
    if (threadIdx.x == 0) {
        int32_t run = 0;
        for (int k = 0; k < kPjBins; ++k) { offs[k] = run; run += hist[k]; cursor[k] = 0; }
    }
}

// A block takes kScatterPer jobs per thread at a time into registers; jobs
// with the same key take consecutive slots of the block's share of that key
// (shared-memory counts, one atomic per warp and key), and the block claims
// its share of each key's range with one global atomic per key it holds. Most
// jobs share a few keys: per-warp global atomics on those keys' cursors
// serialised the scatter.
constexpr int kScatterPer = 4;

__global__ void __launch_bounds__(256) k_pj_scatter(const PJob *jobs, const int32_t *count, int32_t capacity,
                                                    const int32_t *offs, int32_t *cursor, PJob *sorted) {
    __shared__ int32_t s_cnt[kPjBins];
    __shared__ int32_t s_base[kPjBins];
    const int32_t n = min(*count, capacity);
    const int lane = threadIdx.x & 31;
    const int32_t chunk = (int32_t)blockDim.x * kScatterPer;
    for (int32_t c0 = blockIdx.x * chunk; c0 < n; c0 += gridDim.x * chunk) {   // block-uniform
        for (int k = threadIdx.x; k < kPjBins; k += blockDim.x) s_cnt[k] = 0;
        __syncthreads();
        PJob j[kScatterPer];
        int key[kScatterPer], rank[kScatterPer];
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {
            const int32_t t = c0 + u * (int32_t)blockDim.x + (int32_t)threadIdx.x;
            key[u] = kPjBins;                   // no job
            if (t < n) {
                j[u] = jobs[t];
                key[u] = min(j[u].kind >> 8, kPjBins);
            }
            const unsigned same = __match_any_sync(0xffffffffu, key[u]);
            const int leader = __ffs(same) - 1;
            int r = 0;
            if (lane == leader && key[u] < kPjBins) r = atomicAdd(&s_cnt[key[u]], __popc(same));
            r = __shfl_sync(0xffffffffu, r, leader);
            rank[u] = r + __popc(same & ((1u << lane) - 1u));
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kPjBins; k += blockDim.x)
            if (s_cnt[k] > 0) s_base[k] = offs[k] + atomicAdd(&cursor[k], s_cnt[k]);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u)
            if (key[u] < kPjBins) sorted[s_base[key[u]] + rank[u]] = j[u];
        __syncthreads();                        // the counts are reused
    }
}

// At most 80 registers a thread (a few bytes spill), four 128-thread blocks per
// SM: more warps in flight for the long FP64 latencies than 130 registers
// allowed (measured 0.6-0.8 ms less per mixed-cohort step).
__global__ void __launch_bounds__(128, 6) k_pj_eval(const PJob *sorted, const int32_t *count, int32_t capacity, double *pval,
                          const double *bgrat, sf::LargeATab lat) {
    const int32_t n = min(*count, capacity);
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const PJob j = sorted[t];
        const int kind = j.kind & 0xff;
        double p;
        if ((j.kind >> 8) >= kPjKeyLargeA) {
            // the key was taken from these arguments (pjob_key): the expansion
            // applies and its checks are settled, so the incomplete beta is
            // entered directly with the arguments corr_p / t_two_sided / f_sf form
            double a, b, x, y;
            if (kind == kPjCorr) {
                a = 0.5 * (j.a - 2.0); b = 0.5; x = (1.0 - j.s) * (1.0 + j.s); y = j.s * j.s;
            } else if (kind == kPjT) {
                const double t2 = j.s * j.s;
                a = 0.5 * j.a; b = 0.5; x = j.a / (j.a + t2); y = t2 / (j.a + t2);
            } else {
                const double den = j.b + j.a * j.s;
                a = 0.5 * j.b; b = 0.5 * j.a; x = j.b / den; y = j.a * j.s / den;
            }
            p = sf::ibeta_large_a(a, b, x, y, bgrat ? bgrat + ((int)(2.0 * b) - 1) * sf::kBgratTerms : nullptr, lat);
        } else {
            switch (kind) {
                case kPjCorr: p = sf::corr_p(j.s, j.a, bgrat, lat); break;
                case kPjT: p = sf::t_two_sided(j.s, j.a, bgrat, lat); break;
                case kPjF: p = sf::f_sf(j.s, j.a, j.b, bgrat, lat); break;
                default: p = sf::chi2_sf(j.s, j.a); break;
            }
        }
        pval[j.idx] = p;
        if (j.mirror > 0) {
            const int64_t r = j.idx / j.mirror, c = j.idx - r * j.mirror;
            if (r != c) pval[c * j.mirror + r] = p;
        }
    }
}

void launch_pjobs_eval(const PJobQueue &q, PJob *sorted, int32_t *offs, int32_t *cursor, double *pval,
                       cudaStream_t st, int sm_count) {
    if (!pval) return;
    count_launch(3);
    k_pj_scan<<<1, 32, 0, st>>>(q.hist, offs, cursor);
    k_pj_scatter<<<sm_count * 8, 256, 0, st>>>(q.jobs, q.count, q.capacity, offs, cursor, sorted);
    k_pj_eval<<<sm_count * 4, 128, 0, st>>>(sorted, q.count, q.capacity, pval, q.bgrat, q.lat);
}

// the (log M, 1/T^2) table of sf::LargeATab, one thread per entry
__global__ void k_large_a_table(double2 *v, int32_t n2a, int32_t rows) {
    const int64_t cols = (int64_t)n2a + 1, total = (int64_t)rows * cols;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / cols, a2 = t - r * cols;
        const double a = 0.5 * (double)a2, b = 0.5 * (double)(r + 1);
        double logM = __longlong_as_double(0x7ff8000000000000LL), invT2 = logM;
        if (a >= 20.0) sf::large_a_consts(a, b, logM, invT2);
        v[t] = make_double2(logM, invT2);
    }
}

void launch_large_a_table(double2 *v, int32_t n2a, int32_t rows, cudaStream_t st) {
    const int64_t total = (int64_t)rows * ((int64_t)n2a + 1);
    if (total <= 0) return;
    count_launch();
    k_large_a_table<<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16), 256, 0, st>>>(v, n2a, rows);
}

// the table of expansion coefficients c_k(b), 2b = 1..64 (one thread per row)
__global__ void k_bgrat_table(double *tab) {
    const int r = threadIdx.x;
    if (r < sf::kBgratRows) sf::bgrat_coefs(0.5 * (double)(r + 1), tab + r * sf::kBgratTerms);
}

void launch_bgrat_table(double *tab, cudaStream_t st) {
    count_launch();
    k_bgrat_table<<<1, sf::kBgratRows, 0, st>>>(tab);
}

// p-values of caller-supplied statistics (kinds as napg_debug_pvalues)
__global__ void k_debug_pvalues(int32_t kind, const double *s, const double *a, const double *b, int64_t count,
                                double *p, const double *bgrat) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
        double v;
        switch (kind) {
            case 0: v = sf::corr_p(s[t], a[t], bgrat); break;
            case 1: v = sf::t_two_sided(s[t], a[t], bgrat); break;
            case 2: v = sf::f_sf(s[t], a[t], b[t], bgrat); break;
            case 3: v = sf::chi2_sf(s[t], a[t]); break;
            case 4: v = sf::norm_sf(s[t]); break;
            case 5: v = sf::ibeta(a[t], b[t], s[t], 1.0 - s[t], bgrat); break;
            case 6: v = sf::gamma_q(a[t], s[t]); break;
            case 7: { double su; v = sf::erfcx_of_sqrt(s[t], su); } break;
            default: v = erfcx(sqrt(s[t])); break;
        }
        p[t] = v;
    }
}

void launch_debug_pvalues(int32_t kind, const double *s, const double *a, const double *b, int64_t count, double *p,
                          const double *bgrat, cudaStream_t st) {
    if (count <= 0) return;
    count_launch();
    const int64_t blocks = std::min<int64_t>((count + 127) / 128, 152 * 16);
    k_debug_pvalues<<<(unsigned)blocks, 128, 0, st>>>(kind, s, a, b, count, p, bgrat);
}

}  // namespace napg
