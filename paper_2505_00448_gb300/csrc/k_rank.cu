// Rank tests (Sec. 3.5.3 Spearman, 3.5.6 Mann-Whitney U, 3.5.8 Kruskal-Wallis).
//
// Presort (the paper sorts and ranks each feature once, Sec. 3.5.3/3.5.6): every
// continuous variable's observed samples are sorted by value once per cohort
// (ties broken by sample index). A sample context or the other variable of a
// pair only removes samples, so the global order restricted to the survivors is
// still sorted and its tie groups are the global groups restricted likewise.
//
// Pairwise re-rank: for a pair, B[p] = 1 when the sample at sorted position p is
// co-observed. With P(x) = number of co-observed positions < x and a tie group
// spanning positions [gs, ge), a co-observed member has
//   L = P(gs) values strictly below it and t = P(ge) - P(gs) tied with it,
// so its doubled rank is 2R = 2L + t + 1 = P(gs) + P(ge) + 1, an integer.
// Rank sums are accumulated in int64 and are exact.
#include <type_traits>

#include <algorithm>

#include "napg_internal.cuh"

namespace napg {

// ------------------------------------------------------------------ presort --

__device__ __forceinline__ uint64_t order_key(double v) {
    if (v == 0.0) v = 0.0;                       // -0 and +0 tie
    const uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ bool key_less(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

constexpr int kSortSmem = 16384;   // elements sorted in shared memory

// bitonic compare-exchange network over n2 (power of two) elements in shared memory
__device__ void bitonic_smem(uint64_t *key, uint32_t *idx, int n2, int kmin) {
    for (int k = kmin; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < n2; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const bool up = (t & k) == 0;
                    const uint64_t kt = key[t], ku = key[u];
                    const uint32_t it = idx[t], iu = idx[u];
                    const bool sw = up ? key_less(ku, iu, kt, it) : key_less(kt, it, ku, iu);
                    if (sw) { key[t] = ku; key[u] = kt; idx[t] = iu; idx[u] = it; }
                }
            }
            __syncthreads();
        }
    }
}

// stages with stride j >= kSortSmem run on global memory (one CTA per column)
__device__ void bitonic_global_stage(uint64_t *key, uint32_t *idx, int n2, int k, int j) {
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
            const bool up = (t & k) == 0;
            const uint64_t kt = key[t], ku = key[u];
            const uint32_t it = idx[t], iu = idx[u];
            const bool sw = up ? key_less(ku, iu, kt, it) : key_less(kt, it, ku, iu);
            if (sw) { key[t] = ku; key[u] = kt; idx[t] = iu; idx[u] = it; }
        }
    }
    __syncthreads();
}

// Shared-memory stages of the bitonic network on each kSortSmem-aligned block of
// the global array: levels k_lo..k_hi (k_lo == k_hi: only the strides below
// kSortSmem of one level). Directions use the global index.
__device__ void bitonic_local_levels(uint64_t *gkey, uint32_t *gidx, uint64_t *skey, uint32_t *sidx, int n2,
                                     int k_lo, int k_hi) {
    for (int base = 0; base < n2; base += kSortSmem) {
        for (int t = threadIdx.x; t < kSortSmem; t += blockDim.x) { skey[t] = gkey[base + t]; sidx[t] = gidx[base + t]; }
        __syncthreads();
        for (int k = k_lo; k <= k_hi; k <<= 1) {
            for (int j = ((k >> 1) < kSortSmem ? (k >> 1) : (kSortSmem >> 1)); j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < kSortSmem; t += blockDim.x) {
                    const int u = t ^ j;
                    if (u > t) {
                        const bool up = ((base + t) & k) == 0;
                        const uint64_t kt = skey[t], ku = skey[u];
                        const uint32_t it = sidx[t], iu = sidx[u];
                        const bool sw = up ? key_less(ku, iu, kt, it) : key_less(kt, it, ku, iu);
                        if (sw) { skey[t] = ku; skey[u] = kt; sidx[t] = iu; sidx[u] = it; }
                    }
                }
                __syncthreads();
            }
        }
        for (int t = threadIdx.x; t < kSortSmem; t += blockDim.x) { gkey[base + t] = skey[t]; gidx[base + t] = sidx[t]; }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_presort(const T *__restrict__ X, int64_t S, int64_t W,
                                                  const int32_t *__restrict__ contvars, const uint32_t *__restrict__ obs,
                                                  int32_t *__restrict__ perm, int32_t *__restrict__ pos,
                                                  int32_t *__restrict__ nobs, uint32_t *__restrict__ tie,
                                                  int32_t *__restrict__ gsw, int32_t *__restrict__ gew,
                                                  uint64_t *__restrict__ gkey_all, uint32_t *__restrict__ gidx_all,
                                                  int64_t n2max, int cv_base) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *skey = (uint64_t *)smem_raw;
    uint32_t *sidx = (uint32_t *)(skey + kSortSmem);
    __shared__ int s_count;
    const int cv = blockIdx.x + cv_base;     // continuous row
    const int slot = blockIdx.x;             // temp slot of this batch
    const int v = contvars[cv];
    const uint32_t *ob = obs + (int64_t)v * W;
    const T *x = X + (int64_t)v * S;
    // count observed
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    int local = 0;
    for (int64_t w = threadIdx.x; w < W; w += blockDim.x) local += __popc(ob[w]);
    atomicAdd(&s_count, local);
    __syncthreads();
    const int n = s_count;
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    const bool in_smem = n2 <= kSortSmem;
    uint64_t *key = in_smem ? skey : gkey_all + (int64_t)slot * n2max;
    uint32_t *idx = in_smem ? sidx : gidx_all + (int64_t)slot * n2max;
    // compact observed samples in sample order: word prefix counts via a serial scan per warp-chunk
    __shared__ int wbase[1024 + 1];
    const int64_t chunk = (W + blockDim.x - 1) / blockDim.x;
    {
        const int64_t w0 = threadIdx.x * chunk, w1 = min(W, w0 + chunk);
        int c = 0;
        for (int64_t w = w0; w < w1; ++w) c += __popc(ob[w]);
        wbase[threadIdx.x + 1] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        wbase[0] = 0;
        for (int t = 1; t <= (int)blockDim.x; ++t) wbase[t] += wbase[t - 1];
    }
    __syncthreads();
    {
        const int64_t w0 = threadIdx.x * chunk, w1 = min(W, w0 + chunk);
        int o = wbase[threadIdx.x];
        for (int64_t w = w0; w < w1; ++w) {
            uint32_t m = ob[w];
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int64_t s = w * 32 + b;
                key[o] = order_key((double)x[s]);
                idx[o] = (uint32_t)s;
                ++o;
            }
        }
    }
    for (int t = n + threadIdx.x; t < n2; t += blockDim.x) { key[t] = ~0ull; idx[t] = 0xffffffffu; }
    __syncthreads();
    if (in_smem) {
        bitonic_smem(key, idx, n2, 2);
    } else {
        // levels up to kSortSmem entirely in shared memory, then for each larger
        // level the long strides on global memory and the short ones in smem
        bitonic_local_levels(key, idx, skey, sidx, n2, 2, kSortSmem);
        for (int k = kSortSmem << 1; k <= n2; k <<= 1) {
            for (int j = k >> 1; j >= kSortSmem; j >>= 1) bitonic_global_stage(key, idx, n2, k, j);
            bitonic_local_levels(key, idx, skey, sidx, n2, k, k);
        }
    }
    // outputs: perm, pos, tie bits
    int32_t *pm = perm + (int64_t)cv * S;
    int32_t *ps = pos + (int64_t)cv * S;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) ps[s] = -1;
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        pm[p] = (int32_t)idx[p];
        ps[idx[p]] = p;
    }
    uint32_t *tw = tie + (int64_t)cv * W;
    for (int64_t w = threadIdx.x; w < W; w += blockDim.x) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t p = w * 32 + b;
            if (p < n && (p == 0 || key[p] != key[p - 1])) bits |= 1u << b;
        }
        tw[w] = bits;
    }
    __syncthreads();
    // gsw[w] = last group start strictly before position 32w; gew[w] = first group start at or after 32(w+1)
    if (threadIdx.x == 0) {
        int32_t *gs = gsw + (int64_t)cv * W, *ge = gew + (int64_t)cv * W;
        int last = 0;
        for (int64_t w = 0; w < W; ++w) {
            gs[w] = last;
            const uint32_t b = tw[w];
            if (b) last = (int)(w * 32 + 31 - __clz(b));
        }
        int next = n;
        for (int64_t w = W - 1; w >= 0; --w) {
            ge[w] = next;
            const uint32_t b = tw[w];
            if (b) next = (int)(w * 32 + __ffs(b) - 1);
        }
        nobs[cv] = n;
    }
}

constexpr int kPresortBatch = 1024;   // columns per launch on the global-memory path

size_t presort_tmp_bytes(int64_t S, int32_t ncont) {
    int64_t n2 = 1;
    while (n2 < S) n2 <<= 1;
    if (n2 <= kSortSmem) return 16;
    const int64_t cols = ncont < kPresortBatch ? ncont : kPresortBatch;
    return (size_t)cols * (size_t)n2 * (sizeof(uint64_t) + sizeof(uint32_t));
}

void launch_presort(const void *X, int32_t dtype, int64_t S, int64_t W, const int32_t *contvars_dev, int32_t ncont,
                    const uint32_t *obs, int32_t *perm, int32_t *pos, int32_t *nobs, uint32_t *tie, int32_t *gsw,
                    int32_t *gew, void *tmp, size_t tmp_bytes, cudaStream_t st) {
    if (ncont == 0) return;
    int64_t n2 = 1;
    while (n2 < S) n2 <<= 1;
    (void)tmp_bytes;
    uint64_t *gk = nullptr;
    uint32_t *gi = nullptr;
    const int batch = n2 > kSortSmem ? kPresortBatch : ncont;
    if (n2 > kSortSmem) {
        gk = (uint64_t *)tmp;
        gi = (uint32_t *)(gk + (size_t)std::min(ncont, kPresortBatch) * n2);
    }
    const size_t smem = (size_t)kSortSmem * (sizeof(uint64_t) + sizeof(uint32_t));
    cudaFuncSetAttribute(k_presort<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_presort<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int c0 = 0; c0 < ncont; c0 += batch) {
        const int nblk = std::min(batch, ncont - c0);
        if (dtype == NAPG_F32) {
            count_launch();
            k_presort<float><<<nblk, 1024, smem, st>>>((const float *)X, S, W, contvars_dev, obs, perm, pos, nobs, tie,
                                                       gsw, gew, gk, gi, n2, c0);
        }
        else {
            count_launch();
            k_presort<double><<<nblk, 1024, smem, st>>>((const double *)X, S, W, contvars_dev, obs, perm, pos, nobs,
                                                        tie, gsw, gew, gk, gi, n2, c0);
        }
    }
}

// --------------------------------------------------------- rank machinery --

// Per column side of a pair, all in shared memory (W + 1 words each, so that
// position == nobs can be queried). The four values a rank needs from one word
// sit in one 16-byte record, read with a single shared-memory load:
//   R[w].x = B   co-observed bits of the word's 32 sorted positions
//   R[w].y = P   exclusive prefix popcount of B at the word
//   R[w].z = T   tie-group start bits
//   R[w].w = GS  the bound (position, then co-observed prefix) of the group open
//                across the word's start; GE[w] likewise at the word's end.
struct Side {
    uint4 *R;
    int32_t *GE;
    int32_t n;       // observed count of the column
};

__device__ __forceinline__ int32_t prefix_at(const Side &sd, int32_t x) {
    const int w = x >> 5, l = x & 31;
    const uint4 r = sd.R[w];
    return (int32_t)r.y + __popc(r.x & ((1u << l) - 1u));
}

// Doubled rank 2R = P(gs) + P(ge) + 1 of the position at bit l of word w, from
// that word's tie-start bits Tw, co-observed bits Bw and prefix Pw; pgs / pge are
// P at the bounds of the group open across the word's start / end (the side's
// GS / GE after bounds_to_prefix). Below 2^31 for any S.
// group_bounds gives P(gs) and P(ge) themselves: the co-observed tie-group size
// is their difference.
__device__ __forceinline__ void group_bounds(uint32_t Tw, uint32_t Bw, int32_t Pw, int32_t pgs, int32_t pge, int l,
                                             int32_t &lo, int32_t &hi) {
    const uint32_t le = (l == 31) ? 0xffffffffu : ((2u << l) - 1u);
    const uint32_t m_le = Tw & le, m_gt = Tw & ~le;
    lo = m_le ? Pw + __popc(Bw & ((1u << (31 - __clz(m_le))) - 1u)) : pgs;
    hi = m_gt ? Pw + __popc(Bw & ((1u << (__ffs(m_gt) - 1)) - 1u)) : pge;
}

__device__ __forceinline__ uint32_t rank2_word(uint32_t Tw, uint32_t Bw, int32_t Pw, int32_t pgs, int32_t pge,
                                               int l) {
    int32_t lo, hi;
    group_bounds(Tw, Bw, Pw, pgs, pge, l, lo, hi);
    return (uint32_t)(lo + hi + 1);
}

__device__ __forceinline__ uint32_t rank2_at(const Side &sd, int32_t p) {
    const int w = p >> 5;
    const uint4 r = sd.R[w];
    return rank2_word(r.z, r.x, (int32_t)r.y, (int32_t)r.w, sd.GE[w], p & 31);
}

// Build B over the column's sorted positions from the co-observed sample bits,
// then the exclusive word prefix P; with lab_s, also gather the labels la[perm[p]]
// of the co-observed positions into lab_s[p]. Every thread of the block must call it.
__device__ void build_side(Side &sd, const int32_t *__restrict__ perm, const uint32_t *co, int W, int32_t *scan_tmp,
                           const uint8_t *__restrict__ la = nullptr, uint8_t *lab_s = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nw = (sd.n + 31) >> 5;
    for (int w = warp; w <= W; w += nwarps) {
        if (w >= nw) {                          // past the column's observed positions (warp-uniform)
            if (lane == 0) sd.R[w].x = 0u;
            continue;
        }
        const int p = w * 32 + lane;
        bool b = false;
        if (p < sd.n) {
            const int s = perm[p];
            b = (co[s >> 5] >> (s & 31)) & 1u;
            // the label of a co-observed position, in sorted order (others are never read)
            if (lab_s && b) lab_s[p] = la[s];
        }
        const uint32_t bits = __ballot_sync(0xffffffffu, b);
        if (lane == 0) sd.R[w].x = bits;
    }
    __syncthreads();
    // exclusive scan of popc(B[w]) over w = 0..W (W+1 entries), block-wide:
    // per-thread chunks, then a warp-shuffle scan of the chunk totals with one
    // total per warp carried through shared memory
    const int per = (W + 1 + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * per, w1 = min(W + 1, w0 + per);
    int c = 0;
    for (int w = w0; w < w1; ++w) c += __popc(sd.R[w].x);
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) scan_tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int t = lane < nwarps ? scan_tmp[lane] : 0;
        int ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < nwarps) scan_tmp[32 + lane] = ti - t;    // exclusive offset of each warp
    }
    __syncthreads();
    int run = scan_tmp[32 + warp] + incl - c;
    for (int w = w0; w < w1; ++w) { sd.R[w].y = (uint32_t)run; run += __popc(sd.R[w].x); }
    __syncthreads();
    // group bounds (positions) -> co-observed prefix counts at them, in place
    for (int w = threadIdx.x; w <= W; w += blockDim.x) {
        sd.R[w].w = (uint32_t)prefix_at(sd, (int32_t)sd.R[w].w);
        sd.GE[w] = prefix_at(sd, sd.GE[w]);
    }
    __syncthreads();
}

__device__ void load_side_static(Side &sd, const RankData &rd, int crow, int W) {
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        sd.R[w].z = rd.tie[(int64_t)crow * rd.W + w];
        sd.R[w].w = (uint32_t)rd.gsw[(int64_t)crow * rd.W + w];
        sd.GE[w] = rd.gew[(int64_t)crow * rd.W + w];
    }
    if (threadIdx.x == 0) { sd.R[W].z = 0u; sd.R[W].w = 0u; sd.GE[W] = 0; }
    sd.n = rd.nobs[crow];
}

__device__ __forceinline__ int64_t block_sum64(int64_t v, int64_t *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int64_t tot = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    return tot;   // valid in thread 0
}

// smem per side: R[W+1] uint4 (carved where cur is 16-byte aligned: the kernels
// carve every side's records first), GE[W+1] i32
__device__ __forceinline__ void carve_records(Side &sd, unsigned char *&cur, int W) {
    sd.R = (uint4 *)cur;
    cur += (W + 1) * 16;
    sd.n = 0;
}

__device__ __forceinline__ void carve_bounds(Side &sd, unsigned char *&cur, int W) {
    sd.GE = (int32_t *)cur;
    cur += (W + 1) * 4;
}

// ----------------------------------------------------------------- Spearman --
// One CTA per pair. out4[pair] = {n, sum A*B, sum A^2, sum B^2}, A = 2Rx, B = 2Ry.
__global__ void __launch_bounds__(1024, 2) k_spearman(RankData rd, const int32_t *__restrict__ crow_a,
                                                  const int32_t *__restrict__ crow_b, const uint32_t *__restrict__ obs_a,
                                                  const uint32_t *__restrict__ obs_b, int32_t na, int32_t nb,
                                                  int32_t symmetric, int64_t *__restrict__ out4,
                                                  const uint8_t *__restrict__ own) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t scan_tmp[64];
    __shared__ int64_t red4[32][4];
    const int W = (int)rd.W;
    // pair index
    int64_t pid = blockIdx.x;
    int a, b;
    if (symmetric) {
        // upper triangle including the diagonal, row-major: row i starts at
        // i (2 na - i + 1) / 2; closed form, then an exact integer fix-up
        const int64_t nv = na;
        int64_t i = (int64_t)((2.0 * nv + 1.0 - sqrt((2.0 * nv + 1.0) * (2.0 * nv + 1.0) - 8.0 * (double)pid)) / 2.0);
        if (i < 0) i = 0;
        if (i > nv - 1) i = nv - 1;
        while (i > 0 && i * (2 * nv - i + 1) / 2 > pid) --i;
        while ((i + 1) * (2 * nv - i) / 2 <= pid) ++i;
        a = (int)i; b = (int)(i + (pid - i * (2 * nv - i + 1) / 2));
    } else {
        a = (int)(pid / nb); b = (int)(pid - (int64_t)a * nb);
    }
    if (symmetric && own && !own[a]) return;    // another part's row (the whole CTA)
    unsigned char *cur = smem_raw;
    Side si, sj;
    carve_records(si, cur, W);
    carve_records(sj, cur, W);
    carve_bounds(si, cur, W);
    carve_bounds(sj, cur, W);
    uint32_t *co = (uint32_t *)cur; cur += (W + 1) * 4;
    const uint32_t *oa = obs_a + (int64_t)a * W, *ob = obs_b + (int64_t)b * W;
    for (int w = threadIdx.x; w < W; w += blockDim.x) co[w] = oa[w] & ob[w];
    const int ci = crow_a[a], cj = crow_b[b];
    load_side_static(si, rd, ci, W);
    load_side_static(sj, rd, cj, W);
    __syncthreads();
    const int32_t *perm_i = rd.perm + (int64_t)ci * rd.S, *perm_j = rd.perm + (int64_t)cj * rd.S;
    const int32_t *pos_j = rd.pos + (int64_t)cj * rd.S;
    build_side(si, perm_i, co, W, scan_tmp);
    build_side(sj, perm_j, co, W, scan_tmp);
    uint64_t sab = 0, saa = 0, sbb = 0;
    int32_t cnt = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // each warp takes one word of 32 sorted positions of column i at a time
    for (int w = warp; w < ((si.n + 31) >> 5); w += nwarps) {
        const uint4 r = si.R[w];
        const uint32_t Bw = r.x;
        if (Bw == 0u) continue;
        const uint32_t Tw = r.z;
        const int32_t Pw = (int32_t)r.y, pgs = (int32_t)r.w, pge = si.GE[w];
        if ((Bw >> lane) & 1u) {
            const int s = perm_i[w * 32 + lane];
            const int q = pos_j[s];
            const uint32_t A = rank2_word(Tw, Bw, Pw, pgs, pge, lane), B = rank2_at(sj, q);
            // 32 x 32 -> 64-bit products (exact)
            sab += (uint64_t)A * B; saa += (uint64_t)A * A; sbb += (uint64_t)B * B; ++cnt;
        }
    }
    // the four sums over the block: shuffles within each warp, one total per warp
    // through shared memory, then warp 0 (lane k of the result holds sum k)
    int64_t v4[4] = {cnt, (int64_t)sab, (int64_t)saa, (int64_t)sbb};
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) v4[k] += __shfl_down_sync(0xffffffffu, v4[k], o);
    if (lane == 0)
        for (int k = 0; k < 4; ++k) red4[warp][k] = v4[k];
    __syncthreads();
    if (warp == 0) {
        int64_t t[4];
        for (int k = 0; k < 4; ++k) {
            t[k] = lane < nwarps ? red4[lane][k] : 0;
            for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_down_sync(0xffffffffu, t[k], o);
        }
        if (lane == 0) {
            int64_t *o = out4 + 4 * ((int64_t)a * nb + b);
            o[0] = t[0]; o[1] = t[1]; o[2] = t[2]; o[3] = t[3];
        }
    }
}

static size_t rank_smem_bytes(int64_t W, int sides, bool with_co) {
    return (size_t)(W + 1) * 4 * (5 * sides + (with_co ? 1 : 0));
}

// Threads per pair: the per-pair arrays grow with S; once fewer than four
// 256-thread CTAs fit in an SM's shared memory, one 1024-thread CTA per pair
// keeps 32 warps resident instead.
static int rank_threads(size_t smem) { return smem > (size_t)56 * 1024 ? 1024 : 256; }

// Dynamic shared memory a rank CTA may take (below the 227 KB opt-in limit, with
// room for the static scan buffers).
constexpr size_t kRankSmemCap = 210 * 1024;

int rank_threads_default(int64_t W, bool groups) { return rank_threads(rank_smem_bytes(W, groups ? 1 : 2, true)); }

void launch_spearman_pairs(const RankData &rd, const int32_t *crow_a, const int32_t *crow_b, const uint32_t *obs_a,
                           const uint32_t *obs_b, int32_t na, int32_t nb, int32_t symmetric, int64_t *out4,
                           cudaStream_t st, int threads, const uint8_t *own) {
    const int64_t pairs = symmetric ? (int64_t)na * (na + 1) / 2 : (int64_t)na * nb;
    if (pairs == 0) return;
    const size_t smem = rank_smem_bytes(rd.W, 2, true);
    cudaFuncSetAttribute(k_spearman, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    k_spearman<<<(unsigned)pairs, threads > 0 ? threads : rank_threads(smem), smem, st>>>(
        rd, crow_a, crow_b, obs_a, obs_b, na, nb, symmetric, out4, own);
}

// ------------------------------------------------------------ MWU / Kruskal --
// One CTA per (categorical a, continuous j): per level g the count n_g and the
// sum of doubled ranks S_g, plus the tie term sum (t^3 - t) over co-observed
// tie groups. The walk visits j's sorted positions a word (32 positions) per warp
// at a time. With CMAX levels at most (2, 4 or 8), every lane adds into its own
// slot per level, (1 << 40) + 2R as one 64-bit word (sum in the low 40 bits,
// count above: the totals stay below 2^40 and 2^24 for any S the rank tests
// take), and the slots are summed at the end. With CMAX = 0 (up to kMaxLevels
// levels) lanes of one level are grouped by match_any and their leader adds
// into the warp's table. SLAB: the labels are gathered into shared memory in
// sorted order while the co-observed bits are built (otherwise the walk reads
// them from the cohort). P32: the slots are 32-bit words, (1 << 24) + 2R, when a
// lane's totals provably fit (rank_groups_pack32: a lane sees at most m < 256
// positions, and m (2S + 1) < 2^24), which halves the tables.
constexpr int kPackShift = 40, kPackShift32 = 24;

static_assert(kMaxLevels * 12 % 16 == 0, "the level tables keep the records after them 16-byte aligned");

template <int CMAX, bool P32 = false>
__host__ __device__ constexpr size_t rank_group_table_bytes(int nwarp) {
    return CMAX ? (size_t)nwarp * CMAX * 32 * (P32 ? 4 : 8) : (size_t)nwarp * kMaxLevels * 12;
}

// whether every lane's per-level count and doubled-rank sum fit the 32-bit slot:
// a lane sees at most ceil(W / nwarp) positions, each 2R <= 2S + 1
static bool rank_groups_pack32(int64_t S, int64_t W, int nwarp) {
    const int64_t per_lane = (W + nwarp - 1) / nwarp;
    return per_lane < (1 << (32 - kPackShift32)) && per_lane * (2 * S + 1) < ((int64_t)1 << kPackShift32);
}

template <int CMAX, bool SLAB, bool P32>
__global__ void __launch_bounds__(1024, SLAB ? 2 : 1) k_rank_groups(RankData rd, const uint8_t *__restrict__ lab,
                                                     const int32_t *__restrict__ catrow_a, const int32_t *__restrict__ nlev_a,
                                                     const int32_t *__restrict__ levoff_a, int32_t na,
                                                     const int32_t *__restrict__ crow_b, const uint32_t *__restrict__ obs_a,
                                                     const uint32_t *__restrict__ obs_b, int32_t nb, int64_t *__restrict__ rsum,
                                                     int32_t *__restrict__ rcnt, int64_t *__restrict__ tie_term) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t scan_tmp[64];
    __shared__ int64_t red[32];
    const int W = (int)rd.W;
    const int a = (int)(blockIdx.x / nb), j = (int)(blockIdx.x - (int64_t)a * nb);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    unsigned char *cur = smem_raw;
    // CMAX > 0: acc[(warp * CMAX + g) * 32 + lane]; CMAX = 0: lsum / lcnt[warp * kMaxLevels + g]
    using Acc = typename std::conditional<P32, uint32_t, unsigned long long>::type;
    constexpr int kShift = P32 ? kPackShift32 : kPackShift;
    Acc *acc = (Acc *)cur;
    unsigned long long *lsum = (unsigned long long *)cur;
    int *lcnt = (int *)(cur + (size_t)nwarp * kMaxLevels * 8);
    cur += rank_group_table_bytes<CMAX, P32>(nwarp);      // a multiple of 16 bytes
    Side sj;
    carve_records(sj, cur, W);
    carve_bounds(sj, cur, W);
    uint32_t *co = (uint32_t *)cur; cur += (W + 1) * 4;
    uint8_t *lab_s = SLAB ? (uint8_t *)cur : nullptr;   // (W + 1) * 32 bytes
    const uint32_t *oa = obs_a + (int64_t)a * W, *ob = obs_b + (int64_t)j * W;
    for (int w = threadIdx.x; w < W; w += blockDim.x) co[w] = oa[w] & ob[w];
    const int cj = crow_b[j];
    load_side_static(sj, rd, cj, W);
    const int c = nlev_a[a];
    if (CMAX) {
        for (int i = threadIdx.x; i < nwarp * CMAX * 32; i += blockDim.x) acc[i] = 0;
    } else {
        for (int i = threadIdx.x; i < nwarp * kMaxLevels; i += blockDim.x) {
            lsum[i] = 0ull;
            lcnt[i] = 0;
        }
    }
    __syncthreads();
    const int32_t *perm_j = rd.perm + (int64_t)cj * rd.S;
    const uint8_t *la = lab + (int64_t)catrow_a[a] * rd.S;
    build_side(sj, perm_j, co, W, scan_tmp, SLAB ? la : nullptr, lab_s);
    int64_t tsum = 0;
    const int nwj = (sj.n + 31) >> 5;
#pragma unroll 1
    for (int w0 = 0; w0 < nwj; w0 += nwarp) {
        const int w = w0 + warp;               // warps past the end still join the warp-wide steps
        const bool inw = w < nwj;
        const uint4 r = inw ? sj.R[w] : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t Bw = r.x, Tw = r.z;
        const int32_t Pw = (int32_t)r.y, pgs = (int32_t)r.w, pge = inw ? sj.GE[w] : 0;
        const int p = w * 32 + lane;
        const bool on = inw && ((Bw >> lane) & 1u);
        int g = kMaxLevels;                    // no level
        uint32_t r2 = 0;
        if (on) {
            g = SLAB ? lab_s[p] : la[perm_j[p]];
            int32_t lo, hi;
            group_bounds(Tw, Bw, Pw, pgs, pge, lane, lo, hi);
            r2 = (uint32_t)(lo + hi + 1);
            // sum of (t^3 - t) over co-observed tie groups = sum of (t^2 - 1) over
            // their co-observed members, t = P(ge) - P(gs)
            const int64_t t = hi - lo;
            tsum += t * t - 1;
        }
        if (CMAX) {
            if (on) acc[(warp * CMAX + g) * 32 + lane] += ((Acc)1 << kShift) + r2;
        } else {
            // lanes with the same level add their doubled ranks (a warp's sum fits 32 bits)
            const unsigned same = __match_any_sync(0xffffffffu, g);
            const uint32_t sum = __reduce_add_sync(same, r2);
            if (on && lane == __ffs(same) - 1) {
                lsum[warp * kMaxLevels + g] += sum;   // distinct levels per leader: no conflict
                lcnt[warp * kMaxLevels + g] += __popc(same);
            }
        }
    }
    const int64_t T = block_sum64(tsum, red);   // has barriers: the tables are complete after it
    __syncthreads();
    const int off = levoff_a[a];
    if (CMAX) {
        // warp g sums level g over warps (per lane), then over lanes
        if (warp < c) {
            unsigned long long v = 0;
            for (int k = 0; k < nwarp; ++k) {
                const Acc e = acc[(k * CMAX + warp) * 32 + lane];
                v += P32 ? (((unsigned long long)(e >> kShift) << kPackShift) + (e & (((Acc)1 << kShift) - 1)))
                         : (unsigned long long)e;
            }
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) {
                rsum[(int64_t)(off + warp) * nb + j] = (int64_t)(v & ((1ull << kPackShift) - 1ull));
                rcnt[(int64_t)(off + warp) * nb + j] = (int32_t)(v >> kPackShift);
            }
        }
    } else {
        for (int g2 = threadIdx.x; g2 < c; g2 += blockDim.x) {
            unsigned long long su = 0;
            int cn = 0;
            for (int k = 0; k < nwarp; ++k) { su += lsum[k * kMaxLevels + g2]; cn += lcnt[k * kMaxLevels + g2]; }
            rsum[(int64_t)(off + g2) * nb + j] = (int64_t)su;
            rcnt[(int64_t)(off + g2) * nb + j] = cn;
        }
    }
    if (threadIdx.x == 0) tie_term[(int64_t)a * nb + j] = T;
}

template <int CMAX, bool SLAB, bool P32>
static void launch_rank_groups_t(const RankData &rd, const uint8_t *lab, const int32_t *catrow_a,
                                 const int32_t *nlev_a, const int32_t *levoff_a, int32_t na, const int32_t *crow_b,
                                 const uint32_t *obs_a, const uint32_t *obs_b, int32_t nb, int64_t *rsum,
                                 int32_t *rcnt, int64_t *tie_term, int threads, size_t smem, cudaStream_t st) {
    auto kern = k_rank_groups<CMAX, SLAB, P32>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    count_launch();
    kern<<<(unsigned)((int64_t)na * nb), threads, smem, st>>>(rd, lab, catrow_a, nlev_a, levoff_a, na, crow_b, obs_a,
                                                              obs_b, nb, rsum, rcnt, tie_term);
}

void launch_rank_groups(const RankData &rd, const uint8_t *lab, const int32_t *catrow_a, const int32_t *nlev_a,
                        const int32_t *levoff_a, int32_t na, const int32_t *crow_b, const uint32_t *obs_a,
                        const uint32_t *obs_b, int32_t nb, int32_t max_levels, int64_t *rsum, int32_t *rcnt,
                        int64_t *tie_term, cudaStream_t st, int threads_req) {
    const int64_t pairs = (int64_t)na * nb;
    if (pairs == 0) return;
    const size_t side = rank_smem_bytes(rd.W, 1, true);
    const int threads = threads_req > 0 ? threads_req : rank_threads(side);
    const int cmax = max_levels <= 2 ? 2 : max_levels <= 4 ? 4 : max_levels <= 8 ? 8 : 0;
    const int nwarp = threads / 32;
    const size_t labs = (size_t)(rd.W + 1) * 32;
    // per-lane slots (cmax > 0): 32-bit when the totals fit and the labels can be staged
    const size_t tables64 = cmax ? (size_t)nwarp * cmax * 32 * 8 : rank_group_table_bytes<0>(nwarp);
    const bool p32 = cmax > 0 && rank_groups_pack32(rd.S, rd.W, nwarp) && side + tables64 / 2 + labs <= kRankSmemCap;
    const size_t tables = p32 ? tables64 / 2 : tables64;
    const bool slab = side + tables + labs <= kRankSmemCap;
    const size_t smem = side + tables + (slab ? labs : 0);
#define NAPG_RG_ARGS rd, lab, catrow_a, nlev_a, levoff_a, na, crow_b, obs_a, obs_b, nb, rsum, rcnt, tie_term, threads, smem, st
#define NAPG_RG(C)                                                                                                  \
    (p32 ? launch_rank_groups_t<C, true, true>(NAPG_RG_ARGS)                                                        \
         : slab ? launch_rank_groups_t<C, true, false>(NAPG_RG_ARGS) : launch_rank_groups_t<C, false, false>(NAPG_RG_ARGS))
    switch (cmax) {
        case 2: NAPG_RG(2); break;
        case 4: NAPG_RG(4); break;
        case 8: NAPG_RG(8); break;
        default:
            if (slab) launch_rank_groups_t<0, true, false>(NAPG_RG_ARGS);
            else launch_rank_groups_t<0, false, false>(NAPG_RG_ARGS);
            break;
    }
#undef NAPG_RG
#undef NAPG_RG_ARGS
}

// ------------------------------------------------------ exact Mann-Whitney --
// Null distribution of U for group sizes (m, n), m <= n: the coefficients of the
// Gaussian binomial [m+n choose m]_q = prod_{k=1..m} (1 - q^{n+k}) / (1 - q^k)
// count the arrangements with U = u. Built one factor at a time in exact
// 128-bit integers, truncated at the degree needed; then
// p = min(1, 2 P(U <= min(U0, U1))).
typedef unsigned __int128 u128;

__global__ void k_mwu_exact(const double *__restrict__ stat, const int32_t *__restrict__ rcnt,
                            const int32_t *__restrict__ levoff, int32_t nb, const int32_t *__restrict__ flags,
                            const int32_t *__restrict__ nflag, int32_t max_flags, double *__restrict__ pval,
                            u128 *__restrict__ scratch, int64_t cap, uint32_t *__restrict__ err) {
    const int32_t cnt = min(*nflag, max_flags);
    u128 *G = scratch + (int64_t)blockIdx.x * 2 * cap;
    u128 *H = G + cap;
    __shared__ double s_p;
    for (int q = blockIdx.x; q < cnt; q += gridDim.x) {
        const int64_t t = flags[q];
        const int a = (int)(t / nb), j = (int)(t - (int64_t)a * nb);
        const int64_t n0 = rcnt[(int64_t)levoff[a] * nb + j], n1 = rcnt[(int64_t)(levoff[a] + 1) * nb + j];
        const int64_t m = n0 < n1 ? n0 : n1, n = n0 < n1 ? n1 : n0;
        const double U0 = stat[t];
        const double umin_d = fmin(U0, (double)(n0 * n1) - U0);
        const int64_t ulim = (int64_t)floor(umin_d);
        // total = C(m+n, m) exactly; 127-bit overflow guard via lgamma
        const double log2_total = (lgamma((double)(m + n + 1)) - lgamma((double)(m + 1)) - lgamma((double)(n + 1))) /
                                  0.69314718055994530942;
        if (threadIdx.x == 0) s_p = __longlong_as_double(0x7ff8000000000000LL);
        __syncthreads();
        if (ulim + 1 <= cap && log2_total < 126.0 && m <= 64) {
            for (int64_t u = threadIdx.x; u <= ulim; u += blockDim.x) G[u] = (u == 0) ? 1 : 0;
            __syncthreads();
            for (int64_t k = 1; k <= m; ++k) {
                // H = G * (1 - q^{n+k}) (truncated)
                for (int64_t u = threadIdx.x; u <= ulim; u += blockDim.x)
                    H[u] = G[u] - ((u >= n + k) ? G[u - n - k] : (u128)0);
                __syncthreads();
                // G = H / (1 - q^k): prefix sums with stride k, one residue class per thread
                for (int64_t r = threadIdx.x; r < k; r += blockDim.x) {
                    u128 run = 0;
                    for (int64_t u = r; u <= ulim; u += k) { run += H[u]; G[u] = run; }
                }
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                u128 cdf = 0;
                for (int64_t u = 0; u <= ulim; ++u) cdf += G[u];
                u128 total = 1;
                for (int64_t k = 1; k <= m; ++k) total = total * (u128)(n + k) / (u128)k;
                const double pv = 2.0 * ((double)cdf / (double)total);
                s_p = pv > 1.0 ? 1.0 : pv;
            }
        }
        __syncthreads();
        // beyond the exact range the p-value stays NaN and the call reports it
        if (threadIdx.x == 0 && isnan(s_p)) atomicOr(err, kErrExactLimit);
        if (threadIdx.x == 0) pval[t] = s_p;
        __syncthreads();
    }
}

size_t mwu_exact_scratch_bytes(int64_t S, bool forced) {
    // blocks x 2 arrays x (7 S / 2 + 2) entries covers auto mode (min group < 8);
    // forced exact mode: the whole range min(U0, U1) <= S^2 / 8 where that stays
    // within 65,536 entries per array (64 MiB in all), else 7 S / 2 + 2
    int64_t cap = 7 * S / 2 + 2;
    if (forced) cap = std::min<int64_t>(S * S / 8 + 2, std::max<int64_t>(cap, (int64_t)1 << 16));
    return (size_t)32 * 2 * (size_t)cap * sizeof(u128);
}

void launch_mwu_exact(const double *stat, const int32_t *rcnt, const int32_t *levoff, int32_t total_rows, int32_t nb,
                      const int32_t *flag_list, const int32_t *flag_count, int32_t max_flags, double *pval,
                      void *scratch, size_t scratch_bytes, uint32_t *err, cudaStream_t st) {
    (void)total_rows;
    const int64_t cap = (int64_t)(scratch_bytes / (32 * 2 * sizeof(u128)));
    count_launch();
    k_mwu_exact<<<32, 128, 0, st>>>(stat, rcnt, levoff, nb, flag_list, flag_count, max_flags, pval, (u128 *)scratch,
                                    cap, err);
}

}  // namespace napg
