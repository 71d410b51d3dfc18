// Plain FP64 moment contractions on the CUDA cores (the NAPG_FP64_PLAIN form).
//
// Pearson (Sec. 3.5.2): for every pair (i, j) of shifted columns
// x~_i = (x_i - c_i) m_i (zero where unobserved),
//   n_ij = sum m_i m_j,  Sx_ij = sum x~_i m_j,  Sxx_ij = sum x~_i^2 m_j,
//   Sxy_ij = sum x~_i x~_j,
// with Sy_ij = Sx_ji and Syy_ij = Sxx_ji. Tiles with I <= J cover all pairs.
//
// Group sums (Sec. 3.5.5, 3.5.7): for a categorical a and continuous j, per
// level g: n_g = #{co-observed with label g}, S1_g = sum x~_j, S2_g = sum x~_j^2.
#include "napg_internal.cuh"

namespace napg {

constexpr int kPT = 32;   // output tile edge (pairs)
constexpr int kPK = 32;   // samples per stage (one bit word)

__global__ void __launch_bounds__(256) k_pearson_fp64(const double *__restrict__ xs, int64_t S_pad,
                                                      const uint32_t *__restrict__ obsv, int64_t W, int32_t nv,
                                                      double *__restrict__ Sxy, double *__restrict__ Sx,
                                                      double *__restrict__ Sxx, int32_t *__restrict__ nn) {
    // blockIdx.x enumerates upper-triangle tiles (I <= J)
    const int T = (nv + kPT - 1) / kPT;
    int t = blockIdx.x, I = 0;
    while (t >= T - I) { t -= T - I; ++I; }
    const int J = I + t;
    __shared__ double xa[kPT][kPK + 1], xb[kPT][kPK + 1];
    __shared__ uint32_t wa[kPT], wb[kPT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double sxy[2][2] = {}, sx[2][2] = {}, sy[2][2] = {}, sxx[2][2] = {}, syy[2][2] = {};
    int cnt[2][2] = {};
    const int i0 = I * kPT, j0 = J * kPT;
    for (int64_t k0 = 0; k0 < S_pad; k0 += kPK) {
        for (int e = threadIdx.x; e < kPT * kPK; e += 256) {
            const int r = e / kPK, c = e % kPK;
            const int gi = i0 + r, gj = j0 + r;
            xa[r][c] = gi < nv ? xs[(int64_t)gi * S_pad + k0 + c] : 0.0;
            xb[r][c] = gj < nv ? xs[(int64_t)gj * S_pad + k0 + c] : 0.0;
        }
        if (threadIdx.x < kPT) {
            const int gi = i0 + threadIdx.x, gj = j0 + threadIdx.x;
            const int64_t w = k0 >> 5;
            wa[threadIdx.x] = (gi < nv && w < W) ? obsv[(int64_t)gi * W + w] : 0u;
            wb[threadIdx.x] = (gj < nv && w < W) ? obsv[(int64_t)gj * W + w] : 0u;
        }
        __syncthreads();
        uint32_t mi[2], mj[2];
        for (int a = 0; a < 2; ++a) mi[a] = wa[ty + 16 * a];
        for (int b = 0; b < 2; ++b) mj[b] = wb[tx + 16 * b];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) cnt[a][b] += __popc(mi[a] & mj[b]);
#pragma unroll 4
        for (int k = 0; k < kPK; ++k) {
            double xi[2], xj[2], x2i[2], x2j[2];
            bool oi[2], oj[2];
            for (int a = 0; a < 2; ++a) {
                xi[a] = xa[ty + 16 * a][k];
                x2i[a] = xi[a] * xi[a];
                oi[a] = (mi[a] >> k) & 1u;
            }
            for (int b = 0; b < 2; ++b) {
                xj[b] = xb[tx + 16 * b][k];
                x2j[b] = xj[b] * xj[b];
                oj[b] = (mj[b] >> k) & 1u;
            }
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    sxy[a][b] = fma(xi[a], xj[b], sxy[a][b]);
                    sx[a][b] += oj[b] ? xi[a] : 0.0;
                    sxx[a][b] += oj[b] ? x2i[a] : 0.0;
                    sy[a][b] += oi[a] ? xj[b] : 0.0;
                    syy[a][b] += oi[a] ? x2j[b] : 0.0;
                }
        }
        __syncthreads();
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            if (i >= nv || j >= nv) continue;
            const int64_t ij = (int64_t)i * nv + j, ji = (int64_t)j * nv + i;
            Sxy[ij] = sxy[a][b];
            Sx[ij] = sx[a][b];
            Sxx[ij] = sxx[a][b];
            nn[ij] = cnt[a][b];
            if (I != J) {
                Sx[ji] = sy[a][b];
                Sxx[ji] = syy[a][b];
            } else if (i != j) {
                // diagonal tile: thread (i, j) and thread (j, i) both exist; each
                // writes its own (row, column) entry only
            }
        }
}

void launch_pearson_fp64(const double *xs, int64_t S_pad, const uint32_t *obsv, int64_t W, int32_t nv,
                         double *Sxy, double *Sx, double *Sxx, int32_t *nn, cudaStream_t st) {
    if (nv == 0) return;
    const int T = (nv + kPT - 1) / kPT;
    const int tiles = T * (T + 1) / 2;
    count_launch();
    k_pearson_fp64<<<tiles, 256, 0, st>>>(xs, S_pad, obsv, W, nv, Sxy, Sx, Sxx, nn);
}

// One warp per (categorical a, continuous j): lanes stride over samples and keep
// per-level sums in registers (MAXC levels), then reduce across the warp.
template <int MAXC>
__global__ void __launch_bounds__(256) k_groupsum_fp64(
    const uint8_t *__restrict__ lab, int64_t S, const int32_t *__restrict__ catrow, int32_t na,
    const int32_t *__restrict__ levoff, const int32_t *__restrict__ nlev, const double *__restrict__ xs,
    int64_t S_pad, const uint32_t *__restrict__ obsb, int64_t W, int32_t nb, int32_t *__restrict__ gn,
    double *__restrict__ g1, double *__restrict__ g2) {
    const int lane = threadIdx.x & 31;
    const int64_t pair = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pair >= (int64_t)na * nb) return;
    const int a = (int)(pair / nb), j = (int)(pair - (int64_t)a * nb);
    const uint8_t *la = lab + (int64_t)catrow[a] * S;
    const double *xj = xs + (int64_t)j * S_pad;
    const uint32_t *ob = obsb + (int64_t)j * W;
    int c_n[MAXC];
    double c_1[MAXC], c_2[MAXC];
#pragma unroll
    for (int g = 0; g < MAXC; ++g) { c_n[g] = 0; c_1[g] = 0.0; c_2[g] = 0.0; }
    for (int64_t s = lane; s < S; s += 32) {
        const int l = la[s];
        const bool o = (ob[s >> 5] >> (s & 31)) & 1u;
        if (!o || l == kMissingLabel) continue;
        const double v = xj[s];
#pragma unroll
        for (int g = 0; g < MAXC; ++g) {
            if (l == g) { c_n[g] += 1; c_1[g] += v; c_2[g] = fma(v, v, c_2[g]); }
        }
    }
    const int c = nlev[a], off = levoff[a];
#pragma unroll
    for (int g = 0; g < MAXC; ++g) {
        if (g >= c) break;
        int nsum = c_n[g];
        double s1 = c_1[g], s2 = c_2[g];
        for (int o = 16; o > 0; o >>= 1) {
            nsum += __shfl_down_sync(0xffffffffu, nsum, o);
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
            s2 += __shfl_down_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            const int64_t idx = (int64_t)(off + g) * nb + j;
            gn[idx] = nsum;
            g1[idx] = s1;
            g2[idx] = s2;
        }
    }
}

void launch_groupsum_fp64(const uint8_t *lab, int64_t S, const int32_t *catrow_dev, int32_t na,
                          const int32_t *levoff_dev, const int32_t *nlev_dev, const double *xs,
                          int64_t S_pad, const uint32_t *obsb, int64_t W, int32_t nb,
                          int32_t *gn, double *g1, double *g2, int32_t max_levels, cudaStream_t st) {
    const int64_t pairs = (int64_t)na * nb;
    if (pairs == 0) return;
    const unsigned blocks = (unsigned)((pairs + 7) / 8);
    if (max_levels <= 4) {
        count_launch();
        k_groupsum_fp64<4><<<blocks, 256, 0, st>>>(lab, S, catrow_dev, na, levoff_dev, nlev_dev, xs, S_pad, obsb,
                                                   W, nb, gn, g1, g2);
    }
    else if (max_levels <= 10) {
        count_launch();
        k_groupsum_fp64<10><<<blocks, 256, 0, st>>>(lab, S, catrow_dev, na, levoff_dev, nlev_dev, xs, S_pad, obsb,
                                                    W, nb, gn, g1, g2);
    }
    else if (max_levels <= 16) {
        count_launch();
        k_groupsum_fp64<16><<<blocks, 256, 0, st>>>(lab, S, catrow_dev, na, levoff_dev, nlev_dev, xs, S_pad, obsb,
                                                    W, nb, gn, g1, g2);
    }
    else {
        count_launch();
        k_groupsum_fp64<kMaxLevels><<<blocks, 256, 0, st>>>(lab, S, catrow_dev, na, levoff_dev, nlev_dev, xs,
                                                            S_pad, obsb, W, nb, gn, g1, g2);
    }
}

}  // namespace napg
