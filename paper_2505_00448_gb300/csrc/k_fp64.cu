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

#include <cooperative_groups.h>

#include <algorithm>

namespace napg {

constexpr int kPT = 32;   // output tile edge (pairs)
constexpr int kPK = 32;   // samples per stage (one bit word)
constexpr int kMaxSplit = 8;   // portable cluster size

namespace cg = cooperative_groups;

// One thread's 2 x 2 pairs: Sxy, Sx (row sums), Sxx, Sy (column sums), Syy.
struct PairAcc {
    double sxy[2][2], sx[2][2], sy[2][2], sxx[2][2], syy[2][2];
    int cnt[2][2];
};

__device__ __forceinline__ void write_pairs(const PairAcc &r, int I, int J, int tx, int ty, int32_t nv,
                                            double *__restrict__ Sxy, double *__restrict__ Sx,
                                            double *__restrict__ Sxx, int32_t *__restrict__ nn) {
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int i = I * kPT + ty + 16 * a, j = J * kPT + tx + 16 * b;
            if (i >= nv || j >= nv) continue;
            const int64_t ij = (int64_t)i * nv + j, ji = (int64_t)j * nv + i;
            Sxy[ij] = r.sxy[a][b];
            Sx[ij] = r.sx[a][b];
            Sxx[ij] = r.sxx[a][b];
            nn[ij] = r.cnt[a][b];
            // off-diagonal tiles also give the (j, i) column sums; on a diagonal
            // tile thread (j, i) writes its own row entry
            if (I != J) {
                Sx[ji] = r.sy[a][b];
                Sxx[ji] = r.syy[a][b];
            }
        }
}

// Tiles of the upper triangle (I <= J), 32 x 32 pairs, 256 threads with 2 x 2
// pairs each. With split > 1 the CTAs of one cluster share a tile: CTA r sums
// the sample words [r*nw/split, (r+1)*nw/split), then the partials are added in
// rank order through distributed shared memory, each CTA finishing an equal
// share of the tile's values, so the sum order depends only on the split.
__global__ void __launch_bounds__(256) k_pearson_fp64(const double *__restrict__ xs, int64_t S_pad,
                                                      const uint32_t *__restrict__ obsv, int64_t W, int32_t nv,
                                                      int split, double *__restrict__ Sxy,
                                                      double *__restrict__ Sx, double *__restrict__ Sxx,
                                                      int32_t *__restrict__ nn, const uint8_t *__restrict__ own) {
    const int T = (nv + kPT - 1) / kPT;
    int t = blockIdx.x / split, I = 0;
    const int rank = blockIdx.x - t * split;
    while (t >= T - I) { t -= T - I; ++I; }
    const int J = I + t;
    if (!rows_owned(own, (int64_t)I * kPT, kPT, nv)) return;    // another part's rows (every CTA of the tile)
    __shared__ union {
        struct { double xa[kPT][kPK + 1], xb[kPT][kPK + 1], qa[kPT][kPK + 1], qb[kPT][kPK + 1]; } st;
        double part[20][256];
    } u;
    __shared__ int cpart[4][256];
    __shared__ uint32_t wa[kPT], wb[kPT];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    PairAcc r = {};
    const int i0 = I * kPT, j0 = J * kPT;
    const int64_t nw = S_pad / kPK;
    const int64_t wbeg = nw * rank / split, wend = nw * (rank + 1) / split;
    for (int64_t w = wbeg; w < wend; ++w) {
        const int64_t k0 = w * kPK;
        for (int e = threadIdx.x; e < kPT * kPK; e += 256) {
            const int rr = e / kPK, c = e % kPK;
            const int gi = i0 + rr, gj = j0 + rr;
            const double va = gi < nv ? xs[(int64_t)gi * S_pad + k0 + c] : 0.0;
            const double vb = gj < nv ? xs[(int64_t)gj * S_pad + k0 + c] : 0.0;
            u.st.xa[rr][c] = va;
            u.st.xb[rr][c] = vb;
            u.st.qa[rr][c] = va * va;      // squares formed once per staged word
            u.st.qb[rr][c] = vb * vb;
        }
        if (threadIdx.x < kPT) {
            const int gi = i0 + threadIdx.x, gj = j0 + threadIdx.x;
            wa[threadIdx.x] = (gi < nv && w < W) ? obsv[(int64_t)gi * W + w] : 0u;
            wb[threadIdx.x] = (gj < nv && w < W) ? obsv[(int64_t)gj * W + w] : 0u;
        }
        __syncthreads();
        uint32_t mi[2], mj[2];
        for (int a = 0; a < 2; ++a) mi[a] = wa[ty + 16 * a];
        for (int b = 0; b < 2; ++b) mj[b] = wb[tx + 16 * b];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) r.cnt[a][b] += __popc(mi[a] & mj[b]);
#pragma unroll 4
        for (int k = 0; k < kPK; ++k) {
            double xi[2], xj[2], x2i[2], x2j[2];
            bool oi[2], oj[2];
            for (int a = 0; a < 2; ++a) {
                xi[a] = u.st.xa[ty + 16 * a][k];
                x2i[a] = u.st.qa[ty + 16 * a][k];
                oi[a] = (mi[a] >> k) & 1u;
            }
            for (int b = 0; b < 2; ++b) {
                xj[b] = u.st.xb[tx + 16 * b][k];
                x2j[b] = u.st.qb[tx + 16 * b][k];
                oj[b] = (mj[b] >> k) & 1u;
            }
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    r.sxy[a][b] = fma(xi[a], xj[b], r.sxy[a][b]);
                    r.sx[a][b] += oj[b] ? xi[a] : 0.0;
                    r.sxx[a][b] += oj[b] ? x2i[a] : 0.0;
                    r.sy[a][b] += oi[a] ? xj[b] : 0.0;
                    r.syy[a][b] += oi[a] ? x2j[b] : 0.0;
                }
        }
        __syncthreads();
    }
    if (split == 1) {
        write_pairs(r, I, J, tx, ty, nv, Sxy, Sx, Sxx, nn);
        return;
    }
    // partials of this CTA, [quantity][thread slot]: Sxy, Sx, Sxx, Sy, Syy as
    // quantities 4*kind + 2a + b, counts apart (the staging tiles are dead now:
    // the loop ended on a barrier)
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int q = 2 * a + b;
            u.part[q][threadIdx.x] = r.sxy[a][b];
            u.part[4 + q][threadIdx.x] = r.sx[a][b];
            u.part[8 + q][threadIdx.x] = r.sxx[a][b];
            u.part[12 + q][threadIdx.x] = r.sy[a][b];
            u.part[16 + q][threadIdx.x] = r.syy[a][b];
            cpart[q][threadIdx.x] = r.cnt[a][b];
        }
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    // the tile's 24 x 256 values (quantity, thread slot), dealt out in equal
    // contiguous ranges to the CTAs of the cluster; each value sums the ranks'
    // partials in rank order
    constexpr int kVals = 24 * 256;
    const int vbeg = kVals * rank / split, vend = kVals * (rank + 1) / split;
    for (int v = vbeg + (int)threadIdx.x; v < vend; v += 256) {
        const int qd = v >> 8, slot = v & 255;
        const int kind = qd >> 2, a = (qd >> 1) & 1, b = qd & 1;
        const int i = i0 + (slot >> 4) + 16 * a, j = j0 + (slot & 15) + 16 * b;
        double acc = 0.0;
        int cacc = 0;
        if (kind < 5) {
            for (int q = 0; q < split; ++q) acc += cluster.map_shared_rank(&u.part[qd][slot], q)[0];
        } else {
            for (int q = 0; q < split; ++q) cacc += cluster.map_shared_rank(&cpart[qd - 20][slot], q)[0];
        }
        if (i >= nv || j >= nv) continue;
        const int64_t ij = (int64_t)i * nv + j, ji = (int64_t)j * nv + i;
        switch (kind) {
            case 0: Sxy[ij] = acc; break;
            case 1: Sx[ij] = acc; break;
            case 2: Sxx[ij] = acc; break;
            case 3: if (I != J) Sx[ji] = acc; break;
            case 4: if (I != J) Sxx[ji] = acc; break;
            default: nn[ij] = cacc; break;
        }
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

// Split of the sample axis: enough CTAs for two per SM when the triangle has
// few tiles, at most one cluster of 8 and at least one sample word per CTA.
int pearson_fp64_split(int32_t nv, int64_t S_pad) {
    const int T = (nv + kPT - 1) / kPT;
    const int64_t tiles = (int64_t)T * (T + 1) / 2, nw = S_pad / kPK;
    int64_t k = (2 * 152 + tiles - 1) / std::max<int64_t>(tiles, 1);
    k = std::min<int64_t>(k, kMaxSplit);
    k = std::min<int64_t>(k, nw);
    return (int)std::max<int64_t>(k, 1);
}

void launch_pearson_fp64(const double *xs, int64_t S_pad, const uint32_t *obsv, int64_t W, int32_t nv,
                         double *Sxy, double *Sx, double *Sxx, int32_t *nn, cudaStream_t st, const uint8_t *own) {
    if (nv == 0) return;
    const int T = (nv + kPT - 1) / kPT;
    const int tiles = T * (T + 1) / 2;
    const int split = pearson_fp64_split(nv, S_pad);
    count_launch();
    if (split == 1) {
        k_pearson_fp64<<<tiles, 256, 0, st>>>(xs, S_pad, obsv, W, nv, 1, Sxy, Sx, Sxx, nn, own);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(tiles * split));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)split;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_pearson_fp64, xs, S_pad, obsv, W, nv, split, Sxy, Sx, Sxx, nn, own);
}

// One warp per (categorical a, continuous j): lane l takes samples l, l+32, ...
// and adds each into its level's running sums, kept per lane in shared memory
// ([level][lane]), so one sample costs two FP64 operations whatever the level
// count; then the lanes are reduced by a shuffle tree per level.
template <int MAXC>
__global__ void __launch_bounds__(256) k_groupsum_fp64(
    const uint8_t *__restrict__ lab, int64_t S, const int32_t *__restrict__ catrow, int32_t na,
    const int32_t *__restrict__ levoff, const int32_t *__restrict__ nlev, const double *__restrict__ xs,
    int64_t S_pad, const uint32_t *__restrict__ obsb, int64_t W, int32_t nb, int32_t *__restrict__ gn,
    double *__restrict__ g1, double *__restrict__ g2) {
    extern __shared__ double gs_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *c1 = gs_smem + (int64_t)warp * MAXC * 32 * 2, *c2 = c1 + MAXC * 32;
    int *cn = reinterpret_cast<int *>(gs_smem + (int64_t)(blockDim.x >> 5) * MAXC * 32 * 2) + warp * MAXC * 32;
    const int64_t pair = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (pair >= (int64_t)na * nb) return;
    const int a = (int)(pair / nb), j = (int)(pair - (int64_t)a * nb);
    const int c = nlev[a], off = levoff[a];
    for (int g = 0; g < c; ++g) { c1[g * 32 + lane] = 0.0; c2[g * 32 + lane] = 0.0; cn[g * 32 + lane] = 0; }
    const uint8_t *la = lab + (int64_t)catrow[a] * S;
    const double *xj = xs + (int64_t)j * S_pad;
    const uint32_t *ob = obsb + (int64_t)j * W;
    for (int64_t s = lane; s < S; s += 32) {
        const int l = la[s];
        const bool o = (ob[s >> 5] >> (s & 31)) & 1u;
        if (!o || l >= c) continue;
        const double v = xj[s];
        const int e = l * 32 + lane;
        cn[e] += 1;
        c1[e] += v;
        c2[e] = fma(v, v, c2[e]);
    }
    for (int g = 0; g < c; ++g) {
        int nsum = cn[g * 32 + lane];
        double s1 = c1[g * 32 + lane], s2 = c2[g * 32 + lane];
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

template <int MAXC>
static void launch_groupsum_fp64_t(const uint8_t *lab, int64_t S, const int32_t *catrow_dev, int32_t na,
                                   const int32_t *levoff_dev, const int32_t *nlev_dev, const double *xs,
                                   int64_t S_pad, const uint32_t *obsb, int64_t W, int32_t nb, int32_t *gn,
                                   double *g1, double *g2, cudaStream_t st) {
    // shared memory per warp: MAXC x 32 lanes x (two doubles + one int)
    constexpr int kWarps = MAXC <= 16 ? 8 : 4;
    constexpr size_t kSmem = (size_t)kWarps * MAXC * 32 * (2 * sizeof(double) + sizeof(int));
    cudaFuncSetAttribute(k_groupsum_fp64<MAXC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    const int64_t pairs = (int64_t)na * nb;
    const unsigned blocks = (unsigned)((pairs + kWarps - 1) / kWarps);
    count_launch();
    k_groupsum_fp64<MAXC><<<blocks, kWarps * 32, kSmem, st>>>(lab, S, catrow_dev, na, levoff_dev, nlev_dev, xs,
                                                              S_pad, obsb, W, nb, gn, g1, g2);
}

void launch_groupsum_fp64(const uint8_t *lab, int64_t S, const int32_t *catrow_dev, int32_t na,
                          const int32_t *levoff_dev, const int32_t *nlev_dev, const double *xs,
                          int64_t S_pad, const uint32_t *obsb, int64_t W, int32_t nb,
                          int32_t *gn, double *g1, double *g2, int32_t max_levels, cudaStream_t st) {
    if ((int64_t)na * nb == 0) return;
    if (max_levels <= 4)
        launch_groupsum_fp64_t<4>(lab, S, catrow_dev, na, levoff_dev, nlev_dev, xs, S_pad, obsb, W, nb, gn, g1, g2, st);
    else if (max_levels <= 16)
        launch_groupsum_fp64_t<16>(lab, S, catrow_dev, na, levoff_dev, nlev_dev, xs, S_pad, obsb, W, nb, gn, g1, g2,
                                   st);
    else
        launch_groupsum_fp64_t<kMaxLevels>(lab, S, catrow_dev, na, levoff_dev, nlev_dev, xs, S_pad, obsb, W, nb, gn,
                                           g1, g2, st);
}

}  // namespace napg
