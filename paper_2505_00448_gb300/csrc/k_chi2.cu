// Contingency tables (Sec. 3.5.4) as exact integer counts: for level rows r, r'
// (one per (variable, level)) T[r][r'] = popcount(B_r AND B_r') summed over the
// 32-sample words of the level bitmasks, i.e. the number of samples observed in
// both variables (and in the context) with those two labels. The (a, b) block
// of T is the c_a x c_b table of the pair. Only tiles with I <= J are computed;
// the finalize step reads the upper block.
#include "napg_internal.cuh"

namespace napg {

constexpr int kCT = 32;     // cells per tile edge
constexpr int kCK = 32;     // words per stage

__global__ void __launch_bounds__(256) k_contingency(const uint32_t *__restrict__ lb, int64_t W, int32_t R,
                                                     int32_t *__restrict__ T, const uint8_t *__restrict__ own_lev) {
    const int nt = (R + kCT - 1) / kCT;
    int t = blockIdx.x, I = 0;
    while (t >= nt - I) { t -= nt - I; ++I; }
    const int J = I + t;
    if (!rows_owned(own_lev, (int64_t)I * kCT, kCT, R)) return;   // no level of this part's variables
    __shared__ uint32_t sa[kCT][kCK + 1], sb[kCT][kCK + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int acc[2][2] = {};
    const int r0 = I * kCT, c0 = J * kCT;
    for (int64_t w0 = 0; w0 < W; w0 += kCK) {
        for (int e = threadIdx.x; e < kCT * kCK; e += 256) {
            const int r = e / kCK, k = e % kCK;
            const int64_t w = w0 + k;
            sa[r][k] = (r0 + r < R && w < W) ? lb[(int64_t)(r0 + r) * W + w] : 0u;
            sb[r][k] = (c0 + r < R && w < W) ? lb[(int64_t)(c0 + r) * W + w] : 0u;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kCK; ++k) {
            const uint32_t a0 = sa[ty][k], a1 = sa[ty + 16][k];
            const uint32_t b0 = sb[tx][k], b1 = sb[tx + 16][k];
            acc[0][0] += __popc(a0 & b0);
            acc[0][1] += __popc(a0 & b1);
            acc[1][0] += __popc(a1 & b0);
            acc[1][1] += __popc(a1 & b1);
        }
        __syncthreads();
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int r = r0 + ty + 16 * a, c = c0 + tx + 16 * b;
            if (r < R && c < R) {
                T[(int64_t)r * R + c] = acc[a][b];
                T[(int64_t)c * R + r] = acc[a][b];
            }
        }
}

void launch_contingency(const uint32_t *levbits, int64_t W, int32_t R, int32_t *T, const uint8_t *own_lev,
                        cudaStream_t st) {
    if (R == 0) return;
    const int nt = (R + kCT - 1) / kCT;
    count_launch();
    k_contingency<<<nt * (nt + 1) / 2, 256, 0, st>>>(levbits, W, R, T, own_lev);
}

__global__ void k_level_ownership(const uint8_t *own, const int32_t *levoff, const int32_t *nlev, int32_t na,
                                  uint8_t *own_lev) {
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x)
        for (int g = 0; g < nlev[a]; ++g) own_lev[levoff[a] + g] = own[a];
}

void launch_level_ownership(const uint8_t *own, const int32_t *levoff, const int32_t *nlev, int32_t na,
                            uint8_t *own_lev, cudaStream_t st) {
    if (na == 0) return;
    count_launch();
    k_level_ownership<<<(na + 255) / 256, 256, 0, st>>>(own, levoff, nlev, na, own_lev);
}

}  // namespace napg
