// Mixed-precision moment contractions on the 5th-generation tensor cores
// (tcgen05.mma, kind::f16 with FP32 accumulation in tensor memory), fed by TMA.
//
// Operands are "planes": FP16 matrices with one row per variable (or per
// categorical level) and one column per sample, K-major, rows padded to 128.
// For a continuous variable with in-context shift c (FP64 mean of its observed
// values) and v = mean of (x - c)^2:
//   M  = observed (1/0)                        exact
//   Xh + Xl = 2^s x~, x~ = (x - c) m         FP16 hi/lo split of the FP64 value
//   Dh + Dl = 2^t d,  d = ((x - c)^2 - v) m  centred square, FP16 hi/lo
//   H  = one-hot level rows (1/0)              exact
// s and t are per-row powers of two that put the row's largest magnitude in
// [2^14, 2^15), so hi/lo keep 22 significant bits (a bf16 pair keeps only 16,
// too few when one heavy-tailed term carries a large share of a sum); the
// epilogue removes them exactly. FP16 x FP16 products are exact in FP32.
// Sums for Pearson (Sec. 3.5.2):      Sxy ~ Xh Xh^T + Xh Xl^T + Xl Xh^T (split x3),
//                                     n = M M^T, Sx^T = M X~^T, Sxx^T = M D^T + v n
// Group sums (Sec. 3.5.5, 3.5.7):     n_g = H M^T, S1 = H X~^T, S2 = H D^T + v n_g
// Contingency tables (Sec. 3.5.4):    T = H H^T (E4M3 planes, kind::f8f6f4)
// 0/1 operands give integer sums that FP32 holds exactly (S < 2^24): T stays in
// tensor memory for the whole K loop; the pair counts n = M M^T and T take
// their 0/1 planes in FP8 E4M3 (1.0 is exact), at twice the FP16 MMA rate and
// half the operand bytes. In the stacked contractions n_g is drained as
// integers. The other sums are accumulated in short K-chunks in tensor memory
// and drained by the epilogue warps into float-float running sums, which bounds
// the FP32 accumulation error independently of S.
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include "napg_internal.cuh"
#include "umma.cuh"

namespace napg {

using namespace umma;

constexpr int kKB = 64;    // samples per K-block: one 128-byte swizzle row of 16-bit values
constexpr int kKB8 = 128;  // samples per K-block of the E4M3 planes: one 128-byte row
constexpr int kTM = 128;   // rows of an A tile (M of the MMA)

// Triangle tiles (I <= J) of a T x T tile grid in row order: t -> (I, J)
__device__ __forceinline__ void tri_coords(int t, int T, int &I, int &J) {
    int i = 0;
    while (t >= T - i) { t -= T - i; ++i; }
    I = i;
    J = i + t;
}

// Warp roles (10 warps): 0 TMA producer, 1 MMA issuer (and TMEM owner), 2-9
// epilogue (two warps per TMEM lane quadrant, each half the columns).
constexpr int kThreads = 320;

// ----------------------------------------- contingency counts (Sec. 3.5.4) --
//
// T[r][c] = sum_s H[r][s] H[c][s] over 0/1 rows r, c: for one-hot level rows,
// the number of samples in level r of one categorical and level c of another
// (0 where either is missing); for observed-mask rows, the pair counts n. The
// rows are E4M3 bytes (0x38 = 1.0, 0 = 0), 128 samples per K-block, four
// kind::f8f6f4 MMAs of K = 32 each. Integer sums below 2^24 are exact in FP32,
// so the counts stay in tensor memory for the whole K loop. Tiles are 128 rows
// (A) by 256 (B, one MMA of N = 256) over the upper triangle: tile (I, J) for
// J * 256 + 255 >= I * 128; each pair (r, c), r <= c, is written once, at
// (r, c) and (c, r), by the tile that holds it with r in A. Four 48 KB stages.
constexpr int kCountN = 256, kCountStages = 4;

struct CountParams {
    CUtensorMap mapA;              // E4M3 0/1 plane [rows_pad][S_pad8], box 128 x 128
    CUtensorMap mapB;              // the same plane, box 128 x 256
    int rows, tilesA, tilesB, nkb; // rows, 128-row tiles, 256-row tiles, 128-sample K-blocks
    int32_t *out;                  // T [rows][ld], both triangles
    int64_t ld;
    uint32_t *err;
    const uint8_t *own;            // level rows computed (a split call's part; NULL: all)
};

__global__ void __launch_bounds__(kThreads, 1) k_counts(const __grid_constant__ CountParams P) {
    constexpr int N = kCountN;
    constexpr int A_BYTES = kTM * kKB8, B_BYTES = N * kKB8, STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr int HC = N / 2;                  // columns per epilogue thread
    constexpr uint32_t IDESC = idesc_e4m3_f32(kTM, N);

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + kCountStages * STAGE_BYTES);
    uint64_t *empty = full + kCountStages;
    uint64_t *tfull = empty + kCountStages;
    uint32_t *tslot = (uint32_t *)(tfull + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile t -> (I, J): row tile I takes the column tiles J >= I / 2
    int I = 0, J = 0;
    {
        int t = blockIdx.x;
        while (t >= P.tilesB - I / 2) { t -= P.tilesB - I / 2; ++I; }
        J = I / 2 + t;
    }
    pdl_trigger();
    if (!rows_owned(P.own, (int64_t)I * kTM, kTM, P.rows)) { pdl_wait(); return; }   // another part's rows

    if (threadIdx.x == 0) {
        for (int s = 0; s < kCountStages; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(tfull, 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, N);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            prefetch_tmap(&P.mapA);
            prefetch_tmap(&P.mapB);
            int issued = 0;
            for (int kb = 0; kb < P.nkb; ++kb) {
                const int s = kb % kCountStages;
                if (kb >= kCountStages && !mbar_wait(&empty[s], ((kb / kCountStages) - 1) & 1, P.err)) break;
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                uint8_t *st = smem + s * STAGE_BYTES;
                tma_load_2d(st, &P.mapA, &full[s], kb * kKB8, I * kTM);
                tma_load_2d(st + A_BYTES, &P.mapB, &full[s], kb * kKB8, J * N);
                issued = kb + 1;
            }
            // our own copies must have landed before the CTA tears down
            for (int kb = issued - kCountStages < 0 ? 0 : issued - kCountStages; kb < issued; ++kb)
                mbar_wait(&full[kb % kCountStages], (kb / kCountStages) & 1, P.err);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint64_t dbase = sdesc_sw128(smem_u32(smem));
            bool ok = true;
            for (int kb = 0; kb < P.nkb; ++kb) {
                const int s = kb % kCountStages;
                if (!mbar_wait(&full[s], (kb / kCountStages) & 1, P.err)) { ok = false; break; }
                fence_after_sync();
                const uint64_t ds = dbase + (uint64_t)((uint32_t)(s * STAGE_BYTES) >> 4);
#pragma unroll
                for (int k = 0; k < kKB8 / 32; ++k)
                    mma_e4m3(tbase, ds + 2 * k, ds + (A_BYTES >> 4) + 2 * k, IDESC, (kb | k) ? 1u : 0u);
                mma_commit(&empty[s]);             // frees the stage once these MMAs are done
            }
            if (ok) mma_commit(tfull);
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - 2;               // 0..7
        const int q = warp & 3;                // TMEM lane quadrant this warp may access
        const int half = ew >> 2;              // which half of the columns
        const int gi = I * kTM + q * 32 + lane;
        if (mbar_wait(tfull, 0, P.err)) {
            fence_after_sync();
            pdl_wait();
            const uint32_t a0 = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * HC);
#pragma unroll 1
            for (int g = 0; g < HC / 16; ++g) {
                uint32_t r[16];
                tmem_ld16(a0 + g * 16, r);
                tmem_ld_wait();
                if (gi < P.rows) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int col = J * N + half * HC + g * 16 + k;
                        if (col >= gi && col < P.rows) {
                            const int32_t v = (int32_t)__uint_as_float(r[k]);
                            P.out[(int64_t)gi * P.ld + col] = v;
                            P.out[(int64_t)col * P.ld + gi] = v;
                        }
                    }
                }
            }
        }
    }
    pdl_wait();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(tbase, N);
}

// ------------------------------------------------------ Sxy (Sec. 3.5.2) --
//
// Sum over the co-observed samples of x~_i x~_j for the pairs of a triangle
// tile (I <= J) of 128 x 128 variables, from the FP16 planes Xh, Xl of the
// centred, scaled values (zero where a value is missing, so every product off
// the co-observed set vanishes). The split product keeps three of the four
// terms of (Xh + Xl)(Xh + Xl): Xl Xl is below 2^-22 of Xh Xh, about 3.5e-8 of
// the sum for two copies of one column (the residuals then align) and far less
// for independent ones, against the 1e-6 bar on r. Per K-block of 64 samples
// the MMA thread issues the two cross products (Xh Xl, Xl Xh: 2^-11 of Xh Xh,
// random sign) first and Xh Xh last, all into one accumulator that
// starts the K-block at zero: the Xh Xh sum is rounded over its own 4
// instructions, as when drained alone every K-block (correlated pairs add
// same-sign terms, and the accumulator's per-instruction rounding error grows
// with the instructions between restarts). Four such accumulators fill the 512
// columns of tensor memory: a chunk is two K-blocks, each in its own
// accumulator, and two chunks are in flight. The epilogue adds a chunk's two
// K-block sums in FP32 (round to nearest, so the added error has no bias) and
// folds the result into float-float running sums by TwoSum: one TwoSum per two
// K-blocks of MMAs. NEPI epilogue warps (a quarter per tensor-memory lane
// quadrant) split the 128 columns: 16 of them (96 registers a thread) measured
// the same as 8 and leave room for the per-CTA K range; the autotuner picks the
// stage width (64 samples, 128-byte swizzle, or 32, 64-byte swizzle: the outputs
// are bit-identical, each element seeing the same operations in the same order).
constexpr int kSxyStages = 3;

struct SxyParams {
    CUtensorMap mapH, mapL;        // Xh, Xl planes [rows_pad][S_pad], box 64 x 128, 128-byte swizzle
    CUtensorMap mapH32, mapL32;    // the same planes, box 32 x 128, 64-byte swizzle
    int rows, tiles, nkb;          // variables, 128-row tiles, K-blocks
    // triangle tiles from nfull on run as two CTAs, K-blocks [0, kbmid) and
    // [kbmid, nkb), each adding its part into the zeroed output (see launch_sxy)
    int nfull, kbmid;
    double *out;                   // Sxy[i][j] for i in tile I, j in tile J (I <= J), row-major, ld
    int64_t ld;
    const int8_t *sexp;            // per-row scale exponents: the output is divided by 2^(e_i + e_j)
    uint32_t *err;
    const uint8_t *own;            // rows computed (a split call's part; NULL: all)
};

// this CTA's triangle tile and its K-blocks [kb0, kb0 + nk): the tiles from
// nfull on run as two CTAs each, over [0, kbmid) and [kbmid, nkb)
__device__ __forceinline__ int sxy_tile(const SxyParams &P, int &kb0, int &nk) {
    const int t = blockIdx.x;
    kb0 = 0;
    nk = P.nkb;
    if (t < P.nfull) return t;
    const int q = t - P.nfull;
    if (q & 1) { kb0 = P.kbmid; nk = P.nkb - P.kbmid; }
    else nk = P.kbmid;
    return P.nfull + (q >> 1);
}

template <int NEPI, int KS>
__global__ void __launch_bounds__((2 + NEPI) * 32, 1) k_sxy(const __grid_constant__ SxyParams P) {
    // KS samples per pipeline stage: 64 (128-byte swizzle, 3 stages of 64 KB)
    // or 32 (64-byte swizzle, 6 stages of 32 KB: twice the loads in flight)
    static_assert(KS == 64 || KS == 32, "stage width");
    constexpr int SPB = kKB / KS;                      // stages per 64-sample K-block
    constexpr int STAGES = kSxyStages * SPB;
    constexpr int T_BYTES = kTM * KS * 2;              // one 128 x KS FP16 tile
    constexpr int STAGE_BYTES = 4 * T_BYTES;           // Ah, Al, Bh, Bl
    constexpr int N = kTM;
    constexpr int HC = N * 4 / NEPI;                   // columns per epilogue thread
    static_assert(NEPI % 4 == 0 && HC % 8 == 0, "epilogue warps");
    constexpr int H2 = HC / 2;
    constexpr uint32_t IDESC = idesc_f16_f32(kTM, N);

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;       // [2] chunk accumulators ready
    uint64_t *tempty = tfull + 2;           // [2] chunk accumulators drained
    uint64_t *mdone = tempty + 2;
    uint32_t *tslot = (uint32_t *)(mdone + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int I, J;
    {
        int kb0, nk;
        tri_coords(sxy_tile(P, kb0, nk), P.tiles, I, J);
    }
    pdl_trigger();
    if (!rows_owned(P.own, (int64_t)I * kTM, kTM, P.rows)) { pdl_wait(); return; }   // another part's rows
    const bool diag = I == J;                  // B is A: loaded once

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], NEPI); }
        mbar_init(mdone, 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc(tslot, 512);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            const CUtensorMap *mh = KS == 64 ? &P.mapH : &P.mapH32;
            const CUtensorMap *ml = KS == 64 ? &P.mapL : &P.mapL32;
            prefetch_tmap(mh);
            prefetch_tmap(ml);
            const uint32_t bytes = diag ? 2 * T_BYTES : STAGE_BYTES;
            int kb0, nk;
            sxy_tile(P, kb0, nk);
            const int nsb = nk * SPB, x0 = kb0 * kKB;    // stages to fill, first sample
            int issued = 0;
            for (int sb = 0; sb < nsb; ++sb) {
                const int s = sb % STAGES;
                if (sb >= STAGES && !mbar_wait(&empty[s], ((sb / STAGES) - 1) & 1, P.err)) break;
                mbar_arrive_expect_tx(&full[s], bytes);
                uint8_t *st = smem + s * STAGE_BYTES;
                tma_load_2d(st, mh, &full[s], x0 + sb * KS, I * kTM);
                tma_load_2d(st + T_BYTES, ml, &full[s], x0 + sb * KS, I * kTM);
                if (!diag) {
                    tma_load_2d(st + 2 * T_BYTES, mh, &full[s], x0 + sb * KS, J * kTM);
                    tma_load_2d(st + 3 * T_BYTES, ml, &full[s], x0 + sb * KS, J * kTM);
                }
                issued = sb + 1;
            }
            // our own copies must have landed before the CTA tears down
            for (int sb = issued - STAGES < 0 ? 0 : issued - STAGES; sb < issued; ++sb)
                mbar_wait(&full[sb % STAGES], (sb / STAGES) & 1, P.err);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint64_t dbase = KS == 64 ? sdesc_sw128(smem_u32(smem)) : sdesc_sw64(smem_u32(smem));
            // descriptor offsets (16-byte units) of Ah, Al, Bh, Bl within a stage
            constexpr uint32_t oAh = 0, oAl = T_BYTES >> 4;
            const uint32_t oBh = diag ? 0u : (uint32_t)(2 * T_BYTES) >> 4;
            const uint32_t oBl = diag ? (uint32_t)T_BYTES >> 4 : (uint32_t)(3 * T_BYTES) >> 4;
            int kb0, nk;
            sxy_tile(P, kb0, nk);
            const int nchunks = (nk + 1) / 2;
            int kb = 0;
            bool ok = true;
            for (int c = 0; c < nchunks && ok; ++c) {
                const int b = c & 1;
                if (c >= 2 && !mbar_wait(&tempty[b], ((c >> 1) - 1) & 1, P.err)) { ok = false; break; }
                fence_after_sync();
                const int kb_end = min(nk, 2 * c + 2);       // K-blocks counted from kb0
                for (; kb < kb_end && ok; ++kb) {
                    const uint32_t d = tbase + (uint32_t)((2 * b + (kb & 1)) * N);
                    uint64_t ds[SPB];
                    // the cross products of each stage of the K-block as it lands
                    // (the first restarts the accumulator) ...
#pragma unroll
                    for (int h = 0; h < SPB; ++h) {
                        const int sb = kb * SPB + h, s = sb % STAGES;
                        if (!mbar_wait(&full[s], (sb / STAGES) & 1, P.err)) { ok = false; break; }
                        fence_after_sync();
                        ds[h] = dbase + (uint64_t)((uint32_t)(s * STAGE_BYTES) >> 4);
#pragma unroll
                        for (int k = 0; k < KS / 16; ++k) {
                            mma_f16(d, ds[h] + oAh + 2 * k, ds[h] + oBl + 2 * k, IDESC, (h | k) ? 1u : 0u);  // Xh Xl
                            mma_f16(d, ds[h] + oAl + 2 * k, ds[h] + oBh + 2 * k, IDESC, 1u);               // Xl Xh
                        }
                    }
                    if (!ok) break;
                    // ... then Xh Xh over the whole K-block, last
#pragma unroll
                    for (int h = 0; h < SPB; ++h) {
#pragma unroll
                        for (int k = 0; k < KS / 16; ++k)
                            mma_f16(d, ds[h] + oAh + 2 * k, ds[h] + oBh + 2 * k, IDESC, 1u);
                        mma_commit(&empty[(kb * SPB + h) % STAGES]);   // frees the stage once its MMAs are done
                    }
                }
                if (!ok) break;
                mma_commit(&tfull[b]);
            }
            mma_commit(mdone);
        }
        __syncwarp();
        mbar_wait(mdone, 0, P.err);
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - 2;               // 0..NEPI-1
        const int q = warp & 3;                // TMEM lane quadrant this warp may access
        const int half = ew >> 2;              // which group of HC columns
        const int row = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        uint64_t hi[H2], lo[H2];               // float-float running sums, two columns per register pair
#pragma unroll
        for (int k = 0; k < H2; ++k) hi[k] = lo[k] = 0ull;
        int kb0, nk;
        sxy_tile(P, kb0, nk);
        const bool part = (int)blockIdx.x >= P.nfull;     // one of a split tile's two CTAs
        const int nchunks = (nk + 1) / 2;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            if (!mbar_wait(&tfull[b], (c >> 1) & 1, P.err)) { ok = false; break; }
            fence_after_sync();
            const bool two = 2 * c + 1 < nk;
            const uint32_t a0 = tbase + lane_addr + (uint32_t)(2 * b * N + half * HC);
#pragma unroll
            for (int g = 0; g < HC / 4; ++g) {
                uint32_t r0[4], r1[4];
                tmem_ld4(a0 + g * 4, r0);
                if (two) tmem_ld4(a0 + N + g * 4, r1);
                tmem_ld_wait();
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    uint64_t v = pk2(__uint_as_float(r0[2 * k]), __uint_as_float(r0[2 * k + 1]));
                    if (two) v = add2(v, pk2(__uint_as_float(r1[2 * k]), __uint_as_float(r1[2 * k + 1])));
                    two_sum2(hi[g * 2 + k], lo[g * 2 + k], v);
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        pdl_wait();
        if (ok) {
            const int gi = I * kTM + row;
            if (gi < P.rows) {
                const int ei = P.sexp ? (int)P.sexp[gi] : 0;
#pragma unroll
                for (int k = 0; k < H2; ++k) {
                    float h0, h1, l0, l1;
                    unpk2(hi[k], h0, h1);
                    unpk2(lo[k], l0, l1);
#pragma unroll
                    for (int e2 = 0; e2 < 2; ++e2) {
                        const int col = J * N + half * HC + 2 * k + e2;
                        if (col < P.rows) {
                            const double v = (double)(e2 ? h1 : h0) + (double)(e2 ? l1 : l0);
                            const int e = ei + (P.sexp ? (int)P.sexp[col] : 0);
                            if (part) atomicAdd(&P.out[(int64_t)gi * P.ld + col], ldexp(v, -e));   // two parts onto 0: order-free
                            else P.out[(int64_t)gi * P.ld + col] = ldexp(v, -e);
                        }
                    }
                }
            }
        }
    }
    pdl_wait();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 1) tmem_dealloc(tbase, 512);
}

// --------------------------------------------------- stacked contraction --
//
// A 0/1 plane (observed mask or one-hot levels) against the planes M, Xh, Xl,
// Dh, Dl of SV B variables stacked into one operand of N = NPL SV rows: one MMA
// per 16 samples reads the A tile once for all the sums. The MMA spans a pair
// of CTAs on two SMs (cta_group::2, M = 256): each CTA loads 128 rows of A and
// half of the stacked B rows (the first half in the even CTA; with an odd
// number of planes the middle plane is split between the two), so each SM
// streams half of B per sample and the tensor core is fed at its full rate. The
// even CTA's full barrier counts the bytes of both CTAs (the odd CTA's copies
// signal it across the pair); MMA commits arrive in both CTAs; each CTA's
// epilogue warps drain its own 128 accumulator rows and report to the even
// CTA's drain barrier. All blocks of the accumulator restart every chunk and
// are drained: counts as exact integers, the hi sums by TwoSum into float-float
// running sums, the lo sums into the low parts. The sums drained here are
// centred (x - c, (x - c)^2 - v) or exact counts, so a partial sum random-walks
// instead of growing with the chunk, and chunks of 16 K-blocks keep the FP32
// accumulation error far below the statistics' bars.
// SV = B variables per tile (a multiple of 16: the epilogue's two halves read
// 8-column groups); the autotuner picks the width per shape.
constexpr int kSGroup = 8;         // A tile pairs per rasterisation group

struct StackParams {
    CUtensorMap mapA;              // 0/1 plane, box 64 x 128
    CUtensorMap mapB[5];           // the B planes in role order, box 64 x SV
    CUtensorMap mapSplit;          // the plane split between the pair (odd plane counts), box 64 x SV/2
    int rowsA, rowsB;              // valid rows of A and B
    int tilesA, tilesB;            // 128-row A tiles (a pair takes two), SV-row B tiles
    int nkb, chunk;                // K-blocks, K-blocks per drain
    int32_t *out_n;                // counts      [rowsA][ld] (or transposed)
    double *out_s1, *out_s2;       // sum x~, sum (x~^2 - v)
    int64_t ld;
    int out_transpose;
    const int8_t *exp1, *exp2;     // per-B-row scale exponents of X~ and D
    uint32_t *err;
    const uint8_t *own;            // split symmetric calls (A and B rows are the same
                                   // variables): rows computed (NULL: all)
};

// B rows of the stack held by CTA `rank` of the pair: the even CTA holds stacked
// rows [0, N/2), the odd one [N/2, N). Loads the CTA's half for K-block x of B
// tile J into `bh`, counting the bytes on the barrier at cluster address `bar`.
template <int NPL, int SV>
__device__ __forceinline__ void load_b_half(const StackParams &P, uint32_t rank, uint8_t *bh, uint32_t bar, int x,
                                            int J) {
    constexpr int N = NPL * SV, HALF = N / 2;
    constexpr int PS = HALF / SV;              // plane holding stacked row HALF
    constexpr int OS = HALF % SV;              // its rows in the even CTA (0: a plane boundary)
    const int y = J * SV;
    if (rank == 0) {
#pragma unroll
        for (int p = 0; p < PS; ++p) tma_load_2d_pair(bh + p * SV * 128, &P.mapB[p], bar, x, y);
        if (OS) tma_load_2d_pair(bh + PS * SV * 128, &P.mapSplit, bar, x, y);
    } else {
        if (OS) tma_load_2d_pair(bh, &P.mapSplit, bar, x, y + OS);
#pragma unroll
        for (int p = (OS ? PS + 1 : PS); p < NPL; ++p)
            tma_load_2d_pair(bh + (p * SV - HALF) * 128, &P.mapB[p], bar, x, y);
    }
}

// NPL planes stacked, playing the roles ROLE0, ROLE0 + 1, ... of the list (M,
// Xh, Xl, Dh, Dl): all five (counts and both sums), the first three (counts and
// sum x~) or the last two (sum of centred squares alone). Dropping Dl is not an
// option for the group sums: the FP16 rounding of the centred squares leaves
// ~2^-12 / sqrt(n) relative error on the within-group sum, which at n of a few
// hundred and F well above 1 moves the F statistic's effect-scale value by more
// than 1e-6.
// KPS K-blocks per pipeline stage (1 or 2): two put twice the MMAs between
// barrier round trips, which pays when N is small.
template <int NPL, int SV, int STAGES, int ROLE0, int KPS>
__global__ void __launch_bounds__(kThreads, 1) k_umma_stacked(const __grid_constant__ StackParams P) {
    constexpr bool kHasN = ROLE0 == 0;
    constexpr bool kHasS1 = ROLE0 <= 1 && ROLE0 + NPL > 1;
    constexpr bool kHasS2 = ROLE0 + NPL > 3;
    constexpr int kSPerThread = SV / 2;
    static_assert(SV % 16 == 0, "SV");
    constexpr int kSN = NPL * SV;                 // MMA N
    constexpr int HALF = kSN / 2;                 // B rows per CTA
    constexpr int A_BYTES = kTM * kKB * 2;
    constexpr int BH_BYTES = HALF * kKB * 2;
    constexpr int KB_BYTES = A_BYTES + BH_BYTES;  // one K-block: A tile, then this CTA's half of B
    constexpr int STAGE_BYTES = KPS * KB_BYTES;
    static_assert(KPS == 1 || KPS == 2, "K-blocks per stage");
    static_assert(BH_BYTES % 1024 == 0 && STAGE_BYTES % 1024 == 0 && (SV / 2 * 128) % 1024 == 0,
                  "8-row swizzle atoms stay 1024-B aligned");
    static_assert(kSN % 16 == 0 && kSN <= 256, "N");
    constexpr uint32_t IDESC = idesc_f16_f32(2 * kTM, kSN);
    constexpr int BUF = 256;       // tensor-memory columns per accumulator buffer (kSN used)

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *mdone = tempty + 2;
    uint32_t *tslot = (uint32_t *)(mdone + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    // grouped rasterisation over tile pairs: within a group of kSGroup A tile
    // pairs, consecutive pairs step through the group's A tiles, then the B
    // tiles, so a wave of resident pairs covers a block of both operands and
    // streams each from HBM about once
    int I2, J;
    {
        const int tilesA2 = (P.tilesA + 1) / 2;
        const int cl = blockIdx.x >> 1;
        const int per_group = kSGroup * P.tilesB;
        const int g = cl / per_group, r = cl - g * per_group;
        const int gsz = min(kSGroup, tilesA2 - g * kSGroup);
        J = r / gsz;
        I2 = g * kSGroup + (r - J * gsz);
    }
    pdl_trigger();
    if (P.own) {
        // a split call needs the sums of pairs (i, j), i <= j, i owned: tiles with
        // owned A rows and a B column at or after them, or owned B rows and an A
        // row at or after them (both CTAs of the pair decide alike)
        const int64_t a0 = (int64_t)2 * I2 * kTM, c0 = (int64_t)J * SV;
        const bool need = (rows_owned(P.own, a0, 2 * kTM, P.rowsA) && c0 + SV - 1 >= a0) ||
                          (rows_owned(P.own, c0, SV, P.rowsB) && a0 + 2 * kTM - 1 >= c0);
        if (!need) { pdl_wait(); return; }
    }
    const int nchunks = (P.nkb + P.chunk - 1) / P.chunk;   // P.chunk is a multiple of KPS
    const int nsb = (P.nkb + KPS - 1) / KPS;                  // pipeline stages to fill

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], 16); }
        mbar_init(mdone, 1);
        fence_mbar_init();
    }
    if (warp == 1) tmem_alloc_pair(tslot, 512);
    fence_before_sync();
    __syncthreads();
    cluster_sync();                // both CTAs' barriers set up and tensor memory allocated
    fence_after_sync();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            prefetch_tmap(&P.mapA);
            for (int p = 0; p < NPL; ++p) prefetch_tmap(&P.mapB[p]);
            if (NPL & 1) prefetch_tmap(&P.mapSplit);
            const uint32_t full0 = cluster_addr(&full[0], 0);
            int issued = 0;
            for (int sb = 0; sb < nsb; ++sb) {
                const int s = sb % STAGES;
                if (sb >= STAGES && !mbar_wait(&empty[s], ((sb / STAGES) - 1) & 1, P.err)) break;
                const uint32_t bar = full0 + (uint32_t)(s * 8);
                const int nk = min(KPS, P.nkb - sb * KPS);       // K-blocks in this stage
                if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * nk * KB_BYTES);   // both CTAs' bytes
                uint8_t *st = smem + s * STAGE_BYTES;
                for (int h = 0; h < nk; ++h) {
                    const int x = (sb * KPS + h) * kKB;
                    tma_load_2d_pair(st + h * KB_BYTES, &P.mapA, bar, x, (2 * I2 + (int)rank) * kTM);
                    load_b_half<NPL, SV>(P, rank, st + h * KB_BYTES + A_BYTES, bar, x, J);
                }
                issued = sb + 1;
            }
            // the copies of both CTAs are counted on the even CTA's barriers: it
            // waits for the last ones before the pair leaves (the MMA warp has
            // waited for all the others)
            if (rank == 0)
                for (int sb = issued - STAGES < 0 ? 0 : issued - STAGES; sb < issued; ++sb)
                    mbar_wait(&full[sb % STAGES], (sb / STAGES) & 1, P.err);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (rank == 0 && lane == 0) {
            const uint64_t dbase = sdesc_sw128(smem_u32(smem));
            const int spc = P.chunk / KPS;                      // stages per chunk
            int sb = 0;
            bool ok = true;
            for (int c = 0; c < nchunks && ok; ++c) {
                const int b = c & 1;
                if (c >= 2 && !mbar_wait(&tempty[b], ((c >> 1) - 1) & 1, P.err)) { ok = false; break; }
                fence_after_sync();
                const int sb_end = min(nsb, (c + 1) * spc);
                const int sb_chunk0 = sb;
                const uint32_t dcol = tbase + (uint32_t)(b * BUF);
                for (; sb < sb_end; ++sb) {
                    const int s = sb % STAGES;
                    if (!mbar_wait(&full[s], (sb / STAGES) & 1, P.err)) { ok = false; break; }
                    fence_after_sync();
                    const uint64_t ds = dbase + (uint64_t)((uint32_t)(s * STAGE_BYTES) >> 4);
                    const int nk = min(KPS, P.nkb - sb * KPS);
#pragma unroll
                    for (int h = 0; h < KPS; ++h) {
                        if (h < nk) {
                            const uint64_t dh = ds + (uint64_t)((uint32_t)(h * KB_BYTES) >> 4);
#pragma unroll
                            for (int k = 0; k < kKB / 16; ++k)
                                mma_f16_pair(dcol, dh + (uint64_t)(2 * k), dh + (uint64_t)((A_BYTES >> 4) + 2 * k),
                                             IDESC, (sb == sb_chunk0 && h == 0 && k == 0) ? 0u : 1u);
                        }
                    }
                    mma_commit_pair(&empty[s]);
                }
                if (!ok) break;
                mma_commit_pair(&tfull[b]);
            }
            mma_commit_pair(mdone);
        }
        __syncwarp();
        mbar_wait(mdone, 0, P.err);
    } else {
        // ---------------------------------------------------------- epilogue
        const int ew = warp - 2;               // 0..7
        const int q = warp & 3;                // TMEM lane quadrant this warp may access
        const int h = ew >> 2;                 // which half of the SV variables
        const int row = q * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(q * 32) << 16;
        const uint32_t tempty0 = cluster_addr(&tempty[0], 0);
        constexpr int K2 = kSPerThread / 2;
        // columns read per tensor-memory wait: all of a plane's, or 16 where the
        // four sums of 32 columns already hold 128 registers
        constexpr int kLdCols = kSPerThread > 24 && kSPerThread % 16 == 0 ? 16 : kSPerThread;
        int32_t cnt[kSPerThread];
        uint64_t s1h[K2], s1l[K2], s2h[K2], s2l[K2];    // packed float-float sums
#pragma unroll
        for (int k = 0; k < kSPerThread; ++k) cnt[k] = 0;
#pragma unroll
        for (int k = 0; k < K2; ++k) s1h[k] = s1l[k] = s2h[k] = s2l[k] = 0ull;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            if (!mbar_wait(&tfull[b], (c >> 1) & 1, P.err)) { ok = false; break; }
            fence_after_sync();
            const uint32_t col0 = tbase + lane_addr + (uint32_t)(b * BUF + h * kSPerThread);
#pragma unroll
            for (int p = 0; p < NPL; ++p) {
#pragma unroll
                for (int g0 = 0; g0 < kSPerThread; g0 += kLdCols) {
                    uint32_t r[kLdCols];
#pragma unroll
                    for (int g = 0; g < kLdCols / 8; ++g) {
                        uint32_t t8[8];
                        tmem_ld8(col0 + (uint32_t)(p * SV + g0 + g * 8), t8);
#pragma unroll
                        for (int k = 0; k < 8; ++k) r[g * 8 + k] = t8[k];
                    }
                    tmem_ld_wait();
                    const int role = ROLE0 + p;
                    if (role == 0) {
#pragma unroll
                        for (int k = 0; k < kLdCols; ++k) cnt[g0 + k] += (int32_t)__uint_as_float(r[k]);   // exact integers
                    } else {
#pragma unroll
                        for (int k = 0; k < kLdCols / 2; ++k) {
                            const int kk = g0 / 2 + k;
                            const uint64_t v = pk2(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1]));
                            if (role == 1) two_sum2(s1h[kk], s1l[kk], v);
                            else if (role == 2) s1l[kk] = add2(s1l[kk], v);
                            else if (role == 3) two_sum2(s2h[kk], s2l[kk], v);
                            else s2l[kk] = add2(s2l[kk], v);
                        }
                    }
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(tempty0 + (uint32_t)(b * 8));
        }
        pdl_wait();
        if (ok) {
            const int gi = (2 * I2 + (int)rank) * kTM + row;
            if (gi < P.rowsA) {
#pragma unroll
                for (int k = 0; k < K2; ++k) {
                    float a0, a1, b0, b1, c0, c1, d0, d1;
                    unpk2(s1h[k], a0, a1);
                    unpk2(s1l[k], b0, b1);
                    unpk2(s2h[k], c0, c1);
                    unpk2(s2l[k], d0, d1);
#pragma unroll
                    for (int e2 = 0; e2 < 2; ++e2) {
                        const int col = J * SV + h * kSPerThread + 2 * k + e2;
                        if (col < P.rowsB) {
                            const int64_t o = P.out_transpose ? (int64_t)col * P.ld + gi : (int64_t)gi * P.ld + col;
                            if (kHasN) P.out_n[o] = cnt[2 * k + e2];
                            if (kHasS1)
                                P.out_s1[o] = ldexp((double)(e2 ? a1 : a0) + (double)(e2 ? b1 : b0), -(int)P.exp1[col]);
                            if (kHasS2)
                                P.out_s2[o] = ldexp((double)(e2 ? c1 : c0) + (double)(e2 ? d1 : d0), -(int)P.exp2[col]);
                        }
                    }
                }
            }
        }
    }
    pdl_wait();
    fence_before_sync();
    __syncthreads();
    cluster_sync();                // neither CTA leaves while the pair still reads its shared memory
    fence_after_sync();
    if (warp == 1) tmem_dealloc_pair(tbase, 512);
}

// ------------------------------------------------------------ plane prep --

// One block per (padded) row: shift c, v = mean (x - c)^2 over the observed
// samples, the scale exponents s, t, then the FP16 planes M, Xh, Xl, Dh, Dl
// (zero where unobserved, in the padding columns and in padding rows).
__device__ __forceinline__ int scale_exp(double maxabs) {
    if (!(maxabs > 0.0)) return 0;
    int e;
    frexp(maxabs, &e);                 // maxabs in [2^(e-1), 2^e)
    int s = 15 - e;                    // 2^s maxabs in [2^14, 2^15)
    return s < -120 ? -120 : (s > 120 ? 120 : s);
}

// FP32 arithmetic throughout (this GPU's FP64 rate is 1/64 of FP32): the shift
// c and the centring value v need not be exact, only identical in the planes
// and in the finalize step (which adds v n back), so they are FP32 values; x - c
// keeps 24 bits relative to itself (exact when x and c are within a factor of
// two), and the planes keep 22.
// Four consecutive values x[s0 .. s0+3] (zero past S): one 16-byte load (two for
// FP64) when the row is 16-byte aligned and the four are inside it.
// LAST: the values' last use (streaming loads, evicted from L2 first).
template <bool LAST = false, typename T>
__device__ __forceinline__ void load4(const T *__restrict__ x, int64_t s0, int64_t S, bool aligned, T (&v)[4]) {
    if (aligned && s0 + 4 <= S) {
        if constexpr (sizeof(T) == 4) {
            const float4 *p = reinterpret_cast<const float4 *>(x + s0);
            const float4 f = LAST ? __ldcs(p) : *p;
            v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else {
            const double2 *p = reinterpret_cast<const double2 *>(x + s0);
            const double2 a = LAST ? __ldcs(p) : p[0], b = LAST ? __ldcs(p + 1) : p[1];
            v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = s0 + k < S ? x[s0 + k] : T(0);
    }
}

// (count, mean, sum of squared deviations) of two parts of a row, merged
// (Chan, Golub and LeVeque's pairwise update), in FP32
__device__ __forceinline__ void chan_merge(float &n, float &m, float &q, float n2, float m2, float q2) {
    const float nt = n + n2;
    if (nt == 0.f) return;
    const float d = m2 - m, f = n2 / nt;
    m = fmaf(d, f, m);
    q = q + q2 + d * d * n * f;
    n = nt;
}

// Persistent: kPlaneRowsPerSM blocks per SM take the (padded) rows in turn.
// Pass 1 streams the row once for the observed count, mean and squared
// deviations (each thread about its own first observed value, merged across
// threads by chan_merge) and the extremes, which give the largest |x - c| and
// bound |(x - c)^2 - v| by max(max (x - c)^2 - v, v); pass 2 reads the row again
// from L2 (the rows in flight take a few tens of MB; its loads and the plane
// stores are marked streaming, evicted first, so that they do not push the
// rows out) and writes the planes. Four samples per thread and step, several
// steps in flight.
constexpr int kPlaneThreads = 512, kPlaneRowsPerSM = 3;

template <typename T>
__global__ void __launch_bounds__(kPlaneThreads, kPlaneRowsPerSM) k_planes_cont(const T *__restrict__ X, int64_t S, int64_t S_pad,
                                                              const int32_t *__restrict__ vars, int32_t nv,
                                                              int32_t rows_pad, const uint32_t *__restrict__ obsv,
                                                              int64_t W, __half *Pm, __half *Pxh, __half *Pxl,
                                                              __half *Pdh, __half *Pdl, double *shift, double *vsq,
                                                              int8_t *sexp, int8_t *texp) {
    __shared__ float red[5][kPlaneThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nw = kPlaneThreads / 32;
    const int64_t n4 = S_pad / 4, nq = (S + 3) / 4;
    for (int i = blockIdx.x; i < rows_pad; i += gridDim.x) {
        const int64_t base = (int64_t)i * S_pad;
        // the planes are written four samples (8 bytes) per thread and step (S_pad
        // is a multiple of 64, so every row starts 128-byte aligned)
        uint2 *m4 = reinterpret_cast<uint2 *>(Pm + base), *xh4 = reinterpret_cast<uint2 *>(Pxh + base),
              *xl4 = reinterpret_cast<uint2 *>(Pxl + base), *dh4 = reinterpret_cast<uint2 *>(Pdh + base),
              *dl4 = reinterpret_cast<uint2 *>(Pdl + base);
        if (i >= nv) {
            const uint2 z4 = make_uint2(0u, 0u);
            for (int64_t q = threadIdx.x; q < n4; q += kPlaneThreads) {
                __stcs(m4 + q, z4); __stcs(xh4 + q, z4); __stcs(xl4 + q, z4); __stcs(dh4 + q, z4); __stcs(dl4 + q, z4);
            }
            continue;
        }
        const T *x = X + (int64_t)vars[i] * S;
        const uint32_t *ob = obsv + (int64_t)i * W;
        const bool al = (reinterpret_cast<uintptr_t>(x) & 15u) == 0;
        // pass 1
        float cn = 0.f, sh = 0.f, s1 = 0.f, s2 = 0.f;
        T hi = T(-3.0e38f), lo = T(3.0e38f);
        bool have = false;
#pragma unroll 4
        for (int64_t q = threadIdx.x; q < nq; q += kPlaneThreads) {
            const int64_t s0 = 4 * q;
            const uint32_t obits = (ob[s0 >> 5] >> (s0 & 31)) & 0xfu;
            T xv[4];
            load4(x, s0, S, al, xv);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((obits >> k) & 1u) {
                    if (!have) { sh = (float)xv[k]; have = true; }
                    const float d = (float)(xv[k] - (T)sh);
                    cn += 1.f;
                    s1 += d;
                    s2 = fmaf(d, d, s2);
                    hi = xv[k] > hi ? xv[k] : hi;
                    lo = xv[k] < lo ? xv[k] : lo;
                }
        }
        // this thread's (count, mean, squared deviations) about its own mean
        float m = 0.f, qd = 0.f;
        if (cn > 0.f) {
            const float a = s1 / cn;
            m = sh + a;
            qd = fmaxf(fmaf(-a, s1, s2), 0.f);
        }
        float fhi = (float)hi, flo = (float)lo;
        for (int o = 16; o > 0; o >>= 1) {
            const float n2 = __shfl_down_sync(0xffffffffu, cn, o), m2 = __shfl_down_sync(0xffffffffu, m, o),
                        q2 = __shfl_down_sync(0xffffffffu, qd, o);
            chan_merge(cn, m, qd, n2, m2, q2);
            fhi = fmaxf(fhi, __shfl_down_sync(0xffffffffu, fhi, o));
            flo = fminf(flo, __shfl_down_sync(0xffffffffu, flo, o));
        }
        if (lane == 0) { red[0][warp] = cn; red[1][warp] = m; red[2][warp] = qd; red[3][warp] = fhi; red[4][warp] = flo; }
        __syncthreads();
        float tn = 0.f, tm = 0.f, tq = 0.f, thi = -3.0e38f, tlo = 3.0e38f;
        for (int k = 0; k < nw; ++k) {          // every thread, same order
            chan_merge(tn, tm, tq, red[0][k], red[1][k], red[2][k]);
            thi = fmaxf(thi, red[3][k]);
            tlo = fminf(tlo, red[4][k]);
        }
        __syncthreads();                          // red is reused by the next row
        const float c = tn > 0.f ? tm : 0.f;
        const float v = tn > 0.f ? tq / tn : 0.f;
        const float tmx = tn > 0.f ? fmaxf((float)((T)thi - (T)c), (float)((T)c - (T)tlo)) : 0.f;
        const float md = tn > 0.f ? fmaxf(tmx * tmx - v, v) : 0.f;
        const int es = scale_exp((double)tmx), et = scale_exp((double)md);
        if (threadIdx.x == 0) { shift[i] = (double)c; vsq[i] = (double)v; sexp[i] = (int8_t)es; texp[i] = (int8_t)et; }
        const float fs = exp2f((float)es), ft = exp2f((float)et);   // exact powers of two
        // pass 2: the planes, four samples per thread and step
#pragma unroll 2
        for (int64_t q = threadIdx.x; q < n4; q += kPlaneThreads) {
            const int64_t s0 = 4 * q;
            const uint32_t obits = s0 < S ? (ob[s0 >> 5] >> (s0 & 31)) & 0xfu : 0u;
            T xv[4] = {T(0), T(0), T(0), T(0)};
            if (obits) load4<true>(x, s0, S, al, xv);
            __align__(8) __half hm[4];
            __align__(8) __half hxh[4];
            __align__(8) __half hxl[4];
            __align__(8) __half hdh[4];
            __align__(8) __half hdl[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t s = s0 + k;
                const bool o = s < S && ((obits >> k) & 1u);
                float xt = 0.f;
                if (o) xt = (float)(xv[k] - (T)c);
                const float xs = xt * fs;                                  // exact scaling
                const __half h = __float2half_rn(xs);
                const __half l = __float2half_rn(xs - __half2float(h));    // the difference is exact in FP32
                // d = xt^2 - v with the square's rounding error recovered by FMA
                const float sq = xt * xt;
                const float sq_err = fmaf(xt, xt, -sq);
                const float ds = ((sq - v) + sq_err) * ft;
                const __half dh = __float2half_rn(ds);
                const __half dl = __float2half_rn(ds - __half2float(dh));
                const __half z = __float2half(0.f);
                hm[k] = o ? __float2half(1.f) : z;
                hxh[k] = o ? h : z;
                hxl[k] = o ? l : z;
                hdh[k] = o ? dh : z;
                hdl[k] = o ? dl : z;
            }
            __stcs(m4 + q, *reinterpret_cast<const uint2 *>(hm));
            __stcs(xh4 + q, *reinterpret_cast<const uint2 *>(hxh));
            __stcs(xl4 + q, *reinterpret_cast<const uint2 *>(hxl));
            __stcs(dh4 + q, *reinterpret_cast<const uint2 *>(hdh));
            __stcs(dl4 + q, *reinterpret_cast<const uint2 *>(hdl));
        }
    }
}

// one-hot level rows from the level bitmasks (zero padding rows/columns): a
// thread writes eight samples (one 16-byte store) from one byte of a bit word
__global__ void k_planes_onehot(const uint32_t *__restrict__ levbits, int64_t W, int32_t R, int64_t S_pad,
                                __half *H) {
    const int r = blockIdx.x;
    uint4 *h8 = reinterpret_cast<uint4 *>(H + (int64_t)r * S_pad);   // S_pad is a multiple of 64
    const int64_t n8 = S_pad / 8;
    for (int64_t q = threadIdx.x; q < n8; q += blockDim.x) {
        const int64_t s0 = 8 * q, w = s0 >> 5;
        const uint32_t b = (r < R && w < W) ? (levbits[(int64_t)r * W + w] >> (s0 & 31)) & 0xffu : 0u;
        // FP16 1.0 is 0x3c00; two samples per 32-bit word
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            v[k] = ((b >> (2 * k)) & 1u) * 0x3c00u | (((b >> (2 * k + 1)) & 1u) * 0x3c00u) << 16;
        h8[q] = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

// The same rows as E4M3 bytes (1.0 = 0x38) over S_pad8 samples (a multiple of
// 128), sixteen samples (one 16-byte store) per thread and step.
__global__ void k_planes_onehot8(const uint32_t *__restrict__ bits, int64_t W, int32_t R, int64_t S_pad8,
                                 uint8_t *H8) {
    const int r = blockIdx.x;
    uint4 *h16 = reinterpret_cast<uint4 *>(H8 + (int64_t)r * S_pad8);
    const int64_t n16 = S_pad8 / 16;
    for (int64_t q = threadIdx.x; q < n16; q += blockDim.x) {
        const int64_t s0 = 16 * q, w = s0 >> 5;
        const uint32_t b = (r < R && w < W) ? (bits[(int64_t)r * W + w] >> (s0 & 31)) & 0xffffu : 0u;
        uint32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) x |= ((b >> (4 * k + j)) & 1u) * (0x38u << (8 * j));
            v[k] = x;
        }
        h16[q] = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

// ---------------------------------------------------------------- host --

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// FP16 matrix [rows][cols], cols a multiple of 64, box = 64 columns x box_rows rows
// box_k = 64 samples (128-byte rows, 128-byte swizzle) or 32 (64-byte rows,
// 64-byte swizzle)
static bool make_map(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows,
                     uint32_t box_k = kKB) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {box_k, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, box_k == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// a K-major E4M3 plane [rows][cols], box 128 x box_rows (one 128-byte swizzle row)
static bool make_map8(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols};
    cuuint32_t box[2] = {(cuuint32_t)kKB8, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// zeroes the outputs of the split triangle tiles (from nfull on) that this part
// owns, before both halves add into them
__global__ void k_sxy_zero(SxyParams P) {
    pdl_trigger();
    pdl_wait();
    int I, J;
    tri_coords(P.nfull + (int)blockIdx.x, P.tiles, I, J);
    if (!rows_owned(P.own, (int64_t)I * kTM, kTM, P.rows)) return;
    for (int idx = threadIdx.x; idx < kTM * kTM; idx += blockDim.x) {
        const int gi = I * kTM + idx / kTM, col = J * kTM + idx % kTM;
        if (gi < P.rows && col < P.rows) P.out[(int64_t)gi * P.ld + col] = 0.0;
    }
}

// kern<<<grid, block, smem, st>>>(P); with pdl, as a programmatic dependent of
// the stream's previous kernel (the kernel's blocks may start in that kernel's
// tail; the kernel orders its stores and its completion after it by pdl_wait)
template <typename Par>
static cudaError_t launch_chain(void (*kern)(Par), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                                bool pdl, const Par &P) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, P);
}

template <int NEPI, int KS>
static napg_status launch_sxy_v(napg_ctx *ctx, const SxyParams &P, int tiles, cudaStream_t st, bool pdl) {
    const size_t smem = (size_t)kSxyStages * 4 * kTM * kKB * 2 + 1024 + 512;
    NAPG_CU(ctx, cudaFuncSetAttribute(k_sxy<NEPI, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (tiles == 0) return NAPG_OK;
    const int nsplit = tiles - P.nfull;
    if (nsplit > 0) {
        count_launch();
        NAPG_CU(ctx, launch_chain(k_sxy_zero, (unsigned)nsplit, 256, 0, st, pdl, P));
        pdl = true;              // k_sxy's split tiles add into what k_sxy_zero cleared
    }
    count_launch();
    NAPG_CU(ctx, launch_chain(k_sxy<NEPI, KS>, (unsigned)(P.nfull + 2 * nsplit), (2 + NEPI) * 32, smem, st, pdl, P));
    return NAPG_OK;
}

// One CTA per SM: a last wave of R < SMs / 2 tiles would leave most SMs idle
// for a whole tile's time, so those R tiles run as 2R CTAs over half the
// K-blocks each (half a tile's time). The split depends only on the whole
// triangle's tile count and the SM count, so every part of a split call and
// every run of the shape computes each tile the same way.
static napg_status launch_sxy(napg_ctx *ctx, SxyParams P, int tiles, cudaStream_t st, bool pdl) {
    const int sms = ctx->sm_count > 0 ? ctx->sm_count : 152;
    const int rem = tiles % sms;
    P.nfull = tiles;
    P.kbmid = (P.nkb / 4) * 2;                 // an even K-block: the halves' chunks pair K-blocks alike
    if (tiles > sms && rem > 0 && 2 * rem <= sms && P.kbmid >= 2) P.nfull = tiles - rem;
    auto run = [&](int choice) -> napg_status {
        return choice == 0 ? launch_sxy_v<16, 64>(ctx, P, tiles, st, pdl) : launch_sxy_v<16, 32>(ctx, P, tiles, st, pdl);
    };
    const TuneKey key{kTuneSxy, P.rows, P.rows, P.nkb};
    return tuned_launch(ctx, key, 2, run, st);
}

template <int NPL, int SV, int ROLE0, int KPS>
static napg_status launch_stacked_sv(napg_ctx *ctx, const StackParams &P, cudaStream_t st) {
    constexpr int STAGE_BYTES = KPS * (kTM * kKB * 2 + NPL * SV / 2 * kKB * 2);
    constexpr int STAGES = (220 * 1024) / STAGE_BYTES > 8 ? 8 : (220 * 1024) / STAGE_BYTES;
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
    auto kern = k_umma_stacked<NPL, SV, STAGES, ROLE0, KPS>;
    NAPG_CU(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int pairs = ((P.tilesA + 1) / 2) * P.tilesB;
    if (pairs == 0) return NAPG_OK;
    // pairs of CTAs on two SMs (one cluster per tile pair)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * pairs));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    count_launch();
    NAPG_CU(ctx, cudaLaunchKernelEx(&cfg, kern, P));
    return NAPG_OK;
}

// Launch shapes the autotuner chooses from, per plane set: the B-tile width
// (two per set) times 1 or 2 K-blocks per pipeline stage, candidate
// 2 * kps_index + width_index. Every shape gives the same sums: each output
// accumulates the same products in the same order and drains. MMA N = planes x
// width stays a multiple of 16 and at most 256.
enum StackPlanes { kStackAll = 0, kStackNS1 = 1, kStackS2 = 2, kStackSums = 3 };
constexpr int kStackWidths[4][2] = {{48, 32}, {80, 64}, {112, 64}, {64, 48}};
constexpr int kStackPlaneCount[4] = {5, 3, 2, 4};

// A x stacked B planes with the B-tile width chosen by the autotuner for this
// shape (the tensor maps of the B planes are encoded for that width); pb holds
// the planes of the set in role order
static napg_status launch_stacked(napg_ctx *ctx, StackParams P, const void *const *pb, int set, int64_t rows_b_pad,
                                  int64_t S_pad, int kind, cudaStream_t st) {
    auto run = [&](int choice) -> napg_status {
        const int sv = kStackWidths[set][choice & 1];
        const bool two = choice >= 2;
        const int npl = kStackPlaneCount[set];
        for (int k = 0; k < npl; ++k)
            if (!make_map(&P.mapB[k], pb[k], rows_b_pad, S_pad, sv))
                return fail(ctx, NAPG_E_CUDA, "cuTensorMapEncodeTiled failed");
        // an odd number of planes: the middle one is split between the pair
        if ((npl & 1) && !make_map(&P.mapSplit, pb[npl / 2], rows_b_pad, S_pad, sv / 2))
            return fail(ctx, NAPG_E_CUDA, "cuTensorMapEncodeTiled failed");
        P.tilesB = (P.rowsB + sv - 1) / sv;
        if (set == kStackAll)
            return sv == 48 ? (two ? launch_stacked_sv<5, 48, 0, 2>(ctx, P, st) : launch_stacked_sv<5, 48, 0, 1>(ctx, P, st))
                            : (two ? launch_stacked_sv<5, 32, 0, 2>(ctx, P, st) : launch_stacked_sv<5, 32, 0, 1>(ctx, P, st));
        if (set == kStackSums)
            return sv == 64 ? (two ? launch_stacked_sv<4, 64, 1, 2>(ctx, P, st) : launch_stacked_sv<4, 64, 1, 1>(ctx, P, st))
                            : (two ? launch_stacked_sv<4, 48, 1, 2>(ctx, P, st) : launch_stacked_sv<4, 48, 1, 1>(ctx, P, st));
        if (set == kStackNS1)
            return sv == 80 ? (two ? launch_stacked_sv<3, 80, 0, 2>(ctx, P, st) : launch_stacked_sv<3, 80, 0, 1>(ctx, P, st))
                            : (two ? launch_stacked_sv<3, 64, 0, 2>(ctx, P, st) : launch_stacked_sv<3, 64, 0, 1>(ctx, P, st));
        return sv == 112 ? (two ? launch_stacked_sv<2, 112, 3, 2>(ctx, P, st) : launch_stacked_sv<2, 112, 3, 1>(ctx, P, st))
                         : (two ? launch_stacked_sv<2, 64, 3, 2>(ctx, P, st) : launch_stacked_sv<2, 64, 3, 1>(ctx, P, st));
    };
    const TuneKey key{kind, P.rowsA, P.rowsB, P.nkb};
    return tuned_launch(ctx, key, 4, run, st);
}

template <typename T, typename... Rest>
static const T *kern_x_type(void (*)(const T *, Rest...));

struct ContPlanes {
    __half *M, *Xh, *Xl, *Dh, *Dl;
    int8_t *sexp, *texp;        // per-row scale exponents of X~ and D
    int64_t rows_pad, S_pad;
};

static napg_status prep_cont_planes(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st,
                                    const int32_t *vars_dev, int32_t nv, const uint32_t *obsv, int first_slot,
                                    double *shift, double *vsq, ContPlanes &cp,
                                    const std::vector<int32_t> *cache_vars) {
    cp.S_pad = ((c.S + kKB - 1) / kKB) * kKB;
    cp.rows_pad = ((nv + kTM - 1) / kTM) * kTM;
    const size_t plane = sizeof(__half) * (size_t)cp.rows_pad * (size_t)cp.S_pad;
    napg_status st_ = NAPG_OK;
    __half *pl[5];
    for (int k = 0; k < 5; ++k) {
        pl[k] = (__half *)ws_get(ctx, ws, first_slot + k, plane, &st_);
        if (st_) return st_;
    }
    cp.M = pl[0]; cp.Xh = pl[1]; cp.Xl = pl[2]; cp.Dh = pl[3]; cp.Dl = pl[4];
    cp.sexp = (int8_t *)ws_get(ctx, ws, Workspace::kExp, 2 * (size_t)cp.rows_pad, &st_);
    double *pshift = (double *)ws_get(ctx, ws, Workspace::kPlShift, sizeof(double) * (size_t)nv, &st_);
    double *pvsq = (double *)ws_get(ctx, ws, Workspace::kPlVsq, sizeof(double) * (size_t)nv, &st_);
    if (st_) return st_;
    cp.texp = cp.sexp + cp.rows_pad;
    Workspace::PlaneKey &key = ws.plane_key;
    const bool hit = cache_vars && first_slot == Workspace::kTmpA && key.valid && key.gen == c.gen &&
                     key.vars == *cache_vars;
    if (!hit) {
        key.valid = false;
        Stage s_(ctx->trace, st, "planes_f16");
        const unsigned grid = (unsigned)std::min<int64_t>(cp.rows_pad, (int64_t)kPlaneRowsPerSM *
                                                          (ctx->sm_count > 0 ? ctx->sm_count : 152));
        auto launch = [&](auto kern) -> napg_status {
            count_launch();
            kern<<<grid, kPlaneThreads, 0, st>>>((decltype(kern_x_type(kern)))c.X, c.S, cp.S_pad, vars_dev, nv,
                                                 (int32_t)cp.rows_pad, obsv, c.W, cp.M, cp.Xh, cp.Xl, cp.Dh, cp.Dl,
                                                 pshift, pvsq, cp.sexp, cp.texp);
            NAPG_CU(ctx, cudaGetLastError());
            return NAPG_OK;
        };
        if (c.dtype == NAPG_F32) NAPG_ST(launch(k_planes_cont<float>));
        else NAPG_ST(launch(k_planes_cont<double>));
        if (cache_vars && first_slot == Workspace::kTmpA) {
            key.valid = true;
            key.gen = c.gen;
            key.vars = *cache_vars;
        }
    }
    NAPG_CU(ctx, cudaMemcpyAsync(shift, pshift, sizeof(double) * (size_t)nv, cudaMemcpyDeviceToDevice, st));
    NAPG_CU(ctx, cudaMemcpyAsync(vsq, pvsq, sizeof(double) * (size_t)nv, cudaMemcpyDeviceToDevice, st));
    return NAPG_OK;
}

static napg_status prep_onehot(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st, const uint32_t *levbits,
                               int32_t R, int slot, __half **H, int64_t &rows_pad, int64_t &S_pad) {
    S_pad = ((c.S + kKB - 1) / kKB) * kKB;
    rows_pad = ((R + kTM - 1) / kTM) * kTM;
    napg_status st_ = NAPG_OK;
    *H = (__half *)ws_get(ctx, ws, slot, sizeof(__half) * (size_t)rows_pad * (size_t)S_pad, &st_);
    if (st_) return st_;
    Stage s_(ctx->trace, st, "planes_onehot");
    count_launch();
    k_planes_onehot<<<(unsigned)rows_pad, 256, 0, st>>>(levbits, c.W, R, S_pad, *H);
    NAPG_CU(ctx, cudaGetLastError());
    return NAPG_OK;
}

// 0/1 rows from bitmask rows (bits[r * W + w]) as an E4M3 plane, rows padded to
// 128 and samples to 128
static napg_status prep_onehot8(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st, const uint32_t *bits,
                                int32_t R, int slot, uint8_t **H8, int64_t &rows_pad, int64_t &S_pad8) {
    S_pad8 = ((c.S + kKB8 - 1) / kKB8) * kKB8;
    rows_pad = ((R + kTM - 1) / kTM) * kTM;
    napg_status st_ = NAPG_OK;
    *H8 = (uint8_t *)ws_get(ctx, ws, slot, (size_t)rows_pad * (size_t)S_pad8, &st_);
    if (st_) return st_;
    Stage s_(ctx->trace, st, "planes_onehot");
    count_launch();
    k_planes_onehot8<<<(unsigned)rows_pad, 256, 0, st>>>(bits, c.W, R, S_pad8, *H8);
    NAPG_CU(ctx, cudaGetLastError());
    return NAPG_OK;
}

// K-blocks (of 64 samples) between drains of the stacked sums: they are
// counts, centred x~ and centred squares (per variable or per level), whose
// partial sums random-walk instead of growing with the chunk, so their FP32
// accumulation error stays far from the bar; a drain of the stacked
// accumulator takes longer than 4 K-blocks of MMAs, so shorter chunks would
// stall the pair.
constexpr int kChunkStacked = 16;

static napg_status launch_counts(napg_ctx *ctx, const uint8_t *H8, int64_t hrows, int64_t S_pad8, int32_t R, int32_t *T,
                                 const uint8_t *own, cudaStream_t st, bool pdl);

napg_status mixed_pearson(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st, const int32_t *vars_dev, int32_t nv,
                          const uint32_t *obsv, double *Sxy, double *Sx, double *Sxx, int32_t *nn, double *shift,
                          double *vsq, const std::vector<int32_t> *cache_vars, const uint8_t *own) {
    ContPlanes cp;
    NAPG_ST(prep_cont_planes(ctx, c, ws, st, vars_dev, nv, obsv, Workspace::kTmpA, shift, vsq, cp, cache_vars));
    const int nkb = (int)(cp.S_pad / kKB);
    const int T = (int)(cp.rows_pad / kTM);
    // The E4M3 observed rows for the pair counts, built before the chain below
    uint8_t *M8 = nullptr;
    int64_t mrows = 0, S_pad8 = 0;
    NAPG_ST(prep_onehot8(ctx, c, ws, st, obsv, nv, Workspace::kTmpF, &M8, mrows, S_pad8));
    // Three independent contractions over the planes, each launched as a
    // programmatic dependent of the one before, so that its blocks start on the
    // SMs the previous kernel's last, partial wave leaves idle.
    Stage s_(ctx->trace, st, "pearson_moments_tc");
    // P1: all ordered (A tile, B tile) pairs, the mask as A against the four
    // value planes of the B variables stacked: sum_s m_i x~_j = Sx[j][i] and
    // sum_s m_i d_j = D[j][i], written transposed (coalesced stores)
    {
        StackParams P{};
        if (!make_map(&P.mapA, cp.M, cp.rows_pad, cp.S_pad, kTM))
            return fail(ctx, NAPG_E_CUDA, "cuTensorMapEncodeTiled failed");
        const void *pb[4] = {cp.Xh, cp.Xl, cp.Dh, cp.Dl};
        P.rowsA = nv; P.rowsB = nv; P.tilesA = T;
        P.nkb = nkb; P.chunk = kChunkStacked;
        P.out_n = nullptr; P.out_s1 = Sx; P.out_s2 = Sxx; P.ld = nv; P.out_transpose = 1;
        P.exp1 = cp.sexp; P.exp2 = cp.texp; P.err = ctx->dev_err;
        P.own = own;
        NAPG_ST(launch_stacked(ctx, P, pb, kStackSums, cp.rows_pad, cp.S_pad, kTuneStackMask, st));
    }
    // P2: n = M M^T, symmetric, on the triangle (k_counts on the E4M3 rows)
    NAPG_ST(launch_counts(ctx, M8, mrows, S_pad8, nv, nn, own, st, true));
    // P3: Sxy on the triangle tiles (k_sxy)
    {
        SxyParams P{};
        if (!make_map(&P.mapH, cp.Xh, cp.rows_pad, cp.S_pad, kTM) || !make_map(&P.mapL, cp.Xl, cp.rows_pad, cp.S_pad, kTM) ||
            !make_map(&P.mapH32, cp.Xh, cp.rows_pad, cp.S_pad, kTM, 32) ||
            !make_map(&P.mapL32, cp.Xl, cp.rows_pad, cp.S_pad, kTM, 32))
            return fail(ctx, NAPG_E_CUDA, "cuTensorMapEncodeTiled failed");
        P.rows = nv; P.tiles = T; P.nkb = nkb;
        P.out = Sxy; P.ld = nv; P.sexp = cp.sexp; P.err = ctx->dev_err; P.own = own;
        NAPG_ST(launch_sxy(ctx, P, T * (T + 1) / 2, st, true));
    }
    return NAPG_OK;
}

napg_status mixed_groupsum(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st, const uint32_t *levbits, int32_t R,
                           const int32_t *vars_b_dev, int32_t nb, const uint32_t *obsb, int32_t *gn, double *g1,
                           double *g2, double *shift, double *vsq, const std::vector<int32_t> *cache_vars,
                           const uint32_t *obsa, int32_t na, double *g2tot) {
    ContPlanes cp;
    NAPG_ST(prep_cont_planes(ctx, c, ws, st, vars_b_dev, nb, obsb, Workspace::kTmpA, shift, vsq, cp, cache_vars));
    __half *H = nullptr;
    int64_t hrows = 0, S_pad = 0;
    NAPG_ST(prep_onehot(ctx, c, ws, st, levbits, R, Workspace::kTmpF, &H, hrows, S_pad));
    StackParams P{};
    if (!make_map(&P.mapA, H, hrows, S_pad, kTM)) return fail(ctx, NAPG_E_CUDA, "cuTensorMapEncodeTiled failed");
    P.rowsA = R; P.rowsB = nb; P.tilesA = (int)(hrows / kTM);
    P.nkb = (int)(S_pad / kKB); P.chunk = kChunkStacked;
    P.out_n = gn; P.out_s1 = g1; P.out_s2 = g2; P.ld = nb; P.out_transpose = 0;
    P.exp1 = cp.sexp; P.exp2 = cp.texp; P.err = ctx->dev_err;
    if (!g2tot) {
        const void *pb[5] = {cp.M, cp.Xh, cp.Xl, cp.Dh, cp.Dl};
        Stage s_(ctx->trace, st, "groupsum_tc");
        return launch_stacked(ctx, P, pb, kStackAll, cp.rows_pad, cp.S_pad, kTuneStackOneHot, st);
    }
    // One-way ANOVA needs the centred squares summed over all co-observed
    // samples only (SSW = sum x~^2 - sum_g S1_g^2 / n_g): the level rows take
    // the count and sum planes, and each categorical's observed row alone takes
    // the square planes
    {
        const void *pb[3] = {cp.M, cp.Xh, cp.Xl};
        P.out_s2 = nullptr;
        Stage s_(ctx->trace, st, "groupsum_tc");
        NAPG_ST(launch_stacked(ctx, P, pb, kStackNS1, cp.rows_pad, cp.S_pad, kTuneStackOneHotNS1, st));
    }
    __half *O = nullptr;
    int64_t orows = 0;
    NAPG_ST(prep_onehot(ctx, c, ws, st, obsa, na, Workspace::kTmpG, &O, orows, S_pad));
    StackParams Q{};
    if (!make_map(&Q.mapA, O, orows, S_pad, kTM)) return fail(ctx, NAPG_E_CUDA, "cuTensorMapEncodeTiled failed");
    Q.rowsA = na; Q.rowsB = nb; Q.tilesA = (int)(orows / kTM);
    Q.nkb = (int)(S_pad / kKB); Q.chunk = kChunkStacked;
    Q.out_n = nullptr; Q.out_s1 = nullptr; Q.out_s2 = g2tot; Q.ld = nb; Q.out_transpose = 0;
    Q.exp1 = cp.sexp; Q.exp2 = cp.texp; Q.err = ctx->dev_err;
    const void *qb[2] = {cp.Dh, cp.Dl};
    Stage s_(ctx->trace, st, "groupsum_tc");
    return launch_stacked(ctx, Q, qb, kStackS2, cp.rows_pad, cp.S_pad, kTuneStackSquares, st);
}

// T = H H^T over the 0/1 E4M3 rows of H8 (hrows x S_pad8, rows padded to 128):
// both triangles of T[R][R], integers exact; own: rows computed (NULL: all)
static napg_status launch_counts(napg_ctx *ctx, const uint8_t *H8, int64_t hrows, int64_t S_pad8, int32_t R, int32_t *T,
                                 const uint8_t *own, cudaStream_t st, bool pdl) {
    CountParams P{};
    if (!make_map8(&P.mapA, H8, hrows, S_pad8, kTM) || !make_map8(&P.mapB, H8, hrows, S_pad8, kCountN))
        return fail(ctx, NAPG_E_CUDA, "cuTensorMapEncodeTiled failed");
    P.rows = R;
    P.tilesA = (int)(hrows / kTM);
    P.tilesB = (int)((hrows + kCountN - 1) / kCountN);
    P.nkb = (int)(S_pad8 / kKB8);
    P.out = T; P.ld = R; P.err = ctx->dev_err; P.own = own;
    int tiles = 0;
    for (int i = 0; i < P.tilesA; ++i) tiles += P.tilesB - i / 2;
    const size_t smem = (size_t)kCountStages * (kTM + kCountN) * kKB8 + 1024 + 256;
    NAPG_CU(ctx, cudaFuncSetAttribute(k_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (tiles == 0) return NAPG_OK;
    count_launch();
    NAPG_CU(ctx, launch_chain(k_counts, (unsigned)tiles, kThreads, smem, st, pdl, P));
    return NAPG_OK;
}

napg_status mixed_contingency(napg_ctx *ctx, Cohort &c, Workspace &ws, cudaStream_t st, const uint32_t *levbits, int32_t R,
                              int32_t *T, const uint8_t *own_lev) {
    uint8_t *H8 = nullptr;
    int64_t hrows = 0, S_pad8 = 0;
    NAPG_ST(prep_onehot8(ctx, c, ws, st, levbits, R, Workspace::kTmpF, &H8, hrows, S_pad8));
    Stage s_(ctx->trace, st, "contingency_tc");
    return launch_counts(ctx, H8, hrows, S_pad8, R, T, own_lev, st, false);
}

}  // namespace napg
