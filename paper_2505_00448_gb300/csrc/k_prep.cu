// Prep kernels: cohort validation and observed bitmasks (Sec. 3.2 deletion is
// done later as a bitwise AND of these masks), sample-context bits, per-column
// shifts, and per-level bitmasks of categorical variables.
#include "napg_internal.cuh"

namespace napg {

template <typename T>
__device__ __forceinline__ bool is_missing_val(T v, double m, bool m_is_nan) {
    return m_is_nan ? isnan((double)v) : ((double)v == m);
}

// One warp per (variable, 32-sample word): observed bit via ballot; checks finite
// values and integer labels in [0, c); writes labels of categorical variables.
// With copy_to, X is the cohort in (device-mapped) host memory and each value is
// also written to the device copy as it is checked.
template <typename T>
__global__ void k_validate_obs(const T *__restrict__ X, int64_t F, int64_t S, int64_t W, double missing,
                               const uint8_t *__restrict__ vtype, const int32_t *__restrict__ nlev,
                               const int32_t *__restrict__ catrow, uint32_t *__restrict__ obs,
                               uint8_t *__restrict__ lab, uint32_t *err, int64_t v_base, T *__restrict__ copy_to) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t v = (int64_t)blockIdx.y + v_base;
    if (v >= F || warp >= W) return;
    const bool m_nan = isnan(missing);
    const int64_t s = warp * 32 + lane;
    bool ob = false;
    uint32_t e = 0;
    const bool cat = vtype[v] == 1;
    uint8_t lb = kMissingLabel;
    if (s < S) {
        const T x = X[v * S + s];
        if (copy_to) copy_to[v * S + s] = x;
        ob = !is_missing_val(x, missing, m_nan);
        if (ob) {
            const double xd = (double)x;
            if (!isfinite(xd)) {
                e |= kErrNonfinite;
            } else if (cat) {
                if (xd != floor(xd) || xd < 0.0 || xd >= (double)nlev[v]) e |= kErrLabel;
                else lb = (uint8_t)xd;
            }
        }
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, ob);
    if (lane == 0) obs[v * W + warp] = bits;
    if (cat && s < S) lab[(int64_t)catrow[v] * S + s] = ob ? lb : kMissingLabel;
    if (e) atomicOr(err, e);
}

void launch_validate_obs(const void *X, int32_t dtype, int64_t F, int64_t S, int64_t W, double missing,
                         const uint8_t *vtype_dev, const int32_t *nlev_dev, const int32_t *catrow_dev,
                         uint32_t *obs, uint8_t *lab, uint32_t *err, cudaStream_t st, void *copy_to) {
    if (F == 0 || W == 0) return;
    for (int64_t v0 = 0; v0 < F; v0 += 65535) {      // grid.y limit
        dim3 grid((unsigned)((W + 7) / 8), (unsigned)std::min<int64_t>(65535, F - v0));
        if (dtype == NAPG_F32) {
            count_launch();
            k_validate_obs<float><<<grid, 256, 0, st>>>((const float *)X, F, S, W, missing, vtype_dev, nlev_dev,
                                                         catrow_dev, obs, lab, err, v0, (float *)copy_to);
        }
        else {
            count_launch();
            k_validate_obs<double><<<grid, 256, 0, st>>>((const double *)X, F, S, W, missing, vtype_dev, nlev_dev,
                                                          catrow_dev, obs, lab, err, v0, (double *)copy_to);
        }
    }
}

// rows x cols -> cols x rows through a 32x33 shared tile
template <typename T>
__global__ void k_transpose(const T *__restrict__ in, T *__restrict__ out, int64_t rows, int64_t cols) {
    __shared__ T tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][k];
    }
}

void launch_transpose(const void *in, void *out, int32_t dtype, int64_t rows, int64_t cols, cudaStream_t st) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)), block(32, 8);
    if (dtype == NAPG_F32) { count_launch(); k_transpose<float><<<grid, block, 0, st>>>((const float *)in, (float *)out, rows, cols);
    }
    else { count_launch(); k_transpose<double><<<grid, block, 0, st>>>((const double *)in, (double *)out, rows, cols);
    }
}

// context mask (bytes) -> bit words; NULL mask = all samples
__global__ void k_ctx_bits(const uint8_t *__restrict__ mask, int64_t S, int64_t W, uint32_t *__restrict__ ctxw) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (w >= W) return;
    const int64_t s = w * 32 + lane;
    const bool in = (s < S) && (mask == nullptr || mask[s] != 0);
    const uint32_t b = __ballot_sync(0xffffffffu, in);
    if (lane == 0) ctxw[w] = b;
}

void launch_ctx_bits(const uint8_t *mask, int64_t S, int64_t W, uint32_t *ctxw, cudaStream_t st) {
    if (W == 0) return;
    count_launch();
    k_ctx_bits<<<(unsigned)((W + 7) / 8), 256, 0, st>>>(mask, S, W, ctxw);
}

__global__ void k_gather_obs(const uint32_t *__restrict__ obs, const int32_t *__restrict__ vars, int32_t nv,
                             const uint32_t *__restrict__ ctxw, int64_t W, uint32_t *__restrict__ out) {
    const int64_t total = (int64_t)nv * W;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / W, w = t - i * W;
        out[t] = obs[(int64_t)vars[i] * W + w] & ctxw[w];
    }
}

void launch_gather_obs(const uint32_t *obs, const int32_t *vars_dev, int32_t nv, const uint32_t *ctxw,
                       int64_t W, uint32_t *out, cudaStream_t st) {
    const int64_t total = (int64_t)nv * W;
    if (total == 0) return;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
    count_launch();
    k_gather_obs<<<blocks, 256, 0, st>>>(obs, vars_dev, nv, ctxw, W, out);
}

// One block per selected continuous variable: shift c = mean of its observed
// values (FP64), then xs[s] = x[s] - c where observed, 0 elsewhere (and in the
// padding up to S_pad).
template <typename T>
__global__ void k_shift_values(const T *__restrict__ X, int64_t S, int64_t S_pad, const int32_t *__restrict__ vars,
                               const uint32_t *__restrict__ obsv, int64_t W, double *__restrict__ shift,
                               double *__restrict__ xs) {
    const int i = blockIdx.x;
    const T *x = X + (int64_t)vars[i] * S;
    const uint32_t *ob = obsv + (int64_t)i * W;
    double sum = 0.0;
    int cnt = 0;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
        if ((ob[s >> 5] >> (s & 31)) & 1u) { sum += (double)x[s]; ++cnt; }
    }
    __shared__ double red[32];
    __shared__ int redc[32];
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_down_sync(0xffffffffu, sum, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = sum; redc[threadIdx.x >> 5] = cnt; }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        sum = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
        cnt = threadIdx.x < nw ? redc[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_down_sync(0xffffffffu, sum, o);
            cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        }
        if (threadIdx.x == 0) { red[0] = cnt > 0 ? sum / (double)cnt : 0.0; }
    }
    __syncthreads();
    const double c = red[0];
    if (threadIdx.x == 0 && shift) shift[i] = c;
    double *row = xs + (int64_t)i * S_pad;
    for (int64_t s = threadIdx.x; s < S_pad; s += blockDim.x) {
        const bool o = s < S && ((ob[s >> 5] >> (s & 31)) & 1u);
        row[s] = o ? ((double)x[s] - c) : 0.0;
    }
}

void launch_shift_values(const void *X, int32_t dtype, int64_t S, int64_t S_pad, const int32_t *vars_dev,
                         int32_t nv, const uint32_t *obsv, int64_t W, double *shift, double *xs,
                         cudaStream_t st) {
    if (nv == 0) return;
    if (dtype == NAPG_F32) {
        count_launch();
        k_shift_values<float><<<nv, 256, 0, st>>>((const float *)X, S, S_pad, vars_dev, obsv, W, shift, xs);
    }
    else {
        count_launch();
        k_shift_values<double><<<nv, 256, 0, st>>>((const double *)X, S, S_pad, vars_dev, obsv, W, shift, xs);
    }
}

// Level bitmasks of categorical variables: levbits[levoff[i] + g][w] has bit s
// set when sample s is observed (in the context) and has label g. levcnt gets
// the per-level counts (must be zeroed before). Each warp covers 32 words of one
// variable and adds its per-level counts with one atomic per level.
// Level bitmasks of the categorical variables: a thread takes one 32-sample word
// of one categorical, loads its 32 labels once (eight 32-bit words when the row
// is 4-byte aligned) and, per level g, forms the word's bits four labels at a
// time (byte-wise compare, then the four compare results packed into four bits)
// ANDed with the observed word; adjacent threads store adjacent words of a
// level row. The in-context level counts are summed per warp, then one atomic
// per level and warp.
__device__ __forceinline__ uint32_t bits_eq4(uint32_t labels4, uint32_t g4) {
    // 0xff in each byte whose label equals g, then bit 7 of each byte moved to
    // bits 0..3 (byte k -> bit k)
    const uint32_t m = __vcmpeq4(labels4, g4) & 0x80808080u;
    return (m * 0x00204081u) >> 28;
}

__global__ void k_level_bits(const uint8_t *__restrict__ lab, int64_t S, int64_t W,
                             const int32_t *__restrict__ catrow, const int32_t *__restrict__ levoff,
                             const int32_t *__restrict__ nlev, const uint32_t *__restrict__ obsv,
                             uint32_t *__restrict__ levbits, int32_t *__restrict__ levcnt, int i_base) {
    const int i = blockIdx.y + i_base;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = nlev[i], off = levoff[i];
    const uint8_t *la = lab + (int64_t)catrow[i] * S;
    uint32_t L[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) L[k] = 0xffffffffu;   // missing labels past the end
    uint32_t ob = 0;
    if (w < W) {
        ob = obsv[(int64_t)i * W + w];
        const int64_t s0 = w * 32;
        if (s0 + 32 <= S && (((uintptr_t)(la + s0)) & 3u) == 0) {
            const uint32_t *l4 = reinterpret_cast<const uint32_t *>(la + s0);
#pragma unroll
            for (int k = 0; k < 8; ++k) L[k] = l4[k];
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t v = 0;
                for (int b = 0; b < 4; ++b) {
                    const int64_t s = s0 + 4 * k + b;
                    v |= (uint32_t)(s < S ? la[s] : kMissingLabel) << (8 * b);
                }
                L[k] = v;
            }
        }
    }
    for (int g = 0; g < c; ++g) {
        const uint32_t g4 = 0x01010101u * (uint32_t)g;
        uint32_t bits = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) bits |= bits_eq4(L[k], g4) << (4 * k);
        bits &= ob;
        if (w < W) levbits[(int64_t)(off + g) * W + w] = bits;
        int cnt = __popc(bits);
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&levcnt[off + g], cnt);
    }
}

void launch_level_bits(const uint8_t *lab, int64_t S, int64_t W, const int32_t *catrow_dev,
                       const int32_t *levoff_dev, const int32_t *nlev_dev, int32_t nv,
                       const uint32_t *obsv, uint32_t *levbits, int32_t *levcnt, cudaStream_t st) {
    if (nv == 0 || W == 0) return;
    for (int i0 = 0; i0 < nv; i0 += 65535) {        // grid.y limit
        dim3 grid((unsigned)((W + 255) / 256), (unsigned)std::min(65535, nv - i0));
        count_launch();
        k_level_bits<<<grid, 256, 0, st>>>(lab, S, W, catrow_dev, levoff_dev, nlev_dev, obsv, levbits, levcnt, i0);
    }
}

__global__ void k_fill_nan(double *p, int64_t count) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
        p[t] = __longlong_as_double(0x7ff8000000000000LL);
}

void launch_fill_nan(double *p, int64_t count, cudaStream_t st) {
    if (count <= 0 || !p) return;
    count_launch();
    k_fill_nan<<<(unsigned)std::min<int64_t>((count + 255) / 256, 4096), 256, 0, st>>>(p, count);
}

}  // namespace napg
