// napg_pearson_fp64_noalloc: all-pairs Pearson r, p and n (plain FP64 form) for
// a small matrix already on the GPU, using no memory allocation at all.
//
// Some callers cannot allocate device memory: code that runs inside a host
// framework whose allocator owns the whole device (so a cudaMalloc behind its
// back fails or fragments its pool), processes started with a hard device-memory
// cap, and latency-critical paths that must never block in the allocator. This
// entry point serves them: its work space is one fixed array in device memory
// that is part of the library itself. The caller passes only the input matrix
// and the output buffers.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it until the process exits. Host code cannot use the variable's
// name as an address; the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current, and later calls reuse it
// as long as the thread's current CUDA context is the one it was looked up in
// (a call made in another context looks it up again). A device reset
// (cudaDeviceReset) loads the library's device code again and may keep the
// context handle, so the entry point must not be used after resetting the
// device in the same process.
// Every call shares the one array and leaves its contents behind: the counters
// that must start at zero are cleared on the stream at the start of each call,
// and two calls whose work overlaps on the GPU race on the array.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "napg_internal.cuh"

namespace napg {

constexpr int kNoAllocMaxVars = 256;
constexpr int kNoAllocMaxSamples = 8192;
constexpr size_t kNoAllocBytes = (size_t)24 << 20;   // 24 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64] = {};                  // per device, filled on first use
static void *g_noalloc_owner[64] = {};                // the CUDA context each address belongs to

// the calling thread's current driver context (NULL if it cannot be read), to
// tell a reset device's new context from the one an address was looked up in
static void *current_context() {
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuCtxGetCurrent_v4000)p;
    });
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return (void *)c;
}

// observed bits of every row (missing: == sentinel, or isnan when it is NaN);
// a non-missing +-inf/NaN raises bit kErrNonfinite in *err
__global__ void k_noalloc_obs(const double *__restrict__ X, int64_t F, int64_t S, int64_t W, double missing,
                              uint32_t *__restrict__ obs, int32_t *__restrict__ vars, uint32_t *err) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t v = blockIdx.y;
    if (w >= W) return;
    const int64_t s = w * 32 + lane;
    bool ob = false;
    if (s < S) {
        const double x = X[v * S + s];
        ob = isnan(missing) ? !isnan(x) : (x != missing);
        if (ob && !isfinite(x)) atomicOr(err, kErrNonfinite);
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, ob);
    if (lane == 0) obs[v * W + w] = bits;
    if (w == 0 && lane == 0) vars[v] = (int32_t)v;
}

// carve the fixed array: returns false if the request does not fit
struct NoAllocPlan {
    uint32_t *obs, *ctxw, *err;
    int32_t *vars, *nn, *flags, *counter, *pj_meta;
    double *xs, *shift, *Sxy, *Sx, *Sxx;
    PJob *jobs, *sorted;
    int64_t W, S_pad, pairs;
};

static bool carve(unsigned char *base, int64_t nv, int64_t S, NoAllocPlan &pl) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *p = base + off;
        off += (bytes + 255) / 256 * 256;
        return p;
    };
    pl.W = (S + 31) / 32;
    pl.S_pad = pl.W * 32;
    pl.pairs = nv * (nv + 1) / 2;
    pl.obs = (uint32_t *)take(sizeof(uint32_t) * nv * pl.W);
    pl.ctxw = (uint32_t *)take(sizeof(uint32_t) * pl.W);
    pl.err = (uint32_t *)take(sizeof(uint32_t));
    pl.vars = (int32_t *)take(sizeof(int32_t) * nv);
    pl.xs = (double *)take(sizeof(double) * nv * pl.S_pad);
    pl.shift = (double *)take(sizeof(double) * nv);
    pl.Sxy = (double *)take(sizeof(double) * nv * nv);
    pl.Sx = (double *)take(sizeof(double) * nv * nv);
    pl.Sxx = (double *)take(sizeof(double) * nv * nv);
    pl.nn = (int32_t *)take(sizeof(int32_t) * nv * nv);
    pl.flags = (int32_t *)take(sizeof(int32_t) * (pl.pairs + nv + 1));
    pl.counter = (int32_t *)take(sizeof(int32_t) * 4);
    pl.jobs = (PJob *)take(sizeof(PJob) * pl.pairs);
    pl.sorted = (PJob *)take(sizeof(PJob) * pl.pairs);
    pl.pj_meta = (int32_t *)take(sizeof(int32_t) * (1 + 3 * kPjBins));
    return off <= kNoAllocBytes;
}

}  // namespace napg

using namespace napg;

extern "C" napg_status napg_pearson_fp64_noalloc(const double *X, int32_t n_vars, int32_t n_samples, double missing,
                                                 double *r, double *p, int32_t *n, void *stream) {
    if (!X || n_vars < 1 || n_samples < 1) return NAPG_E_ARG;
    if (n_vars > kNoAllocMaxVars || n_samples > kNoAllocMaxSamples) return NAPG_E_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return NAPG_E_CUDA;
    void *base = nullptr;
    {
        // set-up, once per device (and again after a device reset): the array's
        // device address, looked up with this device current
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        void *owner = current_context();    // NULL before the runtime has bound one to this thread
        if (!g_noalloc_ptr[dev] || !owner || owner != g_noalloc_owner[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                (void)cudaGetLastError();
                return NAPG_E_CUDA;
            }
            g_noalloc_ptr[dev] = ptr;
            g_noalloc_owner[dev] = current_context();
        }
        base = g_noalloc_ptr[dev];
    }
    NoAllocPlan pl;
    if (!carve((unsigned char *)base, n_vars, n_samples, pl)) return NAPG_E_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nv = n_vars, S = n_samples;
    // zero what must start at zero: error word, rescue counter, p-job counter and histogram
    if (cudaMemsetAsync(pl.err, 0, sizeof(uint32_t), st) != cudaSuccess ||
        cudaMemsetAsync(pl.counter, 0, sizeof(int32_t) * 4, st) != cudaSuccess ||
        cudaMemsetAsync(pl.pj_meta, 0, sizeof(int32_t) * (1 + kPjBins), st) != cudaSuccess)
        return NAPG_E_CUDA;
    count_launch();
    k_noalloc_obs<<<dim3((unsigned)((pl.W + 7) / 8), (unsigned)nv), 256, 0, st>>>(X, nv, S, pl.W, missing, pl.obs,
                                                                                  pl.vars, pl.err);
    launch_ctx_bits(nullptr, S, pl.W, pl.ctxw, st);
    launch_shift_values(X, NAPG_F64, S, pl.S_pad, pl.vars, n_vars, pl.obs, pl.W, pl.shift, pl.xs, st);
    launch_pearson_fp64(pl.xs, pl.S_pad, pl.obs, pl.W, n_vars, pl.Sxy, pl.Sx, pl.Sxx, pl.nn, st);
    PJobQueue q{};
    if (p) {
        q.jobs = pl.jobs;
        q.count = pl.pj_meta;
        q.hist = pl.pj_meta + 1;
        q.capacity = (int32_t)pl.pairs;
    }
    PearsonFin f{pl.Sxy, pl.Sx, pl.Sxx, pl.nn, pl.shift, n_vars, kPlainRelTol, nullptr, q, nullptr};
    launch_finalize_pearson(f, r, p, n, pl.flags, pl.counter, st);
    RescueArgs rsc{X, NAPG_F64, S, pl.W, pl.ctxw, pl.obs, nullptr, nullptr, pl.vars, nullptr, n_vars, n_vars,
                   NAPG_PEARSON, 1, nullptr, nullptr, nullptr};
    launch_rescue(rsc, pl.flags, pl.counter, (int32_t)(pl.pairs + nv + 1), r, p, n, 1, 0, st);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return NAPG_E_CUDA;
    if (p) launch_pjobs_eval(q, pl.sorted, pl.pj_meta + 1 + kPjBins, pl.pj_meta + 1 + 2 * kPjBins, p, st, sms);
    if (cudaGetLastError() != cudaSuccess) return NAPG_E_CUDA;
    // the non-finite check needs the error word on the host: read it back (synchronous)
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, pl.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NAPG_E_CUDA;
    return (err & kErrNonfinite) ? NAPG_E_NONFINITE : NAPG_OK;
}
