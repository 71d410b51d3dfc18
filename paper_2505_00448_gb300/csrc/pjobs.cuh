// P-value jobs: the finalize kernels compute each pair's statistic and queue
// the p-value as a job; jobs are grouped by a key that predicts the work of the
// special-function evaluation (which function, which branch, and the size of
// the quantity that sets the continued fraction's length) so that the
// evaluation kernel's warps run lanes of similar length together.
#pragma once

#include <cstdint>

namespace napg {

enum PJobKind : int32_t { kPjCorr = 0, kPjT = 1, kPjF = 2, kPjChi2 = 3 };

struct PJob {
    double s;       // statistic (r, t, F or chi2)
    double a, b;    // n (corr); df (t); d1, d2 (F); df (chi2)
    int64_t idx;    // output index
    int32_t kind;
    int32_t mirror; // > 0: also write at the transposed index of an mirror x mirror matrix
};

constexpr int kPjBins = 128;

struct PJobQueue {
    PJob *jobs;         // appended by the finalize kernels
    int32_t *count;     // number of jobs
    int32_t *hist;      // [kPjBins] jobs per key
    int32_t capacity;
};

// bucket of log2(v + 1) clipped to [0, 31]
__device__ __forceinline__ int log_bucket(double v) {
    if (!(v > 0.0)) return 0;
    int e;
    frexp(v + 1.0, &e);
    return e < 0 ? 0 : (e > 31 ? 31 : e);
}

// key: 4 families (beta direct, beta swapped, gamma series, gamma fraction) x 32 buckets
__device__ __forceinline__ int pjob_key(const PJob &j) {
    double a = 0, b = 0, x = 0, y = 0;
    switch (j.kind) {
        case kPjCorr: a = 0.5 * (j.a - 2.0); b = 0.5; y = j.s * j.s; x = 1.0 - y; break;
        case kPjT: { const double t2 = j.s * j.s; a = 0.5 * j.a; b = 0.5; x = j.a / (j.a + t2); y = t2 / (j.a + t2); } break;
        case kPjF: { const double den = j.b + j.a * j.s; a = 0.5 * j.b; b = 0.5 * j.a; x = j.b / den; y = j.a * j.s / den; } break;
        default: {
            const double ga = 0.5 * j.a, gx = 0.5 * j.s;
            return (gx < ga + 1.0 ? 64 : 96) + log_bucket(gx < ga + 1.0 ? gx : ga / (gx + 1e-300) * 32.0);
        }
    }
    const bool swapped = x > (a + 1.0) / (a + b + 2.0);
    return (swapped ? 32 : 0) + log_bucket(swapped ? b * x : a * y);
}

__device__ __forceinline__ void pjob_push(const PJobQueue &q, const PJob &j) {
    const int k = pjob_key(j);
    const int slot = atomicAdd(q.count, 1);
    if (slot < q.capacity) q.jobs[slot] = j;
    atomicAdd(&q.hist[k], 1);
}

}  // namespace napg
