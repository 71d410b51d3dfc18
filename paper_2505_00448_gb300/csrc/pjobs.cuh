// P-value jobs: the finalize kernels compute each pair's statistic and queue
// the p-value as a job; jobs are grouped by a key that predicts the work of the
// special-function evaluation (which function, which branch, and the size of
// the quantity that sets the continued fraction's length) so that the
// evaluation kernel's warps run lanes of similar length together.
#pragma once

#include <cstdint>

#include "specfun.cuh"

namespace napg {

enum PJobKind : int32_t { kPjCorr = 0, kPjT = 1, kPjF = 2, kPjChi2 = 3 };

struct PJob {
    double s;       // statistic (r, t, F or chi2)
    double a, b;    // n (corr); df (t); d1, d2 (F); df (chi2)
    int64_t idx;    // output index
    int32_t kind;   // PJobKind in bits 0-7, key in bits 8 and up once queued
    int32_t mirror; // > 0: also write at the transposed index of an mirror x mirror matrix
};

constexpr int kPjBins = 288;
constexpr int kPjKeyLargeA = 128;   // keys from here on: the incomplete beta's large-a expansion

struct PJobQueue {
    PJob *jobs;         // appended by the finalize kernels
    int32_t *count;     // number of jobs
    int32_t *hist;      // [kPjBins] jobs per key
    int32_t capacity;
    const double *bgrat;   // sf::bgrat_coefs rows for 2b = 1..64 (NULL: formed per job)
    sf::LargeATab lat;     // (log M, 1/T^2) on the half-integer grid (lat.v NULL: formed per job)
};

// bucket of log2(v + 1) clipped to [0, 31]
__device__ __forceinline__ int log_bucket(double v) {
    if (!(v > 0.0)) return 0;
    int e;
    frexp(v + 1.0, &e);
    return e < 0 ? 0 : (e > 31 ? 31 : e);
}

// the incomplete-beta parameters (a, b) and argument (x, y = 1 - x) of a job's
// p-value (false for the chi-squared kind, an incomplete gamma), with one
// reciprocal instead of two divisions: for the job's key and the
// certain-underflow test only, which are decided with margins far above
// rounding (the evaluation forms x and y as corr_p / t_two_sided / f_sf do)
__device__ __forceinline__ bool pjob_beta_key(const PJob &j, double &a, double &b, double &x, double &y) {
    switch (j.kind & 0xff) {
        case kPjCorr: a = 0.5 * (j.a - 2.0); b = 0.5; y = j.s * j.s; x = 1.0 - y; return true;
        case kPjT: { const double t2 = j.s * j.s, inv = 1.0 / (j.a + t2); a = 0.5 * j.a; b = 0.5; x = j.a * inv; y = t2 * inv; } return true;
        case kPjF: { const double inv = 1.0 / (j.b + j.a * j.s); a = 0.5 * j.b; b = 0.5 * j.a; x = j.b * inv; y = j.a * j.s * inv; } return true;
        default: return false;
    }
}

// key: beta continued fraction direct / swapped (32 buckets each, by the
// quantity that sets the fraction's length), gamma finite sums (32, by 2a),
// gamma series / fraction (16 each),
// and the beta large-a expansion (160 buckets: 2b up to 20, then 8 octaves of
// a y, which sets u = -T ln x and with it the branches and the term count).
// The branch tests mirror sf::ibeta and sf::gamma_q.
__device__ __forceinline__ int pjob_key(const PJob &j, bool beta, double a, double b, double x, double y) {
    if (!beta) {
        const double ga = 0.5 * j.a, gx = 0.5 * j.s;
        // finite sums (sf::gamma_q_ladder): work grows with 2a
        if (gx > 0.0 && sf::gamma_ladder_applies(ga)) return 64 + min(31, (int)(2.0 * ga) >> 1);
        return (gx < ga + 1.0 ? 96 : 112) + (log_bucket(gx < ga + 1.0 ? gx : ga / (gx + 1e-300) * 32.0) >> 1);
    }
    if (sf::ibeta_large_a_applies(a, b, x))
        return kPjKeyLargeA + (min(20, (int)(2.0 * b)) - 1) * 8 + min(7, log_bucket(a * y) >> 1);
    const bool swapped = x > (a + 1.0) / (a + b + 2.0);
    return (swapped ? 32 : 0) + log_bucket(swapped ? b * x : a * y);
}

// Appends a job. Lanes of a warp that push together take their slots with one
// atomic, and lanes with equal keys add to the histogram with one atomic (many
// jobs share a key). The key is kept in the job's kind word (bits 8 and up) for
// the scatter.
__device__ __forceinline__ void pjob_push(const PJobQueue &q, PJob j, int k) {
    j.kind |= k << 8;
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(q.count, __popc(act));
    base = __shfl_sync(act, base, leader);
    const int slot = base + __popc(act & ((1u << lane) - 1u));
    if (slot < q.capacity) q.jobs[slot] = j;
    const unsigned same = __match_any_sync(act, k);
    if (lane == __ffs(same) - 1) atomicAdd(&q.hist[k], __popc(same));
}

__device__ __forceinline__ void pjob_push(const PJobQueue &q, const PJob &j) {
    double a = 0, b = 0, x = 0, y = 0;
    const bool beta = pjob_beta_key(j, a, b, x, y);
    pjob_push(q, j, pjob_key(j, beta, a, b, x, y));
}

// Queues the job and returns NaN (its p-value is written by the evaluation), or
// returns the p-value 0 at once when it certainly underflows (sf::ibeta_underflows).
__device__ __forceinline__ double pjob_push_p(const PJobQueue &q, const PJob &j) {
    double a = 0, b = 0, x = 0, y = 0;
    const bool beta = pjob_beta_key(j, a, b, x, y);
    if (beta && isfinite(j.s) && sf::ibeta_underflows(a, b, y)) return 0.0;
    pjob_push(q, j, pjob_key(j, beta, a, b, x, y));
    return __longlong_as_double(0x7ff8000000000000LL);
}

// pjob_push_p for a correlation job (statistic r, n observations), b = 1/2:
// the job's placement (its key and the certain-underflow test) in FP32. Both
// are decided with margins far above FP32 rounding: a job that lands on the
// other side of a key boundary is evaluated by a branch that is accurate there
// too (the large-a expansion also holds just below x = 1/2, and the general
// path re-derives its own branch), and one that lands on the other side of an
// underflow threshold has p below 1e-320 either way. The finalize kernels are
// bound by the FP64 pipe, which this leaves to the statistic.
__device__ __forceinline__ double pjob_push_corr(const PJobQueue &q, double r, double n, int64_t idx,
                                                 int32_t mirror) {
    const float rf = (float)r, nf = (float)n;
    const float a = 0.5f * nf - 1.0f, y = rf * rf, x = 1.0f - y, ay = a * y;
    if (a >= 20.0f && ((y <= 0.5f && (a - 0.25f) * y >= 746.5f) || ay >= 2001.0f)) return 0.0;
    int k;
    if (x >= 0.5f && a >= 20.0f) {
        k = kPjKeyLargeA + min(7, log_bucket((double)ay) >> 1);
    } else {
        const bool swapped = x > (a + 1.0f) / (a + 2.5f);
        k = (swapped ? 32 : 0) + log_bucket((double)(swapped ? 0.5f * x : ay));
    }
    pjob_push(q, PJob{r, n, 0.0, idx, kPjCorr, mirror}, k);
    return __longlong_as_double(0x7ff8000000000000LL);
}

// The same for an F job (statistic F, degrees of freedom d1, d2): x, y and the
// tests in FP32 where d2 + d1 F is within its range, else the generic path.
__device__ __forceinline__ double pjob_push_f(const PJobQueue &q, double F, double d1, double d2, int64_t idx) {
    const PJob j{F, d1, d2, idx, kPjF, 0};
    const double v = d2 + d1 * F;
    if (!(v >= 1e-30 && v <= 1e30)) return pjob_push_p(q, j);
    const float inv = __frcp_rn((float)v), a = 0.5f * (float)d2, b = 0.5f * (float)d1;
    const float y = (float)(d1 * F) * inv, x = (float)d2 * inv;
    if (a >= 20.0f && b <= 32.0f && ((b == 0.5f && y <= 0.5f && (a - 0.25f) * y >= 746.5f) || a * y >= 2001.0f))
        return 0.0;
    int k;
    if (x >= 0.5f && a >= 20.0f && b <= 32.0f && b <= a) {
        k = kPjKeyLargeA + (min(20, (int)(2.0f * b)) - 1) * 8 + min(7, log_bucket((double)(a * y)) >> 1);
    } else {
        const bool swapped = x > (a + 1.0f) / (a + b + 2.0f);
        k = (swapped ? 32 : 0) + log_bucket((double)(swapped ? b * x : a * y));
    }
    pjob_push(q, j, k);
    return __longlong_as_double(0x7ff8000000000000LL);
}

}  // namespace napg
