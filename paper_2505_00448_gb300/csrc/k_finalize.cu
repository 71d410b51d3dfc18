// Finalize: statistic, edge rules and p-value per pair (Sec. 3.5), in FP64,
// from the moments, tables or rank sums the contraction kernels produced.
// Pairs whose sums are numerically degenerate (a variance that vanishes against
// the raw second moment: a constant column or group on the co-observed samples)
// are queued for an exact FP64 two-pass recomputation (k_rescue) instead.
#include "napg_internal.cuh"
#include "specfun.cuh"

namespace napg {

__device__ __forceinline__ double dnan() { return __longlong_as_double(0x7ff8000000000000LL); }

// Mixed form: the planes carry 22 bits relative to each row's largest value;
// over few co-observed samples the centred sums can cancel without the errors
// averaging out, so such pairs are recomputed exactly (cheap at that size).
constexpr int32_t kMixedMinN = 64;
__device__ __forceinline__ double dinf() { return __longlong_as_double(0x7ff0000000000000LL); }

// 1/n for a count n >= 1: the FP32 reciprocal of the FP32 count (relative error
// below 2^-22, also where the count rounds), refined by two Newton steps
// r <- r (2 - n r) in FP64 (each squares the relative error: below 2^-88), so
// within a unit or two in the last place: five FP64 instructions where a
// division takes about a dozen (the finalize kernels are bound by the FP64 pipe)
__device__ __forceinline__ double rcp_count(int32_t n) {
    const double nd = (double)n;
    double r = (double)__frcp_rn(__int2float_rn(n));
    r *= fma(-nd, r, 2.0);
    r *= fma(-nd, r, 2.0);
    return r;
}

// 1/n with one Newton step (relative error below 2^-45): for sums of positive
// terms, where no cancellation magnifies it (the chi-squared cells)
__device__ __forceinline__ double rcp_count1(int32_t n) {
    const double r = (double)__frcp_rn(__int2float_rn(n));
    return r * fma(-(double)n, r, 2.0);
}

__device__ __forceinline__ void put(double *stat, double *pval, int32_t *nout, int64_t idx, double s, double p,
                                    int32_t n) {
    if (stat) stat[idx] = s;
    if (pval) pval[idx] = p;
    if (nout) nout[idx] = n;
}

// ------------------------------------------------------------------ Pearson --
// One CTA per upper-triangle tile (I <= J) of 32 x 32 pairs. The (j, i) sums
// come from the mirrored tile, read row by row and transposed in shared memory,
// and the (j, i) outputs go back the same way, so every global access runs
// along a row.
constexpr int kFinT = 32;

__global__ void __launch_bounds__(256) k_finalize_pearson(PearsonFin f, double *stat, double *pval, int32_t *nout,
                                                          int32_t *flags, int32_t *nflag) {
    const int nv = f.nv;
    const int T = (nv + kFinT - 1) / kFinT;
    int t = blockIdx.x, I = 0;
    while (t >= T - I) { t -= T - I; ++I; }
    const int J = I + t;
    if (!rows_owned(f.own, (int64_t)I * kFinT, kFinT, nv)) return;   // another part's rows
    __shared__ double m_sx[kFinT][kFinT + 1], m_sxx[kFinT][kFinT + 1];   // mirrored tile (rows j, columns i)
    __shared__ double o_r[kFinT][kFinT + 1], o_p[kFinT][kFinT + 1];      // outputs by (i, j) for the mirror
    __shared__ int32_t o_n[kFinT][kFinT + 1];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int i0 = I * kFinT, j0 = J * kFinT;
    for (int ry = ly; ry < kFinT; ry += 8) {
        const int j = j0 + ry, i = i0 + lx;
        if (j < nv && i < nv) {
            m_sx[ry][lx] = f.Sx[(int64_t)j * nv + i];
            m_sxx[ry][lx] = f.Sxx[(int64_t)j * nv + i];
        }
    }
    __syncthreads();
    for (int ry = ly; ry < kFinT; ry += 8) {
        const int i = i0 + ry, j = j0 + lx;
        double r = dnan(), p = dnan();
        int32_t n = 0;
        if (i < nv && j < nv && (I != J || i <= j)) {
            const int64_t ij = (int64_t)i * nv + j;
            n = f.nn[ij];
            if (n > 1) {
                const double nd = (double)n, inv_n = rcp_count(n);
                const double sx = f.Sx[ij], sy = m_sx[lx][ry], sxy = f.Sxy[ij];
                const double sxx = f.vsq ? f.Sxx[ij] + f.vsq[i] * nd : f.Sxx[ij];
                const double syy = f.vsq ? m_sxx[lx][ry] + f.vsq[j] * nd : m_sxx[lx][ry];
                const double cxx = sxx - sx * sx * inv_n, cyy = syy - sy * sy * inv_n, cxy = sxy - sx * sy * inv_n;
                if (!(cxx > f.rel_tol * sxx) || !(cyy > f.rel_tol * syy) || (f.vsq && n < kMixedMinN)) {
                    const int q = atomicAdd(nflag, 1);
                    flags[q] = (int32_t)ij;
                } else {
                    // a variable against itself: r = 1 exactly, as the two-pass
                    // definition gives (its centred cross sum is its sum of squares)
                    const bool same = f.vars ? f.vars[i] == f.vars[j] : i == j;
                    r = same ? 1.0 : cxy * rsqrt(cxx * cyy);
                    r = fmin(1.0, fmax(-1.0, r));
                    if (n <= 2) p = dnan();
                    else if (fabs(r) >= 1.0) p = 0.0;
                    else if (f.q.jobs) p = pjob_push_corr(f.q, r, nd, ij, (int32_t)nv);
                }
            }
            put(stat, pval, nout, ij, r, p, n);       // p of a queued job is written by the evaluation
        }
        o_r[ry][lx] = r;
        o_p[ry][lx] = p;
        o_n[ry][lx] = n;
    }
    __syncthreads();
    // the mirrored outputs (j, i), i < j: row j of the (J, I) tile
    for (int ry = ly; ry < kFinT; ry += 8) {
        const int j = j0 + ry, i = i0 + lx;
        if (i < nv && j < nv && (I != J || i < j))
            put(stat, pval, nout, (int64_t)j * nv + i, o_r[lx][ry], o_p[lx][ry], o_n[lx][ry]);
    }
}

void launch_finalize_pearson(const PearsonFin &f, double *stat, double *pval, int32_t *nout, int32_t *flag_list,
                             int32_t *flag_count, cudaStream_t st) {
    if (f.nv == 0) return;
    const int64_t T = (f.nv + kFinT - 1) / kFinT;
    count_launch();
    k_finalize_pearson<<<(unsigned)(T * (T + 1) / 2), 256, 0, st>>>(f, stat, pval, nout, flag_list, flag_count);
}

// --------------------------------------------------- ANOVA / Welch / Student --
__global__ void k_finalize_groups(GroupFin f, double *stat, double *pval, int32_t *nout, int32_t *flags,
                                  int32_t *nflag) {
    const int64_t total = (int64_t)f.na * f.nb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / f.nb), j = (int)(t - (int64_t)a * f.nb);
        const int c = f.nlev[a], off = f.levoff[a];
        int64_t n = 0;
        int k = 0;
        bool empty = false;
        for (int g = 0; g < c; ++g) {
            const int32_t ng = f.gn[(int64_t)(off + g) * f.nb + j];
            n += ng;
            if (f.present[off + g]) {
                ++k;
                if (ng == 0) empty = true;
            }
        }
        double s = dnan(), p = dnan(), es = dnan(), dof = dnan();
        if (f.test == NAPG_ANOVA) {
            if (!empty && k >= 2 && n - k >= 1) {
                double s1 = 0.0, raw = 0.0;
                for (int g = 0; g < c; ++g) {
                    const int64_t idx = (int64_t)(off + g) * f.nb + j;
                    s1 += f.g1[idx];
                    if (!f.g2tot) raw += f.g2[idx] + (f.vsq ? f.vsq[j] * (double)f.gn[idx] : 0.0);
                }
                // sum of squares over all co-observed samples: per level, or one total
                if (f.g2tot) raw = f.g2tot[t] + (f.vsq ? f.vsq[j] * (double)n : 0.0);
                const double gm = s1 * rcp_count((int32_t)n);
                double ssb = 0.0, ssw = f.g2tot ? raw : 0.0;
                for (int g = 0; g < c; ++g) {
                    if (!f.present[off + g]) continue;
                    const int64_t idx = (int64_t)(off + g) * f.nb + j;
                    const int32_t ngi = f.gn[idx];
                    const double ng = (double)ngi, mg = f.g1[idx] * rcp_count(ngi);
                    ssb += ng * (mg - gm) * (mg - gm);
                    if (f.g2tot) {
                        ssw -= f.g1[idx] * mg;
                    } else {
                        const double s2 = f.g2[idx] + (f.vsq ? f.vsq[j] * ng : 0.0);
                        ssw += s2 - f.g1[idx] * mg;
                    }
                }
                if (!(ssw > f.rel_tol * raw) || (f.vsq && n < kMixedMinN)) {
                    flags[atomicAdd(nflag, 1)] = (int32_t)t;
                } else {
                    const double d1 = (double)(k - 1), d2 = (double)(n - k);
                    s = (ssb * d2) / (ssw * d1);          // (ssb / d1) / (ssw / d2), one division
                    if (f.q.jobs) p = pjob_push_f(f.q, s, d1, d2, t);
                }
            }
        } else {  // two-sample t (levels 0 and 1)
            const int64_t i0 = (int64_t)off * f.nb + j, i1 = (int64_t)(off + 1) * f.nb + j;
            const int32_t n0 = f.gn[i0], n1 = f.gn[i1];
            if (n0 >= 2 && n1 >= 2 && n >= 3) {
                const double m0 = f.g1[i0] * rcp_count(n0), m1 = f.g1[i1] * rcp_count(n1);
                const double r0 = f.g2[i0] + (f.vsq ? f.vsq[j] * (double)n0 : 0.0);
                const double r1 = f.g2[i1] + (f.vsq ? f.vsq[j] * (double)n1 : 0.0);
                const double q0 = r0 - f.g1[i0] * m0, q1 = r1 - f.g1[i1] * m1;
                if (!(q0 > f.rel_tol * r0) || !(q1 > f.rel_tol * r1) || (f.vsq && n < kMixedMinN)) {
                    flags[atomicAdd(nflag, 1)] = (int32_t)t;
                } else if (f.welch) {
                    const double e0 = q0 / (double)(n0 - 1) / (double)n0, e1 = q1 / (double)(n1 - 1) / (double)n1;
                    const double se2 = e0 + e1;
                    s = (m0 - m1) / sqrt(se2);
                    const double nu = se2 * se2 / (e0 * e0 / (double)(n0 - 1) + e1 * e1 / (double)(n1 - 1));
                    if (f.q.jobs) p = pjob_push_p(f.q, PJob{s, nu, 0.0, t, kPjT, 0});
                    // Cohen's d over the mean of the two variances
                    es = (m0 - m1) / sqrt(0.5 * (q0 / (double)(n0 - 1) + q1 / (double)(n1 - 1)));
                    dof = nu;
                } else {
                    const double df = (double)(n - 2);
                    const double sp2 = (q0 + q1) / df;
                    s = (m0 - m1) / sqrt(sp2 * (1.0 / n0 + 1.0 / n1));
                    if (f.q.jobs) p = pjob_push_p(f.q, PJob{s, df, 0.0, t, kPjT, 0});
                    es = (m0 - m1) / sqrt(sp2);      // Cohen's d over the pooled SD
                    dof = df;
                }
            }
        }
        put(stat, pval, nout, t, s, p, (int32_t)n);
        if (f.es) f.es[t] = es;
        if (f.es2) f.es2[t] = dof;
    }
}

void launch_finalize_groups(const GroupFin &f, double *stat, double *pval, int32_t *nout, int32_t *flag_list,
                            int32_t *flag_count, cudaStream_t st) {
    const int64_t total = (int64_t)f.na * f.nb;
    if (total == 0) return;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 127) / 128, 152 * 32);
    count_launch();
    k_finalize_groups<<<blocks, 128, 0, st>>>(f, stat, pval, nout, flag_list, flag_count);
}

// -------------------------------------------------------------- chi-squared --
// One thread per pair (the upper triangle only, for symmetric calls). Each cell
// contributes (O - E)^2 / E = (n O - r c)^2 / (n r c): the centred numerator is
// exact in integers and the reciprocals of n and of the margins are formed once,
// so no cell divides. MAXC bounds the levels per variable: tables up to 16 x 16
// keep their margins in registers (fully unrolled, predicated loops); larger
// ones run the same body without unrolling.
#define NAPG_CHI2_KERNEL(NAME, MAXC, UNROLL) \
__global__ void NAME(Chi2Fin f, double *stat, double *pval, int32_t *nout) { \
    const int64_t nn = f.na; \
    const int64_t total = f.symmetric ? nn * (nn + 1) / 2 : (int64_t)f.na * f.nb; \
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; \
         t += (int64_t)gridDim.x * blockDim.x) { \
        int a, b; \
        if (f.symmetric) { \
            /* row from an FP32 estimate, corrected exactly in integers below */ \
            const float q2 = (float)(2 * nn + 1); \
            int64_t i = (int64_t)((q2 - sqrtf(fmaxf(q2 * q2 - 8.0f * (float)t, 0.0f))) * 0.5f); \
            if (i < 0) i = 0; \
            if (i > nn - 1) i = nn - 1; \
            while (i > 0 && i * (2 * nn - i + 1) / 2 > t) --i; \
            while ((i + 1) * (2 * nn - i) / 2 <= t) ++i; \
            a = (int)i; \
            b = (int)(i + (t - i * (2 * nn - i + 1) / 2)); \
        } else { \
            a = (int)(t / f.nb); \
            b = (int)(t - (int64_t)a * f.nb); \
        } \
        if (f.symmetric && f.own && !f.own[a]) continue;   /* another part's row */ \
        const int64_t ab = (int64_t)a * f.nb + b; \
        const int ca = f.nlev_a[a], cb = f.nlev_b[b]; \
        const int oa = f.levoff_a[a], ob = f.levoff_b[b]; \
        const int32_t *Tb = f.T + (int64_t)oa * f.R + ob; \
        int32_t row[MAXC], col[MAXC]; \
UNROLL \
        for (int g = 0; g < MAXC; ++g) { row[g] = 0; col[g] = 0; } \
        int64_t n = 0; \
UNROLL \
        for (int g = 0; g < MAXC; ++g) { \
            if (g >= ca) break; \
UNROLL \
            for (int h = 0; h < MAXC; ++h) { \
                if (h >= cb) break; \
                const int32_t o = Tb[(int64_t)g * f.R + h]; \
                row[g] += o; \
                col[h] += o; \
                n += o; \
            } \
        } \
        int ka = 0, kb = 0; \
        bool empty = (n == 0); \
UNROLL \
        for (int g = 0; g < MAXC; ++g) \
            if (g < ca && f.present[oa + g]) { ++ka; if (row[g] == 0) empty = true; } \
UNROLL \
        for (int h = 0; h < MAXC; ++h) \
            if (h < cb && f.present[ob + h]) { ++kb; if (col[h] == 0) empty = true; } \
        double s = dnan(), p = dnan(); \
        if (!empty) { \
            const bool yates = f.yates && ka == 2 && kb == 2; \
            const double nd = (double)n, inv_n = rcp_count1((int32_t)n); \
            double icol[MAXC]; \
UNROLL \
            for (int h = 0; h < MAXC; ++h) icol[h] = (h < cb && col[h] > 0) ? rcp_count1(col[h]) : 0.0; \
            double chi = 0.0; \
UNROLL \
            for (int g = 0; g < MAXC; ++g) { \
                if (g >= ca) break; \
                if (!f.present[oa + g]) continue; \
                const double irow = rcp_count1(row[g]); \
                double acc = 0.0; \
UNROLL \
                for (int h = 0; h < MAXC; ++h) { \
                    if (h >= cb) break; \
                    if (!f.present[ob + h]) continue; \
                    const int64_t D = n * (int64_t)Tb[(int64_t)g * f.R + h] - (int64_t)row[g] * col[h];   /* exact */ \
                    double d = fabs((double)D); \
                    if (yates) d = fmax(d - 0.5 * nd, 0.0);      /* |O - E| - 1/2, times n */ \
                    acc += d * d * icol[h]; \
                } \
                chi += acc * irow; \
            } \
            s = chi * inv_n; \
            const int df = (ka - 1) * (kb - 1); \
            if (df > 0 && f.q.jobs) pjob_push(f.q, PJob{s, (double)df, 0.0, ab, kPjChi2, f.symmetric ? f.nb : 0}); \
        } \
        put(stat, pval, nout, ab, s, p, (int32_t)n); \
        if (f.symmetric && a != b) put(stat, pval, nout, (int64_t)b * f.nb + a, s, p, (int32_t)n); \
    } \
}

NAPG_CHI2_KERNEL(k_finalize_chi2_small, 16, _Pragma("unroll"))
NAPG_CHI2_KERNEL(k_finalize_chi2_large, kMaxLevels, _Pragma("unroll 1"))
#undef NAPG_CHI2_KERNEL

void launch_finalize_chi2(const Chi2Fin &f, double *stat, double *pval, int32_t *nout, cudaStream_t st) {
    const int64_t total = f.symmetric ? (int64_t)f.na * (f.na + 1) / 2 : (int64_t)f.na * f.nb;
    if (total == 0) return;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 127) / 128, 152 * 32);
    count_launch();
    if (f.maxc <= 16) k_finalize_chi2_small<<<blocks, 128, 0, st>>>(f, stat, pval, nout);
    else k_finalize_chi2_large<<<blocks, 128, 0, st>>>(f, stat, pval, nout);
}

// ----------------------------------------------------------------- Spearman --
__global__ void k_finalize_spearman(SpearmanFin f, double *stat, double *pval, int32_t *nout) {
    const int64_t total = (int64_t)f.na * f.nb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / f.nb), b = (int)(t - (int64_t)a * f.nb);
        if (f.symmetric && b < a) continue;
        if (f.symmetric && f.own && !f.own[a]) continue;   // another part's row
        const int64_t *q = f.q + 4 * t;
        const int64_t n = q[0];
        double r = dnan(), p = dnan();
        if (n > 1) {
            // doubled ranks A = 2Rx, B = 2Ry: sum A = sum B = n(n+1) = K
            const __int128 K = (__int128)n * (n + 1);
            const __int128 num = (__int128)n * q[1] - K * K;
            const __int128 da = (__int128)n * q[2] - K * K;
            const __int128 db = (__int128)n * q[3] - K * K;
            if (da > 0 && db > 0) {
                // identical or reversed rankings (|rho| = 1) decided exactly in integers
                if (da == db && (num == da || num == -da)) r = num > 0 ? 1.0 : -1.0;
                else r = (double)num / (sqrt((double)da) * sqrt((double)db));
                r = fmin(1.0, fmax(-1.0, r));
                if (n <= 2) p = dnan();
                else if (fabs(r) >= 1.0) p = 0.0;
                else if (f.pq.jobs) p = pjob_push_corr(f.pq, r, (double)n, t, f.symmetric ? f.nb : 0);
            }
        }
        put(stat, pval, nout, t, r, p, (int32_t)n);
        if (f.symmetric && a != b) put(stat, pval, nout, (int64_t)b * f.nb + a, r, p, (int32_t)n);
    }
}

void launch_finalize_spearman(const SpearmanFin &f, double *stat, double *pval, int32_t *nout, cudaStream_t st) {
    const int64_t total = (int64_t)f.na * f.nb;
    if (total == 0) return;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 127) / 128, 152 * 32);
    count_launch();
    k_finalize_spearman<<<blocks, 128, 0, st>>>(f, stat, pval, nout);
}

// ------------------------------------------------------------ MWU / Kruskal --
__global__ void k_finalize_rankgroups(RankGroupFin f, double *stat, double *pval, int32_t *nout, int32_t *flags,
                                      int32_t *nflag) {
    const int64_t total = (int64_t)f.na * f.nb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / f.nb), j = (int)(t - (int64_t)a * f.nb);
        const int c = f.nlev[a], off = f.levoff[a];
        int64_t n = 0;
        int k = 0;
        bool empty = false;
        for (int g = 0; g < c; ++g) {
            const int32_t ng = f.rcnt[(int64_t)(off + g) * f.nb + j];
            n += ng;
            if (f.present[off + g]) { ++k; if (ng == 0) empty = true; }
        }
        const int64_t T = f.tie_term[t];
        double s = dnan(), p = dnan();
        if (f.test == NAPG_MWU) {
            const int64_t i0 = (int64_t)off * f.nb + j, i1 = (int64_t)(off + 1) * f.nb + j;
            const int64_t n0 = f.rcnt[i0], n1 = f.rcnt[i1];
            if (n0 > 0 && n1 > 0) {
                const int64_t two_u0 = f.rsum[i0] - n0 * (n0 + 1);   // 2 U0 (exact)
                const int64_t two_nn = 2 * n0 * n1;
                const int64_t two_u = two_u0 > two_nn - two_u0 ? two_u0 : two_nn - two_u0;
                s = 0.5 * (double)two_u0;
                const bool exact = f.mwu_mode == 1 || (f.mwu_mode == 0 && T == 0 && (n0 < 8 || n1 < 8));
                if (exact) {
                    flags[atomicAdd(nflag, 1)] = (int32_t)t;
                } else {
                    const int64_t num = n * n * n - n - T;           // 12 n (n-1) sigma^2 / (n0 n1)
                    if (num > 0) {
                        const double sigma = sqrt((double)n0 * (double)n1 * (double)num /
                                                  (12.0 * (double)n * (double)(n - 1)));
                        const double cc = f.mwu_cc ? 1.0 : 0.0;
                        const double z = ((double)(two_u - n0 * n1) - cc) / (2.0 * sigma);
                        p = fmin(1.0, 2.0 * sf::norm_sf(z));
                    }
                }
            }
        } else {  // Kruskal-Wallis
            if (!empty && k >= 2) {
                const int64_t denom = n * n * n - n;
                const int64_t cnum = denom - T;
                if (cnum > 0) {
                    double acc = 0.0;
                    for (int g = 0; g < c; ++g) {
                        if (!f.present[off + g]) continue;
                        const int64_t idx = (int64_t)(off + g) * f.nb + j;
                        const int64_t ng = f.rcnt[idx];
                        const double D = (double)(f.rsum[idx] - ng * (n + 1));   // 2 n_g (Rbar_g - (n+1)/2)
                        acc += D * D / (double)ng;
                    }
                    const double h0 = 3.0 * acc / ((double)n * (double)(n + 1));
                    s = h0 / ((double)cnum / (double)denom);
                    if (f.q.jobs) pjob_push(f.q, PJob{s, (double)(k - 1), 0.0, t, kPjChi2, 0});
                }
            }
        }
        put(stat, pval, nout, t, s, p, (int32_t)n);
    }
}

void launch_finalize_rankgroups(const RankGroupFin &f, double *stat, double *pval, int32_t *nout,
                                int32_t *flag_list, int32_t *flag_count, cudaStream_t st) {
    const int64_t total = (int64_t)f.na * f.nb;
    if (total == 0) return;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 127) / 128, 152 * 32);
    count_launch();
    k_finalize_rankgroups<<<blocks, 128, 0, st>>>(f, stat, pval, nout, flag_list, flag_count);
}

// ---------------------------------------------------------- exact rescue --
// One thread per queued pair: the textbook two-pass computation over the
// co-observed samples read straight from the cohort, with exact constancy
// checks (a constant column or group is detected by comparing values, not by a
// rounded variance).
template <typename T>
__device__ double load_val(const void *X, int64_t idx) { return (double)((const T *)X)[idx]; }

__device__ __forceinline__ double xval(const RescueArgs &r, int64_t idx) {
    return r.dtype == NAPG_F32 ? load_val<float>(r.X, idx) : load_val<double>(r.X, idx);
}

__device__ __forceinline__ bool bit(const uint32_t *w, int64_t s) { return (w[s >> 5] >> (s & 31)) & 1u; }

// The p-value of a rescued pair with statistic s and parameters a, b (n for r;
// d1, d2 for F; the degrees of freedom for t). With a job queue the pair's job
// joins the others (the evaluation kernels write p; 0 at once when it certainly
// underflows), so that one thread of the rescue does not run the special
// function alone while its block waits; without one it is formed here.
__device__ __forceinline__ double rescue_p(const RescueArgs &r, int kind, double s, double a, double b, int64_t idx,
                                           int32_t mirror) {
    if (kind == kPjCorr && fabs(s) >= 1.0) return 0.0;
    if (r.q.jobs) return pjob_push_p(r.q, PJob{s, a, b, idx, kind, mirror});
    if (kind == kPjCorr) return sf::corr_p(s, a);
    if (kind == kPjF) return sf::f_sf(s, a, b);
    return sf::t_two_sided(s, a);
}

// f(k) for this thread's share of the samples k < S set in ctx, oa and ob: one
// 32-sample word per thread and step, the set samples of each byte of the word
// in one unrolled group, so that their loads are in flight together (a loop
// over single samples waits out one memory latency per sample). The order in
// which a thread visits its samples is fixed, so the sums are reproducible.
template <typename F>
__device__ __forceinline__ void for_co_observed(const uint32_t *ctxw, const uint32_t *oa, const uint32_t *ob,
                                                int64_t S, F &&f) {
    const int64_t W = (S + 31) >> 5;
    for (int64_t w = threadIdx.x; w < W; w += blockDim.x) {
        uint32_t m = ctxw[w] & oa[w] & ob[w];
        if (w == W - 1 && (S & 31)) m &= (1u << (S & 31)) - 1u;
        if (!m) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t bq = (m >> (8 * q)) & 0xffu;
            if (!bq) continue;
#pragma unroll
            for (int b = 0; b < 8; ++b)
                if ((bq >> b) & 1u) f(w * 32 + 8 * q + b);
        }
    }
}

__global__ void k_rescue(RescueArgs r, const int32_t *flags, const int32_t *nflag, int32_t max_flags,
                         double *stat, double *pval, int32_t *nout, int32_t symmetric) {
    const int32_t cnt = min(*nflag, max_flags);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
        const int64_t t = flags[q];
        const int ncols = symmetric ? r.na : r.nb;
        const int ia = (int)(t / ncols), ib = (int)(t - (int64_t)ia * ncols);
        const int va = r.va[ia], vb = symmetric ? r.va[ib] : r.vb[ib];
        const uint32_t *oa = r.obs + (int64_t)va * r.W, *ob = r.obs + (int64_t)vb * r.W;
        double s = dnan(), p = dnan();
        if (r.test == NAPG_PEARSON) {
            int64_t n = 0;
            double mx = 0.0, my = 0.0, fx = 0.0, fy = 0.0;
            bool cx = true, cy = true;
            for (int64_t k = 0; k < r.S; ++k) {
                if (!(bit(r.ctxw, k) && bit(oa, k) && bit(ob, k))) continue;
                const double x = xval(r, (int64_t)va * r.S + k), y = xval(r, (int64_t)vb * r.S + k);
                if (n == 0) { fx = x; fy = y; } else { cx &= (x == fx); cy &= (y == fy); }
                mx += x; my += y; ++n;
            }
            if (n > 1 && !cx && !cy) {
                mx /= (double)n; my /= (double)n;
                double sxx = 0.0, syy = 0.0, sxy = 0.0;
                for (int64_t k = 0; k < r.S; ++k) {
                    if (!(bit(r.ctxw, k) && bit(oa, k) && bit(ob, k))) continue;
                    const double dx = xval(r, (int64_t)va * r.S + k) - mx, dy = xval(r, (int64_t)vb * r.S + k) - my;
                    sxx += dx * dx; syy += dy * dy; sxy += dx * dy;
                }
                s = (va == vb) ? 1.0 : fmin(1.0, fmax(-1.0, sxy / (sqrt(sxx) * sqrt(syy))));
                p = (n <= 2) ? dnan() : rescue_p(r, kPjCorr, s, (double)n, 0.0, t, symmetric ? ncols : 0);
            }
            put(stat, pval, nout, t, s, p, (int32_t)n);
            if (symmetric) put(stat, pval, nout, (int64_t)ib * ncols + ia, s, p, (int32_t)n);
            continue;
        }
        // group tests: a categorical (labels), b continuous
        const uint8_t *la = r.lab + (int64_t)r.catrow[ia] * r.S;
        const int c = r.nlev_a[ia], off = r.levoff[ia];
        int64_t ng[kMaxLevels];
        double sum[kMaxLevels], first[kMaxLevels], ss[kMaxLevels];
        bool cst[kMaxLevels];
        for (int g = 0; g < c; ++g) { ng[g] = 0; sum[g] = 0.0; first[g] = 0.0; ss[g] = 0.0; cst[g] = true; }
        int64_t n = 0;
        double tot = 0.0;
        for (int64_t k = 0; k < r.S; ++k) {
            if (!(bit(r.ctxw, k) && bit(oa, k) && bit(ob, k))) continue;
            const int g = la[k];
            const double y = xval(r, (int64_t)vb * r.S + k);
            if (ng[g] == 0) first[g] = y; else cst[g] &= (y == first[g]);
            sum[g] += y; ng[g] += 1; tot += y; ++n;
        }
        double mean[kMaxLevels];                 // the level means, formed once
        for (int g = 0; g < c; ++g) mean[g] = ng[g] > 0 ? sum[g] / (double)ng[g] : 0.0;
        for (int64_t k = 0; k < r.S; ++k) {
            if (!(bit(r.ctxw, k) && bit(oa, k) && bit(ob, k))) continue;
            const int g = la[k];
            const double d = xval(r, (int64_t)vb * r.S + k) - mean[g];
            ss[g] += d * d;
        }
        for (int g = 0; g < c; ++g) if (cst[g]) ss[g] = 0.0;
        if (r.test == NAPG_ANOVA) {
            int k = 0;
            bool all_const = true, differ = false;
            double ref = 0.0;
            bool have_ref = false;
            for (int g = 0; g < c; ++g) {
                if (!r.present[off + g]) continue;
                ++k;
                all_const &= cst[g];
                if (!have_ref) { ref = first[g]; have_ref = true; } else if (first[g] != ref) differ = true;
            }
            if (all_const) {
                if (differ) { s = dinf(); p = 0.0; }
            } else {
                const double gm = tot / (double)n;
                double ssb = 0.0, ssw = 0.0;
                for (int g = 0; g < c; ++g) {
                    if (!r.present[off + g]) continue;
                    const double mg = sum[g] / (double)ng[g];
                    ssb += (double)ng[g] * (mg - gm) * (mg - gm);
                    ssw += ss[g];
                }
                const double d1 = (double)(k - 1), d2 = (double)(n - k);
                s = (ssb / d1) / (ssw / d2);
                p = rescue_p(r, kPjF, s, d1, d2, t, 0);
            }
        } else {  // t-test
            const int64_t n0 = ng[0], n1 = ng[1];
            const double m0 = sum[0] / (double)n0, m1 = sum[1] / (double)n1;
            if (!r.welch) {
                if (!(cst[0] && cst[1])) {
                    const double df = (double)(n - 2);
                    const double sp2 = (ss[0] + ss[1]) / df;
                    s = (m0 - m1) / sqrt(sp2 * (1.0 / (double)n0 + 1.0 / (double)n1));
                    p = rescue_p(r, kPjT, s, df, 0.0, t, 0);
                }
            } else if (cst[0] && cst[1]) {
                if (first[0] != first[1]) { s = first[0] > first[1] ? dinf() : -dinf(); p = 0.0; }
            } else {
                const double e0 = ss[0] / (double)(n0 - 1) / (double)n0, e1 = ss[1] / (double)(n1 - 1) / (double)n1;
                const double se2 = e0 + e1;
                s = (m0 - m1) / sqrt(se2);
                const double nu = se2 * se2 / (e0 * e0 / (double)(n0 - 1) + e1 * e1 / (double)(n1 - 1));
                p = rescue_p(r, kPjT, s, nu, 0.0, t, 0);
            }
        }
        put(stat, pval, nout, t, s, p, (int32_t)n);
    }
}

// Block-parallel form of the rescue: one block per queued pair, each thread a
// fixed strided subset of the samples, reductions in a fixed order (results do
// not depend on scheduling). Group tests keep per-level sums in registers for up
// to MAXC levels; wider variables go through k_rescue.
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// op: 0 sum, 1 min, 2 max; result broadcast to every thread
__device__ double block_reduce(double v, int op, double *sh) {
    v = op == 0 ? warp_sum(v) : (op == 1 ? warp_min(v) : warp_max(v));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = op == 0 ? t + sh[w] : (op == 1 ? fmin(t, sh[w]) : fmax(t, sh[w]));
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// NT threads a pair: the few rescued pairs run on a few SMs while the others
// idle, so the time is one pair's instruction latency chain, which more threads
// shorten (512 up to 10 levels; 256 for 16, whose per-level sums need the
// registers)
template <int MAXC, int NT>
__global__ void __launch_bounds__(NT) k_rescue_block(RescueArgs r, const int32_t *flags, const int32_t *nflag,
                                                      int32_t max_flags, double *stat, double *pval, int32_t *nout,
                                                      int32_t symmetric) {
    __shared__ double sh[33];
    const int32_t cnt = min(*nflag, max_flags);
    const double inf = dinf();
    for (int q = blockIdx.x; q < cnt; q += gridDim.x) {
        const int64_t t = flags[q];
        const int ncols = symmetric ? r.na : r.nb;
        const int ia = (int)(t / ncols), ib = (int)(t - (int64_t)ia * ncols);
        const int va = r.va[ia], vb = symmetric ? r.va[ib] : r.vb[ib];
        const uint32_t *oa = r.obs + (int64_t)va * r.W, *ob = r.obs + (int64_t)vb * r.W;
        double s = dnan(), p = dnan(), es = dnan(), dof = dnan();
        if (r.test == NAPG_PEARSON) {
            double n = 0, sx = 0, sy = 0, mnx = inf, mxx = -inf, mny = inf, mxy = -inf;
            for_co_observed(r.ctxw, oa, ob, r.S, [&](int64_t k) {
                const double x = xval(r, (int64_t)va * r.S + k), y = xval(r, (int64_t)vb * r.S + k);
                n += 1; sx += x; sy += y;
                mnx = fmin(mnx, x); mxx = fmax(mxx, x); mny = fmin(mny, y); mxy = fmax(mxy, y);
            });
            n = block_reduce(n, 0, sh); sx = block_reduce(sx, 0, sh); sy = block_reduce(sy, 0, sh);
            mnx = block_reduce(mnx, 1, sh); mxx = block_reduce(mxx, 2, sh);
            mny = block_reduce(mny, 1, sh); mxy = block_reduce(mxy, 2, sh);
            const int64_t ni = (int64_t)n;
            if (ni > 1 && mnx != mxx && mny != mxy) {
                const double mx = sx / n, my = sy / n;
                double sxx = 0, syy = 0, sxy = 0;
                for_co_observed(r.ctxw, oa, ob, r.S, [&](int64_t k) {
                    const double dx = xval(r, (int64_t)va * r.S + k) - mx, dy = xval(r, (int64_t)vb * r.S + k) - my;
                    sxx += dx * dx; syy += dy * dy; sxy += dx * dy;
                });
                sxx = block_reduce(sxx, 0, sh); syy = block_reduce(syy, 0, sh); sxy = block_reduce(sxy, 0, sh);
                s = (va == vb) ? 1.0 : fmin(1.0, fmax(-1.0, sxy / (sqrt(sxx) * sqrt(syy))));
                if (threadIdx.x == 0) p = (ni <= 2) ? dnan() : rescue_p(r, kPjCorr, s, n, 0.0, t, symmetric ? ncols : 0);
            }
            if (threadIdx.x == 0) {
                put(stat, pval, nout, t, s, p, (int32_t)ni);
                if (symmetric) put(stat, pval, nout, (int64_t)ib * ncols + ia, s, p, (int32_t)ni);
            }
            __syncthreads();
            continue;
        }
        const uint8_t *la = r.lab + (int64_t)r.catrow[ia] * r.S;
        const int c = r.nlev_a[ia], off = r.levoff[ia];
        double ng[MAXC], sum[MAXC], mn[MAXC], mx[MAXC], ss[MAXC];
#pragma unroll
        for (int g = 0; g < MAXC; ++g) { ng[g] = 0; sum[g] = 0; mn[g] = inf; mx[g] = -inf; ss[g] = 0; }
        for_co_observed(r.ctxw, oa, ob, r.S, [&](int64_t k) {
            const int l = la[k];
            const double y = xval(r, (int64_t)vb * r.S + k);
#pragma unroll
            for (int g = 0; g < MAXC; ++g)
                if (l == g) { ng[g] += 1; sum[g] += y; mn[g] = fmin(mn[g], y); mx[g] = fmax(mx[g], y); }
        });
#pragma unroll
        for (int g = 0; g < MAXC; ++g) {
            if (g >= c) break;
            ng[g] = block_reduce(ng[g], 0, sh); sum[g] = block_reduce(sum[g], 0, sh);
            mn[g] = block_reduce(mn[g], 1, sh); mx[g] = block_reduce(mx[g], 2, sh);
        }
        double mean[MAXC];                       // the level means, formed once
#pragma unroll
        for (int g = 0; g < MAXC; ++g) mean[g] = (g < c && ng[g] > 0) ? sum[g] / ng[g] : 0.0;
        for_co_observed(r.ctxw, oa, ob, r.S, [&](int64_t k) {
            const int l = la[k];
            const double y = xval(r, (int64_t)vb * r.S + k);
#pragma unroll
            for (int g = 0; g < MAXC; ++g)
                if (l == g) { const double d = y - mean[g]; ss[g] += d * d; }
        });
#pragma unroll
        for (int g = 0; g < MAXC; ++g) {
            if (g >= c) break;
            ss[g] = block_reduce(ss[g], 0, sh);
        }
        if (threadIdx.x == 0) {
            double n = 0, tot = 0;
            bool cst[MAXC];
#pragma unroll
            for (int g = 0; g < MAXC; ++g) {
                cst[g] = (g < c) && (mn[g] == mx[g]);
                if (g < c) { n += ng[g]; tot += sum[g]; if (cst[g]) ss[g] = 0.0; }
            }
            if (r.test == NAPG_ANOVA) {
                int k = 0;
                bool all_const = true, differ = false, have_ref = false;
                double ref = 0.0;
#pragma unroll
                for (int g = 0; g < MAXC; ++g) {
                    if (g >= c || !r.present[off + g]) continue;
                    ++k;
                    all_const &= cst[g];
                    if (!have_ref) { ref = mn[g]; have_ref = true; } else if (mn[g] != ref) differ = true;
                }
                if (all_const) {
                    if (differ) { s = inf; p = 0.0; }
                } else {
                    const double gm = tot / n;
                    double ssb = 0.0, ssw = 0.0;
#pragma unroll
                    for (int g = 0; g < MAXC; ++g) {
                        if (g >= c || !r.present[off + g]) continue;
                        const double mg = sum[g] / ng[g];
                        ssb += ng[g] * (mg - gm) * (mg - gm);
                        ssw += ss[g];
                    }
                    const double d1 = (double)(k - 1), d2 = n - (double)k;
                    s = (ssb / d1) / (ssw / d2);
                    p = rescue_p(r, kPjF, s, d1, d2, t, 0);
                }
            } else {
                const double n0 = ng[0], n1 = ng[1];
                const double m0 = sum[0] / n0, m1 = sum[1] / n1;
                if (!r.welch) {
                    if (!(cst[0] && cst[1])) {
                        const double df = n - 2.0;
                        const double sp2 = (ss[0] + ss[1]) / df;
                        s = (m0 - m1) / sqrt(sp2 * (1.0 / n0 + 1.0 / n1));
                        p = rescue_p(r, kPjT, s, df, 0.0, t, 0);
                        es = (m0 - m1) / sqrt(sp2);
                        dof = df;
                    }
                } else if (cst[0] && cst[1]) {
                    // Cohen's d undefined: the two variances sum to zero
                    if (mn[0] != mn[1]) { s = mn[0] > mn[1] ? inf : -inf; p = 0.0; }
                } else {
                    const double e0 = ss[0] / (n0 - 1.0) / n0, e1 = ss[1] / (n1 - 1.0) / n1;
                    const double se2 = e0 + e1;
                    s = (m0 - m1) / sqrt(se2);
                    const double nu = se2 * se2 / (e0 * e0 / (n0 - 1.0) + e1 * e1 / (n1 - 1.0));
                    p = rescue_p(r, kPjT, s, nu, 0.0, t, 0);
                    es = (m0 - m1) / sqrt(0.5 * (ss[0] / (n0 - 1.0) + ss[1] / (n1 - 1.0)));
                    dof = nu;
                }
            }
            put(stat, pval, nout, t, s, p, (int32_t)n);
            if (r.es && r.test == NAPG_TTEST) r.es[t] = es;
            if (r.es2 && r.test == NAPG_TTEST) r.es2[t] = dof;
        }
        __syncthreads();
    }
}

void launch_rescue(const RescueArgs &r, const int32_t *flag_list, const int32_t *flag_count, int32_t max_flags,
                   double *stat, double *pval, int32_t *nout, int32_t symmetric, int32_t max_levels,
                   cudaStream_t st) {
    const unsigned blocks = 152 * 8;
    if (r.test == NAPG_PEARSON || max_levels <= 4) {
        count_launch();
        k_rescue_block<4, 512><<<blocks, 512, 0, st>>>(r, flag_list, flag_count, max_flags, stat, pval, nout, symmetric);
    } else if (max_levels <= 10) {
        count_launch();
        k_rescue_block<10, 512><<<blocks, 512, 0, st>>>(r, flag_list, flag_count, max_flags, stat, pval, nout, symmetric);
    } else if (max_levels <= 16) {
        count_launch();
        k_rescue_block<16, 256><<<blocks, 256, 0, st>>>(r, flag_list, flag_count, max_flags, stat, pval, nout, symmetric);
    } else {
        launch_rescue_serial(r, flag_list, flag_count, max_flags, stat, pval, nout, symmetric, st);
    }
}

void launch_rescue_serial(const RescueArgs &r, const int32_t *flag_list, const int32_t *flag_count, int32_t max_flags,
                          double *stat, double *pval, int32_t *nout, int32_t symmetric, cudaStream_t st) {
    count_launch();
    k_rescue<<<64, 64, 0, st>>>(r, flag_list, flag_count, max_flags, stat, pval, nout, symmetric);
}

}  // namespace napg
