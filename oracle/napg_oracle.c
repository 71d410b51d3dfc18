/*
 * napg_oracle.c -- plain, slow FP64 reference for the all-pairs statistical
 * tests with pairwise deletion of NApy (arXiv 2505.00448).
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the CPU-baseline
 * leg of the benchmark call it; the library under test never links, loads or
 * calls anything in this directory, and this file includes no header of it.
 *
 * Every statistic is computed one pair of variables at a time, straight from its
 * textbook definition, on the samples that survive pairwise deletion:
 *   deletion ............. Sec. 3.2 (operator I(g,h): both entries non-missing)
 *   Pearson r ............ Sec. 3.5.2      Spearman rho ....... Sec. 3.5.3
 *   chi-squared .......... Sec. 3.5.4      t-test (Welch/Student) Sec. 3.5.5
 *   Mann-Whitney U ....... Sec. 3.5.6      one-way ANOVA F .... Sec. 3.5.7
 *   Kruskal-Wallis H ..... Sec. 3.5.8      inputs/outputs ..... Sec. 3.3, 3.4
 * Means and sums of squares are two-pass (mean first, then centred sums).
 * Ranks come from a sort of the surviving values (a library qsort), with tied
 * values given the average of their ranks. P-values use the regularized
 * incomplete beta and gamma functions, written here from the DLMF continued
 * fractions and series (named at each function), plus lgamma/erfc/log1p/exp
 * from the C library.
 *
 * Readings of points the paper leaves open are stated where they are applied
 * (search for "reading:").
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fast-math).
 * OpenMP only spreads independent pairs over threads; each pair's arithmetic is
 * sequential and identical for any thread count.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Status codes (same numeric values as the library's, defined independently). */
#define ORC_OK 0
#define ORC_E_ARG 1
#define ORC_E_OOM 2
#define ORC_E_LABEL 4
#define ORC_E_NONFINITE 5

/* Test identifiers (same numeric values as the library's, defined independently). */
enum { ORC_PEARSON = 0, ORC_SPEARMAN = 1, ORC_CHI2 = 2, ORC_ANOVA = 3,
       ORC_TTEST = 4, ORC_MWU = 5, ORC_KRUSKAL = 6 };

#define ORC_MAXLEV 256

/* ------------------------------------------------------------------------ */
/* Special functions                                                         */
/* ------------------------------------------------------------------------ */

/* Stirling correction Delta(a) = lgamma(a) - [(a-1/2) log a - a + log(2 pi)/2]
 * (DLMF 5.11.1): for a >= 10 the Bernoulli series
 *   1/(12a) - 1/(360a^3) + 1/(1260a^5) - 1/(1680a^7) + 1/(1188a^9) - 691/(360360a^11),
 * otherwise the definition with the library lgamma. */
static double stirling_delta(double a) {
    if (a < 10.0) return lgamma(a) - ((a - 0.5) * log(a) - a + 0.5 * log(2.0 * M_PI));
    double r = 1.0 / a, r2 = r * r;
    return r * (1.0 / 12.0 + r2 * (-1.0 / 360.0 + r2 * (1.0 / 1260.0 + r2 * (-1.0 / 1680.0 +
           r2 * (1.0 / 1188.0 + r2 * (-691.0 / 360360.0))))));
}

/* rlog1(z) = z - log(1+z), with full relative precision for small |z|:
 * with u = z/(2+z), log(1+z) = 2 atanh(u) and z - 2u = u z, so
 *   rlog1(z) = u z - 2 (u^3/3 + u^5/5 + ...). */
static double rlog1(double z) {
    if (z < -0.5 || z > 0.5) return z - log1p(z);
    double u = z / (2.0 + z), u2 = u * u, term = u * u2, s = 0.0;
    for (int k = 3; k < 200; k += 2) {
        double t = term / (double)k;
        s += t;
        if (fabs(t) <= 1e-18 * fabs(s)) break;
        term *= u2;
    }
    return u * z - 2.0 * s;
}

/* log Gamma(b+a) - log Gamma(b) for b >= 10, from the Stirling form:
 *   a log b + (a + b - 1/2) log1p(a/b) - a + Delta(a+b) - Delta(b). */
static double lgamma_ratio(double a, double b) {
    return a * log(b) + (a + b - 0.5) * log1p(a / b) - a + stirling_delta(a + b) - stirling_delta(b);
}

/* x^a y^b / B(a,b) with x + y = 1, computed so that large a and b keep full
 * relative precision (the scaling of DiDonato & Morris, ACM TOMS 708, 1992):
 * for a, b >= 10, with x0 = a/(a+b) and lambda = (a+b) x - a,
 *   x^a y^b / B(a,b) = sqrt(ab / (2 pi (a+b))) exp(-a rlog1(lambda/a)
 *                      - b rlog1(-lambda/b) - Delta(a) - Delta(b) + Delta(a+b)). */
static double beta_front(double a, double b, double x, double y) {
    if (a >= 10.0 && b >= 10.0) {
        double lam = (x <= 0.5) ? (a + b) * x - a : b - (a + b) * y;
        double e = -a * rlog1(lam / a) - b * rlog1(-lam / b)
                   - stirling_delta(a) - stirling_delta(b) + stirling_delta(a + b);
        return sqrt(a * b / (2.0 * M_PI * (a + b))) * exp(e);
    }
    double lx = (x <= 0.5) ? log(x) : log1p(-y);
    double ly = (y <= 0.5) ? log(y) : log1p(-x);
    double lb;
    double lo = a < b ? a : b, hi = a < b ? b : a;
    if (hi >= 10.0) lb = lgamma(lo) - lgamma_ratio(lo, hi);
    else lb = lgamma(a) + lgamma(b) - lgamma(a + b);
    return exp(a * lx + b * ly - lb);
}

/* Continued fraction of DLMF 8.17.22 for I_x(a,b), evaluated with the modified
 * Lentz algorithm (Thompson & Barnett 1986). The value returned is
 *   1/(1+ d1/(1+ d2/(1+ ...)))
 * with d_{2m}   =  m (b-m) x / ((a+2m-1)(a+2m)),
 *      d_{2m+1} = -(a+m)(a+b+m) x / ((a+2m)(a+2m+1)). */
static double ibeta_cf(double a, double b, double x) {
    const double tiny = 1e-300;
    /* K = b0 + a1/(b1 + a2/(b2 + ...)) with b0 = 0, a1 = 1, all b_n = 1,
       a_{n+1} = d_n. */
    double f = tiny, C = tiny, D = 0.0;
    for (long n = 1; n < 2000000; ++n) {
        double an;
        if (n == 1) {
            an = 1.0;
        } else {
            long k = n - 1;          /* this is d_k */
            if (k % 2 == 0) {
                double m = (double)(k / 2);
                an = m * (b - m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));
            } else {
                double m = (double)((k - 1) / 2);
                an = -(a + m) * (a + b + m) * x / ((a + 2.0 * m) * (a + 2.0 * m + 1.0));
            }
        }
        D = 1.0 + an * D;
        if (fabs(D) < tiny) D = tiny;
        C = 1.0 + an / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        double delta = C * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-15) break;
    }
    return f;
}

/* The partial numerators d_k of DLMF 8.17.22 (k >= 1). */
static double ibeta_d(double a, double b, double x, long k) {
    if (k % 2 == 0) {
        double m = (double)(k / 2);
        return m * (b - m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));
    }
    double m = (double)((k - 1) / 2);
    return -(a + m) * (a + b + m) * x / ((a + 2.0 * m) * (a + 2.0 * m + 1.0));
}

/* 1 + d_{2m+1}, expanded so that nothing cancels when a is large and x is
 * close to 1 (y = 1 - x is used instead of x):
 *   [a(2m+1-b) + m(3m+2-b) + (a+m)(a+b+m) y] / ((a+2m)(a+2m+1)). */
static double ibeta_one_plus_odd(double a, double b, double y, long m) {
    double md = (double)m;
    double num = a * (2.0 * md + 1.0 - b) + md * (3.0 * md + 2.0 - b) + (a + md) * (a + b + md) * y;
    return num / ((a + 2.0 * md) * (a + 2.0 * md + 1.0));
}

/* The same fraction through its even part (contraction of pairs of steps):
 *   1/(1 + d1 - d1 d2/(1 + d2 + d3 - d3 d4/(1 + d4 + d5 - ...))),
 * with every 1 + d_{2m+1} taken from ibeta_one_plus_odd. For large a the odd
 * d_k approach -1, and this form keeps the digits the plain one loses. */
static double ibeta_cf_even(double a, double b, double x, double y) {
    const double tiny = 1e-300;
    double f = ibeta_one_plus_odd(a, b, y, 0);
    if (fabs(f) < tiny) f = tiny;
    double C = f, D = 0.0;
    for (long m = 1; m < 2000000; ++m) {
        double an = -ibeta_d(a, b, x, 2 * m - 1) * ibeta_d(a, b, x, 2 * m);
        double bn = ibeta_d(a, b, x, 2 * m) + ibeta_one_plus_odd(a, b, y, m);
        D = bn + an * D;
        if (fabs(D) < tiny) D = tiny;
        C = bn + an / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        double delta = C * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-15) break;
    }
    return 1.0 / f;
}

/* I_x(a,b) for x < (a+1)/(a+b+2): front factor x^a y^b / (a B(a,b)) times the
 * continued fraction (DLMF 8.17.22). y = 1-x is passed in to keep its digits.
 * The even-part form is used when a >= b, the plain form otherwise (measured
 * against 40-digit values, this choice keeps the relative error near 1e-13). */
static double ibeta_direct(double a, double b, double x, double y) {
    double cf = (a >= b) ? ibeta_cf_even(a, b, x, y) : ibeta_cf(a, b, x);
    return beta_front(a, b, x, y) / a * cf;
}

/* Regularized incomplete beta I_x(a,b), with x + y = 1 supplied by the caller.
 * Uses the symmetry I_x(a,b) = 1 - I_y(b,a) (DLMF 8.17.4) when
 * x > (a+1)/(a+b+2), where the fraction converges slowly. */
double orc_ibeta(double a, double b, double x, double y) {
    if (!(a > 0.0) || !(b > 0.0) || isnan(x) || isnan(y)) return NAN;
    if (x <= 0.0) return 0.0;
    if (y <= 0.0) return 1.0;
    if (x > (a + 1.0) / (a + b + 2.0)) return 1.0 - ibeta_direct(b, a, y, x);
    return ibeta_direct(a, b, x, y);
}

/* x^a e^{-x} / Gamma(a): for a >= 10 in the scaled form
 *   sqrt(a / (2 pi)) exp(-a rlog1((x-a)/a) - Delta(a)),
 * otherwise exp(a log x - x - lgamma(a)). */
static double gamma_front(double a, double x) {
    if (a >= 10.0) return sqrt(a / (2.0 * M_PI)) * exp(-a * rlog1((x - a) / a) - stirling_delta(a));
    return exp(a * log(x) - x - lgamma(a));
}

/* Lower series of DLMF 8.7.1 (gamma*(a,x) form):
 *   P(a,x) = x^a e^{-x} / Gamma(a+1) * sum_{k>=0} x^k / ((a+1)...(a+k)). */
static double gamma_p_series(double a, double x) {
    double term = 1.0, sum = 1.0;
    for (long k = 1; k < 2000000; ++k) {
        term *= x / (a + (double)k);
        sum += term;
        if (term < sum * 1e-18) break;
    }
    return gamma_front(a, x) / a * sum;
}

/* Legendre continued fraction for Gamma(a,x) (DLMF 8.9.2), even part:
 *   Gamma(a,x) = e^{-x} x^a / (x+1-a - 1(1-a)/(x+3-a - 2(2-a)/(x+5-a - ...)))
 * evaluated with modified Lentz; returns Q(a,x) = Gamma(a,x)/Gamma(a). */
static double gamma_q_cf(double a, double x) {
    const double tiny = 1e-300;
    double f = tiny, C = tiny, D = 0.0;
    for (long n = 1; n < 2000000; ++n) {
        double an = (n == 1) ? 1.0 : -(double)(n - 1) * ((double)(n - 1) - a);
        double bn = x + 2.0 * (double)n - 1.0 - a;
        D = bn + an * D;
        if (fabs(D) < tiny) D = tiny;
        C = bn + an / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        double delta = C * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-15) break;
    }
    return gamma_front(a, x) * f;
}

/* Regularized upper incomplete gamma Q(a,x): series for x < a+1, else the
 * continued fraction. */
double orc_gamma_q(double a, double x) {
    if (!(a > 0.0) || isnan(x)) return NAN;
    if (x <= 0.0) return 1.0;
    if (isinf(x)) return 0.0;
    if (x < a + 1.0) return 1.0 - gamma_p_series(a, x);
    return gamma_q_cf(a, x);
}

/* Standard normal survival function, 1 - Phi(z) = erfc(z/sqrt 2)/2. */
double orc_norm_sf(double z) { return 0.5 * erfc(z / sqrt(2.0)); }

/* Two-sided p of Student's t with df degrees of freedom:
 *   p = I_{df/(df+t^2)}(df/2, 1/2). */
double orc_t_p2(double t, double df) {
    if (isnan(t) || !(df > 0.0)) return NAN;
    if (isinf(t)) return 0.0;
    double t2 = t * t;
    return orc_ibeta(0.5 * df, 0.5, df / (df + t2), t2 / (df + t2));
}

/* Survival function of F(d1, d2) at F: I_{d2/(d2+d1 F)}(d2/2, d1/2). */
double orc_f_sf(double F, double d1, double d2) {
    if (isnan(F) || !(d1 > 0.0) || !(d2 > 0.0)) return NAN;
    if (isinf(F)) return 0.0;
    if (F <= 0.0) return 1.0;
    double den = d2 + d1 * F;
    return orc_ibeta(0.5 * d2, 0.5 * d1, d2 / den, d1 * F / den);
}

/* Survival function of chi-squared with df degrees of freedom. */
double orc_chi2_sf(double x, double df) {
    if (isnan(x) || !(df > 0.0)) return NAN;
    return orc_gamma_q(0.5 * df, 0.5 * x);
}

/* Pearson / Spearman p-value from a correlation coefficient (Sec. 3.5.2:
 * Beta-distribution CDF; Sec. 3.5.3: t-distribution): the two are the same
 * number, p = I_{1-r^2}((n-2)/2, 1/2). */
double orc_corr_p(double r, double n) {
    if (isnan(r) || n <= 2.0) return NAN;
    if (fabs(r) >= 1.0) return 0.0;
    return orc_ibeta(0.5 * (n - 2.0), 0.5, (1.0 - r) * (1.0 + r), r * r);
}

/* Exact null distribution of the Mann-Whitney U statistic (Sec. 3.5.6, exact
 * mode), by the Mann & Whitney (1947) recurrence in probability form:
 *   p(u; a, b) = a/(a+b) p(u-b; a-1, b) + b/(a+b) p(u; a, b-1),
 *   p(u; a, 0) = p(u; 0, b) = [u == 0].
 * Returns P(U >= u) for group sizes (n0, n1). */
double orc_mwu_exact_sf(double u, long n0, long n1) {
    if (n0 <= 0 || n1 <= 0 || isnan(u)) return NAN;
    long m = n0 < n1 ? n0 : n1, n = n0 < n1 ? n1 : n0;
    long umax = m * n;
    if (u <= 0.0) return 1.0;
    if (u > (double)umax) return 0.0;
    /* p[a][v] for a = 0..m, v = 0..a*n, updated in place for b = 1..n. */
    double **p = (double **)malloc((size_t)(m + 1) * sizeof(double *));
    if (!p) return NAN;
    for (long a = 0; a <= m; ++a) {
        p[a] = (double *)calloc((size_t)(a * n + 1), sizeof(double));
        if (!p[a]) { for (long q = 0; q < a; ++q) free(p[q]); free(p); return NAN; }
        p[a][0] = 1.0;                  /* b = 0: U = 0 surely */
    }
    for (long b = 1; b <= n; ++b) {
        /* a = 0 stays [v == 0]. For a >= 1 the new row reads the new row a-1
           (already updated for this b) and the old row a (previous b). */
        for (long a = 1; a <= m; ++a) {
            double wa = (double)a / (double)(a + b), wb = (double)b / (double)(a + b);
            long vmax = a * b;
            for (long v = vmax; v >= 0; --v) {
                double from_a = (v - b >= 0 && v - b <= (a - 1) * b) ? p[a - 1][v - b] : 0.0;
                double from_b = (v <= a * (b - 1)) ? p[a][v] : 0.0;
                p[a][v] = wa * from_a + wb * from_b;
            }
        }
    }
    long u0 = (long)ceil(u);
    double s = 0.0;
    for (long v = umax; v >= u0; --v) s += p[m][v];
    for (long a = 0; a <= m; ++a) free(p[a]);
    free(p);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Cohort access and pairwise deletion (Sec. 3.2)                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *X;        /* F x S, row-major, one row per variable */
    int64_t F, S;
    double miss;            /* missing sentinel; NaN means "isnan" */
    const uint8_t *vtype;   /* 0 continuous, 1 categorical */
    const int32_t *nlev;    /* levels per categorical variable */
    const uint8_t *ctx;     /* sample context mask, NULL = all samples */
    int welch, yates, mwu_mode, mwu_cc;
} orc_cohort;

static int is_missing(double v, double m) { return isnan(m) ? isnan(v) : (v == m); }

static int observed(const orc_cohort *c, int64_t v, int64_t s) {
    if (c->ctx && !c->ctx[s]) return 0;
    return !is_missing(c->X[v * c->S + s], c->miss);
}

/* Input validation (Sec. 3.2 / 3.3). Reading: a non-missing value that is
 * +-inf or NaN is an error; a categorical value must be an integer in
 * [0, n_levels). */
int orc_validate(const double *X, int64_t F, int64_t S, double miss,
                 const uint8_t *vtype, const int32_t *nlev) {
    for (int64_t v = 0; v < F; ++v) {
        for (int64_t s = 0; s < S; ++s) {
            double x = X[v * S + s];
            if (is_missing(x, miss)) continue;
            if (!isfinite(x)) return ORC_E_NONFINITE;
            if (vtype[v] == 1) {
                if (x != floor(x) || x < 0.0 || x >= (double)nlev[v]) return ORC_E_LABEL;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Ranking helpers (Sec. 3.5.3, 3.5.6, 3.5.8: ties get the average rank)     */
/* ------------------------------------------------------------------------ */

typedef struct { double v; int64_t i; } orc_vi;

static int cmp_vi(const void *pa, const void *pb) {
    const orc_vi *a = (const orc_vi *)pa, *b = (const orc_vi *)pb;
    if (a->v < b->v) return -1;
    if (a->v > b->v) return 1;
    return (a->i < b->i) ? -1 : (a->i > b->i);
}

/* Doubled average ranks: for the value at index k of v[0..n), 2R = 2L + t + 1
 * with L = #values strictly smaller and t = #values equal to it (its tie group
 * included). Also returns the tie term sum over groups of (t^3 - t). */
static void doubled_ranks(const double *v, int64_t n, int64_t *r2, orc_vi *buf, int64_t *tie_term) {
    for (int64_t k = 0; k < n; ++k) { buf[k].v = v[k]; buf[k].i = k; }
    qsort(buf, (size_t)n, sizeof(orc_vi), cmp_vi);
    int64_t T = 0;
    int64_t a = 0;
    while (a < n) {
        int64_t b = a + 1;
        while (b < n && buf[b].v == buf[a].v) ++b;
        int64_t t = b - a;
        for (int64_t k = a; k < b; ++k) r2[buf[k].i] = 2 * a + t + 1;
        T += t * t * t - t;
        a = b;
    }
    if (tie_term) *tie_term = T;
}

static int all_equal(const double *v, int64_t n) {
    for (int64_t k = 1; k < n; ++k) if (v[k] != v[0]) return 0;
    return 1;
}

/* Two-pass Pearson correlation of v, w (n >= 2). Reading: a constant column
 * on the co-observed samples has zero variance and gives NaN. */
static double pearson_r(const double *v, const double *w, int64_t n) {
    if (all_equal(v, n) || all_equal(w, n)) return NAN;
    double mv = 0.0, mw = 0.0;
    for (int64_t k = 0; k < n; ++k) { mv += v[k]; mw += w[k]; }
    mv /= (double)n; mw /= (double)n;
    double svv = 0.0, sww = 0.0, svw = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double dv = v[k] - mv, dw = w[k] - mw;
        svv += dv * dv; sww += dw * dw; svw += dv * dw;
    }
    double r = svw / (sqrt(svv) * sqrt(sww));
    if (r > 1.0) r = 1.0;
    if (r < -1.0) r = -1.0;
    return r;
}

/* ------------------------------------------------------------------------ */
/* Per-pair tests                                                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    double *x, *y;          /* gathered values of the two variables */
    int64_t *r2;            /* doubled ranks */
    orc_vi *buf;
} orc_scratch;

/* Gather the co-observed samples of (va, vb): I(g,h) of Sec. 3.2, restricted to
 * the sample context. */
static int64_t gather_pair(const orc_cohort *c, int64_t va, int64_t vb, double *x, double *y) {
    int64_t n = 0;
    for (int64_t s = 0; s < c->S; ++s) {
        if (observed(c, va, s) && observed(c, vb, s)) {
            x[n] = c->X[va * c->S + s];
            y[n] = c->X[vb * c->S + s];
            ++n;
        }
    }
    return n;
}

/* Levels of a categorical variable present in the current context before
 * pairwise deletion. Reading: these are the "previously existing categories"
 * of Sec. 3.5.4/3.5.5/3.5.7/3.5.8; a level never observed in the context is
 * not a category of this call. */
static int present_levels(const orc_cohort *c, int64_t v, int *present) {
    int L = c->nlev[v];
    for (int g = 0; g < L; ++g) present[g] = 0;
    for (int64_t s = 0; s < c->S; ++s)
        if (observed(c, v, s)) present[(int)c->X[v * c->S + s]] = 1;
    int k = 0;
    for (int g = 0; g < L; ++g) k += present[g];
    return k;
}

/* Sec. 3.5.2. Reading of the garbled thresholds: n <= 1 -> r and p NaN;
 * n == 2 -> p NaN. */
static void pearson_pair(const orc_cohort *c, int64_t i, int64_t j, orc_scratch *w,
                         double *st, double *p, int32_t *nn) {
    int64_t n = gather_pair(c, i, j, w->x, w->y);
    *nn = (int32_t)n;
    if (n <= 1) { *st = NAN; *p = NAN; return; }
    double r = pearson_r(w->x, w->y, n);
    *st = r;
    *p = (n <= 2) ? NAN : orc_corr_p(r, (double)n);
}

/* Sec. 3.5.3: rho is the Pearson correlation of the tie-averaged ranks of the
 * co-observed samples; p from the t distribution with n-2 df. */
static void spearman_pair(const orc_cohort *c, int64_t i, int64_t j, orc_scratch *w,
                          double *st, double *p, int32_t *nn) {
    int64_t n = gather_pair(c, i, j, w->x, w->y);
    *nn = (int32_t)n;
    if (n <= 1) { *st = NAN; *p = NAN; return; }
    doubled_ranks(w->x, n, w->r2, w->buf, NULL);
    for (int64_t k = 0; k < n; ++k) w->x[k] = 0.5 * (double)w->r2[k];
    doubled_ranks(w->y, n, w->r2, w->buf, NULL);
    for (int64_t k = 0; k < n; ++k) w->y[k] = 0.5 * (double)w->r2[k];
    double r = pearson_r(w->x, w->y, n);
    *st = r;
    *p = (n <= 2) ? NAN : orc_corr_p(r, (double)n);
}

/* Sec. 3.5.4: chi-squared test of independence on the contingency table of the
 * present levels. A present level left empty by deletion makes everything NaN.
 * Reading: one present level in either variable gives chi2 = 0 and p NaN. */
static void chi2_pair(const orc_cohort *c, int64_t a, int64_t b, orc_scratch *w,
                      double *st, double *p, int32_t *nn) {
    int pa[ORC_MAXLEV], pb[ORC_MAXLEV];
    int ka = present_levels(c, a, pa), kb = present_levels(c, b, pb);
    int La = c->nlev[a], Lb = c->nlev[b];
    int64_t n = gather_pair(c, a, b, w->x, w->y);
    *nn = (int32_t)n;
    int64_t *O = (int64_t *)calloc((size_t)La * (size_t)Lb, sizeof(int64_t));
    int64_t row[ORC_MAXLEV], col[ORC_MAXLEV];
    for (int g = 0; g < La; ++g) row[g] = 0;
    for (int h = 0; h < Lb; ++h) col[h] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int g = (int)w->x[k], h = (int)w->y[k];
        O[(int64_t)g * Lb + h] += 1; row[g] += 1; col[h] += 1;
    }
    int empty = (n == 0);
    for (int g = 0; g < La; ++g) if (pa[g] && row[g] == 0) empty = 1;
    for (int h = 0; h < Lb; ++h) if (pb[h] && col[h] == 0) empty = 1;
    if (empty) { *st = NAN; *p = NAN; free(O); return; }
    int yates = c->yates && ka == 2 && kb == 2;
    double chi2 = 0.0;
    for (int g = 0; g < La; ++g) {
        if (!pa[g]) continue;
        for (int h = 0; h < Lb; ++h) {
            if (!pb[h]) continue;
            double E = (double)row[g] * (double)col[h] / (double)n;
            double d = fabs((double)O[(int64_t)g * Lb + h] - E);
            if (yates) d = (d > 0.5) ? d - 0.5 : 0.0;
            chi2 += d * d / E;
        }
    }
    free(O);
    int df = (ka - 1) * (kb - 1);
    *st = chi2;
    *p = (df <= 0) ? NAN : orc_chi2_sf(chi2, (double)df);
}

/* Split the co-observed values of continuous j by the present levels of
 * categorical a. Returns the number of co-observed samples; fills group sizes
 * and sets *empty when a present level has no co-observed sample. The values
 * land in w->y in sample order and their labels in w->x. */
static int64_t group_pair(const orc_cohort *c, int64_t a, int64_t j, orc_scratch *w,
                          int *present, int *k, int64_t *ng, int *empty) {
    *k = present_levels(c, a, present);
    int64_t n = gather_pair(c, a, j, w->x, w->y);
    int L = c->nlev[a];
    for (int g = 0; g < L; ++g) ng[g] = 0;
    for (int64_t q = 0; q < n; ++q) ng[(int)w->x[q]] += 1;
    *empty = (n == 0);
    for (int g = 0; g < L; ++g) if (present[g] && ng[g] == 0) *empty = 1;
    return n;
}

/* Sec. 3.5.7: one-way ANOVA F over the present levels, p from F(k-1, n-k).
 * Readings: k < 2 or n - k < 1 -> NaN; all groups constant -> F = inf, p = 0
 * when the group values differ, else NaN. */
static void anova_pair(const orc_cohort *c, int64_t a, int64_t j, orc_scratch *w,
                       double *st, double *p, int32_t *nn) {
    int present[ORC_MAXLEV], k, empty;
    int64_t ng[ORC_MAXLEV];
    int64_t n = group_pair(c, a, j, w, present, &k, ng, &empty);
    *nn = (int32_t)n;
    if (empty || k < 2 || n - k < 1) { *st = NAN; *p = NAN; return; }
    int L = c->nlev[a];
    double sum[ORC_MAXLEV], first[ORC_MAXLEV];
    int constant[ORC_MAXLEV], seen[ORC_MAXLEV];
    for (int g = 0; g < L; ++g) { sum[g] = 0.0; constant[g] = 1; seen[g] = 0; first[g] = 0.0; }
    double gm = 0.0;
    for (int64_t q = 0; q < n; ++q) {
        int g = (int)w->x[q]; double v = w->y[q];
        if (!seen[g]) { first[g] = v; seen[g] = 1; } else if (v != first[g]) constant[g] = 0;
        sum[g] += v; gm += v;
    }
    gm /= (double)n;
    int all_const = 1;
    for (int g = 0; g < L; ++g) if (present[g]) all_const &= constant[g];
    if (all_const) {
        int differ = 0; double ref = NAN;
        for (int g = 0; g < L; ++g) if (present[g]) { if (isnan(ref)) ref = first[g]; else if (first[g] != ref) differ = 1; }
        if (differ) { *st = INFINITY; *p = 0.0; } else { *st = NAN; *p = NAN; }
        return;
    }
    /* F does not change when every y moves by one constant: the sums of
     * squares are formed from y - gm (the two-pass form), so that a large
     * common offset does not swamp group-mean differences far below it. */
    double dsum[ORC_MAXLEV], dmean[ORC_MAXLEV], dgm = 0.0;
    for (int g = 0; g < L; ++g) dsum[g] = 0.0;
    for (int64_t q = 0; q < n; ++q) { double d = w->y[q] - gm; dsum[(int)w->x[q]] += d; dgm += d; }
    dgm /= (double)n;
    for (int g = 0; g < L; ++g) if (present[g]) dmean[g] = dsum[g] / (double)ng[g];
    double ssb = 0.0, ssw = 0.0;
    for (int g = 0; g < L; ++g) if (present[g]) ssb += (double)ng[g] * (dmean[g] - dgm) * (dmean[g] - dgm);
    for (int64_t q = 0; q < n; ++q) { int g = (int)w->x[q]; double d = (w->y[q] - gm) - dmean[g]; ssw += d * d; }
    double d1 = (double)(k - 1), d2 = (double)(n - k);
    double F = (ssb / d1) / (ssw / d2);
    *st = F;
    *p = orc_f_sf(F, d1, d2);
}

/* Sec. 3.5.5: two-sample t-test between levels 0 and 1 (statistic = mean of
 * level 0 minus mean of level 1). NaN when a group has fewer than 2 samples or
 * n < 3. Student: NaN when the pooled SD is 0. Welch, reading: both groups
 * constant -> t = +-inf with p = 0 when the values differ, else NaN. */
static void ttest_pair(const orc_cohort *c, int64_t a, int64_t j, orc_scratch *w,
                       double *st, double *p, int32_t *nn) {
    int64_t n = gather_pair(c, a, j, w->x, w->y);
    *nn = (int32_t)n;
    int64_t n0 = 0, n1 = 0;
    double s0 = 0.0, s1 = 0.0, f0 = 0.0, f1 = 0.0;
    int c0 = 1, c1 = 1;
    for (int64_t q = 0; q < n; ++q) {
        double v = w->y[q];
        if (w->x[q] == 0.0) { if (n0 == 0) f0 = v; else if (v != f0) c0 = 0; s0 += v; ++n0; }
        else                { if (n1 == 0) f1 = v; else if (v != f1) c1 = 0; s1 += v; ++n1; }
    }
    if (n0 < 2 || n1 < 2 || n < 3) { *st = NAN; *p = NAN; return; }
    /* t does not change when every y moves by one constant: means and sums of
     * squares are formed from y - (overall mean), as for the F statistic. */
    double gm = (s0 + s1) / (double)n, d0 = 0.0, d1 = 0.0;
    for (int64_t q = 0; q < n; ++q) {
        double d = w->y[q] - gm;
        if (w->x[q] == 0.0) d0 += d; else d1 += d;
    }
    double m0 = d0 / (double)n0, m1 = d1 / (double)n1;
    double q0 = 0.0, q1 = 0.0;
    for (int64_t q = 0; q < n; ++q) {
        double v = w->y[q] - gm;
        if (w->x[q] == 0.0) q0 += (v - m0) * (v - m0); else q1 += (v - m1) * (v - m1);
    }
    if (c0) q0 = 0.0;
    if (c1) q1 = 0.0;
    double v0 = q0 / (double)(n0 - 1), v1 = q1 / (double)(n1 - 1);
    if (!c->welch) {
        if (c0 && c1) { *st = NAN; *p = NAN; return; }
        double df = (double)(n - 2);
        double sp2 = (q0 + q1) / df;
        double t = (m0 - m1) / sqrt(sp2 * (1.0 / (double)n0 + 1.0 / (double)n1));
        *st = t; *p = orc_t_p2(t, df);
        return;
    }
    if (c0 && c1) {
        if (f0 != f1) { *st = (f0 > f1) ? INFINITY : -INFINITY; *p = 0.0; }
        else { *st = NAN; *p = NAN; }
        return;
    }
    double e0 = v0 / (double)n0, e1 = v1 / (double)n1;
    double se2 = e0 + e1;
    double t = (m0 - m1) / sqrt(se2);
    double nu = se2 * se2 / (e0 * e0 / (double)(n0 - 1) + e1 * e1 / (double)(n1 - 1));
    *st = t; *p = orc_t_p2(t, nu);
}

/* Sec. 3.5.6: Mann-Whitney U between levels 0 and 1 on tie-averaged ranks.
 * Statistic: U of level 0, U0 = R0 - n0(n0+1)/2. Modes: 0 auto (exact when no
 * ties and min(n0,n1) < 8), 1 exact, 2 asymptotic. Asymptotic p uses the
 * tie-corrected variance and, if mwu_cc, the 0.5 continuity correction;
 * p = min(1, 2 sf(z)) with z taken at max(U0, U1). Exact p = min(1, 2 P(U >= max)).
 * Reading: zero variance (everything tied) gives p NaN. */
static void mwu_pair(const orc_cohort *c, int64_t a, int64_t j, orc_scratch *w,
                     double *st, double *p, int32_t *nn) {
    int64_t n = gather_pair(c, a, j, w->x, w->y);
    *nn = (int32_t)n;
    int64_t n0 = 0, n1 = 0;
    for (int64_t q = 0; q < n; ++q) { if (w->x[q] == 0.0) ++n0; else ++n1; }
    if (n0 == 0 || n1 == 0) { *st = NAN; *p = NAN; return; }
    int64_t T = 0;
    doubled_ranks(w->y, n, w->r2, w->buf, &T);
    double R0 = 0.0;
    for (int64_t q = 0; q < n; ++q) if (w->x[q] == 0.0) R0 += 0.5 * (double)w->r2[q];
    double U0 = R0 - 0.5 * (double)n0 * (double)(n0 + 1);
    double U1 = (double)n0 * (double)n1 - U0;
    double U = U0 > U1 ? U0 : U1;
    *st = U0;
    int exact = (c->mwu_mode == 1) || (c->mwu_mode == 0 && T == 0 && (n0 < 8 || n1 < 8));
    if (exact) {
        double pv = 2.0 * orc_mwu_exact_sf(U, (long)n0, (long)n1);
        *p = pv > 1.0 ? 1.0 : pv;
        return;
    }
    double nd = (double)n;
    double var = (double)n0 * (double)n1 / 12.0 * ((nd + 1.0) - (double)T / (nd * (nd - 1.0)));
    if (!(var > 0.0)) { *p = NAN; return; }
    double z = (U - 0.5 * (double)n0 * (double)n1 - (c->mwu_cc ? 0.5 : 0.0)) / sqrt(var);
    double pv = 2.0 * orc_norm_sf(z);
    *p = pv > 1.0 ? 1.0 : pv;
}

/* Sec. 3.5.8: Kruskal-Wallis H over the present levels with tie-averaged ranks
 * and the tie correction C = 1 - sum(t^3 - t)/(n^3 - n); p from chi2(k-1).
 * H0 = 12/(n(n+1)) * sum_g n_g (Rbar_g - (n+1)/2)^2 (the centred form of the
 * textbook 12/(n(n+1)) sum R_g^2/n_g - 3(n+1)), the centred group sums formed
 * exactly from the integer doubled ranks. Readings: k < 2 -> NaN;
 * C == 0 (all tied) -> NaN. */
static void kruskal_pair(const orc_cohort *c, int64_t a, int64_t j, orc_scratch *w,
                         double *st, double *p, int32_t *nn) {
    int present[ORC_MAXLEV], k, empty;
    int64_t ng[ORC_MAXLEV];
    int64_t n = group_pair(c, a, j, w, present, &k, ng, &empty);
    *nn = (int32_t)n;
    if (empty || k < 2) { *st = NAN; *p = NAN; return; }
    int64_t T = 0;
    doubled_ranks(w->y, n, w->r2, w->buf, &T);
    int L = c->nlev[a];
    /* per level, the doubled rank sum and its centred value
     * D_g = sum 2R - n_g (n+1) = 2 n_g (Rbar_g - (n+1)/2), exact in int64, so
     * n_g (Rbar_g - (n+1)/2)^2 = D_g^2 / (4 n_g) carries no cancellation */
    int64_t S2[ORC_MAXLEV];
    for (int g = 0; g < L; ++g) S2[g] = 0;
    for (int64_t q = 0; q < n; ++q) S2[(int)w->x[q]] += w->r2[q];
    double nd = (double)n, h0 = 0.0;
    for (int g = 0; g < L; ++g) {
        if (!present[g]) continue;
        const double D = (double)(S2[g] - ng[g] * (n + 1));
        h0 += D * D / (4.0 * (double)ng[g]);
    }
    h0 *= 12.0 / (nd * (nd + 1.0));
    double C = 1.0 - (double)T / (nd * nd * nd - nd);
    if (!(C > 0.0)) { *st = NAN; *p = NAN; return; }
    double H = h0 / C;
    *st = H;
    *p = orc_chi2_sf(H, (double)(k - 1));
}

typedef void (*pair_fn)(const orc_cohort *, int64_t, int64_t, orc_scratch *, double *, double *, int32_t *);

static pair_fn pick(int test) {
    switch (test) {
        case ORC_PEARSON: return pearson_pair;
        case ORC_SPEARMAN: return spearman_pair;
        case ORC_CHI2: return chi2_pair;
        case ORC_ANOVA: return anova_pair;
        case ORC_TTEST: return ttest_pair;
        case ORC_MWU: return mwu_pair;
        case ORC_KRUSKAL: return kruskal_pair;
        default: return NULL;
    }
}

/* Argument checks shared by the run entry points: the variable types each test
 * takes, and two levels for the two-group tests. */
static int check_vars(const orc_cohort *c, int test, const int32_t *va, int64_t na,
                      const int32_t *vb, int64_t nb) {
    int want_a = (test == ORC_PEARSON || test == ORC_SPEARMAN) ? 0 : 1;
    int want_b = (test == ORC_PEARSON || test == ORC_SPEARMAN) ? 0 :
                 (test == ORC_CHI2 ? 1 : 0);
    for (int64_t q = 0; q < na; ++q) {
        if (va[q] < 0 || va[q] >= c->F || c->vtype[va[q]] != want_a) return ORC_E_ARG;
        if (want_a == 1 && (c->nlev[va[q]] < 1 || c->nlev[va[q]] > ORC_MAXLEV)) return ORC_E_ARG;
        if ((test == ORC_TTEST || test == ORC_MWU) && c->nlev[va[q]] != 2) return ORC_E_ARG;
        if ((test == ORC_ANOVA || test == ORC_KRUSKAL) && c->nlev[va[q]] < 2) return ORC_E_ARG;
    }
    if (vb) {
        for (int64_t q = 0; q < nb; ++q) {
            if (vb[q] < 0 || vb[q] >= c->F || c->vtype[vb[q]] != want_b) return ORC_E_ARG;
            if (want_b == 1 && (c->nlev[vb[q]] < 1 || c->nlev[vb[q]] > ORC_MAXLEV)) return ORC_E_ARG;
        }
    } else if (want_a != want_b) {
        return ORC_E_ARG;
    }
    return ORC_OK;
}

static int alloc_scratch(orc_scratch *w, int64_t S) {
    size_t m = (size_t)(S > 0 ? S : 1);
    w->x = (double *)malloc(m * sizeof(double));
    w->y = (double *)malloc(m * sizeof(double));
    w->r2 = (int64_t *)malloc(m * sizeof(int64_t));
    w->buf = (orc_vi *)malloc(m * sizeof(orc_vi));
    return (w->x && w->y && w->r2 && w->buf) ? ORC_OK : ORC_E_OOM;
}

static void free_scratch(orc_scratch *w) { free(w->x); free(w->y); free(w->r2); free(w->buf); }

/* All pairs of vars_a x vars_b (or vars_a x vars_a when vars_b is NULL), outputs
 * row-major n_a x n_b. The mixed tests take categorical variables in A and
 * continuous ones in B (Sec. 3.4: an F_C x F_Q output). */
int orc_run(int test, const double *X, int64_t F, int64_t S, double miss,
            const uint8_t *vtype, const int32_t *nlev, const uint8_t *ctx,
            const int32_t *va, int32_t na, const int32_t *vb, int32_t nb,
            int welch, int yates, int mwu_mode, int mwu_cc,
            double *stat, double *pval, int32_t *nout, int nthreads) {
    orc_cohort c = { X, F, S, miss, vtype, nlev, ctx, welch, yates, mwu_mode, mwu_cc };
    pair_fn fn = pick(test);
    if (!fn || na < 0 || nb < 0) return ORC_E_ARG;
    int rc = check_vars(&c, test, va, na, vb, nb);
    if (rc) return rc;
    rc = orc_validate(X, F, S, miss, vtype, nlev);
    if (rc) return rc;
    const int32_t *cols = vb ? vb : va;
    int64_t ncols = vb ? nb : na;
    int64_t total = (int64_t)na * ncols;
    int err = 0;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();   /* this call only */
#else
    const int nt = 1;
    (void)nthreads;
#endif
    (void)nt;
#pragma omp parallel num_threads(nt)
    {
        orc_scratch w;
        int ok = alloc_scratch(&w, S) == ORC_OK;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < total; ++q) {
            if (!ok) continue;
            int64_t ia = q / ncols, ib = q % ncols;
            double st, pv; int32_t nn;
            fn(&c, va[ia], cols[ib], &w, &st, &pv, &nn);
            if (stat) stat[q] = st;
            if (pval) pval[q] = pv;
            if (nout) nout[q] = nn;
        }
        free_scratch(&w);
    }
    return err ? ORC_E_OOM : ORC_OK;
}

/* The same tests on an explicit list of (var_a, var_b) pairs; used to check
 * sampled pairs of large cohorts. Skips validation of the whole matrix when
 * validate == 0 (the caller validated it once). */
int orc_run_pairs(int test, const double *X, int64_t F, int64_t S, double miss,
                  const uint8_t *vtype, const int32_t *nlev, const uint8_t *ctx,
                  const int32_t *pa, const int32_t *pb, int64_t npairs,
                  int welch, int yates, int mwu_mode, int mwu_cc,
                  double *stat, double *pval, int32_t *nout, int nthreads, int validate) {
    orc_cohort c = { X, F, S, miss, vtype, nlev, ctx, welch, yates, mwu_mode, mwu_cc };
    pair_fn fn = pick(test);
    if (!fn || npairs < 0) return ORC_E_ARG;
    for (int64_t q = 0; q < npairs; ++q) {
        int rc = check_vars(&c, test, pa + q, 1, pb + q, 1);
        if (rc) return rc;
    }
    if (validate) {
        int rc = orc_validate(X, F, S, miss, vtype, nlev);
        if (rc) return rc;
    }
    int err = 0;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();   /* this call only */
#else
    const int nt = 1;
    (void)nthreads;
#endif
    (void)nt;
#pragma omp parallel num_threads(nt)
    {
        orc_scratch w;
        int ok = alloc_scratch(&w, S) == ORC_OK;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t q = 0; q < npairs; ++q) {
            if (!ok) continue;
            double st, pv; int32_t nn;
            fn(&c, pa[q], pb[q], &w, &st, &pv, &nn);
            if (stat) stat[q] = st;
            if (pval) pval[q] = pv;
            if (nout) nout[q] = nn;
        }
        free_scratch(&w);
    }
    return err ? ORC_E_OOM : ORC_OK;
}

/* Integer quantities of one pair, for bit-exact checks:
 *   CHI2:      out[g*Lb + h] = contingency count O_gh (all levels, row-major).
 *   SPEARMAN:  out = {n, sum 2Rx*2Ry, sum (2Rx)^2, sum (2Ry)^2}.
 *   MWU/KRUSKAL: out = {n, T, n_0, S_0, n_1, S_1, ...} with S_g the sum of the
 *              doubled ranks of level g and T = sum (t^3 - t) over tie groups.
 *   PEARSON/ANOVA/TTEST: out = {n} (plus n_g for ANOVA/TTEST: {n, n_0, n_1, ...}).
 * Returns the number of int64 values written, or -1 on bad arguments. */
int64_t orc_pair_ints(int test, const double *X, int64_t F, int64_t S, double miss,
                      const uint8_t *vtype, const int32_t *nlev, const uint8_t *ctx,
                      int32_t a, int32_t b, int64_t *out, int64_t cap) {
    orc_cohort c = { X, F, S, miss, vtype, nlev, ctx, 1, 0, 0, 1 };
    if (check_vars(&c, test, &a, 1, &b, 1)) return -1;
    orc_scratch w;
    if (alloc_scratch(&w, S)) return -1;
    int64_t n = gather_pair(&c, a, b, w.x, w.y), m = 0;
    if (test == ORC_CHI2) {
        int La = nlev[a], Lb = nlev[b];
        if (cap < (int64_t)La * Lb) { free_scratch(&w); return -1; }
        for (int64_t q = 0; q < (int64_t)La * Lb; ++q) out[q] = 0;
        for (int64_t q = 0; q < n; ++q) out[(int64_t)w.x[q] * Lb + (int64_t)w.y[q]] += 1;
        m = (int64_t)La * Lb;
    } else if (test == ORC_SPEARMAN) {
        if (cap < 4) { free_scratch(&w); return -1; }
        int64_t *rx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        doubled_ranks(w.x, n, rx, w.buf, NULL);
        doubled_ranks(w.y, n, w.r2, w.buf, NULL);
        int64_t sab = 0, saa = 0, sbb = 0;
        for (int64_t q = 0; q < n; ++q) { sab += rx[q] * w.r2[q]; saa += rx[q] * rx[q]; sbb += w.r2[q] * w.r2[q]; }
        free(rx);
        out[0] = n; out[1] = sab; out[2] = saa; out[3] = sbb; m = 4;
    } else if (test == ORC_MWU || test == ORC_KRUSKAL) {
        int L = nlev[a];
        if (cap < 2 + 2 * (int64_t)L) { free_scratch(&w); return -1; }
        int64_t T = 0;
        doubled_ranks(w.y, n, w.r2, w.buf, &T);
        out[0] = n; out[1] = T;
        for (int g = 0; g < L; ++g) { out[2 + 2 * g] = 0; out[3 + 2 * g] = 0; }
        for (int64_t q = 0; q < n; ++q) { int g = (int)w.x[q]; out[2 + 2 * g] += 1; out[3 + 2 * g] += w.r2[q]; }
        m = 2 + 2 * (int64_t)L;
    } else if (test == ORC_ANOVA || test == ORC_TTEST) {
        int L = nlev[a];
        if (cap < 1 + (int64_t)L) { free_scratch(&w); return -1; }
        out[0] = n;
        for (int g = 0; g < L; ++g) out[1 + g] = 0;
        for (int64_t q = 0; q < n; ++q) out[1 + (int)w.x[q]] += 1;
        m = 1 + (int64_t)L;
    } else {
        if (cap < 1) { free_scratch(&w); return -1; }
        out[0] = n; m = 1;
    }
    free_scratch(&w);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Effect sizes (Table 2)                                                    */
/* ------------------------------------------------------------------------ */

/* One pair's effect sizes, from the test's own statistic on the co-observed
 * samples (NaN wherever that statistic is NaN):
 *   Pearson: e1 = r^2.  Spearman: e1 = rho.
 *   chi-squared: e1 = phi = sqrt(chi2 / n); e2 = Cramer's V =
 *     sqrt(chi2 / (n (min(k_a, k_b) - 1))) over the present levels, NaN when a
 *     variable has a single level (Sec. 3.5.4).
 *   t-test: e1 = Cohen's d = (mean_0 - mean_1) / s, s the pooled SD (Student)
 *     or sqrt((v_0 + v_1) / 2) (Welch); NaN when s = 0 (Sec. 3.5.5); e2 = the
 *     degrees of freedom of the t distribution (Welch-Satterthwaite, or
 *     n0 + n1 - 2), NaN when t is infinite.
 *   Mann-Whitney: e1 = Pearson's r = |z| / sqrt(n), z = (U_0 - n_0 n_1 / 2) / sigma
 *     with the tie-corrected sigma and no continuity correction; NaN when sigma = 0.
 *   ANOVA: e1 = partial eta^2 = SSB / (SSB + SSW) (one-way: the same as eta^2);
 *     1 when every group is constant and the groups differ (F = inf).
 *   Kruskal-Wallis: e1 = eta^2 = (H - k + 1) / (n - k); NaN when n <= k (Sec. 3.5.8).
 * e2 is NaN except for chi-squared. */
static void effect_pair(const orc_cohort *c, int test, int64_t a, int64_t b, orc_scratch *w,
                        double *e1, double *e2) {
    double st, pv;
    int32_t nn;
    *e1 = NAN;
    *e2 = NAN;
    pick(test)(c, a, b, w, &st, &pv, &nn);
    if (isnan(st)) return;
    const double n = (double)nn;
    switch (test) {
    case ORC_PEARSON:
        *e1 = st * st;
        return;
    case ORC_SPEARMAN:
        *e1 = st;
        return;
    case ORC_CHI2: {
        int pa[ORC_MAXLEV], pb[ORC_MAXLEV];
        int ka = present_levels(c, a, pa), kb = present_levels(c, b, pb);
        int m = (ka < kb ? ka : kb) - 1;
        *e1 = sqrt(st / n);
        if (m >= 1) *e2 = sqrt(st / (n * (double)m));
        return;
    }
    case ORC_TTEST: {
        int64_t cnt = gather_pair(c, a, b, w->x, w->y);
        double s0 = 0.0, s1 = 0.0;
        int64_t n0 = 0, n1 = 0;
        for (int64_t q = 0; q < cnt; ++q) {
            if (w->x[q] == 0.0) { s0 += w->y[q]; ++n0; } else { s1 += w->y[q]; ++n1; }
        }
        const double m0 = s0 / (double)n0, m1 = s1 / (double)n1;
        double q0 = 0.0, q1 = 0.0;
        for (int64_t q = 0; q < cnt; ++q) {
            if (w->x[q] == 0.0) q0 += (w->y[q] - m0) * (w->y[q] - m0);
            else q1 += (w->y[q] - m1) * (w->y[q] - m1);
        }
        const double v0 = q0 / (double)(n0 - 1), v1 = q1 / (double)(n1 - 1);
        const double s2 = c->welch ? 0.5 * (v0 + v1) : (q0 + q1) / (double)(n0 + n1 - 2);
        if (s2 > 0.0) *e1 = (m0 - m1) / sqrt(s2);
        /* second output: the degrees of freedom of the t distribution the
         * p-value comes from (Sec. 3.5.5): Welch-Satterthwaite for Welch,
         * n0 + n1 - 2 for Student; none when t is infinite */
        if (!isinf(st)) {
            if (c->welch) {
                const double a0 = v0 / (double)n0, a1 = v1 / (double)n1;
                *e2 = (a0 + a1) * (a0 + a1) / (a0 * a0 / (double)(n0 - 1) + a1 * a1 / (double)(n1 - 1));
            } else {
                *e2 = (double)(n0 + n1 - 2);
            }
        }
        return;
    }
    case ORC_MWU: {
        int64_t cnt = gather_pair(c, a, b, w->x, w->y);
        int64_t n0 = 0, n1 = 0, T = 0;
        for (int64_t q = 0; q < cnt; ++q) { if (w->x[q] == 0.0) ++n0; else ++n1; }
        doubled_ranks(w->y, cnt, w->r2, w->buf, &T);
        double R0 = 0.0;
        for (int64_t q = 0; q < cnt; ++q) if (w->x[q] == 0.0) R0 += 0.5 * (double)w->r2[q];
        const double U0 = R0 - 0.5 * (double)n0 * (double)(n0 + 1);
        const double var = (double)n0 * (double)n1 / 12.0 * ((n + 1.0) - (double)T / (n * (n - 1.0)));
        if (var > 0.0) *e1 = fabs((U0 - 0.5 * (double)n0 * (double)n1) / sqrt(var)) / sqrt(n);
        return;
    }
    case ORC_ANOVA: {
        if (isinf(st)) { *e1 = 1.0; return; }
        int present[ORC_MAXLEV], k, empty;
        int64_t ng[ORC_MAXLEV];
        int64_t cnt = group_pair(c, a, b, w, present, &k, ng, &empty);
        int L = c->nlev[a];
        double gm = 0.0, sum[ORC_MAXLEV];
        for (int g = 0; g < L; ++g) sum[g] = 0.0;
        for (int64_t q = 0; q < cnt; ++q) gm += w->y[q];
        gm /= (double)cnt;
        for (int64_t q = 0; q < cnt; ++q) sum[(int)w->x[q]] += w->y[q] - gm;
        double ssb = 0.0, ssw = 0.0;
        for (int g = 0; g < L; ++g)
            if (present[g]) ssb += sum[g] * sum[g] / (double)ng[g];
        for (int64_t q = 0; q < cnt; ++q) {
            const int g = (int)w->x[q];
            const double d = (w->y[q] - gm) - sum[g] / (double)ng[g];
            ssw += d * d;
        }
        if (ssb + ssw > 0.0) *e1 = ssb / (ssb + ssw);
        return;
    }
    case ORC_KRUSKAL: {
        int present[ORC_MAXLEV];
        int k = present_levels(c, a, present);
        if (n > (double)k) *e1 = (st - (double)k + 1.0) / (n - (double)k);
        return;
    }
    default:
        return;
    }
}

/* Effect sizes of all pairs, laid out as orc_run's outputs. */
int orc_effects(int test, const double *X, int64_t F, int64_t S, double miss,
                const uint8_t *vtype, const int32_t *nlev, const uint8_t *ctx,
                const int32_t *va, int32_t na, const int32_t *vb, int32_t nb,
                int welch, int yates, double *e1, double *e2, int nthreads) {
    orc_cohort c = { X, F, S, miss, vtype, nlev, ctx, welch, yates, 2, 1 };
    if (!pick(test) || na < 0 || nb < 0) return ORC_E_ARG;
    int rc = check_vars(&c, test, va, na, vb, nb);
    if (rc) return rc;
    rc = orc_validate(X, F, S, miss, vtype, nlev);
    if (rc) return rc;
    const int32_t *cols = vb ? vb : va;
    int64_t ncols = vb ? nb : na;
    int64_t total = (int64_t)na * ncols;
    int err = 0;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();   /* this call only */
#else
    const int nt = 1;
    (void)nthreads;
#endif
    (void)nt;
#pragma omp parallel num_threads(nt)
    {
        orc_scratch w;
        int ok = alloc_scratch(&w, S) == ORC_OK;
        if (!ok) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < total; ++q) {
            if (!ok) continue;
            double x1, x2;
            effect_pair(&c, test, va[q / ncols], cols[q % ncols], &w, &x1, &x2);
            if (e1) e1[q] = x1;
            if (e2) e2[q] = x2;
        }
        free_scratch(&w);
    }
    return err ? ORC_E_OOM : ORC_OK;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
