// Device FP64 special functions for the p-values of Sec. 3.5 (Pearson/Spearman:
// Beta CDF; t: t survival; ANOVA: F survival; chi-squared and Kruskal-Wallis:
// chi-squared survival; Mann-Whitney: normal survival).
//
// Methods (published; this file is written from the mathematics):
//  * I_x(a,b): continued fraction of DLMF 8.17.22, evaluated by the modified
//    Lentz method. When the first parameter is the larger one its odd partial
//    numerators approach -1, so the fraction is evaluated through its even part
//    with 1 + d_{2m+1} expanded algebraically (no cancellation). The symmetry
//    I_x(a,b) = 1 - I_{1-x}(b,a) (DLMF 8.17.4) is used for x > (a+1)/(a+b+2).
//  * The prefactor x^a (1-x)^b / B(a,b) follows the scaling of DiDonato &
//    Morris (ACM TOMS 708, 1992): for a, b >= 10 it is written with the
//    Stirling remainder Delta(.) (DLMF 5.11.1, Bernoulli series) and
//    rlog1(z) = z - log(1+z), which keeps full precision for large degrees of
//    freedom.
//  * Q(a,x): series of DLMF 8.7.1 for x < a+1, Legendre's continued fraction
//    (DLMF 8.9.2, even part) otherwise, with the same scaled prefactor.
// CUDA's own lgamma/log/log1p/exp/erfc/sqrt are called, never re-implemented.
#pragma once

#include <math.h>

namespace napg {
namespace sf {

// log Gamma(k/2), k = 1..40, from Gamma(n) = (n-1)! and
// Gamma(n + 1/2) = (2n)! sqrt(pi) / (4^n n!) (evaluated to 40 digits, rounded).
__constant__ double kLogGammaHalf[40] = {
    0.5723649429247001,
    0.0,
    -0.12078223763524522,
    0.0,
    0.2846828704729192,
    0.6931471805599453,
    1.2009736023470743,
    1.791759469228055,
    2.4537365708424423,
    3.1780538303479458,
    3.9578139676187165,
    4.787491742782046,
    5.662562059857142,
    6.579251212010101,
    7.534364236758733,
    8.525161361065415,
    9.549267257300997,
    10.60460290274525,
    11.689333420797269,
    12.801827480081469,
    13.940625219403763,
    15.104412573075516,
    16.292000476567242,
    17.502307845873887,
    18.734347511936445,
    19.987214495661885,
    21.2600761562447,
    22.552163853123425,
    23.862765841689086,
    25.19122118273868,
    26.536914491115613,
    27.89927138384089,
    29.277754515040815,
    30.671860106080672,
    32.08111489594735,
    33.50507345013689,
    34.943315776876815,
    36.39544520803305,
    37.861086508961094,
    39.339884187199495};

// log Gamma(a): table for the half-integers the test p-values use (degrees of
// freedom / 2), the library function otherwise.
__device__ __forceinline__ double lgamma_fast(double a) {
    const double k = 2.0 * a;
    if (k >= 1.0 && k <= 40.0 && k == floor(k)) return kLogGammaHalf[(int)k - 1];
    return lgamma(a);
}

__device__ __forceinline__ double stirling_rem(double a) {
    // Delta(a) = lgamma(a) - ((a - 1/2) log a - a + log(2 pi)/2)
    if (a < 10.0) return lgamma_fast(a) - ((a - 0.5) * log(a) - a + 0.91893853320467274178);
    const double inv = 1.0 / a, q = inv * inv;
    // Bernoulli terms B_{2k} / (2k (2k-1) a^{2k-1}), k = 1..6
    double s = -691.0 / 360360.0;
    s = s * q + 1.0 / 1188.0;
    s = s * q - 1.0 / 1680.0;
    s = s * q + 1.0 / 1260.0;
    s = s * q - 1.0 / 360.0;
    s = s * q + 1.0 / 12.0;
    return s * inv;
}

__device__ __forceinline__ double rlog1(double z) {
    // z - log(1+z); for |z| <= 1/2 via u = z/(2+z): z - log(1+z) = u z - 2 sum_{k>=1} u^{2k+1}/(2k+1)
    if (z < -0.5 || z > 0.5) return z - log1p(z);
    const double u = z / (2.0 + z), u2 = u * u;
    double pw = u * u2, acc = 0.0;
    for (int k = 3; k < 121; k += 2) {
        const double t = pw / (double)k;
        acc += t;
        if (fabs(t) <= 1e-18 * fabs(acc)) break;
        pw *= u2;
    }
    return u * z - 2.0 * acc;
}

// log Gamma(big + small) - log Gamma(big), big >= 10
__device__ __forceinline__ double lgamma_shift(double small, double big) {
    return small * log(big) + (small + big - 0.5) * log1p(small / big) - small
           + stirling_rem(big + small) - stirling_rem(big);
}

// x^a y^b / B(a,b) with x + y = 1
static __device__ double beta_prefactor(double a, double b, double x, double y) {
    if (a >= 10.0 && b >= 10.0) {
        const double lam = (x <= 0.5) ? ((a + b) * x - a) : (b - (a + b) * y);
        const double e = -a * rlog1(lam / a) - b * rlog1(-lam / b)
                         - stirling_rem(a) - stirling_rem(b) + stirling_rem(a + b);
        return sqrt(a * b / (6.283185307179586477 * (a + b))) * exp(e);
    }
    const double lx = (x <= 0.5) ? log(x) : log1p(-y);
    const double ly = (y <= 0.5) ? log(y) : log1p(-x);
    const double lo = fmin(a, b), hi = fmax(a, b);
    const double lbeta = (hi >= 10.0) ? (lgamma_fast(lo) - lgamma_shift(lo, hi))
                                      : (lgamma_fast(a) + lgamma_fast(b) - lgamma_fast(a + b));
    return exp(a * lx + b * ly - lbeta);
}

// partial numerator d_k of DLMF 8.17.22
__device__ __forceinline__ double cf_d(double a, double b, double x, int k) {
    if ((k & 1) == 0) {
        const double m = (double)(k >> 1);
        return m * (b - m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));
    }
    const double m = (double)(k >> 1);
    return -(a + m) * (a + b + m) * x / ((a + 2.0 * m) * (a + 2.0 * m + 1.0));
}

// 1 + d_{2m+1} without cancellation (y = 1 - x)
__device__ __forceinline__ double cf_one_plus_odd(double a, double b, double y, int m) {
    const double md = (double)m;
    const double num = a * (2.0 * md + 1.0 - b) + md * (3.0 * md + 2.0 - b) + (a + md) * (a + b + md) * y;
    return num / ((a + 2.0 * md) * (a + 2.0 * md + 1.0));
}

constexpr int kMaxIter = 200000;
constexpr double kTiny = 1e-300;

// value of 1/(1 + d1/(1 + d2/(1 + ...)))
static __device__ double cf_plain(double a, double b, double x) {
    double f = kTiny, C = kTiny, D = 0.0;
    for (int n = 1; n < kMaxIter; ++n) {
        const double an = (n == 1) ? 1.0 : cf_d(a, b, x, n - 1);
        D = 1.0 + an * D;
        D = (fabs(D) < kTiny) ? kTiny : D;
        C = 1.0 + an / C;
        C = (fabs(C) < kTiny) ? kTiny : C;
        D = 1.0 / D;
        const double del = C * D;
        f *= del;
        if (fabs(del - 1.0) < 1e-15) break;
    }
    return f;
}

// the same value through the even part 1/(1 + d1 - d1 d2/(1 + d2 + d3 - d3 d4/(...)))
static __device__ double cf_even(double a, double b, double x, double y) {
    double f = cf_one_plus_odd(a, b, y, 0);
    f = (fabs(f) < kTiny) ? kTiny : f;
    double C = f, D = 0.0;
    for (int m = 1; m < kMaxIter; ++m) {
        const double d_odd = cf_d(a, b, x, 2 * m - 1), d_even = cf_d(a, b, x, 2 * m);
        const double an = -d_odd * d_even;
        const double bn = d_even + cf_one_plus_odd(a, b, y, m);
        D = bn + an * D;
        D = (fabs(D) < kTiny) ? kTiny : D;
        C = bn + an / C;
        C = (fabs(C) < kTiny) ? kTiny : C;
        D = 1.0 / D;
        const double del = C * D;
        f *= del;
        if (fabs(del - 1.0) < 1e-15) break;
    }
    return 1.0 / f;
}

static __device__ double ibeta_lower(double a, double b, double x, double y) {
    const double cf = (a >= b) ? cf_even(a, b, x, y) : cf_plain(a, b, x);
    return beta_prefactor(a, b, x, y) / a * cf;
}

// regularized I_x(a,b) with x + y = 1 supplied
static __device__ double ibeta(double a, double b, double x, double y) {
    if (!(a > 0.0) || !(b > 0.0) || isnan(x) || isnan(y)) return nan("");
    if (x <= 0.0) return 0.0;
    if (y <= 0.0) return 1.0;
    if (x > (a + 1.0) / (a + b + 2.0)) return 1.0 - ibeta_lower(b, a, y, x);
    return ibeta_lower(a, b, x, y);
}

// x^a e^{-x} / Gamma(a)
__device__ __forceinline__ double gamma_prefactor(double a, double x) {
    if (a >= 10.0) return sqrt(a / 6.283185307179586477) * exp(-a * rlog1((x - a) / a) - stirling_rem(a));
    return exp(a * log(x) - x - lgamma_fast(a));
}

// regularized upper incomplete gamma Q(a, x)
static __device__ double gamma_q(double a, double x) {
    if (!(a > 0.0) || isnan(x)) return nan("");
    if (x <= 0.0) return 1.0;
    if (isinf(x)) return 0.0;
    if (x < a + 1.0) {
        double term = 1.0, sum = 1.0;
        for (int k = 1; k < kMaxIter; ++k) {
            term *= x / (a + (double)k);
            sum += term;
            if (term < sum * 1e-18) break;
        }
        return 1.0 - gamma_prefactor(a, x) / a * sum;
    }
    double f = kTiny, C = kTiny, D = 0.0;
    for (int n = 1; n < kMaxIter; ++n) {
        const double an = (n == 1) ? 1.0 : -(double)(n - 1) * ((double)(n - 1) - a);
        const double bn = x + 2.0 * (double)n - 1.0 - a;
        D = bn + an * D;
        D = (fabs(D) < kTiny) ? kTiny : D;
        C = bn + an / C;
        C = (fabs(C) < kTiny) ? kTiny : C;
        D = 1.0 / D;
        const double del = C * D;
        f *= del;
        if (fabs(del - 1.0) < 1e-15) break;
    }
    return gamma_prefactor(a, x) * f;
}

// two-sided p of Student t with df degrees of freedom
__device__ __forceinline__ double t_two_sided(double t, double df) {
    if (isnan(t) || !(df > 0.0)) return nan("");
    if (isinf(t)) return 0.0;
    const double t2 = t * t;
    return ibeta(0.5 * df, 0.5, df / (df + t2), t2 / (df + t2));
}

// p of a correlation coefficient with n observations: I_{1-r^2}((n-2)/2, 1/2)
__device__ __forceinline__ double corr_p(double r, double n) {
    if (isnan(r) || n <= 2.0) return nan("");
    if (fabs(r) >= 1.0) return 0.0;
    return ibeta(0.5 * (n - 2.0), 0.5, (1.0 - r) * (1.0 + r), r * r);
}

// survival function of F(d1, d2)
__device__ __forceinline__ double f_sf(double F, double d1, double d2) {
    if (isnan(F) || !(d1 > 0.0) || !(d2 > 0.0)) return nan("");
    if (isinf(F)) return 0.0;
    if (F <= 0.0) return 1.0;
    const double den = d2 + d1 * F;
    return ibeta(0.5 * d2, 0.5 * d1, d2 / den, d1 * F / den);
}

__device__ __forceinline__ double chi2_sf(double x, double df) {
    if (isnan(x) || !(df > 0.0)) return nan("");
    return gamma_q(0.5 * df, 0.5 * x);
}

__device__ __forceinline__ double norm_sf(double z) { return 0.5 * erfc(z * 0.70710678118654752440); }

}  // namespace sf
}  // namespace napg
