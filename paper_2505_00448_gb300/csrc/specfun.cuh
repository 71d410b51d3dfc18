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
//  * For a >= 20, b <= 32 (integer or half-integer) and x >= 1/2, an
//    expansion of the integrand in w = -ln t around the Gamma(b) limit
//    (the idea of DiDonato & Morris's large-a expansion, derived in full at
//    ibeta_large_a): a few terms in 1/T^2 replace about sqrt(a) fraction steps.
//  * Q(a,x): series of DLMF 8.7.1 for x < a+1, Legendre's continued fraction
//    (DLMF 8.9.2, even part) otherwise, with the same scaled prefactor.
// CUDA's own lgamma/log/log1p/exp/erfc/erfcx/sqrt are called, never re-implemented.
#pragma once

#include <math.h>

namespace napg {
namespace sf {

// log Gamma(k/2), k = 1..40, from Gamma(n) = (n-1)! and
// Gamma(n + 1/2) = (2n)! sqrt(pi) / (4^n n!) (evaluated to 40 digits, rounded).
static __constant__ double kLogGammaHalf[40] = {
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

// Delta(a) = lgamma(a) - ((a - 1/2) log a - a + log(2 pi)/2) for a >= 10 from
// inv = 1/a: Bernoulli terms B_{2k} / (2k (2k-1) a^{2k-1}), k = 1..6
__device__ __forceinline__ double stirling_series(double inv) {
    const double q = inv * inv;
    double s = -691.0 / 360360.0;
    s = s * q + 1.0 / 1188.0;
    s = s * q - 1.0 / 1680.0;
    s = s * q + 1.0 / 1260.0;
    s = s * q - 1.0 / 360.0;
    s = s * q + 1.0 / 12.0;
    return s * inv;
}

__device__ __forceinline__ double stirling_rem(double a) {
    if (a < 10.0) return lgamma_fast(a) - ((a - 0.5) * log(a) - a + 0.91893853320467274178);
    return stirling_series(1.0 / a);
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
    const double pf = beta_prefactor(a, b, x, y);
    if (pf == 0.0) return 0.0;   // underflowed: the (bounded) fraction cannot lift it
    const double cf = (a >= b) ? cf_even(a, b, x, y) : cf_plain(a, b, x);
    return pf / a * cf;
}

// k e_k = (-1)^(k+1) zeta(2k) / (2 pi)^(2k), k = 1..20: the Taylor coefficients
// of (d/ds) s log(sinh(w/2)/(w/2)) in s = w^2 (B_2k = (-1)^(k+1) 2 (2k)! zeta(2k)
// / (2 pi)^(2k)); evaluated to 40 digits, rounded.
static __constant__ double kSinhLogCoef[20] = {
    4.1666666666666667e-2, -6.9444444444444444e-4, 1.6534391534391534e-5, -4.1335978835978836e-7,
    1.0438378493934049e-8, -2.6420950693437466e-10, 6.6912682653423394e-12, -1.6948401481612914e-13,
    4.2930310281389223e-15, -1.0874343492790309e-16, 2.7545014141801148e-18, -6.9772323429062617e-20,
    1.7673535198147337e-21, -4.4767587135187734e-23, 1.1339762261688415e-24, -2.8723953344361012e-26,
    7.2758623780743245e-28, -1.8429974703326551e-29, 4.6683671285475223e-31, -1.182511207850315e-32};

// I_x(a,b) is below the smallest subnormal when a >= 20, b <= 32 and a y >= 2000:
// then -a ln x >= a y >= 2000 while the remaining factor of the integral,
// Gamma(a+b) / (Gamma(a+1) Gamma(b)) max(1, y^(b-1)), stays far below e^1200.
// I_x(a, b) certainly below half the least subnormal (so 0 in FP64):
// a y >= 2000 for b <= 32 (the expansion below: p <= 2 e^-u u^(b+41), u >= a y);
// for b = 1/2 with x = 1 - y >= 1/2, u = -T log x >= T y >= 746 already does
// it (the expansion's sum is erfcx(sqrt u) (1 + e), |e| < 0.05, since its first
// correction is at most (1/64) 1.33 u^2 / T^2 with u <= T log 2; M < 1.001; and
// erfcx(z) <= 1 / (z sqrt(pi)), so p < 1.06 e^-u / sqrt(pi u) < 2^-1075).
__device__ __forceinline__ bool ibeta_underflows(double a, double b, double y) {
    if (b == 0.5 && a >= 20.0 && y <= 0.5 && (a - 0.25) * y >= 746.0) return true;
    return a >= 20.0 && b <= 32.0 && a * y >= 2000.0;
}

// erfcx(sqrt u) = e^u erfc(sqrt u) for u >= 0, and sqrt u in su: the library's
// own erfcx for the p-value expansions, near-minimax polynomials fitted to the
// function in 40-digit arithmetic (erfcx_fit.py writes erfcx_coefs.inc; within
// 3.2e-16 relative of it over 0 <= z <= 1e4, checked against CUDA's erfcx in the
// tests). For z = sqrt u >= 4 it takes g(w) = sqrt(pi) z erfcx(z) as a
// polynomial in w = 1/u, with z and 1/z from one reciprocal square root: about 25
// FP64 instructions where sqrt and erfcx take about 58; below, eight pieces of
// width 1/2 in z.
#include "erfcx_coefs.inc"

__device__ __forceinline__ double erfcx_of_sqrt(double u, double &su) {
    if (u >= 16.0) {
        const double r = rsqrt(u), w = r * r;
        su = u * r;
        double g;
        if (w >= 0.015625) {
            g = kErfcxMid[kErfcxMidTerms - 1];
#pragma unroll
            for (int i = kErfcxMidTerms - 2; i >= 0; --i) g = fma(g, w, kErfcxMid[i]);
        } else {
            g = kErfcxFar[kErfcxFarTerms - 1];
#pragma unroll
            for (int i = kErfcxFarTerms - 2; i >= 0; --i) g = fma(g, w, kErfcxFar[i]);
        }
        return g * r * 0.56418958354775628695;       // 1 / sqrt(pi)
    }
    su = sqrt(u);
    const int k = min(7, (int)(su * 2.0));          // piece [k/2, k/2 + 1/2)
    const double t = su - (0.5 * (double)k + 0.25);
    const double *c = kErfcxPiece + k * kErfcxPieceTerms;
    double acc = c[kErfcxPieceTerms - 1];
#pragma unroll
    for (int i = kErfcxPieceTerms - 2; i >= 0; --i) acc = fma(acc, t, c[i]);
    return acc;
}

// The expansion below applies to I_x(a,b) with a large, b a moderate integer or
// half-integer and x >= 1/2 (the p-values of t, F and r near the null, where the
// continued fraction needs about sqrt(a) steps).
__device__ __forceinline__ bool ibeta_large_a_applies(double a, double b, double x) {
    return x >= 0.5 && a >= 20.0 && b <= 32.0 && b <= a && 2.0 * b == floor(2.0 * b);
}

// I_x(a,b) for large a. With t = e^-w the integrand of I_x is
// e^{-T w} w^{b-1} phi(w), T = a + (b-1)/2, phi(w) = (sinh(w/2)/(w/2))^{b-1}
// (even in w). Expanding phi = sum_k g_k w^{2k} and integrating term by term
// from w0 = -ln x gives
//   I_x(a,b) = M sum_k g_k (b)_{2k} Q(b+2k, u) / T^{2k},  u = T w0,
//   M = Gamma(a+b) / (Gamma(a) T^b) = 1 + O(1/T^2),
// an expansion in 1/T^2 (and, in the tail, a convergent series in (w0/2pi)^2).
// phi = exp((b-1) sum_k e_k w^{2k}) gives g_n = ((b-1)/n) sum_{k<=n} k e_k g_{n-k}.
// Q(b+j, u) climbs from Q(1/2,u) = erfc(sqrt u) or Q(1,u) = e^-u by
// Q(s+1,u) = Q(s,u) + e^-u u^s / Gamma(s+1); the ladder is kept scaled by e^u
// (erfcx) so that it does not underflow before the final product.
// 2/m, m = 1..160 (entry 0 unused): 1/s for the half-integer steps s = m/2 of
// the ladder below, correctly rounded
static __constant__ double kInvHalf[161] = {
    0.0, 2.0, 1.0, 0.6666666666666666, 0.5, 0.4, 0.3333333333333333, 0.2857142857142857,
    0.25, 0.2222222222222222, 0.2, 0.18181818181818182, 0.16666666666666666, 0.15384615384615385, 0.14285714285714285, 0.13333333333333333,
    0.125, 0.11764705882352941, 0.1111111111111111, 0.10526315789473684, 0.1, 0.09523809523809523, 0.09090909090909091, 0.08695652173913043,
    0.08333333333333333, 0.08, 0.07692307692307693, 0.07407407407407407, 0.07142857142857142, 0.06896551724137931, 0.06666666666666667, 0.06451612903225806,
    0.0625, 0.06060606060606061, 0.058823529411764705, 0.05714285714285714, 0.05555555555555555, 0.05405405405405406, 0.05263157894736842, 0.05128205128205128,
    0.05, 0.04878048780487805, 0.047619047619047616, 0.046511627906976744, 0.045454545454545456, 0.044444444444444446, 0.043478260869565216, 0.0425531914893617,
    0.041666666666666664, 0.04081632653061224, 0.04, 0.0392156862745098, 0.038461538461538464, 0.03773584905660377, 0.037037037037037035, 0.03636363636363636,
    0.03571428571428571, 0.03508771929824561, 0.034482758620689655, 0.03389830508474576, 0.03333333333333333, 0.03278688524590164, 0.03225806451612903, 0.031746031746031744,
    0.03125, 0.03076923076923077, 0.030303030303030304, 0.029850746268656716, 0.029411764705882353, 0.028985507246376812, 0.02857142857142857, 0.028169014084507043,
    0.027777777777777776, 0.0273972602739726, 0.02702702702702703, 0.02666666666666667, 0.02631578947368421, 0.025974025974025976, 0.02564102564102564, 0.02531645569620253,
    0.025, 0.024691358024691357, 0.024390243902439025, 0.024096385542168676, 0.023809523809523808, 0.023529411764705882, 0.023255813953488372, 0.022988505747126436,
    0.022727272727272728, 0.02247191011235955, 0.022222222222222223, 0.02197802197802198, 0.021739130434782608, 0.021505376344086023, 0.02127659574468085, 0.021052631578947368,
    0.020833333333333332, 0.020618556701030927, 0.02040816326530612, 0.020202020202020204, 0.02, 0.019801980198019802, 0.0196078431372549, 0.019417475728155338,
    0.019230769230769232, 0.01904761904761905, 0.018867924528301886, 0.018691588785046728, 0.018518518518518517, 0.01834862385321101, 0.01818181818181818, 0.018018018018018018,
    0.017857142857142856, 0.017699115044247787, 0.017543859649122806, 0.017391304347826087, 0.017241379310344827, 0.017094017094017096, 0.01694915254237288, 0.01680672268907563,
    0.016666666666666666, 0.01652892561983471, 0.01639344262295082, 0.016260162601626018, 0.016129032258064516, 0.016, 0.015873015873015872, 0.015748031496062992,
    0.015625, 0.015503875968992248, 0.015384615384615385, 0.015267175572519083, 0.015151515151515152, 0.015037593984962405, 0.014925373134328358, 0.014814814814814815,
    0.014705882352941176, 0.014598540145985401, 0.014492753623188406, 0.014388489208633094, 0.014285714285714285, 0.014184397163120567, 0.014084507042253521, 0.013986013986013986,
    0.013888888888888888, 0.013793103448275862, 0.0136986301369863, 0.013605442176870748, 0.013513513513513514, 0.013422818791946308, 0.013333333333333334, 0.013245033112582781,
    0.013157894736842105, 0.013071895424836602, 0.012987012987012988, 0.012903225806451613, 0.01282051282051282, 0.012738853503184714, 0.012658227848101266, 0.012578616352201259,
    0.0125};

// 4 / ((m + 2)(m + 4)), m = 0..156: two rungs of the ladder below at once,
// correctly rounded
static __constant__ double kInvQuad[157] = {
    0.5, 0.26666666666666666, 0.16666666666666666, 0.11428571428571428, 0.08333333333333333, 0.06349206349206349, 0.05, 0.04040404040404041,
    0.03333333333333333, 0.027972027972027972, 0.023809523809523808, 0.020512820512820513, 0.017857142857142856, 0.01568627450980392, 0.013888888888888888, 0.01238390092879257,
    0.011111111111111112, 0.010025062656641603, 0.00909090909090909, 0.008281573498964804, 0.007575757575757576, 0.006956521739130435, 0.00641025641025641, 0.005925925925925926,
    0.005494505494505495, 0.005108556832694764, 0.004761904761904762, 0.004449388209121246, 0.004166666666666667, 0.0039100684261974585, 0.003676470588235294, 0.003463203463203463,
    0.0032679738562091504, 0.003088803088803089, 0.0029239766081871343, 0.002772002772002772, 0.002631578947368421, 0.0025015634771732333, 0.002380952380952381, 0.0022688598979013048,
    0.0021645021645021645, 0.0020671834625322996, 0.001976284584980237, 0.0018912529550827422, 0.0018115942028985507, 0.0017368649587494573, 0.0016666666666666668, 0.001600640256102441,
    0.0015384615384615385, 0.0014798372179060304, 0.0014245014245014246, 0.0013722126929674098, 0.0013227513227513227, 0.0012759170653907496, 0.0012315270935960591, 0.0011894142134998512,
    0.0011494252873563218, 0.0011114198388441233, 0.001075268817204301, 0.0010408534998698933, 0.0010080645161290322, 0.0009768009768009768, 0.000946969696969697, 0.0009184845005740528,
    0.00089126559714795, 0.0008652390222799049, 0.0008403361344537816, 0.0008164931618697694, 0.0007936507936507937, 0.0007717538105344395, 0.0007507507507507507, 0.0007305936073059361,
    0.0007112375533428165, 0.0006926406926406926, 0.0006747638326585695, 0.0006575702778234424, 0.000641025641025641, 0.0006250976715111736, 0.0006097560975609756, 0.0005949724825226833,
    0.0005807200929152149, 0.0005669737774627923, 0.0005537098560354374, 0.0005409060175794456, 0.0005285412262156448, 0.0005165956347668862, 0.000505050505050505, 0.0004938881343375726,
    0.0004830917874396135, 0.0004726456339359565, 0.00046253469010175765, 0.0004527447651386531, 0.0004432624113475177, 0.0004340748779164406, 0.00042517006802721087, 0.0004165364990107258,
    0.00040816326530612246, 0.00040004000400040005, 0.000392156862745098, 0.00038450446986446215, 0.0003770739064856712, 0.0003698566805362922, 0.000362844702467344, 0.00035603026257231867,
    0.00034940600978336826, 0.0003429649318357198, 0.0003367003367003367, 0.00033060583519299114, 0.0003246753246753247, 0.0003189029737702304, 0.0003132832080200501, 0.00030781069642170063,
    0.00030248033877797946, 0.00029728725380899295, 0.0002922267679719462, 0.0002872944049414638, 0.0002824858757062147, 0.0002777970692409195, 0.000273224043715847, 0.00026876301820869447,
    0.00026441036488630354, 0.00026016260162601624, 0.0002560163850486431, 0.0002519685039370079, 0.000248015873015873, 0.00024415552707074406, 0.0002403846153846154, 0.0002367003964731641,
    0.0002331002331002331, 0.00022958158755667795, 0.0002261420171867933, 0.0002227791701475912, 0.00021949078138718174, 0.00021627466882941334, 0.00021312872975277067, 0.00021005093735230792,
    0.00020703933747412008, 0.00020409204551252616, 0.00020120724346076458, 0.00019838317710658135, 0.00019561815336463224, 0.00019291053773812393, 0.0001902587519025875, 0.00018766127140511376,
    0.00018511662347278786, 0.00018262338492443957, 0.00018018018018018018, 0.00017778567936352726, 0.00017543859649122806, 0.00017313768774618015, 0.00017088174982911826, 0.0001686696183849884,
    0.0001665001665001665, 0.00016437230326689953, 0.0001622849724115547, 0.0001602371509834555, 0.00015822784810126583};

// binary exponent field of a double (0 for zero and subnormals): magnitude
// comparisons on the integer pipe
__device__ __forceinline__ int expo_field(double v) { return (__double2hiint(v) >> 20) & 0x7FF; }

// ln(1 - y) for 0 <= y < 2^-7 from its Taylor series (DLMF 4.6.1),
// -(y + y^2 (1/2 + y/3 + ... + y^6/8)): the first omitted term, y^9/9, is below
// 2^-56 of the sum, and the leading term y is exact, so the result is within
// about one unit in the last place. Eight FP64 instructions where log1p takes
// about two dozen; the large-a expansion's jobs mostly have such y (r^2 of
// weak correlations, the beta argument of small F and t).
__device__ __forceinline__ double log1m_small(double y) {
    double p = 0.125;
    p = fma(p, y, 1.0 / 7.0);
    p = fma(p, y, 1.0 / 6.0);
    p = fma(p, y, 0.2);
    p = fma(p, y, 0.25);
    p = fma(p, y, 1.0 / 3.0);
    p = fma(p, y, 0.5);
    return -fma(y * y, p, y);
}

// c_k(b) = g_k (b)_{2k}, k = 1..20: the coefficients of the expansion below for
// one b (row 2b - 1 of a table of kBgratRows rows), by the recurrence for g_k
constexpr int kBgratTerms = 20, kBgratRows = 64;

__device__ __forceinline__ void bgrat_coefs(double b, double *c) {
    const double beta = b - 1.0;
    double g[kBgratTerms + 1];
    g[0] = 1.0;
    double poch = 1.0;
#pragma unroll
    for (int k = 1; k <= kBgratTerms; ++k) {
        double acc = 0.0;
#pragma unroll
        for (int i = 1; i <= k; ++i) acc = fma(kSinhLogCoef[i - 1], g[k - i], acc);
        g[k] = beta * acc * (1.0 / (double)k);
        poch *= (b + (double)(2 * k - 2)) * (b + (double)(2 * k - 1));
        c[k - 1] = g[k] * poch;
    }
}

// log M for b = 1/2: log Gamma(T + 3/4) - log Gamma(T - 1/4) - (1/2) log T
// = -sum_m 2 B_{2m+1}(3/4) / (2m (2m+1) T^{2m}) (DLMF 5.11.8; the odd powers
// cancel because 3/4 + 1/4 = 1); six terms reach 1e-20 at T = 20.
__device__ __forceinline__ double log_m_half(double invT2) {
    double s = -0.0067123894890149434408;
    s = fma(s, invT2, 0.0024090290069580078125);
    s = fma(s, invT2, -0.00132083892822265625);
    s = fma(s, invT2, 0.0012410481770833333333);
    s = fma(s, invT2, -0.00244140625);
    s = fma(s, invT2, 0.015625);
    return s * invT2;
}

// log M and 1/T^2 of the expansion below for one (a, b), T = a + (b - 1)/2
__device__ __forceinline__ void large_a_consts(double a, double b, double &logM, double &invT2) {
    const double T = a + 0.5 * (b - 1.0);
    invT2 = 1.0 / (T * T);
    if (b == 0.5) {
        logM = log_m_half(invT2);
    } else {
        // log M from the Stirling forms of log Gamma(a+b) and log Gamma(a)
        const double inv_a = 1.0 / a;
        logM = (a + b - 0.5) * log1p(b * inv_a) - b * log1p((b - 1.0) * 0.5 * inv_a) - b
               + stirling_series(1.0 / (a + b)) - stirling_series(inv_a);
    }
}

// large_a_consts on the half-integer grid the test p-values use (a = df/2,
// b = d1/2): v[(2b - 1) (n2a + 1) + 2a] = {log M, 1/T^2} for 2a = 0..n2a,
// 2b = 1..rows (entries with a < 20 unused). Formed once by the same function,
// so a lookup gives the values the job would compute.
struct LargeATab {
    const double2 *v;
    int32_t n2a, rows;
};

// coef: the table row c_k(b) (see bgrat_coefs), or NULL to form it here;
// lat: the (log M, 1/T^2) table (lat.v NULL: formed here)
static __device__ double ibeta_large_a(double a, double b, double x, double y, const double *coef,
                                       LargeATab lat) {
    const double T = a + 0.5 * (b - 1.0);
    const double u = -T * ((x <= 0.5) ? log(x) : (y < 0.0078125 ? log1m_small(y) : log1p(-y)));
    // the result is below the smallest subnormal: for b = 1/2 once u >= 746
    // (see ibeta_underflows), else when p <= 2 e^-u u^(b+41) is
    if (b == 0.5 && u >= 746.0) return 0.0;
    if (u > 700.0 && u - (b + 41.0) * log(u) > 760.0) return 0.0;
    double logM, invT2;
    const double a2 = 2.0 * a, b2 = 2.0 * b;    // b2 is an integer here
    if (lat.v && a2 <= (double)lat.n2a && b2 <= (double)lat.rows && a2 == floor(a2)) {
        const double2 e = lat.v[((int64_t)b2 - 1) * ((int64_t)lat.n2a + 1) + (int64_t)a2];
        logM = e.x;
        invT2 = e.y;
    } else {
        large_a_consts(a, b, logM, invT2);
    }
    int m;             // 2 s
    double Q, th;      // Q = e^u Q(s,u), th = u^s / Gamma(s+1)
    if (b == floor(b)) {
        m = 2; Q = 1.0; th = u;
    } else {
        double su;
        m = 1; Q = erfcx_of_sqrt(u, su); th = su * 1.1283791670955125739;   // sqrt(u) / Gamma(3/2)
    }
    const int mb = (int)(2.0 * b);
    while (m < mb) {
        Q += th;
        m += 2;
        th *= u * kInvHalf[m];
    }
    double cbuf[kBgratTerms];
    const double *c = coef;
    if (!c) {
        bgrat_coefs(b, cbuf);
        c = cbuf;
    }
    double sum = Q, pw = 1.0;
    const double u2 = u * u;
    int small = 0;
#pragma unroll
    for (int k = 1; k <= kBgratTerms; ++k) {
        // two rungs: Q += th + th u 2/(m+2), th <- th u^2 4/((m+2)(m+4))
        Q = fma(th, fma(u, kInvHalf[m + 2], 1.0), Q);
        th *= u2 * kInvQuad[m];
        m += 4;
        pw *= invT2;
        const double term = c[k - 1] * pw * Q;
        sum += term;
        // two consecutive negligible terms, |term| < 2^-56 |sum| (a single c_k
        // can vanish for some b)
        if (expo_field(term) + 57 <= expo_field(sum)) {
            if (++small == 2) break;
        } else {
            small = 0;
        }
    }
    const double e = logM - u;
    if (e > -700.0) return exp(e) * sum;
    return exp(e + log(sum));
}

// regularized I_x(a,b) with x + y = 1 supplied; bgrat: table of c_k(b) rows
// for 2b = 1..kBgratRows (or NULL); lat: see LargeATab (or empty)
static __device__ double ibeta(double a, double b, double x, double y, const double *bgrat = nullptr,
                               LargeATab lat = LargeATab{nullptr, 0, 0}) {
    if (!(a > 0.0) || !(b > 0.0) || isnan(x) || isnan(y)) return nan("");
    if (x <= 0.0) return 0.0;
    if (y <= 0.0) return 1.0;
    if (ibeta_underflows(a, b, y)) return 0.0;
    if (ibeta_large_a_applies(a, b, x))
        return ibeta_large_a(a, b, x, y, bgrat ? bgrat + ((int)(2.0 * b) - 1) * kBgratTerms : nullptr, lat);
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
    const double pf = gamma_prefactor(a, x);
    if (pf == 0.0) return 0.0;
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
    return pf * f;
}

// Q(a, x) for 2a a positive integer up to kInvHalf's range (the chi-squared
// p-values: a = df / 2), x > 0 finite, as the finite sums of DLMF 8.4.10-8.4.11
// (repeated integration by parts of Gamma(a, x)):
//   a = n:        Q = e^-x sum_{j<n} x^j / j!
//   a = n + 1/2:  Q = erfc(sqrt x) + e^-x sum_{j<n} x^{j+1/2} / Gamma(j + 3/2).
// Every term is positive (no cancellation; relative error about a + 25 units
// in the last place) and there are at most a of them, where the series or the
// continued fraction would take tens to hundreds of steps with a division each.
// The sum is formed scaled by e^x (erfc(sqrt x) e^x = erfcx(sqrt x)) with the
// ladder th <- th x 2/s of the large-a expansion below.
constexpr int kGammaLadderMax = 160;     // 2a up to kInvHalf's last entry

__device__ __forceinline__ bool gamma_ladder_applies(double a) {
    const double m = 2.0 * a;
    return m >= 1.0 && m <= (double)kGammaLadderMax && m == floor(m);
}

static __device__ double gamma_q_ladder(double a, double x) {
    // a <= 80 and x > 1e4: Q < x^a e^-x < e^(737 - 10000), below the least subnormal
    // (and the terms x^j / j! would overflow further out)
    if (x > 1.0e4) return 0.0;
    const int m = (int)(2.0 * a);
    double S, th;
    int s;
    if (m & 1) {
        double sx;
        S = erfcx_of_sqrt(x, sx);
        th = sx * 1.1283791670955125739;     // x^(1/2) / Gamma(3/2)
        s = 3;
    } else {
        S = 0.0;
        th = 1.0;
        s = 2;
    }
    for (; s <= m; s += 2) {
        S += th;
        th *= x * kInvHalf[s];
    }
    if (x <= 700.0) return exp(-x) * S;
    const double e = log(S) - x;
    return e < -746.0 ? 0.0 : exp(e);
}

// two-sided p of Student t with df degrees of freedom
__device__ __forceinline__ double t_two_sided(double t, double df, const double *bgrat = nullptr,
                                              LargeATab lat = LargeATab{nullptr, 0, 0}) {
    if (isnan(t) || !(df > 0.0)) return nan("");
    if (isinf(t)) return 0.0;
    const double t2 = t * t;
    return ibeta(0.5 * df, 0.5, df / (df + t2), t2 / (df + t2), bgrat, lat);
}

// p of a correlation coefficient with n observations: I_{1-r^2}((n-2)/2, 1/2)
__device__ __forceinline__ double corr_p(double r, double n, const double *bgrat = nullptr,
                                         LargeATab lat = LargeATab{nullptr, 0, 0}) {
    if (isnan(r) || n <= 2.0) return nan("");
    if (fabs(r) >= 1.0) return 0.0;
    return ibeta(0.5 * (n - 2.0), 0.5, (1.0 - r) * (1.0 + r), r * r, bgrat, lat);
}

// survival function of F(d1, d2)
__device__ __forceinline__ double f_sf(double F, double d1, double d2, const double *bgrat = nullptr,
                                       LargeATab lat = LargeATab{nullptr, 0, 0}) {
    if (isnan(F) || !(d1 > 0.0) || !(d2 > 0.0)) return nan("");
    if (isinf(F)) return 0.0;
    if (F <= 0.0) return 1.0;
    const double den = d2 + d1 * F;
    return ibeta(0.5 * d2, 0.5 * d1, d2 / den, d1 * F / den, bgrat, lat);
}

__device__ __forceinline__ double chi2_sf(double x, double df) {
    if (isnan(x) || !(df > 0.0)) return nan("");
    const double a = 0.5 * df, hx = 0.5 * x;
    if (hx > 0.0 && !isinf(hx) && gamma_ladder_applies(a)) return gamma_q_ladder(a, hx);
    return gamma_q(a, hx);
}

__device__ __forceinline__ double norm_sf(double z) { return 0.5 * erfc(z * 0.70710678118654752440); }

}  // namespace sf
}  // namespace napg
