"""The finalize kernels place each p-value job (its branch key and the test
that its p-value certainly underflows) in FP32 arithmetic. A job that the FP32
test resolves to p = 0 at once must have a p-value that FP64 cannot tell from
0 either: these tests redo the FP32 test in numpy float32 (both with and without
the fused multiply-add the compiler may form) on grids that straddle its
thresholds, and check every job it zeroes against the oracle's p-function
(Sec. 3.5.2 for r, Sec. 3.5.5 for F)."""
import numpy as np

from oracle import oracle as O

f32 = np.float32


def corr_zeroed(r, n, fused):
    """The correlation job's FP32 certain-underflow test, b = 1/2."""
    rf, nf = f32(r), f32(n)
    a = f32(f32(0.5) * nf - f32(1.0)) if not fused else f32(0.5 * np.float64(nf) - 1.0)
    y = f32(rf * rf)
    t = f32(f32(a - f32(0.25)) * y)
    ay = f32(a * y)
    return (a >= 20.0) & (((y <= 0.5) & (t >= f32(746.5))) | (ay >= f32(2001.0)))


def f_zeroed(F, d1, d2):
    """The F job's FP32 certain-underflow test (the denominator within FP32's range)."""
    v = d2 + d1 * F
    inv = f32(1.0) / f32(v)
    a, b = f32(0.5) * f32(d2), f32(0.5) * f32(d1)
    y = f32(f32(d1 * F) * inv)
    half = (b == f32(0.5)) & (y <= 0.5) & (f32(f32(a - f32(0.25)) * y) >= f32(746.5))
    return (a >= 20.0) & (b <= 32.0) & (half | (f32(a * y) >= f32(2001.0)))


def test_correlation_jobs_zeroed_only_where_p_underflows():
    rng = np.random.default_rng(5)
    checked = 0
    for n in (42.0, 43.0, 100.0, 1000.0, 30_011.0, 50_000.0, 1_000_003.0):
        a = 0.5 * (n - 2.0)
        # |r| around the two thresholds, (a - 1/4) r^2 = 746.5 and a r^2 = 2001
        r0 = [np.sqrt(746.5 / (a - 0.25)), np.sqrt(2001.0 / a)]
        rs = [min(0.999999, x * (1.0 + e)) for x in r0 for e in np.linspace(-1e-3, 1e-3, 41)]
        rs += list(rng.uniform(0.0, 1.0, 200))
        rs = np.array([x for x in rs if 0.0 <= x < 1.0])
        for fused in (False, True):
            z = corr_zeroed(rs, n, fused)
            if z.any():
                p = O.corr_p(rs[z], np.full(z.sum(), n))
                assert (p < 1e-300).all(), (n, rs[z][p >= 1e-300][:3], p[p >= 1e-300][:3])
                checked += int(z.sum())
    assert checked > 100


def test_f_jobs_zeroed_only_where_p_underflows():
    rng = np.random.default_rng(6)
    checked = 0
    for d1 in (1.0, 2.0, 3.0, 5.0, 9.0):
        for d2 in (40.0, 41.0, 1000.0, 49_990.0):
            a, b = 0.5 * d2, 0.5 * d1
            # F around a y = 2001 (and (a - 1/4) y = 746.5 for b = 1/2), y = d1 F / (d2 + d1 F)
            ys = [2001.0 / a] + ([746.5 / (a - 0.25)] if b == 0.5 else [])
            Fs = []
            for y0 in ys:
                if y0 < 1.0:
                    F0 = y0 * d2 / (d1 * (1.0 - y0))
                    Fs += [F0 * (1.0 + e) for e in np.linspace(-1e-3, 1e-3, 41)]
            Fs += list(np.exp(rng.uniform(-3.0, 12.0, 200)))
            Fs = np.array([F for F in Fs if 1e-30 <= d2 + d1 * F <= 1e30])
            z = f_zeroed(Fs, d1, d2)
            if z.any():
                p = O.f_sf(Fs[z], np.full(z.sum(), d1), np.full(z.sum(), d2))
                assert (p < 1e-300).all(), (d1, d2, Fs[z][p >= 1e-300][:3], p[p >= 1e-300][:3])
                checked += int(z.sum())
    assert checked > 100
