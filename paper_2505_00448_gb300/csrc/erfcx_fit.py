"""Coefficients of the library's own erfcx(z) = exp(z^2) erfc(z), z >= 0, for
the p-value expansion (specfun.cuh, erfcx_fast): near-minimax polynomials fitted
in 40-digit arithmetic (mpmath's Chebyshev fit) to the function defined by
mpmath's erfc, then rounded to doubles.

* 0 <= z < 4: eight pieces of width 1/2, each a polynomial in t = z - z_c (the
  piece's midpoint, |t| <= 1/4).
* z >= 4: g(w) = sqrt(pi) z erfcx(z) as a polynomial in w = 1/z^2, on
  [1/64, 1/16] (4 <= z <= 8) and on [0, 1/64] (z >= 8); g -> 1 as w -> 0 (the
  function's asymptotic series 1 - w/2 + 3 w^2/4 - ...), and it is smooth on the
  closed interval, so a polynomial of a few terms holds it to the last bit.

Run: python erfcx_fit.py > erfcx_coefs.inc (the file the CUDA source includes).
"""
import mpmath as mp

mp.mp.dps = 40
TOL = mp.mpf(2) ** -56          # fit error relative to the smallest value on the piece


def erfcx(z):
    return mp.exp(z * z) * mp.erfc(z)


def g(w):
    if w == 0:
        return mp.mpf(1)
    z = 1 / mp.sqrt(w)
    return mp.sqrt(mp.pi) * z * erfcx(z)


def fit(f, a, b, nmin=4, nmax=24):
    """Lowest degree whose Chebyshev fit on [a, b] keeps |error| below TOL * min|f|;
    coefficients in ascending powers of the argument."""
    fmin = min(abs(f(a)), abs(f(b)), abs(f((a + b) / 2)))
    for n in range(nmin, nmax + 1):
        poly, err = mp.chebyfit(f, [a, b], n, error=True)
        if err <= TOL * fmin:
            return list(reversed(poly)), err / fmin
    raise RuntimeError("no fit on [%s, %s]" % (a, b))


def emit(name, coefs):
    vals = ", ".join(repr(float(c)) for c in coefs)
    return "static __constant__ double %s[%d] = {%s};" % (name, len(coefs), vals)


def main():
    out = ["// generated by erfcx_fit.py (mpmath %s, %d digits): do not edit" % (mp.__version__, mp.mp.dps)]
    degs = []
    pieces = []
    for k in range(8):
        zc = mp.mpf(k) / 2 + mp.mpf(1) / 4
        c, rel = fit(lambda t, zc=zc: erfcx(zc + t), -mp.mpf(1) / 4, mp.mpf(1) / 4)
        pieces.append(c)
        degs.append(len(c))
    nmax = max(degs)
    # one table of 8 rows, padded with zeros to the longest piece (Horner from the top)
    rows = [c + [mp.mpf(0)] * (nmax - len(c)) for c in pieces]
    flat = [v for r in rows for v in r]
    out.append("constexpr int kErfcxPieceTerms = %d;   // terms per piece (0 <= z < 4), zero-padded" % nmax)
    out.append(emit("kErfcxPiece", flat))
    cm, rm = fit(g, mp.mpf(1) / 64, mp.mpf(1) / 16)
    cs, rs = fit(g, mp.mpf(0), mp.mpf(1) / 64)
    out.append("constexpr int kErfcxMidTerms = %d, kErfcxFarTerms = %d;" % (len(cm), len(cs)))
    out.append(emit("kErfcxMid", cm) + "   // g(w), 1/64 <= w <= 1/16")
    out.append(emit("kErfcxFar", cs) + "   // g(w), 0 <= w <= 1/64")
    print("\n".join(out))


if __name__ == "__main__":
    main()
