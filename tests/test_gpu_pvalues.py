"""The device p-value functions (Sec. 3.5: Beta CDF for r and t, F, chi-squared and
normal survival functions) against the oracle's, on a grid that reaches every
branch: the incomplete beta continued fraction in both orientations, the
large-parameter expansion, the incomplete gamma series and fraction, and the
parameter ranges of the workloads (n up to 10^6, 1 to 64 levels)."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

P_REL = 1e-12
TINY = 1e-300


@pytest.fixture(scope="module")
def ctx():
    from paper_2505_00448_gb300 import napg
    c = napg.Context()
    yield c
    c.close()


def _check(got, want, label):
    got = np.asarray(got)
    want = np.asarray(want)
    nan_w = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan_w), f"{label}: NaN pattern differs"
    g, w = got[~nan_w], want[~nan_w]
    both_tiny = (np.abs(g) < TINY) & (np.abs(w) < TINY)
    rel = np.abs(g - w) / np.maximum(np.abs(w), TINY)
    rel[both_tiny] = 0.0
    k = int(np.argmax(rel))
    assert rel[k] <= P_REL, f"{label}: rel err {rel[k]:.3e} (gpu {g[k]!r}, oracle {w[k]!r}) at flat index {k}"


def _grid(*axes):
    m = np.meshgrid(*axes, indexing="ij")
    return [x.ravel() for x in m]


def test_corr_p(ctx):
    n = np.array([3, 4, 5, 10, 30, 41, 42, 43, 100, 1000, 9999, 25000, 50000, 1_000_000], float)
    r = np.concatenate([[0.0, 1e-9, 1e-6, 1e-4, 0.003, 0.011, 0.05, 0.2, 0.5, 0.7071, 0.75, 0.9, 0.99,
                         0.999999, 1.0], -np.array([1e-5, 0.1, 0.6, 0.95])])
    rr, nn = _grid(r, n)
    _check(ctx.debug_pvalues("corr", rr, nn), O.corr_p(rr, nn), "corr_p")


def test_t_two_sided(ctx):
    df = np.array([1, 2, 3, 5.5, 19.9, 39, 40, 41, 80, 1000.3, 24998, 99997.25, 1e6])
    t = np.concatenate([[0.0], np.logspace(-8, 2.5, 40), -np.logspace(-3, 1, 5), [np.inf, -np.inf]])
    tt, dd = _grid(t, df)
    _check(ctx.debug_pvalues("t", tt, dd), O.t_p2(tt, dd), "t_two_sided")


def test_f_sf(ctx):
    d1 = np.array([1, 2, 3, 4, 5, 6, 7, 8, 9, 20, 63, 64, 65, 100], float)
    d2 = np.array([1, 2, 5, 39, 40, 41, 100, 1000, 24990, 99990], float)
    F = np.concatenate([[0.0], np.logspace(-5, 3.5, 30), [np.inf]])
    ff, aa, bb = _grid(F, d1, d2)
    _check(ctx.debug_pvalues("f", ff, aa, bb), O.f_sf(ff, aa, bb), "f_sf")


def test_chi2_sf(ctx):
    df = np.concatenate([np.arange(1, 82), [99, 200, 1000, 4000]]).astype(float)
    rows = []
    for d in df:
        rows.append(np.concatenate([[0.0], d * np.logspace(-3, 1.2, 25), d + np.sqrt(2 * d) * np.linspace(-3, 3, 7)]))
    x = np.concatenate(rows)
    dd = np.repeat(df, [len(r) for r in rows])
    x = np.maximum(x, 0.0)
    _check(ctx.debug_pvalues("chi2", x, dd), O.chi2_sf(x, dd), "chi2_sf")


def test_chi2_sf_far_tail(ctx):
    """The finite sums for integer and half-integer df / 2 out to the log-form
    branch (x / 2 > 700), the underflow to subnormals and zero, and the cut-off
    past x / 2 = 10^4; df 161 and 4000 take the series / fraction instead."""
    df = np.array([1, 2, 3, 4, 9, 10, 41, 80, 81, 159, 160, 161, 4000], float)
    hx = np.array([1e-300, 1e-12, 0.3, 599.0, 699.9, 700.1, 712.0, 730.0, 740.0, 745.0, 748.0, 752.0, 760.0, 800.0,
                   900.0, 2000.0, 9999.0, 10001.0, 1e5])
    xx, dd = _grid(2.0 * hx, df)
    _check(ctx.debug_pvalues("chi2", xx, dd), O.chi2_sf(xx, dd), "chi2_sf far tail")


def test_erfcx_of_sqrt_against_cuda(ctx):
    """The library's own erfcx (fitted polynomials, used by the p-value
    expansions for half-integer b and the chi-squared finite sums) against CUDA's
    erfcx on the same arguments: across every piece of 0 <= z < 4 and its
    boundaries, both large-argument polynomials (1/64 <= 1/z^2 <= 1/16 and below)
    and far out. The fit is within 3.2e-16 of the function; CUDA's own error adds
    a few units in the last place."""
    edges = np.arange(0.0, 8.01, 0.5)
    z = np.concatenate([np.linspace(0.0, 4.0, 4001), np.linspace(4.0, 30.0, 5201), np.geomspace(30.0, 1e4, 2001),
                        (edges[:, None] + np.array([-1e-9, 0.0, 1e-9])).ravel()])
    z = z[z >= 0.0]
    u = z * z
    mine = ctx.debug_pvalues("erfcx_sqrt", u)
    cuda = ctx.debug_pvalues("erfcx_sqrt_cuda", u)
    rel = np.abs(mine - cuda) / cuda
    k = int(np.argmax(rel))
    assert rel[k] <= 1.5e-15, f"erfcx(sqrt u): rel diff {rel[k]:.3e} at u = {u[k]!r}"


def test_norm_sf(ctx):
    z = np.concatenate([np.linspace(-40, 40, 801), [np.inf, -np.inf]])
    _check(ctx.debug_pvalues("norm", z), O.norm_sf(z), "norm_sf")


def test_ibeta_branches(ctx):
    """I_x(a,b) over both continued-fraction orientations and the large-a expansion,
    including its edges (a = 20, b = 32, x = 1/2) and non-half-integer b."""
    a = np.array([0.5, 1, 2.5, 10, 19.99, 20, 20.5, 33, 100.25, 1e3, 12499, 1e5, 1e6])
    b = np.array([0.5, 1, 1.5, 2, 3.5, 4.5, 7.3, 10, 15.5, 31.5, 32, 32.5, 50])
    x = np.concatenate([[0.0, 1e-12, 1e-3, 0.1, 0.3, 0.4999999, 0.5, 0.5000001, 0.7, 0.9, 0.99],
                        1 - np.logspace(-12, -2.5, 12), [1.0]])
    xx, aa, bb = _grid(x, a, b)
    _check(ctx.debug_pvalues("ibeta", xx, aa, bb), O.ibeta(aa, bb, xx), "ibeta")


def test_gamma_q(ctx):
    a = np.array([0.5, 1, 1.5, 2, 4.5, 10, 40.5, 100, 2048])
    x = np.concatenate([[0.0], np.logspace(-6, 3.6, 40)])
    xx, aa = _grid(x, a)
    _check(ctx.debug_pvalues("gamma_q", xx, aa), O.gamma_q(aa, xx), "gamma_q")
