"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a copy of napg_oracle.c (a dropped term, a
wrong sign or index, a wrong degree of freedom, a transposed operand), builds it
on the CPU, and runs the pin tests against the copy: at least one pin must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "napg_oracle.c")
PINS = ["tests/test_oracle_special.py", "tests/test_oracle_stats.py", "tests/test_oracle_effects.py"]

MUTANTS = {
    "pearson_uncentred_y": ("double dv = v[k] - mv, dw = w[k] - mw;", "double dv = v[k] - mv, dw = w[k];"),
    "tie_rank_off_by_one": ("r2[buf[k].i] = 2 * a + t + 1;", "r2[buf[k].i] = 2 * a + t;"),
    "chi2_expected_wrong_n": ("double E = (double)row[g] * (double)col[h] / (double)n;",
                              "double E = (double)row[g] * (double)col[h] / (double)(n + 1);"),
    "anova_df_within": ("double d1 = (double)(k - 1), d2 = (double)(n - k);",
                        "double d1 = (double)(k - 1), d2 = (double)(n - k + 1);"),
    "welch_df_term": ("e1 * e1 / (double)(n1 - 1));", "e1 * e1 / (double)(n1));"),
    "mwu_continuity_sign": ("(c->mwu_cc ? 0.5 : 0.0)", "(c->mwu_cc ? -0.5 : 0.0)"),
    "kruskal_no_tie_correction": ("double C = 1.0 - (double)T / (nd * nd * nd - nd);", "double C = 1.0;"),
    "ibeta_even_term_sign": ("return m * (b - m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));",
                             "return m * (b + m) * x / ((a + 2.0 * m - 1.0) * (a + 2.0 * m));"),
    "gamma_cf_sign": ("-(double)(n - 1) * ((double)(n - 1) - a)", "(double)(n - 1) * ((double)(n - 1) - a)"),
    "deletion_one_sided": ("if (observed(c, va, s) && observed(c, vb, s)) {", "if (observed(c, va, s)) {"),
    "transposed_operand": ("y[n] = c->X[vb * c->S + s];", "y[n] = c->X[va * c->S + s];"),
    "context_ignored": ("if (c->ctx && !c->ctx[s]) return 0;", ""),
    "anova_uncentred": ("{ double d = w->y[q] - gm; dsum[(int)w->x[q]] += d; dgm += d; }",
                        "{ double d = w->y[q]; dsum[(int)w->x[q]] += d; dgm += d; }"),
    "cramer_v_max_levels": ("int m = (ka < kb ? ka : kb) - 1;", "int m = (ka > kb ? ka : kb) - 1;"),
    "cohen_d_welch_pooled": ("const double s2 = c->welch ? 0.5 * (v0 + v1) : (q0 + q1) / (double)(n0 + n1 - 2);",
                             "const double s2 = (q0 + q1) / (double)(n0 + n1 - 2);"),
    "mwu_r_uncorrected_ties": ("((n + 1.0) - (double)T / (n * (n - 1.0)));\n        if (var > 0.0) *e1",
                               "((n + 1.0));\n        if (var > 0.0) *e1"),
    "kruskal_eta_k_off_by_one": ("*e1 = (st - (double)k + 1.0) / (n - (double)k);",
                                 "*e1 = (st - (double)k) / (n - (double)k);"),
    "ttest_uncentred": ("double gm = (s0 + s1) / (double)n, d0 = 0.0, d1 = 0.0;",
                        "double gm = 0.0, d0 = 0.0, d1 = 0.0;"),
}


def _run_mutant(name, workdir):
    """Build the oracle with one planted mistake and run the pins against it;
    returns (pins' exit status, the end of their output)."""
    old, new = MUTANTS[name]
    src = open(SRC).read()
    if src.count(old) < 1:
        return None, f"mutation site for {name} not found"
    d = os.path.join(workdir, name)
    os.makedirs(d, exist_ok=True)
    csrc = os.path.join(d, "mutant.c")
    with open(csrc, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(d, "libmutant.so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                    "-o", so, csrc, "-lm"], check=True)
    env = dict(os.environ, NAPG_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    """Every mutant's pin run, several at a time (each is an independent process)."""
    from concurrent.futures import ThreadPoolExecutor
    workdir = str(tmp_path_factory.mktemp("mutants"))
    names = sorted(MUTANTS)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda n: _run_mutant(n, workdir), names))
    return dict(zip(names, results))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, mutant_results):
    rc, out = mutant_results[name]
    assert rc is not None, out
    assert rc != 0, f"no pin caught mutant {name}:\n{out}"
