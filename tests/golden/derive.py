"""Writes the hand-derived golden cases in this folder.

The paper (NApy, arXiv 2505.00448) prints no worked example, so each case here
is a tiny input whose statistic and p-value follow in closed form from the
test's textbook definition; the derivation is stored beside the numbers. Only
the `math` module is used: no value comes from the oracle or from the GPU path.

Run: python tests/golden/derive.py
"""
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
N = None  # missing entry (NaN)


def t3_two_sided(ratio):
    """Two-sided p of Student t with 3 df, given t/sqrt(3) = ratio:
    F(t) = 1/2 + (1/pi) [ (t/sqrt3) / (1 + t^2/3) + atan(t/sqrt3) ]."""
    return 1.0 - (2.0 / math.pi) * (ratio / (1.0 + ratio * ratio) + math.atan(ratio))


cases = {
    "pearson_deletion_5pairs": {
        "cite": "Sec. 3.2 (pairwise deletion), Sec. 3.5.2 (Pearson, Beta-CDF p)",
        "derivation": "co-observed pairs (1,2),(2,1),(3,4),(4,3),(5,5): means 3,3; "
                      "sum dx*dy = 8, sum dx^2 = sum dy^2 = 10, r = 0.8; t/sqrt(3) = r/sqrt(1-r^2) = 4/3; "
                      "p = 1 - (2/pi)(12/25 + atan(4/3))",
        "test": "pearson", "vtype": [0, 0], "nlev": [0, 0],
        "X": [[1, 2, N, 3, 4, 5, 8], [2, 1, 6, 4, 3, 5, N]],
        "vars_a": [0, 1], "pair": [0, 1], "n": 5,
        "stat": 0.8, "p": t3_two_sided(4.0 / 3.0), "rtol": 1e-13,
    },
    "spearman_tie_average": {
        "cite": "Sec. 3.5.3 (Spearman, tie-averaged ranks, t-distribution p)",
        "derivation": "ranks x = 1..5, ranks y = 1,2,3.5,5,3.5; dx.dy = 8, dx^2 = 10, dy^2 = 9.5; "
                      "rho = 8/sqrt(95); rho/sqrt(1-rho^2) = 8/sqrt(31)",
        "test": "spearman", "vtype": [0, 0], "nlev": [0, 0],
        "X": [[1, 2, 3, 4, 5, N], [5, 6, 7, 8, 7, 1]],
        "vars_a": [0, 1], "pair": [0, 1], "n": 5,
        "stat": 8.0 / math.sqrt(95.0), "p": t3_two_sided(8.0 / math.sqrt(31.0)), "rtol": 1e-13,
    },
    "chi2_2x3": {
        "cite": "Sec. 3.5.4 (chi-squared test, chi2 survival function)",
        "derivation": "O = [[10,20,30],[20,20,20]], rows 60,60, cols 30,40,50, n = 120; "
                      "E = [[15,20,25],[15,20,25]]; chi2 = 2(25/15 + 25/25) = 16/3, df = 2, p = exp(-8/3)",
        "test": "chi2", "vtype": [1, 1], "nlev": [2, 3],
        "X": [[0] * 60 + [1] * 60,
              [0] * 10 + [1] * 20 + [2] * 30 + [0] * 20 + [1] * 20 + [2] * 20],
        "vars_a": [0, 1], "pair": [0, 1], "n": 120,
        "stat": 16.0 / 3.0, "p": math.exp(-8.0 / 3.0), "rtol": 1e-13,
    },
    "anova_3_groups": {
        "cite": "Sec. 3.5.7 (one-way ANOVA, F survival function)",
        "derivation": "groups {1,2,3},{4,5,6},{7,8,9}: grand mean 5, SSB = 3(9+0+9) = 54, SSW = 6; "
                      "F = (54/2)/(6/6) = 27; F(2,6) sf = (6/(6+2*27))^3 = 1e-3",
        "test": "anova", "vtype": [1, 0], "nlev": [3, 0],
        "X": [[0, 0, 0, 1, 1, 1, 2, 2, 2, 1], [1, 2, 3, 4, 5, 6, 7, 8, 9, N]],
        "vars_a": [0], "vars_b": [1], "pair": [0, 0], "n": 9,
        "stat": 27.0, "p": 1e-3, "rtol": 1e-12,
    },
    "welch_t": {
        "cite": "Sec. 3.5.5 (Welch t)",
        "derivation": "groups {1,2,3,4} (mean 2.5, var 5/3) and {2,4,6,8,10} (mean 6, var 10); "
                      "se^2 = 5/12 + 2 = 29/12; t = -3.5/sqrt(29/12)",
        "test": "ttest", "vtype": [1, 0], "nlev": [2, 0],
        "X": [[0, 0, 0, 0, 1, 1, 1, 1, 1], [1, 2, 3, 4, 2, 4, 6, 8, 10]],
        "vars_a": [0], "vars_b": [1], "pair": [0, 0], "n": 9,
        "stat": -3.5 / math.sqrt(29.0 / 12.0), "p": None, "rtol": 1e-14,
    },
    "kruskal_no_ties": {
        "cite": "Sec. 3.5.8 (Kruskal-Wallis H, chi2(k-1) survival function)",
        "derivation": "groups {1,2,3},{4,5,6}: rank sums 6, 15, n = 6; "
                      "H = 12/42 (36/3 + 225/3) - 21 = 27/7; df 1: p = erfc(sqrt(27/14))",
        "test": "kruskal", "vtype": [1, 0], "nlev": [2, 0],
        "X": [[0, 0, 0, 1, 1, 1], [1, 2, 3, 4, 5, 6]],
        "vars_a": [0], "vars_b": [1], "pair": [0, 0], "n": 6,
        "stat": 27.0 / 7.0, "p": math.erfc(math.sqrt(27.0 / 14.0)), "rtol": 1e-13,
    },
    "mwu_exact_extreme": {
        "cite": "Sec. 3.5.6 (Mann-Whitney U, exact mode for small groups without ties)",
        "derivation": "groups {1,2,3} vs {4,5,6}: U0 = 6 - 3*4/2 = 0, max(U0,U1) = 9; "
                      "P(U >= 9) = 1/C(6,3) = 1/20; p = 2/20",
        "test": "mwu", "vtype": [1, 0], "nlev": [2, 0],
        "X": [[0, 0, 0, 1, 1, 1], [1, 2, 3, 4, 5, 6]],
        "vars_a": [0], "vars_b": [1], "pair": [0, 0], "n": 6,
        "stat": 0.0, "p": 0.1, "rtol": 1e-14,
    },
}

if __name__ == "__main__":
    for name, case in cases.items():
        with open(os.path.join(HERE, name + ".json"), "w") as fh:
            json.dump(case, fh, indent=1)
    print(f"wrote {len(cases)} cases")
