"""Checks of the paper's printed worked example (Sec. IV) and complexity tables (Tables I-III).

These pin readings of the paper that the oracle and the library rely on: the band-index rule of
eq. (k_var) (k1 = b_N - Delta_N/2 + 1, L_V = Delta_N - 1, M = N - L + 1) and the garbled adder count
C_a,F of Sec. III-D, read as (3/2) N log2 N - (5/2) N + 4.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2406_14116_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_example.json")))


def test_example_geometry():
    d = GOLD["design"]
    N, L, M, DN = d["N"], d["L"], d["M"], d["Delta_N"]
    assert M == N - L + 1                       # Sec. II: L = N - M + 1
    assert d["L_V"] == DN - 1                   # Sec. III-B: L_V = Delta_N - 1
    assert DN == round(GOLD["spec"]["Delta_over_pi"] * N / 2)   # Delta = Delta_N * 2 pi / N
    lo, hi = d["b_N"]
    assert lo == math.ceil(GOLD["spec"]["b_over_pi"][0] * N / 2)
    assert hi == math.floor(GOLD["spec"]["b_over_pi"][1] * N / 2)
    # every b_N of the example gives a k1 the oracle accepts, and the range ends exactly at the
    # paper's upper bound b_N <= N/2 - Delta_N/2 - 1
    V = np.linspace(0.95, 0.05, d["L_V"])
    for bN in range(lo, hi + 1):
        k1 = bN - DN // 2 + 1
        hr = oracle.HR(N, V, k1)
        assert hr[k1 - 1] == 1.0 and hr[k1 + d["L_V"]] == 0.0
    assert hi - DN // 2 + 1 == wl.max_band(N, d["L_V"])
    with pytest.raises(ValueError):
        oracle.HR(N, V, hi - DN // 2 + 2)


def table1_rates(N, L, LV, c2_shortcut=True):
    """Table I with Sec. III-D's counts; with (L-1)/N = 1/4 (c = 2) the fixed exponent multiply
    costs 2 mults + 2 adds on odd k only, over the N/2 conjugate-symmetric bins."""
    lg = math.log2(N)
    C_mf_F = 0.5 * N * lg - 1.5 * N + 2
    C_a_F = 1.5 * N * lg - 2.5 * N + 4
    C_mf_H = N / 2 if c2_shortcut else 1.5 * N
    C_a_H = N / 2 if c2_shortcut else 1.5 * N
    R = N - L + 1
    return (2 * C_mf_F + C_mf_H) / R, 2 * LV / R, (2 * C_a_F + C_a_H) / R


def test_table1_general_form_matches_printed_expressions():
    for N, L, LV in ((128, 33, 15), (1024, 257, 12)):
        rmf, rmv, ra = table1_rates(N, L, LV, c2_shortcut=False)
        lg = math.log2(N)
        assert rmf == pytest.approx((N * lg - 1.5 * N + 4) / (N - L + 1))
        assert ra == pytest.approx((3 * N * lg - 3.5 * N + 8) / (N - L + 1))
        assert rmv == pytest.approx(2 * LV / (N - L + 1))


def test_table2_proposed_row_and_savings():
    t = GOLD["table2"]
    p = t["FD/FD (prop.)"]
    rmf, rmv, ra = table1_rates(p["N"], p["L"], GOLD["design"]["L_V"])
    assert round(rmf, 1) == p["R_mf"] and round(rmv, 1) == p["R_mv"] and round(ra, 1) == p["R_a"]
    f = t["TD/TD"]
    sav = [100 * (1 - a / b) for a, b in ((rmf, f["R_mf"]), (rmv, f["R_mv"]), (ra, f["R_a"]))]
    assert [round(s, 1) for s in sav] == t["saving_vs_TD/TD_percent"]
    # the TD/FD rates are printed rounded to one decimal, so its savings agree to ~1 point
    g = t["TD/FD"]
    sav2 = [100 * (1 - a / b) for a, b in ((rmf, g["R_mf"]), (rmv, g["R_mv"]), (ra, g["R_a"]))]
    for s, want in zip(sav2, t["saving_vs_TD/FD_percent"]):
        assert abs(s - want) < 2.0


def test_table3_design_cost_is_the_table_size():
    """A bandwidth change costs no arithmetic; the stored state is the L_V transition samples."""
    assert GOLD["table3_prop"] == {"R_md": 0, "R_ad": 0, "Mem": GOLD["design"]["L_V"]}
