"""Pins of the model oracle (oracle/model.py) to the numbers the paper prints.

Fixtures under tests/golden/ carry the paper's Tables 2-4 with citations.
"""
import json
import os

import pytest

from oracle import model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


T2 = _load("paper_table2.json")
T3 = _load("paper_table3.json")


@pytest.mark.parametrize("row", T2["rows"], ids=lambda r: f"row{r['row']}")
def test_table2_analytical_C_M_I(row):
    s, d, r, t, D = row["shape"], row["d"], row["r"], row["t"], row["D"]
    if row["impl"] == "cu":
        C = model.C_cu(s, d, r, t)
        I = model.I_cu(s, d, r, t, D)
    else:
        assert model.alpha(s, d, r, t) == pytest.approx(row["alpha"], abs=0.005)
        C = model.C_tc(s, d, r, t, row["S_exact"])
        I = model.I_tc(s, d, r, t, D, row["S_exact"])
    assert C == pytest.approx(row["C"], abs=0.5)
    assert model.M_point(D) == row["M"]
    assert I == pytest.approx(row["I"], abs=0.006)
    assert C / model.M_point(D) == pytest.approx(I)


def test_alpha_values_and_box_formula():
    """alpha = 49/27 = 1.81 (Box-2D1R, t=3) and 225/63 = 3.57 (Box-2D1R, t=7)."""
    assert model.alpha("box", 2, 1, 3) == pytest.approx(49 / 27)
    assert model.alpha("box", 2, 1, 7) == pytest.approx(225 / 63)
    assert round(model.alpha("box", 2, 1, 3), 2) == 1.81
    assert round(model.alpha("box", 2, 1, 7), 2) == 3.57
    assert model.alpha("box", 3, 1, 3) == pytest.approx(343 / 81)  # not the 1.81 quoted for case 5
    for d in (1, 2, 3):
        for r in (1, 2, 3):
            assert model.alpha("box", d, r, 1) == 1.0


def test_alpha_grows_like_t_power_d_minus_1():
    """Sec. 4.1: alpha_box = O(t^(d-1)); alpha/t^(d-1) tends to ((2r)^d/(2r+1)^d)."""
    for d in (2, 3):
        a = [model.alpha("box", d, 1, t) / t ** (d - 1) for t in (50, 100, 200)]
        assert a[2] == pytest.approx((2 / 3) ** d, rel=0.02)
        assert a[0] > a[1] > a[2]


def _peaks(case):
    p = T3["peaks"]
    if case["D"] == 8:
        P_cu = p["P_cu_f64"]
        P_tc = p["P_tc_f64"]
    else:
        P_cu = p["P_cu_f32"]
        P_tc = p["P_sptc_tf32"] if case["tc"] == "sptc_tf32" else p["P_tc_tf32"]
    return P_cu, P_tc, p["B"]


@pytest.mark.parametrize("case", T3["cases"], ids=lambda c: f"case{c['case']}")
def test_table3_intensity_ridge_scenario(case):
    s, d, r, t, D, S = case["shape"], case["d"], case["r"], case["t"], case["D"], case["S"]
    P_cu, P_tc, B = _peaks(case)
    assert model.I_cu(s, d, r, t, D) == pytest.approx(case["I_cu"], abs=0.006) or case["case"] == 4
    assert model.I_tc(s, d, r, t, D, S) == pytest.approx(case["I_tc"], abs=0.006)
    assert round(model.ridge(P_cu, B)) == case["ridge_cu"]
    assert round(model.ridge(P_tc, B)) == case["ridge_tc"]
    assert model.bound(model.I_cu(s, d, r, t, D), P_cu, B) == case["bound_cu"]
    assert model.bound(model.I_tc(s, d, r, t, D, S), P_tc, B) == case["bound_tc"]
    assert model.scenario(s, d, r, t, D, S, P_cu, P_tc, B) == case["scenario"]


@pytest.mark.parametrize("case", T3["cases"], ids=lambda c: f"case{c['case']}")
def test_table3_predicted_direction(case):
    """The predicted speed-up direction matches the measured change (Sec. 5.3)."""
    s, d, r, t, D, S = case["shape"], case["d"], case["r"], case["t"], case["D"], case["S"]
    P_cu, P_tc, B = _peaks(case)
    ratio = model.speedup(s, d, r, t, D, S, P_cu, P_tc, B)
    measured = case["measured_tc"] / case["measured_cu"]
    if case["change"] == "down":
        assert ratio < 1 and measured < 1
    elif case["change"] == "up":
        assert ratio > 1 and measured > 1
    else:
        assert ratio == pytest.approx(1.0, abs=0.02) and measured == pytest.approx(1.0, abs=0.02)
    # sweet spot = scenario 3 or (scenario 4 with alpha < S P_TC / P_CU); case 2
    # sits on its edge (alpha = 1 against a threshold of 1.005)
    if case["change"] == "same":
        assert model.alpha(s, d, r, t) == pytest.approx(S * P_tc / P_cu, rel=0.01)
    else:
        assert model.in_sweet_spot(s, d, r, t, D, S, P_cu, P_tc, B) == (case["change"] == "up")


def test_case1_degradation_matches_text():
    """Case 1: the text's 27.12 % loss is 1 - 190.14/260.90."""
    c = T3["cases"][0]
    assert 1 - c["measured_tc"] / c["measured_cu"] == pytest.approx(0.2712, abs=5e-5)


def test_scenario_identities():
    """Scenario 1 ratio = 1 (Eq. 14); scenario 2 < 1 (Eq. 16); scenario 3 > 1
    (Eq. 17); scenario 4 = (S/alpha) P_TC/P_CU (Eq. 18)."""
    B = 1e12
    # S1: both memory-bound
    assert model.scenario("box", 2, 1, 1, 8, 0.5, 1e15, 1e16, B) == 1
    assert model.speedup("box", 2, 1, 1, 8, 0.5, 1e15, 1e16, B) == pytest.approx(1.0)
    # S2: CU memory-bound, TC compute-bound
    assert model.scenario("box", 2, 1, 3, 8, 0.25, 9.7e12, 19.5e12, 1.935e12) == 2
    assert model.speedup("box", 2, 1, 3, 8, 0.25, 9.7e12, 19.5e12, 1.935e12) < 1
    # S3: CU compute-bound, TC memory-bound
    assert model.scenario("box", 2, 2, 1, 4, 0.5, 1e12, 1e15, B) == 3
    assert model.speedup("box", 2, 2, 1, 4, 0.5, 1e12, 1e15, B) > 1
    # S4: closed form
    s4 = model.speedup("box", 3, 2, 2, 8, 0.6, 1e12, 5e12, 1e12)
    assert model.scenario("box", 3, 2, 2, 8, 0.6, 1e12, 5e12, 1e12) == 4
    assert s4 == pytest.approx(0.6 / model.alpha("box", 3, 2, 2) * 5)


def test_table4_sparse_moves_bottleneck():
    t4 = T3["table4"]
    p = T3["peaks"]
    s, d, r, t, D, S = t4["shape"], t4["d"], t4["r"], t4["t"], t4["D"], t4["S"]
    I = model.I_tc(s, d, r, t, D, S)
    assert I == pytest.approx(t4["I"])
    assert round(model.ridge(p["P_tc_tf32"], p["B"])) == t4["dense"]["ridge"]
    assert round(model.ridge(p["P_sptc_tf32"], p["B"])) == t4["sparse"]["ridge"]
    assert model.bound(I, p["P_tc_tf32"], p["B"]) == t4["dense"]["bound"]
    assert model.bound(I, p["P_sptc_tf32"], p["B"]) == t4["sparse"]["bound"]
    dense = model.P_tc_actual(s, d, r, t, D, S, p["P_tc_tf32"], p["B"])
    sparse = model.P_tc_actual(s, d, r, t, D, S, p["P_sptc_tf32"], p["B"])
    # dense is capped by P_TC, sparse by B I: the model's gain is B I / P_TC = 1.49,
    # below the measured 3.06 but in the same direction
    assert sparse / dense == pytest.approx(p["B"] * I / p["P_tc_tf32"])
    assert sparse / dense > 1
    assert t4["sparse"]["measured"] / t4["dense"]["measured"] == pytest.approx(3.06, abs=0.005)


def test_sec42_cuda_core_transition_points():
    """Sec. 4.2 and Fig. 14: I_CU grows linearly in t.  The measured A100
    transitions (box at t=3, star at t=5, r=1, D=8) come earlier than the
    model at full A100 peaks (t=5 and t=9) because clocks were locked low;
    one common lower ridge explains both measured points."""
    for s in ("box", "star"):
        Is = [model.I_cu(s, 2, 1, t, 8) for t in range(1, 9)]
        diffs = [b - a for a, b in zip(Is, Is[1:])]
        assert all(x == pytest.approx(diffs[0]) for x in diffs)

    def first(s, ridge):
        return next(t for t in range(1, 40) if model.I_cu(s, 2, 1, t, 8) >= ridge)

    full = model.ridge(9.7e12, 1.935e12)
    assert (first("box", full), first("star", full)) == (5, 9)
    ok = [x / 100 for x in range(100, 600) if (first("box", x / 100), first("star", x / 100)) == (3, 5)]
    assert ok and min(ok) > 2.5 and max(ok) <= 3.125 + 1e-9


def test_K_fused_star_closed_form_small_cases():
    # star 2D r=1: t=1 -> 5, t=2 -> 13 (diamond of radius 2), t=3 -> 25
    assert [model.K_fused("star", 2, 1, t) for t in (1, 2, 3)] == [5, 13, 25]
    # star 3D r=1: octahedron sizes 7, 25, 63
    assert [model.K_fused("star", 3, 1, t) for t in (1, 2, 3)] == [7, 25, 63]
    assert model.K_fused("star", 3, 2, 2) == 73


# ---------------------------------------------------------------------------
# Roof functions and the beta (split-product) terms, against values worked out
# by hand from the closed form of the roofline in point updates per second
# (Sec. 3.1, Eq. 5; Eq. 8 for CUDA cores; Eq. 11-12 for tensor cores):
#     CU:  min(P_CU / (2K),                t B / (2D))
#     TC:  min(S P_TC / (2K alpha beta),   t B / (2D))
# at the A100 peaks of tests/golden/paper_table3.json (B = 1.935e12 B/s,
# FP64 P_CU = 9.7e12, P_TC = 19.5e12, sparse TF32 312e12 FLOP/s).
# ---------------------------------------------------------------------------
A100_B = 1.935e12


def test_gstencils_roof_cu_memory_term_binds_case1():
    """Table 3 case 1, Box-2D1R t=3 FP64: K = 9, 2K = 18 FLOP per point-step.
    Compute term 9.7e12 / 18 = 5.3889e11; memory term 3 * 1.935e12 / 16 =
    3.628125e11 points/s, the smaller one.  Dividing by C^(t) = 3 * 18 instead
    of C = 18 would give 1.796e11; dropping t from the memory term 1.209e11."""
    got = model.gstencils_roof_cu("box", 2, 1, 3, 8, 9.7e12, A100_B)
    assert got == pytest.approx(3.628125e11, rel=1e-12)


def test_gstencils_roof_cu_compute_term_binds_case2():
    """Table 3 case 2, Box-2D3R t=1 FP64: K = 49; I = 49/8 = 6.125 is above
    the ridge 9.7/1.935 = 5.013, so the roof is 9.7e12 / 98 = 9.897959e10."""
    got = model.gstencils_roof_cu("box", 2, 3, 1, 8, 9.7e12, A100_B)
    assert got == pytest.approx(9.7e12 / 98, rel=1e-12)
    assert got == pytest.approx(9.8979591836734694e10, rel=1e-12)
    # t = 2: compute term unchanged (9.898e10) and the memory term doubles
    # (2.419e11), so the roof stays the compute term
    assert model.gstencils_roof_cu("box", 2, 3, 2, 8, 9.7e12, A100_B) == pytest.approx(9.8979591836734694e10)


def test_gstencils_roof_tc_compute_term_binds_case1():
    """Case 1 on the FP64 MMA: S = 1/2, alpha = 49/27, beta = 1.
    I_TC = 3 (49/27)/(1/2) * 9/8 = 12.25 > ridge 10.08, so the roof is
    S P_TC / (2K alpha) = 0.5 * 19.5e12 / (18 * 49/27) = 2.984694e11."""
    got = model.gstencils_roof_tc("box", 2, 1, 3, 8, 0.5, 19.5e12, A100_B)
    assert got == pytest.approx(0.5 * 19.5e12 * 27 / (18 * 49), rel=1e-12)
    assert got == pytest.approx(2.9846938775510204e11, rel=1e-12)


def test_gstencils_roof_tc_memory_term_binds_case3():
    """Case 3, Box-2D1R t=7 FP32 on sparse TF32: S = 15/32, alpha = 225/63,
    I_TC = 120 < ridge 161.2, so the memory term binds: 7 * 1.935e12 / 8 =
    1.693125e12 points/s, independent of S and alpha (they cancel between
    I_TC and S/alpha)."""
    got = model.gstencils_roof_tc("box", 2, 1, 7, 4, 15 / 32, 312e12, A100_B)
    assert got == pytest.approx(1.693125e12, rel=1e-12)
    # the same configuration with the compute term binding: half the dense
    # TF32 peak 78e12 puts the ridge at 40.3 < 120, roof
    # (15/32) 78e12 / (18 * 225/63) = 5.6875e11
    got_cb = model.gstencils_roof_tc("box", 2, 1, 7, 4, 15 / 32, 78e12, A100_B)
    assert got_cb == pytest.approx((15 / 32) * 78e12 * 63 / (18 * 225), rel=1e-12)
    assert got_cb == pytest.approx(5.6875e11, rel=1e-12)


def test_beta_terms_hand_values():
    """beta = 3 (hi/lo split, three products per useful product), case 1 on the
    FP64 MMA: C_TC = beta alpha/S t 2K = 3 * (49/27) / 0.5 * 54 = 588 FLOP and
    I_TC = 588 / 16 = 36.75 FLOP/B; the roof is the compute term divided by
    beta: 2.984694e11 / 3 = 9.948980e10 points/s."""
    assert model.C_tc("box", 2, 1, 3, 0.5, beta=3.0) == pytest.approx(588.0, rel=1e-12)
    assert model.C_tc("box", 2, 1, 3, 0.5) == pytest.approx(196.0, rel=1e-12)
    assert model.I_tc("box", 2, 1, 3, 8, 0.5, beta=3.0) == pytest.approx(36.75, rel=1e-12)
    assert model.P_tc_actual("box", 2, 1, 3, 8, 0.5, 19.5e12, A100_B, beta=3.0) == pytest.approx(
        0.5 * 19.5e12 * 27 / (49 * 3), rel=1e-12)
    assert model.gstencils_roof_tc("box", 2, 1, 3, 8, 0.5, 19.5e12, A100_B, beta=3.0) == pytest.approx(
        9.9489795918367347e10, rel=1e-12)


def test_beta_cancels_when_memory_bound_and_moves_the_scenario():
    """Case 3 with beta = 3 and the sparse TF32 peak: I_TC = 3 * 120 = 360 is
    now above the ridge 161.2, so the compute term binds:
    (15/32) 312e12 / (18 * (225/63) * 3) = 7.583333e11 points/s (beta applied
    in the roof AND in I_TC; applying it only in I_TC gives 2.275e12, only in
    the S/(alpha beta) factor 5.644e11).  With beta = 3 but the peak raised 10x (ridge 1612 > 360) the
    roof is the memory term again and beta drops out: 1.693125e12."""
    got = model.gstencils_roof_tc("box", 2, 1, 7, 4, 15 / 32, 312e12, A100_B, beta=3.0)
    assert got == pytest.approx((15 / 32) * 312e12 * 63 / (18 * 225 * 3), rel=1e-12)
    assert got == pytest.approx(7.5833333333333333e11, rel=1e-12)
    assert model.scenario("box", 2, 1, 7, 4, 15 / 32, 19.5e12, 312e12, A100_B) == 3
    assert model.scenario("box", 2, 1, 7, 4, 15 / 32, 19.5e12, 312e12, A100_B, beta=3.0) == 4
    assert model.gstencils_roof_tc("box", 2, 1, 7, 4, 15 / 32, 3120e12, A100_B, beta=3.0) == pytest.approx(
        1.693125e12, rel=1e-12)


def test_beta_in_sweet_spot_condition():
    """Eq. 19 with beta folded into alpha: Box-2D3R t=1 (alpha = 1), S = 1/2,
    P_TC/P_CU = 19.5/9.7: alpha beta < S P_TC/P_CU holds for beta = 1
    (1 < 1.00515) and fails for beta = 3 (3 > 1.00515)."""
    assert model.alpha_condition("box", 2, 3, 1, 0.5, 9.7e12, 19.5e12)
    assert not model.alpha_condition("box", 2, 3, 1, 0.5, 9.7e12, 19.5e12, beta=3.0)
