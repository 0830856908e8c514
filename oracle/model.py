"""The paper's performance model, written out plainly in FP64 (Python floats).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The product has its
own C++ implementation of the same model (used as its dispatch rule); tests
compare the two and pin this one to the numbers the paper prints.

Notation follows the paper's nomenclature (Table 1): d, r, t, K, C, M, I, P,
the peaks P_hw and bandwidth B, the sparsity factor S and the fusion
redundancy factor alpha.

* K: box (2r+1)^d (Sec. 3.2.1).  The paper writes no star count; a star has
  one centre and r points on each side of each axis, 2dr+1.
* K^(t): number of points of the fused kernel.  Box: (2rt+1)^d (Eq. 10).  Star
  (not given by the paper): the t-fold sum of star offsets is the set of p
  with sum_i ceil(|p_i|/r) <= t, whose size is
  sum_j C(d,j) C(t,j) (2r)^j.
* C = 2K, M = 2D, I = K/D (Sec. 3.2.1).
* CUDA cores with temporal fusion: C^(t) = tC, M^(t) = M, I = tK/D,
  P = min(P_CU, B I) (Eq. 8).
* Tensor cores with kernel fusion: C_TC^(t) = (alpha/S) C^(t) (Eq. 3),
  alpha = K^(t)/(tK) (Eq. 9), I_TC = t (alpha/S) K/D,
  P_TC,actual = (S/alpha) min(P_TC, B I_TC) (Eq. 11-12).
* Speedup ratio and the four scenarios (Sec. 4.1, Eqs. 13-19); the sweet spot
  is scenario 3 plus the part of scenario 4 where alpha < S P_TC/P_CU.
* Sparse tensor cores: same intensity, peak P_SpTC (Sec. 4.3, Eq. 20).

One extension that is not in the paper: beta = products issued per useful
product (1 for a single-precision MMA, 3 for hi/lo split forms), which
multiplies the issued work like alpha/S does.
"""
from __future__ import annotations

from math import comb


def K_points(shape: str, d: int, r: int) -> int:
    if shape == "box":
        return (2 * r + 1) ** d
    if shape == "star":
        return 2 * d * r + 1
    raise ValueError(shape)


def K_fused(shape: str, d: int, r: int, t: int) -> int:
    """K^(t): points of the t-fold fused kernel."""
    if shape == "box":
        return (2 * r * t + 1) ** d
    if shape == "star":
        return sum(comb(d, j) * comb(t, j) * (2 * r) ** j for j in range(0, min(d, t) + 1))
    raise ValueError(shape)


def alpha(shape: str, d: int, r: int, t: int) -> float:
    """Fusion redundancy factor alpha = K^(t) / (t K)  (Eq. 9)."""
    return K_fused(shape, d, r, t) / (t * K_points(shape, d, r))


def C_point(shape, d, r) -> float:
    """Floating-point operations per point update, C = 2K."""
    return 2.0 * K_points(shape, d, r)


def M_point(D: int) -> float:
    """Bytes per point update, M = 2D (one read, one write)."""
    return 2.0 * D


def I_cu(shape, d, r, t, D) -> float:
    """CUDA-core intensity with temporal fusion, I = t K / D  (Eq. 8)."""
    return t * K_points(shape, d, r) / D


def C_cu(shape, d, r, t) -> float:
    return t * C_point(shape, d, r)


def C_tc(shape, d, r, t, S, beta=1.0) -> float:
    """Executed tensor-core operations per fused point update (Eq. 3), times beta."""
    return beta * alpha(shape, d, r, t) / S * C_cu(shape, d, r, t)


def I_tc(shape, d, r, t, D, S, beta=1.0) -> float:
    """Tensor-core intensity I_TC = t (alpha/S) K/D  (Eq. 11-12), times beta."""
    return beta * t * alpha(shape, d, r, t) / S * K_points(shape, d, r) / D


def roofline(P_peak: float, B: float, I: float) -> float:
    """P = min(P_peak, B I)  (Eq. 5)."""
    return min(P_peak, B * I)


def ridge(P_peak: float, B: float) -> float:
    """Ridge point I* = P_peak / B."""
    return P_peak / B


def P_cu_actual(shape, d, r, t, D, P_cu, B) -> float:
    return roofline(P_cu, B, I_cu(shape, d, r, t, D))


def P_tc_actual(shape, d, r, t, D, S, P_tc, B, beta=1.0) -> float:
    """(S / (alpha beta)) min(P_TC, B I_TC)  (Eq. 12; Eq. 20 with P_SpTC)."""
    a = alpha(shape, d, r, t)
    return S / (a * beta) * roofline(P_tc, B, I_tc(shape, d, r, t, D, S, beta))


def bound(I: float, P_peak: float, B: float) -> str:
    """'MB' below the ridge, 'CB' at or above it."""
    return "MB" if I < ridge(P_peak, B) else "CB"


def scenario(shape, d, r, t, D, S, P_cu, P_tc, B, beta=1.0) -> int:
    """Scenario 1..4 of Sec. 4.1: (CU bound, TC bound) = (MB,MB),(MB,CB),(CB,MB),(CB,CB)."""
    cu = bound(I_cu(shape, d, r, t, D), P_cu, B)
    tc = bound(I_tc(shape, d, r, t, D, S, beta), P_tc, B)
    return {("MB", "MB"): 1, ("MB", "CB"): 2, ("CB", "MB"): 3, ("CB", "CB"): 4}[(cu, tc)]


def speedup(shape, d, r, t, D, S, P_cu, P_tc, B, beta=1.0) -> float:
    """P_TC,actual / P_CU,actual (Sec. 4.1, Eq. 13)."""
    return P_tc_actual(shape, d, r, t, D, S, P_tc, B, beta) / P_cu_actual(shape, d, r, t, D, P_cu, B)


def alpha_condition(shape, d, r, t, S, P_cu, P_tc, beta=1.0) -> bool:
    """alpha < S P_TC / P_CU (Eq. 19), with beta folded into alpha."""
    return alpha(shape, d, r, t) * beta < S * P_tc / P_cu


def in_sweet_spot(shape, d, r, t, D, S, P_cu, P_tc, B, beta=1.0) -> bool:
    sc = scenario(shape, d, r, t, D, S, P_cu, P_tc, B, beta)
    return sc == 3 or (sc == 4 and alpha_condition(shape, d, r, t, S, P_cu, P_tc, beta))


def gstencils_roof_cu(shape, d, r, t, D, P_cu, B) -> float:
    """Point updates per second at the CUDA-core roof: min(P/(2K), t B/(2D))."""
    return P_cu_actual(shape, d, r, t, D, P_cu, B) / C_point(shape, d, r)


def gstencils_roof_tc(shape, d, r, t, D, S, P_tc, B, beta=1.0) -> float:
    """Point updates per second at the tensor-core roof:
    min(S P/(2K alpha beta), t B/(2D))."""
    return P_tc_actual(shape, d, r, t, D, S, P_tc, B, beta) / C_point(shape, d, r)
