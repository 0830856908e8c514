"""Error bounds of the tensor-core precision forms, derived from their arithmetic.

Per fused sweep, with positive weights summing to 1 (the sweep is then
non-expansive in the max norm, so errors add up over sweeps):
  * operand rounding P: TF32 rounds the field and the weights to 11
    significant bits (P = 2 * 2^-11); the hi+lo forms leave a lo part rounded
    to the form's precision plus the dropped lo*lo product (TF32x3:
    P = 2^-21; BF16x3, 8-bit parts: P = 2^-15);
  * accumulation: every MMA adds into an FP32 accumulator in TMEM, which may
    lose up to one unit in the last place (2^-23) per accumulation, and there
    are n_mma accumulations per output and sweep.
The bound after n sweeps is n * (P + n_mma * 2^-23) relative to max|u|.

n_mma is counted here from the band geometry of the composite kernel (the
Toeplitz formulation of Sec. 2.2), not read from the library: line a of the
composite (radius R = t r) has half-width h_a = R for a box and
r (t - ceil(|a|/r)) for a star; with MMA width N and K step k its window of
N + 2R columns is padded to nkb = ceil((N + 2R)/k) blocks, of which the
blocks holding a column in [R - h_a, R + h_a + N - 1] are issued.  The
library's exported layout must issue exactly that many (checked), so a
kernel that issued extra MMAs could not loosen its own tolerance.  For the
2:4 sparse form (M = 16 output columns, logical K = 16 per instruction, the
window of 16 + 2R columns cut into 4-column chunks that are paired) any
valid pairing needs at most ceil(nc / 2) instructions per line, nc =
ceil((16 + 2R)/4); that independent count is the sparse n_mma.
"""
from paper_2603_00477_gb300 import binding as B

# F16 / F16X3 (FP16 operands scaled by a power of two per tile and for the
# weights) keep 11 significant bits relative to the tile's largest value, like
# TF32 (normwise), and hi + lo 22 bits, like TF32x3
P_FORM = {"tf32": 2.0 * 2 ** -11, "tf32x3": 2.0 ** -21, "bf16x3": 2.0 ** -15,
          "f16": 2.0 * 2 ** -11, "f16x3": 2.0 ** -21}


def line_half(shape: str, r: int, t: int, a: int) -> int:
    """Half-width of line a of the t-fold composite kernel (-1: empty line)."""
    R = t * r
    if shape == "box":
        return R
    ca = (abs(a) + r - 1) // r
    return -1 if ca > t else r * (t - ca)


def dense_mma_per_output(shape: str, r: int, t: int, n_tile: int, k_inst: int) -> int:
    """MMAs (per accumulator) that add into one output of a fused sweep."""
    R = t * r
    nkb = -(-(n_tile + 2 * R) // k_inst)
    total = 0
    for a in range(-R, R + 1):
        h = line_half(shape, r, t, a)
        if h < 0:
            continue
        lo = (R - h) // k_inst
        hi = min(nkb - 1, (R + h + n_tile - 1) // k_inst)
        total += hi - lo + 1
    return total


def sparse_mma_bound(shape: str, r: int, t: int) -> int:
    """Upper bound of the mma.sp instructions that add into one output."""
    R = t * r
    nc = -(-(16 + 2 * R) // 4)
    per_line = -(-nc // 2)
    return sum(per_line for a in range(-R, R + 1) if line_half(shape, r, t, a) >= 0)


def sweeps(steps: int, t: int) -> int:
    return steps // t + (1 if steps % t else 0)


def mma_per_output(plan_handle, shape: str, r: int, t: int, split: bool) -> int:
    lay, lo, hi, _ = B.stencil_plan_tc_layout(plan_handle, t, with_B=False)
    n = dense_mma_per_output(shape, r, t, lay["n_tile"], lay["k_inst"])
    issued = sum(max(0, h - l + 1) for l, h in zip(lo, hi))
    assert issued == n, f"the exported layout issues {issued} MMAs per output, the band needs {n}"
    return n * (3 if split else 1)


def tc_bound(form: str, steps: int, t: int, plan_handle, shape: str, r: int) -> float:
    n_mma = mma_per_output(plan_handle, shape, r, t, form not in ("tf32", "f16"))
    return sweeps(steps, t) * (P_FORM[form] + n_mma * 2.0 ** -23)


def sp_bound(plan_handle, shape: str, r: int, steps: int, t: int) -> float:
    n_mma = sparse_mma_bound(shape, r, t)
    mask = B.stencil_plan_sptc_layout(plan_handle, t)[3]
    issued = int(sum(bin(int(m)).count("1") for m in mask))
    assert issued <= n_mma, f"the exported layout issues {issued} sparse MMAs per output (bound {n_mma})"
    return sweeps(steps, t) * (2.0 * 2 ** -11 + n_mma * 2.0 ** -23)
