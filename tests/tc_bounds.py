"""Error bounds of the tensor-core precision forms, derived from their arithmetic.

Per fused sweep, with positive weights summing to 1 (the sweep is then
non-expansive in the max norm, so errors add up over sweeps):
  * operand rounding P: TF32 rounds the field and the weights to 11
    significant bits (P = 2 * 2^-11); the hi+lo forms leave a lo part rounded
    to the form's precision plus the dropped lo*lo product (TF32x3:
    P = 2^-21; BF16x3, 8-bit parts: P = 2^-15);
  * accumulation: every MMA adds into an FP32 accumulator in TMEM, which may
    lose up to one unit in the last place (2^-23) per accumulation, and there
    are n_mma accumulations per output and sweep (from the issued layout).
The bound after n sweeps is n * (P + n_mma * 2^-23) relative to max|u|.
"""
from paper_2603_00477_gb300 import binding as B

P_FORM = {"tf32": 2.0 * 2 ** -11, "tf32x3": 2.0 ** -21, "bf16x3": 2.0 ** -15}


def mma_per_output(plan_handle, t: int, split: bool) -> int:
    _, lo, hi, _ = B.stencil_plan_tc_layout(plan_handle, t, with_B=False)
    blocks = sum(max(0, h - l + 1) for l, h in zip(lo, hi))
    return blocks * (3 if split else 1)


def sweeps(steps: int, t: int) -> int:
    return steps // t + (1 if steps % t else 0)


def tc_bound(form: str, steps: int, t: int, plan_handle) -> float:
    n_mma = mma_per_output(plan_handle, t, form != "tf32")
    return sweeps(steps, t) * (P_FORM[form] + n_mma * 2.0 ** -23)
