"""Tolerances of the parity tests against the FP64 oracle (relative L2 per
field): round-off for FP64 storage, 1e-5 for FP32 storage and 1e-3 for the
16-bit formats (the targets the library is held to).

The 16-bit formats keep the moments f^0, J in FP32 and the pair sums'
non-equilibrium parts in 16 bits a value.  Where the accumulated rounding
of those parts exceeds 1e-3 for BF16 or FP16 (BF16's 8-bit significand on
fast waves, a_0 <= 0.99, or on the 10^4-step waves; FP16 on the 10^4-step
waves, the paper's tension and shear squares and fast rough cases) the run
is reported as an expected failure (xfail) with its measured error, and must
still stay below a regression bound per format: a known precision limit of
the format, not a passing test.  BFP13 has no such bound: it is held to
1e-3 on every case.
"""
import pytest

TARGET = {"f64": 1e-10, "f32": 1e-5, "bf16": 1e-3, "f16": 1e-3, "bfp13": 1e-3}
# regression bounds of the runs that miss the 16-bit target (largest
# measured: BF16 1.4e-2, a_0 = 0.9 mixed rectangle; FP16 1.7e-3, same case)
LIMIT_16 = {"bf16": 2e-2, "f16": 2e-3}


def judge(errs, storage, what=""):
    """Pass if every field meets the target; for a 16-bit format that misses
    it but stays within LIMIT_16, xfail with the measured error; else fail."""
    worst = max(errs.values())
    print(f"rel-L2 {storage} {worst:.3e} {what}")
    if worst <= TARGET[storage]:
        return errs
    if storage in LIMIT_16 and worst <= LIMIT_16[storage]:
        pytest.xfail(f"{storage} rel-L2 {worst:.2e} > {TARGET[storage]:g}: 16-bit precision limit {what}")
    raise AssertionError((what, storage, errs))
