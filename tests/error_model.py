"""Error models of the two GPU paths' arithmetic, handed to the oracle's running error bound (test helper).

Each describes how a path evaluates Eq. 12 in the deviation form (the oracle's `segment_bound` turns it into a
first-order bound per segment average and per cell moment):

* FP64 (path 0): every operation in binary64 (u = 2^-53); exp and expm1 with relative error at most 2^-51
  (two units in the last place, above the one-ulp accuracy of CUDA's double-precision exp and expm1); every term
  omega (A/V) Omega.. Ibar added to the cell sums one by one in any order (recursive summation, gamma_{n-1}).
* FP32 (path 1): operations in binary32 (u = 2^-24); e^-tau as the square of 2^x from ex2.approx.ftz.f32 and 1/x
  from rcp.approx.ftz.f32, each taken with relative error at most 2^-21 and 2^-22 (above the errors the PTX ISA
  states for these approximations; the GPU test of the attenuation checks E1 against them over twelve decades of
  tau); a moment term passes through k_sum = n_polar + 18 roundings of relative u32 on its way into the two-word
  sums: the polar fold (n_polar additions and a coefficient w sin^2 zeta of five roundings), the area fraction
  (one), the run of at most 8 same-pair segments (eight), the angular factor cos^2 phi times the run sum (four);
  the two-word sums and the FP64 assembly add errors of order u32^2 and u64, covered by the bound's 8 u64 term.
  The FP32 state works in units scaled by a power of two (max(B, boundary) near 2^100); a result below the normal
  FP32 range there carries an absolute error of 2^-126 in scaled units, about 1e-68 of that maximum.
"""

import numpy as np

FP64 = {"path": 0, "u": 2.0 ** -53, "e_exp": 2.0 ** -51}
FP32_E_EX2 = 2.0 ** -21
FP32_E_RCP = 2.0 ** -22


def fp32_scale(B, bnd) -> float:
    """The FP32 state's scale: the power of two that maps max(B, boundary) into [2^99, 2^100)."""
    m = max(float(np.max(B)), float(np.max(bnd)))
    return 2.0 ** (100 - (np.frexp(m)[1] if m > 0 else 0))


def model(prec: str, n_polar: int, B=None, bnd=None, Bref=None) -> dict:
    """The error model of a path; for FP32, B and bnd fix the state's scale, below which results leave the normal
    FP32 range (absolute error 2^-126 / scale per operation)."""
    if prec == "fp64":
        m = dict(FP64)
    else:
        # the path keeps a scale while the scaled maximum stays within 2^-7 .. 2^8 of its target: the smallest
        # scale it may sweep with is 2^-7 of fp32_scale
        m = {"path": 1, "u": 2.0 ** -24, "e_exp": FP32_E_EX2, "e_rcp": FP32_E_RCP, "k_sum": n_polar + 18.0,
             "abs_unit": 2.0 ** -126 * 2.0 ** 7 / fp32_scale(B, bnd)}
    if Bref is not None:
        m["Bref"] = Bref
    return m
