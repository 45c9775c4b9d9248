"""Error bounds of the precision forms, derived from the operand rounding.

A non-negative sum of products whose operands carry a relative rounding error
<= u_op each, accumulated in FP32 (<= 144 terms; u_acc = 2^-16 covers their
roundings and the few ulp of the power; 2^-15 in the tensor-core forms, whose
hardware power and pooling keys (the maximum's last 5 bits) add to that), has relative error <= r_0 = (1 +
u_op)^2 (1 + u_acc) - 1.  Pooling and averaging non-negative values keep a
relative error bound, and x -> x^lambda turns a factor (1 + r) into (1 +
r)^lambda, so the unrectified values of level l carry at most r_l = (1 +
r_0)^(lambda^l) - 1 and the stored (rectified) maps eps_l = (1 +
r_0)^(lambda^(l+1)) - 1; u_op = 0 (FP32), 2^-9 (BF16: 8 mantissa bits), 2^-4
(E4M3: 3 mantissa bits; the per-patch power-of-two scaling is exact).

Decisions.  An argmax between candidates x1 > x2 can only change if x2 / x1 >
(1 - r_l) / (1 + r_l), i.e. where the FP64 gap of the rectified values
(reading c23) is below 1 - ((1 - r_l) / (1 + r_l))^lambda.  BestAt and
BestAt' compare path scores, sums of terms each within eps_L, which can only
change below a gap of 2 eps_L / (1 - eps_L).  So a patch's match can only
differ from the FP64 oracle's where one of its decisions (c23) is within
match_tol of a tie.
"""
import numpy as np

LAM = 1.4
U_OP = {"fp32": 0.0, "bf16": 2.0 ** -9, "fp8": 2.0 ** -4}
# FP32 arithmetic of the level-0 value: the FP32 path's fma chain and power;
# the tensor-core forms also carry the hardware power (lg2 / ex2 approximations)
# and the pooling keys, which keep the maximum to within 31 units of its last
# place (2^-18)
U_ACC = {"fp32": 2.0 ** -16, "bf16": 2.0 ** -15, "fp8": 2.0 ** -15}


def r_level(prec, l):
    """Bound on the relative error of the unrectified values of level l."""
    return ((1 + U_OP[prec]) ** 2 * (1 + U_ACC[prec])) ** (LAM ** l) - 1.0


def eps_level(prec, l):
    """Bound on the relative error of the stored (rectified) maps of level l."""
    return (1.0 + r_level(prec, l)) ** LAM - 1.0


def argmax_tol(prec, l):
    r = r_level(prec, l)
    return 1.0 - ((1.0 - r) / (1.0 + r)) ** LAM if r < 1 else 1.0


def match_tol(prec, L):
    e = eps_level(prec, L)
    return max(argmax_tol(prec, L - 1), 2 * e / (1 - e) if e < 1 else np.inf)
