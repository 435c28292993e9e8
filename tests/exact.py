"""Exact rational evaluation of the track position, for pinning the oracle.

Every FP64 input (v/c, n, t, f1, T_SFT) is converted to the exact rational it represents
and the real-valued track position of Eq. (track) (a_p = 0, with the f1 term)

    x = (K0 + j + f1 (t - t0) T_SFT) (1 + v . n) - k_lo

is evaluated with no rounding at all, then rounded half-up to a bin.  This involves none
of the oracle's code and none of its FP64 operation order.
"""
from fractions import Fraction as F


def position(K0, k_lo, j, f1, t_mid, t0, t_sft, v, n):
    eps = F(float(v[0])) * F(float(n[0])) + F(float(v[1])) * F(float(n[1])) + F(float(v[2])) * F(float(n[2]))
    tau = (F(float(t_mid)) - F(float(t0))) * F(float(t_sft))
    return (F(int(K0) + int(j)) + F(float(f1)) * tau) * (1 + eps) - int(k_lo)


def bin_and_tie_distance(x: F):
    """Round-half-up bin of x and |x - nearest half-integer| (as a float)."""
    y = x + F(1, 2)
    k = y.numerator // y.denominator
    frac = y - k
    d = min(frac, 1 - frac)
    return int(k), float(d)
