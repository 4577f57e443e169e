"""Coefficients of the float32 scaled complementary error function used by
the short-range kernel: erfcx(x) = erfc(x) exp(x^2) ~= sum_k c_k t^k with
t = 1 / (1 + x / 2), a least-squares fit weighted for relative error on
[0, 8] (degree 10).  Prints the C array; run once, paste into k_short.cu.
"""
import numpy as np
from scipy.special import erfcx

P, DEG, XMAX = 0.5, 10, 8.0


def fit():
    xs = np.linspace(0.0, XMAX, 200001)
    h = erfcx(xs)
    t = 1.0 / (1.0 + P * xs)
    A = np.vander(t, DEG + 1, increasing=True)
    c, *_ = np.linalg.lstsq(A / h[:, None], np.ones_like(h), rcond=None)
    return xs, h, c


def float32_rel_error(xs, h, c):
    t = (np.float32(1) / (np.float32(1) + np.float32(P) * xs.astype(np.float32))).astype(np.float32)
    v = np.zeros_like(t)
    for ck in c[::-1].astype(np.float32):
        v = (v * t + ck).astype(np.float32)
    return float(np.max(np.abs(v.astype(np.float64) - h) / h))


if __name__ == "__main__":
    xs, h, c = fit()
    print("// max relative error in float32: %.2e" % float32_rel_error(xs, h, c))
    print("{ " + ", ".join("%.9ef" % v for v in c) + " }")
