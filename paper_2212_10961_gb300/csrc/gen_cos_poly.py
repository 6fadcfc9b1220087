"""Coefficients of the FP32 polynomial cosine used on the FMA pipe.

cos(2 pi f) for f in [-1/2, 1/2] (f in turns) is written as a polynomial in
s = f^2 on [0, 1/4],  c_0 + c_1 s + ... + c_6 s^6, evaluated by Horner's rule
in FP32.  The coefficients are the least-squares fit on Chebyshev nodes of
the first kind (a near-minimax fit; see e.g. Trefethen, "Approximation Theory
and Approximation Practice", ch. 4), computed in FP64 and then rounded to
FP32.  The script prints the coefficients and the error of the FP32
Horner evaluation against numpy's FP64 cosine on a dense grid.

Run: python gen_cos_poly.py
"""
import numpy as np

DEGREE = 6  # in s = f^2, i.e. degree 12 in f


def fit(degree=DEGREE, nodes=4096):
    k = np.arange(nodes)
    # Chebyshev nodes on [0, 1/4]
    s = 0.125 + 0.125 * np.cos((2 * k + 1) * np.pi / (2 * nodes))
    f = np.sqrt(s)
    y = np.cos(2 * np.pi * f)
    # weights: relative to nothing (absolute error matters for the field sum)
    V = np.vander(s, degree + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V, y, rcond=None)
    return c


def horner_fp32(c32, f):
    f = np.asarray(f, dtype=np.float32)
    s = (f * f).astype(np.float32)
    acc = np.float32(c32[-1]) * np.ones_like(s)
    for cc in c32[-2::-1]:
        acc = (acc * s + np.float32(cc)).astype(np.float32)
    return acc


def main():
    c = fit()
    c32 = c.astype(np.float32)
    f = np.linspace(-0.5, 0.5, 2_000_001)
    err = np.max(np.abs(horner_fp32(c32, f).astype(np.float64) - np.cos(2 * np.pi * f)))
    print("max abs error of the FP32 Horner evaluation on [-1/2, 1/2]: %.3e" % err)
    for i, v in enumerate(c32):
        print("c%d = %.9ef" % (i, float(v)))


if __name__ == "__main__":
    main()
