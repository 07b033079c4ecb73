"""Derive the coefficients of the kernels' sine/cosine of a quarter turn.

The azimuth of a sample is 2 pi m / 2^24 for a 24-bit integer m.  The kernels
split m exactly into a quarter-turn index q and a remainder y in [-1/2, 1/2)
(in quarter turns), and evaluate sin(pi y / 2) = y P(y^2), cos(pi y / 2) = Q(y^2).
P (degree 3) and Q (degree 4) are fitted here by weighted least squares on
Chebyshev nodes of y^2 in [0, 1/4], refined with a few Lawson iterations towards
the minimax fit, and rounded to float32.  Run to print the coefficients and the
float32 Horner error over every y on the 2^-22 grid.
"""
import numpy as np


def fit(func, deg, n=4000, iters=60):
    t = 0.125 * (1 - np.cos(np.pi * (np.arange(n) + 0.5) / n))  # Chebyshev nodes of y^2 in [0, 1/4]
    y = np.sqrt(t)
    target = func(y)
    A = np.vander(t, deg + 1, increasing=True)
    w = np.ones(n)
    for _ in range(iters):                                     # Lawson: weights follow the error
        c, *_ = np.linalg.lstsq(A * w[:, None], target * w, rcond=None)
        err = np.abs(A @ c - target)
        w = w * np.sqrt(err / err.max() + 1e-30)
        w /= w.max()
    return c


def main():
    P = fit(lambda y: np.where(y > 0, np.sin(np.pi * y / 2) / np.where(y > 0, y, 1), np.pi / 2), 3)
    Q = fit(lambda y: np.cos(np.pi * y / 2), 4)
    P32 = P.astype(np.float32)
    Q32 = Q.astype(np.float32)
    Q32[0] = np.float32(1.0)
    print("P (y, y^3, y^5, y^7):", [float(v) for v in P32])
    print("Q (1, y^2, y^4, y^6, y^8):", [float(v) for v in Q32])
    f = np.arange(-(1 << 21), 1 << 21, dtype=np.int64)
    y = (f.astype(np.float32) * np.float32(2.0 ** -22)).astype(np.float32)
    y2 = (y * y).astype(np.float32)
    ps = P32[3]
    for c in P32[2::-1]:
        ps = (ps * y2 + c).astype(np.float32)
    s = (y * ps).astype(np.float32)
    pc = Q32[4]
    for c in Q32[3::-1]:
        pc = (pc * y2 + c).astype(np.float32)
    es = np.abs(s.astype(np.float64) - np.sin(np.pi * y.astype(np.float64) / 2)).max()
    ec = np.abs(pc.astype(np.float64) - np.cos(np.pi * y.astype(np.float64) / 2)).max()
    print(f"max abs error (float32 Horner, no FMA): sin {es:.3e}, cos {ec:.3e}")


if __name__ == "__main__":
    main()
