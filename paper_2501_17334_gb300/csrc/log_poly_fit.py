"""Reproduces the polynomial of log_poly.h: Q(f) ~ (log1p(f) - f) / f^2 on [sqrt(1/2) - 1,
sqrt(2) - 1], degree 8, by Lawson's iteratively reweighted least squares (converges to the
minimax fit).  Prints the coefficients, lowest degree first."""
import numpy as np


def fit(deg=8, iters=200):
    a, b = np.sqrt(0.5) - 1, np.sqrt(2) - 1
    f = np.linspace(a, b, 20001)
    f = f[np.abs(f) > 1e-6]
    y = (np.log1p(f) - f) / (f * f)
    V = np.vander(f, deg + 1, increasing=True)
    w = np.ones_like(f)
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * sw[:, None], y * sw, rcond=None)
        e = np.abs(V @ c - y)
        w = w * e
        w /= w.sum()
    return c, float(np.abs(V @ c - y).max())


if __name__ == "__main__":
    c, err = fit()
    print("max |Q error| = %.3e" % err)
    for v in c:
        print(repr(float(v)))
