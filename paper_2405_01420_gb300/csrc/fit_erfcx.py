"""Fit the rational approximation of erfcx(x) = exp(x^2) erfc(x) used by the kernels.

The force kernel needs erfc(beta r) for Ewald real-space Coulomb. It writes
erfc(x) = exp(-x^2) * R(x) with R(x) = P(x) / Q(x), P and Q of degree 4,
Q(0) = 1, fitted here for minimum relative error on [0, X_MAX] by
Sanathanan-Koerner iteration (linearised weighted least squares) in FP64.
Ewald parameters in use have beta * rc = 3.1234 (erfc(beta rc) = 1e-5),
so pairs inside the cutoff have x < 3.2.

Run ``python fit_erfcx.py`` to print the coefficients as they appear in
``nb_pair.cuh`` and the FP32 error of that evaluation order.
"""
import numpy as np
from scipy.special import erfcx

X_MAX = 3.2
DEG = 4


def fit(deg: int = DEG, x_max: float = X_MAX, iters: int = 40):
    xs = np.linspace(0.0, x_max, 40001)
    y = erfcx(xs)
    w = 1.0 / y
    qv = np.ones_like(xs)
    for _ in range(iters):
        vp = np.vander(xs, deg + 1, increasing=True)
        vq = np.vander(xs, deg + 1, increasing=True)[:, 1:]
        a = np.hstack([vp, -(y[:, None] * vq)]) * (w / qv)[:, None]
        c, *_ = np.linalg.lstsq(a, y * (w / qv), rcond=None)
        p = c[: deg + 1]
        q = np.concatenate([[1.0], c[deg + 1:]])
        qv = np.vander(xs, deg + 1, increasing=True) @ q
    return p, q


def fp32_error(p, q, x_max: float = X_MAX):
    """Max relative error of FMA-Horner P/Q evaluated in FP32 on a fine grid."""
    p32 = p.astype(np.float32)
    q32 = q.astype(np.float32)
    x = np.linspace(0.0, x_max, 200001).astype(np.float32)

    def horner(c):
        acc = np.full_like(x, c[-1])
        for k in range(len(c) - 2, -1, -1):
            acc = (acc.astype(np.float64) * x.astype(np.float64) + np.float64(c[k])).astype(np.float32)
        return acc

    r = horner(p32).astype(np.float64) / horner(q32).astype(np.float64)
    ref = erfcx(x.astype(np.float64))
    return float(np.abs(r / ref - 1.0).max())


if __name__ == "__main__":
    p, q = fit()
    print("P:", ", ".join(f"{v:.9e}f" for v in p.astype(np.float32)))
    print("Q:", ", ".join(f"{v:.9e}f" for v in q.astype(np.float32)))
    print("max rel error (FP32 Horner):", fp32_error(p, q))
