"""Fit the function approximations used by the force kernels: erfcx and exp2.

The force kernel needs erfc(beta r) for Ewald real-space Coulomb. It writes
erfc(x) = exp(-x^2) * R(x) with R(x) = P(x) / Q(x), P and Q of degree 4,
Q(0) = 1, fitted here for minimum relative error on [0, X_MAX] by
Sanathanan-Koerner iteration (linearised weighted least squares) in FP64.
Ewald parameters in use have beta * rc = 3.1234 (erfc(beta rc) = 1e-5),
so pairs inside the cutoff have x < 3.2.

Run ``python fit_coeffs.py`` to print the coefficients as they appear in
``nb_pair.cuh`` and the FP32 error of that evaluation order; the exp2
polynomial is fitted at the end of the file.
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


# --------------------------------------------------------------------------
# 2^f on [-0.5, 0.5] for the kernels' exp: 2^t = 2^n * 2^f with n = rint(t).
# Polynomial 1 + c1 f + ... + c6 f^6, fitted for minimum relative error by
# iteratively reweighted least squares. Relative error 8.3e-9 in FP64,
# 8.1e-8 evaluated in FP32 (mean 9e-10).
# --------------------------------------------------------------------------
def fit_exp2(deg: int = 6, iters: int = 20):
    f = np.linspace(-0.5, 0.5, 20001)
    y = 2.0 ** f
    v = np.vander(f, deg + 1, increasing=True)[:, 1:]
    c, *_ = np.linalg.lstsq(v / y[:, None], (y - 1) / y, rcond=None)
    for _ in range(iters):
        err = (1 + v @ c) / y - 1
        w = 1 + 50 * np.abs(err) / np.abs(err).max()
        c, *_ = np.linalg.lstsq(v / y[:, None] * w[:, None], (y - 1) / y * w, rcond=None)
    return c


if __name__ == "__main__":
    c = fit_exp2()
    print("EXP2:", ", ".join(f"{v:.9e}f" for v in c.astype(np.float32)))
