"""Exact FP32 helpers for tests: IEEE fused multiply-add emulated in numpy.

``fma32(a, b, c)`` returns round-to-nearest-even of a*b + c for float32
arrays, computed exactly: a*b is exact in float64, TwoSum gives the exact
error of the float64 addition, and the only case where rounding the float64
sum to float32 can differ from rounding the exact value (a sum exactly on a
float32 midpoint) is resolved by the sign of that error.
"""
import numpy as np

f32 = np.float32
f64 = np.float64


def fma32(a, b, c):
    a = np.asarray(a, f32)
    b = np.asarray(b, f32)
    c = np.asarray(c, f32)
    p = a.astype(f64) * b.astype(f64)
    cd = c.astype(f64)
    s = p + cd
    bb = s - p
    err = (p - (s - bb)) + (cd - bb)
    r = s.astype(f32)
    rd = r.astype(f64)
    diff = s - rd
    toward = np.where(diff > 0, np.inf, -np.inf).astype(f32)
    nbr = np.nextafter(r, toward)
    mid = (rd + nbr.astype(f64)) * 0.5
    at_mid = (diff != 0) & (s == mid)
    pick_nbr = at_mid & (err != 0) & (np.sign(err) == np.sign(nbr.astype(f64) - rd))
    return np.where(pick_nbr, nbr, r).astype(f32)


def r2_contract(dx, dy, dz):
    """r2 = fma(dz, dz, fma(dy, dy, dx*dx)) in FP32 (the kernels' order)."""
    dx = np.asarray(dx, f32)
    return fma32(dz, dz, fma32(dy, dy, (dx * dx).astype(f32)))
