"""Coefficients of the polynomials of smpc_device.cuh: the sin/cos pair
(sincos_quadrant, used by joint_sincos and the Box-Muller angle) and the
logarithm of the Box-Muller radius (ln_unit).

On r in [-R, R], R = 1.01 pi/4 (the remainder of a Cody-Waite reduction by
pi/2, with room for the rounding of x 2/pi):
    sin r ~ r + r^3 (S0 + S1 z + S2 z^2 + S3 z^3),   z = r^2
    cos r ~ 1 + z   (C0 + C1 z + C2 z^2 + C3 z^3)
Each bracket is a least-squares fit, in z, of (sin sqrt(z) - sqrt(z)) / z^1.5
and (cos sqrt(z) - 1) / z on 4000 Chebyshev nodes of [0, R^2] (close to the
minimax fit), rounded to float32.  Prints the constants and the worst error
of the float32 evaluation (emulated: every operation rounded to float32)
against sin and cos in float64, in float32 ulps of the result.

ln m for m in [sqrt(1/2), sqrt(2)) is 2 atanh(s), s = (m - 1) / (m + 1),
|s| <= S_MAX = (sqrt(2) - 1) / (sqrt(2) + 1):
    atanh(s) ~ s (1 + z (L0 + L1 z + L2 z^2 + L3 z^3)),   z = s^2
with the bracket a least-squares fit of (atanh(s)/s - 1) / z on 4000
Chebyshev nodes of [0, (1.001 S_MAX)^2], rounded to float32.

    python paper_2512_22575_b300/csrc/gen_sincos_poly.py
"""
import numpy as np

R = 1.01 * np.pi / 4
S_MAX = (np.sqrt(2.0) - 1.0) / (np.sqrt(2.0) + 1.0)
N_NODES = 4000


def fit(f, deg, zmax=R * R):
    k = np.arange(N_NODES)
    z = 0.5 * zmax * (1.0 - np.cos(np.pi * (k + 0.5) / N_NODES))
    A = np.vstack([z ** i for i in range(deg + 1)]).T
    c, *_ = np.linalg.lstsq(A, f(z), rcond=None)
    return c.astype(np.float32)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def fma32(a, b, c):
    # a*b exact in float64 (two 24-bit significands); one rounding to float32
    # after the add (the double rounding through float64 is not modelled)
    return f32(a * b + c)


def evaluate(r, S, C):
    z = f32(r * r)
    ps, pc = f32(S[3]), f32(C[3])
    for i in (2, 1, 0):
        ps = fma32(z, ps, f32(S[i]))
        pc = fma32(z, pc, f32(C[i]))
    s = fma32(f32(r * z), ps, r)
    c = fma32(z, pc, 1.0)
    return s, c


def fit_ln():
    return fit(lambda z: (np.arctanh(np.sqrt(z)) / np.sqrt(z) - 1.0) / z, 3, (1.001 * S_MAX) ** 2)


def ln_unit(u, L):
    """ln u as the kernels evaluate it, for float32 u in [2^-24, 1) (emulated)."""
    b = np.asarray(u, dtype=np.float32).view(np.uint32).astype(np.int64)
    e = ((b - 0x3F3504F3).astype(np.int32)) >> 23
    m = ((b - (e.astype(np.int64) << 23)) & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    f = f32(m - 1.0)
    s = f32(f / f32(2.0 + f))
    z = f32(s * s)
    p = f32(L[3])
    for i in (2, 1, 0):
        p = fma32(z, p, f32(L[i]))
    s2 = f32(s + s)
    lnm = fma32(f32(s2 * z), p, s2)
    ef = e.astype(np.float64)
    hi = f32(np.log(2.0))
    lo = f32(np.log(2.0) - hi)
    return fma32(ef, hi, fma32(ef, lo, lnm))


def main():
    S = fit(lambda z: (np.sin(np.sqrt(z)) - np.sqrt(z)) / z ** 1.5, 3)
    C = fit(lambda z: (np.cos(np.sqrt(z)) - 1.0) / z, 3)
    r = f32(np.linspace(-R, R, 400001))
    r = r[r != 0]
    s, c = evaluate(r, S, C)
    us = np.spacing(np.abs(np.sin(r)).astype(np.float32)).astype(np.float64)
    uc = np.spacing(np.abs(np.cos(r)).astype(np.float32)).astype(np.float64)
    print("sin coefficients", ", ".join(f"{float(x):.9e}f" for x in S))
    print("cos coefficients", ", ".join(f"{float(x):.9e}f" for x in C))
    print(f"worst error on [-R, R]: sin {np.max(np.abs(s - np.sin(r)) / us):.3f} ulp, "
          f"cos {np.max(np.abs(c - np.cos(r)) / uc):.3f} ulp")
    L = fit_ln()
    i = np.arange(0, 1 << 23, 3, dtype=np.int64)
    u = f32((i + 0.5) * 2.0 ** -23)
    ln = ln_unit(u, L)
    ul = np.spacing(np.abs(np.log(u)).astype(np.float32)).astype(np.float64)
    print("ln coefficients", ", ".join(f"{float(x):.9e}f" for x in L))
    print(f"worst error of ln on the uniforms (i + 1/2) 2^-23: {np.max(np.abs(ln - np.log(u)) / ul):.3f} ulp")


if __name__ == "__main__":
    main()
