"""Coefficients of the joint sin/cos polynomials of smpc_device.cuh (joint_sincos).

On r in [-R, R], R = 1.01 pi/4 (the remainder of a Cody-Waite reduction by
pi/2, with room for the rounding of x 2/pi):
    sin r ~ r + r^3 (S0 + S1 z + S2 z^2 + S3 z^3),   z = r^2
    cos r ~ 1 + z   (C0 + C1 z + C2 z^2 + C3 z^3)
Each bracket is a least-squares fit, in z, of (sin sqrt(z) - sqrt(z)) / z^1.5
and (cos sqrt(z) - 1) / z on 4000 Chebyshev nodes of [0, R^2] (close to the
minimax fit), rounded to float32.  Prints the constants and the worst error
of the float32 evaluation (emulated: every operation rounded to float32)
against sin and cos in float64, in float32 ulps of the result.

    python paper_2512_22575_b300/csrc/gen_sincos_poly.py
"""
import numpy as np

R = 1.01 * np.pi / 4
N_NODES = 4000


def fit(f, deg):
    k = np.arange(N_NODES)
    z = 0.5 * R * R * (1.0 - np.cos(np.pi * (k + 0.5) / N_NODES))
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


if __name__ == "__main__":
    main()
