"""CPU checks of the polynomials the kernels use for the joint sin/cos
(Eq. 6) and the Box-Muller radius and angle (Eq. 27).

The coefficients in smpc_device.cuh (kSinCosPoly, kLnP0-3) must be those
that gen_sincos_poly.py fits, and the float32 evaluation (every operation
rounded to float32, as emulated by that script) must stay within one ulp of
sin and cos on the reduced range [-1.01 pi/4, 1.01 pi/4] and within two ulps
of ln u on the sampler's uniforms u = (i + 1/2) 2^-23.  Taylor checks pin the
fits: the leading sin/cos coefficients are -1/6 and -1/2 to float32
rounding, the next ones 1/120 and 1/24 within 1e-5 relative; the atanh
series' 1/3 and 1/5 within 1e-5.
"""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_22575_b300", "csrc")


def load_generator():
    spec = importlib.util.spec_from_file_location("gen_sincos_poly", os.path.join(CSRC, "gen_sincos_poly.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def header_coefficients():
    src = open(os.path.join(CSRC, "smpc_device.cuh")).read()
    body = re.search(r"constexpr float2 kSinCosPoly\[4\] = \{(.*?)\};", src, re.S).group(1)
    vals = [float(v) for v in re.findall(r"(-?\d\.\d+e[-+]\d+)f", body)]
    assert len(vals) == 8
    pairs = np.array(vals).reshape(4, 2)          # (sin, cos), highest degree first
    return pairs[::-1, 0].astype(np.float32), pairs[::-1, 1].astype(np.float32)


def test_header_matches_generator():
    gen = load_generator()
    S = gen.fit(lambda z: (np.sin(np.sqrt(z)) - np.sqrt(z)) / z ** 1.5, 3)
    C = gen.fit(lambda z: (np.cos(np.sqrt(z)) - 1.0) / z, 3)
    hs, hc = header_coefficients()
    np.testing.assert_allclose(hs, S, rtol=2e-7)
    np.testing.assert_allclose(hc, C, rtol=2e-7)


def test_taylor_pins():
    hs, hc = header_coefficients()
    assert hs[0] == np.float32(-1.0 / 6.0) and hc[0] == np.float32(-0.5)
    assert abs(hs[1] / (1.0 / 120.0) - 1.0) < 1e-5 and abs(hc[1] / (1.0 / 24.0) - 1.0) < 1e-5
    assert abs(hs[2] / (-1.0 / 5040.0) - 1.0) < 1e-3 and abs(hc[2] / (-1.0 / 720.0) - 1.0) < 1e-3


def test_float32_evaluation_within_one_ulp():
    gen = load_generator()
    hs, hc = header_coefficients()
    r = gen.f32(np.linspace(-gen.R, gen.R, 200_001))
    r = r[r != 0]
    s, c = gen.evaluate(r, hs, hc)
    us = np.spacing(np.abs(np.sin(r)).astype(np.float32)).astype(np.float64)
    uc = np.spacing(np.abs(np.cos(r)).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(s - np.sin(r)) / us) < 1.0
    assert np.max(np.abs(c - np.cos(r)) / uc) < 1.0


def header_ln_coefficients():
    src = open(os.path.join(CSRC, "smpc_device.cuh")).read()
    vals = [float(re.search(r"kLnP%d = (-?\d\.\d+e[-+]\d+)f" % i, src).group(1)) for i in range(4)]
    return np.array(vals, dtype=np.float32)


def test_ln_header_matches_generator_and_taylor():
    gen = load_generator()
    L = header_ln_coefficients()
    np.testing.assert_allclose(L, gen.fit_ln(), rtol=2e-7)
    assert abs(L[0] * 3.0 - 1.0) < 1e-5 and abs(L[1] * 5.0 - 1.0) < 1e-5


def test_ln_float32_evaluation_within_two_ulps():
    gen = load_generator()
    L = header_ln_coefficients()
    i = np.concatenate([np.arange(0, 1 << 23, 5), np.arange((1 << 23) - 4096, 1 << 23)]).astype(np.int64)
    u = gen.f32((i + 0.5) * 2.0 ** -23)
    ln = gen.ln_unit(u, L)
    ulp = np.spacing(np.abs(np.log(u)).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(ln - np.log(u)) / ulp) < 2.0
