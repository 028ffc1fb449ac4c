"""The joint sin/cos of the forward kinematics (Eq. 6) on the GPU.

The kernels evaluate sin and cos of every joint angle with their own routine
(a Cody-Waite reduction by pi/2, then polynomials on [-pi/4, pi/4] whose
Horner steps run in packed FP32 FMAs; smpc_device.cuh, joint_sincos).
pm_joint_sincos runs that device function.  Checks:
  * against sin/cos in float64 of the same float32 argument, over the joint
    range, near every multiple of pi/4 up to |x| = 64, at random arguments
    up to 1e4 and at a few up to 2^22: within 2 float32 ulps of the result
    for |x| <= 64, within 2^-23 absolute up to 1e4 and 2^-21 beyond;
  * against CUDA's own sincosf of the same arguments: within 2^-23;
  * sin^2 + cos^2 = 1 within 4 ulps; sin = 0 (of either sign) and cos = 1
    at +-0, sin x = x at +-1e-30; NaN for +-inf and NaN.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2512_22575_b300 as pm  # noqa: E402

DEV = torch.device("cuda", 0)


def run(x):
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(DEV)
    sc = torch.empty((xt.numel(), 2), dtype=torch.float32, device=DEV)
    ref = torch.empty_like(sc)
    pm.joint_sincos(xt, sc, ref)
    torch.cuda.synchronize()
    return sc.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)


def arguments():
    rng = np.random.default_rng(7)
    q = np.linspace(-3.0 * np.pi, 3.0 * np.pi, 200_001)            # joint range (with offsets)
    k = np.arange(-81, 82)[:, None] * (np.pi / 4)                  # multiples of pi/4 to |x| ~ 64
    near = (k + np.linspace(-1e-3, 1e-3, 201)[None, :]).ravel()
    ulps = (k.astype(np.float32).astype(np.float64) + 0.0).ravel()
    wide = rng.uniform(-1e4, 1e4, 200_000)
    big = rng.uniform(-(2.0 ** 22), 2.0 ** 22, 2_000)
    x = np.concatenate([q, near, ulps, wide, big]).astype(np.float32)
    return x


def test_against_float64_and_cuda_sincosf():
    x = arguments()
    sc, ref = run(x)
    xd = x.astype(np.float64)
    truth = np.stack([np.sin(xd), np.cos(xd)], axis=1)
    err = np.abs(sc - truth)
    ulp = np.spacing(np.abs(truth).astype(np.float32)).astype(np.float64)
    small = np.abs(xd) <= 1e4
    joint = np.abs(xd) <= 64.0
    assert err[small].max() <= 2.0 ** -23, err[small].max()
    # relative to the result (near its zeros the reduction's absolute error
    # counts in ulps of a small number, so over the joint angles)
    assert (err[joint] / ulp[joint]).max() <= 2.0, (err[joint] / ulp[joint]).max()
    # beyond 1e4 the reduction's second constant leaves up to |n| 2^-50 more
    assert err[~small].max() <= 2.0 ** -21, err[~small].max()
    assert np.abs(sc[small] - ref[small]).max() <= 2.0 ** -23
    print(f"max abs error {err.max():.3e}, max ulps (|x| <= 64) {(err[joint] / ulp[joint]).max():.2f}, "
          f"max |ours - sincosf| {np.abs(sc - ref)[small].max():.3e}")


def test_identity_and_special_values():
    x = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-30, -1e-30], dtype=np.float32)
    sc, _ = run(x)
    assert sc[0, 0] == 0.0 and sc[0, 1] == 1.0
    assert sc[1, 0] == 0.0 and sc[1, 1] == 1.0
    assert np.isnan(sc[2:5]).all()
    assert sc[5, 0] == np.float32(1e-30) and sc[6, 0] == np.float32(-1e-30) and (sc[5:7, 1] == 1.0).all()
    xs = arguments()[:200_001]
    s2, _ = run(xs)
    one = s2[:, 0] ** 2 + s2[:, 1] ** 2
    assert np.abs(one - 1.0).max() <= 4 * 2.0 ** -24
