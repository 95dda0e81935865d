"""The float32 atan2 of the bicycle inverse (atan2_poly in
paper_2310_08710_b300/csrc/wsim_phases.cuh) on the CPU: its coefficients are
read from the kernel source, the same steps are evaluated in float32 with
numpy, and the result is compared with the exact angle (float64 arctan2)
over every octant, the octant boundaries, signed zeros and magnitudes from
1e-30 to 1e30.  The coefficients must also be the ones the committed fit
script produces (Lawson's method, degree 7 in t^2)."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2310_08710_b300", "csrc", "wsim_phases.cuh")


def _coefficients():
    s = open(SRC).read()
    body = s[s.index("float atan2_poly("):]
    body = body[:body.index("return copysignf")]
    first = re.search(r"float q = ([-0-9.e+]+)f;", body).group(1)
    rest = re.findall(r"q = fmaf\(q, s, ([-0-9.e+]+)f\);", body)
    return np.array([first] + rest, dtype=np.float32)  # highest degree first


def atan2_poly(y, x, c):
    y = np.asarray(y, np.float32)
    x = np.asarray(x, np.float32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    with np.errstate(invalid="ignore", divide="ignore"):
        t = np.where(mx > 0, mn / np.where(mx > 0, mx, 1), 0).astype(np.float32)
    s = (t * t).astype(np.float32)
    q = np.full_like(t, c[0])
    for k in c[1:]:
        q = (q * s + k).astype(np.float32)  # the device uses fma: within an ulp of this
    r = (t * q).astype(np.float32)
    r = np.where(ay > ax, np.float32(1.57079637) - r, r).astype(np.float32)
    r = np.where(x < 0, np.float32(3.14159274) - r, r).astype(np.float32)
    return np.copysign(r, y)


def test_coefficients_are_the_fit():
    sys.path.insert(0, os.path.join(ROOT, "paper_2310_08710_b300", "csrc"))
    import gen_atan_poly
    c, rel = gen_atan_poly.fit()
    assert rel < 2e-7
    assert np.array_equal(c[::-1], _coefficients())


def test_every_direction_within_4e7():
    c = _coefficients()
    rng = np.random.default_rng(0)
    ang = np.concatenate([rng.uniform(-np.pi, np.pi, 200000),
                          np.arange(-4, 5) * np.pi / 4,
                          np.arange(-4, 5) * np.pi / 4 + 1e-7, np.arange(-4, 5) * np.pi / 4 - 1e-7])
    mag = 10.0 ** rng.uniform(-30, 30, ang.size)
    x = (mag * np.cos(ang)).astype(np.float32)
    y = (mag * np.sin(ang)).astype(np.float32)
    got = atan2_poly(y, x, c).astype(np.float64)
    want = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(got - want)
    err = np.minimum(err, 2 * np.pi - err)  # +-pi on the negative x axis
    assert err.max() <= 4e-7, err.max()


def test_axes_and_signed_zeros():
    c = _coefficients()
    cases = [(0.0, 1.0, 0.0), (1.0, 0.0, np.pi / 2), (0.0, -1.0, np.pi), (-0.0, -1.0, -np.pi),
             (-1.0, 0.0, -np.pi / 2), (-1.0, -0.0, -np.pi / 2), (1.0, 1.0, np.pi / 4), (0.0, 0.0, 0.0),
             (-0.0, 0.0, -0.0)]
    for y, x, want in cases:
        got = float(atan2_poly(np.float32(y), np.float32(x), c))
        assert abs(got - want) <= 4e-7 and np.signbit(got) == np.signbit(want), (y, x, got, want)
