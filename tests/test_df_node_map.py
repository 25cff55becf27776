"""The double-float evaluation of the Doppler node map (Sec. 3: each star's
spectrum shifted by its line-of-sight velocity and resampled).

The reading maps output bin j to the fractional SSP node position
t(j) = ((l0 + j dl) / ((1 + z)(1 + v/c)) - ls0) / dls = B + j A, in FP64.
The setup kernel computes A and B without FP64 arithmetic: with
g = (v/c) / (1 + v/c), A = A_z (1 - g) and B = B_z - L g, every operation
on pairs of FP32 numbers (an exact product from the FMA residual, Knuth's
two-sum), and stores B = bi + bf and A = a_hi + a_lo (a_hi of 11 significant
bits, so that j a_hi is exact in FP32). This test replays those operations
with NumPy float32 arithmetic (an FMA through exact rationals) for
velocities over +-900 km/s and two redshifts, and checks that the stored
record reproduces the FP64 t(j) to 2e-7 node units for every bin."""
from fractions import Fraction

import numpy as np

F32 = np.float32
C_KMS = 299792.458


def _fma(a, b, c):
    return F32(float(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))))


def _norm(hi, lo):
    s = F32(hi + lo)
    return s, F32(lo - F32(s - hi))


def _of(x):
    hi = F32(x)
    return hi, F32(x - float(hi))


def _add(a, b):
    s = F32(a[0] + b[0])
    z = F32(s - a[0])
    e = F32(F32(a[0] - F32(s - z)) + F32(b[0] - z))
    return _norm(s, F32(e + F32(a[1] + b[1])))


def _neg(a):
    return (F32(-a[0]), F32(-a[1]))


def _mul(a, b):
    p = F32(a[0] * b[0])
    e = _fma(a[0], b[0], -p)
    return _norm(p, _fma(a[0], b[1], _fma(a[1], b[0], e)))


def _mul_f(a, b):
    p = F32(a[0] * b)
    e = _fma(a[0], b, -p)
    return _norm(p, _fma(a[1], b, e))


def _record(v, l0, dl, ls0, dls, z):
    alpha_z = 1.0 / ((1.0 + z) * dls)
    Az, L = _of(dl * alpha_z), _of(l0 * alpha_z)
    Bz, invc = _of(l0 * alpha_z - ls0 / dls), _of(1.0 / C_KMS)
    b = _mul_f(invc, F32(v))
    q = _add((F32(1.0), F32(0.0)), b)
    g0 = F32(b[0] / q[0])
    res = _add(b, _neg(_mul_f(q, g0)))
    g = _norm(g0, F32(res[0] / q[0]))
    A = _add(Az, _neg(_mul(Az, g)))
    B = _add(Bz, _neg(_mul(L, g)))
    fb = np.floor(B[0])
    bi = int(fb)
    bf = F32(F32(B[0] - F32(fb)) + B[1])
    if bf < 0:
        bf = F32(bf + F32(1.0))
        bi -= 1
    a_hi = np.array([A[0]], np.float32).view(np.uint32) & np.uint32(~((1 << 13) - 1) & 0xFFFFFFFF)
    a_hi = a_hi.view(np.float32)[0]
    a_lo = F32(F32(A[0] - a_hi) + A[1])
    return bi, bf, a_hi, a_lo


def test_double_float_node_map_matches_fp64():
    rng = np.random.default_rng(0)
    ls0, dls = 4700.0, (9450.0 - 4700.0) / 3720
    l0, dl, n = 4750.0, 1.25, 3721
    j = np.arange(n, dtype=np.float64)
    worst = 0.0
    for z in (0.0, 0.02):
        for v in list(rng.uniform(-900.0, 900.0, 60)) + [0.0, 1e-3, -1e-3, 899.9]:
            v = float(np.float32(v))
            bi, bf, a_hi, a_lo = _record(v, l0, dl, ls0, dls, z)
            # 11 significant bits: j * a_hi exact in FP32 for j < 2^13
            assert float(F32(F32(n) * a_hi)) == float(n) * float(a_hi)
            t_rec = bi + float(bf) + j * float(a_hi) + j * float(a_lo)
            t_64 = ((l0 + j * dl) / ((1.0 + z) * (1.0 + v / C_KMS)) - ls0) / dls
            worst = max(worst, float(np.abs(t_rec - t_64).max()))
            assert 0.0 <= bf <= 1.0
    assert worst <= 2e-7, worst
