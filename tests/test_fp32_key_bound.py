"""The error bound behind the GPU's FP32 decision of spaxel keys (Sec. 3,
spaxel assignment).

The key reading is FP64 with every product and sum rounded once. The GPU
first evaluates the key coordinate u = (x' - x_lo) / size in FP32 (R and
x_lo rounded to FP32, x' by two FMAs after one product) and takes floor(u)
from it only when no integer lies within err = 2^-19 (mag + |est| + 1) of the
estimate, mag = (|R0 x| + |R1 y| + |R2 z| + |x_lo|) / size; otherwise it
evaluates the FP64 expression. That is exact if |est - u| stays below the
roundings' bound 2^-21 mag, which this test checks on random orientations,
positions over and beyond the fields used here and extreme magnitudes, with
NumPy's IEEE float32 arithmetic (an FMA emulated by an exact float64 product
and one float64 sum before the float32 rounding). It also checks, on the
same samples, that a decision made this way equals the FP64 key.
"""
import math

import numpy as np

import _edges


def _fma32(a, b, c):
    # a*b is exact in float64 for float32 a, b; the float64 sum rounds at
    # 2^-53, far below the float32 rounding that follows
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _fp32_estimate(R, x, y, z, x_lo, inv):
    f = np.float32
    Rf = [f(r) for r in R]
    xp = _fma32(np.full_like(x, Rf[2]), z, _fma32(np.full_like(x, Rf[1]), y, (Rf[0] * x).astype(np.float32)))
    est = ((xp - f(x_lo)) * f(inv)).astype(np.float32)
    mag = ((np.abs(Rf[0] * x) + np.abs(Rf[1] * y) + np.abs(Rf[2] * z) + abs(f(x_lo))) * f(inv)).astype(np.float32)
    return est, mag


def _fp64_coord(R, x, y, z, x_lo, inv):
    xp, _ = _edges.project(R, x, y, z)
    return (xp - x_lo) * inv


def test_fp32_key_estimate_within_bound_and_decisions_exact():
    rng = np.random.default_rng(11)
    worst = 0.0
    for trial in range(40):
        R = _edges.rotation(rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi), rng.uniform(-math.pi, math.pi))
        size = float(rng.choice([0.1, 0.2, 0.5, 0.3]))
        nx = int(rng.integers(20, 400))
        x_lo = (-0.5 * nx) * size
        inv = 1.0 / size
        scale = float(rng.choice([1.0, 10.0, 60.0, 1e3]))
        n = 20000
        x = (rng.standard_normal(n) * scale).astype(np.float32)
        y = (rng.standard_normal(n) * scale).astype(np.float32)
        z = (rng.standard_normal(n) * scale * 0.1).astype(np.float32)
        est, mag = _fp32_estimate(R, x, y, z, x_lo, inv)
        u = _fp64_coord(R, x, y, z, x_lo, inv)
        ratio = np.abs(est.astype(np.float64) - u) / (mag.astype(np.float64) * 2.0 ** -21)
        worst = max(worst, float(ratio.max()))
        # the decision rule of the kernel, in float32 as there
        err = (np.float32(2.0 ** -19) * (mag + np.abs(est) + np.float32(1.0))).astype(np.float32)
        lo = np.floor((est - err).astype(np.float32))
        hi = np.floor((est + err).astype(np.float32))
        decided = lo == hi
        assert np.array_equal(lo[decided], np.floor(u[decided])), trial
        if scale <= 60.0:  # fields and galaxies of the workloads here: the FP64 fallback stays rare
            assert decided.mean() > 0.99, (trial, scale, decided.mean())
    assert worst <= 1.0, worst


def test_fp32_key_decisions_on_near_edge_particles():
    """Particles placed within a few FP64 ulps of spaxel edges: every one the
    FP32 rule decides gets the FP64 key, and (being that close) almost all
    fall back to FP64."""
    from paper_2412_08265_gb300 import synth
    tel = synth.serving_telescope(57)
    size = tel.spaxel_size
    x_lo = (-0.5 * tel.nx) * size
    inv = 1.0 / size
    R = _edges.rotation(0.83, 0.0, 0.61)
    rng = np.random.default_rng(3)
    xs, ys, zs = [], [], []
    for k in rng.integers(1, tel.nx - 1, 40):
        target = _edges.crossing(x_lo, inv, size, int(k))
        x = np.float32(target * R[0])
        y = np.float32(target * R[1])
        for dz in (0.0, 1e-12, -1e-12):
            xs.append(x)
            ys.append(y)
            zs.append(np.float32(dz))
    x, y, z = (np.array(a, np.float32) for a in (xs, ys, zs))
    est, mag = _fp32_estimate(R, x, y, z, x_lo, inv)
    u = _fp64_coord(R, x, y, z, x_lo, inv)
    err = (np.float32(2.0 ** -19) * (mag + np.abs(est) + np.float32(1.0))).astype(np.float32)
    lo = np.floor((est - err).astype(np.float32))
    hi = np.floor((est + err).astype(np.float32))
    decided = lo == hi
    assert np.array_equal(lo[decided], np.floor(u[decided]))
    near = np.abs(u - np.round(u)) < 1e-6
    assert not decided[near].any()
