"""Test inputs: 3-D particles whose rotated coordinates sit within a few FP64
ulps of a spaxel edge (spaxel assignment, Sec. 3).

The orientation reading (R = Rz(q) Rx(i) Rz(a), every product and sum of the
matrix elements and of x' = (R00 x + R01 y) + R02 z rounded once in FP64)
fixes the key of a particle bit for bit. A particle whose x' lies within an
ulp of an edge changes spaxel if any element of R, or any rounding of the
projection, differs by one ulp -- so a GPU path whose host builds R with a
fused multiply-add, or in another order, fails a bitwise key comparison on
these particles, while ordinary random particles (about 1e-7 kpc from the
nearest edge at best) cannot tell.

Construction: x and y are float32 values near the rotated-back target; among
their float32 neighbours the pair whose S = fl(R00 x) + fl(R01 y) comes
closest to E leaves a residual of order 1e-11, which the small z then
cancels: fl(R02 z) for such a z moves in steps far below an ulp of x', so
x' can be placed on E or a few ulps from it.

Python floats and NumPy float64 arrays round every operation (no
contraction), so `project` below is the same arithmetic as the reading.
"""
from __future__ import annotations

import math

import numpy as np


def rotation(incl: float, azim: float, pa: float):
    ca, sa, ci, si = math.cos(azim), math.sin(azim), math.cos(incl), math.sin(incl)
    cq, sq = math.cos(pa), math.sin(pa)
    return [cq * ca - sq * (ci * sa), -(cq * sa) - sq * (ci * ca), sq * si,
            sq * ca + cq * (ci * sa), cq * (ci * ca) - sq * sa, -(cq * si),
            si * sa, si * ca, ci]


def project(R, x, y, z):
    x = np.asarray(x, np.float32).astype(np.float64)
    y = np.asarray(y, np.float32).astype(np.float64)
    z = np.asarray(z, np.float32).astype(np.float64)
    xp = (R[0] * x + R[1] * y) + R[2] * z
    yp = (R[3] * x + R[4] * y) + R[5] * z
    return xp, yp


def keys(xp, yp, tel):
    size = tel.spaxel_size
    x_lo = (-0.5 * tel.nx) * size
    y_lo = (-0.5 * tel.ny) * size
    inv = 1.0 / size
    ix = np.floor((np.asarray(xp) - x_lo) * inv)
    iy = np.floor((np.asarray(yp) - y_lo) * inv)
    ok = (ix >= 0) & (ix < tel.nx) & (iy >= 0) & (iy < tel.ny)
    k = (iy * tel.nx + ix).astype(np.int64)
    return np.where(ok, k, tel.nx * tel.ny).astype(np.int32)


def crossing(lo: float, inv: float, size: float, k: int) -> float:
    """Smallest double c with floor((c - lo) * inv) >= k (the key's edge k)."""
    c = lo + k * size
    f = lambda v: math.floor((v - lo) * inv) >= k
    if f(c):
        while f(math.nextafter(c, -math.inf)):
            c = math.nextafter(c, -math.inf)
    else:
        while not f(c):
            c = math.nextafter(c, math.inf)
    return c


def near_edge_particles(tel, incl: float, azim: float, pa: float, n_edges: int = 48, seed: int = 0,
                        ulps: int = 3):
    """float32 (x, y, z) arrays of particles whose x' (first half of the edges)
    or y' (second half) lies within `ulps` FP64 ulps of an interior spaxel
    edge, with the other coordinate inside the field. Needs R02, R12 != 0
    (an inclined galaxy with a position angle off 0 and pi/2) and the
    in-plane block [[R00, R01], [R10, R11]] invertible (not edge-on)."""
    R = rotation(incl, azim, pa)
    if abs(R[2]) < 1e-3 or abs(R[5]) < 1e-3:
        raise ValueError("angles give R02 or R12 near 0")
    rng = np.random.default_rng(seed)
    size = tel.spaxel_size
    inv = 1.0 / size
    lo = {0: (-0.5 * tel.nx) * size, 1: (-0.5 * tel.ny) * size}
    nn = {0: tel.nx, 1: tel.ny}
    xs, ys, zs = [], [], []
    M2 = np.array([[R[0], R[1]], [R[3], R[4]]])
    for e in range(n_edges):
        axis = 0 if e < n_edges // 2 else 1
        k = int(rng.integers(1, nn[axis]))
        E = crossing(lo[axis], inv, size, k)
        other = 1 - axis
        o = lo[other] + (rng.uniform(0.1, 0.9) * nn[other]) * size
        tgt = np.zeros(2)
        tgt[axis] = E
        tgt[other] = o
        # (x, y) with z = 0 that project onto the target
        r = np.linalg.solve(M2, tgt)
        x32, y32 = np.float32(r[0]), np.float32(r[1])
        a0, a1, a2 = (R[0], R[1], R[2]) if axis == 0 else (R[3], R[4], R[5])
        # float32 neighbours of (x, y) whose S = fl(a0 x) + fl(a1 y) comes closest to E
        steps = np.arange(-96, 97, dtype=np.int32)
        xc = (np.array(x32).view(np.int32) + steps).view(np.float32).astype(np.float64)
        yc = (np.array(y32).view(np.int32) + steps).view(np.float32).astype(np.float64)
        S = (a0 * xc)[:, None] + (a1 * yc)[None, :]
        best = np.argsort(np.abs(S - E), axis=None)[:4]
        for b in best:
            i, j = np.unravel_index(b, S.shape)
            Sij = float(S[i, j])
            z = np.float32((E - Sij) / a2)
            cands = [z]
            up, dn = z, z
            for _ in range(8):
                up = np.nextafter(up, np.float32(np.inf))
                dn = np.nextafter(dn, np.float32(-np.inf))
                cands += [up, dn]
            for zc in cands:
                v = Sij + a2 * float(zc)
                if abs(v - E) <= ulps * math.ulp(E):
                    xs.append(np.float32(xc[i]))
                    ys.append(np.float32(yc[j]))
                    zs.append(zc)
    x = np.array(xs, np.float32)
    y = np.array(ys, np.float32)
    z = np.array(zs, np.float32)
    xp, yp = project(R, x, y, z)
    inside = (keys(xp, yp, tel) < tel.nx * tel.ny)
    return x[inside], y[inside], z[inside]


def perturbed(R, i: int, direction: float):
    Rp = list(R)
    Rp[i] = math.nextafter(Rp[i], direction)
    return Rp
