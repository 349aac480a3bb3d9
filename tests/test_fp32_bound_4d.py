"""The error bound behind the 4D percolation's FP32 tests, on the host.

The CUDA path decides the percolation in FP32 where a rigorous bound e_a on
|xi_a(FP32) - x_a(FP64)| settles the decision, x_a = (Q_a - Q_m,a)/dm_a being
the FP64 inverse map in the fixed order of the exact test.  This test
restates the FP32 record (A, B, K and the row norms nA, nB) and the FP32
evaluation with its bound, emulating each fused multiply-add as an exact
product and sum rounded once to FP32, and checks the bound against the
oracle's FP64 evaluation (the one the exact test reproduces) on random,
strongly distorted elements and offsets, including offsets far outside an
element's own cell.  No GPU.
"""
import numpy as np
import pytest

import oracle.oracle4d as Q

f32 = np.float32


def fmaf(a, b, c):
    """fmaf(a, b, c): exact a*b + c rounded once to FP32 (the product of two
    FP32 values is exact in FP64; the FP64 sum's own rounding is below the
    FP32 ulp by far)."""
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def sym(b, c):
    if b > c:
        b, c = c, b
    return 4 * b - (b * (b - 1)) // 2 + (c - b)


def record(t, dm):
    """FP32 record of a Taylor record t (64 doubles): A[16], B[40], K[4], nA[4], nB[4]."""
    Ti = t[4:20].reshape(4, 4)
    G = t[20:60].reshape(4, 10)
    r = np.zeros(72, dtype=f32)
    inv_dm = 1.0 / dm
    for a in range(4):
        for b in range(4):
            r[4 * a + b] = f32(Ti[a, b] * dm[b] * inv_dm[a])
        kmax = 0.0
        for l in range(4):
            gm = 0.0
            for b in range(4):
                for c in range(b, 4):
                    gm = max(gm, abs(G[l, sym(b, c)]) * dm[b] * dm[c])
            kmax += abs(Ti[a, l]) * gm
        r[56 + a] = f32(0.5 * kmax * inv_dm[a] * 1.0000001)
        for b in range(4):
            for c in range(b, 4):
                v = sum(Ti[a, l] * G[l, sym(b, c)] for l in range(4))
                r[16 + 10 * a + sym(b, c)] = f32(-0.5 * (1.0 if b == c else 2.0) * v * dm[b] * dm[c] * inv_dm[a])
    for a in range(4):
        na = f32(0)
        nb = f32(0)
        for b in range(4):
            na = f32(na + abs(r[4 * a + b]))
        for q in range(10):
            nb = f32(nb + abs(r[16 + 10 * a + q]))
        r[60 + a] = f32(na * f32(1.000001))
        r[64 + a] = f32(nb * f32(1.000001))
    return r


def eval32(R, p, dp):
    """xi (FP32) and its bound e, in the device's order."""
    kRel, kAbs = f32(2.0e-6), f32(1.0e-9)
    pm = max(abs(p[0]), abs(p[1]), abs(p[2]), abs(p[3]))
    dm = max(dp)
    dpp = fmaf(f32(2) * pm, dm, f32(dm * dm))
    S = f32(4) * pm
    pp = np.zeros(10, dtype=f32)
    for b in range(4):
        for c in range(b, 4):
            pp[sym(b, c)] = f32(p[b] * p[c])
    xi = np.zeros(4, dtype=f32)
    e = np.zeros(4, dtype=f32)
    for a in range(4):
        v = f32(0)
        for b in range(4):
            v = fmaf(R[4 * a + b], p[b], v)
        for q in range(10):
            v = fmaf(R[16 + 10 * a + q], pp[q], v)
        xi[a] = v
        nA, nB = R[60 + a], R[64 + a]
        E = fmaf(nB, f32(pm * pm), f32(nA * pm))
        Ep = fmaf(nB, dpp, f32(nA * dm))
        e[a] = f32(f32(f32(kRel * E) + f32(kAbs * f32(1 + E))) + f32(f32(1.00001) * Ep)) + \
            f32(f32(f32(1e-13) * R[56 + a]) * f32(S * S)) * f32(16)
    return xi, e


def d2_32(xi, e):
    d2 = f32(0)
    b = f32(0)
    for a in range(4):
        d2 = fmaf(xi[a], xi[a], d2)
        b = fmaf(e[a], f32(f32(2) * abs(xi[a])) + e[a], b)
    return d2, f32(b + f32(6e-7) * d2) + f32(1e-30)


@pytest.mark.parametrize("scale", [0.05, 0.3, 1.0])
def test_fp32_offsets_and_distances_stay_within_their_bounds(scale):
    rng = np.random.default_rng(int(scale * 1000))
    dm = np.array([0.13, 0.11, 0.19, 0.21])
    worst = 0.0
    for _ in range(60):
        T = np.eye(4) + scale * rng.normal(size=(4, 4))
        if abs(np.linalg.det(T)) < 0.05:
            continue
        H = scale * 3.0 * rng.normal(size=40)
        Pm = rng.normal(size=4)
        el = np.concatenate([Pm, T.ravel(), H])
        t = Q.taylor_one(el, rng.normal(size=4))
        R = record(t, dm)
        d = dm / 4.0                       # grid spacing, element stride 4
        h = np.array([f32(d[b] * (1.0 / dm[b])) for b in range(4)], dtype=f32)
        Pst = Pm + d * rng.integers(-6, 7, size=4) + d * rng.uniform(-0.5, 0.5, size=4)
        for k in range(20):
            if k % 2 == 0:
                # the resample's form: p from the FP64 offset, rounded once
                P = Pm + dm * rng.uniform(-3.0, 3.0, size=4)
                dP = P - t[:4]
                p = np.array([f32(f32(dP[b]) * f32(1.0 / dm[b])) for b in range(4)], dtype=f32)
                dp = np.array([f32(1.8e-7) * abs(p[b]) + f32(1e-12) for b in range(4)], dtype=f32)
            else:
                # the percolation's form: p = j h + r from the integer offset j
                # of the site from a reference site and the FP32 offset r of it
                j = rng.integers(-12, 13, size=4)
                P = Pst + j * d
                r = np.array([f32((Pst[b] - t[b]) * (1.0 / dm[b])) for b in range(4)], dtype=f32)
                jh = np.array([f32(f32(j[b]) * h[b]) for b in range(4)], dtype=f32)
                p = np.array([f32(jh[b] + r[b]) for b in range(4)], dtype=f32)
                dp = np.array([f32(f32(6.0e-8) * f32(abs(r[b]) + f32(2) * abs(jh[b]) + abs(p[b]))) + f32(1e-12)
                               for b in range(4)], dtype=f32)
            xi, e = eval32(R, p, dp)
            x64 = Q.qofp(t, P) * (1.0 / dm)
            err = np.abs(xi.astype(np.float64) - x64)
            assert (err <= e.astype(np.float64)).all(), (err, e)
            worst = max(worst, float((err / e).max()))
            d2, bd = d2_32(xi, e)
            d64 = float(np.sum(x64 * x64))
            assert abs(float(d2) - d64) <= float(bd), (d2, d64, bd)
    # the bound is not vacuous: the observed error reaches a fair part of it
    assert 1e-4 < worst < 1.0, worst
