"""Oracle pins for the building blocks: the Cash-Karp stepper (order test), the
interpolant's analytic gradient, the Hilbert curve, the Sobel FLEDGE operator
and the Hilbert -> rectilinear converter (Sec. "Adaptive refinements")."""
import math

import numpy as np
import pytest

from paper_1609_00724_gb300 import inputs


# ---------------------------------------------------------------- Cash-Karp
def _integrate(oracle_mod, M, y0, T, N):
    y = np.array(y0, dtype=float)
    h = T / N
    for _ in range(N):
        y, _ = oracle_mod.ck_linear_step(M, y, h)
    return y


@pytest.mark.parametrize("M,y0,exact", [
    (np.array([[1.0]]), [1.0], lambda T: np.array([math.exp(T)])),
    (np.array([[0.0, 1.0], [-1.0, 0.0]]), [1.0, 0.0], lambda T: np.array([math.cos(T), -math.sin(T)])),
])
def test_cash_karp_is_fifth_order(oracle_mod, M, y0, exact):
    T = 2.0
    errs = [np.abs(_integrate(oracle_mod, M, y0, T, N) - exact(T)).max() for N in (8, 16, 32)]
    for a, b in zip(errs, errs[1:]):
        assert 28 < a / b < 36, errs  # 2^5 = 32


def test_cash_karp_error_estimate_is_fourth_order_local(oracle_mod):
    """The embedded error estimate of one step scales as h^5 (a 4th-order
    method's local error)."""
    M = np.array([[0.0, 1.0], [-1.0, 0.0]])
    est = [np.abs(oracle_mod.ck_linear_step(M, [1.0, 0.0], h)[1]).max() for h in (0.2, 0.1, 0.05)]
    for a, b in zip(est, est[1:]):
        assert 28 < a / b < 36, est


# ------------------------------------------------------- interpolant gradient
@pytest.mark.parametrize("mode", [0, 1])
def test_analytic_gradient_matches_central_differences(oracle_mod, mode):
    """Inside a cell the interpolant is smooth; its analytic gradient (the
    gradient acting on the kernels f_v) must match central differences."""
    import torch
    ch = inputs.random_charges(4, 2, depth=(0.15, 0.3))
    gf = inputs.to_numpy64(inputs.charge_field(ch, (9, 11, 7), dtype=torch.float64))
    # a rectilinear (non-uniform) grid: stretch the x axis
    xc = np.sign(gf.xc) * np.abs(gf.xc) ** 1.3
    F = oracle_mod.Field(gf.bx, gf.by, gf.bz, xc, gf.yc, gf.zc, mode=mode)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(50):
        # pick a point well inside a random cell
        i, j, k = rng.integers(0, 8), rng.integers(0, 10), rng.integers(0, 6)
        f = rng.uniform(0.2, 0.8, 3)
        x = np.array([xc[i] + f[0] * (xc[i + 1] - xc[i]), gf.yc[j] + f[1] * (gf.yc[j + 1] - gf.yc[j]),
                      gf.zc[k] + f[2] * (gf.zc[k + 1] - gf.zc[k])])
        b, g, _ = F.interp(x)
        for jj in range(3):
            e = np.zeros(3)
            e[jj] = h
            bp, _, _ = F.interp(x + e)
            bm, _, _ = F.interp(x - e)
            fd = (bp - bm) / (2 * h)
            assert np.allclose(g[:, jj], fd, rtol=1e-6, atol=1e-6 * (1 + np.abs(g).max()))


def test_paper_mode_vertex_values_are_unit(oracle_mod):
    import torch
    ch = inputs.random_charges(2, 9)
    gf = inputs.to_numpy64(inputs.charge_field(ch, 6, dtype=torch.float64))
    F = oracle_mod.Field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, mode=0)
    for (i, j, k) in [(0, 0, 0), (3, 2, 5), (5, 5, 0)]:
        b, _, m = F.interp(np.array([gf.xc[i], gf.yc[j], gf.zc[k]]))
        B = np.array([gf.bx[k, j, i], gf.by[k, j, i], gf.bz[k, j, i]])
        assert abs(np.linalg.norm(b) - 1) < 1e-14
        assert np.allclose(b, B / np.linalg.norm(B), atol=1e-14)
        assert abs(m - np.linalg.norm(B)) < 1e-12 * np.linalg.norm(B)


# ----------------------------------------------------------------- Hilbert
@pytest.mark.parametrize("ndim,bits", [(2, 1), (2, 2), (2, 5), (2, 7), (3, 1), (3, 2), (3, 4)])
def test_hilbert_bijection_adjacency_blocks(oracle_mod, ndim, bits):
    n = 1 << (ndim * bits)
    pts = [oracle_mod.hilbert_coords(k, ndim, bits) for k in range(n)]
    assert pts[0] == (0,) * ndim  # starts at the origin
    assert len(set(pts)) == n  # bijection onto the lattice
    for c in pts:
        assert all(0 <= v < (1 << bits) for v in c)
    for k in range(0, n, max(1, n // 200)):
        assert oracle_mod.hilbert_key(pts[k], ndim, bits) == k
    # successive cells are lattice neighbours
    for a, b in zip(pts, pts[1:]):
        assert sum(abs(x - y) for x, y in zip(a, b)) == 1
    # every aligned 2^l block is a contiguous key range (what the converter uses)
    for lev in range(1, bits):
        blk = 1 << (ndim * lev)
        for k0 in range(0, n, blk):
            cells = {tuple(v >> lev for v in pts[k]) for k in range(k0, k0 + blk)}
            assert len(cells) == 1


def test_hilbert_large_order_roundtrip(oracle_mod):
    rng = np.random.default_rng(3)
    for ndim, bits in ((2, 13), (3, 11), (3, 21)):
        for _ in range(200):
            c = tuple(int(v) for v in rng.integers(0, 1 << bits, ndim))
            k = oracle_mod.hilbert_key(c, ndim, bits)
            assert k < (1 << (ndim * bits))
            assert oracle_mod.hilbert_coords(k, ndim, bits) == c


# ------------------------------------------------------------------- Sobel
def test_sobel_ramp_2d(oracle_mod):
    a, b = 0.3, -1.7
    I, J = np.meshgrid(np.arange(20), np.arange(30), indexing="ij")
    L = (a * I + b * J).astype(np.float32)
    S = oracle_mod.fledge(L)
    # interior: d/di = (1+2+1) * 2a = 8a
    assert np.allclose(S[1:-1, 1:-1], 8 * math.hypot(a, b), rtol=1e-6)
    # reflect boundary at i = 0: difference L(1) - L(0) = a, so 4a along that axis
    assert np.allclose(S[0, 1:-1], math.hypot(4 * a, 8 * b), rtol=1e-6)
    assert np.allclose(S[0, 0], math.hypot(4 * a, 4 * b), rtol=1e-6)


def test_sobel_ramp_3d_and_nan_fill(oracle_mod):
    a, b, c = 0.5, 0.25, -2.0
    I, J, K = np.meshgrid(np.arange(9), np.arange(10), np.arange(11), indexing="ij")
    L = (a * I + b * J + c * K).astype(np.float32)
    S = oracle_mod.fledge(L)
    assert np.allclose(S[1:-1, 1:-1, 1:-1], 32 * math.sqrt(a * a + b * b + c * c), rtol=1e-6)
    # a NaN (skipped line) is replaced by the largest finite length of the map
    L2 = np.zeros((5, 6), dtype=np.float32)
    L2[2, 3] = 2.0
    L2[0, 0] = np.nan
    S2 = oracle_mod.fledge(L2)
    L3 = L2.copy()
    L3[0, 0] = 2.0
    assert np.array_equal(S2, oracle_mod.fledge(L3))
    assert S2[2, 3] == 0.0  # symmetric neighbourhood of a single spike


# --------------------------------------------------------------- converter
def test_converter_max_and_log_interpolation(oracle_mod):
    ndim, p = 2, 3
    ext = (8, 8, 0)
    key_of = lambda x, y: oracle_mod.hilbert_key((x, y), ndim, p)
    # two samples in the same output cell at out_order 2 -> maximum wins
    k1, k2 = key_of(0, 0), key_of(1, 0)
    k3 = key_of(7, 0)  # last cell of the curve? (its key is whatever the curve gives)
    keys = np.array(sorted([k1, k2, k3]), dtype=np.uint64)
    vals = {k1: 10.0, k2: 1000.0, k3: 1e5}
    v = np.array([vals[int(k)] for k in keys])
    out = oracle_mod.convert(keys, v, ndim, p, ext, 2, True)
    assert out.shape == (4, 4)
    assert out[0, 0] == 1000.0
    # an empty output cell between keys k2 and k3 on the curve: log10 interpolation
    blk = 4
    for oy in range(4):
        for ox in range(4):
            if (ox, oy) in ((0, 0), (3, 0)):
                continue
            k0 = (key_of(2 * ox, 2 * oy) // blk) * blk
            kc = k0 + 0.5 * (blk - 1)
            ks = [int(k) for k in keys]
            pred = max([k for k in ks if k < k0], default=None)
            succ = min([k for k in ks if k >= k0 + blk], default=None)
            if pred is None:
                exp = vals[succ]
            elif succ is None:
                exp = vals[pred]
            else:
                t = (kc - pred) / (succ - pred)
                exp = 10 ** ((1 - t) * math.log10(vals[pred]) + t * math.log10(vals[succ]))
            assert abs(out[oy, ox] / exp - 1) < 1e-12, (ox, oy)
    # identity at full order: every sampled cell keeps its value
    out3 = oracle_mod.convert(keys, v, ndim, p, ext, 3, False)
    assert out3[0, 0] == 10.0 and out3[0, 1] == 1000.0 and out3[0, 7] == 1e5
