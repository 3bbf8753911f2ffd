"""Oracle pins for the higher-order interpolation schemes (Sec. "Interpolation
schemes": triquadratic and tricubic kernels of the cited methods), from
properties of the kernels rather than their formulas: interpolation at the
vertices, reproduction of polynomials (linear for both, quadratic for the
cubic kernel), C1 continuity of the cubic interpolant across cell faces,
analytic gradients equal to differences of the interpolant, and the order of
convergence under grid refinement; then the tracer's Q and L converge faster
with the cubic kernel than with the trilinear one."""
import numpy as np
import pytest

from paper_1609_00724_gb300 import inputs


def grid_field(oracle_mod, fn, n, order, mode=1, box=((-1.0, 1.0), (-1.0, 1.0), (0.0, 1.0))):
    ax = [np.linspace(lo, hi, n) for lo, hi in box]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    bx, by, bz = fn(X, Y, Z)
    return oracle_mod.Field(bx, by, bz, ax[0], ax[1], ax[2], mode=mode, order=order), ax


def quad(X, Y, Z):
    return (0.3 + 0.2 * X - 0.1 * Y + 0.4 * X * Y - 0.25 * Y ** 2,
            -0.2 + 0.5 * Z + 0.3 * X ** 2 - 0.2 * Y * Z,
            1.0 + 0.1 * X + 0.2 * Y + 0.3 * Z ** 2)


def lin(X, Y, Z):
    return 0.3 + 0.2 * X - 0.1 * Y + 0.5 * Z, -0.2 + 0.5 * Z + 0.3 * X, 1.0 + 0.1 * X + 0.2 * Y - 0.3 * Z


def interior_points(n_pts, seed, margin=0.25):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0, 1, size=(n_pts, 3))
    lo = np.array([-1 + margin, -1 + margin, margin / 2])
    hi = np.array([1 - margin, 1 - margin, 1 - margin / 2])
    return lo + p * (hi - lo)


def test_orders_validated(oracle_mod):
    with pytest.raises(ValueError):
        grid_field(oracle_mod, lin, 9, 4)
    ax = np.array([0.0, 0.1, 0.3, 0.6, 1.0])  # non-uniform: higher orders refused
    b = np.ones((5, 5, 5))
    with pytest.raises(ValueError):
        oracle_mod.Field(b, b, b, ax, ax, ax, mode=1, order=3)


@pytest.mark.parametrize("order", [2, 3])
def test_interpolation_at_vertices_and_linear_reproduction(oracle_mod, order):
    F, ax = grid_field(oracle_mod, quad, 17, order)
    # at interior vertices the interpolant equals the sample (raw mode: B itself)
    for i, j, k in [(3, 5, 7), (8, 8, 8), (11, 2, 13)]:
        x = np.array([ax[0][i], ax[1][j], ax[2][k]])
        b, _, m = F.interp(x)
        want = np.array(quad(*x))
        assert np.allclose(b * m, want, rtol=0, atol=1e-12)
    F1, _ = grid_field(oracle_mod, lin, 17, order)
    for x in interior_points(40, order):
        b, g, m = F1.interp(x)
        want = np.array(lin(*x))
        assert np.allclose(b * m, want, rtol=0, atol=1e-12)


def test_cubic_reproduces_quadratics_and_quadratic_kernel_does_not(oracle_mod):
    F3, _ = grid_field(oracle_mod, quad, 17, 3)
    F2, _ = grid_field(oracle_mod, quad, 17, 2)
    F1, _ = grid_field(oracle_mod, quad, 17, 1)
    e3 = e2 = e1 = 0.0
    for x in interior_points(60, 3):
        want = np.array(quad(*x))
        e3 = max(e3, np.abs(F3.interp(x)[0] * F3.interp(x)[2] - want).max())
        e2 = max(e2, np.abs(F2.interp(x)[0] * F2.interp(x)[2] - want).max())
        e1 = max(e1, np.abs(F1.interp(x)[0] * F1.interp(x)[2] - want).max())
    assert e3 < 1e-12
    assert e2 > 1e-6 and e1 > 1e-6


def test_cubic_interpolant_is_c1_across_cell_faces(oracle_mod):
    """Paper mode (the interpolated normalised field is used as is): value and
    gradient of the cubic interpolant are continuous across a cell face."""
    F, ax = grid_field(oracle_mod, lambda X, Y, Z: (np.sin(2 * X) + Y, np.cos(3 * Y) * Z + 1.5, 2 + X * Z), 13, 3,
                       mode=0)
    xf = ax[0][6]
    for eps in (1e-7,):
        a = F.interp(np.array([xf - eps, 0.13, 0.41]))
        b = F.interp(np.array([xf + eps, 0.13, 0.41]))
        assert np.allclose(a[0], b[0], atol=1e-6)
        assert np.allclose(a[1], b[1], atol=1e-5)
    F1, _ = grid_field(oracle_mod, lambda X, Y, Z: (np.sin(2 * X) + Y, np.cos(3 * Y) * Z + 1.5, 2 + X * Z), 13, 1,
                       mode=0)
    a = F1.interp(np.array([xf - 1e-7, 0.13, 0.41]))
    b = F1.interp(np.array([xf + 1e-7, 0.13, 0.41]))
    assert np.abs(a[1] - b[1]).max() > 1e-3  # the trilinear gradient jumps there


@pytest.mark.parametrize("order", [2, 3])
def test_gradient_is_the_derivative_of_the_interpolant(oracle_mod, order):
    F, _ = grid_field(oracle_mod, lambda X, Y, Z: (np.sin(2 * X) + Y, np.cos(3 * Y) * Z + 1.5, 2 + X * Z), 13, order,
                      mode=0)
    h = 1e-6
    for x in interior_points(20, 10 + order):
        _, g, _ = F.interp(x)
        for j in range(3):
            d = np.zeros(3)
            d[j] = h
            fd = (F.interp(x + d)[0] - F.interp(x - d)[0]) / (2 * h)
            # the quadratic kernel's derivative jumps at mid-cell: skip points near it
            assert np.allclose(g[:, j], fd, atol=1e-5) or order == 2 and _near_mid(x, j)


def _near_mid(x, j, n=13):
    box = ((-1.0, 1.0), (-1.0, 1.0), (0.0, 1.0))[j]
    u = (x[j] - box[0]) / (box[1] - box[0]) * (n - 1)
    return abs((u % 1.0) - 0.5) < 1e-5


def test_convergence_orders(oracle_mod):
    """RMS interpolation error of a smooth field over 300 fixed interior points
    falls by about 2^2 per grid doubling for the trilinear and quadratic
    kernels and by about 2^3 for the cubic one."""
    fn = lambda X, Y, Z: (np.sin(2 * X) * np.cos(Y), np.cos(3 * Y) * Z + 1.5, np.exp(0.5 * X) * (1 + Z ** 2))
    pts = interior_points(300, 21)
    ratios = {}
    for order in (1, 2, 3):
        errs = []
        for n in (33, 65):
            F, _ = grid_field(oracle_mod, fn, n, order)
            e = [np.abs(F.interp(x)[0] * F.interp(x)[2] - np.array(fn(*x))).max() for x in pts]
            errs.append(np.sqrt(np.mean(np.square(e))))
        ratios[order] = errs[0] / errs[1]
    assert 3.5 < ratios[1] < 4.6, ratios
    assert 3.5 < ratios[2] < 4.6, ratios
    assert 7.0 < ratios[3] < 9.5, ratios


def test_tracer_converges_faster_with_the_cubic_kernel(oracle_mod):
    """Q_perp and L of charge-field lines against a 129^3 cubic reference: at
    33^3 the cubic kernel's length error is well below the trilinear one (third
    against second order) and its Q error below it (Q uses the gradient, one
    order lower for both)."""
    import torch
    ch = inputs.random_charges(2, 21)
    seeds = inputs.random_seeds(40, 5, margin=0.1)

    def field(n, order):
        gf = inputs.to_numpy64(inputs.charge_field(ch, n, dtype=torch.float64))
        return oracle_mod.Field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, mode=1, order=order)

    o = oracle_mod.default_opts(tol_abs=1e-10, tol_rel=1e-10)
    ref = oracle_mod.trace_seeds(field(129, 3), seeds, o)
    err = {}
    for order in (1, 3):
        r = oracle_mod.trace_seeds(field(33, order), seeds, o)
        ok = (r["face_f"] == ref["face_f"]) & (r["face_b"] == ref["face_b"]) & np.isfinite(ref["q_perp"])
        assert ok.sum() >= 30
        err[order] = (np.median(np.abs(r["q_perp"][ok] / ref["q_perp"][ok] - 1)),
                      np.median(np.abs(r["L"][ok] / ref["L"][ok] - 1)))
    assert err[3][1] < 0.3 * err[1][1] and err[3][0] < 0.7 * err[1][0], err
