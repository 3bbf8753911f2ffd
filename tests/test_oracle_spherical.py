"""Oracle pins for spherical geometry (Sec. "Integrating field lines",
Eq. fl_sph; Sec. "Field-line deviation using linearization", Eq. dev_sph):
axes (phi, theta, r) = longitude, latitude (radians) and radius, field
components in the local orthonormal basis (phi^, theta^, r^)."""
import numpy as np
import pytest

PHI, TH, R = (-0.4, 0.4), (-0.3, 0.3), (1.0, 1.5)


def sph_field(oracle_mod, fn, n=(33, 33, 33), box=(PHI, TH, R), mode=1, order=1):
    ax = [np.linspace(lo, hi, k) for (lo, hi), k in zip(box, n)]
    T, Th, Ph = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")  # [r, theta, phi] = [z, y, x]
    bp, bt, br = fn(Ph, Th, T)
    return oracle_mod.Field(bp, bt, br, ax[0], ax[1], ax[2], mode=mode, order=order, geometry=1)


def test_geometry_validated(oracle_mod):
    with pytest.raises(ValueError):
        sph_field(oracle_mod, lambda p, t, r: (0 * r, 0 * r, 1 + 0 * r), box=(PHI, (-1.6, 0.3), R))
    with pytest.raises(ValueError):
        sph_field(oracle_mod, lambda p, t, r: (0 * r, 0 * r, 1 + 0 * r), box=(PHI, TH, (-0.5, 1.0)))


def test_monopole_lines_are_radial_with_q_two(oracle_mod):
    """B = r^/r^2: lines keep (phi, theta), run from r = 1 to r = 1.5 (L = 0.5),
    and neighbouring lines separate in proportion to r in both transverse
    directions, so Q_det = 2 exactly; Q_perp = 2 and zero flux residuals hold
    up to the trilinear interpolation error of |B| = 1/r^2."""
    F = sph_field(oracle_mod, lambda p, t, r: (0 * r, 0 * r, 1.0 / r ** 2))
    rng = np.random.default_rng(3)
    seeds = np.column_stack([rng.uniform(-0.3, 0.3, 20), rng.uniform(-0.25, 0.25, 20), rng.uniform(1.05, 1.45, 20)])
    r = oracle_mod.trace_seeds(F, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    assert np.all(r["face_f"] == 5) and np.all(r["face_b"] == 4)
    assert np.allclose(r["xf"][:, :2], seeds[:, :2], atol=1e-10) and np.allclose(r["xf"][:, 2], 1.5, atol=1e-12)
    assert np.allclose(r["xb"][:, :2], seeds[:, :2], atol=1e-10) and np.allclose(r["xb"][:, 2], 1.0, atol=1e-12)
    assert np.allclose(r["L"], 0.5, rtol=1e-10)
    assert np.allclose(r["q_det"], 2.0, rtol=1e-8)
    assert np.allclose(r["q_perp"], 2.0, rtol=1e-3)
    assert np.allclose(r["flux"], 0.0, atol=1e-3) and np.allclose(r["flux_b"], 0.0, atol=1e-3)


def test_twisted_field_closed_form(oracle_mod):
    """B = (Omega r, 0, 1) (linear in r, so interpolated exactly): at fixed
    latitude theta0 the longitude advances as phi = phi0 + Omega (r - r0) /
    cos(theta0) (Eq. fl_sph), and the length is the integral of
    sqrt(1 + (Omega r)^2) dr."""
    om = 0.3
    F = sph_field(oracle_mod, lambda p, t, r: (om * r, 0 * r, 1 + 0 * r))
    rng = np.random.default_rng(5)
    seeds = np.column_stack([rng.uniform(-0.2, 0.2, 20), rng.uniform(-0.25, 0.25, 20), rng.uniform(1.05, 1.45, 20)])
    r = oracle_mod.trace_seeds(F, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    assert np.all(r["face_f"] == 5) and np.all(r["face_b"] == 4)

    def prim(rr):  # antiderivative of sqrt(1 + om^2 r^2)
        return 0.5 * (rr * np.sqrt(1 + (om * rr) ** 2) + np.arcsinh(om * rr) / om)

    ct = np.cos(seeds[:, 1])
    assert np.allclose(r["xf"][:, 0], seeds[:, 0] + om * (1.5 - seeds[:, 2]) / ct, atol=1e-9)
    assert np.allclose(r["xb"][:, 0], seeds[:, 0] + om * (1.0 - seeds[:, 2]) / ct, atol=1e-9)
    assert np.allclose(r["xf"][:, 1], seeds[:, 1], atol=1e-9)
    assert np.allclose(r["L"], prim(1.5) - prim(1.0), rtol=1e-9)


def _phys_basis(u):
    t = np.array([1.0, 0, 0]) if abs(u[0]) < 0.9 else np.array([0, 1.0, 0])
    a = np.cross(u, t)
    a /= np.linalg.norm(a)
    return a, np.cross(u, a)


def _scale(q):
    return np.array([q[2] * np.cos(q[1]), q[2], 1.0])


def test_deviations_match_finite_differences_far_from_the_centre(oracle_mod):
    """Eq. dev_sph leaves out terms of relative size (field scale)/r. Far from
    the centre (r ~ 100, field varying over ~0.3) the tangent-space Q_det
    agrees with finite differences of traced neighbouring lines (seeds moved
    along the seed's orthonormal deviation vectors, end displacements taken
    as physical vectors and projected perpendicular to the end field) to a
    few 1e-3; a wrong metric factor in the deviation equations misses by
    about (1 - cos 0.6) = 17 %."""
    th0 = 0.6
    box = ((-0.004, 0.004), (th0 - 0.004, th0 + 0.004), (100.0, 100.5))
    lam = 0.3

    def fn(p, t, r):
        X = 100.0 * np.cos(th0) * p
        Y = 100.0 * (t - th0)
        Z = r - 100.0
        return (0.5 * np.sin(2 * np.pi * Y / lam) + 0.2 * Z, 0.4 * np.cos(2 * np.pi * X / lam), 1.0 + 0.2 * np.sin(
            2 * np.pi * (X + Y) / lam))

    F = sph_field(oracle_mod, fn, n=(33, 33, 33), box=box, mode=0)
    rng = np.random.default_rng(8)
    seeds = np.column_stack([rng.uniform(-0.002, 0.002, 30), th0 + rng.uniform(-0.002, 0.002, 30),
                             rng.uniform(100.1, 100.4, 30)])
    o = oracle_mod.default_opts(tol_abs=1e-12, tol_rel=1e-12)
    r = oracle_mod.trace_seeds(F, seeds, o)
    eps = 1e-6
    errs = []
    for i, q0 in enumerate(seeds):
        if not (r["st_f"][i] == 0 and r["st_b"][i] == 0):
            continue
        b, _, _ = F.interp(q0)
        a, bb = _phys_basis(b / np.linalg.norm(b))
        ends = {}
        for name, d in (("a", a), ("b", bb)):
            for sgn in (1, -1):
                ends[name, sgn] = oracle_mod.trace_seeds(F, (q0 + sgn * eps * d / _scale(q0))[None, :], o)
        if not all(e["face_f"][0] == r["face_f"][i] and e["face_b"][0] == r["face_b"][i] for e in ends.values()):
            continue
        vecs = {}
        for side, key in (("F", "xf"), ("B", "xb")):
            qe = r[key][i]
            be, _, _ = F.interp(qe)
            ue = be / np.linalg.norm(be)
            P = np.eye(3) - np.outer(ue, ue)
            for name in ("a", "b"):
                dq = (ends[name, 1][key][0] - ends[name, -1][key][0]) / (2 * eps)
                vecs[side, name] = P @ (dq * _scale(qe))
        gF = np.array([[vecs["F", "a"] @ vecs["F", "a"], vecs["F", "a"] @ vecs["F", "b"]],
                       [vecs["F", "a"] @ vecs["F", "b"], vecs["F", "b"] @ vecs["F", "b"]]])
        gB = np.array([[vecs["B", "a"] @ vecs["B", "a"], vecs["B", "a"] @ vecs["B", "b"]],
                       [vecs["B", "a"] @ vecs["B", "b"], vecs["B", "b"] @ vecs["B", "b"]]])
        adjB = np.array([[gB[1, 1], -gB[0, 1]], [-gB[0, 1], gB[0, 0]]])
        q_fd = np.trace(gF @ adjB) / np.sqrt(np.linalg.det(gF) * np.linalg.det(gB))
        errs.append(abs(q_fd / r["q_det"][i] - 1))
    assert len(errs) >= 15
    assert max(errs) < 1e-2, sorted(errs)[-5:]
