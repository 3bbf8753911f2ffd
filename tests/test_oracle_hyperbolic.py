"""Oracle pins on the linear hyperbolic field B = (lam x, -lam y, B0).

The flow map of dx/dt = B is (x0 e^{lam t}, y0 e^{-lam t}, z0 + B0 t), so:
* a line from (x0, y0, 0) leaves through z = 1 at t = 1/B0 when |x0| < e^{-lam/B0},
  otherwise through x = +-1 at t = ln(1/|x0|)/lam (never through y = +-1 in the box);
* footpoint Q (Jacobian of the boundary-to-boundary map, Titov 2002) is
  k^2 + k^-2 with k = e^{lam/B0} for top exits and lam (x0^2 + y0^2)/B0 + B0/(lam x0^2)
  for side exits;
* perpendicular Q (Eq. finalQ with dx_perp) is ||P_e D [a b]||_F^2 |B_e|/|B_s| with
  D = diag(e^{lam t}, e^{-lam t}, 1), P_e the projector orthogonal to B_e = D B_s, and
  (a, b) any orthonormal pair orthogonal to B_s (Q does not depend on the pair);
* the length is the arc length integral of |B(x(t))| dt.
In raw mode trilinear interpolation reproduces this linear field exactly, so the
oracle must meet the closed forms to integration tolerance.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_1609_00724_gb300 import inputs

LAM, B0 = 3.0, 1.0


def closed_forms(x0, y0):
    k = math.exp(LAM / B0)
    top = abs(x0) < math.exp(-LAM / B0)
    if top:
        te = 1.0 / B0
        qf = k * k + 1.0 / (k * k)
        face = 5
    else:
        te = math.log(1.0 / abs(x0)) / LAM
        qf = LAM * (x0 * x0 + y0 * y0) / B0 + B0 / (LAM * x0 * x0)
        face = 1 if x0 > 0 else 0
    Bs = np.array([LAM * x0, -LAM * y0, B0])
    D = np.diag([math.exp(LAM * te), math.exp(-LAM * te), 1.0])
    Be = D @ Bs
    # any orthonormal pair orthogonal to Bs
    u = Bs / np.linalg.norm(Bs)
    t = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    a = np.cross(u, t)
    a /= np.linalg.norm(a)
    b = np.cross(u, a)
    ue = Be / np.linalg.norm(Be)
    P = np.eye(3) - np.outer(ue, ue)
    M = P @ D @ np.column_stack([a, b])
    qp = float(np.sum(M * M)) * np.linalg.norm(Be) / np.linalg.norm(Bs)
    L, _ = integrate.quad(lambda s: math.sqrt((LAM * x0) ** 2 * math.exp(2 * LAM * s)
                                              + (LAM * y0) ** 2 * math.exp(-2 * LAM * s) + B0 ** 2),
                          0.0, te, epsabs=1e-14, epsrel=1e-13, limit=200)
    return qf, qp, L, face


@pytest.fixture(scope="module")
def raw_field(oracle_mod):
    gf = inputs.hyperbolic_field(64)
    return oracle_mod.Field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, mode=1)


def test_trilinear_exact_for_linear_field(raw_field):
    rng = np.random.default_rng(7)
    for _ in range(200):
        x = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0, 1)])
        b, g, m = raw_field.interp(x)
        B = np.array([LAM * x[0], -LAM * x[1], B0])
        n = np.linalg.norm(B)
        assert np.allclose(b, B / n, rtol=0, atol=1e-13)
        assert abs(m - n) < 1e-12
        J = np.diag([LAM, -LAM, 0.0])
        u = B / n
        G = (np.eye(3) - np.outer(u, u)) @ J / n
        assert np.allclose(g, G, rtol=0, atol=1e-12)


def test_config1_map_matches_closed_forms(oracle_mod, raw_field):
    """256 x 256 pixel centres on z = 0 (every 3rd pixel row/column plus all 12
    top-exit columns), raw mode, tol 1e-11."""
    nu = nv = 256
    seeds = oracle_mod.plane_seeds([0, 0, 0], [2, 0, 0], [0, 2, 0], nu, nv).reshape(nv, nu, 3)
    cols = sorted(set(range(0, nu, 3)) | set(range(122, 134)))
    rows = list(range(0, nv, 3))
    pick = seeds[np.ix_(rows, cols)].reshape(-1, 3)
    o = oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11)
    r = oracle_mod.trace_seeds(raw_field, pick, o)
    n_top = 0
    for i, (x0, y0, _) in enumerate(pick):
        qf, qp, L, face = closed_forms(x0, y0)
        n_top += face == 5
        assert r["st_f"][i] == 0 and r["st_b"][i] == 0
        assert r["face_f"][i] == face, (x0, y0)
        assert r["face_b"][i] == 4  # the seed is on z = 0 and B_z > 0: zero-length backward side
        assert r["lam_b"][i] == 0.0
        assert abs(r["q_foot"][i] / qf - 1) < 1e-8, (x0, y0, r["q_foot"][i], qf)
        assert abs(r["q_perp"][i] / qp - 1) < 1e-8, (x0, y0, r["q_perp"][i], qp)
        assert abs(r["L"][i] / L - 1) < 1e-10, (x0, y0, r["L"][i], L)
        assert r["q_det"][i] >= 2.0
    # pixel columns 122..133 are exactly the top-exit lines (|x0| < e^-3)
    assert n_top == 12 * len(rows)


def test_top_exit_columns(oracle_mod):
    xs = -1 + (np.arange(256) + 0.5) * 2 / 256
    top = np.nonzero(np.abs(xs) < math.exp(-3.0))[0]
    assert list(top) == list(range(122, 134))


def test_endpoint_lands_exactly_on_face(oracle_mod, raw_field):
    pick = np.array([[0.01, 0.2, 0.0], [0.4, -0.3, 0.0], [-0.2, 0.6, 0.0]])
    r = oracle_mod.trace_seeds(raw_field, pick, oracle_mod.default_opts(tol_abs=1e-8, tol_rel=1e-8))
    for i in range(3):
        f = r["face_f"][i]
        ax, up = f // 2, f % 2
        bound = [(-1, 1), (-1, 1), (0, 1)][ax][up]
        assert r["xf"][i][ax] == bound


def test_paper_mode_converges_second_order(oracle_mod):
    """Normalise-then-interpolate (paper mode) is not exact for this field; its
    footpoint-Q error must fall about 4x per grid doubling."""
    seed = np.array([[0.01, 0.3, 0.0]])
    qf, _, _, _ = closed_forms(0.01, 0.3)
    errs = []
    for n in (33, 65, 129):
        gf = inputs.hyperbolic_field(n)
        F = oracle_mod.Field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, mode=0)
        r = oracle_mod.trace_seeds(F, seed, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
        errs.append(abs(r["q_foot"][0] / qf - 1))
    assert errs[0] > errs[1] > errs[2]
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 5.5, errs


def test_max_length_cutoff(oracle_mod, raw_field):
    o = oracle_mod.default_opts(tol_abs=1e-10, tol_rel=1e-10, max_length=0.25)
    r = oracle_mod.trace_seeds(raw_field, np.array([[0.0, 0.0, 0.5]]), o)
    assert r["st_f"][0] == oracle_mod.ST_MAXLEN and r["st_b"][0] == oracle_mod.ST_MAXLEN
    assert abs(r["L"][0] - 0.5) < 1e-14
    # on the centre line B = (0, 0, 1): the line is the z axis
    assert abs(r["xf"][0][2] - 0.75) < 1e-12 and abs(r["xb"][0][2] - 0.25) < 1e-12
    assert np.isnan(r["q_foot"][0]) and np.isfinite(r["q_perp"][0])


def test_seed_outside_and_skip_open(oracle_mod, raw_field):
    o = oracle_mod.default_opts(tol_abs=1e-8, tol_rel=1e-8, skip_open=1)
    r = oracle_mod.trace_seeds(raw_field, np.array([[0.0, 0.0, -0.1], [0.2, 0.1, 0.0]]), o)
    assert r["st_f"][0] == oracle_mod.ST_OUTSIDE and np.isnan(r["L"][0])
    # every line of this field is open (reaches the top or a side): Q is skipped
    assert np.isnan(r["q_perp"][1]) and np.isfinite(r["L"][1])


def load_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hyperbolic_closed_forms.txt")
    return np.loadtxt(path, comments="#")


def test_golden_fixture(oracle_mod, raw_field):
    g = load_golden()
    seeds = np.column_stack([g[:, 2], g[:, 3], np.zeros(len(g))])
    r = oracle_mod.trace_seeds(raw_field, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    assert np.all(r["face_f"] == g[:, 7].astype(int))
    assert np.allclose(r["q_foot"], g[:, 4], rtol=1e-8, atol=0)
    assert np.allclose(r["q_perp"], g[:, 5], rtol=1e-8, atol=0)
    assert np.allclose(r["L"], g[:, 6], rtol=1e-10, atol=0)


def test_euler_is_first_order(oracle_mod, raw_field):
    """Fixed-step Euler (Sec. "Integration methods"): against the closed forms,
    the length, footpoint Q and perpendicular Q errors halve with the step
    (first order), the exit faces are exact at every step, and Richardson
    extrapolation of two steps, 2 X(h/2) - X(h), removes the first-order term
    (error at least 20x smaller). A dropped or mis-signed term would leave an
    O(1) error or another order."""
    seeds = np.array([[0.02, 0.3, 0.0], [-0.03, -0.5, 0.0], [0.3, 0.2, 0.0], [-0.6, 0.7, 0.0],
                      [0.1, -0.1, 0.0]])
    cf = [closed_forms(x, y) for x, y, _ in seeds]
    exact = {"q_foot": np.array([c[0] for c in cf]), "q_perp": np.array([c[1] for c in cf]),
             "L": np.array([c[2] for c in cf])}
    res = {}
    for eh in (0.2, 0.1, 0.05):
        r = oracle_mod.trace_seeds(raw_field, seeds, oracle_mod.default_opts(integrator=1, euler_h=eh))
        assert np.all(r["st_f"] == oracle_mod.ST_OK) and np.all(r["st_b"] == oracle_mod.ST_OK)
        assert list(r["face_f"]) == [c[3] for c in cf] and np.all(r["face_b"] == 4)
        res[eh] = r
    for key, ex in exact.items():
        err = {eh: np.abs(res[eh][key] / ex - 1) for eh in res}
        assert np.all(err[0.05] > 1e-7), key  # not exact: a genuine fixed-step method
        for a, b in ((0.2, 0.1), (0.1, 0.05)):
            ratio = err[a] / err[b]
            assert np.all((ratio > 1.8) & (ratio < 2.2)), (key, ratio)
        rich = np.abs((2 * res[0.05][key] - res[0.1][key]) / ex - 1)
        assert np.all(rich <= err[0.05] / 20), (key, rich / err[0.05])


def test_length_only_matches_closed_form_lengths(oracle_mod, raw_field):
    """Lengths-only tracing (no deviation equations; the mode of the refinement
    passes' decision traces) meets the closed-form lengths and exit faces: to
    1e-10 at tol 1e-11, and to 1e-7 at the decision traces' settings (tol 1e-5,
    step cap 4 smallest spacings); its Q outputs are NaN."""
    seeds = oracle_mod.plane_seeds([0, 0, 0], [2, 0, 0], [0, 2, 0], 64, 64).reshape(-1, 3)[::7]
    for tol, h_max, bar in ((1e-11, 2.0, 1e-10), (1e-5, 4.0, 1e-7)):
        r = oracle_mod.trace_seeds(raw_field, seeds, oracle_mod.default_opts(tol_abs=tol, tol_rel=tol, length_only=1,
                                                                             h_max=h_max))
        assert np.all(np.isnan(r["q_perp"]))
        for i, (x0, y0, _) in enumerate(seeds):
            _, _, L, face = closed_forms(x0, y0)
            assert r["face_f"][i] == face and r["face_b"][i] == 4
            assert abs(r["L"][i] / L - 1) < bar, (tol, x0, y0, r["L"][i], L)
