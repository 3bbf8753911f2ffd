"""Oracle pins on point-charge fields: invariants of Q and brute-force
(Pariat-style finite-difference) squashing factors.

* Q_det (the Eq. finalQ bracket over the true Gram determinants) is >= 2 for
  every line (AM-GM on a 2 x 2 map).
* Q_perp = Q_det (1 + flux_F)(1 + flux_B): Eq. finalQ substitutes flux
  conservation for the determinant; the residuals are reported per end.
* Q is the same when traced from either end of a line and from a mid-line seed
  (it depends only on the end cross-sections).
* Finite differences of traced neighbouring lines (the method the paper
  replaces, Sec. "Field-line deviation using linearization") reproduce the
  tangent-space Q_det to 1e-5 where no neighbour changes end face.
"""
import numpy as np
import pytest

from paper_1609_00724_gb300 import inputs


def make_field(oracle_mod, n, count, seed, mode, depth=(0.15, 0.3)):
    ch = inputs.random_charges(count, seed, depth=depth)
    gf = inputs.to_numpy64(inputs.charge_field(ch, n, dtype=__import__("torch").float64))
    return oracle_mod.Field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, mode=mode)


@pytest.fixture(scope="module")
def fields(oracle_mod):
    return {mode: make_field(oracle_mod, 24, 4, 11, mode) for mode in (0, 1)}


def test_qdet_at_least_two_and_flux_identity(oracle_mod, fields):
    seeds = inputs.random_seeds(400, 3, margin=0.0)
    seeds[:100, 2] = 0.0  # footpoint seeds on the bottom face
    for mode, F in fields.items():
        r = oracle_mod.trace_seeds(F, seeds, oracle_mod.default_opts(tol_abs=1e-9, tol_rel=1e-9))
        ok = np.isfinite(r["q_det"])
        assert ok.sum() > 300
        assert np.all(r["q_det"][ok] >= 2.0 - 1e-9)
        pred = r["q_det"] * (1 + r["flux"]) * (1 + r["flux_b"])
        assert np.allclose(r["q_perp"][ok], pred[ok], rtol=1e-9, atol=0)
        # lengths are the sum of both sides
        assert np.allclose(r["L"], r["lam_f"] - r["lam_b"], rtol=1e-15, atol=0)


def test_flux_residual_converges_in_raw_mode(oracle_mod):
    """The interpolated field is only approximately solenoidal; the flux
    residual of Eq. finalQ must shrink with grid refinement (raw mode)."""
    seeds = inputs.random_seeds(60, 5, margin=0.05)
    worst = []
    for n in (17, 33, 65):
        F = make_field(oracle_mod, n, 2, 21, 1)
        r = oracle_mod.trace_seeds(F, seeds, oracle_mod.default_opts(tol_abs=1e-10, tol_rel=1e-10))
        ok = (r["st_f"] == 0) & (r["st_b"] == 0)
        worst.append(np.median(np.abs(r["flux"][ok])))
    assert worst[0] > worst[1] > worst[2], worst
    assert worst[2] < 1e-2


def test_same_q_from_either_footpoint_and_midline(oracle_mod, fields):
    F = fields[1]
    o = oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11)
    seeds = inputs.random_seeds(40, 8, margin=0.05)
    seeds[:, 2] = 0.0
    r = oracle_mod.trace_seeds(F, seeds, o)
    good = np.nonzero((r["st_f"] == 0) & (r["st_b"] == 0) & (r["lam_f"] - r["lam_b"] > 0.05))[0]
    assert len(good) > 10
    # the far end of each line
    far = np.where((r["lam_f"][good] > 0)[:, None], r["xf"][good], r["xb"][good])
    r2 = oracle_mod.trace_seeds(F, far, o)
    assert np.allclose(r2["q_det"], r["q_det"][good], rtol=1e-6)
    assert np.allclose(r2["L"], r["L"][good], rtol=1e-8)
    fl = np.abs(r["flux"][good]) + np.abs(r["flux_b"][good])
    assert np.all(np.abs(r2["q_perp"] / r["q_perp"][good] - 1) <= 3 * fl + 1e-6)
    # a mid-line seed: stop the line half-way with the maximum-length option
    half = 0.5 * r["L"][good]
    mids = []
    for i, g in enumerate(good):
        s = 1 if r["lam_f"][g] > 0 else -1
        o2 = oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11, max_length=half[i])
        r3 = oracle_mod.trace_seeds(F, seeds[g:g + 1], o2)
        mids.append(r3["xf"][0] if s > 0 else r3["xb"][0])
    r4 = oracle_mod.trace_seeds(F, np.array(mids), o)
    assert np.allclose(r4["q_det"], r["q_det"][good], rtol=1e-6)
    assert np.allclose(r4["L"], r["L"][good], rtol=1e-8)


def _basis(u):
    t = np.array([1.0, 0, 0]) if abs(u[0]) < 0.9 else np.array([0, 1.0, 0])
    a = np.cross(u, t)
    a /= np.linalg.norm(a)
    return a, np.cross(u, a)


def _qdet_from_gram(aF, bF, aB, bB):
    gF = np.array([[aF @ aF, aF @ bF], [aF @ bF, bF @ bF]])
    gB = np.array([[aB @ aB, aB @ bB], [aB @ bB, bB @ bB]])
    adjB = np.array([[gB[1, 1], -gB[0, 1]], [-gB[0, 1], gB[0, 0]]])
    return np.trace(gF @ adjB) / np.sqrt(np.linalg.det(gF) * np.linalg.det(gB))


@pytest.mark.parametrize("mode,n", [(1, 12), (0, 16)])
def test_finite_difference_q_matches_tangent_space(oracle_mod, mode, n):
    F = make_field(oracle_mod, n, 4, 31 + n, mode)
    cell = 1.0 / (n - 1)
    eps = 1e-5 * cell  # central-difference error falls as eps^2: about 2e-7 here
    o = oracle_mod.default_opts(tol_abs=1e-12, tol_rel=1e-12)
    seeds = inputs.random_seeds(30, 40 + n, margin=0.1)
    r = oracle_mod.trace_seeds(F, seeds, o)
    checked = 0
    for i, x0 in enumerate(seeds):
        if not (r["st_f"][i] == 0 and r["st_b"][i] == 0):
            continue
        b, _, _ = F.interp(x0)
        a, bb = _basis(b / np.linalg.norm(b))
        ends = {}
        for name, d in (("a", a), ("b", bb)):
            for sgn in (1, -1):
                rr = oracle_mod.trace_seeds(F, (x0 + sgn * eps * d)[None, :], o)
                ends[name, sgn] = rr
        faces_same = all(e["face_f"][0] == r["face_f"][i] and e["face_b"][0] == r["face_b"][i]
                         for e in ends.values())
        if not faces_same:
            continue
        vecs = {}
        for side, key in (("F", "xf"), ("B", "xb")):
            xe = r[key][i]
            be, _, _ = F.interp(xe)
            ue = be / np.linalg.norm(be)
            P = np.eye(3) - np.outer(ue, ue)
            for name in ("a", "b"):
                dx = (ends[name, 1][key][0] - ends[name, -1][key][0]) / (2 * eps)
                vecs[side, name] = P @ dx
        q_fd = _qdet_from_gram(vecs["F", "a"], vecs["F", "b"], vecs["B", "a"], vecs["B", "b"])
        assert abs(q_fd / r["q_det"][i] - 1) < 1e-5, (x0, q_fd, r["q_det"][i])
        checked += 1
    assert checked >= 10


def test_footpoint_fd_on_bottom_face(oracle_mod):
    """Footpoint Q from finite differences of the boundary-to-boundary map
    (seeds on z = 0, in-plane perturbations) in raw mode on a fine grid: the
    Jacobian form must agree with Eq. finalQ's footpoint variant up to the
    flux residual of the interpolated field."""
    n = 33
    F = make_field(oracle_mod, n, 2, 5, 1, depth=(0.2, 0.3))
    cell = 1.0 / (n - 1)
    eps = 1e-5 * cell
    o = oracle_mod.default_opts(tol_abs=1e-12, tol_rel=1e-12)
    seeds = inputs.random_seeds(25, 77, margin=0.2)
    seeds[:, 2] = 0.0
    r = oracle_mod.trace_seeds(F, seeds, o)
    checked = 0
    for i, x0 in enumerate(seeds):
        if not (r["st_f"][i] == 0 and r["st_b"][i] == 0) or not np.isfinite(r["q_foot"][i]):
            continue
        s_key = "xf" if r["lam_f"][i] > 0 else "xb"
        f_key = "face_f" if r["lam_f"][i] > 0 else "face_b"
        face = r[f_key][i]
        cols = []
        same = True
        for d in (np.array([1.0, 0, 0]), np.array([0, 1.0, 0])):
            e = [oracle_mod.trace_seeds(F, (x0 + sgn * eps * d)[None, :], o) for sgn in (1, -1)]
            if any(ee[f_key][0] != face for ee in e):
                same = False
            cols.append((e[0][s_key][0] - e[1][s_key][0]) / (2 * eps))
        if not same:
            continue
        keep = [k for k in range(3) if k != face // 2]
        J = np.array([[cols[0][keep[0]], cols[1][keep[0]]], [cols[0][keep[1]], cols[1][keep[1]]]])
        q_fd = np.sum(J * J) / abs(np.linalg.det(J))
        fl = abs(r["flux"][i]) + abs(r["flux_b"][i])
        assert abs(q_fd / r["q_foot"][i] - 1) < 3 * fl + 1e-5, (x0, q_fd, r["q_foot"][i], fl)
        checked += 1
    assert checked >= 8


@pytest.mark.parametrize("mode", [0, 1])
def test_loop_from_face_is_continuous(oracle_mod, fields, mode):
    """A seed on z = 0 where the field points weakly inward can loop back to
    the same face: the line's length is the later crossing, continuous in the
    seed. Moving the seed a distance d inside changes L by O(d), so the
    difference must shrink tenfold from d = 1e-9 to d = 1e-10 (a landing that
    stops at the start point would give L = 0 and a difference of L)."""
    F = fields[mode]
    n = 24
    xs = np.linspace(-0.97, 0.97, 90)
    s = np.stack(np.meshgrid(xs, xs, indexing="ij"), -1).reshape(-1, 2)
    seeds = np.concatenate([s, np.zeros((len(s), 1))], 1)
    o = oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11)
    r = oracle_mod.trace_seeds(F, seeds, o)
    loop = (r["face_f"] == 4) & (r["face_b"] == 4) & (r["L"] < 0.5 / (n - 1))
    near_zero = np.where(loop)[0]
    assert len(near_zero) >= 10
    idx = near_zero[:30]
    diffs = []
    for d in (1e-9, 1e-10):
        s2 = seeds[idx].copy()
        s2[:, 2] += d
        r2 = oracle_mod.trace_seeds(F, s2, o)
        diffs.append(np.abs(r2["L"] - r["L"][idx]))
    assert np.all(r["L"][idx] > 0)
    assert np.all(diffs[1] <= 0.2 * diffs[0] + 1e-12), np.c_[r["L"][idx], diffs[0], diffs[1]]
