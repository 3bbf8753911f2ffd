"""GPU parity of spherical geometry (Eq. fl_sph, Eq. dev_sph) against the FP64
oracle, through the C ABI: Cash-Karp in FP32 and FP64, paper and raw modes,
higher-order interpolation, spherical slices through qsl_q_map_2d, and the
monopole's exact Q."""
import numpy as np
import pytest
import torch

from gpu_helpers import GPU_TOL, compare_lines

pytestmark = pytest.mark.gpu

PHI, TH, R = (-0.4, 0.4), (-0.3, 0.3), (1.0, 1.5)
LO, HI = (PHI[0], TH[0], R[0]), (PHI[1], TH[1], R[1])


@pytest.fixture(scope="module")
def qsl():
    from paper_1609_00724_gb300 import qsl as q
    q.lib()
    return q


def dipole_twist(p, t, r):
    """A dipole tilted off the grid's pole plus a twist, in (phi^, theta^, r^)."""
    c = np.cos(t)
    br = 2.0 * (np.sin(t) * 0.8 + c * np.cos(p - 0.2) * 0.6) / r ** 3
    bt = -(np.cos(t) * 0.8 - np.sin(t) * np.cos(p - 0.2) * 0.6) / r ** 3 + 0.05
    bp = 0.6 * np.sin(p - 0.2) / r ** 3 + 0.3 * (r - 1.0) * c
    return bp, bt, br


def fields(qsl, oracle_mod, fn, n, mode, order=1):
    ax = [np.linspace(lo, hi, k) for (lo, hi), k in zip((PHI, TH, R), n)]
    T, Th, Ph = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    bp, bt, br = (np.ascontiguousarray(a, dtype=np.float64) for a in fn(Ph, Th, T))
    b32 = [torch.as_tensor(a.astype(np.float32)).cuda() for a in (bp, bt, br)]
    F = qsl.qsl_load_field(*b32, ax[0], ax[1], ax[2], interp_mode=mode)
    qsl.qsl_set_geometry(F, qsl.QSL_GEOM_SPHERICAL)
    f32 = [a.astype(np.float32).astype(np.float64) for a in (bp, bt, br)]
    Fo = oracle_mod.Field(*f32, ax[0], ax[1], ax[2], mode=mode, order=order, geometry=1)
    cq = min(np.diff(a).min() for a in ax)
    return F, Fo, cq


def seeds_in_box(n, seed):
    rng = np.random.default_rng(seed)
    s = np.column_stack([rng.uniform(-0.35, 0.35, n), rng.uniform(-0.27, 0.27, n), rng.uniform(1.0, 1.45, n)])
    s[: n // 4, 2] = 1.0  # footpoints on the inner sphere
    return s


def rec_dict(rec):
    return {"q_perp": rec["q_perp"], "q_foot": rec["q_foot"], "q_det": rec["q_det"], "L": rec["length"],
            "face_f": rec["face_f"], "face_b": rec["face_b"], "xf": rec["x_f"], "xb": rec["x_b"],
            "st_f": rec["status_f"], "st_b": rec["status_b"]}


@pytest.mark.parametrize("mode,prec,integ,order", [(1, 0, 0, 1), (0, 0, 0, 1), (1, 1, 0, 1), (0, 0, 1, 1),
                                                   (1, 0, 0, 3)])
def test_spherical_matches_oracle(qsl, oracle_mod, mode, prec, integ, order):
    F, Fo, cq = fields(qsl, oracle_mod, dipole_twist, (33, 25, 33), mode, order)
    seeds = seeds_in_box(200, 4 + mode + 2 * prec)
    kw = dict(integrator=qsl.QSL_EULER, euler_h=0.2) if integ else dict(tol_abs=GPU_TOL, tol_rel=GPU_TOL)
    if prec:
        kw.update(tol_abs=1e-10, tol_rel=1e-10, precision=qsl.QSL_FP64)
    o = qsl.qsl_opts_default(interp_order=order, **kw)
    rec = qsl.qsl_trace_seeds(F, seeds, o)
    if integ:
        ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(integrator=1, euler_h=0.2))
        tol = dict(q_rtol=1e-4, l_rtol=1e-5)
    else:
        ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
        tol = dict(q_rtol=2e-6, l_rtol=3e-7) if prec else {}
    rep = compare_lines(rec_dict(rec), ref, cq, LO, HI, **tol)
    assert rep["q_checked"] > 100
    assert np.array_equal(rec["status_f"], ref["st_f"]) and np.array_equal(rec["status_b"], ref["st_b"])


def test_spherical_slice_map(qsl, oracle_mod):
    """A spherical slice at r0 = 1.2 through qsl_q_map_2d (a plane in
    (phi, theta, r)), sampled pixels against the oracle."""
    F, Fo, cq = fields(qsl, oracle_mod, dipole_twist, (33, 25, 33), 1)
    nu, nv = 128, 96
    q = torch.empty(nu * nv, device="cuda")
    L = torch.empty(nu * nv, device="cuda")
    fc = torch.empty(2 * nu * nv, dtype=torch.uint8, device="cuda")
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL)
    qsl.qsl_q_map_2d(F, (0.0, 0.0, 1.2), (0.7, 0, 0), (0, 0.5, 0), nu, nv, o, q=q, length=L, faces=fc)
    torch.cuda.synchronize()
    seeds = oracle_mod.plane_seeds([0.0, 0.0, 1.2], [0.7, 0, 0], [0, 0.5, 0], nu, nv)
    idx = np.random.default_rng(1).choice(nu * nv, 150, replace=False)
    ref = oracle_mod.trace_seeds(Fo, seeds[idx], oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    f2 = fc.cpu().numpy().reshape(-1, 2)[idx]
    gd = {"q_perp": q.cpu().numpy()[idx], "L": L.cpu().numpy()[idx], "face_f": f2[:, 0], "face_b": f2[:, 1]}
    compare_lines(gd, ref, cq, LO, HI)


def test_spherical_monopole_q_is_two_and_argument_checks(qsl, oracle_mod):
    F, Fo, cq = fields(qsl, oracle_mod, lambda p, t, r: (0 * r, 0 * r, 1.0 / r ** 2), (33, 33, 33), 1)
    seeds = seeds_in_box(100, 9)
    seeds[:, 2] = np.clip(seeds[:, 2], 1.02, 1.45)
    rec = qsl.qsl_trace_seeds(F, seeds, qsl.qsl_opts_default(tol_abs=1e-10, tol_rel=1e-10, precision=qsl.QSL_FP64))
    assert np.all(rec["face_f"] == 5) and np.all(rec["face_b"] == 4)
    assert np.allclose(rec["length"], 0.5, rtol=1e-6)
    assert np.allclose(rec["q_det"], 2.0, rtol=1e-8)
    with pytest.raises(qsl.QslError) as e:
        qsl.qsl_trace_seeds(F, seeds, qsl.qsl_opts_default(integrator=qsl.QSL_DOPRI5_CELL))
    assert e.value.code == qsl.QSL_EINVAL
    ax = np.linspace(-1.7, 1.7, 5)  # latitudes beyond the poles
    b = np.ones((5, 5, 5))
    Fb = qsl.qsl_load_field(b, b, b, ax, ax, np.linspace(1, 2, 5), qsl.QSL_RAW_B)
    with pytest.raises(qsl.QslError):
        qsl.qsl_set_geometry(Fb, qsl.QSL_GEOM_SPHERICAL)
