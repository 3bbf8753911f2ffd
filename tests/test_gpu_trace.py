"""GPU parity of the tracer (qsl_trace_seeds, qsl_q_map_2d, qsl_q_volume_3d)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_1609_00724_gb300 import inputs
from gpu_helpers import GPU_TOL, L_RTOL, compare_lines

pytestmark = pytest.mark.gpu

BOX_LO, BOX_HI = (-1.0, -1.0, 0.0), (1.0, 1.0, 1.0)


@pytest.fixture(scope="module")
def qsl():
    from paper_1609_00724_gb300 import qsl as q
    q.lib()
    return q


def _gpu_field(qsl, gf, mode):
    t = [torch.as_tensor(np.ascontiguousarray(a)).cuda() if not isinstance(a, torch.Tensor) else a.cuda()
         for a in (gf.bx, gf.by, gf.bz)]
    return qsl.qsl_load_field(*t, gf.xc, gf.yc, gf.zc, interp_mode=mode)


def _oracle_field(oracle_mod, gf, mode):
    g = inputs.to_numpy64(gf)
    return oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=mode)


def _rec_to_dict(rec):
    return {"q_perp": rec["q_perp"], "q_foot": rec["q_foot"], "q_det": rec["q_det"], "L": rec["length"],
            "face_f": rec["face_f"], "face_b": rec["face_b"], "xf": rec["x_f"], "xb": rec["x_b"],
            "st_f": rec["status_f"], "st_b": rec["status_b"]}


@pytest.mark.parametrize("mode,integ,lanes", [(0, 0, 0), (1, 0, 0), (0, 2, 1), (1, 2, 1), (0, 2, 3), (1, 2, 3)])
def test_trace_seeds_charge_field(qsl, oracle_mod, mode, integ, lanes):
    """lanes: 1 = one lane per line (cell_kernel_f32/_f64), 3 = a group of three lanes
    per line (cell_coop_kernel)."""
    tol = GPU_TOL
    ch = inputs.random_charges(4, 2)
    gf = inputs.charge_field(ch, 64, dtype=torch.float32)
    F = _gpu_field(qsl, gf, mode)
    Fo = _oracle_field(oracle_mod, gf, mode)
    seeds = inputs.random_seeds(600, 17)
    seeds[:150, 2] = 0.0     # footpoints on the bottom face
    seeds[150:160, 0] = 1.0  # on the x+ face
    o = qsl.qsl_opts_default(tol_abs=tol, tol_rel=tol, integrator=integ, line_lanes=lanes)
    rec = qsl.lines_to_numpy(qsl.qsl_trace_seeds(F, torch.as_tensor(seeds).cuda(), o))
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    g = _rec_to_dict(rec)
    rep = compare_lines(g, ref, 1.0 / 63, BOX_LO, BOX_HI)
    rep2 = compare_lines(g, ref, 1.0 / 63, BOX_LO, BOX_HI, "q_foot", "q_foot")
    rep3 = compare_lines(g, ref, 1.0 / 63, BOX_LO, BOX_HI, "q_det", "q_det")
    print(rep["worst_q"], rep["worst_l"], rep2["worst_q"], rep3["worst_q"])
    assert rep["q_checked"] > 300
    # statuses agree
    assert np.array_equal(rec["status_f"], ref["st_f"]) and np.array_equal(rec["status_b"], ref["st_b"])
    # host-memory path gives the same records as the device path
    rec_h = qsl.qsl_trace_seeds(F, seeds, o)
    assert np.array_equal(rec_h["face_f"], rec["face_f"])
    assert np.allclose(rec_h["length"], rec["length"], rtol=1e-6)


@pytest.mark.parametrize("mode,integ,tol", [(1, 0, GPU_TOL), (0, 0, GPU_TOL), (1, 2, GPU_TOL), (0, 2, GPU_TOL)])
def test_config1_hyperbolic_map(qsl, oracle_mod, mode, integ, tol):
    """The 256 x 256 map of the linear hyperbolic field on z = 0: raw mode
    against the closed forms (golden fixture), both modes against the oracle
    on a subsample that includes the 12 top-exit columns."""
    gf = inputs.hyperbolic_field(64)
    F = _gpu_field(qsl, gf, mode)
    n = 256
    q = torch.empty(n * n, device="cuda")
    L = torch.empty(n * n, device="cuda")
    faces = torch.empty(2 * n * n, dtype=torch.uint8, device="cuda")
    st = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    o = qsl.qsl_opts_default(tol_abs=tol, tol_rel=tol, q_form=qsl.QSL_Q_FOOT, integrator=integ)
    qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), n, n, o, q, L, faces, st)
    torch.cuda.synchronize()
    q, L, faces, st = q.cpu().numpy(), L.cpu().numpy(), faces.cpu().numpy().reshape(-1, 2), st.cpu().numpy()
    assert np.all(st & 0x3f == 0)
    if mode == 1:
        import os
        g = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "hyperbolic_closed_forms.txt"))
        idx = g[:, 1].astype(int) * n + g[:, 0].astype(int)
        assert np.array_equal(faces[idx, 0], g[:, 7].astype(int))
        assert np.all(np.abs(q[idx] / g[:, 4] - 1) < 1e-3)
        assert np.all(np.abs(L[idx] / g[:, 6] - 1) < 1e-5)
    Fo = _oracle_field(oracle_mod, gf, mode)
    cols = sorted(set(range(0, n, 7)) | set(range(122, 134)))
    rows = list(range(3, n, 11))
    pix = np.array([j * n + i for j in rows for i in cols])
    seeds = oracle_mod.plane_seeds([0, 0, 0], [2, 0, 0], [0, 2, 0], n, n)[pix]
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    g = {"q_foot": q[pix], "L": L[pix], "face_f": faces[pix, 0], "face_b": faces[pix, 1]}
    compare_lines(g, ref, 1.0 / 63, BOX_LO, BOX_HI, "q_foot", "q_foot")


@pytest.mark.parametrize("integ,tol", [(0, GPU_TOL), (2, GPU_TOL)])
def test_volume_map_matches_oracle(qsl, oracle_mod, integ, tol):
    ch = inputs.random_charges(8, 3)
    gf = inputs.charge_field(ch, 48, dtype=torch.float32)
    F = _gpu_field(qsl, gf, 0)
    nx, ny, nz = 40, 36, 17  # ragged against any tiling
    N = nx * ny * nz
    q = torch.empty(N, device="cuda")
    L = torch.empty(N, device="cuda")
    faces = torch.empty(2 * N, dtype=torch.uint8, device="cuda")
    st = torch.empty(N, dtype=torch.uint8, device="cuda")
    o = qsl.qsl_opts_default(tol_abs=tol, tol_rel=tol, integrator=integ)
    qsl.qsl_q_volume_3d(F, BOX_LO, BOX_HI, nx, ny, nz, o, q, L, faces, st)
    torch.cuda.synchronize()
    Fo = _oracle_field(oracle_mod, gf, 0)
    idx = inputs.subsample(N, 500, 99)
    seeds = oracle_mod.volume_seeds(BOX_LO, BOX_HI, nx, ny, nz)[idx]
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    fc = faces.cpu().numpy().reshape(-1, 2)
    g = {"q_perp": q.cpu().numpy()[idx], "L": L.cpu().numpy()[idx], "face_f": fc[idx, 0], "face_b": fc[idx, 1]}
    compare_lines(g, ref, 1.0 / 47, BOX_LO, BOX_HI)


@pytest.mark.parametrize("integ,lanes", [(0, 0), (2, 1), (2, 3)])
def test_fp64_precision_matches_oracle_tightly(qsl, oracle_mod, integ, lanes):
    ch = inputs.random_charges(4, 5)
    gf = inputs.charge_field(ch, 32, dtype=torch.float64)
    F = _gpu_field(qsl, gf, 1)
    Fo = _oracle_field(oracle_mod, gf, 1)
    seeds = inputs.random_seeds(200, 23)
    o = qsl.qsl_opts_default(tol_abs=1e-10, tol_rel=1e-10, precision=qsl.QSL_FP64, integrator=integ,
                             line_lanes=lanes)
    rec = qsl.qsl_trace_seeds(F, seeds, o)
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    # lengths are stored as float32 in the record: 3e-7 covers their rounding
    compare_lines(_rec_to_dict(rec), ref, 1.0 / 31, BOX_LO, BOX_HI, q_rtol=2e-6, l_rtol=3e-7)


def test_euler_matches_oracle_euler(qsl, oracle_mod):
    """Fixed-step Euler (Sec. "Integration methods"): same steps on both sides."""
    gf = inputs.hyperbolic_field(32)
    F = _gpu_field(qsl, gf, 1)
    Fo = _oracle_field(oracle_mod, gf, 1)
    seeds = inputs.random_seeds(100, 4, margin=0.05)
    o = qsl.qsl_opts_default(integrator=qsl.QSL_EULER, euler_h=0.2, precision=qsl.QSL_FP64)
    rec = qsl.qsl_trace_seeds(F, seeds, o)
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(integrator=1, euler_h=0.2))
    compare_lines(_rec_to_dict(rec), ref, 1.0 / 31, BOX_LO, BOX_HI, q_rtol=1e-9, l_rtol=2e-7)


def test_edge_cases(qsl, oracle_mod):
    gf = inputs.hyperbolic_field(16)
    F = _gpu_field(qsl, gf, 1)
    o = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6)
    # no seeds
    out = qsl.qsl_trace_seeds(F, np.zeros((0, 3)), o)
    assert out.shape == (0,)
    # outside, on a face moving out, max length cutoff
    seeds = np.array([[0.0, 0.0, -0.5], [0.3, 0.2, 0.0], [0.0, 0.0, 0.5]])
    o2 = qsl.qsl_opts_default(tol_abs=1e-7, tol_rel=1e-7, max_length=0.2)
    rec = qsl.qsl_trace_seeds(F, seeds, o2)
    assert rec["status_f"][0] == qsl.QSL_LINE_OUTSIDE and np.isnan(rec["length"][0])
    assert rec["face_b"][1] == 4 and rec["lam_b"][1] == 0.0
    assert rec["status_f"][2] == qsl.QSL_LINE_MAXLEN and abs(rec["length"][2] - 0.4) < 1e-6
    # zero field: the line cannot start
    z = np.zeros((4, 4, 4))
    ax = np.linspace(0, 1, 4)
    Fz = qsl.qsl_load_field(z, z, z, ax, ax, ax, qsl.QSL_RAW_B)
    rz = qsl.qsl_trace_seeds(Fz, np.array([[0.5, 0.5, 0.5]]), o)
    assert rz["status_f"][0] == qsl.QSL_LINE_NULL
    # non-finite field values are rejected
    zb = z.copy()
    zb[1, 1, 1] = np.nan
    with pytest.raises(qsl.QslError) as e:
        qsl.qsl_load_field(zb, z, z, ax, ax, ax)
    assert e.value.code == qsl.QSL_ENONFINITE
    # bad arguments
    with pytest.raises(qsl.QslError) as e:
        qsl.qsl_trace_seeds(F, seeds, qsl.qsl_opts_default(tol_abs=-1.0))
    assert e.value.code == qsl.QSL_EINVAL
    with pytest.raises(qsl.QslError):
        qsl.qsl_load_field(z, z, z, ax, ax[::-1].copy(), ax)


def test_skip_open_and_retrace_flag(qsl, oracle_mod):
    ch = inputs.random_charges(4, 2)
    gf = inputs.charge_field(ch, 64, dtype=torch.float32)
    F = _gpu_field(qsl, gf, 0)
    n = 128
    q = torch.empty(n * n, device="cuda")
    st = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    faces = torch.empty(2 * n * n, dtype=torch.uint8, device="cuda")
    o = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6, skip_open=1, retrace_q=1e3)
    qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), n, n, o, q=q, faces=faces, status=st)
    torch.cuda.synchronize()
    q, st, fc = q.cpu().numpy(), st.cpu().numpy(), faces.cpu().numpy().reshape(-1, 2)
    closed = (fc[:, 0] == 4) & (fc[:, 1] == 4)
    assert np.all(np.isnan(q[~closed]))
    assert np.all((st[~closed] & qsl.QSL_FLAG_OPEN_SKIPPED) != 0)
    assert np.all(np.isfinite(q[closed]))
    s = qsl.qsl_last_stats()
    ret = (st & qsl.QSL_FLAG_RETRACED) != 0
    assert s["retraced"] == ret.sum()
    assert np.all(q[ret & closed] > 1e3 * 0.99)


def test_config3_volume_full_size_sampled(qsl, oracle_mod):
    """8 charges on 384^3 (FP32), Q/FLL at 512 x 512 x 256 cell-centre seeds and
    the 3D FLEDGE of the length volume, in the launch configuration the bench
    uses; sampled seeds against the FP64 oracle, FLEDGE against the oracle's
    Sobel on a sub-block."""
    ch = inputs.random_charges(8, 3)
    gf = inputs.charge_field(ch, 384, dtype=torch.float32, device="cuda", slab=32)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
    nx, ny, nz = 512, 512, 256
    N = nx * ny * nz
    q = torch.empty(N, device="cuda")
    L = torch.empty(N, device="cuda")
    faces = torch.empty(2 * N, dtype=torch.uint8, device="cuda")
    st = torch.empty(N, dtype=torch.uint8, device="cuda")
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL, integrator=qsl.QSL_DOPRI5_CELL)
    qsl.qsl_q_volume_3d(F, BOX_LO, BOX_HI, nx, ny, nz, o, q, L, faces, st)
    S = torch.empty((nz, ny, nx), device="cuda")
    qsl.qsl_fledge(L.view(nz, ny, nx), S)
    torch.cuda.synchronize()
    idx = inputs.subsample(N, 120, 11)
    g = inputs.GridField(*(a.cpu().numpy().astype(np.float64) for a in (gf.bx, gf.by, gf.bz)), gf.xc, gf.yc, gf.zc)
    del gf
    Fo = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    del g
    seeds = oracle_mod.volume_seeds(BOX_LO, BOX_HI, nx, ny, nz)[idx]
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    del Fo
    fc = faces.cpu().numpy().reshape(-1, 2)
    gd = {"q_perp": q.cpu().numpy()[idx], "L": L.cpu().numpy()[idx], "face_f": fc[idx, 0], "face_b": fc[idx, 1]}
    compare_lines(gd, ref, 1.0 / 383, BOX_LO, BOX_HI)
    # 3D FLEDGE on a block of the GPU length volume (the Sobel input is that same array)
    Lb = L.view(nz, ny, nx)[100:140, 200:260, 300:350].contiguous().cpu().numpy()
    Sb = S[101:139, 201:259, 301:349].cpu().numpy()
    want = oracle_mod.fledge(Lb)[1:-1, 1:-1, 1:-1]
    assert np.allclose(Sb, want, rtol=1e-4, atol=1e-4 * want.max())


@pytest.mark.parametrize("integ,prec,lanes", [(0, 0, 0), (2, 0, 1), (2, 0, 3), (0, 1, 0), (2, 1, 1), (2, 1, 3)])
def test_loops_from_the_bottom_face(qsl, oracle_mod, integ, prec, lanes):
    """Seeds on z = 0 whose lines curve back out through z = 0 within a fraction
    of a cell (chosen by the oracle): the end is the re-crossing, not the seed.
    Both kernels, FP32 and FP64."""
    n = 40
    gf = inputs.charge_field(inputs.random_charges(4, 3), n, dtype=torch.float32)
    Fo = _oracle_field(oracle_mod, gf, 0)
    xs = np.linspace(-0.99, 0.99, 160)
    s = np.stack(np.meshgrid(xs, xs, indexing="ij"), -1).reshape(-1, 2)
    cand = np.concatenate([s, np.zeros((len(s), 1))], 1)
    oo = oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11, nthreads=8)
    r = oracle_mod.trace_seeds(Fo, cand, oo)
    loop = (r["face_f"] == 4) & (r["face_b"] == 4) & (r["L"] > 0) & (r["L"] < 0.5 / (n - 1))
    seeds = cand[loop][:64]
    assert len(seeds) >= 8
    F = _gpu_field(qsl, gf, 0)
    tol = 1e-10 if prec else GPU_TOL
    o = qsl.qsl_opts_default(tol_abs=tol, tol_rel=tol, integrator=integ, precision=prec, line_lanes=lanes)
    rec = qsl.qsl_trace_seeds(F, seeds, o)
    ref = oracle_mod.trace_seeds(Fo, seeds, oo)
    assert np.all(rec["length"] > 0)
    compare_lines(_rec_to_dict(rec), ref, 1.0 / (n - 1), BOX_LO, BOX_HI)


@pytest.mark.parametrize("order,mode,prec", [(3, 1, 0), (3, 0, 0), (2, 1, 0), (3, 1, 1), (2, 0, 1)])
def test_higher_order_interpolation_matches_oracle(qsl, oracle_mod, order, mode, prec):
    """Triquadratic (2) and tricubic (3) interpolation (Sec. "Interpolation
    schemes") with the Cash-Karp tracer: Q, L and end faces against the oracle
    with the same kernels; FP32 at the parity bar, FP64 tightly."""
    ch = inputs.random_charges(4, 2)
    gf = inputs.charge_field(ch, 48, dtype=torch.float32)
    F = _gpu_field(qsl, gf, mode)
    g = inputs.to_numpy64(gf)
    Fo = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=mode, order=order)
    seeds = inputs.random_seeds(200, 19)
    seeds[:50, 2] = 0.0
    if prec:
        o = qsl.qsl_opts_default(tol_abs=1e-10, tol_rel=1e-10, precision=qsl.QSL_FP64, interp_order=order)
    else:
        o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL, interp_order=order)
    rec = qsl.qsl_trace_seeds(F, seeds, o)
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    kw = dict(q_rtol=2e-6, l_rtol=3e-7) if prec else {}
    rep = compare_lines(_rec_to_dict(rec), ref, 1.0 / 47, BOX_LO, BOX_HI, **kw)
    assert rep["q_checked"] > 120
    # the interpolation order matters: trilinear gives visibly different Q here
    tri = qsl.qsl_trace_seeds(F, seeds, qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL))
    ok = np.isfinite(ref["q_perp"]) & (ref["q_perp"] < 1e6)
    assert np.median(np.abs(tri["q_perp"][ok] / ref["q_perp"][ok] - 1)) > 1e-4


def test_higher_order_euler_and_argument_checks(qsl, oracle_mod):
    gf = inputs.hyperbolic_field(24)
    F = _gpu_field(qsl, gf, 1)
    g = inputs.to_numpy64(gf)
    Fo = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=1, order=3)
    seeds = inputs.random_seeds(60, 8, margin=0.05)
    o = qsl.qsl_opts_default(integrator=qsl.QSL_EULER, euler_h=0.2, precision=qsl.QSL_FP64, interp_order=3)
    rec = qsl.qsl_trace_seeds(F, seeds, o)
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(integrator=1, euler_h=0.2))
    compare_lines(_rec_to_dict(rec), ref, 1.0 / 23, BOX_LO, BOX_HI, q_rtol=1e-9, l_rtol=2e-7)
    for bad in (dict(interp_order=4), dict(interp_order=3, integrator=qsl.QSL_DOPRI5_CELL)):
        with pytest.raises(qsl.QslError) as e:
            qsl.qsl_trace_seeds(F, seeds, qsl.qsl_opts_default(**bad))
        assert e.value.code == qsl.QSL_EINVAL
    ax = np.array([0.0, 0.1, 0.3, 0.6, 1.0])
    b = np.ones((5, 5, 5))
    Fn = qsl.qsl_load_field(b, b, b, ax, ax, ax, qsl.QSL_RAW_B)
    with pytest.raises(qsl.QslError) as e:
        qsl.qsl_trace_seeds(Fn, np.array([[0.5, 0.5, 0.5]]), qsl.qsl_opts_default(interp_order=2))
    assert e.value.code == qsl.QSL_EINVAL


@pytest.mark.parametrize("mode,lanes", [(0, 1), (0, 3), (1, 1), (1, 3)])
def test_length_only_matches_oracle(qsl, oracle_mod, mode, lanes):
    """Lengths only (qsl_opts.length_only, the mode of the refinement passes)
    on the cell-wise kernels, which evaluate the cell's trilinear polynomial:
    one lane per line (for a launch this small the kernel of the refinement
    passes) and the queue-refilled three-lane kernel. Lengths and end faces
    against the oracle's lengths-only trace; Q outputs are NaN."""
    ch = inputs.random_charges(4, 2)
    gf = inputs.charge_field(ch, 64, dtype=torch.float32)
    F = _gpu_field(qsl, gf, mode)
    Fo = _oracle_field(oracle_mod, gf, mode)
    seeds = inputs.random_seeds(600, 41)
    seeds[:200, 2] = 0.0     # footpoints on the bottom face
    seeds[200:210, 1] = -1.0  # on the y- face
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL, integrator=qsl.QSL_DOPRI5_CELL, line_lanes=lanes,
                             length_only=1)
    rec = qsl.lines_to_numpy(qsl.qsl_trace_seeds(F, torch.as_tensor(seeds).cuda(), o))
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11, length_only=1))
    assert np.all(np.isnan(rec["q_perp"])) and np.all(np.isnan(ref["q_perp"]))
    rep = compare_lines(_rec_to_dict(rec), ref, 1.0 / 63, BOX_LO, BOX_HI)
    assert rep["labels_checked"] > 550
    assert np.array_equal(rec["status_f"], ref["st_f"]) and np.array_equal(rec["status_b"], ref["st_b"])


@pytest.mark.parametrize("mode,tol", [(0, 1e-5), (0, 1e-7), (1, 1e-5)])
def test_cash_karp_decision_lengths_match_oracle(qsl, oracle_mod, mode, tol):
    """The refinement passes' decision tracer (lengths only, the Cash-Karp
    stepper across cells, step cap 4 smallest spacings) against the oracle's
    lengths-only Cash-Karp trace with the same tolerance and step cap: the
    same method in FP64. End faces equal; lengths within the length bar where
    the cap sets the steps (tol 1e-5), within D_RTOL where the error estimate
    sets some of them (tol 1e-7: the two runs step differently near faces)."""
    from gpu_helpers import D_RTOL
    ch = inputs.random_charges(4, 2)
    gf = inputs.charge_field(ch, 64, dtype=torch.float32)
    F = _gpu_field(qsl, gf, mode)
    Fo = _oracle_field(oracle_mod, gf, mode)
    seeds = inputs.random_seeds(600, 47)
    seeds[:200, 2] = 0.0
    o = qsl.qsl_opts_default(tol_abs=tol, tol_rel=tol, integrator=qsl.QSL_RKCK54, length_only=1, h_max=4.0)
    rec = qsl.lines_to_numpy(qsl.qsl_trace_seeds(F, torch.as_tensor(seeds).cuda(), o))
    ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=tol, tol_rel=tol, length_only=1,
                                                                    h_max=4.0))
    assert np.all(np.isnan(rec["q_perp"]))
    rep = compare_lines(_rec_to_dict(rec), ref, 1.0 / 63, BOX_LO, BOX_HI, l_rtol=L_RTOL if tol >= 1e-5 else D_RTOL)
    assert rep["labels_checked"] > 550


@pytest.mark.parametrize("integ,lanes,len_only", [(0, 0, 0), (2, 1, 0), (2, 3, 0), (0, 0, 1), (2, 1, 1)])
def test_watchdog_expires_and_handle_stays_usable(qsl, oracle_mod, integ, lanes, len_only):
    """The device watchdog (qsl_opts.timeout_s): with a limit of one
    microsecond every tracer kernel stops its lines after its next check (every
    64 loop iterations), lines still running end with QSL_LINE_TIMEOUT,
    qsl_last_stats reports QSL_ETIMEOUT, and the next call on the same field
    handle runs to completion. Nothing waits on anything: the kernels only
    return early. Lengths only (len_only): the one-lane Cash-Karp and
    cell-wise kernels of the refinement passes."""
    ch = inputs.random_charges(4, 2)
    gf = inputs.charge_field(ch, 64, dtype=torch.float32)
    F = _gpu_field(qsl, gf, 0)
    seeds = inputs.random_seeds(4000, 43)
    seeds[:, 2] = 0.0
    sd = torch.as_tensor(seeds).cuda()
    o = qsl.qsl_opts_default(tol_abs=1e-9, tol_rel=1e-9, integrator=integ, line_lanes=lanes, retrace_q=0.0,
                             timeout_s=1e-6, length_only=len_only)
    rec = qsl.lines_to_numpy(qsl.qsl_trace_seeds(F, sd, o))
    with pytest.raises(qsl.QslError) as e:
        qsl.qsl_last_stats()
    assert e.value.code == qsl.QSL_ETIMEOUT
    st = np.concatenate([rec["status_f"], rec["status_b"]])
    assert np.sum(st == qsl.QSL_LINE_TIMEOUT) > 100
    assert np.all((st == qsl.QSL_LINE_TIMEOUT) | (st == qsl.QSL_LINE_OK))
    timed = (rec["status_f"] == qsl.QSL_LINE_TIMEOUT) | (rec["status_b"] == qsl.QSL_LINE_TIMEOUT)
    assert np.all(rec["face_f"][rec["status_f"] == qsl.QSL_LINE_TIMEOUT] == qsl.QSL_NO_FACE)
    o.timeout_s = 0.0
    rec2 = qsl.lines_to_numpy(qsl.qsl_trace_seeds(F, sd, o))
    qsl.qsl_last_stats()  # no watchdog: no error
    assert np.all(rec2["status_f"] == qsl.QSL_LINE_OK) and np.all(rec2["status_b"] == qsl.QSL_LINE_OK)
    # lines the watchdog did not reach are the same as without it
    done = ~timed
    assert done.sum() > 0
    assert np.array_equal(rec["face_f"][done], rec2["face_f"][done])
    assert np.allclose(rec["length"][done], rec2["length"][done], rtol=1e-6)


def test_fp64_newton_reciprocals_match_cuda(qsl):
    """The FP64 Newton-Raphson reciprocal square root and reciprocal of the
    field pack and the Q assembly against CUDA's 1 / sqrt(x) and 1 / x, over
    values log-uniform on 1e-35..1e35 (both sides of the FP32 range, where the
    FP64 operations take over) and powers of two and their neighbours."""
    rng = np.random.default_rng(5)
    x = 10.0 ** rng.uniform(-35, 35, 200000)
    p2 = 2.0 ** np.arange(-99, 100)
    x = np.concatenate([x, p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), [1.0, 3.0, 0.5]])
    r = qsl.qsl_check_fp64_newton(x)
    print("max ulps:", r)
    assert r["rsqrt_ulp"] <= 2.0 and r["rcp_ulp"] <= 2.0
