"""GPU parity of FLEDGE (Sobel), the Hilbert curve, the converter and the
refinement driver against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_1609_00724_gb300 import inputs
from gpu_helpers import D_RTOL, GPU_TOL, L_RTOL, Q_RTOL, length_err, min_spacing

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsl():
    from paper_1609_00724_gb300 import qsl as q
    q.lib()
    return q


@pytest.mark.parametrize("ndim,bits", [(2, 1), (2, 10), (2, 16), (2, 31), (3, 1), (3, 7), (3, 10), (3, 21)])
def test_hilbert_bit_exact(qsl, oracle_mod, ndim, bits):
    rng = np.random.default_rng(bits * 10 + ndim)
    n = 3000
    coords = rng.integers(0, 1 << bits, size=(n, ndim), dtype=np.uint64).astype(np.uint32)
    keys = np.zeros(n, dtype=np.uint64)
    qsl.qsl_hilbert_encode(coords, ndim, bits, keys)
    want = np.array([oracle_mod.hilbert_key(tuple(c), ndim, bits) for c in coords[:400]], dtype=np.uint64)
    assert np.array_equal(keys[:400], want)
    back = np.zeros_like(coords)
    qsl.qsl_hilbert_decode(keys, ndim, bits, back)
    assert np.array_equal(back, coords)
    # device memory path
    kd = torch.zeros(n, dtype=torch.int64, device="cuda")
    qsl.qsl_hilbert_encode(torch.as_tensor(coords.astype(np.int32)).cuda(), ndim, bits, kd)
    assert np.array_equal(kd.cpu().numpy().view(np.uint64), keys)


@pytest.mark.parametrize("shape", [(77, 1003), (1, 5), (37, 50, 41), (3, 2, 65)])
def test_fledge_matches_oracle(qsl, oracle_mod, shape):
    rng = np.random.default_rng(len(shape) * 100 + shape[-1])
    L = rng.uniform(0, 3, size=shape).astype(np.float32)
    L.reshape(-1)[rng.integers(0, L.size, size=max(1, L.size // 200))] = np.nan
    want = oracle_mod.fledge(L)
    got = np.zeros(shape, dtype=np.float32)
    qsl.qsl_fledge(L, got)
    assert np.allclose(got, want, rtol=1e-5, atol=1e-5 * np.nanmax(want))
    gd = torch.empty(shape, device="cuda")
    qsl.qsl_fledge(torch.as_tensor(L).cuda(), gd)
    assert np.allclose(gd.cpu().numpy(), want, rtol=1e-5, atol=1e-5 * np.nanmax(want))


@pytest.mark.parametrize("ndim,p,ext,out_order", [(2, 6, (64, 64), 6), (2, 6, (64, 48), 4), (3, 4, (16, 16, 8), 3),
                                                  (3, 5, (32, 32, 32), 5)])
def test_converter_matches_oracle(qsl, oracle_mod, ndim, p, ext, out_order):
    rng = np.random.default_rng(p + ndim)
    ncell = int(np.prod(ext))
    cells = rng.choice(ncell, size=ncell // 7, replace=False)
    coords = []
    for c in cells:
        cc = []
        for a in range(ndim):
            cc.append(c % ext[a])
            c //= ext[a]
        coords.append(cc)
    coords = np.array(coords, dtype=np.uint32)
    keys = np.zeros(len(coords), dtype=np.uint64)
    qsl.qsl_hilbert_encode(coords, ndim, p, keys)
    keys = np.sort(keys)
    vals = rng.uniform(2, 1e4, size=len(keys)).astype(np.float32)
    for log_interp in (True, False):
        want = oracle_mod.convert(keys, vals.astype(np.float64), ndim, p, list(ext) + [0] * (3 - ndim), out_order,
                                  log_interp)
        got = np.zeros(want.shape, dtype=np.float32)
        qsl.qsl_convert(keys, vals, ndim, p, list(ext), out_order, log_interp, got)
        assert np.allclose(got, want, rtol=2e-6), np.abs(got / want - 1).max()


def _fields(qsl, oracle_mod, n=48, seed=2, mode=0):
    ch = inputs.random_charges(4, seed)
    gf = inputs.charge_field(ch, n, dtype=torch.float32)
    F = qsl.qsl_load_field(gf.bx.cuda(), gf.by.cuda(), gf.bz.cuda(), gf.xc, gf.yc, gf.zc, interp_mode=mode)
    g = inputs.to_numpy64(gf)
    Fo = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=mode)
    Fo.cell = min_spacing(gf)
    return F, Fo


def _alloc(cap, dev="cuda"):
    return {"key": torch.zeros(cap, dtype=torch.int64, device=dev), "q": torch.zeros(cap, device=dev),
            "L": torch.zeros(cap, device=dev), "faces": torch.zeros(2 * cap, dtype=torch.uint8, device=dev),
            "st": torch.zeros(cap, dtype=torch.uint8, device=dev)}


def _positions(qsl, keys, spec):
    nd, p = spec.ndim, spec.max_order
    c = np.zeros((len(keys), nd), dtype=np.uint32)
    qsl.qsl_hilbert_decode(keys, nd, p, c)
    ext = [spec.extent[a] or (1 << p) for a in range(nd)]
    if nd == 2:
        a = (c[:, 0] + 0.5) / ext[0] - 0.5
        b = (c[:, 1] + 0.5) / ext[1] - 0.5
        return np.array(spec.center)[None] + a[:, None] * np.array(spec.u)[None] + b[:, None] * np.array(spec.v)[None]
    lo, hi = np.array(spec.lo), np.array(spec.hi)
    return lo[None] + (c + 0.5) / np.array(ext)[None] * (hi - lo)[None]


def test_refine_dense_and_values(qsl, oracle_mod):
    """tau < 0 without the shifted pass: every cell between the first and last
    coarse sample along the curve; each traced value matches the oracle."""
    F, Fo = _fields(qsl, oracle_mod)
    sp = qsl.refine_spec(ndim=2, coarse_order=3, max_order=5, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), tau=-1.0,
                         shift=0)
    b = _alloc(1024)
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL)
    n, iters, traced, rc = qsl.qsl_refine(F, sp, o, b["key"], b["q"], b["L"], b["faces"], b["st"])
    keys = b["key"].cpu().numpy()[:n].view(np.uint64)
    spo = oracle_mod.refine_spec(ndim=2, coarse_order=3, max_order=5, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0),
                                 tau=-1.0, shift=0)
    ref = oracle_mod.refine_fn(lambda x: (np.ones(len(x)), np.zeros(len(x))), spo)  # sample set only
    k0, k1 = int(ref["key"].min()), int(ref["key"].max())
    assert traced == n
    assert list(keys) == list(range(k0, k1 + 1))
    pos = _positions(qsl, keys, sp)
    r = oracle_mod.trace_seeds(Fo, pos, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    q = b["q"].cpu().numpy()[:n]
    L = b["L"].cpu().numpy()[:n]
    ok = np.isfinite(r["q_perp"]) & (r["q_perp"] < 1e6)
    assert np.all(np.abs(q[ok] / r["q_perp"][ok] - 1) <= Q_RTOL)
    good = np.isfinite(r["L"])
    assert np.all(length_err(L[good], r["L"][good], Fo.cell) <= L_RTOL)


def _refine_case(ndim):
    if ndim == 2:
        return dict(ndim=2, coarse_order=4, max_order=7, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0),
                    tau=0.05), 128 * 128
    return dict(ndim=3, coarse_order=2, max_order=4, extent=(16, 16, 8), lo=(-1, -1, 0), hi=(1, 1, 1),
                tau=0.05), 16 * 16 * 8


def _gpu_refine(qsl, F, kw, cap, o):
    """qsl_refine through the C ABI; returns host copies of the sample set with
    the pass that added each sample."""
    b = _alloc(cap)
    org = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    n, iters, traced, rc = qsl.qsl_refine(F, qsl.refine_spec(**kw), o, b["key"], b["q"], b["L"], b["faces"], b["st"],
                                          origin=org)
    assert rc == qsl.QSL_OK
    fa = b["faces"].cpu().numpy()[:2 * n].reshape(-1, 2)
    return {"key": b["key"].cpu().numpy()[:n].view(np.uint64).copy(), "q": b["q"].cpu().numpy()[:n],
            "L": b["L"].cpu().numpy()[:n], "face_f": fa[:, 0], "face_b": fa[:, 1],
            "origin": org.cpu().numpy()[:n], "iters": iters, "traced": traced}


class _Truth:
    """Oracle lines (tangent space, tol 1e-11) of the refinement samples it is
    asked for, remembered by key, so the replay and the comparison share one
    trace. A sample is marked undetermined when a seed moved by 1e-5 cells
    (ten times the GPU's position error, on the axes of the sample lattice)
    ends on other faces or with a length that jumps by more than 1e-3 of the
    line: its line runs along a separatrix within that distance (or grazes a
    face), so its end depends on the integration and no bar applies to it.

    `decide` (oracle opts, lengths only): the tracer of the GPU passes'
    decision lengths. Batches after the first (the coarse pass) then return
    the lengths of that trace, undetermined when the tangent-space line is or
    when the same perturbation changes the decision trace's end; the stored
    lines and their own undetermined flags stay the tangent-space ones."""

    def __init__(self, oracle_mod, Fo, ndim, decide=None):
        self.o, self.Fo, self.ndim = oracle_mod, Fo, ndim
        self.opts = oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11)
        self.opts_len = oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11, length_only=1)
        self.decide = decide
        self.lines = {}
        self.calls = 0

    def _unsure(self, x, r, opts):
        unsure = np.zeros(len(x), dtype=bool)
        d = 1e-5 * self.Fo.cell
        for ax in range(self.ndim):
            for sg in (1.0, -1.0):
                xp = x.copy()
                xp[:, ax] += sg * d
                rp = self.o.trace_seeds(self.Fo, xp, opts)
                unsure |= (rp["face_f"] != r["face_f"]) | (rp["face_b"] != r["face_b"])
                unsure |= ~(np.abs(rp["L"] - r["L"]) <= 1e-3 * np.maximum(r["L"], self.Fo.cell))
        return unsure

    def __call__(self, x, keys):
        r = self.o.trace_seeds(self.Fo, x, self.opts)
        unsure = self._unsure(x, r, self.opts_len)
        for i, k in enumerate(keys):
            self.lines[int(k)] = dict({name: r[name][i] for name in r}, unsure=bool(unsure[i]))
        first = self.calls == 0
        self.calls += 1
        if self.decide is None or first:
            return r["q_perp"], r["L"], unsure
        rd = self.o.trace_seeds(self.Fo, x, self.decide)
        return r["q_perp"], rd["L"], unsure | self._unsure(x, rd, self.decide)

    def records(self, keys):
        names = self.lines[int(keys[0])].keys()
        return {name: np.array([self.lines[int(k)][name] for k in keys]) for name in names}


def _determined(ref, n_max_frac=0.005):
    """Mask of the samples whose line the oracle determines; few are not."""
    un = ref["unsure"]
    print("undetermined samples (line along a separatrix within 1e-5 cells): %d of %d" % (un.sum(), len(un)))
    assert un.sum() <= max(2, n_max_frac * len(un))
    return ~un


def _band(cell, rtol=L_RTOL):
    """Band of the threshold within which a refinement decision may differ
    between the GPU and the oracle: each length is within rtol max(L, cell) of
    the oracle's, so a pair's |dL| within 2 rtol (max L + cell)."""
    return 2 * rtol * cell, 2 * rtol


def _check_replay(oracle_mod, g, rep, what):
    """The replay's sample set (and the pass that added each sample) is the
    GPU's, key for key."""
    gk, rk = g["key"], rep["key"]
    only_g = np.setdiff1d(gk, rk)
    only_r = np.setdiff1d(rk, gk)
    print("%s: %d samples, %d iterations; replay %d samples; only GPU %d, only replay %d" % (
        what, len(gk), g["iters"], len(rk), len(only_g), len(only_r)))
    assert len(only_g) == 0 and len(only_r) == 0, (what, only_g[:8], only_r[:8])
    assert np.array_equal(rep["origin"], g["origin"]), what


@pytest.mark.parametrize("ndim", [2, 3])
def test_refine_length_only_decisions_replay_exactly(qsl, oracle_mod, ndim):
    """Lengths-only refinement (the mode of the refinement passes): (1) the
    oracle's refinement driver fed the GPU's own lengths makes the GPU's sample
    set, key for key and pass for pass (the flagging, midpoint, shifted-curve and
    merge logic is exact); (2) every GPU length is within the parity bar of the
    oracle's and the end faces are the oracle's; (3) the oracle's driver on its
    own lengths reproduces the GPU set once the pairs whose |dL| lies within the
    GPU's stated length error of tau are decided by the GPU's choice, so every
    key where the two sets differ comes from such a pair. The cell-wise
    integrator: the refinement passes trace lengths only with it alone (the
    Cash-Karp stepper across cell faces meets the length bar only in tangent
    space at this tolerance)."""
    from gpu_helpers import compare_lines
    F, Fo = _fields(qsl, oracle_mod, n=40, seed=3)
    kw, cap = _refine_case(ndim)
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL, length_only=1, integrator=qsl.QSL_DOPRI5_CELL)
    g = _gpu_refine(qsl, F, kw, cap, o)
    assert g["iters"] > 0 and g["traced"] == len(g["key"])
    spo = oracle_mod.refine_spec(**kw)
    own = dict(zip(g["key"].tolist(), g["L"].astype(np.float64).tolist()))
    exact = oracle_mod.refine_replay(lambda x, k: (np.full(len(k), np.nan), np.array([own.get(int(v), np.nan)
                                                                                     for v in k])), spo)
    _check_replay(oracle_mod, g, exact, "exact replay on GPU lengths")
    truth = _Truth(oracle_mod, Fo, ndim)
    ba, br = _band(Fo.cell)
    rep = oracle_mod.refine_replay(truth, spo, g["key"], g["origin"], band_abs=ba, band_rel=br)
    _check_replay(oracle_mod, g, rep, "replay on oracle lengths")
    ref = truth.records(g["key"])
    plain = oracle_mod.refine(Fo, spo, truth.opts)
    print("oracle's own refinement: %d samples (symmetric difference with the GPU set %d)" % (
        len(plain["key"]), len(np.setxor1d(plain["key"], g["key"]))))
    ok = _determined(ref)
    ref_len = {k: v[ok] for k, v in ref.items()}
    ref_len["q_perp"] = np.full(ok.sum(), np.nan)  # lengths only: no Q to compare
    compare_lines({k: v[ok] for k, v in g.items() if k in ("L", "face_f", "face_b")}, ref_len, Fo.cell,
                  (-1, -1, 0), (1, 1, 1))


@pytest.mark.parametrize("integrator,stepper", [("ck", 0), ("cell", 0), ("cell", 1), ("ck", 2)])
@pytest.mark.parametrize("ndim", [2, 3])
def test_refine_sample_set_matches_oracle(qsl, oracle_mod, ndim, integrator, stepper):
    """Default refinement (tangent-space coarse pass, lengths-only passes, one
    tangent-space trace of the pass samples): the oracle's driver on its own
    lines reproduces the GPU sample set key for key once the pairs within the
    stated length error of tau follow the GPU's choice; every sample's Q, L and
    end faces match the oracle's; the converted grids keep the sampled values.
    Pass decision tracers (spec.pass_stepper): 0, the default, lengths-only
    Cash-Karp across cells with a step cap of 4 spacings, replayed on the
    oracle's trace with the same settings and a band of the decision lengths'
    error (D_RTOL); 1 with the cell-wise integrator,
    its own lengths-only trace, replayed on the oracle's tight lines (it meets
    the length bar); 2 the tangent-space passes themselves."""
    from gpu_helpers import compare_lines
    F, Fo = _fields(qsl, oracle_mod, n=40, seed=3)
    kw, cap = _refine_case(ndim)
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL,
                             integrator=qsl.QSL_DOPRI5_CELL if integrator == "cell" else qsl.QSL_RKCK54)
    sp = qsl.refine_spec(pass_stepper=stepper, **kw)
    b = _alloc(cap)
    org = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    qg = torch.zeros(cap, device="cuda")
    lg = torch.zeros(cap, device="cuda")
    n, iters, traced, rc = qsl.qsl_refine(F, sp, o, b["key"], b["q"], b["L"], b["faces"], b["st"], q_grid=qg,
                                          l_grid=lg, origin=org)
    assert rc == qsl.QSL_OK
    keys = b["key"].cpu().numpy()[:n].view(np.uint64)
    assert np.all(np.diff(keys.astype(np.int64)) > 0)
    fa = b["faces"].cpu().numpy()[:2 * n].reshape(-1, 2)
    g = {"key": keys.copy(), "q_perp": b["q"].cpu().numpy()[:n], "L": b["L"].cpu().numpy()[:n], "face_f": fa[:, 0],
         "face_b": fa[:, 1], "origin": org.cpu().numpy()[:n], "iters": iters}
    spo = oracle_mod.refine_spec(**kw)
    decide = (oracle_mod.default_opts(tol_abs=GPU_TOL, tol_rel=GPU_TOL, length_only=1, h_max=4.0)
              if stepper == 0 else None)
    truth = _Truth(oracle_mod, Fo, ndim, decide)
    ba, br = _band(Fo.cell, D_RTOL if stepper == 0 else L_RTOL)
    rep = oracle_mod.refine_replay(truth, spo, keys, g["origin"], band_abs=ba, band_rel=br)
    _check_replay(oracle_mod, g, rep, "replay on oracle lines")
    st = qsl.qsl_last_refine_stats()
    assert (st["deferred_ms"] > 0) == (stepper == 0 or integrator == "cell" and stepper == 1)
    ref = truth.records(keys)
    ok = _determined(ref)
    compare_lines({k: v[ok] for k, v in g.items() if k in ("q_perp", "L", "face_f", "face_b")},
                  {k: v[ok] for k, v in ref.items()}, Fo.cell, (-1, -1, 0), (1, 1, 1))
    # converted grids keep the sampled values in their cells
    c = np.zeros((n, ndim), dtype=np.uint32)
    qsl.qsl_hilbert_decode(keys, ndim, sp.max_order, c)
    ext = [sp.extent[a] or (1 << sp.max_order) for a in range(ndim)]
    flat = c[:, 0].astype(np.int64) + ext[0] * c[:, 1].astype(np.int64)
    if ndim == 3:
        flat += ext[0] * ext[1] * c[:, 2].astype(np.int64)
    assert np.array_equal(lg.cpu().numpy()[flat], b["L"].cpu().numpy()[:n])
    # both grids (converted in one pass) equal qsl_convert of each sample array
    for vals, grid, log_interp in ((b["q"], qg, 1), (b["L"], lg, 0)):
        want = torch.full_like(grid, float("nan"))
        qsl.qsl_convert(b["key"][:n], vals[:n], ndim, sp.max_order, ext, sp.max_order, log_interp, want)
        w, gg = want.cpu().numpy(), grid.cpu().numpy()
        m = int(np.prod(ext))
        assert np.array_equal(np.isnan(w[:m]), np.isnan(gg[:m])) and np.array_equal(w[:m][~np.isnan(w[:m])],
                                                                                      gg[:m][~np.isnan(gg[:m])])


@pytest.mark.parametrize("stride", [1, 2])
def test_refine_proposal_traces_every_cell_of_flagged_coarse_cells(qsl, oracle_mod, stride):
    """Proposal step (one byte per coarse cell, x fastest) with no refinement
    iteration after it: the sample set is the coarse samples plus the
    effective cells of the flagged coarse cells at the proposal stride (every
    cell; every other cell per axis at offset 1), key for key (keys from the
    oracle's Hilbert curve), and the lines traced there match the oracle."""
    from gpu_helpers import compare_lines
    F, Fo = _fields(qsl, oracle_mod, n=40, seed=3)
    p0, p = 4, 6
    R, nc = 1 << (p - p0), 1 << p0
    mask = (np.random.default_rng(11).random(nc * nc) < 0.15).astype(np.uint8)
    mask[0] = mask[nc * nc - 1] = 1  # both ends of the coarse lattice
    kw = dict(ndim=2, coarse_order=p0, max_order=p, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), tau=0.05,
              max_iters=0)
    mask_dev = torch.as_tensor(mask).cuda()
    sp = qsl.refine_spec(proposal=mask_dev, proposal_stride=stride, **kw)
    cap = (nc * R) ** 2
    b = _alloc(cap)
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL)
    n, iters, traced, rc = qsl.qsl_refine(F, sp, o, b["key"], b["q"], b["L"], b["faces"], b["st"])
    assert rc == qsl.QSL_OK and iters == 0 and traced == n
    keys = b["key"].cpu().numpy()[:n].view(np.uint64)
    want = set()
    for j in range(nc):
        for i in range(nc):
            want.add(oracle_mod.hilbert_key((i * R + R // 2, j * R + R // 2), 2, p))
            if mask[i + nc * j]:
                for bb in range(stride // 2, R, stride):
                    for aa in range(stride // 2, R, stride):
                        want.add(oracle_mod.hilbert_key((i * R + aa, j * R + bb), 2, p))
    assert n == len(want) and list(keys) == sorted(want)
    # the lines: a seeded sample of the samples against the oracle
    idx = np.sort(np.random.default_rng(12).choice(n, 80, replace=False))
    pos = _positions(qsl, keys[idx], sp)
    ref = oracle_mod.trace_seeds(Fo, pos, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    fc = b["faces"].cpu().numpy()[:2 * n].reshape(-1, 2)[idx]
    gd = {"q_perp": b["q"].cpu().numpy()[:n][idx], "L": b["L"].cpu().numpy()[:n][idx], "face_f": fc[:, 0],
          "face_b": fc[:, 1]}
    compare_lines(gd, ref, Fo.cell, (-1, -1, 0), (1, 1, 1))


def test_refine_resume_capacity_and_host_path(qsl, oracle_mod):
    F, _ = _fields(qsl, oracle_mod, n=40, seed=5)
    kw = dict(ndim=2, coarse_order=4, max_order=7, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), tau=0.05)
    o = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6)
    full = _alloc(128 * 128)
    n_full, it_full, _, _ = qsl.qsl_refine(F, qsl.refine_spec(**kw), o, full["key"], full["q"], full["L"],
                                           full["faces"], full["st"])
    # resume: two iterations, then the rest
    part = _alloc(128 * 128)
    n1, it1, _, _ = qsl.qsl_refine(F, qsl.refine_spec(max_iters=2, **kw), o, part["key"], part["q"], part["L"],
                                   part["faces"], part["st"])
    assert it1 == 2 and n1 < n_full
    kw2 = dict(kw)
    n2, it2, _, _ = qsl.qsl_refine(F, qsl.refine_spec(**kw2), o, part["key"], part["q"], part["L"], part["faces"],
                                   part["st"], count=n1)
    # the shift alternates with the iteration index, so compare sets loosely
    assert n2 >= n1
    # capacity: a small buffer ends with QSL_ECAPACITY and sorted valid samples
    small = _alloc(300)
    ns, _, _, rc = qsl.qsl_refine(F, qsl.refine_spec(**kw), o, small["key"], small["q"], small["L"],
                                  small["faces"], small["st"])
    assert rc == qsl.QSL_ECAPACITY and ns <= 300
    ks = small["key"].cpu().numpy()[:ns].view(np.uint64)
    assert np.all(np.diff(ks.astype(np.int64)) > 0)
    # host memory path = device path
    h = {k: v.cpu().numpy() for k, v in _alloc(128 * 128, "cpu").items()}
    nh, ith, _, _ = qsl.qsl_refine(F, qsl.refine_spec(**kw), o, h["key"], h["q"], h["L"], h["faces"], h["st"])
    assert nh == n_full and ith == it_full
    assert np.array_equal(h["key"][:nh], full["key"].cpu().numpy()[:n_full])
    assert np.array_equal(h["L"][:nh], full["L"].cpu().numpy()[:n_full])


def test_refine_time_accounting(qsl, oracle_mod):
    """qsl_last_refine_stats: the parts of the last refine add up, and the line
    counts agree with what qsl_refine reports."""
    F, _ = _fields(qsl, oracle_mod, n=40, seed=3)
    sp = qsl.refine_spec(ndim=2, coarse_order=5, max_order=7, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), tau=0.05)
    b = _alloc(128 * 128)
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL, integrator=qsl.QSL_DOPRI5_CELL)
    n, iters, traced, rc = qsl.qsl_refine(F, sp, o, b["key"], b["q"], b["L"], b["faces"], b["st"])
    assert rc == qsl.QSL_OK
    st = qsl.qsl_last_refine_stats()
    assert st["iters"] == iters
    assert st["coarse_lines"] == 32 * 32
    assert st["coarse_lines"] + st["pass_lines"] == traced == n
    assert 1 <= st["passes"] <= 2 * max(iters, 1)
    assert st["deferred_ms"] > 0 and st["deferred_stage_evals"] > 0  # the tangent-space trace of pass samples
    assert st["total_ms"] > 0 and st["coarse_ms"] > 0
    assert st["coarse_ms"] + st["passes_ms"] + st["deferred_ms"] <= st["total_ms"] * 1.001
    assert st["coarse_stage_evals"] > 0 and (st["pass_stage_evals"] > 0) == (st["pass_lines"] > 0)
    # the pool's cached blocks go back to the driver; a later refine allocates again
    qsl.qsl_trim_pool()
    n2, _, _, rc2 = qsl.qsl_refine(F, sp, o, b["key"], b["q"], b["L"], b["faces"], b["st"])
    assert rc2 == qsl.QSL_OK and n2 == n


@pytest.mark.parametrize("ndim", [2, 3])
def test_refine_q_threshold_criterion_matches_oracle(qsl, oracle_mod, ndim):
    """The Q-threshold criterion (QSL_REFINE_Q_THRESHOLD): the oracle's driver
    on its own lines reproduces the GPU sample set key for key once the pairs
    whose Q lies within the Q parity bar of the threshold follow the GPU's
    choice; every sample matches the oracle's line; at termination no pair with
    a gap has a sample above the threshold."""
    from gpu_helpers import compare_lines
    F, Fo = _fields(qsl, oracle_mod, n=40, seed=3)
    kw, cap = _refine_case(ndim)
    thr = 30.0 if ndim == 2 else 10.0  # the 3D coarse samples stay below 30
    kw.update(criterion=qsl.QSL_REFINE_Q_THRESHOLD, q_threshold=thr)
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL)
    g = _gpu_refine(qsl, F, kw, cap, o)
    assert g["iters"] > 0
    assert len(g["key"]) > (1 << (kw["coarse_order"] * ndim)) * 1.05  # it refined
    spo = oracle_mod.refine_spec(**kw)
    truth = _Truth(oracle_mod, Fo, ndim)
    rep = oracle_mod.refine_replay(truth, spo, g["key"], g["origin"], band_rel=Q_RTOL / (1 - Q_RTOL))
    _check_replay(oracle_mod, g, rep, "replay on oracle Q")
    ref = truth.records(g["key"])
    ok = _determined(ref)
    gd = {"q_perp": g["q"][ok], "L": g["L"][ok], "face_f": g["face_f"][ok], "face_b": g["face_b"][ok]}
    compare_lines(gd, {k: v[ok] for k, v in ref.items()}, Fo.cell, (-1, -1, 0), (1, 1, 1))
    qa, keys = g["q"], g["key"]
    hot = (np.nan_to_num(qa[:-1]) > thr) | (np.nan_to_num(qa[1:]) > thr)
    gaps = np.diff(keys.astype(np.int64))
    if ndim == 2:  # full square lattice: every gap has cells to insert
        assert not np.any(hot & (gaps > 1) & (g["iters"] < kw.get("max_iters", 64)))


def test_bench_refined_map_full_size_sampled(qsl, oracle_mod):
    """The refined-map workload at full size in the settings the bench times
    after tuning (4 charges, seed 2, on 256^3 FP32; 1024^2 z = 0 map refined to
    4096^2; tol 1e-5, step cap 4 smallest spacings, 4 warps per block, 32
    blocks per SM, refill 8): coarse and refined samples against the FP64
    oracle, and FLEDGE of the converted length grid against the oracle's
    Sobel on a block."""
    from gpu_helpers import compare_lines
    gf = inputs.charge_field(inputs.random_charges(4, 2), 256, dtype=torch.float32, device="cuda", slab=32)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    sp = qsl.refine_spec(ndim=2, coarse_order=10, max_order=12, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0),
                         tau=0.05, shift=1, max_iters=64)
    o = qsl.qsl_opts_default(tol_abs=1e-5, tol_rel=1e-5, integrator=qsl.QSL_DOPRI5_CELL, h_max=4.0)
    o.warps_per_block, o.blocks_per_sm, o.refill_min = 4, 32, 8
    eff = 4096
    b = _alloc(eff * eff)
    qg = torch.empty(eff * eff, device="cuda")
    lg = torch.empty(eff * eff, device="cuda")
    n, iters, traced, rc = qsl.qsl_refine(F, sp, o, b["key"], b["q"], b["L"], b["faces"], b["st"], q_grid=qg,
                                          l_grid=lg)
    assert rc == qsl.QSL_OK and iters > 0 and n > 1024 * 1024
    S = torch.empty((eff, eff), device="cuda")
    qsl.qsl_fledge(lg.view(eff, eff), S)
    torch.cuda.synchronize()
    keys = b["key"].cpu().numpy()[:n].view(np.uint64)
    assert np.all(np.diff(keys.astype(np.int64)) > 0)
    # 150 coarse (index 2 modulo 4 on both axes) and 150 refined samples
    c = np.zeros((n, 2), dtype=np.uint32)
    qsl.qsl_hilbert_decode(keys, 2, 12, c)
    coarse = (c[:, 0] % 4 == 2) & (c[:, 1] % 4 == 2)
    assert coarse.sum() == 1024 * 1024
    ci = np.where(coarse)[0][inputs.subsample(int(coarse.sum()), 150, 31)]
    ri = np.where(~coarse)[0][inputs.subsample(int((~coarse).sum()), 150, 32)]
    idx = np.concatenate([ci, ri])
    pos = np.column_stack([(c[idx, 0] + 0.5) / eff * 2 - 1, (c[idx, 1] + 0.5) / eff * 2 - 1, np.zeros(len(idx))])
    g = inputs.GridField(*(a.cpu().numpy().astype(np.float64) for a in (gf.bx, gf.by, gf.bz)), gf.xc, gf.yc, gf.zc)
    del gf
    Fo = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    cell = min_spacing(g)
    del g
    ref = oracle_mod.trace_seeds(Fo, pos, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    fa = b["faces"].cpu().numpy()[:2 * n].reshape(-1, 2)
    gd = {"q_perp": b["q"].cpu().numpy()[:n][idx], "L": b["L"].cpu().numpy()[:n][idx], "face_f": fa[idx, 0],
          "face_b": fa[idx, 1]}
    compare_lines(gd, ref, cell, (-1, -1, 0), (1, 1, 1))
    # FLEDGE of the converted length grid on a block (Sobel input is that same grid)
    Lb = lg.view(eff, eff)[2000:2100, 1500:1620].contiguous().cpu().numpy()
    Sb = S[2001:2099, 1501:1619].cpu().numpy()
    want = oracle_mod.fledge(Lb)[1:-1, 1:-1]
    assert np.allclose(Sb, want, rtol=1e-5, atol=1e-6 * float(np.abs(Lb).max()))
