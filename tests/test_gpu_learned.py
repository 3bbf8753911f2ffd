"""GPU test of the learned refinement proposal at small scale: tracer-generated
training maps, training with the hand-written CNN kernels, calibration, and a
learned refinement (proposal traced in one launch, plain FLL-jump criterion as
fallback) against the plain refinement of a held-out field."""
import numpy as np
import pytest
import torch

from paper_1609_00724_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_learned_proposal_end_to_end():
    from paper_1609_00724_gb300 import learned, qsl
    o = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6, integrator=qsl.QSL_DOPRI5_CELL)
    # tau large enough that smooth length variation across one coarse cell
    # (spacing 2/64) does not trigger refinement
    X, Y, _ = learned.make_training_set(40, grid=64, coarse=64, levels=2, tau=0.15, seed0=6000, opts=o)
    assert 0.0 < float(Y.mean()) < 0.6, float(Y.mean())
    net, hist, pw = learned.train(X[:32], Y[:32], epochs=40, batch=8, lr=3e-3)
    assert hist[-1] < 0.7 * hist[0], hist
    thr, frac = learned.calibrate(net, X[32:], Y[32:], recall=0.99)
    assert 0 < thr < 1
    # held-out field
    gf = inputs.charge_field(inputs.random_charges(7, 6999), 64, dtype=torch.float32, device="cuda")
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
    spec = learned.plane_spec(64, 2, 0.15)
    cap = 256 * 256
    plain = learned.Samples(cap)
    n_plain, it_plain, tr_plain, _ = plain.refine(F, spec, o)
    # learned: coarse pass only, CNN proposal, then the plain criterion as fallback
    lrn = learned.Samples(cap)
    lrn.refine(F, learned.plane_spec(64, 2, 0.15, max_iters=0), o)
    L, Q, _ = learned.coarse_grids(lrn, 2, spec.max_order, 2, (64, 64))
    mask = learned.propose(net, learned.features(L, Q)[None], thr)[0].contiguous()
    n_l, it_l, tr_l, _ = lrn.refine(F, learned.plane_spec(64, 2, 0.15, proposal=mask), o)
    kp = set(plain.key[:n_plain].cpu().numpy().tolist())
    kl = set(lrn.key[:n_l].cpu().numpy().tolist())
    recall = len(kp & kl) / len(kp)
    assert recall >= 0.97, recall
    # (what the network gains is shown on the volume workload, at equal iterations, below)
    # sample keys stay unique and sorted
    k = lrn.key[:n_l].cpu().numpy()
    assert np.all(np.diff(k) > 0)


def test_config5_learned_volume_full_size_sampled(oracle_mod):
    """The learned-proposal workload at full size: an 8-charge field on 512^3,
    a 256 x 256 x 128 coarse cell-centre volume refined two orders (1024 x 1024
    x 512 effective) after a CNN proposal on its z-slices, with the plain
    criterion as fallback. The network here is a quick one (40 small training
    maps): what is checked is the tracer on this volume, on seeded samples of
    each kind (coarse, proposed, refinement passes) against the FP64 oracle."""
    from gpu_helpers import compare_lines
    from paper_1609_00724_gb300 import learned, qsl
    o = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6, integrator=qsl.QSL_DOPRI5_CELL)
    X, Y, _ = learned.make_training_set(40, grid=64, coarse=64, levels=2, tau=0.05, seed0=6100, opts=o)
    net, hist, pw = learned.train(X[:32], Y[:32], epochs=20, batch=8, lr=3e-3)
    thr, _ = learned.calibrate(net, X[32:], Y[32:], recall=0.99)
    gf = inputs.charge_field(inputs.random_charges(8, 5), 512, dtype=torch.float32, device="cuda", slab=16)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
    coarse = (256, 256, 128)
    cap = 96 * 1024 * 1024
    smp = learned.Samples(cap)
    org = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    spec0 = learned.volume_spec(coarse, 2, 0.05, max_iters=0)
    n0, _, _, rc = qsl.qsl_refine(F, spec0, o, smp.key, smp.q, smp.L, smp.faces, smp.status, 0, origin=org)
    assert rc == qsl.QSL_OK and n0 == 256 * 256 * 128
    smp.count = n0
    Lc, Qc, _ = learned.coarse_grids(smp, 3, spec0.max_order, 2, coarse[::-1])
    budget = int(0.8 * (cap - n0) / 64)
    mask = learned.propose(net, learned.features_slices(Lc, Qc), thr, budget=budget).contiguous()
    assert 0 < int(mask.sum().item()) <= budget
    spec = learned.volume_spec(coarse, 2, 0.05, proposal=mask)
    n, iters, traced, rc = qsl.qsl_refine(F, spec, o, smp.key, smp.q, smp.L, smp.faces, smp.status, n0, origin=org)
    assert rc == qsl.QSL_OK and n > n0 and iters > 0
    keys = smp.key[:n].cpu().numpy().view(np.uint64)
    assert np.all(np.diff(keys.astype(np.int64)) > 0)
    og = org[:n].cpu().numpy()
    c = np.zeros((n, 3), dtype=np.uint32)
    qsl.qsl_hilbert_decode(keys, 3, spec.max_order, c)
    on_coarse = np.all((c % 4) == 2, axis=1)
    kinds = {"coarse": np.where(on_coarse)[0], "proposed": np.where(~on_coarse & (og == 0))[0],
             "passes": np.where(og > 0)[0]}
    idx = np.concatenate([v[inputs.subsample(len(v), min(60, len(v)), 40 + j)] for j, v in enumerate(kinds.values())])
    assert len(kinds["proposed"]) > 0 and len(kinds["passes"]) > 0
    ext = np.array([1024, 1024, 512])
    lo, hi = np.array([-1.0, -1.0, 0.0]), np.array([1.0, 1.0, 1.0])
    pos = lo[None] + (c[idx] + 0.5) / ext[None] * (hi - lo)[None]
    g = inputs.to_numpy64(gf)
    del gf
    Fo = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    del g
    ref = oracle_mod.trace_seeds(Fo, pos, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
    fa = smp.faces[:2 * n].view(-1, 2).cpu().numpy()
    gd = {"q_perp": smp.q[:n].cpu().numpy()[idx], "L": smp.L[:n].cpu().numpy()[idx], "face_f": fa[idx, 0],
          "face_b": fa[idx, 1]}
    rep = compare_lines(gd, ref, 1.0 / 511, tuple(lo), tuple(hi))
    assert rep["q_checked"] > 100


def _qsl_cells(smp, spec, ext):
    """Output cells (one order below the sample lattice) holding a sample with Q >= 100."""
    hot = torch.nan_to_num(smp.q[:smp.count], nan=0.0) >= 100.0
    cc = smp.coords(3, spec.max_order)[hot] >> 1
    eo = [e >> 1 for e in ext]
    return torch.unique(cc[:, 0] + eo[0] * (cc[:, 1] + eo[1] * cc[:, 2]))


def test_learned_volume_gains_over_the_plain_criterion_at_equal_iterations():
    """What the trained network gains (volume workload at small scale, the
    setting of the learned bench): trained on z-slices of tracer-generated
    volumes, calibrated on held-out QSL samples, its dilated proposal plus two
    fallback iterations recalls at least 99 % of the QSL pixels of the plain
    criterion run to convergence (output cells holding a plain sample with
    Q >= 100), strictly more than the plain criterion stopped after the same
    two iterations, and with fewer sequential iterations than the plain run
    needs."""
    from paper_1609_00724_gb300 import learned, qsl
    o = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6, integrator=qsl.QSL_DOPRI5_CELL)
    tr = (32, 32, 16)
    X, Y, W, _ = learned.make_training_volumes(40, grid=64, coarse=tr, levels=2, tau=0.05, seed0=7000, opts=o)
    n_fit = 32 * tr[2]
    net, hist, pw = learned.train(X[:n_fit], Y[:n_fit], epochs=30, batch=16, lr=3e-3)
    assert hist[-1] < 0.8 * hist[0], hist
    thr, frac, rec = learned.calibrate_qsl(net, X[n_fit:], W[n_fit:], tr[2], recall=0.995, dilate=True)
    assert rec >= 0.995 and frac < 0.9, (thr, frac, rec)
    gf = inputs.charge_field(inputs.random_charges(8, 7999), 64, dtype=torch.float32, device="cuda")
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
    spec = learned.volume_spec(tr, 2, 0.05)
    ext = [c * 4 for c in tr]
    cap = int(np.prod(ext))
    plain = learned.Samples(cap)
    n_p, it_p, _, _ = plain.refine(F, spec, o)
    cells = _qsl_cells(plain, spec, ext)
    assert cells.numel() > 50
    K = 2
    assert it_p > K + 1, it_p

    def recall(smp):
        q = learned.converted_q(smp, 3, spec.max_order, ext, spec.max_order - 1).reshape(-1)
        return float((torch.nan_to_num(q[cells], nan=0.0) >= 100.0).float().mean().item())

    trunc = learned.Samples(cap)
    trunc.refine(F, learned.volume_spec(tr, 2, 0.05, max_iters=K), o)
    lrn = learned.Samples(cap)
    lrn.refine(F, learned.volume_spec(tr, 2, 0.05, max_iters=0), o)
    L, Q, _ = learned.coarse_grids(lrn, 3, spec.max_order, 2, tr[::-1])
    mask = learned.propose(net, learned.features_slices(L, Q), thr, dilate=True)
    n_l, it_l, _, _ = lrn.refine(F, learned.volume_spec(tr, 2, 0.05, proposal=mask, max_iters=K), o)
    r_l, r_t = recall(lrn), recall(trunc)
    print("QSL-pixel recall: learned %.4f (%d samples), plain stopped after %d iterations %.4f (%d samples), "
          "plain to convergence %d iterations (%d samples); proposed %.3f of the coarse cells" % (
              r_l, n_l, K, r_t, trunc.count, it_p, n_p, float(mask.float().mean().item())))
    assert r_l >= 0.99 and r_l > r_t and it_l <= K < it_p
