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
    # what the network gains: fewer sequential refinement iterations after the proposal
    assert it_l <= it_plain, (it_l, it_plain)
    # sample keys stay unique and sorted
    k = lrn.key[:n_l].cpu().numpy()
    assert np.all(np.diff(k) > 0)
