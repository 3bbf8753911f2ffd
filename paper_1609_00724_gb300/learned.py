"""Learned refinement proposal: a CNN that predicts, from a coarse Q/FLL map,
which coarse cells the FLL-jump refinement (Sec. "Adaptive refinements") will
sample, so that those cells are traced in one launch before the plain
criterion runs as the fallback.

Pipeline (every computation runs in libqsl.so kernels; torch holds device
memory and does index bookkeeping):
* training data: coarse cell-centre volumes of random 4-12-charge fields,
  refined by the plain criterion; each z-slice is one example, with input
  (FLEDGE / max FLEDGE of the slice, (log10 Q - 2) / 2) of the coarse volume,
  label = coarse cells that received refined samples, and weight = the number
  of samples with Q >= 100 (QSL samples) of the plain run in each cell;
* training: mean BCE with a positive-class weight, Adam, BF16 weights;
* inference: coarse volume -> per-slice CNN -> probability per coarse cell ->
  threshold -> 3 x 3 x 3 dilation -> proposal mask; the threshold is the
  largest whose dilated mask holds the required fraction of the held-out
  QSL samples.
"""
import math
import time

import numpy as np
import torch

from . import inputs, qsl

NPARAMS = 32 * 2 * 9 + 32 + 32 * 32 * 9 + 32 + 32 * 9 + 1


def init_params(seed):
    """Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for cout, cin in ((32, 2), (32, 32), (1, 32)):
        bound = math.sqrt(6.0 / (cin * 9))
        parts.append(rng.uniform(-bound, bound, size=cout * cin * 9))
        parts.append(np.zeros(cout))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == NPARAMS
    return p


def plane_spec(coarse, levels, tau, shift=1, max_iters=64, proposal=None, proposal_stride=1):
    p0 = int(round(math.log2(coarse)))
    return qsl.refine_spec(ndim=2, coarse_order=p0, max_order=p0 + levels, center=(0, 0, 0), u=(2, 0, 0),
                           v=(0, 2, 0), tau=tau, shift=shift, max_iters=max_iters, proposal=proposal,
                           proposal_stride=proposal_stride)


def volume_spec(coarse_xyz, levels, tau, lo=(-1, -1, 0), hi=(1, 1, 1), max_iters=64, proposal=None,
                proposal_stride=1):
    R = 1 << levels
    p0 = int(round(math.log2(max(coarse_xyz))))
    ext = [c * R for c in coarse_xyz]
    return qsl.refine_spec(ndim=3, coarse_order=p0, max_order=p0 + levels, extent=ext, lo=lo, hi=hi, tau=tau,
                           max_iters=max_iters, proposal=proposal, proposal_stride=proposal_stride)


class Samples:
    """Device sample arrays for qsl_refine."""

    def __init__(self, capacity, device="cuda"):
        self.key = torch.zeros(capacity, dtype=torch.int64, device=device)
        self.q = torch.zeros(capacity, device=device)
        self.L = torch.zeros(capacity, device=device)
        self.faces = torch.zeros(2 * capacity, dtype=torch.uint8, device=device)
        self.status = torch.zeros(capacity, dtype=torch.uint8, device=device)
        self.count = 0

    def refine(self, field, spec, opts, count=None):
        n, iters, traced, rc = qsl.qsl_refine(field, spec, opts, self.key, self.q, self.L, self.faces, self.status,
                                              self.count if count is None else count)
        self.count = n
        return n, iters, traced, rc

    def coords(self, ndim, bits):
        """Decoded lattice coordinates (int64, count x ndim) of the samples."""
        c = torch.zeros((self.count, ndim), dtype=torch.int32, device=self.key.device)
        qsl.qsl_hilbert_decode(self.key[:self.count], ndim, bits, c)
        return c.long()


def coarse_grids(smp, ndim, max_order, levels, coarse_shape):
    """Coarse-lattice L and Q (and a mask of refined cells) from a sample set.
    coarse_shape is (ny, nx) or (nz, ny, nx); coarse samples sit at index
    R/2 modulo R (R = 2^levels) on every axis."""
    R = 1 << levels
    c = smp.coords(ndim, max_order)
    on = torch.ones(c.shape[0], dtype=torch.bool, device=c.device)
    for a in range(ndim):
        on &= (c[:, a] % R) == (R // 2)
    cc = c // R
    flat = cc[:, 0]
    mult = 1
    shape_xyz = list(coarse_shape)[::-1]
    for a in range(1, ndim):
        mult *= shape_xyz[a - 1]
        flat = flat + cc[:, a] * mult
    n = int(np.prod(coarse_shape))
    L = torch.full((n,), float("nan"), device=c.device)
    Q = torch.full((n,), float("nan"), device=c.device)
    L[flat[on]] = smp.L[:smp.count][on]
    Q[flat[on]] = smp.q[:smp.count][on]
    refined = torch.zeros(n, dtype=torch.float32, device=c.device)
    refined[flat[~on]] = 1.0
    return L.view(coarse_shape), Q.view(coarse_shape), refined.view(coarse_shape)


def features(L2d, Q2d):
    """CNN input [2, H, W] from coarse L and Q maps (device tensors)."""
    S = torch.empty_like(L2d)
    qsl.qsl_fledge(L2d.contiguous(), S)
    X = torch.empty((1, 2) + tuple(L2d.shape), device=L2d.device)
    qsl.qsl_cnn_features(S, Q2d.contiguous(), X)
    return X[0]


def features_slices(L3, Q3):
    """Per z-slice features [nz, 2, ny, nx] of a coarse volume (3D FLEDGE
    sliced, log10 Q)."""
    S = torch.empty_like(L3)
    qsl.qsl_fledge(L3.contiguous(), S)
    X = torch.empty((L3.shape[0], 2) + tuple(L3.shape[1:]), device=L3.device)
    qsl.qsl_cnn_features(S, Q3.contiguous(), X)
    return X


def qsl_counts(smp, ndim, max_order, levels, coarse_shape, q_qsl=100.0):
    """Number of samples with Q >= q_qsl (QSL samples) in each coarse cell."""
    R = 1 << levels
    c = smp.coords(ndim, max_order)
    cc = c // R
    flat = cc[:, 0]
    mult = 1
    shape_xyz = list(coarse_shape)[::-1]
    for a in range(1, ndim):
        mult *= shape_xyz[a - 1]
        flat = flat + cc[:, a] * mult
    hot = torch.nan_to_num(smp.q[:smp.count], nan=0.0) >= q_qsl
    W = torch.zeros(int(np.prod(coarse_shape)), dtype=torch.float32, device=c.device)
    W.index_add_(0, flat[hot], torch.ones(int(hot.sum().item()), device=c.device))
    return W.view(coarse_shape)


def make_training_volumes(n_vol, grid=128, coarse=(64, 64, 32), levels=2, tau=0.05, seed0=5000, opts=None,
                          device="cuda", charges=(4, 12), log_every=0):
    """Tracer-generated training slices: volume i is the coarse cell-centre
    lattice `coarse` (x, y, z) of a field with k ~ U{charges} charges (seed
    seed0 + i) on grid^3, refined `levels` orders by the plain criterion.
    Returns X [n_vol * nz, 2, ny, nx], Y [.., ny, nx] (refined cells), W [..]
    (QSL samples per cell), all device tensors, and the time spent."""
    if opts is None:
        opts = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6, integrator=qsl.QSL_DOPRI5_CELL)
    nx, ny, nz = coarse
    X = torch.empty((n_vol * nz, 2, ny, nx), device=device)
    Y = torch.empty((n_vol * nz, ny, nx), device=device)
    W = torch.empty((n_vol * nz, ny, nx), device=device)
    R = 1 << levels
    smp = Samples(nx * ny * nz * R ** 3, device)
    spec = volume_spec(coarse, levels, tau)
    t0 = time.perf_counter()
    for i in range(n_vol):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        k = int(rng.integers(charges[0], charges[1] + 1))
        gf = inputs.charge_field(inputs.random_charges(k, seed0 + i), grid, dtype=torch.float32, device=device)
        F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
        del gf
        smp.count = 0
        smp.refine(F, spec, opts)
        L, Q, refined = coarse_grids(smp, 3, spec.max_order, levels, (nz, ny, nx))
        X[i * nz:(i + 1) * nz] = features_slices(L, Q)
        Y[i * nz:(i + 1) * nz] = refined
        W[i * nz:(i + 1) * nz] = qsl_counts(smp, 3, spec.max_order, levels, (nz, ny, nx))
        del F
        if log_every and (i + 1) % log_every == 0:
            print("training volumes: %d / %d" % (i + 1, n_vol), flush=True)
    torch.cuda.synchronize()
    return X, Y, W, time.perf_counter() - t0


def make_training_set(n_maps, grid=128, coarse=128, levels=2, tau=0.05, seed0=5000, opts=None, device="cuda",
                      charges=(4, 12), log_every=0):
    """Tracer-generated maps: field i has k ~ U{charges} charges (seed
    seed0 + i), sampled on grid^3; its coarse^2 z = 0 cut is refined `levels`
    orders by the plain criterion. Returns X [n, 2, coarse, coarse], Y [n,
    coarse, coarse] (device) and the time spent."""
    if opts is None:
        opts = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6, integrator=qsl.QSL_DOPRI5_CELL)
    X = torch.empty((n_maps, 2, coarse, coarse), device=device)
    Y = torch.empty((n_maps, coarse, coarse), device=device)
    cap = (coarse << levels) ** 2
    smp = Samples(cap, device)
    spec = plane_spec(coarse, levels, tau)
    t0 = time.perf_counter()
    for i in range(n_maps):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        k = int(rng.integers(charges[0], charges[1] + 1))
        gf = inputs.charge_field(inputs.random_charges(k, seed0 + i), grid, dtype=torch.float32, device=device)
        F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
        del gf
        smp.count = 0
        smp.refine(F, spec, opts)
        L, Q, refined = coarse_grids(smp, 2, spec.max_order, levels, (coarse, coarse))
        X[i] = features(L, Q)
        Y[i] = refined
        del F
        if log_every and (i + 1) % log_every == 0:
            print("training maps: %d / %d" % (i + 1, n_maps), flush=True)
    torch.cuda.synchronize()
    return X, Y, time.perf_counter() - t0


def train(X, Y, epochs=20, batch=32, lr=2e-3, pos_weight=None, seed=11, log=None):
    """Trains a fresh network on (X, Y); returns (Cnn, loss history)."""
    n = X.shape[0]
    if pos_weight is None:
        frac = float(Y.mean().item())
        pos_weight = min(50.0, max(1.0, (1 - frac) / max(frac, 1e-6)))
    net = qsl.Cnn(init_params(seed))
    loss = torch.zeros(1, device=X.device)
    grad = torch.zeros(NPARAMS, device=X.device)
    rng = np.random.Generator(np.random.PCG64(seed))
    hist = []
    for ep in range(epochs):
        order = torch.as_tensor(rng.permutation(n), device=X.device)
        tot = 0.0
        nb = 0
        for b0 in range(0, n, batch):
            idx = order[b0:b0 + batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            net.loss_grad(xb, yb, pos_weight, loss, grad)
            net.adam(grad, lr=lr)
            tot += float(loss.item())
            nb += 1
        hist.append(tot / max(nb, 1))
        if log:
            log("epoch %d loss %.4f" % (ep, hist[-1]))
    return net, hist, pos_weight


def predict(net, X, batch=64):
    out = torch.empty((X.shape[0],) + tuple(X.shape[2:]), device=X.device)
    for b0 in range(0, X.shape[0], batch):
        xb = X[b0:b0 + batch].contiguous()
        out[b0:b0 + batch] = net.forward(xb)
    return out


def calibrate(net, X, Y, recall=0.995):
    """Largest probability threshold whose label recall on (X, Y) reaches
    `recall`; also returns the fraction of cells it proposes."""
    P = predict(net, X)
    pos = P[Y > 0.5]
    if pos.numel() == 0:
        return 0.5, 0.0
    thr = float(torch.quantile(pos.float(), 1.0 - recall).item()) if pos.numel() > 1 else float(pos.item())
    thr = max(min(thr, 0.999), 1e-6)
    frac = float((P >= thr).float().mean().item())
    return thr, frac


def propose(net, X, thr, budget=None, dilate=False):
    """uint8 mask (same layout as X's spatial dims: one volume [nz, ny, nx]
    or one map [ny, nx]) of cells with p >= thr, dilated by one cell in every
    direction if asked; with a budget, only the `budget` most probable of them
    (before dilation)."""
    P = predict(net, X)
    mask = P >= thr
    if budget is not None and int(mask.sum().item()) > budget:
        flat = torch.where(mask, P, torch.zeros_like(P)).reshape(-1)
        top = torch.topk(flat, int(budget)).indices
        mask = torch.zeros_like(flat, dtype=torch.bool)
        mask[top] = True
        mask = mask.view(P.shape)
    mask = mask.to(torch.uint8).contiguous()
    if dilate:
        out = torch.empty_like(mask)
        qsl.qsl_mask_dilate(mask, out)
        mask = out
    return mask


def calibrate_qsl(net, X, W, nz, recall=0.995, dilate=True, steps=30):
    """Largest probability threshold whose mask (dilated per volume of nz
    slices, if asked) holds `recall` of the QSL samples W of held-out
    volumes; also returns the fraction of cells it proposes and the recall."""
    P = predict(net, X)
    nv = X.shape[0] // nz
    Pv = P.view(nv, nz, *P.shape[1:])
    Wv = W.view(nv, nz, *W.shape[1:])
    total = float(Wv.sum().item())
    if total == 0:
        return 0.5, 0.0, 1.0

    def at(thr):
        m = (Pv >= thr).to(torch.uint8).contiguous()
        if dilate:
            d = torch.empty_like(m)
            for v in range(nv):
                qsl.qsl_mask_dilate(m[v], d[v])
            m = d
        return float((Wv * m.float()).sum().item()) / total, float(m.float().mean().item())

    lo, hi = 0.0, 1.0  # recall(lo) = 1
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        r, _ = at(mid)
        if r >= recall:
            lo = mid
        else:
            hi = mid
    r, frac = at(lo)
    return max(lo, 1e-6), frac, r


def converted_q(smp, ndim, max_order, extent, out_order):
    """Q of a sample set on the rectilinear output lattice (qsl_convert)."""
    d = max_order - out_order
    shape = [extent[a] >> d for a in range(ndim)][::-1]
    out = torch.empty(int(np.prod(shape)), device=smp.key.device)
    qsl.qsl_convert(smp.key[:smp.count], smp.q[:smp.count], ndim, max_order, list(extent), out_order, True, out)
    return out.view(shape)
