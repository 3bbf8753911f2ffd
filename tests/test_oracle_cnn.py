"""Pins of the FP64 CNN oracle: the hand-written backward pass against central
finite differences of the loss, the BF16 rounding against known values, and
the transposed-convolution identity <conv(x, w), dy> = <x, conv_data_grad(dy, w)>."""
import numpy as np

from oracle import cnn


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7 + 2 ** -8 + 2 ** -10, -3.14159265, 65504.0, 1.0 + 2 ** -7 + 2 ** -9],
                    dtype=np.float32)
    r = cnn.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0  # halfway to the next bf16 value: ties to even
    assert r[2] == 1.0 + 2 ** -6  # above halfway: rounds up
    assert r[5] == 1.0 + 2 ** -7  # below halfway: rounds down
    assert abs(r[3] - (-3.140625)) < 1e-12
    assert r[4] == 65536.0


def test_transpose_identity():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 7, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    dy = rng.normal(size=(2, 4, 7, 9))
    lhs = np.sum(cnn.conv(x, w) * dy)
    rhs = np.sum(x * cnn.conv_data_grad(dy, w))
    assert abs(lhs - rhs) < 1e-9 * abs(lhs)
    # weight gradient: d<conv(x,w), dy>/dw
    gw = cnn.conv_weight_grad(x, dy)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (3, 2, 1, 2), (1, 1, 2, 0)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += eps
        wm[idx] -= eps
        fd = (np.sum(cnn.conv(x, wp) * dy) - np.sum(cnn.conv(x, wm) * dy)) / (2 * eps)
        assert abs(fd - gw[idx]) < 1e-6 * (1 + abs(gw[idx]))


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = cnn.init_params(3).astype(np.float64)
    # biases nonzero so that ReLU kinks are away from the probed points
    d = cnn.unflatten(params)
    d["b1"] = rng.uniform(-0.1, 0.1, 32)
    d["b2"] = rng.uniform(-0.1, 0.1, 32)
    d["b3"] = np.array([0.05])
    params = cnn.flatten(d)
    x = rng.normal(size=(2, 2, 6, 7))
    y = (rng.uniform(size=(2, 6, 7)) > 0.7).astype(np.float64)
    loss, g = cnn.loss_grad(params, x, y, pos_w=3.0)
    # the passes use BF16 weights: probe the biases (exact in the passes) and
    # weights through their BF16 values (steps that keep the BF16 rounding)
    eps = 1e-6
    offs = {"b1": 32 * 2 * 9, "b2": 32 * 2 * 9 + 32 + 32 * 32 * 9, "b3": cnn.NPARAMS - 1}
    for name, o in offs.items():
        for k in range(3 if name != "b3" else 1):
            pp, pm = params.copy(), params.copy()
            pp[o + k] += eps
            pm[o + k] -= eps
            fd = (cnn.loss_grad(pp, x, y, 3.0)[0] - cnn.loss_grad(pm, x, y, 3.0)[0]) / (2 * eps)
            assert abs(fd - g[o + k]) < 1e-6 * (1 + abs(g[o + k])), (name, k, fd, g[o + k])
    # weights: evaluate the loss with BF16-exact weights perturbed in the
    # un-rounded forward (the gradient is d loss / d w_bf16)
    def loss_with(wflat):
        d2 = cnn.unflatten(wflat)
        z1 = cnn.conv(x, d2["w1"], d2["b1"])
        a1 = np.maximum(z1, 0)
        a2 = np.maximum(cnn.conv(a1, d2["w2"], d2["b2"]), 0)
        z = cnn.conv(a2, d2["w3"], d2["b3"])[:, 0]
        return np.sum(3.0 * y * cnn.softplus(-z) + (1 - y) * cnn.softplus(z)) / z.size
    base = cnn.unflatten(params)
    for nm in ("w1", "w2", "w3"):
        base[nm] = cnn.bf16(base[nm])
    flat = cnn.flatten(base)
    for o in (5, 32 * 2 * 9 + 32 + 100, cnn.NPARAMS - 10):
        pp, pm = flat.copy(), flat.copy()
        pp[o] += eps
        pm[o] -= eps
        fd = (loss_with(pp) - loss_with(pm)) / (2 * eps)
        assert abs(fd - g[o]) < 1e-6 * (1 + abs(g[o])), (o, fd, g[o])
