"""FP64 oracle of the refinement-proposal CNN (TEST INFRASTRUCTURE).

conv3x3 2->32 + ReLU, conv3x3 32->32 + ReLU, conv3x3 32->1 (logit), zero
padding; loss = mean over pixels of pos_w * y * softplus(-z) + (1 - y) *
softplus(z). The weights enter the passes rounded to BF16 (round to nearest
even), as the model specifies; everything else is float64. The backward pass
is the chain rule written out layer by layer; tests pin it with central finite
differences. Parameters are flattened as w1[32][2][3][3], b1[32],
w2[32][32][3][3], b2[32], w3[1][32][3][3], b3[1].
"""
import numpy as np

SHAPES = [("w1", (32, 2, 3, 3)), ("b1", (32,)), ("w2", (32, 32, 3, 3)), ("b2", (32,)), ("w3", (1, 32, 3, 3)),
          ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(p):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(d):
    return np.concatenate([d[name].reshape(-1) for name, _ in SHAPES])


def bf16(a):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed):
    """Kaiming-uniform weights, zero biases (numpy PCG64 with `seed`)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = {}
    for name, shp in SHAPES:
        if name.startswith("w"):
            fan_in = shp[1] * 9
            bound = np.sqrt(6.0 / fan_in)
            d[name] = rng.uniform(-bound, bound, size=shp)
        else:
            d[name] = np.zeros(shp)
    return flatten(d).astype(np.float32)


def conv(x, w, b=None):
    """x [n][ci][h][w], w [co][ci][3][3] -> [n][co][h][w], zero padding."""
    n, ci, h, wd = x.shape
    xp = np.zeros((n, ci, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    out = np.zeros((n, w.shape[0], h, wd))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], xp[:, :, ky:ky + h, kx:kx + wd])
    if b is not None:
        out += b[None, :, None, None]
    return out


def conv_weight_grad(x, dy):
    n, ci, h, wd = x.shape
    xp = np.zeros((n, ci, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    g = np.zeros((dy.shape[1], ci, 3, 3))
    for ky in range(3):
        for kx in range(3):
            g[:, :, ky, kx] = np.einsum("nohw,nchw->oc", dy, xp[:, :, ky:ky + h, kx:kx + wd])
    return g


def conv_data_grad(dy, w):
    """Gradient w.r.t. the input of conv(x, w): correlation with the flipped,
    transposed kernel."""
    wt = np.transpose(w[:, :, ::-1, ::-1], (1, 0, 2, 3))
    return conv(dy, wt)


def softplus(z):
    return np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z)))


def forward(params, x):
    p = unflatten(params)
    w1, w2, w3 = bf16(p["w1"]), bf16(p["w2"]), bf16(p["w3"])
    z1 = conv(x, w1, p["b1"])
    a1 = np.maximum(z1, 0)
    z2 = conv(a1, w2, p["b2"])
    a2 = np.maximum(z2, 0)
    z = conv(a2, w3, p["b3"])[:, 0]
    return z, (x, a1, a2, w1, w2, w3)


def loss_grad(params, x, y, pos_w):
    """Returns (loss, flat gradient) of the mean weighted BCE."""
    z, (x, a1, a2, w1, w2, w3) = forward(params, x)
    npx = z.size
    loss = np.sum(pos_w * y * softplus(-z) + (1 - y) * softplus(z)) / npx
    s = 1.0 / (1.0 + np.exp(-z))
    dz = ((-pos_w * y * (1 - s) + (1 - y) * s) / npx)[:, None]
    g = {"w3": conv_weight_grad(a2, dz), "b3": dz.sum(axis=(0, 2, 3))}
    d2 = conv_data_grad(dz, w3) * (a2 > 0)
    g["w2"] = conv_weight_grad(a1, d2)
    g["b2"] = d2.sum(axis=(0, 2, 3))
    d1 = conv_data_grad(d2, w2) * (a1 > 0)
    g["w1"] = conv_weight_grad(x, d1)
    g["b1"] = d1.sum(axis=(0, 2, 3))
    return loss, flatten(g)


def adam(params, m, v, grad, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    c1, c2 = 1 - b1 ** step, 1 - b2 ** step
    return params - lr * (m / c1) / (np.sqrt(v / c2) + eps), m, v
