"""GPU parity of the refinement-proposal CNN kernels against the FP64 oracle
(oracle/cnn.py): forward probabilities, loss, the parameter gradient (BF16
weights, FP32 accumulation) and the Adam update."""
import numpy as np
import pytest
import torch

from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsl():
    from paper_1609_00724_gb300 import qsl as q
    q.lib()
    return q


def _problem(seed, n=3, h=37, w=45):
    rng = np.random.default_rng(seed)
    params = ocnn.init_params(seed)
    d = ocnn.unflatten(params)
    d["b1"] = rng.uniform(-0.1, 0.1, 32)
    d["b2"] = rng.uniform(-0.1, 0.1, 32)
    d["b3"] = np.array([-0.5])
    params = ocnn.flatten(d).astype(np.float32)
    x = rng.normal(size=(n, 2, h, w)).astype(np.float32)
    y = (rng.uniform(size=(n, h, w)) > 0.8).astype(np.float32)
    return params, x, y


def test_forward_loss_and_gradient_match_oracle(qsl):
    params, x, y = _problem(4)
    net = qsl.Cnn(params)
    xd, yd = torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda()
    prob = net.forward(xd).cpu().numpy()
    z, _ = ocnn.forward(params.astype(np.float64), x.astype(np.float64))
    want = 1 / (1 + np.exp(-z))
    assert np.abs(prob - want).max() < 1e-5
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(qsl.QSL_CNN_NPARAMS, device="cuda")
    net.loss_grad(xd, yd, 4.0, loss, grad)
    L, g = ocnn.loss_grad(params.astype(np.float64), x.astype(np.float64), y.astype(np.float64), 4.0)
    assert abs(loss.item() / L - 1) < 1e-5
    gg = grad.cpu().numpy().astype(np.float64)
    # FP32 accumulation over up to n*h*w*288 terms: relative to each block's scale
    o = 0
    for name, shp in ocnn.SHAPES:
        k = int(np.prod(shp))
        a, b = gg[o:o + k], g[o:o + k]
        assert np.abs(a - b).max() <= 1e-4 * np.abs(b).max() + 1e-9, name
        o += k


def test_adam_step_matches_oracle(qsl):
    params, x, y = _problem(5, n=2, h=16, w=16)
    net = qsl.Cnn(params)
    rng = np.random.default_rng(0)
    m = np.zeros(params.size)
    v = np.zeros(params.size)
    p64 = params.astype(np.float64)
    for step in range(1, 4):
        gr = rng.normal(size=params.size).astype(np.float32)
        net.adam(torch.as_tensor(gr).cuda(), lr=1e-2)
        p64, m, v = ocnn.adam(p64, m, v, gr.astype(np.float64), step, lr=1e-2)
    torch.cuda.synchronize()
    assert np.abs(net.params() - p64).max() < 1e-5


def test_training_reduces_loss(qsl):
    """A toy target (pixels where channel 0 exceeds 0.5) is learned."""
    rng = np.random.default_rng(7)
    x = rng.normal(size=(16, 2, 32, 32)).astype(np.float32)
    y = (x[:, 0] > 0.5).astype(np.float32)
    net = qsl.Cnn(ocnn.init_params(11))
    xd, yd = torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda()
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(qsl.QSL_CNN_NPARAMS, device="cuda")
    first = None
    for it in range(200):
        net.loss_grad(xd, yd, 1.0, loss, grad)
        if first is None:
            first = loss.item()
        net.adam(grad, lr=3e-3)
    net.loss_grad(xd, yd, 1.0, loss, grad)
    assert loss.item() < 0.3 * first, (first, loss.item())
