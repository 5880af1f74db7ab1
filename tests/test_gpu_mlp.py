"""Closure network on the GPU against the FP64 oracle with bfloat16 emulation.

The oracle rounds the inputs, weights, hidden activations and each layer's output gradient to
bfloat16 exactly where the CUDA kernels do and computes the rest in FP64, so the two differ
by FP32 accumulation (and a rare bfloat16 rounding flip it causes). Bars: outputs within
1e-2 of max|y|, every gradient tensor within 1e-2 of its largest entry, the loss within 1e-3;
Adam within FP32 round-off of the oracle's update applied to the same gradients; training
on a learnable target lowers the loss tenfold.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from paper_1105_2904_gb300 import lbmp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1105_2904_gb300 import build as B
    B.build()


def _params(sizes, seed):
    p = M.init_params(sizes, seed)
    g = np.random.Generator(np.random.PCG64(seed + 100))
    for l in range(len(p)):
        p[l][1] = g.normal(0, 0.2, p[l][1].shape)
    return p


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


SHAPES = [[256, 128, 128, 6], [7, 33, 5], [64, 96, 6]]


@pytest.mark.parametrize("sizes", SHAPES, ids=["256-128-128-6", "7-33-5", "64-96-6"])
@pytest.mark.parametrize("rows", [300, 64, 5])
def test_forward_and_gradients_match_oracle(sizes, rows):
    g = np.random.Generator(np.random.PCG64(rows + len(sizes)))
    X = g.normal(0, 1, (rows, sizes[0]))
    T = g.normal(0, 1, (rows, sizes[-1]))
    p = _params(sizes, 7)
    net = lbmp.MLP(sizes)
    net.set_params(p)
    xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    td = torch.tensor(T, dtype=torch.float32, device="cuda")
    Y = net.forward(xd).cpu().double().numpy()
    # the oracle sees the same FP32-rounded data and parameters
    Xf, Tf = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
    pf = [[W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)] for W, b in p]
    Yr, _ = M.forward(pf, Xf, bf16=True)
    assert _rel(Y, Yr) <= 1e-2
    loss = net.loss_grad(xd, td)
    lr_, gr = M.loss_and_grads(pf, Xf, Tf, bf16=True)
    assert abs(loss - lr_) <= 1e-3 * lr_
    gg = net.grads()
    for l in range(len(sizes) - 1):
        assert _rel(gg[l][0], gr[l][0]) <= 1e-2, ("W", l)
        assert _rel(gg[l][1], gr[l][1]) <= 1e-2, ("b", l)
    net.close()


def test_adam_step_matches_oracle_update():
    sizes = [16, 32, 6]
    g = np.random.Generator(np.random.PCG64(3))
    X = torch.tensor(g.normal(0, 1, (128, 16)), dtype=torch.float32, device="cuda")
    T = torch.tensor(g.normal(0, 1, (128, 6)), dtype=torch.float32, device="cuda")
    p = _params(sizes, 11)
    net = lbmp.MLP(sizes)
    net.set_params(p)
    pf = [[W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)] for W, b in p]
    m, v = M.adam_init(pf)
    for t in range(1, 4):
        net.loss_grad(X, T)
        gr = net.grads()
        net.adam_step(1e-2)
        M.adam_step(pf, gr, m, v, t, lr=1e-2)
        got = net.params()
        for l in range(len(sizes) - 1):
            for k in range(2):
                assert np.max(np.abs(got[l][k] - pf[l][k])) <= 1e-5 * max(1.0, np.max(np.abs(pf[l][k]))), (t, l, k)
        pf = got  # continue from the GPU's FP32 masters
    net.close()


def test_training_learns_a_smooth_target():
    sizes = [32, 64, 64, 6]
    g = np.random.Generator(np.random.PCG64(5))
    A = g.normal(0, 1, (6, 32)) / np.sqrt(32)
    X = g.normal(0, 1, (4096, 32))
    Y = np.tanh(X @ A.T) + 0.3 * (X @ A.T) ** 2
    net = lbmp.MLP(sizes)
    net.set_params(M.init_params(sizes, 1))
    xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.tensor(Y, dtype=torch.float32, device="cuda")
    losses = net.train(xd, yd, batch=256, epochs=30, lr=2e-3, seed=9)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.1 * losses[0]
    net.close()


def test_input_scaling_matches_oracle_on_scaled_inputs():
    # the kernel standardises each input in FP32, (x - shift) * scale, before rounding it to
    # bfloat16: the oracle sees the same FP32 values
    sizes = [7, 33, 5]
    g = np.random.Generator(np.random.PCG64(21))
    X = (g.normal(3.0, 2.0, (50, 7))).astype(np.float32)
    shift = g.normal(3.0, 0.5, 7)
    scale = 1.0 / g.uniform(1.0, 3.0, 7)
    p = _params(sizes, 13)
    net = lbmp.MLP(sizes)
    net.set_params(p)
    net.set_input_scaling(shift, scale)
    Y = net.forward(torch.tensor(X, device="cuda")).cpu().double().numpy()
    Xs = ((X - shift.astype(np.float32)) * scale.astype(np.float32)).astype(np.float64)
    pf = [[W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)] for W, b in p]
    Yr, _ = M.forward(pf, Xs, bf16=True)
    assert _rel(Y, Yr) <= 1e-2
    net.set_input_scaling(None, None)   # removed: plain inputs again
    Y0 = net.forward(torch.tensor(X, device="cuda")).cpu().double().numpy()
    Y0r, _ = M.forward(pf, X.astype(np.float64), bf16=True)
    assert _rel(Y0, Y0r) <= 1e-2
    net.close()
