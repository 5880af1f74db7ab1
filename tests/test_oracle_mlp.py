"""Pins of the FP64 closure-network oracle (oracle/mlp_oracle.py) against what the
mathematics fixes: central finite differences of the loss for every gradient, the closed
form of Adam's first step, bfloat16 rounding against torch's own conversion, and a forward
pass small enough to write out by hand."""
import numpy as np
import pytest
import torch

from oracle import mlp_oracle as M


def test_bf16_round_matches_torch_and_ties_to_even():
    g = np.random.Generator(np.random.PCG64(0))
    x = np.concatenate([g.normal(0, 1, 5000), g.normal(0, 1e-30, 100), g.normal(0, 1e30, 100),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.5 + 2 ** -9]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x), ref)
    assert M.bf16_round([1.0 + 2 ** -8])[0] == 1.0                 # tie: even mantissa kept
    assert M.bf16_round([1.0 + 3 * 2 ** -8])[0] == 1.0 + 2 ** -6    # tie: rounds up to even


def test_forward_by_hand():
    params = [[np.array([[1.0, -2.0], [0.5, 0.25]]), np.array([0.1, -1.0])],
              [np.array([[2.0, -1.0]]), np.array([0.5])]]
    X = np.array([[1.0, 1.0], [2.0, -1.0]])
    # row 0: z1 = (1 - 2 + 0.1, 0.5 + 0.25 - 1) = (-0.9, -0.25) -> h = (0, 0) -> y = 0.5
    # row 1: z1 = (2 + 2 + 0.1, 1 - 0.25 - 1) = (4.1, -0.25) -> h = (4.1, 0) -> y = 8.2 + 0.5
    Y, _ = M.forward(params, X)
    assert np.allclose(Y[:, 0], [0.5, 8.7], rtol=0, atol=1e-15)


def test_gradients_match_central_differences():
    g = np.random.Generator(np.random.PCG64(1))
    params = M.init_params([7, 5, 4, 3], seed=2)
    for l in range(3):
        params[l][1] = g.normal(0, 0.3, params[l][1].shape)
    X = g.normal(0, 1, (11, 7))
    T = g.normal(0, 1, (11, 3))
    _, grads = M.loss_and_grads(params, X, T)
    h = 1e-6
    for l in range(3):
        for k in range(2):
            P = params[l][k]
            num = np.zeros_like(P)
            for idx in np.ndindex(P.shape):
                old = P[idx]
                P[idx] = old + h
                lp, _ = M.loss_and_grads(params, X, T)
                P[idx] = old - h
                lm, _ = M.loss_and_grads(params, X, T)
                P[idx] = old
                num[idx] = (lp - lm) / (2 * h)
            scale = np.max(np.abs(num)) + 1e-12
            assert np.max(np.abs(num - grads[l][k])) <= 1e-7 * scale, (l, k)


def test_adam_first_step_closed_form():
    # after one step m_hat = g and v_hat = g^2, so the update is -lr g / (|g| + eps)
    params = [[np.array([[1.0, -2.0, 3.0]]), np.array([0.5])]]
    grads = [[np.array([[0.1, -0.02, 0.0]]), np.array([-3.0])]]
    m, v = M.adam_init(params)
    M.adam_step(params, grads, m, v, 1, lr=0.01, eps=1e-8)
    want = np.array([[1.0 - 0.01 * 0.1 / (0.1 + 1e-8), -2.0 + 0.01 * 0.02 / (0.02 + 1e-8), 3.0]])
    assert np.allclose(params[0][0], want, rtol=0, atol=1e-15)
    assert np.isclose(params[0][1][0], 0.5 + 0.01 * 3.0 / (3.0 + 1e-8), rtol=0, atol=1e-15)


def test_training_reduces_the_loss_on_a_linear_target():
    g = np.random.Generator(np.random.PCG64(3))
    A = g.normal(0, 1, (4, 9))
    X = g.normal(0, 1, (64, 9))
    T = X @ A.T
    params = M.init_params([9, 16, 16, 4], seed=4)
    m, v = M.adam_init(params)
    l0, _ = M.loss_and_grads(params, X, T)
    for t in range(1, 301):
        _, gr = M.loss_and_grads(params, X, T)
        M.adam_step(params, gr, m, v, t, lr=3e-3)
    l1, _ = M.loss_and_grads(params, X, T)
    assert l1 < 0.05 * l0


def test_bf16_emulation_stays_close_to_fp64():
    # bfloat16 keeps 8 significant bits; batch sums of mixed-sign terms amplify the relative
    # error of a gradient entry (measured: 7 % of the largest entry in the hidden layers)
    g = np.random.Generator(np.random.PCG64(5))
    params = M.init_params([32, 16, 16, 6], seed=6)
    X = g.normal(0, 1, (40, 32))
    T = g.normal(0, 1, (40, 6))
    l64, g64 = M.loss_and_grads(params, X, T)
    l16, g16 = M.loss_and_grads(params, X, T, bf16=True)
    assert abs(l16 - l64) <= 2e-2 * l64
    for a, b in zip(g64, g16):
        assert np.max(np.abs(a[0] - b[0])) <= 0.15 * np.max(np.abs(a[0]))


def test_stencil_features_interpolate_linear_fields_exactly():
    # trilinear interpolation reproduces a linear field; nodes are kept away from the wrap
    nz, ny, nx = 20, 22, 24
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rho = 1.0 + 1e-3 * (0.5 * x - 0.25 * y + 0.125 * z)
    u = np.stack([2e-3 * x + 1e-4, -1e-3 * y, 5e-4 * (x + z)], axis=-1)
    centers = np.array([[11.3, 10.7, 9.2], [12.05, 11.5, 10.0]])
    up = np.array([[1e-4, 0.0, -2e-4], [0.0, 0.0, 0.0]])
    n, h, U = 4, 1.7, 2e-3
    F = M.stencil_features(rho, u, centers, up, n, h, U)
    for p in range(2):
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    X = centers[p] + h * (np.array([i, j, k]) - 1.5)
                    q = (k * n + j) * n + i
                    want = [1e-3 * (0.5 * X[0] - 0.25 * X[1] + 0.125 * X[2]) / U,
                            (2e-3 * X[0] + 1e-4 - up[p, 0]) / U, (-1e-3 * X[1] - up[p, 1]) / U,
                            (5e-4 * (X[0] + X[2]) - up[p, 2]) / U]
                    assert np.allclose(F[p, 4 * q:4 * q + 4], want, rtol=0, atol=1e-12)
