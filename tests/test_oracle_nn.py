"""Pins of the warm-start network oracle (oracle/nn.py) on the CPU.

The convolution is checked against a brute-force sum over voxels, offsets
and channels; its backward pass against the exact adjoint identities of a
linear map; pooling and up-sampling against their adjoint identities and
constant fields; the whole network's backward pass against central finite
differences of its forward pass; Adam's first step against its closed
form; and the bfloat16 rounding against torch's conversion.
"""
import numpy as np
import pytest

from oracle import nn


def _brute_conv(X, W, b):
    nz, ny, nx, ci = X.shape
    co = W.shape[1]
    Z = np.zeros((nz, ny, nx, co))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for o in range(co):
                    s = b[o]
                    for dz in (-1, 0, 1):
                        for dy in (-1, 0, 1):
                            for dx in (-1, 0, 1):
                                kk, jj, ii = k + dz, j + dy, i + dx
                                if 0 <= kk < nz and 0 <= jj < ny and 0 <= ii < nx:
                                    t = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                                    for c in range(ci):
                                        s += X[kk, jj, ii, c] * W[t, o, c]
                    Z[k, j, i, o] = s
    return Z


def test_conv_matches_brute_force():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((3, 4, 5, 2))
    W = rng.standard_normal((27, 3, 2))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(nn.conv(X, W, b), _brute_conv(X, W, b), rtol=1e-13, atol=1e-13)


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((4, 3, 5, 3))
    W = rng.standard_normal((27, 4, 3))
    G = rng.standard_normal((4, 3, 5, 4))
    dX, dW, db = nn.conv_backward(X, W, G)
    zero = np.zeros(4)
    # <conv(X), G> is linear in X and in W separately
    np.testing.assert_allclose(np.sum(nn.conv(X, W, zero) * G), np.sum(X * dX), rtol=1e-12)
    W2 = rng.standard_normal(W.shape)
    np.testing.assert_allclose(np.sum(nn.conv(X, W2, zero) * G), np.sum(W2 * dW), rtol=1e-12)
    np.testing.assert_allclose(db, G.sum(axis=(0, 1, 2)), rtol=1e-12)


@pytest.mark.parametrize("shape", [(4, 6, 8), (3, 5, 7), (1, 1, 3)])
def test_pool_and_up_adjoints(shape):
    rng = np.random.default_rng(3)
    X = rng.standard_normal(shape + (2,))
    cs = nn.coarse_shape(shape)
    C = rng.standard_normal(cs + (2,))
    G = rng.standard_normal(cs + (2,))
    H = rng.standard_normal(shape + (2,))
    np.testing.assert_allclose(np.sum(nn.pool(X) * G), np.sum(X * nn.pool_backward(shape, G)), rtol=1e-12)
    np.testing.assert_allclose(np.sum(nn.up(C, shape) * H), np.sum(C * nn.up_backward(H, cs)), rtol=1e-12)
    # constants survive pooling; pooling an up-sampled field gives it back
    np.testing.assert_allclose(nn.pool(np.full(shape + (1,), 2.5)), 2.5)
    np.testing.assert_allclose(nn.pool(nn.up(C, shape)), C, rtol=1e-12)


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    shape = (3, 5, 6)                      # odd sizes: ragged pooling at every level
    P = nn.init_params(5)
    for name in P:                         # non-zero biases so that they matter
        W, b = P[name]
        P[name] = (W, 0.1 * rng.standard_normal(b.shape))
    F = rng.standard_normal(shape + (8,))
    T = rng.standard_normal(shape + (8,))
    Y, cache = nn.forward(P, F)
    g = nn.backward(P, cache, Y, T)
    h = 1e-6
    checked = 0
    for name, ci, co, _ in nn.LAYERS:
        W, b = P[name]
        for which in ("W", "b"):
            A = W if which == "W" else b
            G = g[name][0] if which == "W" else g[name][1]
            for _ in range(2):
                idx = tuple(rng.integers(0, s) for s in A.shape)
                old = A[idx]
                A[idx] = old + h
                lp = nn.loss(nn.forward(P, F)[0], T)
                A[idx] = old - h
                lm = nn.loss(nn.forward(P, F)[0], T)
                A[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - G[idx]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (name, which, idx, fd, G[idx])
                checked += 1
    assert checked == 4 * len(nn.LAYERS)


def test_loss_definition():
    Y = np.zeros((1, 1, 2, 8))
    T = np.zeros((1, 1, 2, 8))
    Y[0, 0, 0, :3] = (1.0, 2.0, 50.0)      # channel 2 is not predicted: ignored
    assert nn.loss(Y, T) == pytest.approx(0.5 * (1.0 + 4.0) / 2)


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, m, v = nn.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected moments of the first step are g and g^2
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14)


def test_adam_constant_gradient_every_step():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2 at every step t (m_t = (1 - beta1^t) g, v_t = (1 - beta2^t) g^2), so
    each step moves p by lr g / (|g| + eps)."""
    g = np.array([0.3, -4.0, 1e-3, 7.5])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 8):
        p_new, m, v = nn.adam_step(p, g, m, v, t, lr=0.01)
        np.testing.assert_allclose(p - p_new, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
        p = p_new


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(6).standard_normal(10000) * np.exp(np.random.default_rng(7).uniform(-20, 20, 10000))
    x = np.concatenate([x, [0.0, 1.0, -1.0, 1.00390625, 1.01171875]])     # ties to even
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(nn.bf16_round(x), ref)
