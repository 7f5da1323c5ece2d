"""CPU FP64 oracle of the learned warm start's network (numpy).

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product
path).  The paper has no network; the warm start is an extension whose
architecture is this reading of a "3D convolutional network with 4 levels,
32 channels, 3x3x3 kernels":

* tensors are (nz, ny, nx, C) arrays: cell (i, j, k) of the reservoir grid
  is element [k, j, i], so the flattened voxel order is the simulator's
  natural cell order i + nx (j + ny k);
* conv: Z[v, o] = b[o] + sum over the 27 offsets d in {-1,0,1}^3 and input
  channels c of X[v + d, c] W[t(d), o, c], with X = 0 outside the grid and
  t(d) = (dx+1) + 3 (dy+1) + 9 (dz+1); followed by ReLU except in the head;
* pool: average of the (up to 8) children that exist, coarse size
  ceil(n / 2) per axis;  up: nearest neighbour (fine cell takes its parent);
* U-Net over 4 resolution levels: two convs per encoder level, average pool
  down, two convs at the bottom, nearest up-sampling, concatenation
  [up-sampled, skip] (64 channels), two convs per decoder level, and a head
  conv to 8 output channels of which the first 2 are the prediction;
* loss: 0.5 / n * sum over voxels and the 2 predicted channels of
  (Y - T)^2.

Each function is the plain definition: sums over offsets and channels,
written with numpy slicing; no blocking or reordering beyond that.
"""
from __future__ import annotations

import numpy as np

# (input channels, output channels, relu) per layer, in forward order
LAYERS = [
    ("c00", 8, 32, True), ("c01", 32, 32, True),
    ("c10", 32, 32, True), ("c11", 32, 32, True),
    ("c20", 32, 32, True), ("c21", 32, 32, True),
    ("c30", 32, 32, True), ("c31", 32, 32, True),
    ("d20", 64, 32, True), ("d21", 32, 32, True),
    ("d10", 64, 32, True), ("d11", 32, 32, True),
    ("d00", 64, 32, True), ("d01", 32, 32, True),
    ("h", 32, 8, False),
]
N_IN, N_OUT, N_PRED = 8, 8, 2

OFFSETS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # index = tap


def _shift(X, dx, dy, dz):
    """S[k, j, i] = X[k + dz, j + dy, i + dx] (zero outside)."""
    nz, ny, nx = X.shape[:3]
    S = np.zeros_like(X)
    zs, ys, xs = slice(max(0, -dz), nz - max(0, dz)), slice(max(0, -dy), ny - max(0, dy)), \
        slice(max(0, -dx), nx - max(0, dx))
    zt, yt, xt = slice(max(0, dz), nz - max(0, -dz)), slice(max(0, dy), ny - max(0, -dy)), \
        slice(max(0, dx), nx - max(0, -dx))
    S[zs, ys, xs] = X[zt, yt, xt]
    return S


def conv(X, W, b):
    """Z = conv(X) + b.  X (nz,ny,nx,Ci), W (27,Co,Ci), b (Co,)."""
    Z = np.zeros(X.shape[:3] + (W.shape[1],))
    for t, (dx, dy, dz) in enumerate(OFFSETS):
        Z += _shift(X, dx, dy, dz) @ W[t].T
    return Z + b


def conv_backward(X, W, G):
    """Gradients of sum(G * conv(X, W, b)): (dX, dW, db)."""
    dX = np.zeros_like(X)
    dW = np.zeros_like(W)
    Gf = G.reshape(-1, G.shape[-1])
    for t, (dx, dy, dz) in enumerate(OFFSETS):
        S = _shift(X, dx, dy, dz)
        dW[t] = Gf.T @ S.reshape(-1, S.shape[-1])
        # X[v + d] contributed to Z[v]: move G back by -d
        dX += _shift(G @ W[t], -dx, -dy, -dz)
    return dX, dW, Gf.sum(axis=0)


def coarse_shape(shape):
    return tuple((n + 1) // 2 for n in shape)


def pool(X):
    """Average over the existing children of each coarse cell."""
    nz, ny, nx, c = X.shape
    Nz, Ny, Nx = coarse_shape((nz, ny, nx))
    S = np.zeros((Nz, Ny, Nx, c))
    cnt = np.zeros((Nz, Ny, Nx, 1))
    for k in range(2):
        for j in range(2):
            for i in range(2):
                part = X[k::2, j::2, i::2]
                S[:part.shape[0], :part.shape[1], :part.shape[2]] += part
                cnt[:part.shape[0], :part.shape[1], :part.shape[2]] += 1
    return S / cnt


def pool_backward(shape, G):
    """Gradient of sum(G * pool(X)) with respect to X of the given fine shape."""
    nz, ny, nx = shape
    cnt = np.zeros(G.shape[:3] + (1,))
    for k in range(2):
        for j in range(2):
            for i in range(2):
                sz, sy, sx = len(range(k, nz, 2)), len(range(j, ny, 2)), len(range(i, nx, 2))
                cnt[:sz, :sy, :sx] += 1
    Gs = G / cnt
    return up(Gs, shape)


def up(C, shape):
    """Fine cell (i, j, k) takes coarse cell (i//2, j//2, k//2)."""
    nz, ny, nx = shape
    return C.repeat(2, 0).repeat(2, 1).repeat(2, 2)[:nz, :ny, :nx]


def up_backward(G, coarse):
    """Gradient of sum(G * up(C)) with respect to C: sum over the children."""
    S = np.zeros(tuple(coarse) + (G.shape[-1],))
    for k in range(2):
        for j in range(2):
            for i in range(2):
                part = G[k::2, j::2, i::2]
                S[:part.shape[0], :part.shape[1], :part.shape[2]] += part
    return S


def init_params(seed=0):
    """He-normal weights, zero biases (any deterministic draw will do for tests)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co, _ in LAYERS:
        P[name] = (rng.standard_normal((27, co, ci)) * np.sqrt(2.0 / (27 * ci)), np.zeros(co))
    return P


def forward(P, F, rnd=None):
    """Network output Y (nz,ny,nx,8) for features F (nz,ny,nx,8) and the cache.

    rnd (default: none) is applied where a kernel stores an activation in a
    narrower type (the input, every ReLU output and every pooled tensor), so
    the oracle can take the same storage precision as the implementation
    under test; the arithmetic between those points stays FP64."""
    r = rnd if rnd is not None else (lambda a: a)
    cache = {"rnd": r}

    def layer(name, X, relu=True):
        W, b = P[name]
        Z = conv(X, W, b)
        A = r(np.maximum(Z, 0.0)) if relu else Z
        cache[name] = (X, A)
        return A

    F = r(F)
    s0 = F.shape[:3]
    s1 = coarse_shape(s0); s2 = coarse_shape(s1); s3 = coarse_shape(s2)
    e0 = layer("c01", layer("c00", F))
    e1 = layer("c11", layer("c10", r(pool(e0))))
    e2 = layer("c21", layer("c20", r(pool(e1))))
    b3 = layer("c31", layer("c30", r(pool(e2))))
    b2 = layer("d21", layer("d20", np.concatenate([up(b3, s2), e2], axis=-1)))
    b1 = layer("d11", layer("d10", np.concatenate([up(b2, s1), e1], axis=-1)))
    b0 = layer("d01", layer("d00", np.concatenate([up(b1, s0), e0], axis=-1)))
    Y = layer("h", b0, relu=False)
    cache["shapes"] = (s0, s1, s2, s3)
    return Y, cache


def loss(Y, T):
    """0.5 / n * sum of squared errors over the predicted channels."""
    n = Y.shape[0] * Y.shape[1] * Y.shape[2]
    E = Y[..., :N_PRED] - T[..., :N_PRED]
    return 0.5 * float(np.sum(E * E)) / n


def backward(P, cache, Y, T):
    """Gradients {name: (dW, db)} of loss(Y, T) for the forward pass cached.
    The cache's rounding (see forward) is applied where a kernel stores a
    gradient tensor: the loss gradient, every data gradient, and the sums
    formed at up-sampling and pooling joins."""
    r = cache["rnd"]
    n = Y.shape[0] * Y.shape[1] * Y.shape[2]
    G = np.zeros_like(Y)
    G[..., :N_PRED] = r((Y[..., :N_PRED] - T[..., :N_PRED]) / n)
    grads = {}
    s0, s1, s2, s3 = cache["shapes"]

    def layer_back(name, dA, below_relu=True):
        # dA arrives already multiplied by this layer's ReLU mask (the
        # mask is applied where the gradient of its output is formed)
        X, A = cache[name]
        dX, dW, db = conv_backward(X, P[name][0], dA)
        grads[name] = (dW, db)
        return r(dX * (X > 0)) if below_relu else r(dX)

    def masked(name, dA):
        return dA * (cache[name][1] > 0)

    db0 = layer_back("h", G)                        # input of h is a ReLU output
    dcat0 = layer_back("d00", layer_back("d01", db0))
    db1 = r(up_backward(dcat0[..., :32], s1))
    dcat1 = layer_back("d10", layer_back("d11", db1))
    db2 = r(up_backward(dcat1[..., :32], s2))
    dcat2 = layer_back("d20", layer_back("d21", db2))
    db3 = r(up_backward(dcat2[..., :32], s3))
    dp3 = layer_back("c30", layer_back("c31", db3), below_relu=False)
    de2 = r(masked("c21", dcat2[..., 32:] + pool_backward(s2, dp3)))
    dp2 = layer_back("c20", layer_back("c21", de2), below_relu=False)
    de1 = r(masked("c11", dcat1[..., 32:] + pool_backward(s1, dp2)))
    dp1 = layer_back("c10", layer_back("c11", de1), below_relu=False)
    de0 = r(masked("c01", dcat0[..., 32:] + pool_backward(s0, dp1)))
    layer_back("c00", layer_back("c01", de0), below_relu=False)
    return grads


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1) of parameter p with
    gradient g at step t (1-based); returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
