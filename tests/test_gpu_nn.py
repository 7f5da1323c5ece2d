"""The learned warm start's network on the GPU (BF16 tensor-core kernels,
FP32 accumulation) against the FP64 network oracle (oracle/nn.py).

Both sides start from the same parameters: the GPU's FP32 master weights,
which the oracle takes rounded to BF16 exactly as the kernels do.  The
oracle also rounds to BF16 at the points where the kernels store an
activation or a gradient, so the remaining differences come from FP32
accumulation order and the occasional rounding-boundary flip they cause:
the forward output must match element by element (the largest voxel
difference of each output channel over that channel's largest value) to
1e-2, every parameter gradient tensor element by element to 1e-2 (and in
Frobenius norm to 3e-2); Adam's update (FP32) to 1e-5.  Without the
emulated rounding (plain FP64 oracle) the output still agrees to 5e-2.
Odd grid sizes make every pooling level ragged.  The forward and backward
checks run with the tcgen05 convolution kernels and with the mma.sync ones
(the default).
"""
import numpy as np
import pytest

import paper_1701_06254_gb300 as R
from paper_1701_06254_gb300 import inputs as I
from oracle import nn

pytestmark = pytest.mark.gpu


def _to_dict(flat):
    P, q = {}, 0
    for name, ci, co, _ in nn.LAYERS:
        W = flat[q:q + 27 * co * ci].reshape(27, co, ci).astype(np.float64); q += 27 * co * ci
        b = flat[q:q + co].astype(np.float64); q += co
        P[name] = (W, b)
    assert q == flat.size
    return P


def _to_flat(P):
    return np.concatenate([np.concatenate([P[name][0].ravel(), P[name][1].ravel()]) for name, *_ in nn.LAYERS])


def _bf16_weights(P):
    return {k: (nn.bf16_round(W), b) for k, (W, b) in P.items()}


def _setup(shape=(5, 7, 9), seed=3, tc=True):
    ws = R.WarmStart(seed=seed)
    ws.use_tcgen05(tc)
    rng = np.random.default_rng(seed)
    flat = ws.params()
    # non-zero biases so that they are exercised
    P = _to_dict(flat)
    for k in P:
        P[k] = (P[k][0], 0.05 * rng.standard_normal(P[k][1].shape))
    flat = _to_flat(P).astype(np.float32)
    ws.set_params(flat)
    P = _to_dict(flat)
    F = nn.bf16_round(rng.standard_normal(shape + (8,)))
    T = rng.standard_normal(shape + (2,))
    return ws, P, F, T


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _maxrel(a, b):
    """Element by element: the largest |a - b| over the largest |b|."""
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-30))


@pytest.mark.parametrize("tc", [True, False], ids=["tcgen05", "mma_sync"])
def test_forward_matches_oracle(tc):
    ws, P, F, T = _setup(tc=tc)
    y = ws.forward(F.astype(np.float32))
    yo, _ = nn.forward(_bf16_weights(P), F, rnd=nn.bf16_round)
    for ch in range(2):                         # the prediction's two channels, voxel by voxel
        assert _maxrel(y[..., ch], yo[..., ch]) <= 1e-2, (ch, _maxrel(y[..., ch], yo[..., ch]))
    assert _rel(y, yo) <= 1e-2, _rel(y, yo)
    yp, _ = nn.forward(_bf16_weights(P), F)
    assert _rel(y, yp) <= 5e-2, _rel(y, yp)


@pytest.mark.parametrize("tc", [True, False], ids=["tcgen05", "mma_sync"])
def test_backward_matches_oracle(tc):
    ws, P, F, T = _setup(shape=(6, 5, 11), seed=4, tc=tc)
    ws.zero_grad()
    loss = ws.backward(F.astype(np.float32), T.astype(np.float32))
    g = _to_dict(ws.params(which=1))
    Pb = _bf16_weights(P)
    yo, cache = nn.forward(Pb, F, rnd=nn.bf16_round)
    To = np.zeros(yo.shape); To[..., :2] = T
    go = nn.backward(Pb, cache, yo, To)
    assert loss == pytest.approx(nn.loss(yo, To), rel=2e-2)
    worst = []
    for name, *_ in nn.LAYERS:
        for k in range(2):
            e = _rel(g[name][k], go[name][k])
            m = _maxrel(g[name][k], go[name][k])     # element by element over the tensor
            worst.append((m, name, "W" if k == 0 else "b"))
            assert e <= 3e-2, (name, "W" if k == 0 else "b", e)
    assert max(worst)[0] <= 1e-2, sorted(worst)[-3:]


def test_adam_step_matches_oracle():
    ws, P, F, T = _setup(shape=(4, 6, 5), seed=5)
    ws.zero_grad()
    ws.backward(F.astype(np.float32), T.astype(np.float32))
    g = ws.params(which=1).astype(np.float64)
    p0 = ws.params().astype(np.float64)
    ws.adam(1e-3)
    p1 = ws.params().astype(np.float64)
    pe, _, _ = nn.adam_step(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, 1e-3)
    assert np.max(np.abs(p1 - pe)) <= 1e-5 * 1e-3 + 1e-6 * np.max(np.abs(p0)), np.max(np.abs(p1 - pe))


def test_gradients_accumulate_over_samples():
    ws, P, F, T = _setup(shape=(3, 4, 5), seed=6)
    ws.zero_grad()
    ws.backward(F.astype(np.float32), T.astype(np.float32))
    g1 = ws.params(which=1)
    ws.backward(F.astype(np.float32), T.astype(np.float32))
    g2 = ws.params(which=1)             # mean over two identical samples
    np.testing.assert_allclose(g2, g1, rtol=1e-5, atol=1e-9)


def _run(case, steps, ws=None, rec=None, **opts):
    g = R.Sim(case, **opts)
    g.init_hydrostatic()
    if ws is not None:
        g.attach_warm_start(ws)
    if rec is not None:
        g.record_to(rec)
    g.advance(steps)
    return g


def test_training_on_recorded_solves_lowers_the_loss():
    ws = R.WarmStart(seed=11)
    for k in range(3):
        c = I.ensemble_member(k, seed0=5100, size_lo=(12, 12, 4), size_hi=(16, 16, 6))
        _run(c, 3, rec=ws, precision=R.PREC_MIXED)
    n = ws.dataset_size()
    assert n >= 6
    l0 = ws.eval()
    l1 = ws.train(epochs=30, batch=2, lr=2e-3, seed=1)
    assert np.isfinite(l1) and ws.eval() < 0.9 * l0, (l0, l1, ws.eval())


def test_warm_start_keeps_the_converged_solution():
    """With a network attached (trained briefly), every solve still meets its
    tolerance: the run matches the FP64 oracle with the whole-run tolerances,
    and every solve took either the prediction or the fallback."""
    import oracle
    ws = R.WarmStart(seed=12)
    for k in range(2):
        _run(I.ensemble_member(k, seed0=5200, size_lo=(12, 12, 4), size_hi=(16, 16, 6)), 3, rec=ws,
             precision=R.PREC_MIXED)
    ws.train(epochs=20, batch=2, lr=2e-3, seed=2)
    c = I.ensemble_member(7, seed0=5200, size_lo=(12, 12, 4), size_hi=(16, 16, 6))
    o = oracle.Sim(c)
    o.init_hydrostatic()
    g = R.Sim(c, precision=R.PREC_MIXED)
    g.init_hydrostatic()
    g.attach_warm_start(ws)
    for k in range(3):
        assert o.advance(1) == 0
        g.advance(1)
        po, so, _, to = o.get_state()
        pg, sg, _, tg = g.get_state()
        assert tg == to
        assert np.max(np.abs(pg - po) / np.abs(po)) <= 1e-6, k
        assert np.max(np.abs(sg - so)) <= 1e-6, k
    st = g.stats()
    assert st["ws_used"] + st["ws_fallback"] == st["linear_solves"]


def test_untrained_network_falls_back_to_the_plain_guess():
    """A fresh network's head is zero, so its prediction adds nothing: every
    solve falls back to the previous step's first update where there is one
    (the first Newton iteration of every step after the first), whose
    residual is below the zero guess's, and to zero elsewhere."""
    c = I.ensemble_member(4, seed0=5300, size_lo=(10, 10, 4), size_hi=(12, 12, 5))
    g = _run(c, 3, ws=R.WarmStart(seed=14), precision=R.PREC_MIXED)
    st = g.stats()
    assert st["ws_used"] == 0 and st["ws_fallback"] == st["linear_solves"] > 0
    assert st["ws_r0"] < st["linear_solves"]          # some solves started below ||b||, none above


def test_warm_start_iteration_savings():
    """What the warm start gains: the same model run with and without a
    trained network attached; FGMRES iterations per solve and the mean
    initial residual ||b - A x0|| / ||b|| are reported, and iterations must
    not grow."""
    kw = dict(seed0=5300, size_lo=(14, 14, 5), size_hi=(16, 16, 6))
    ws = R.WarmStart(seed=13)
    for k in range(3):
        _run(I.ensemble_member(k, **kw), 3, rec=ws, precision=R.PREC_MIXED)
    ws.train(epochs=20, batch=2, lr=1e-3, seed=3)
    c = I.ensemble_member(9, **kw)
    plain = _run(c, 4, precision=R.PREC_MIXED).stats()
    learned = _run(c, 4, ws=ws, precision=R.PREC_MIXED).stats()
    per_plain = plain["linear_its"] / plain["linear_solves"]
    per_ws = learned["linear_its"] / learned["linear_solves"]
    print(f"FGMRES iterations per solve: plain {per_plain:.2f} ({plain['linear_solves']} solves), "
          f"warm start {per_ws:.2f} ({learned['linear_solves']} solves, mean ||r0||/||b|| "
          f"{learned['ws_r0'] / learned['linear_solves']:.3f}, network term kept in {learned['ws_used']})")
    assert per_ws <= per_plain, (per_ws, per_plain)


def test_tcgen05_and_mma_sync_agree_on_a_large_grid():
    """Several 128-voxel tiles with a ragged last one: the two kernel
    families give the same network output to BF16 rounding."""
    rng = np.random.default_rng(9)
    F = nn.bf16_round(rng.standard_normal((6, 23, 37, 8))).astype(np.float32)
    a = R.WarmStart(seed=21)
    P = _to_dict(a.params())
    for k in P:
        P[k] = (P[k][0], 0.05 * rng.standard_normal(P[k][1].shape))
    a.set_params(_to_flat(P).astype(np.float32))
    a.use_tcgen05(True)
    ya = a.forward(F)
    a.use_tcgen05(False)
    yb = a.forward(F)
    assert _rel(ya, yb) <= 1e-2, _rel(ya, yb)
