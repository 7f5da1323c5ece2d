"""Train the learned warm start on solves the simulator records itself.

The network (a 3D U-Net, see include/resim.h) predicts the Newton update
from the Newton residual, ln k, s_w and the previous update.  Its training
data are the linear systems of ordinary simulator runs: `--members` seeded
permeability realisations of the 1M-cell case's physics (channelised
two-facies field, 13 wells scaled to the grid, 10-day steps) on a 64x64x16
grid, each advanced `--steps` time steps with every solve recorded (its
features and its solved update), on the GPU.  Training runs the network's
own BF16 forward and backward kernels with Adam; the recorded systems stay in
device memory (about 2.6 MB each).

The weights are written to an .npz file (the flat FP32 parameter vector in
the layout of sim_ws_params, plus a description of the data), which
bench.py loads for its learned-warm-start variant.

  python -m paper_1701_06254_gb300.train_warm_start [--members 200] [--steps 28]
         [--epochs 3] [--out paper_1701_06254_gb300/warm_start_64x64x16.npz]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "warm_start_64x64x16.npz")


def record_and_train(members=200, steps=28, epochs=3, batch=4, lr=1e-3, seed0=1000, grid=(64, 64, 16),
                     precision=None, decoupling=2, log=print):
    """Record the solves of `members` realisations (seeds seed0 + k) and
    train a fresh network on them; returns (network, info)."""
    import torch  # noqa: F401  (device context for the library)
    import paper_1701_06254_gb300 as R
    from paper_1701_06254_gb300 import inputs as I
    prec = R.PREC_MIXED_BF16 if precision is None else precision
    ws = R.WarmStart(seed=7)
    t0 = time.perf_counter()
    failed = 0
    for k in range(members):
        c = I.ensemble_member(k, seed0=seed0, size_lo=grid, size_hi=grid)
        g = R.Sim(c, precision=prec, decoupling=decoupling, max_lin=200)
        g.init_hydrostatic()
        g.record_to(ws)
        try:
            g.advance(steps)
        except R.SimError:
            failed += 1                      # a member that stalls keeps the solves it recorded
        g.record_to(None)
        del g
        if log and (k + 1) % 20 == 0:
            log(f"recorded {k + 1} members, {ws.dataset_size()} systems, {time.perf_counter() - t0:.0f} s")
    t1 = time.perf_counter()
    n = ws.dataset_size()
    l0 = ws.eval()
    losses = []
    for e in range(epochs):
        losses.append(ws.train(epochs=1, batch=batch, lr=lr, seed=11 + e))
        if log:
            log(f"epoch {e + 1}: mean loss {losses[-1]:.4f}")
    t2 = time.perf_counter()
    info = {"train_grid": "x".join(str(v) for v in grid), "members": members, "seeds": [seed0, seed0 + members - 1],
            "steps": steps, "samples": n, "epochs": epochs, "batch": batch, "lr": lr, "loss_before": l0,
            "epoch_losses": losses, "loss_after": ws.eval(), "record_s": t1 - t0, "train_s": t2 - t1,
            "members_stopped_early": failed}
    return ws, info


def save(ws, info, path=DEFAULT_OUT):
    np.savez(path, params=ws.params(), info=json.dumps(info))


def load(path=DEFAULT_OUT):
    """(flat FP32 parameters, info dict) from a file written by save()."""
    d = np.load(path, allow_pickle=False)
    return d["params"].astype(np.float32), json.loads(str(d["info"]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--members", type=int, default=200)
    ap.add_argument("--steps", type=int, default=28)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=DEFAULT_OUT)
    a = ap.parse_args()
    ws, info = record_and_train(a.members, a.steps, a.epochs, a.batch, a.lr)
    save(ws, info, a.out)
    print(json.dumps(info))


if __name__ == "__main__":
    main()
