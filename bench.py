"""Benchmark: cell-timesteps/s of the GPU CPR-FGMRES Newton path.

A step is one time step of the 200x200x25 channelised case (1M cells,
13 wells, dt = 10 days): Newton iterations with assembly, Quasi-IMPES
decoupling (ABF with --decoupling abf), per-subdomain potential reordering,
RAS/BILU(0) and PMIS-AMG setup and
CPR-FGMRES solves to relres 1e-6, all on the device.  Inputs are resident
in HBM when the timed region starts; the working set (2x2 BSR Jacobian,
Krylov basis) is larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed_bf16|mixed|fp64]
                  [--decoupling qi|abf|none] [--no-reorder] [--breakdown]
  python bench.py --impl reference     # the CPU oracle on the same workload
  python bench.py --workload ensemble  # 128 independent models (~16.6M cells) on one GPU
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-timesteps/s at 1M cells, relres 1e-6: mixed+learned vs plain FP64; %HBM peak"
# decoupling codes, the same in the CUDA library (SIM_DEC_*) and the oracle
DECOUPLING = {"none": 0, "abf": 1, "qi": 2}
KRYLOV = {"fgmres": 0, "bicgstab": 1}
INTERP = {"direct": 0, "exti": 1}
NEWTON = {"standard": 0, "inexact": 1}


def oracle_opts(args):
    """The oracle's options for the configuration the GPU arm runs."""
    tx, ty = (int(v) for v in args.tile.split("x"))
    o = dict(max_lin=args.max_lin, decoupling=DECOUPLING[args.decoupling], reorder=0 if args.no_reorder else 1,
             tile_x=tx, tile_y=ty, krylov=KRYLOV[args.krylov], overlap=args.overlap, interp=INTERP[args.interp])
    if args.newton:
        o["newton"] = NEWTON[args.newton]
    return o


UNIT = "cell-timesteps/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clock, power and throttle reasons."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            v = [x.strip() for x in line.split(",")]
            if len(v) >= 9:
                try:
                    rows.append((float(v[1]), float(v[2]), float(v[3]), v[5], v[6], v[7], v[8]))
                except ValueError:
                    pass
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        for r in rows:
            for name, flag in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[3:]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


def ras_bytes(ls, precision):
    """Algorithmic bytes of one RAS apply with the packed per-subdomain
    factors: every off-diagonal factor block (values + 2-byte column) and
    every row's record (gather index, six 2-byte row/level indices, inverse
    diagonal block) read once, the extended right-hand side gathered and the
    owned rows written.  In mixed precision both applications of Algorithm 2
    read an FP32 input (the basis vector's hi plane, then the FP32 residual);
    the first overwrites its output, the second accumulates into it, so the
    output bytes are their average."""
    vb = {"mixed": 16, "mixed_bf16": 8, "fp64": 32}[precision]
    nsub = ls.ras_count()
    nnz = nxt = own = 0
    for s in range(nsub):
        o, e, z = ls.ras_sizes(s)
        own += o; nxt += e; nnz += z
    off = nnz - nxt
    if precision == "fp64":
        gather, scatter = 16.0, 24.0          # double2 in; write, or read + write
    else:
        gather, scatter = 8.0, 12.0           # float2 in; float2 write, or read + write
    return off * (vb + 2) + nxt * (4 + 12 + vb) + nxt * gather + own * scatter


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
# ncu captures summarised in profiles/, keyed by (kernel family, precision,
# decoupling): a capture is quoted only for the configuration it was taken in
# (null otherwise, and null once the kernel changes)
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# ncu captures of the benchmark's own command (profiles/dram_traffic_channelised_1m.md),
# keyed on (kernel family, precision, decoupling); a configuration without a
# capture of the current kernels reports null
NCU_TRAFFIC = {("ras", "mixed_bf16", "qi"): 202.0e6, ("spmv_prec", "mixed_bf16", "qi"): 165.7e6,
               ("spmv64", "mixed_bf16", "qi"): 271.3e6, ("vcycle", "mixed_bf16", "qi"): 351.7e6}


def ncu_traffic(kernel, args):
    return NCU_TRAFFIC.get((kernel, args.precision, args.decoupling))


def spmv_bytes(nb, nnzb, val_b, x_b, f_b, y_b):
    return nnzb * (val_b + 4) + (nb + 1) * 4 + 2 * nb * (x_b + f_b + y_b)


def spmv_prec_bytes(nb, nnzb, n, precision):
    """The FP32 residual SpMV of a CPR application (r = v - A z): in mixed
    precision the first of its two launches also writes the pressure residual
    (4 B per cell) and the second reads the pressure correction and writes
    the corrected iterate (4 + 8 B per block row); the mean per launch is
    counted."""
    if precision == "fp64":
        return spmv_bytes(nb, nnzb, 32, 8, 8, 8)
    return spmv_bytes(nb, nnzb, 16, 4, 4, 4) + (4 * n + 4 * n + 8 * nb) // 2


def vcycle_bytes(ls, precision):
    """Algorithmic bytes of one V-cycle: on every level but the coarsest the
    pre- and post-smoothing sweeps each read A_l (value + column) and its row
    pointers once, the restriction reads R = P^T, the prolongation P, and
    each sweep reads / writes its vectors once (pre: f, D^-1 in, x, r out;
    restriction: r in, f_c, D_c^-1 f_c out and D_c^-1 in; prolongation: x,
    e in, t out; post: f, t, D^-1 in, x out); the coarsest level reads its
    dense FP64 inverse."""
    vb = 8 if precision == "fp64" else 4
    total = 0
    nlev = ls.amg_nlev()
    for l in range(nlev):
        d = ls.amg_level(l)
        n, nnz = d["n"], d["nnz"]
        if l == nlev - 1:
            total += (n * n * 8 + 2 * n * vb) if d["coarse_dense"] else 10 * (nnz * (vb + 4) + (n + 1) * 4 + 4 * n * vb)
            break
        nc, nnzP = d["nc"], d["nnzP"]
        a = nnz * (vb + 4) + (n + 1) * 4
        total += 2 * a + 8 * n * vb                              # pre + post: matrix twice, 8 vectors
        total += nnzP * (vb + 4) + (nc + 1) * 4 + n * vb + 3 * nc * vb      # restriction
        total += nnzP * (vb + 4) + (n + 1) * 4 + 2 * n * vb + nc * vb       # prolongation
    return total


def state_difference(a, b):
    """Largest per-cell differences between two states (p, s_w) of the same
    grid: relative in pressure (to b's), absolute in water saturation."""
    pa, sa = (np.asarray(x, np.float64) for x in a[:2])
    pb, sb = (np.asarray(x, np.float64) for x in b[:2])
    return {"p_rel_max": float(np.max(np.abs(pa - pb) / np.abs(pb))), "sw_abs_max": float(np.max(np.abs(sa - sb)))}


def _host_state(sim):
    """(p, s_w) copied to the host, or None (never raises: a comparison is
    reported, not required)."""
    try:
        p, sw = sim.get_state()[:2]
        return np.array(p), np.array(sw)
    except Exception:
        return None


def oracle_timed_step(case, opts, state, omp):
    """One time step of the CPU oracle from a given state (p, s_w, p_b, t):
    the same step the GPU arm times first, on one core (omp=False) or with
    the OpenMP build on all host cores (bit-identical results).  Returns
    (seconds, Newton iterations, FGMRES iterations, return code)."""
    import oracle
    s = oracle.Sim(case, omp=omp, **opts)
    p, sw, pb, t = state
    s.set_state(np.asarray(p, np.float64), np.asarray(sw, np.float64), np.asarray(pb, np.float64), t)
    t0 = time.perf_counter()
    rc = s.advance(1)
    t1 = time.perf_counter()
    st = s.stats()
    return t1 - t0, st["newton"], st["lin"], rc


def oracle_newton_iteration(case, opts):
    """One Newton iteration of the CPU oracle on the first time step of the
    case (assembly + decoupling + reordering + RAS/AMG setup + CPR-FGMRES)."""
    import oracle
    s = oracle.Sim(case, **opts)
    s.init_hydrostatic()
    s.store_old(); s.set_dt(case.dt)
    t0 = time.perf_counter()
    s.assemble()
    rc, y, its, rel = s.linear_solve(case.lin_tol)
    t1 = time.perf_counter()
    return t1 - t0, its


def oracle_full_step(case, opts):
    import oracle
    s = oracle.Sim(case, **opts)
    s.init_hydrostatic()
    t0 = time.perf_counter()
    rc = s.advance(1)
    t1 = time.perf_counter()
    return t1 - t0, rc, s.stats()


def run_reference(args, case, rank):
    if rank != 0:
        return
    dt, rc, st = oracle_full_step(case, oracle_opts(args))
    value = case.n / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": 1, "warmup": 0, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": case.name, "cells": case.n, "dt_days": case.dt, "relres": case.lin_tol,
                   "precision": "fp64", "decoupling": args.decoupling, "reorder": not args.no_reorder},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"the CPU oracle's complete first time step of {case.name} "
                                   f"({st['newton']} Newton iterations, {st['lin']} FGMRES iterations, rc={rc}); "
                                   "--steps/--warmup are not applied: one step is the bounded sample"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def train_warm_start(R, args, opts):
    """The learned warm start's network: the weights trained offline by
    paper_1701_06254_gb300/train_warm_start.py on the solves of 200
    64x64x16 realisations of the 1M-cell case's physics when that file is
    present (--ws-file), else a quick stand-in: record the solves of
    --ws-members 64x64x16 models (seeds 3000 + k, --ws-steps steps each) and
    train on them for --ws-epochs epochs (outside the timed region)."""
    from paper_1701_06254_gb300 import inputs as I
    if args.ws_file and os.path.exists(args.ws_file):
        from paper_1701_06254_gb300 import train_warm_start as T
        params, info = T.load(args.ws_file)
        ws = R.WarmStart(seed=7)
        ws.set_params(params)
        info = dict(info, source=os.path.basename(args.ws_file) + " (trained offline by train_warm_start.py)")
        return ws, info
    t0 = time.perf_counter()
    ws = R.WarmStart(seed=7)
    for k in range(args.ws_members):
        c = I.ensemble_member(k, seed0=3000, size_lo=(64, 64, 16), size_hi=(64, 64, 16))
        g = R.Sim(c, **opts)
        g.init_hydrostatic()
        g.record_to(ws)
        g.advance(args.ws_steps)
        del g
    t1 = time.perf_counter()
    n = ws.dataset_size()
    l0 = ws.eval()
    loss = ws.train(epochs=args.ws_epochs, batch=4, lr=1e-3, seed=1)
    t2 = time.perf_counter()
    return ws, {"train_grid": "64x64x16", "members": args.ws_members, "steps": args.ws_steps, "samples": n,
                "epochs": args.ws_epochs, "loss_before": l0, "loss_after": ws.eval(), "last_epoch_loss": loss,
                "record_s": t1 - t0, "train_s": t2 - t1}


def measure_variant(R, torch, case, opts, args, ws=None):
    """One more configuration of the same workload, timed like the main run
    (W warm-up steps, K timed steps between CUDA events on the device)."""
    sim = R.Sim(case, **opts)
    sim.init_hydrostatic()
    if ws is not None:
        sim.attach_warm_start(ws)
        sim.ls.kernel_timer([R.T_WARMSTART, R.T_NETWORK])   # before the warm-up, as in the main run
    for _ in range(args.warmup):
        sim.advance(1)
    if ws is not None:
        sim.ls.kernel_timer([R.T_WARMSTART, R.T_NETWORK])   # counters reset
    st0 = sim.stats()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sim.advance(1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st1 = sim.stats()
    dn = st1["newton"] - st0["newton"]
    dl = max(1, st1["linear_solves"] - st0["linear_solves"])
    out = {"value": case.n * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
           "newton_per_step": dn / args.steps, "fgmres_its_per_newton": (st1["linear_its"] - st0["linear_its"]) / max(1, dn)}
    if ws is not None:
        out["warm_start"] = {"ms_per_step": sim.ls.kernel_time(R.T_WARMSTART)[1] / args.steps,
                             "network_ms_per_step": sim.ls.kernel_time(R.T_NETWORK)[1] / args.steps,
                             "network_term_kept": st1["ws_used"] - st0["ws_used"],
                             "network_term_dropped": st1["ws_fallback"] - st0["ws_fallback"],
                             "mean_r0_over_b": (st1["ws_r0"] - st0["ws_r0"]) / dl}
    out["_state"] = _host_state(sim)          # dropped before printing
    del sim
    return out


# ---- cross-rank reductions (one process per GPU; gloo on CPU in the tests)
def rank_max(x, dist, device):
    """Largest x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_sum(x, dist, device):
    """Sum of x over all ranks (units processed by the whole job)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def ensemble_seed0(rank, members):
    """First member seed of a rank: ranks draw disjoint seed ranges."""
    return 2000 + rank * members


def time_ensemble(R, torch, args, cases, prec, dec, dist, local, steps, warmup):
    """Advance the members together through the ensemble driver (host
    workers chosen by the autotuner unless --workers is a number): `warmup`
    untimed steps, then `steps` timed ones between device-wide
    synchronisations (members run on streams of their own), on the host
    clock, max over ranks."""
    auto = args.workers == "auto"
    batch = R.Batch(cases, workers=0 if auto else int(args.workers), precision=prec, max_lin=args.max_lin,
                    decoupling=dec)
    batch.init_hydrostatic()
    tuned = None
    if auto:
        chosen, secs = batch.autotune(candidates=(4, 8, 16, 32))
        tuned = {"chosen": chosen, "seconds_per_candidate": secs}
    for _ in range(warmup):
        batch.advance(1)
    st0 = [m.stats() for m in batch.members]
    clocks = Clocks(local)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = R.launch_count()
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(steps):
        batch.advance(1)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    ck = clocks.stop()
    launches = R.launch_count() - l0
    sec = rank_max(sec, dist, "cuda")
    st1 = [m.stats() for m in batch.members]
    out = {"seconds": sec, "launches": launches, "clocks": ck, "autotune": tuned, "workers": batch.workers,
           "newton": sum(b["newton"] - a["newton"] for a, b in zip(st0, st1)),
           "linear_its": sum(b["linear_its"] - a["linear_its"] for a, b in zip(st0, st1))}
    del batch
    return out


def run_ensemble(args, rank, world, local):
    """--members independent models (grids drawn from U{32..128}^2 x U{8..32},
    seeds 2000 + k) advanced together by the ensemble driver.  Each rank of a
    multi-GPU run takes the same number of members with its own seeds (weak
    scaling, no collective on the data path).  Members run on streams of their
    own, so the timed region is bracketed by device-wide synchronisations and
    read on the host clock."""
    from paper_1701_06254_gb300 import inputs as I
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the single-model workload; "
                              "run it without --workload ensemble"}), flush=True)
        return
    import torch
    import paper_1701_06254_gb300 as R
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = {"mixed": R.PREC_MIXED, "mixed_bf16": R.PREC_MIXED_BF16, "fp64": R.PREC_FP64}[args.precision]
    cases = I.ensemble(args.members, seed0=ensemble_seed0(rank, args.members))
    cells = sum(c.n for c in cases)
    dec = DECOUPLING[args.decoupling]
    e = time_ensemble(R, torch, args, cases, prec, dec, dist, local, args.steps, args.warmup)
    sec, launches, ck, tuned, workers_used = e["seconds"], e["launches"], e["clocks"], e["autotune"], e["workers"]
    cells_all = rank_sum(cells, dist, "cuda")           # each rank's members differ in size
    newton, lin = e["newton"], e["linear_its"]
    # the same ensemble with the learned warm start: the network is trained
    # first (outside the timing) and every member gets its own copy of it
    # (same parameters; a network serves one caller at a time, so members
    # sharing one would queue on it)
    variants = None
    if not args.no_variants:
        ws, info = train_warm_start(R, args, dict(precision=prec, max_lin=args.max_lin, decoupling=dec))
        params = ws.params()
        b2 = R.Batch(cases, workers=workers_used, precision=prec, max_lin=args.max_lin, decoupling=dec)
        b2.init_hydrostatic()
        copies = []
        for m in b2.members:
            w = R.WarmStart(seed=7)
            w.set_params(params)
            copies.append(w)
            m.attach_warm_start(w)
        for _ in range(args.warmup):
            b2.advance(1)
        s0 = [m.stats() for m in b2.members]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            b2.advance(1)
        torch.cuda.synchronize()
        sec2 = rank_max(time.perf_counter() - t1, dist, "cuda")
        s1 = [m.stats() for m in b2.members]
        n2 = sum(b["newton"] - a["newton"] for a, b in zip(s0, s1))
        variants = {"learned": {"value": cells_all * args.steps / sec2, "ms_per_step": sec2 * 1e3 / args.steps,
                                "fgmres_its_per_newton": sum(b["linear_its"] - a["linear_its"]
                                                             for a, b in zip(s0, s1)) / max(n2, 1),
                                "network_term_kept": sum(b["ws_used"] - a["ws_used"] for a, b in zip(s0, s1)),
                                "fallback": sum(b["ws_fallback"] - a["ws_fallback"] for a, b in zip(s0, s1)),
                                "training": info}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": cells_all * args.steps / sec, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f64+f32", "mixed_bf16": "f64+f32+bf16", "fp64": "f64"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"ensemble_{args.members}", "members": args.members, "cells": cells,
                       "cells_all_ranks": int(cells_all),
                       "precision": args.precision, "decoupling": args.decoupling, "workers": workers_used,
                       "autotune": tuned,
                       "timer": "host clock between device-wide synchronisations (members on their own streams)",
                       "newton_per_member_step": newton / (len(cases) * args.steps),
                       "fgmres_its_per_newton": lin / max(newton, 1),
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "working set larger than L2 (no flush needed)"},
            "roofline": None, "gpu_launches": launches, "e2e": None, "cpu_baseline": None, "clocks": ck,
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="channelised", choices=["lognormal", "fivespot", "channelised"],
                    help="workload: the 1M-cell channelised case (default), the 200k-cell five-spot or the "
                         "2,000-cell log-normal case")
    ap.add_argument("--precision", default="mixed_bf16", choices=["mixed", "mixed_bf16", "fp64"],
                    help="preconditioner precision: FP32 AMG/ILU with BF16 RAS values (the 1M-cell case's "
                         "setting), FP32 throughout, or FP64")
    ap.add_argument("--max-lin", type=int, default=200)
    ap.add_argument("--tile", default="4x4", help="RAS subdomain tile, columns x rows of cells")
    ap.add_argument("--decoupling", default="qi", choices=["abf", "qi", "none"],
                    help="decoupling of the Newton system (eq. 29): Quasi-IMPES (default, with the potential "
                         "reordering the paper's configuration for its SPE10 runs), ABF or none")
    ap.add_argument("--no-reorder", action="store_true", help="switch off the local potential reordering")
    ap.add_argument("--krylov", default="fgmres", choices=["fgmres", "bicgstab"],
                    help="Krylov method: FGMRES(50) (default) or BiCGSTAB, both right-preconditioned by CPR")
    ap.add_argument("--newton", default=None, choices=["standard", "inexact"],
                    help="Newton variant (default: the workload's own; the 1M-cell case runs standard Newton "
                         "at relres 1e-6)")
    ap.add_argument("--overlap", type=int, default=1, choices=[1, 2], help="RAS overlap")
    ap.add_argument("--interp", default="direct", choices=["direct", "exti"], help="AMG interpolation")
    ap.add_argument("--fp64-basis", action="store_true",
                    help="mixed precision with the FGMRES basis, w = A z and Gram-Schmidt in FP64 instead of "
                         "double-float")
    ap.add_argument("--roofline", default="ras", choices=["ras", "spmv64", "spmv_prec"])
    ap.add_argument("--workload", default="single", choices=["single", "ensemble"],
                    help="single: the 1M-cell case; ensemble: --members independent models advanced together")
    ap.add_argument("--members", type=int, default=128)
    ap.add_argument("--ens-members", type=int, default=32,
                    help="members of the ensemble variant of the single-model run (0: none)")
    ap.add_argument("--ens-steps", type=int, default=2)
    ap.add_argument("--workers", default="auto", help="ensemble host workers, or 'auto' for the autotuner")
    ap.add_argument("--learned", action="store_true",
                    help="train the warm-start network on recorded 64x64x16 solves first and attach it")
    ap.add_argument("--ws-file", default=os.path.join(ROOT, "paper_1701_06254_gb300", "warm_start_64x64x16.npz"),
                    help="trained warm-start weights (train_warm_start.py); when missing, a short stand-in training")
    ap.add_argument("--ws-members", type=int, default=8)
    ap.add_argument("--ws-steps", type=int, default=5)
    ap.add_argument("--ws-epochs", type=int, default=10)
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the plain-FP64 and mixed+learned comparison runs")
    ap.add_argument("--exti-variant", action="store_true", help="also time extended+i interpolation")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra-rooflines", action="store_true",
                    help="skip the extra step that times the SpMVs and the V-cycle for their rooflines")
    ap.add_argument("--breakdown", action="store_true",
                    help="time every kernel family with CUDA events (adds event records between launches)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_1701_06254_gb300 import inputs as I
    if args.workload == "ensemble":
        run_ensemble(args, rank, world, local)
        return
    case = I.CASES[args.config]()
    if args.impl == "reference":
        run_reference(args, case, rank)
        return

    import torch
    import paper_1701_06254_gb300 as R
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = {"mixed": R.PREC_MIXED, "mixed_bf16": R.PREC_MIXED_BF16, "fp64": R.PREC_FP64}[args.precision]
    tx, ty = (int(v) for v in args.tile.split("x"))
    opts = dict(precision=prec, max_lin=args.max_lin, tile_x=tx, tile_y=ty,
                decoupling=DECOUPLING[args.decoupling],
                reorder=0 if args.no_reorder else 1, krylov=KRYLOV[args.krylov], overlap=args.overlap,
                interp=INTERP[args.interp], fp64_basis=1 if args.fp64_basis else 0)
    if args.newton:
        opts["newton"] = NEWTON[args.newton]
    ws_info = False
    ws = None
    if args.learned:
        ws, ws_info = train_warm_start(R, args, opts)
    sim = R.Sim(case, **opts)
    sim.init_hydrostatic()
    if ws is not None:
        sim.attach_warm_start(ws)
    # timers on before the warm-up: enabling them changes what the Arnoldi-step
    # graph records, and that recording belongs in the warm-up, not the timed steps
    fam = {"ras": R.T_RAS, "spmv64": R.T_SPMV64, "spmv_prec": R.T_SPMV_PREC}[args.roofline]
    fams = range(1, R.T_NFAMILIES) if args.breakdown else [fam]
    sim.ls.kernel_timer(fams)
    for _ in range(args.warmup):
        sim.advance(1)
    # the state the timed steps start from, so that the end-to-end pass below
    # replays exactly the same steps
    saved = None
    if not (args.no_e2e and args.no_cpu_baseline):
        nw = len(case.wells)
        saved = (torch.empty(case.n, dtype=torch.float64, pin_memory=True),
                 torch.empty(case.n, dtype=torch.float64, pin_memory=True),
                 torch.empty(max(nw, 1), dtype=torch.float64, pin_memory=True))
        t_saved = sim.get_state(saved)[3]
    sim.ls.kernel_timer(fams)                 # same families: counters reset, recording kept
    st0 = sim.stats()
    clocks = Clocks(local)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = R.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    e0.record()
    for _ in range(args.steps):
        sim.advance(1)
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = R.launch_count() - l0
    ms = rank_max(ms, dist, "cuda")
    if dist:
        dist.barrier()
    st1 = sim.stats()
    end_state = _host_state(sim)              # after the timed region; compared with the FP64 variant below
    nk, kms = sim.ls.kernel_time(fam)
    breakdown = None
    if args.breakdown:
        breakdown = {}
        for f, name in R.T_NAMES.items():
            n_, t_ = sim.ls.kernel_time(f)
            breakdown[name] = {"launches": n_, "ms_per_step": t_ / args.steps, "share": t_ / ms}
    value = world * case.n * args.steps / (ms / 1e3)
    newton_per_step = (st1["newton"] - st0["newton"]) / args.steps
    its_per_newton = (st1["linear_its"] - st0["linear_its"]) / max(1, st1["newton"] - st0["newton"])

    # level structure of the reordered subdomain factors (sets the latency of the RAS solves)
    nsub = sim.ls.ras_count()
    lv = [sim.ls.ras_levels(s_)[:2] for s_ in range(0, nsub, max(1, nsub // 64))]
    ras_levels = {"subdomains": nsub, "sampled": len(lv),
                  "L_mean": float(np.mean([a for a, _ in lv])), "L_max": int(max(a for a, _ in lv)),
                  "U_mean": float(np.mean([b_ for _, b_ in lv])), "U_max": int(max(b_ for _, b_ in lv))}

    # roofline of the chosen kernel family (algorithmic bytes / event time)
    rp = sim.ls.export(R.X_ROWPTR, 0, np.int32)
    nb, nnzb = len(rp) - 1, int(rp[-1])
    if args.roofline == "ras":
        bpl = ras_bytes(sim.ls, args.precision)
    elif args.roofline == "spmv64":
        bpl = spmv_bytes(nb, nnzb, 32, 8 if args.precision == "fp64" else 4, 0, 8)
    else:
        bpl = spmv_prec_bytes(nb, nnzb, case.n, args.precision)
    peak, src = peaks()
    achieved = bpl / (kms / nk * 1e-3) / 1e9 if nk else 0.0
    roof = {"kernel": args.roofline, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": src, "traffic": ncu_traffic(args.roofline, args),
            "launches": nk,
            "ms_per_launch": kms / nk if nk else None, "algorithmic_bytes_per_launch": bpl}

    # the other memory-bound kernels: one more step with their timers on
    # (a pass of its own, so that the timed steps carry one timer family only)
    rooflines = None
    if not args.no_extra_rooflines:
        others = [("spmv_prec", R.T_SPMV_PREC,
                   spmv_prec_bytes(nb, nnzb, case.n, args.precision)),
                  ("spmv_w", R.T_SPMV64, spmv_bytes(nb, nnzb, 32, 8 if args.precision == "fp64" else 4, 0, 8)),
                  ("vcycle", R.T_VCYCLE, vcycle_bytes(sim.ls, args.precision))]
        sim.ls.kernel_timer([f for _, f, _ in others])
        sim.advance(1)
        rooflines = {}
        for name, f, b in others:
            n_, t_ = sim.ls.kernel_time(f)
            ach = b / (t_ / n_ * 1e-3) / 1e9 if n_ else 0.0
            key = {"spmv_prec": "spmv_prec", "spmv_w": "spmv64", "vcycle": "vcycle"}.get(name)
            rooflines[name] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                               "ms_per_launch": t_ / n_ if n_ else None, "algorithmic_bytes_per_launch": b,
                               "launches": n_, "traffic": ncu_traffic(key, args)}
        sim.ls.kernel_timer(fams)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        nw = len(case.wells)
        hp, hs, hb = (x.clone().pin_memory() for x in saved)   # the timed steps' starting state
        tt = t_saved
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sim.set_state(hp, hs, hb, tt)
            sim.advance(1)
            tt = sim.get_state((hp, hs, hb))[3]
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te = rank_max(te, dist, "cuda")
        e2e = {"value": world * case.n * args.steps / te, "unit": UNIT,
               "h2d_bytes_per_step": (2 * case.n + nw) * 8, "d2h_bytes_per_step": (2 * case.n + nw) * 8}

    # the method's two reference points on the same workload: plain FP64
    # CPR-FGMRES and the mixed-precision path with the learned warm start
    variants = None
    if not args.no_variants:
        variants = {"plain_fp64": measure_variant(R, torch, case, dict(opts, precision=R.PREC_FP64), args)}
        if ws is None:
            ws, info = train_warm_start(R, args, opts)
        else:
            info = ws_info
        lv = measure_variant(R, torch, case, opts, args, ws)
        lv["training"] = info
        variants[args.precision + "_learned"] = lv
        if prec != R.PREC_FP64:
            # the precision split as first specified: FP32/BF16 preconditioner,
            # FGMRES basis, w = A z and Gram-Schmidt in FP64
            variants[args.precision + "_fp64_basis"] = measure_variant(R, torch, case, dict(opts, fp64_basis=1), args)
        # the paper's other solver settings on the same workload: inexact Newton
        # (eq. 26, Eisenstat-Walker forcing), BiCGSTAB (Tables 2, 3, 6) and
        # RAS overlap 2 (Table 9); extended+i AMG only with --exti-variant
        # (without truncation of P its coarse operators grow dense here)
        variants["inexact_newton"] = measure_variant(R, torch, case, dict(opts, newton=1), args)
        variants["bicgstab"] = measure_variant(R, torch, case, dict(opts, krylov=1, max_lin=300), args)
        variants["ras_overlap2"] = measure_variant(R, torch, case, dict(opts, overlap=2), args)
        if args.exti_variant:
            variants["amg_exti"] = measure_variant(R, torch, case, dict(opts, interp=1), args)
        if args.ens_members > 0:
            # the batched ensemble: --ens-members independent models (grids
            # drawn from U{32..128}^2 x U{8..32}) advanced together
            cases_e = I.ensemble(args.ens_members, seed0=ensemble_seed0(rank, args.ens_members))
            e = time_ensemble(R, torch, args, cases_e, prec, DECOUPLING[args.decoupling], dist, local,
                              args.ens_steps, 3)
            cells_e = rank_sum(sum(c.n for c in cases_e), dist, "cuda")
            variants["ensemble"] = {
                "workload": f"ensemble_{args.ens_members}", "members": args.ens_members, "cells_all_ranks": int(cells_e),
                "value": cells_e * args.ens_steps / e["seconds"], "unit": UNIT,
                "ms_per_step": e["seconds"] * 1e3 / args.ens_steps, "steps": args.ens_steps, "warmup": 3,
                "workers": e["workers"], "autotune": e["autotune"], "gpu_launches": e["launches"],
                "newton_per_member_step": e["newton"] / (args.ens_members * args.ens_steps),
                "fgmres_its_per_newton": e["linear_its"] / max(e["newton"], 1), "clocks": e["clocks"],
                "timer": "host clock between device-wide synchronisations (members on their own streams)"}
    precision_error = None
    if variants is not None:
        states = {k: v.pop("_state", None) for k, v in variants.items()}
        ref = states.pop("plain_fp64", None)
        try:
            if ref is not None and end_state is not None:
                precision_error = {
                    "reference": "the plain FP64 GPU method over the same warm-up and timed steps "
                                 "(it matches the FP64 oracle to 1e-6 in the parity tests)",
                    args.precision: state_difference(end_state, ref)}
                for k, st_ in states.items():
                    if st_ is not None:
                        precision_error[k] = state_difference(st_, ref)
        except Exception as e:                # reported, never fatal
            precision_error = {"error": str(e)[:200]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the first timed step, re-seeded: the oracle starts from the GPU's
        # state at the start of the timed region and advances the same step,
        # once on one core and once with its OpenMP build on all host cores
        import oracle
        state = (saved[0].numpy(), saved[1].numpy(), saved[2].numpy()[:len(case.wells)], t_saved)
        t1c, nn1, li1, rc1 = oracle_timed_step(case, oracle_opts(args), state, omp=False)
        tac, nna, lia, rca = oracle_timed_step(case, oracle_opts(args), state, omp=True)
        thr = oracle.omp_threads()
        cpu = {"value": case.n / t1c, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first timed step of {case.name} (t = {t_saved:g} d, dt = {case.dt:g} d) re-seeded from "
                         f"the GPU state at the start of the timed region: {nn1} Newton and {li1} FGMRES iterations, "
                         f"{t1c:.1f} s on one core (rc {rc1})",
               "all_cores": {"value": case.n / tac, "cores": thr, "nproc": os.cpu_count(), "seconds": tac,
                             "newton": nna, "linear_its": lia, "rc": rca,
                             "build": "OpenMP on the oracle's element-wise loops (bit-identical results)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"mixed": "f64+f32", "mixed_bf16": "f64+f32+bf16", "fp64": "f64"}[args.precision], "data": "synthetic",
            "config": {"workload": case.name, "cells": case.n, "wells": len(case.wells), "dt_days": case.dt,
                       "relres": case.lin_tol, "precision": args.precision, "learned_warm_start": ws_info,
                       "krylov": {"method": args.krylov,
                                  "basis": "fp64" if (args.precision == "fp64" or args.fp64_basis) else "double-float"},
                       "newton": args.newton or case.newton, "ras_overlap": args.overlap, "amg_interp": args.interp,
                       "ras_tile": args.tile, "decoupling": args.decoupling, "reorder": not args.no_reorder,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "working set larger than L2 (no flush needed)",
                       "newton_per_step": newton_per_step, "fgmres_its_per_newton": its_per_newton,
                       "ras_levels": ras_levels},
            "roofline": roof, "rooflines_other": rooflines, "gpu_launches": launches, "e2e": e2e,
            "cpu_baseline": cpu, "clocks": ck,
            "phases_ms_per_step": {k: (st1[k] - st0[k]) / args.steps for k in ("ms_assemble", "ms_setup", "ms_solve")},
            "warm_start": ({"used": st1["ws_used"] - st0["ws_used"], "fallback": st1["ws_fallback"] - st0["ws_fallback"],
                            "mean_r0": (st1["ws_r0"] - st0["ws_r0"]) / max(1, st1["linear_solves"] - st0["linear_solves"])}
                           if ws is not None else None),
            "kernel_breakdown": breakdown,
            "variants": variants,
            "precision_error_vs_fp64": precision_error,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
