"""Learned warm start: training data from the method's own solves, training
of the warm-start network on the GPU, and the warm-vs-cold evaluation.

The network (include/spfom_mlp.h) maps per-resource features of an instance
to its bid prices y / mean(r). Training targets are the averaged duals at
which the plain binary64 method reaches KKT <= 1e-4, obtained with batched
solves (spfom_load_batch); features come from spfom_features; forward,
backward and Adam run in the library's tensor-core kernels. Nothing here
computes any part of the method: this module marshals instances, calls the
C ABI and keeps the bookkeeping.

Command line (one GPU):

    python -m paper_2602_22421_gb300.warmstart --train 10000 --test 512 \\
        --out paper_2602_22421_gb300/data/warmstart_mlp.npz --report report.json
"""
from __future__ import annotations

import argparse
import json
import os
import time
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import get_context

import numpy as np

from .spfom import MLP, MLP_PARAMS, Solver

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "warmstart_mlp.npz")
TRAIN_SEED, TEST_SEED = 5, 6


def _make(args):
    from instances import warm_family
    seed, k, lo, hi = args
    return warm_family(seed, k, lo, hi)


def instances(seed: int, ks, L_lo: float = 1e4, L_hi: float = 5e4, pool=None):
    """warm_family instances for the indices ks (in a process pool if given)."""
    jobs = [(seed, int(k), L_lo, L_hi) for k in ks]
    return list(pool.map(_make, jobs)) if pool is not None else [_make(j) for j in jobs]


def solve_batch(insts, precision: int = 64, **params):
    """Batched plain solve to KKT <= 1e-4: (per-instance averaged duals, stats)."""
    with Solver(None, device=0, precision=precision, **params) as s:
        s.load_batch(insts)
        s.solve()
        y = s.duals(averaged=True)
        per = s.batch_stats()
    out, i0 = [], 0
    for inst in insts:
        out.append(y[i0:i0 + inst.m].copy())
        i0 += inst.m
    return out, per


def features_of(insts, solver=None):
    """Per-resource features [sum m, 16] (float32, host) of each instance."""
    own = solver is None
    s = solver or Solver(None, device=0)
    try:
        rows = []
        for inst in insts:
            s.load(inst)
            rows.append(s.features().cpu().numpy().copy())
        return rows
    finally:
        if own:
            s.close()


def build_dataset(n_inst: int, seed: int = TRAIN_SEED, chunk: int = 64, L_lo: float = 1e4, L_hi: float = 5e4,
                  workers: int = 8, log=print, **params):
    """Generate, solve and featurise n_inst instances in chunks (generation of
    the next chunk overlaps the solves of the current one). Returns X [R, 16],
    T [R] (targets y* / mean(r)) as float32 host arrays and a summary."""
    X, T = [], []
    unconverged = 0
    t0 = time.time()
    ctx = get_context("spawn")
    with ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as pool, Solver(None, device=0) as fs:
        starts = list(range(0, n_inst, chunk))
        nxt = pool.map(_make, [(seed, k, L_lo, L_hi) for k in range(0, min(chunk, n_inst))])
        for ci, a in enumerate(starts):
            insts = list(nxt)
            if ci + 1 < len(starts):
                b = starts[ci + 1]
                nxt = pool.map(_make, [(seed, k, L_lo, L_hi) for k in range(b, min(b + chunk, n_inst))])
            ys, per = solve_batch(insts, **params)
            unconverged += sum(1 for p in per if not p["converged"])
            feats = features_of(insts, fs)
            for inst, y, f in zip(insts, ys, feats):
                X.append(f)
                T.append((y / float(np.mean(inst.r))).astype(np.float32))
            if log and (ci % 16 == 0 or ci + 1 == len(starts)):
                log(f"  dataset: {min(a + chunk, n_inst)}/{n_inst} instances, {time.time() - t0:.1f} s")
    return np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32), {
        "instances": n_inst, "rows": int(sum(len(t) for t in T)), "unconverged": unconverged,
        "seconds": time.time() - t0}


def train(X, T, epochs: int = 30, batch_rows: int = 16384, lr: float = 1e-3, seed: int = 0, log=print):
    """Train a new network on (X, T) with minibatch Adam; returns it."""
    import torch
    net = MLP(0, seed=seed)
    rng = np.random.default_rng(seed)
    R = len(T)
    steps = 0
    for ep in range(epochs):
        perm = rng.permutation(R)
        xs = torch.from_numpy(X[perm]).cuda()
        ts = torch.from_numpy(T[perm]).cuda()
        tot, cnt = 0.0, 0
        rate = lr * (0.5 * (1 + np.cos(np.pi * ep / epochs)))  # cosine decay over the epochs
        for a in range(0, R, batch_rows):
            b = min(R, a + batch_rows)
            if b - a < 64:
                continue
            loss = net.train_step(xs[a:b], ts[a:b], rate)
            tot += loss * (b - a)
            cnt += b - a
            steps += 1
        if log and (ep % 5 == 0 or ep + 1 == epochs):
            log(f"  epoch {ep}: mse {tot / max(cnt, 1):.4e} (lr {rate:.2e}, {steps} steps)")
    return net


def save(net: MLP, path: str, meta: dict | None = None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez_compressed(path, params=net.params, meta=json.dumps(meta or {}))


def load(path: str = DEFAULT_WEIGHTS) -> MLP:
    d = np.load(path)
    p = d["params"].astype(np.float32)
    if p.shape != (MLP_PARAMS,):
        raise ValueError(f"{path}: expected {MLP_PARAMS} parameters, got {p.shape}")
    net = MLP(0)
    net.params = p
    return net


def evaluate(net: MLP, insts, precision: int = 64, log=None, **params):
    """Cold (spfom_solve from y = 0) and warm (spfom_solve_warm) solves of each
    instance, timed on the host around the call (the warm time includes the
    features and the forward pass). Each instance first runs one evaluation
    period untimed, so that both timed solves replay already captured graphs.
    Returns per-instance records."""
    import torch
    out = []
    with Solver(None, device=0, precision=precision, **params) as s:
        for k, inst in enumerate(insts):
            s.load(inst)
            s.step(s.params.eval_every)
            torch.cuda.synchronize()
            t = time.perf_counter()
            cold = s.solve()
            tc = time.perf_counter() - t
            t = time.perf_counter()
            warm, mode = s.solve_warm(net)
            tw = time.perf_counter() - t
            rec = {"name": inst.name, "cold_s": tc, "warm_s": tw, "cold_iters": cold["iters"],
                   "warm_iters": warm["iters"], "mode": mode, "cold_conv": cold["converged"],
                   "warm_conv": warm["converged"], "cold_dual": cold["dual_avg"], "warm_dual": warm["dual_avg"],
                   "cold_kkt": cold["kkt"], "warm_kkt": warm["kkt"]}
            out.append(rec)
            if log and k % 64 == 0:
                log(f"  eval {k}: cold {tc * 1e3:.1f} ms / {cold['iters']} it, warm {tw * 1e3:.1f} ms / "
                    f"{warm['iters']} it (mode {mode})")
    return out


def summarize(recs) -> dict:
    c = np.array([r["cold_s"] for r in recs])
    w = np.array([r["warm_s"] for r in recs])
    ci = np.array([r["cold_iters"] for r in recs])
    wi = np.array([r["warm_iters"] for r in recs])
    rel = np.array([abs(r["warm_dual"] - r["cold_dual"]) / max(abs(r["cold_dual"]), 1e-30) for r in recs])
    modes = [r["mode"] for r in recs]
    return {"instances": len(recs), "cold_mean_s": float(c.mean()), "warm_mean_s": float(w.mean()),
            "cold_median_s": float(np.median(c)), "warm_median_s": float(np.median(w)),
            "speedup_mean": float(c.mean() / w.mean()), "cold_mean_iters": float(ci.mean()),
            "warm_mean_iters": float(wi.mean()), "warm_faster_frac": float(np.mean(w < c)),
            "mode_counts": {str(k): modes.count(k) for k in (0, 1, 2)},
            "all_converged": bool(all(r["cold_conv"] and r["warm_conv"] for r in recs)),
            "max_objective_rel_diff": float(rel.max()), "max_kkt": float(max(max(r["cold_kkt"], r["warm_kkt"])
                                                                              for r in recs))}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train", type=int, default=10_000)
    ap.add_argument("--test", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--workers", type=int, default=12)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--report", default=None)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    t0 = time.time()
    X, T, info = build_dataset(a.train, TRAIN_SEED, a.chunk, workers=a.workers)
    print(f"dataset: {info}", flush=True)
    t1 = time.time()
    net = train(X, T, epochs=a.epochs, lr=a.lr)
    train_s = time.time() - t1
    save(net, a.out, {"train_instances": a.train, "rows": int(len(T)), "epochs": a.epochs, "lr": a.lr,
                      "train_seed": TRAIN_SEED, "family": "warm_family(n=2000,m=400,L=10^U(4,4.7),K=U{10..30},c=0.4d)"})
    ctx = get_context("spawn")
    with ProcessPoolExecutor(max_workers=a.workers, mp_context=ctx) as pool:
        test = instances(TEST_SEED, range(a.test), pool=pool)
    recs = evaluate(net, test, log=print)
    summ = summarize(recs)
    summ.update({"dataset": info, "train_seconds": train_s, "total_seconds": time.time() - t0})
    print(json.dumps(summ, indent=1), flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump({"summary": summ, "records": recs}, f)


if __name__ == "__main__":
    main()
