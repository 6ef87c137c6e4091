"""Batched multi-period re-solves for bid-price control (Section 5.1).

A network of resources sells over `periods` periods. Each period re-solves
the choice-based LP of every base instance with what is left: the capacity
of period k is the remaining inventory spread over the remaining periods,
c_k = inv_k / (periods - k), the arrival rates are the base rates scaled by
rho[k] ~ U(0.5, 1.5), and the averaged duals of the solve are the bid prices
of the period. The period then sells what bid-price control sells -- every
segment is offered its best assortment at the bid prices, expected sales
s = spfom_sales_at(y) -- and the inventory drops by the consumption A s
(clipped at zero). The initial inventory is `periods` times the base
capacity (c = 0.6 x one period's full-offer demand).

Both take the solver's parameters; the family's smallest instances (about
1e3 segments over thousands of products) need restart_tau_balance > 0 to
reach KKT <= 1e-4 with either form.

``run_batched`` solves all base instances of a period in one batch
(spfom_load_batch once, spfom_update per period, warm-started from the
previous period's bid prices), in the binary32 bulk iteration with the
segment kernel chosen by spfom_autotune and the evaluation periods replayed
as CUDA graphs. ``run_sequential`` re-solves the same (instance, period)
problems one at a time with the plain binary64 method from y = 0, the
reference point of the comparison. The consumption update is host
bookkeeping of the simulation, not part of the method.
"""
from __future__ import annotations

import time

import numpy as np

from .spfom import Solver


def consumption(inst, sales) -> np.ndarray:
    """A s for one instance (host)."""
    a_val = inst.a_val if inst.a_val is not None else np.ones(len(inst.a_idx))
    prod_of = np.repeat(np.arange(inst.n), np.diff(inst.a_ptr))
    return np.bincount(inst.a_idx, weights=a_val * sales[prod_of], minlength=inst.m)


def _split(vec, sizes):
    out, i0 = [], 0
    for k in sizes:
        out.append(vec[i0:i0 + k])
        i0 += k
    return out


def run_batched(insts, rho, periods: int = 16, precision: int = 32, tune: bool = True, log=None, **params):
    """Solve every period of every instance, one batch per period (solver
    parameters `params`). Returns (per-period records, the capacity and rate
    path, per-(period, instance) stats)."""
    import torch
    ms = [i.m for i in insts]
    ns = [i.n for i in insts]
    inv = [periods * np.asarray(i.c, np.float64) for i in insts]
    path, per_stats, recs = [], [], []
    with Solver(None, device=0, precision=precision, **params) as s:
        t = time.perf_counter()
        s.load_batch(insts)
        load_s = time.perf_counter() - t
        choice = s.autotune(64) if tune else None
        y = None
        for k in range(periods):
            c_k = [v / (periods - k) for v in inv]
            lam_k = [i.lam * rho[k, b] for b, i in enumerate(insts)]
            s.update(np.concatenate(c_k), np.concatenate(lam_k))
            torch.cuda.synchronize()
            t = time.perf_counter()
            st = s.solve(y)
            y = s.duals(averaged=True)
            solve_s = time.perf_counter() - t
            stats = s.batch_stats()
            sales = _split(s.sales_at(y), ns)
            for b, inst in enumerate(insts):
                inv[b] = np.maximum(0.0, inv[b] - consumption(inst, sales[b]))
            path.append((c_k, lam_k))
            per_stats.append(stats)
            recs.append({"period": k, "seconds": solve_s, "iters": st["iters"], "converged": st["converged"],
                         "kkt": st["kkt"], "members_converged": sum(p["converged"] for p in stats),
                         "mean_member_iters": float(np.mean([p["iters"] for p in stats]))})
            if log:
                log(f"  period {k}: {solve_s * 1e3:.1f} ms, {st['iters']} it (slowest member), "
                    f"{recs[-1]['members_converged']}/{len(insts)} converged")
    return {"records": recs, "load_seconds": load_s, "autotune_choice": choice}, path, per_stats


def run_sequential(insts, path, which=None, precision: int = 64, log=None, **params):
    """Plain re-solves of the (period, instance) problems on the recorded
    capacity path, one instance at a time from y = 0. `which` selects
    instance indices (default all). Returns per-solve records."""
    import torch
    idx = list(range(len(insts))) if which is None else list(which)
    out = []
    with Solver(None, device=0, precision=precision, **params) as s:
        for b in idx:
            inst = insts[b]
            s.load(inst)
            for k, (c_k, lam_k) in enumerate(path):
                s.update(c_k[b], lam_k[b])
                torch.cuda.synchronize()
                t = time.perf_counter()
                st = s.solve()
                out.append({"instance": b, "period": k, "seconds": time.perf_counter() - t, "iters": st["iters"],
                            "converged": st["converged"], "dual": st["dual_avg"], "kkt": st["kkt"]})
            if log:
                log(f"  sequential instance {b}: {sum(r['seconds'] for r in out if r['instance'] == b):.3f} s")
    return out
