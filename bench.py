#!/usr/bin/env python3
"""SPFOM iteration benchmark on the mid GAM instance (1e4 products, 2000
resources, 1e6 segments with 5-15 products each; seeded synthetic data).

A step is ``--iters-per-step`` SPFOM iterations (default 64 = one KKT
evaluation period), so every step covers margins, segment solves, the sales
aggregate, the dual step, averaging and one KKT / restart evaluation. The JSON
line reports iterations per second of the whole job, the segment kernel's HBM
roofline fraction, the end-to-end rate through host buffers, the time to KKT
<= 1e-4, and the FP64 oracle timed on the host as the CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Under torchrun (N > 1) every rank solves its own seeded instance (replicas;
the iteration has no cross-GPU exchange here), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to-1e-4 KKT (s) & SPFOM iters/s: GPU plain vs FP32/batched/learned"
CSRC = os.path.join(ROOT, "paper_2602_22421_gb300", "csrc")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
BYTES_PER_NNZ = 20      # seg_prod int32 + v f64 + (v - w) f64
BYTES_PER_SEGMENT = 24  # seg_ptr int64 + lambda f64 + (v0 + sum w) f64
BYTES_PER_NNZ_F32 = 12      # seg_prod int32 + v f32 + (v - w) f32
BYTES_PER_SEGMENT_F32 = 16  # seg_ptr int64 + lambda f32 + (v0 + sum w) f32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--iters-per-step", type=int, default=64)
    ap.add_argument("--segments", type=int, default=1_000_000)
    ap.add_argument("--tiling64", type=int, default=0,
                    help="segment-kernel tiling of the precision-64 legs (0: spfom_autotune picks)")
    ap.add_argument("--tiling32", type=int, default=0,
                    help="segment-kernel tiling of the precision-32 legs (0: spfom_autotune picks)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-huge", action="store_true", help="skip the 1e7-segment instance")
    ap.add_argument("--huge-segments", type=int, default=10_000_000)
    ap.add_argument("--huge-steps", type=int, default=6)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched multi-period re-solves")
    ap.add_argument("--batched-count", type=int, default=256)
    ap.add_argument("--periods", type=int, default=16)
    ap.add_argument("--seq-sample", type=int, default=16,
                    help="instances of the batched family re-solved one at a time for the plain reference "
                         "(0 = all)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm start")
    ap.add_argument("--no-paper-shaped", action="store_true",
                    help="skip the instance of the paper's speedup-study shape (sets of all 100 products)")
    ap.add_argument("--learned-test", type=int, default=128)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(args, seed):
    from instances import mid_gam
    return mid_gam(seed, L=args.segments)


def config_of(inst, args, extra=None):
    import numpy as np
    K = np.diff(inst.seg_ptr)
    cfg = {"workload": f"mid GAM instance: n={inst.n} products, m={inst.m} resources (1-3 per product), "
                       f"L={inst.L} segments, |C_l|~U{{{int(K.min())}..{int(K.max())}}}",
           "n": inst.n, "m": inst.m, "L": inst.L, "nnz": inst.nnz,
           "iterations_per_step": args.iters_per_step, "eval_every": 64,
           "input_bytes": inst.nbytes(),
           "l2": f"inputs {inst.nbytes() / 1e9:.2f} GB > L2 (129 MB); L2 not flushed between iterations",
           "parallelism": "replicas" if args.gpus > 1 else "single GPU"}
    if extra:
        cfg.update(extra)
    return cfg


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(index), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def code_digest(path):
    """SHA-256 of a source file's code: line comments and blank lines dropped,
    so that a capture stays valid across comment-only edits."""
    lines = []
    for line in open(path, encoding="utf-8"):
        code = line.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def kernel_of(precision, path, fast_path, tiling):
    """Name and source file of the iterate pass's segment kernel."""
    if precision == 32:
        return ("k_seg_rows32", "spfom_segments_rows.cu") if tiling == 9 else ("k_seg_f32", "spfom_segments_fast.cu")
    if not fast_path:
        return "k_segments", "spfom_kernels.cu"
    if path == 2:
        return "k_seg_dd", "spfom_segments_dd.cu"
    return ("k_seg_rows", "spfom_segments_rows.cu") if tiling == 4 else ("k_seg_fast", "spfom_segments_fast.cu")


def kernel_traffic(kernel, tiling, src, nnz):
    """DRAM bytes per launch of `kernel` in `tiling` from the committed ncu
    summary, if it was taken on the current kernel source; scaled by nonzeros."""
    if not os.path.exists(TRAFFIC):
        return None, None
    with open(TRAFFIC) as f:
        d = json.load(f).get(f"{kernel}/tiling{tiling}")
    if not d:
        return None, None
    if d.get("kernel_code_sha256") != code_digest(os.path.join(CSRC, src)):
        return None, "kernel changed since the ncu capture"
    return d["dram_bytes_per_launch"] * nnz / d["nnz"], d.get("capture")


def host_cpu() -> str:
    """CPU model and core count of this host (lscpu, else /proc/cpuinfo)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    import platform
    return f"{model or platform.machine()}, {os.cpu_count()} cores"


def cpu_baseline(inst, seconds):
    """The FP64 oracle as it stands, single thread, full iterations of the
    same instance for about `seconds` (at least 2 iterations); and its
    OpenMP timing build (segments over all host cores) for a third of that."""
    from oracle import Oracle, Params

    def rate(omp, secs):
        run = Oracle(inst, omp=omp).run(Params(kkt_tol=0.0))
        run.step(1)
        t0, it = time.perf_counter(), 0
        while True:
            run.step(1)
            it += 1
            el = time.perf_counter() - t0
            if (el >= secs and it >= 2) or el >= 3 * secs:
                return it, el

    it, el = rate(False, seconds)
    out = {"value": it / el, "unit": "iters/s", "cores": 1, "kind": "oracle",
           "sample": f"{it} full iterations of the {inst.L}-segment instance ({el:.1f} s, single thread)",
           "host": host_cpu()}
    try:
        it2, el2 = rate(True, seconds / 3)
        out["all_cores"] = {"value": it2 / el2, "unit": "iters/s", "cores": os.cpu_count(),
                            "kind": "oracle, OpenMP timing build (segments over all cores)",
                            "sample": f"{it2} full iterations ({el2:.1f} s)"}
    except Exception as e:  # the timing build needs gcc's OpenMP; the single-thread number stands alone
        out["all_cores"] = {"unavailable": str(e)[:200]}
    return out


def pinned_arrays(inst):
    """Host copies of the instance in page-locked memory (the e2e inputs)."""
    import numpy as np
    import torch
    from paper_2602_22421_gb300 import InstanceArrays
    arrs = InstanceArrays(inst)
    keep = {}
    for k, a in arrs.keep.items():
        if a is None:
            keep[k] = None
            continue
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        keep[k] = t
    class _I:  # noqa: N801
        pass
    fake = _I()
    for k, t in keep.items():
        setattr(fake, k, None if t is None else t.numpy())
    fake.n, fake.m, fake.L = inst.n, inst.m, inst.L
    pinned = InstanceArrays(fake)
    pinned.torch_keep = keep
    return pinned


def run_gpu(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_2602_22421_gb300 import Solver

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def allmax(x):
        if not dist:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    inst = workload(args, seed=1 + rank)
    ips = args.iters_per_step
    stream = torch.cuda.Stream()  # a real stream handle: the ctx runs on it, the events bracket it

    def measure(precision, with_clocks, path=0, solve=True):
        """Timed iterations (kkt_tol = 0: nothing is skipped), then a profiled
        pass for the segment kernel's roofline, then a solve to KKT <= 1e-4."""
        forced = (args.tiling64 if precision == 64 else args.tiling32) if path == 0 else 0
        s = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=0.0, precision=precision, path=path,
                   tiling=forced)
        tiling = forced or (s.autotune(ips) if path != 1 else 0)  # segment-kernel tiling for this instance
        s.step(args.warmup * ips)
        barrier()
        clk = Clocks(local) if (rank == 0 and with_clocks) else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        st = s.step(args.steps * ips)
        e1.record(stream)
        barrier()
        clocks = clk.stop() if clk else None
        ms = allmax(e0.elapsed_time(e1))
        s.close()
        out = {"value": ws * args.steps * ips / (ms * 1e-3), "ms": ms, "launches": st["kernel_launches"],
               "clocks": clocks, "iter_precision": st["iter_precision"], "tiling": tiling}
        if rank == 0:
            sp = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=0.0, profile=1, precision=precision,
                        path=path, tiling=tiling)
            sp.step(2 * ips)
            pst = sp.step(min(args.steps, 10) * ips)
            sp.close()
            per_launch = pst["seg_kernel_seconds"] / max(1, pst["seg_kernel_launches"])
            if precision == 32:
                alg = BYTES_PER_NNZ_F32 * inst.nnz + BYTES_PER_SEGMENT_F32 * inst.L
            else:
                alg = BYTES_PER_NNZ * inst.nnz + BYTES_PER_SEGMENT * inst.L
            kname, ksrc = kernel_of(precision, path, pst["fast_path"], tiling)
            peak, src = measured_peaks()
            achieved = alg / per_launch / 1e9
            traffic, cap = kernel_traffic(kname, tiling, ksrc, inst.nnz)
            solves = (2 + min(args.steps, 10)) * ips * inst.L
            out["roofline"] = {"bound": "hbm", "kernel": kname + " (iterate)", "achieved": achieved, "peak": peak,
                               "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                               "algorithmic_bytes_per_launch": alg, "launch_ms": per_launch * 1e3,
                               "peak_source": f"{src} hbm_gbs", "traffic_note": cap,
                               "binary64_redo_fraction": pst["fallback_segments"] / solves}
        if solve and not args.no_solve:
            sv = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=1e-4, max_iters=20000,
                        precision=precision, path=path, tiling=tiling)
            barrier()
            w0 = time.perf_counter()
            sst = sv.solve()
            wall = time.perf_counter() - w0
            out["ttk"] = {"seconds_device": sst["seconds"], "seconds_wall": wall, "iterations": sst["iters"],
                          "converged": bool(sst["converged"]), "kkt": sst["kkt"], "dual_obj": sst["dual_avg"],
                          "primal_obj": sst["primal_avg"], "restarts": sst["restarts"],
                          "final_iter_precision": sst["iter_precision"]}
            sv.close()
        return out

    m64 = measure(64, True)
    m32 = measure(32, False)
    m64b = measure(64, False, path=2, solve=False)  # double-float values (k_seg_dd), autotuned tiling
    value, ms, launches, clocks = m64["value"], m64["ms"], m64["launches"], m64["clocks"]
    roof = m64.get("roofline")
    ttk = m64.get("ttk")
    fp32 = {"value": m32["value"], "unit": "iters/s", "ms_per_step": m32["ms"] / args.steps, "tiling": m32["tiling"],
            "roofline": m32.get("roofline"), "time_to_kkt_1e-4": m32.get("ttk"), "gpu_launches": m32["launches"],
            "dtype": "f32 segment solves, f64 dual step / residuals / evaluations"}
    f64_dd = {"value": m64b["value"], "unit": "iters/s", "ms_per_step": m64b["ms"] / args.steps,
              "roofline": m64b.get("roofline"), "gpu_launches": m64b["launches"], "tiling": m64b["tiling"],
              "dtype": "f64 inputs/outputs: certified decisions, values in double-binary32 arithmetic (path 2)"}
    if ttk and m32.get("ttk"):
        fp32["objective_rel_diff_vs_f64"] = abs(m32["ttk"]["dual_obj"] / ttk["dual_obj"] - 1)
        fp32["speedup_time_to_kkt_vs_f64"] = ttk["seconds_device"] / m32["ttk"]["seconds_device"]
    # --- end to end through host buffers -------------------------------------
    e2e = None
    if not args.no_e2e:
        pinned = pinned_arrays(inst)
        # the measured tiling (each load builds its copy anew: the row-exact copy on the
        # device), except the slot-major copy, whose host sort of the segments by size costs
        # more than it saves per step: then the shared-margin tiling
        e2e_tiling = 2 if m64["tiling"] == 3 else m64["tiling"]
        se = Solver(None, stream=stream.cuda_stream, device=local, kkt_tol=0.0, tiling=e2e_tiling)
        ysink = np.empty(inst.m)
        se.load(pinned)
        se.step(ips)
        se.duals()
        barrier()
        k = max(3, min(args.steps, 20))
        w0 = time.perf_counter()
        for _ in range(k):
            se.load(pinned)              # host -> device copy of the instance, validation
            se.step(ips)
            ysink[:] = se.duals()        # device -> host read of the result
        barrier()
        wall = allmax(time.perf_counter() - w0)
        se.close()
        e2e = {"value": ws * k * ips / wall, "unit": "iters/s", "steps": k, "tiling": e2e_tiling,
               "h2d_bytes_per_step": pinned.nbytes(), "d2h_bytes_per_step": inst.m * 8 + 160}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(inst, args.cpu_seconds)
    legs = {}
    if rank == 0:
        for name, skip, fn in (("paper_shaped", args.no_paper_shaped, lambda: paper_shaped_leg(args, stream, local)),
                               ("huge", args.no_huge, lambda: huge_leg(args, stream, local)),
                               ("batched", args.no_batched, lambda: batched_leg(args, local)),
                               ("learned", args.no_learned, lambda: learned_leg(args, local))):
            if skip:
                continue
            t0 = time.perf_counter()
            legs[name] = fn()
            legs[name]["leg_seconds"] = time.perf_counter() - t0
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "dtype_note": "binary64 throughout; segment decisions taken in binary32 and certified exact "
                             "(binary64 redo otherwise)",
               "data": "synthetic (seeded generator)",
               "config": config_of(inst, args), "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
               "roofline": roof, "cpu_baseline": cpu, "time_to_kkt_1e-4": ttk, "fp32_bulk": fp32,
               "f64_double_float_values": f64_dd, "tiling": m64["tiling"]}
        out.update(legs)
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def roofline_of(s_prof, inst, precision, ips, steps, tiling=0):
    """Segment-kernel roofline of a profiled solver (the per-launch time of the
    iterate pass from its CUDA event pairs)."""
    pst = s_prof.step(steps * ips)
    per_launch = pst["seg_kernel_seconds"] / max(1, pst["seg_kernel_launches"])
    if precision == 32:
        alg = BYTES_PER_NNZ_F32 * inst.nnz + BYTES_PER_SEGMENT_F32 * inst.L
    else:
        alg = BYTES_PER_NNZ * inst.nnz + BYTES_PER_SEGMENT * inst.L
    kname = kernel_of(precision, 0, pst["fast_path"], tiling)[0]
    peak, src = measured_peaks()
    achieved = alg / per_launch / 1e9
    return {"bound": "hbm", "kernel": kname + " (iterate)", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "algorithmic_bytes_per_launch": alg, "launch_ms": per_launch * 1e3,
            "peak_source": f"{src} hbm_gbs", "traffic": None,
            "binary64_redo_fraction": pst["fallback_segments"] / (steps * ips * inst.L)}


def paper_shaped_leg(args, stream, local):
    """The shape of the paper's speedup study (Section 4.5): n = m = 100, one
    resource per product, every segment considers all 100 products, MNL,
    c, r, v ~ U(0,1), lambda = 1, here with 1e5 segments (1e7 nonzeros):
    iterations/s and the segment kernel's roofline in both precisions."""
    import torch
    from instances import paper_shaped
    from paper_2602_22421_gb300 import Solver
    inst = paper_shaped(3, L=100_000, n=100)
    out = {"workload": f"paper-shaped: n=m={inst.n}, A=I, L={inst.L}, |C_l|={inst.n} (all products), MNL, "
                       "c, r, v ~ U(0,1), lambda = 1", "nnz": inst.nnz}
    ips = args.iters_per_step
    for precision in (64, 32):
        s = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=0.0, precision=precision)
        tiling = s.autotune(16)
        s.step(2 * ips)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(4 * ips)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s.close()
        sp = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=0.0, profile=1, precision=precision,
                    tiling=tiling)
        sp.step(ips)
        roof = roofline_of(sp, inst, precision, ips, 2, tiling)
        sp.close()
        out[f"f{precision}"] = {"value": 4 * ips / (ms * 1e-3), "unit": "iters/s", "tiling": tiling,
                                "ms_per_iter": ms / (4 * ips), "roofline": roof}
    return out


def huge_leg(args, stream, local):
    """The 1e7-segment GAM instance (|C_l| ~ U{10..30}, ~2e8 nonzeros, c = 0.4 x
    demand): iterations/s and the segment kernel's roofline in binary64 and in
    the binary32 bulk mode, and the binary32 solve to KKT <= 1e-4 (with its
    binary64 residuals and polish)."""
    import torch
    from instances import huge_gam
    from paper_2602_22421_gb300 import Solver
    t0 = time.perf_counter()
    inst = huge_gam(2, L=args.huge_segments, workers=12)
    gen_s = time.perf_counter() - t0
    out = {"workload": f"huge GAM instance: n={inst.n}, m={inst.m}, L={inst.L}, nnz={inst.nnz}, "
                       "|C_l|~U{10..30}, c = 0.4 x demand", "nnz": inst.nnz, "generate_seconds": gen_s}
    ips = args.iters_per_step
    for precision in (64, 32):
        t0 = time.perf_counter()
        forced = args.tiling64 if precision == 64 else args.tiling32
        s = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=0.0, precision=precision, tiling=forced)
        load_s = time.perf_counter() - t0
        tiling = forced or s.autotune(16)
        s.step(2 * ips)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(args.huge_steps * ips)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s.close()
        sp = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=0.0, profile=1, precision=precision,
                    tiling=tiling)
        sp.step(ips)
        roof = roofline_of(sp, inst, precision, ips, 2, tiling)
        sp.close()
        out[f"f{precision}"] = {"value": args.huge_steps * ips / (ms * 1e-3), "unit": "iters/s", "tiling": tiling,
                                "ms_per_iter": ms / (args.huge_steps * ips), "load_seconds": load_s,
                                "roofline": roof}
    sv = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=1e-4, max_iters=20000, precision=32,
                tiling=out["f32"]["tiling"])
    w0 = time.perf_counter()
    st = sv.solve()
    out["f32"]["time_to_kkt_1e-4"] = {"seconds_wall": time.perf_counter() - w0, "seconds_device": st["seconds"],
                                      "iterations": st["iters"], "converged": bool(st["converged"]),
                                      "kkt": st["kkt"], "dual_obj": st["dual_avg"],
                                      "final_iter_precision": st["iter_precision"]}
    sv.close()
    # the plain binary64 solve to 1e-4, measured the same way
    sd = Solver(inst, stream=stream.cuda_stream, device=local, kkt_tol=1e-4, max_iters=20000, precision=64,
                tiling=out["f64"]["tiling"])
    w0 = time.perf_counter()
    sd_st = sd.solve()
    out["f64"]["time_to_kkt_1e-4"] = {"seconds_wall": time.perf_counter() - w0, "seconds_device": sd_st["seconds"],
                                      "iterations": sd_st["iters"], "converged": bool(sd_st["converged"]),
                                      "kkt": sd_st["kkt"], "dual_obj": sd_st["dual_avg"]}
    sd.close()
    out["f32"]["time_to_kkt_1e-4"]["speedup_vs_f64"] = sd_st["seconds"] / st["seconds"] if st["seconds"] > 0 else None
    out["f32"]["time_to_kkt_1e-4"]["objective_rel_diff_vs_f64"] = abs(st["dual_avg"] / sd_st["dual_avg"] - 1.0)
    # the oracle on one host core: two full iterations, and its time to 1e-4 extrapolated with the
    # GPU solve's iteration count (same iterates)
    if not args.no_cpu_baseline:
        from oracle import Oracle, Params
        run = Oracle(inst).run(Params(kkt_tol=0.0))
        t0 = time.perf_counter()
        run.step(2)
        per = (time.perf_counter() - t0) / 2
        out["cpu_baseline"] = {"seconds_per_iteration": per, "cores": 1, "kind": "oracle",
                               "sample": "2 full iterations of the 1e7-segment instance, single thread",
                               "time_to_kkt_1e-4_extrapolated_s": per * st["iters"]}
    return out


def batched_leg(args, local):
    """Batched multi-period re-solves (count base instances of uneven size, 16
    periods each): all instances of a period in one batch, binary32 bulk,
    autotuned segment kernel, graph-replayed evaluation periods, warm-started
    from the previous period's bid prices -- against the plain binary64 method
    re-solving the same problems one at a time from y = 0 (on a seeded sample
    of the instances when seq-sample > 0, scaled to all of them)."""
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import get_context

    import numpy as np
    from instances import batch_base, period_rates
    from paper_2602_22421_gb300 import periods as PR
    count = args.batched_count
    t0 = time.perf_counter()
    with ProcessPoolExecutor(12, mp_context=get_context("spawn")) as pool:
        insts = list(pool.map(batch_base, [4] * count, range(count)))
    gen_s = time.perf_counter() - t0
    rho = period_rates(4, count, args.periods)
    prm = dict(restart_tau_balance=0.5, restart_tau_decay=0.9, max_iters=40000)
    summary, path, per = PR.run_batched(insts, rho, periods=args.periods, precision=32, **prm)
    batched_s = sum(r["seconds"] for r in summary["records"])
    # the same periods with each solve phase as one launch (device-side loop over evaluation periods)
    loop_summary, _, loop_per = PR.run_batched(insts, rho, periods=args.periods, precision=32, device_loop=1, **prm)
    loop_s = sum(r["seconds"] for r in loop_summary["records"])
    loop_same = all(a["iters"] == b["iters"] and a["converged"] == b["converged"]
                    for pa, pb in zip(per, loop_per) for a, b in zip(pa, pb))
    if args.seq_sample and args.seq_sample < count:
        which = sorted(np.random.default_rng(7).choice(count, args.seq_sample, replace=False).tolist())
    else:
        which = list(range(count))
    seq = PR.run_sequential(insts, path, which=which, precision=64, **prm)
    seq_s = sum(r["seconds"] for r in seq)
    nnz_all = sum(i.nnz for i in insts)
    nnz_sample = sum(insts[b].nnz for b in which)
    scale = len(insts) / len(which)
    rel = [abs(per[r["period"]][r["instance"]]["dual_avg"] / r["dual"] - 1) for r in seq]
    return {"workload": f"{count} GAM instances, n~U{{200..5000}}, m=ceil(n/5), L=10^U(3,5), |C_l|~U{{3..20}}, "
                        f"{args.periods} periods (capacity = remaining inventory / remaining periods, "
                        f"lambda x U(0.5,1.5))",
            "solver_params": prm,
            "instances": count, "periods": args.periods, "nnz_total": nnz_all, "generate_seconds": gen_s,
            "batched_seconds": batched_s, "batched_load_seconds": summary["load_seconds"],
            "device_loop": {"batched_seconds": loop_s, "periods_converged":
                            sum(r["converged"] for r in loop_summary["records"]),
                            "same_members_iterations_as_period_by_period": loop_same,
                            "note": "each solve phase one graph launch: a conditional WHILE node replays the "
                                    "evaluation period until the device-side test ends the phase"},
            "autotune_choice": summary["autotune_choice"],
            "periods_converged": sum(r["converged"] for r in summary["records"]),
            "batched_iterations_per_period": [r["iters"] for r in summary["records"]],
            "sequential_plain_seconds": seq_s * scale, "sequential_sample": len(which),
            "sequential_scale": scale, "sequential_sample_nnz_share": nnz_sample / nnz_all,
            "speedup_vs_sequential_plain": seq_s * scale / batched_s,
            "max_objective_rel_diff_vs_plain": max(rel),
            "sequential_all_converged": all(r["converged"] for r in seq)}


def learned_leg(args, local):
    """Learned warm start: the committed network, on held-out instances of its
    training family (n=2000, m=400, L=10^U(4,4.7), |C_l|~U{10..30}, c=0.4 x
    demand): cold and warm solves to KKT <= 1e-4 per instance, wall clock."""
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import get_context

    from paper_2602_22421_gb300 import warmstart as W
    if not os.path.exists(W.DEFAULT_WEIGHTS):
        return {"unavailable": f"no trained network at {os.path.relpath(W.DEFAULT_WEIGHTS, ROOT)}"}
    with ProcessPoolExecutor(8, mp_context=get_context("spawn")) as pool:
        test = W.instances(W.TEST_SEED, range(args.learned_test), pool=pool)
    net = W.load()
    recs = W.evaluate(net, test)
    net.close()
    out = W.summarize(recs)
    # the training step of the network on the tensor cores (BF16 tcgen05 products)
    from paper_2602_22421_gb300 import mlpbench
    import contextlib
    import io
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        mlpbench.main(["--rows", "262144", "--steps", "20"])
    tr = json.loads(buf.getvalue().strip().splitlines()[-1])
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peak = float(json.load(f)["bf16_tflops"])
    out["training_step"] = {"rows": tr["rows"], "ms": tr["ms_per_step"],
                            "roofline": {"bound": "tensor", "achieved": tr["tflops"], "peak": peak or 1900.0,
                                         "unit": "TFLOP/s", "frac": tr["tflops"] / (peak or 1900.0),
                                         "peak_source": "measured bf16_tflops" if peak else "fallback"}}
    out["workload"] = ("held-out warm_family(seed 6) instances: n=2000, m=400, L=10^U(4,4.7), |C_l|~U{10..30}, "
                       "c=0.4 x demand")
    return out


def sub_instance(inst, Ls):
    """The first Ls segments of inst, capacities scaled by their share of the
    arrival mass (a bounded sample of the same workload)."""
    from instances import Instance
    e = int(inst.seg_ptr[Ls])
    frac = float(inst.lam[:Ls].sum() / inst.lam.sum())
    return Instance(n=inst.n, m=inst.m, L=Ls, r=inst.r, c=inst.c * frac, a_ptr=inst.a_ptr, a_idx=inst.a_idx,
                    a_val=inst.a_val, seg_ptr=inst.seg_ptr[:Ls + 1].copy(), seg_prod=inst.seg_prod[:e],
                    v=inst.v[:e], w=None if inst.w is None else inst.w[:e], lam=inst.lam[:Ls], v0=inst.v0[:Ls],
                    name=inst.name + f"[:{Ls}]")


def run_reference(args):
    """The FP64 oracle as it stands on the host cores: each step runs
    iters-per-step oracle iterations on the first 1e4 segments of the same
    instance; the rate is scaled to full-instance iterations by nonzeros."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import Oracle, Params
    inst = workload(args, seed=1)
    Ls = min(inst.L, 10_000)
    sub = sub_instance(inst, Ls)
    run = Oracle(sub).run(Params(kkt_tol=0.0))
    ips = args.iters_per_step
    for _ in range(args.warmup):
        run.step(ips)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run.step(ips)
    el = time.perf_counter() - t0
    scale = sub.nnz / inst.nnz
    value = args.steps * ips / el * scale
    sample = (f"{ips} oracle iterations per step on the first {Ls} of {inst.L} segments ({sub.nnz} of {inst.nnz} "
              f"nonzeros); rate scaled by the nonzero share to full-instance iterations")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded generator)", "config": config_of(inst, args),
           "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
