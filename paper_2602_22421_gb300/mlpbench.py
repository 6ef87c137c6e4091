"""Throughput of the warm-start network's training step (forward, backward and
Adam on the tensor-core kernels of include/spfom_mlp.h) on synthetic rows.

    python -m paper_2602_22421_gb300.mlpbench [--rows 262144] [--steps 20]

Prints one JSON line: milliseconds per step and the BF16 tensor-core rate of
the step's matrix products (2 flops per multiply-add, over the products'
useful shapes: the padding of the 16-wide input and output layers is not
counted).
"""
from __future__ import annotations

import argparse
import json


def flops_per_step(rows: int) -> int:
    f, h = 16, 256
    fwd = rows * (f * h + h * h + h)          # three layers
    bwd = rows * (h + h * h + h * h + h * f + h * f)  # dw3, dH2, dW2, dH1, dW1
    return 2 * (fwd + bwd)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--rows", type=int, default=262144)
    ap.add_argument("--steps", type=int, default=20)
    a = ap.parse_args(argv)
    import numpy as np
    import torch
    from . import build
    build.build()
    from .spfom import MLP
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.standard_normal((a.rows, 16)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.uniform(0, 1, a.rows).astype(np.float32)).cuda()
    net = MLP(0, seed=1)
    for _ in range(4):
        net.train_step(x, t, 1e-3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        net.train_step(x, t, 1e-3)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    net.close()
    print(json.dumps({"rows": a.rows, "ms_per_step": ms, "tflops": flops_per_step(a.rows) / ms / 1e9}))


if __name__ == "__main__":
    main()
