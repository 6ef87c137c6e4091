"""Segment-sharded iteration on CPU ranks (gloo, world size 2).

The iteration shards by segments: each rank solves the inner problems of a
contiguous, nonzero-balanced range of segments, one all-reduce of the
m-vector g (and of the scalars sum z, P) gives every rank the full aggregate,
and each rank then applies the identical dual step (Algorithm 3's workers and
aggregation, with the workers on different devices). This test runs that
pattern with the oracle as the per-rank solver and checks it against the
single-rank oracle. The benchmark itself runs replicas: each run here uses one
GPU.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from instances import Instance, mid_gam, seeded_duals  # noqa: E402


def shard_bounds(seg_ptr, world):
    """Segment boundaries giving each rank about nnz / world nonzeros."""
    nnz = int(seg_ptr[-1])
    cuts = [0]
    for r in range(1, world):
        cuts.append(int(np.searchsorted(seg_ptr, r * nnz / world)))
    cuts.append(len(seg_ptr) - 1)
    return cuts


def segment_slice(inst, a, b):
    p0, p1 = int(inst.seg_ptr[a]), int(inst.seg_ptr[b])
    return Instance(n=inst.n, m=inst.m, L=b - a, r=inst.r, c=inst.c, a_ptr=inst.a_ptr, a_idx=inst.a_idx,
                    a_val=inst.a_val, seg_ptr=inst.seg_ptr[a:b + 1] - p0, seg_prod=inst.seg_prod[p0:p1],
                    v=inst.v[p0:p1], w=None if inst.w is None else inst.w[p0:p1], lam=inst.lam[a:b],
                    v0=inst.v0[a:b], name=f"{inst.name}[{a}:{b}]")


def _instance():
    return mid_gam(1, L=3001, n=300, m=60)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import Oracle
    inst = _instance()
    cuts = shard_bounds(inst.seg_ptr, world)
    part = Oracle(segment_slice(inst, cuts[rank], cuts[rank + 1]))
    y = np.zeros(inst.m)
    tau = Oracle(inst).default_tau(0.1)
    ys = []
    for t in range(5):  # five full-batch iterations, mu = 0
        sw = part.sweep(y)
        g = torch.from_numpy(sw["g"].copy())
        zs = torch.tensor([sw["zsum"], sw["P"]], dtype=torch.float64)
        dist.all_reduce(g)
        dist.all_reduce(zs)
        y = np.maximum(0.0, y - tau * (inst.c - g.numpy()))
        ys.append(y.copy())
    gathered = [torch.zeros(inst.m, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(y))
    if rank == 0:
        out.put((np.array(ys), [x.numpy() for x in gathered], zs.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_aggregate_matches_single_rank():
    from oracle import Oracle, Params
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    ys, finals, zs = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    inst = _instance()
    run = Oracle(inst).run(Params(eval_every=0))
    for t in range(5):
        run.step(1)
        np.testing.assert_allclose(ys[t], run.y, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(finals[0], finals[1])  # every rank holds the same duals
    st = run.stats()
    assert zs[1] == pytest.approx(st["P"], rel=1e-12)
    assert zs[0] == pytest.approx(st["z_sum"], rel=1e-12)


def test_shard_bounds_balance_nonzeros():
    inst = _instance()
    cuts = shard_bounds(inst.seg_ptr, 4)
    assert cuts[0] == 0 and cuts[-1] == inst.L and cuts == sorted(cuts)
    per = np.diff(inst.seg_ptr[cuts])
    assert per.max() - per.min() <= 2 * int(np.diff(inst.seg_ptr).max())
    y = seeded_duals(inst.m, 3, 5.0)
    from oracle import Oracle
    whole = Oracle(inst).sweep(y)
    parts = [Oracle(segment_slice(inst, cuts[r], cuts[r + 1])).sweep(y) for r in range(4)]
    np.testing.assert_allclose(sum(p["g"] for p in parts), whole["g"], rtol=1e-12, atol=1e-12)
