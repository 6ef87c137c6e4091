"""Batched re-solves (spfom_load_batch) against per-instance oracle runs, and
the multi-period update (needs a GPU).

A batch is the block-diagonal union of its instances with per-instance step
size, averages, KKT, restarts and convergence, so every instance of a batch
must follow exactly the iterates of its own single-instance run.
"""
import numpy as np
import pytest

from instances import make_instance, mid_gam, seeded_duals, tiny_mnl
from oracle import Oracle
from oracle import Params as OracleParams

pytestmark = pytest.mark.gpu
ITER_RTOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def Solver(**kw):
    from paper_2602_22421_gb300 import Solver as S
    return S(None, device=0, **kw)


def nrel(a, b):
    scale = float(np.abs(b).max()) if np.size(b) else 0.0
    return float(np.abs(np.asarray(a) - np.asarray(b)).max()) / (scale if scale > 0 else 1.0) if np.size(b) else 0.0


def members():
    return [tiny_mnl(0), make_instance(n=30, m=8, L=600, kmin=3, kmax=8, gam=True, tightness=0.6, seed=5),
            mid_gam(1, L=5000, n=300, m=60), mid_gam(7, L=2500, n=150, m=40, kmin=3, kmax=12)]


def slices(insts):
    out, i0 = [], 0
    for inst in insts:
        out.append(slice(i0, i0 + inst.m))
        i0 += inst.m
    return out


def test_batch_members_track_their_own_oracle_runs():
    insts = members()
    runs = [Oracle(i).run(OracleParams()) for i in insts]
    with Solver() as s:
        s.load_batch(insts)
        done = 0
        for t in (1, 5, 64, 65, 128, 200):
            s.step(t - done)
            done = t
            y = s.duals()
            per = s.batch_stats()
            for k, (inst, run, sl) in enumerate(zip(insts, runs, slices(insts))):
                run.step(t - run.stats()["t"])
                ost = run.stats()
                assert per[k]["iters"] == ost["t"] == t
                assert per[k]["restarts"] == ost["restarts"] and per[k]["evals"] == ost["evals"]
                assert nrel(y[sl], run.y) <= ITER_RTOL, (k, t)
                assert per[k]["dual_iter"] == pytest.approx(ost["dual_iter"], rel=ITER_RTOL)
                if ost["evals"]:
                    assert per[k]["kkt"] == pytest.approx(ost["kkt"], rel=1e-5)
                    assert per[k]["dual_avg"] == pytest.approx(ost["dual_avg"], rel=ITER_RTOL)


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_solve_converges_every_member(precision):
    insts = members()[1:]  # the 40-segment instance needs a decaying step (see the oracle pins)
    refs = []
    for inst in insts:
        run = Oracle(inst).run(OracleParams())
        for _ in range(300):
            ost = run.step(64)
            if ost["converged"]:
                break
        assert ost["converged"]
        refs.append(ost)
    with Solver(precision=precision) as s:
        s.load_batch(insts)
        st = s.solve()
        per = s.batch_stats()
    assert st["converged"] == 1 and st["kkt"] <= 1e-4
    for k, ref in enumerate(refs):
        assert per[k]["converged"] == 1 and per[k]["kkt"] <= 1e-4
        assert per[k]["dual_avg"] == pytest.approx(ref["dual_avg"], rel=1e-6 if precision == 64 else 1e-4)
        if precision == 64:
            assert per[k]["iters"] == ref["t"]


def test_sales_at_matches_oracle_sweep():
    inst = mid_gam(1, L=20_000, n=1000, m=200)
    y = seeded_duals(inst.m, 3, float(np.mean(inst.r)) / 4)
    from paper_2602_22421_gb300 import Solver as S
    with S(inst, device=0) as s:
        got = s.sales_at(y)
        assert s.stats()["iters"] == 0
    np.testing.assert_allclose(got, Oracle(inst).sweep(y)["s"], rtol=1e-12, atol=1e-12 * got.max())


def test_multi_period_update_with_warm_start():
    """Period 2 of a two-instance batch: capacities lowered by period 1's
    expected sales under its bid prices, arrival rates rescaled, duals kept."""
    insts = members()[2:]
    with Solver() as s:
        s.load_batch(insts)
        s.step(256)
        y1 = s.duals()
        sales = s.sales_at(y1)
        c_new, lam_new = [], []
        rng = np.random.default_rng(11)
        for inst, j0 in zip(insts, np.cumsum([0] + [i.n for i in insts])[:-1]):
            A = np.zeros((inst.m, inst.n))
            for j in range(inst.n):
                A[inst.a_idx[inst.a_ptr[j]:inst.a_ptr[j + 1]], j] = 1.0
            used = A @ sales[j0:j0 + inst.n]
            c_new.append(np.maximum(0.0, 2.0 * inst.c - used))
            lam_new.append(inst.lam * rng.uniform(0.5, 1.5))
        s.update(np.concatenate(c_new), np.concatenate(lam_new))
        s.reset(y1)
        s.step(130)
        y2 = s.duals()
        per = s.batch_stats()
    for k, (inst, sl) in enumerate(zip(insts, slices(insts))):
        upd = inst.with_capacity(c_new[k])
        upd.lam = lam_new[k]
        run = Oracle(upd).run(OracleParams(), y0=y1[sl])
        ost = run.step(130)
        assert nrel(y2[sl], run.y) <= ITER_RTOL
        assert per[k]["restarts"] == ost["restarts"] and per[k]["tau"] == ost["tau_used"]


@pytest.mark.parametrize("batch", [False, True])
def test_autotune_keeps_the_duals_and_the_solution(batch):
    """spfom_autotune times the segment kernels' tilings, keeps the faster one
    and restarts from the duals it was given; the solve that follows reaches the
    same objective as the untuned one."""
    insts = members()[2:] if batch else [mid_gam(3, L=30_000, n=800, m=160)]

    def loaded(s):
        s.load_batch(insts) if batch else s.load(insts[0])

    with Solver(precision=32) as s:
        loaded(s)
        ref = s.solve()
    with Solver(precision=32) as s:
        loaded(s)
        s.step(70)
        y = s.duals()
        choice = s.autotune(16)
        assert 1 <= choice <= 9 and not (batch and choice in (2, 4, 8, 9))
        assert s.stats()["iters"] == 0
        np.testing.assert_array_equal(s.duals(), y)
        st = s.solve()
    assert st["converged"] == 1 and st["kkt"] <= 1e-4
    assert st["dual_avg"] == pytest.approx(ref["dual_avg"], rel=1e-4)
    with Solver(precision=64) as s:
        loaded(s)
        s.step(70)
        y = s.duals()
        assert s.autotune(4) in ((1, 2, 3) if batch else (1, 2, 3, 4))
        np.testing.assert_array_equal(s.duals(), y)
        st = s.solve()
    assert st["converged"] == 1
    assert st["dual_avg"] == pytest.approx(ref["dual_avg"], rel=2e-4)


def test_instance_chunked_batch_kernel_equals_plain_loads():
    """Tiling 6 (chunks of one instance's segments with shared-memory sums of
    that instance's products) computes what tiling 3 computes on a batch wide
    enough for global sums: the fixed-point sales make duals and sales equal
    bit for bit."""
    from instances import batch_base
    insts = [batch_base(12, k) for k in range(14)]
    out = {}
    for tiling in (3, 6):
        with Solver(precision=32, tiling=tiling) as s:
            s.load_batch(insts)
            st = s.step(130)
            out[tiling] = (s.duals(), s.vector(5), st, s.batch_stats())
    np.testing.assert_array_equal(out[3][0], out[6][0])
    np.testing.assert_array_equal(out[3][1], out[6][1])
    assert [p["restarts"] for p in out[3][3]] == [p["restarts"] for p in out[6][3]]


@pytest.mark.parametrize("precision", [64, 32])
def test_device_loop_equals_period_by_period_solve(precision):
    """params.device_loop: each phase of the solve is one graph launch whose
    conditional node replays the evaluation period until the device-side test
    ends it. The kernels and their order are those of the period-by-period
    solve, so a batch (binary32 phase, switch to binary64, confirmation) and a
    single instance reach the same iterations, restarts and duals bit for bit;
    a cap that is not a multiple of the evaluation period finishes on the host."""
    from paper_2602_22421_gb300 import Solver
    from instances import batch_base
    insts = [batch_base(4, k) for k in (0, 2, 5, 100)]
    out = {}
    for loop in (0, 1):
        with Solver(None, device=0, precision=precision, device_loop=loop, restart_tau_balance=0.5) as s:
            s.load_batch(insts)
            st = s.solve()
            out[loop] = (st, s.batch_stats(), s.duals(averaged=True))
    assert out[0][0]["converged"] == out[1][0]["converged"] == 1
    assert out[0][0]["iters"] == out[1][0]["iters"]
    for a, b in zip(out[0][1], out[1][1]):
        assert (a["iters"], a["restarts"], a["converged"]) == (b["iters"], b["restarts"], b["converged"])
    np.testing.assert_array_equal(out[0][2], out[1][2])
    inst = mid_gam(1, L=20_000, n=1000, m=200)
    res = {}
    for loop in (0, 1):
        with Solver(inst, device=0, precision=precision, device_loop=loop, max_iters=1000) as s:
            try:
                st = s.solve()
            except Exception:
                st = s.stats()
            res[loop] = (st["iters"], st["restarts"], st["converged"], s.duals())
    assert res[0][:3] == res[1][:3]
    np.testing.assert_array_equal(res[0][3], res[1][3])
