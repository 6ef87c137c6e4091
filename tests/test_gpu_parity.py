"""CUDA path against the FP64 oracle, through the C ABI (needs a GPU).

Tolerance: the FP64 iterates must track the oracle to 1e-6 relative for the
first 200 iterations (norm-relative: max_i |a_i - b_i| / max_i |b_i|). Both
sides compute in binary64; they differ only in summation order (the GPU adds
sales with atomics and scans prefixes as a tree), which moves results by a few
ulps per iteration, so the bar has ample room while still catching any
algorithmic difference (a wrong prefix, a dropped term, a missed restart).
Per-segment values at a fixed dual point are compared at 1e-12.
"""
import numpy as np
import pytest

from instances import make_instance, mid_gam, seeded_duals, tiny_mnl
from oracle import Oracle
from oracle import Params as OracleParams

pytestmark = pytest.mark.gpu

ITER_RTOL = 1e-6
VALUE_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def Solver(inst, **kw):
    from paper_2602_22421_gb300 import Solver as S
    return S(inst, device=0, **kw)


def nrel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    if a.size == 0:
        return 0.0
    scale = float(np.abs(b).max())
    return float(np.abs(a - b).max()) / (scale if scale > 0 else 1.0)


def small_gam():
    return make_instance(n=30, m=8, L=600, kmin=3, kmax=8, gam=True, tightness=0.6, seed=5, name="small_gam")


def edge_instance():
    """Empty and 32-product consideration sets, zero arrival rates, items with
    w = v, a segment count that leaves a ragged last tile."""
    inst = make_instance(n=50, m=10, L=3001, kmin=0, kmax=32, gam=True, tightness=0.5, seed=11, name="edge")
    rng = np.random.default_rng(12)
    inst.lam[rng.uniform(size=inst.L) < 0.05] = 0.0
    pick = rng.uniform(size=inst.nnz) < 0.05
    inst.w[pick] = inst.v[pick]
    return inst


def mid_small():
    return mid_gam(1, L=40_001, n=2000, m=400)


def wide():
    """More products than a block's shared memory holds as sums (global atomics)."""
    return mid_gam(1, L=20_001, n=30_000, m=500)


CASES = {"tiny_mnl": lambda: tiny_mnl(0), "small_gam": small_gam, "edge": edge_instance, "mid_small": mid_small,
         "wide": wide}


@pytest.mark.parametrize("path,tiling", [(0, 0), (0, 2), (0, 3), (0, 4), (1, 0), (2, 1), (2, 2), (2, 3)],
                         ids=["certified", "certified_shared_margins", "certified_slot_major", "certified_row_exact",
                              "general", "double_float_t1", "double_float_t2", "double_float_t3"])
@pytest.mark.parametrize("name", list(CASES))
def test_iterates_track_oracle_200(name, path, tiling):
    if (path, tiling) == (0, 2) and name == "wide":
        pytest.skip("margins in shared memory need the shared-memory product sums (n <= 14464)")
    inst = CASES[name]()
    o = Oracle(inst)
    run = o.run(OracleParams())
    done = 0
    with Solver(inst, path=path, tiling=tiling) as s:
        assert s.stats()["fast_path"] == (0 if path == 1 else 1)
        for t in (1, 2, 5, 63, 64, 65, 128, 129, 200):
            while done < t:
                marg_prev = o.margins(run.y)  # margins the coming iteration uses
                run.step(1)
                done += 1
            st = s.step(t - st_iters(s))
            ost = run.stats()
            assert st["iters"] == ost["t"] == t
            assert st["restarts"] == ost["restarts"] and st["evals"] == ost["evals"]
            assert st["epoch_iters"] == ost["count"]
            assert nrel(s.duals(), run.y) <= ITER_RTOL, (t, nrel(s.duals(), run.y))
            assert nrel(s.vector(2), run.sum_y) <= ITER_RTOL
            assert nrel(s.vector(3), run.sum_g) <= ITER_RTOL
            assert nrel(s.vector(4), run.g) <= ITER_RTOL
            assert nrel(s.vector(5), run.s) <= ITER_RTOL
            assert nrel(s.vector(6), marg_prev) <= ITER_RTOL
            assert st["revenue"] == pytest.approx(ost["P"], rel=ITER_RTOL)
            assert st["z_sum"] == pytest.approx(ost["z_sum"], rel=ITER_RTOL)
            assert st["dual_iter"] == pytest.approx(ost["dual_iter"], rel=ITER_RTOL)
            assert st["tau"] == ost["tau_used"]
            if ost["evals"]:
                for k in ("kkt", "pinf", "gap"):
                    assert st[k] == pytest.approx(ost[k], rel=1e-5, abs=1e-12), k
                assert st["dual_avg"] == pytest.approx(ost["dual_avg"], rel=ITER_RTOL)
                assert st["primal_avg"] == pytest.approx(ost["primal_avg"], rel=ITER_RTOL)
        # binary64 redos stay rare (each iteration solves L segments, each evaluation L more)
        assert st["fallback_segments"] <= max(5, 1e-3 * inst.L * (200 + 3))


def tie_instance():
    """Three MNL segments over products {0, 1} with v = (1/2, 1/4), v0 = 1 and
    prices (3, 1): at y = 0 adding product 1 leaves N/D = 1 unchanged, an exact
    tie that no binary32 certificate can settle."""
    from instances import Instance
    return Instance(n=2, m=1, L=3, r=np.array([3.0, 1.0]), c=np.array([1e30]),
                    a_ptr=np.array([0, 1, 2], np.int32), a_idx=np.array([0, 0], np.int32), a_val=None,
                    seg_ptr=np.array([0, 2, 4, 6], np.int64), seg_prod=np.array([0, 1] * 3, np.int32),
                    v=np.array([0.5, 0.25] * 3), w=None, lam=np.ones(3), v0=np.ones(3), name="tie")


def test_exact_tie_falls_back_to_binary64_and_keeps_smallest_set():
    inst = tie_instance()
    run = Oracle(inst).run(OracleParams(eval_every=0))
    run.step(1)
    np.testing.assert_array_equal(run.s, [1.0, 0.0])
    with Solver(inst, eval_every=0) as s:
        st = s.step(1)
        assert st["fast_path"] == 1 and st["fallback_segments"] == 3
        np.testing.assert_allclose(s.vector(5), run.s, rtol=1e-15, atol=1e-15)
        assert st["z_sum"] == pytest.approx(3.0, rel=1e-15)


def tie_crowd(n_pairs, L):
    """L segments, each the tie of tie_instance on its own product pair
    (pairs reused cyclically over n_pairs): every segment of every block is
    uncertified in binary32."""
    from instances import Instance
    pair = np.arange(L) % n_pairs
    prod = np.stack([2 * pair, 2 * pair + 1], axis=1).ravel().astype(np.int32)
    n = 2 * n_pairs
    return Instance(n=n, m=1, L=L, r=np.tile([3.0, 1.0], n_pairs), c=np.array([1e30]),
                    a_ptr=np.arange(n + 1, dtype=np.int32), a_idx=np.zeros(n, np.int32), a_val=None,
                    seg_ptr=np.arange(0, 2 * L + 1, 2, dtype=np.int64), seg_prod=prod,
                    v=np.tile([0.5, 0.25], L), w=None, lam=np.ones(L), v0=np.ones(L), name="tie_crowd")


@pytest.mark.parametrize("n_pairs", [1, 15_000], ids=["block_sums", "global_sums"])
def test_row_exact_redo_of_a_crowd_of_ties(n_pairs):
    """Row-exact tiling with every segment a binary32 tie: each block's list in
    shared memory overflows into the global list (worked off by the fold kernel
    with per-block sums, by the separate redo kernel with global sums), and the
    sales are those of the binary64 decision, the smallest optimal set."""
    inst = tie_crowd(n_pairs, 40_000)
    run = Oracle(inst).run(OracleParams(eval_every=0))
    run.step(2)
    with Solver(inst, eval_every=0, tiling=4) as s:
        st = s.step(2)
        assert st["fast_path"] == 1 and st["fallback_segments"] == 2 * inst.L
        # the oracle adds 40 000 binary64 terms in order, the kernel rounds each to fixed point
        np.testing.assert_allclose(s.vector(5), run.s, rtol=VALUE_RTOL, atol=0)
        np.testing.assert_array_equal(s.vector(5)[1::2], 0.0)
        np.testing.assert_array_equal(s.duals(), run.y)


def st_iters(s):
    return s.stats()["iters"]


@pytest.mark.parametrize("name", list(CASES))
def test_evaluate_matches_oracle_per_segment(name):
    inst = CASES[name]()
    o = Oracle(inst)
    with Solver(inst) as s:
        for seed in (0, 1, 2):
            y = np.zeros(inst.m) if seed == 0 else seeded_duals(inst.m, seed, float(np.mean(inst.r)) / 3)
            ref = o.sweep(y)
            dual, z = s.evaluate(y, per_segment=True)
            np.testing.assert_allclose(z, ref["z"], rtol=VALUE_RTOL, atol=VALUE_RTOL * max(1.0, np.abs(ref["z"]).max()))
            assert dual == pytest.approx(o.dual(y), rel=VALUE_RTOL)
        # evaluation leaves the iteration state alone
        assert s.stats()["iters"] == 0 and np.all(s.duals() == 0)


def test_uncapacitated_duals_stay_zero():
    inst = tiny_mnl(0, capacity="inf")
    o = Oracle(inst)
    with Solver(inst) as s:
        st = s.step(100)
        assert np.all(s.duals() == 0.0)
        assert st["converged"] == 1 and st["iters"] == 64
        assert st["dual_avg"] == pytest.approx(o.dual(np.zeros(inst.m)), rel=VALUE_RTOL)


@pytest.mark.parametrize("p", [0.3, 0.05])
def test_sampled_iterates_track_oracle(p):
    inst = mid_gam(1, L=20_000, n=1000, m=200)
    prm = dict(batch_frac=p, seed=42)
    run = Oracle(inst).run(OracleParams(**prm))
    with Solver(inst, **prm) as s:
        for t in (1, 3, 64, 150):
            run.step(t - run.stats()["t"])
            st = s.step(t - st_iters(s))
            assert st["iters"] == t and st["restarts"] == run.stats()["restarts"]
            assert nrel(s.duals(), run.y) <= ITER_RTOL
            assert nrel(s.vector(5), run.s) <= ITER_RTOL
            assert np.isnan(st["z_sum"])


@pytest.mark.parametrize("mu,decay,balance", [(0.05, 1.0, 0.0), (0.0, 0.5, 0.0), (0.0, 1.0, 0.5)])
def test_regularised_and_decayed_steps_track_oracle(mu, decay, balance):
    inst = small_gam()
    prm = dict(mu=mu, restart_tau_decay=decay, restart_tau_balance=balance, eval_every=16)
    run = Oracle(inst).run(OracleParams(**prm))
    run.step(200)
    with Solver(inst, **prm) as s:
        st = s.step(200)
        assert st["restarts"] == run.stats()["restarts"] > 0
        assert st["mu"] == run.stats()["mu_cur"]
        # the balanced step depends on pinf / gap, whose last bits differ between the two sides
        assert st["tau"] == pytest.approx(run.stats()["tau_used"], rel=0 if balance == 0 else 1e-12)
        assert nrel(s.duals(), run.y) <= ITER_RTOL


def test_solve_reaches_tolerance_like_oracle():
    inst = mid_gam(1, L=20_000, n=1000, m=200)
    run = Oracle(inst).run(OracleParams())
    for _ in range(200):
        ost = run.step(64)
        if ost["converged"]:
            break
    assert ost["converged"] == 1
    with Solver(inst) as s:
        st = s.solve()
        assert st["converged"] == 1 and st["iters"] == ost["t"] and st["restarts"] == ost["restarts"]
        assert st["dual_avg"] == pytest.approx(ost["dual_avg"], rel=1e-6)
        assert st["kkt"] <= 1e-4
        assert nrel(s.duals(averaged=True), run.ybar) <= ITER_RTOL


@pytest.mark.parametrize("schedule", [dict(restart_tau_decay=0.5), dict(restart_tau_balance=0.5)],
                         ids=["halving", "balanced"])
def test_tiny_capacitated_instance_solves_to_the_lp_optimum(schedule):
    """The tiny MNL instance with c = 0.5 x demand (40 segments, 12 products,
    6 resources) solved to KKT <= 1e-4 on the GPU: the same iteration count,
    restarts and averaged objective as the oracle, and the dual bound at the
    averaged duals above the HiGHS optimum of the SBLP by at most 1e-4 relative
    with the step halved at every restart (this instance's schedule; the
    oracle pin converges at iteration 4544), 3e-4 with tau balanced at
    epoch-length restarts (KKT 1e-4 bounds the gap |Dual - Pbar| by
    1e-4 (1 + |Dual| + |Pbar|), about 2e-4 relative). The default constant
    step stalls on this instance (KKT 1.2e-2)."""
    from pins import sblp_highs
    inst = tiny_mnl(0)
    opt, _ = sblp_highs(inst)
    run = Oracle(inst).run(OracleParams(**schedule))
    for _ in range(400):
        ost = run.step(64)
        if ost["converged"]:
            break
    assert ost["converged"] == 1
    with Solver(inst, **schedule) as s:
        st = s.solve()
        assert st["converged"] == 1 and st["kkt"] <= 1e-4
        assert st["iters"] == ost["t"] and st["restarts"] == ost["restarts"]
        assert st["dual_avg"] == pytest.approx(ost["dual_avg"], rel=1e-6)
        assert nrel(s.duals(averaged=True), run.ybar) <= ITER_RTOL
        bound = 1e-4 if "restart_tau_decay" in schedule else 3e-4
        assert opt * (1 - 1e-9) <= st["dual_avg"] <= opt * (1 + bound)
        assert np.all(s.duals() >= 0)


def test_full_size_mid_instance_first_iterations():
    """The 1e6-segment GAM instance in the benchmark's launch configuration:
    three iterations element by element, and every segment's value at a
    seeded dual point."""
    inst = mid_gam(1)
    o = Oracle(inst)
    run = o.run(OracleParams())
    run.step(3)
    y = seeded_duals(inst.m, 7, float(np.mean(inst.r)) / 4)
    ref = o.sweep(y)
    with Solver(inst) as s:
        st = s.step(3)
        assert nrel(s.duals(), run.y) <= ITER_RTOL
        assert nrel(s.vector(4), run.g) <= ITER_RTOL
        assert nrel(s.vector(5), run.s) <= ITER_RTOL
        assert st["dual_iter"] == pytest.approx(run.stats()["dual_iter"], rel=ITER_RTOL)
        dual, z = s.evaluate(y, per_segment=True)
        np.testing.assert_allclose(z, ref["z"], rtol=VALUE_RTOL, atol=VALUE_RTOL * np.abs(ref["z"]).max())
        assert dual == pytest.approx(ref["zsum"] + float(inst.c @ y), rel=1e-10)


@pytest.mark.slow
@pytest.mark.parametrize("precision", [64, 32])
def test_full_size_huge_instance_sampled(precision):
    """The 1e7-segment, 2e8-nonzero GAM instance in the benchmark's launch
    configuration: one iteration from y = 0 against the oracle's sweep (the
    product sales and consumption it scatters), and the value of a seeded
    sample of 4000 segments at a seeded dual point, each solved on its own by
    the oracle."""
    from instances import huge_gam
    inst = huge_gam(2, workers=12)
    o = Oracle(inst)
    ref0 = o.sweep(np.zeros(inst.m))
    y = seeded_duals(inst.m, 9, float(np.mean(inst.r)) / 4)
    marg = o.margins(y)
    sample = np.sort(np.random.default_rng(3).choice(inst.L, 4000, replace=False))
    with Solver(inst, precision=precision) as s:
        assert s.autotune(8) >= 1
        s.reset()
        s.step(1)
        # binary32 decisions of segments near a tie may differ from the exact ones
        # (reported by the binary32 error test, not bounded): a looser check
        tol = ITER_RTOL if precision == 64 else 1e-3
        assert nrel(s.vector(5), ref0["s"]) <= tol
        assert nrel(s.vector(4), ref0["g"]) <= tol
        _, z = s.evaluate(y, per_segment=True)
    want = np.array([o.segment_solve(int(l), marg)[0] for l in sample])
    np.testing.assert_allclose(z[sample], want, rtol=VALUE_RTOL, atol=VALUE_RTOL * np.abs(want).max())


def _bad(mut):
    inst = tiny_mnl(0)
    inst.v = inst.v.copy()
    inst.seg_prod = inst.seg_prod.copy()
    inst.a_idx = inst.a_idx.copy()
    inst.v0 = inst.v0.copy()
    mut(inst)
    return inst


@pytest.mark.parametrize("mut,status,needle", [
    (lambda I: I.v.__setitem__(3, 0.0), 1, "v["),
    (lambda I: I.v0.__setitem__(2, -1.0), 1, "v0["),
    (lambda I: I.seg_prod.__setitem__(1, I.seg_prod[0]), 1, "repeated"),
    (lambda I: I.a_idx.__setitem__(0, 99), 1, "out of range"),
    (lambda I: setattr(I, "w", I.v * 1.5), 1, "w["),
])
def test_invalid_instances_are_rejected(mut, status, needle):
    from paper_2602_22421_gb300 import SpfomError
    inst = _bad(mut)
    with pytest.raises(SpfomError) as ei:
        Solver(inst)
    assert ei.value.status == status and needle in str(ei.value)


def test_first_failing_nonzero_is_reported():
    """The per-nonzero checks run on the device; the message names the first
    failing nonzero in CSR order, as a host loop would, whatever fails later."""
    from paper_2602_22421_gb300 import SpfomError

    def two_faults(I):
        I.v[7] = -1.0                    # an earlier nonzero: bad attraction
        I.seg_prod[30] = I.n + 5         # a later one: id out of range
    with pytest.raises(SpfomError) as ei:
        Solver(_bad(two_faults))
    assert ei.value.status == 1 and "v[7]" in str(ei.value)

    def id_first(I):
        I.seg_prod[2] = -3
        I.v[9] = 0.0
    with pytest.raises(SpfomError) as ei:
        Solver(_bad(id_first))
    assert ei.value.status == 1 and "seg_prod[2]" in str(ei.value)


def test_segment_checks_run_in_segment_order():
    """Offsets, lambda and v0 are checked on the device too; the message names
    the first failure of a host loop over segments (a segment's own checks
    before its nonzeros, earlier segments first)."""
    from paper_2602_22421_gb300 import SpfomError

    def lam_then_item(I):
        I.lam = I.lam.copy()
        I.lam[6] = -1.0                  # segment 6
        I.v[6 * 4 + 1] = -2.0            # a nonzero of segment 6: reported after its lambda
        I.seg_prod[30 * 4] = -1          # a later segment
    with pytest.raises(SpfomError) as ei:
        Solver(_bad(lam_then_item))
    assert ei.value.status == 1 and "lam[6]" in str(ei.value)

    def order(I):
        I.seg_ptr = I.seg_ptr.copy()
        I.seg_ptr[12] = I.seg_ptr[11] - 1  # segment 11 ends before it starts
        I.v0[20] = 0.0
    with pytest.raises(SpfomError) as ei:
        Solver(_bad(order))
    assert ei.value.status == 1 and "not monotone at 11" in str(ei.value)


def test_binary32_range_is_checked_for_precision_32():
    """Precision 32 keeps binary32 images of v and v - w: an attraction below
    binary32's normal range is unsupported there (ENOTSUP) and fine in
    precision 64."""
    from paper_2602_22421_gb300 import SpfomError
    inst = _bad(lambda I: I.v.__setitem__(5, 1e-40))
    with pytest.raises(SpfomError) as ei:
        Solver(inst, precision=32)
    assert ei.value.status == 7 and "precision 32" in str(ei.value) and "at 5 " in str(ei.value)
    with Solver(inst) as s:
        assert s.step(3)["iters"] == 3


def test_large_consideration_set_is_unsupported():
    """Sets of more than 128 products are rejected; sets of 33..128 need the
    certified-decision path (the sorting kernel takes at most 32)."""
    from paper_2602_22421_gb300 import SpfomError
    with pytest.raises(SpfomError) as ei:
        Solver(make_instance(n=200, m=5, L=10, kmin=129, kmax=129, seed=3))
    assert ei.value.status == 7 and "at most 128" in str(ei.value)
    wide_sets = make_instance(n=60, m=5, L=10, kmin=33, kmax=40, seed=3)
    with pytest.raises(SpfomError) as ei:
        Solver(wide_sets, path=1)
    assert ei.value.status == 7
    with Solver(wide_sets) as s:
        assert s.step(2)["iters"] == 2
        with pytest.raises(SpfomError) as ei:
            s.sales_at(np.zeros(5))
        assert ei.value.status == 7


def paper_shaped_small():
    """The paper's speedup-study shape (Section 4.5): every segment considers
    all 100 products, MNL, one resource per product, at 2000 segments."""
    from instances import paper_shaped
    return paper_shaped(3, L=2000, n=100)


def wide_sets_gam():
    """GAM instance with sets of 60..100 of 120 products."""
    return make_instance(n=120, m=60, L=3000, kmin=60, kmax=100, gam=True, tightness=0.6, seed=3, name="wide_sets")


@pytest.mark.parametrize("tiling", [0, 4], ids=["lanes_16x8", "row_exact"])
@pytest.mark.parametrize("make", [paper_shaped_small, wide_sets_gam], ids=["paper_shaped_mnl", "gam_60_100"])
def test_sets_of_100_products_track_oracle(make, tiling):
    """Sets of up to 100 products (16 lanes x 8 slots per segment, or 8 lanes
    x <= 13 exact rows in the row-exact tiling): the binary64 iterates track
    the oracle as for small sets."""
    inst = make()
    o = Oracle(inst)
    run = o.run(OracleParams())
    done = 0
    with Solver(inst, tiling=tiling) as s:
        assert s.stats()["fast_path"] == 1
        for t in (1, 2, 63, 64, 65, 200):
            while done < t:
                run.step(1)
                done += 1
            st = s.step(t - st_iters(s))
            ost = run.stats()
            assert st["iters"] == ost["t"] == t and st["restarts"] == ost["restarts"]
            assert nrel(s.duals(), run.y) <= ITER_RTOL, (t, nrel(s.duals(), run.y))
            assert nrel(s.vector(5), run.s) <= ITER_RTOL
            assert st["z_sum"] == pytest.approx(ost["z_sum"], rel=ITER_RTOL)
            if ost["evals"]:
                assert st["kkt"] == pytest.approx(ost["kkt"], rel=1e-5, abs=1e-12)


def test_row_exact_tiling_mixes_every_lane_class():
    """One instance whose sets span 0..128 products, so the row-exact copy holds
    all four lane classes (1, 2, 4, 8 lanes per segment), partial chunks at each
    class boundary and empty sets: 200 iterations track the oracle."""
    inst = make_instance(n=400, m=40, L=3001, kmin=0, kmax=128, gam=True, tightness=0.6, seed=21,
                         name="all_classes")
    o = Oracle(inst)
    run = o.run(OracleParams())
    done = 0
    with Solver(inst, tiling=4) as s:
        for t in (1, 64, 65, 200):
            while done < t:
                run.step(1)
                done += 1
            st = s.step(t - st_iters(s))
            ost = run.stats()
            assert st["iters"] == ost["t"] == t and st["restarts"] == ost["restarts"]
            assert nrel(s.duals(), run.y) <= ITER_RTOL, (t, nrel(s.duals(), run.y))
            assert nrel(s.vector(5), run.s) <= ITER_RTOL
            assert st["z_sum"] == pytest.approx(ost["z_sum"], rel=ITER_RTOL)


@pytest.mark.parametrize("n,L", [(200, 100_000), (16_000, 20_001), (22_000, 20_001)],
                         ids=["two_sums_blocks", "shared_margins", "one_sums_block"])
def test_row_exact_forms_by_product_count(n, L):
    """The row-exact kernels take their form from the product count. The
    binary64 pass keeps per-block sums in shared memory at two 768-thread
    blocks per SM while two such blocks fit (n up to about 14 400; n = 200
    here, with 5000 slots per product), then the sums and binary32 margins in
    one 1024-thread block (n = 16 000), then one block of shared sums
    (n = 22 000), then global sums (the wide instance of the other tests). The
    binary32 pass keeps shared margins up to about 19 300 products and shared
    sums beyond. The binary64 iterates track the oracle for 200 iterations, and
    the binary32 solve reaches the binary64 objective."""
    inst = mid_gam(1, L=L, n=n, m=min(400, n // 2))
    run = Oracle(inst).run(OracleParams())
    done = 0
    with Solver(inst, tiling=4) as s:
        for t in (1, 64, 65, 200):
            while done < t:
                run.step(1)
                done += 1
            st = s.step(t - st_iters(s))
            ost = run.stats()
            assert st["iters"] == ost["t"] == t and st["restarts"] == ost["restarts"]
            assert nrel(s.duals(), run.y) <= ITER_RTOL, (t, nrel(s.duals(), run.y))
            assert nrel(s.vector(5), run.s) <= ITER_RTOL
        s.reset()
        ref = s.solve()
    with Solver(inst, precision=32, tiling=9) as s:
        st = s.solve()
    assert ref["converged"] == 1 and st["converged"] == 1 and st["kkt"] <= 1e-4
    assert st["dual_avg"] == pytest.approx(ref["dual_avg"], rel=1e-4)


@pytest.mark.parametrize("precision,tiling", [(64, 2), (64, 4), (32, 9)])
def test_solvers_of_different_sizes_coexist(precision, tiling):
    """A kernel's shared-memory limit is one setting per process and context.
    Loading a smaller instance into a second solver (a smaller shared-memory
    plan) must not lower the limit that the first solver's kernels launch
    with: both go on with the iterates a solver alone computes."""
    big = mid_gam(1, L=20_001, n=10_000, m=400)
    small = mid_gam(2, L=5_001, n=1_000, m=100)
    ref = {}
    for name, inst in (("big", big), ("small", small)):
        with Solver(inst, precision=precision, tiling=tiling) as s:
            s.step(65)
            ref[name] = s.duals()
    a = Solver(big, precision=precision, tiling=tiling)
    b = Solver(small, precision=precision, tiling=tiling)
    try:
        b.step(65)
        a.step(65)
        np.testing.assert_array_equal(a.duals(), ref["big"])
        np.testing.assert_array_equal(b.duals(), ref["small"])
    finally:
        b.close()
        a.close()


def test_sets_of_100_products_binary32_solve():
    """The binary32 bulk mode (32 lanes x 4 slots, 16 x 8, or the row-exact
    layout) on sets of up to 100 products solves to KKT <= 1e-4 at the binary64
    solve's objective."""
    inst = wide_sets_gam()
    with Solver(inst) as s:
        ref = s.solve()
    with Solver(inst, precision=32) as s:
        assert s.autotune(8) in (1, 3, 9)
        st = s.solve()
    assert ref["converged"] == 1 and st["converged"] == 1 and st["kkt"] <= 1e-4
    assert st["dual_avg"] == pytest.approx(ref["dual_avg"], rel=1e-4)


# -- binary32 bulk mode (precision 32) --------------------------------------
FP32_ERRORS = {}


@pytest.mark.parametrize("name", ["mid_small", "wide", "edge"])
def test_fp32_bulk_error_against_fp64_oracle(name, tiling=0):
    """Binary32 segment solves with binary64 residuals: the error against the
    FP64 oracle is reported per result (FP32_ERRORS) and bounded: one iteration
    from y = 0 is within binary32 rounding; after 200 iterations the iterates
    stay close although binary32 decisions near ties may differ."""
    inst = CASES[name]()
    run = Oracle(inst).run(OracleParams())
    with Solver(inst, precision=32, tiling=tiling) as s:
        st = s.step(1)
        run.step(1)
        assert st["iter_precision"] == 32 and st["fast_path"] == 1
        e = {"y@1": nrel(s.duals(), run.y), "s@1": nrel(s.vector(5), run.s), "g@1": nrel(s.vector(4), run.g),
             "z_sum@1": abs(st["z_sum"] / run.stats()["z_sum"] - 1)}
        assert max(e.values()) <= 1e-5, e
        st = s.step(199)
        run.step(199)
        ost = run.stats()
        e.update({"y@200": nrel(s.duals(), run.y), "g@200": nrel(s.vector(4), run.g),
                  "dual_avg@200": abs(st["dual_avg"] / ost["dual_avg"] - 1),
                  "kkt@200": abs(st["kkt"] - ost["kkt"])})
        FP32_ERRORS[name] = e
        print(f"binary32 vs FP64 oracle errors ({name}): {e}")
        assert e["y@200"] <= 1e-2 and e["dual_avg@200"] <= 1e-5 and e["kkt@200"] <= 1e-4, e


def test_fp32_bulk_solve_matches_fp64_objective():
    """Time-to-KKT form: binary32 iterations, binary64 KKT checks and a binary64
    polish reach KKT <= 1e-4 with the dual objective within 1e-4 of the FP64
    oracle's at its own KKT <= 1e-4."""
    inst = mid_gam(1, L=20_000, n=1000, m=200)
    run = Oracle(inst).run(OracleParams())
    for _ in range(200):
        ost = run.step(64)
        if ost["converged"]:
            break
    with Solver(inst, precision=32) as s:
        st = s.solve()
        assert st["converged"] == 1 and st["kkt"] <= 1e-4 and st["iter_precision"] == 64
        assert st["dual_avg"] == pytest.approx(ost["dual_avg"], rel=1e-4)
        assert st["primal_avg"] == pytest.approx(ost["primal_avg"], rel=1e-4)
    with Solver(inst, precision=32, polish=0) as s:
        st = s.solve()
        assert st["converged"] == 1 and st["iter_precision"] == 32
        assert st["dual_avg"] == pytest.approx(ost["dual_avg"], rel=1e-4)


@pytest.mark.parametrize("precision", [64, 32])
def test_graph_replay_equals_direct_launches(precision):
    """Whole evaluation periods replayed from a CUDA graph give bit-identical
    iterates to direct launches (the sums are fixed point, the partial sums
    fold in block order)."""
    inst = mid_small()
    out = {}
    for graphs in (0, 1):
        with Solver(inst, precision=precision, graphs=graphs) as s:
            s.step(5)      # leaves the period boundary: the next call starts with direct launches
            st = s.step(195)
            out[graphs] = (s.duals(), s.vector(3), st["kkt"], st["restarts"], st["kernel_launches"])
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] and out[0][3] == out[1][3] and out[0][4] == out[1][4]


@pytest.mark.parametrize("name", ["mid_small", "wide", "edge"])
def test_pipeline_equals_plain_loads(name):
    """The warp-specialised bulk-copy pipeline computes what the plain-load
    certified kernel computes: fixed-point sales make s, g and y identical;
    only the block grouping of the z partial sums differs."""
    inst = CASES[name]()
    out = {}
    for pipeline in (0, 1):
        with Solver(inst, pipeline=pipeline) as s:
            st = s.step(130)
            out[pipeline] = (s.duals(), s.vector(5), st)
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][2]["restarts"] == out[1][2]["restarts"]
    assert out[0][2]["z_sum"] == pytest.approx(out[1][2]["z_sum"], rel=1e-13)


@pytest.mark.parametrize("name", ["mid_small", "wide", "edge"])
def test_fp32_cooperative_staging_equals_plain_loads(name):
    """Tiling 4 (tiles streamed into shared memory by the whole block) runs the
    same slot layout and summation order as tiling 3 (plain loads, 8 products
    per lane): duals, sales and segment values agree bit for bit."""
    inst = CASES[name]()
    out = {}
    for tiling in (3, 4):
        with Solver(inst, precision=32, tiling=tiling) as s:
            st = s.step(130)
            out[tiling] = (s.duals(), s.vector(5), st)
    np.testing.assert_array_equal(out[3][0], out[4][0])
    np.testing.assert_array_equal(out[3][1], out[4][1])
    assert out[3][2]["restarts"] == out[4][2]["restarts"]
    assert out[3][2]["z_sum"] == pytest.approx(out[4][2]["z_sum"], rel=1e-6)


@pytest.mark.parametrize("name", ["mid_small", "edge", "tiny_mnl", "wide"])
@pytest.mark.parametrize("precision,plain,shared", [(64, 1, 2), (32, 3, 7), (64, 1, 3), (32, 3, 8)],
                         ids=["f64_shared_margins", "f32_shared_margins", "f64_slot_major", "f32_slot_major"])
def test_tilings_equal_plain_loads(name, precision, plain, shared):
    """The margins-in-shared-memory kernels (precision 64 tiling 2, precision
    32 tiling 7) and the slot-major kernels (tilings 3 and 8: segments sorted
    by set size, slot rows of 32 entries) solve every segment as the
    plain-load kernel of the same lane layout does (tilings 1 and 3): the same
    products in each lane's slots, summed in the same order. The product sums
    are exact fixed point, so duals and sales agree bit for bit; only the order
    of the per-thread segment-value sums differs."""
    if name == "wide" and shared in (2, 7):
        pytest.skip("margins in shared memory need the shared-memory product sums (n <= 14464)")
    inst = CASES[name]()
    out = {}
    for tiling in (plain, shared):
        with Solver(inst, precision=precision, tiling=tiling) as s:
            st = s.step(130)
            out[tiling] = (s.duals(), s.vector(5), st)
    np.testing.assert_array_equal(out[plain][0], out[shared][0])
    np.testing.assert_array_equal(out[plain][1], out[shared][1])
    assert out[plain][2]["restarts"] == out[shared][2]["restarts"]
    assert out[plain][2]["z_sum"] == pytest.approx(out[shared][2]["z_sum"], rel=1e-6 if precision == 32 else 1e-12)


@pytest.mark.parametrize("tiling", [1, 3, 5, 7, 8, 9])
def test_fp32_tilings_solve_to_the_binary64_objective(tiling):
    """Each plain-load binary32 tiling (4, 8 or 16 products per lane, the
    slot-major and the row-exact copies) solves the mid-size instance to KKT
    <= 1e-4 (with binary64 polish) at the binary64 solve's objective."""
    inst = mid_small()
    with Solver(inst) as s:
        ref = s.solve()
    with Solver(inst, precision=32, tiling=tiling) as s:
        st = s.solve()
    assert st["converged"] == 1 and st["kkt"] <= 1e-4
    assert st["dual_avg"] == pytest.approx(ref["dual_avg"], rel=1e-4)


@pytest.mark.parametrize("name", ["mid_small", "wide", "edge"])
def test_fp32_row_exact_error_against_fp64_oracle(name):
    """The row-exact binary32 pass (tiling 9) keeps the bulk mode's error bounds
    against the FP64 oracle (one iteration within binary32 rounding, 200
    iterations close)."""
    test_fp32_bulk_error_against_fp64_oracle(name, tiling=9)
