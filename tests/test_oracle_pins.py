"""The FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it pins. A plausible slip anywhere in the oracle
(a dropped attraction term, a wrong sign in the margins or the dual step, a
transposed incidence, a wrong tie rule) fails at least one of them.
"""
import math

import numpy as np
import pytest

from instances import make_instance, mid_gam, seeded_duals, tiny_mnl
from oracle import Oracle, Params, sample_hash

from pins import (brute_force_all_products, brute_force_segment, cblp_highs, dense_A, sales_of,
                  sblp_highs)


def small_gam(seed=5, L=60, n=30, m=8, kmin=3, kmax=8, tightness=0.6):
    return make_instance(n=n, m=m, L=L, kmin=kmin, kmax=kmax, gam=True, tightness=tightness, seed=seed,
                         name="small_gam")


def with_zero_vt(inst, frac=0.2, seed=9):
    """Copy with w = v on a random fraction of items (vt = 0: the item never
    enlarges the denominator)."""
    rng = np.random.default_rng(seed)
    w = inst.w.copy()
    pick = rng.uniform(size=w.size) < frac
    w[pick] = inst.v[pick]
    out = inst.with_capacity(inst.c)
    out.w = w
    return out


def dual_points(inst, k=4):
    scale = float(np.mean(inst.r)) / 3.0
    return [np.zeros(inst.m)] + [seeded_duals(inst.m, 100 + s, scale) for s in range(k)]


# -- a1: margins ------------------------------------------------------------
@pytest.mark.parametrize("make", [tiny_mnl, small_gam])
def test_margins_equal_dense_product(make):
    """m = r - A^T y (Section 4.1 inner objective, eq. new_NRM_1 incidence), via a dense matmul."""
    inst = make()
    o = Oracle(inst)
    A = dense_A(inst)
    for y in dual_points(inst):
        np.testing.assert_allclose(o.margins(y), inst.r - A.T @ y, rtol=0, atol=1e-12)


# -- a2: exact best response ------------------------------------------------
@pytest.mark.parametrize("make", [tiny_mnl, small_gam, lambda: with_zero_vt(small_gam())])
def test_best_response_equals_brute_force(make):
    """z_l(y) equals the best of all 2^K assortments under the closed-form pi'
    of Section 3, and the returned sales are that assortment's sales."""
    inst = make()
    o = Oracle(inst)
    for y in dual_points(inst):
        marg = o.margins(y)
        for l in range(inst.L):
            z, x, kstar = o.segment_solve(l, marg)
            zb, sets = brute_force_segment(inst, l, marg)
            assert z == pytest.approx(zb, rel=1e-12, abs=1e-12)
            assert any(np.allclose(x, sales_of(inst, l, S), rtol=1e-12, atol=1e-14) for S in sets)
            assert int((x > 0).sum()) == kstar


def test_best_response_picks_smallest_optimal_set():
    """Ties: when adding the next product leaves N/D unchanged the response
    keeps the smaller prefix. Dyadic data make the tie exact: v = (1/2, 1/4),
    v0 = 1, margins (3, 1) give N/D = 1.5/1.5 = 1.75/1.75 = 1."""
    inst = tiny_mnl(0)
    l = 0
    b = int(inst.seg_ptr[l])
    inst.v = inst.v.copy()
    inst.v[b:b + 2] = [0.5, 0.25]
    o = Oracle(inst)
    prod, v, _ = inst.segment(l)
    marg = np.zeros(inst.n)
    marg[prod[0]], marg[prod[1]] = 3.0, 1.0
    z, x, kstar = o.segment_solve(l, marg)
    assert kstar == 1
    assert x[1] == 0.0 and x[0] == inst.lam[l] * 0.5 / 1.5
    assert z == inst.lam[l] * 1.0


def test_uncapacitated_brute_force_over_whole_catalogue():
    """Tiny plain instance with c = infinity: Dual(0) = sum_l max over all 2^n
    assortments of the catalogue (products outside C_l have no attraction), and
    the iteration never moves y off 0."""
    inst = tiny_mnl(0, capacity="inf")
    o = Oracle(inst)
    marg = o.margins(np.zeros(inst.m))
    np.testing.assert_array_equal(marg, inst.r)
    want = sum(brute_force_all_products(inst, l, marg) for l in range(inst.L))
    assert o.dual(np.zeros(inst.m)) == pytest.approx(want, rel=1e-12)
    run = o.run(Params(eval_every=16))
    st = run.step(200)
    assert np.all(run.y == 0.0)
    assert st["converged"] == 1
    assert st["dual_avg"] == pytest.approx(want, rel=1e-12)


# -- Lemma 1: Algorithm 1 + golden section -----------------------------------
@pytest.mark.parametrize("make", [tiny_mnl, small_gam, lambda: with_zero_vt(small_gam())])
def test_fast_inner_and_golden_section_reach_exact_value(make):
    """Algorithm 1 at the optimal no-purchase level reproduces the exact
    response, and golden-section search over it converges to z_l (Lemma 1)."""
    inst = make()
    o = Oracle(inst)
    for y in dual_points(inst, 2):
        marg = o.margins(y)
        for l in range(inst.L):
            z, x, kstar = o.segment_solve(l, marg)
            zg = o.golden(l, marg, 1e-12)
            assert zg <= z * (1 + 1e-12) + 1e-12
            assert zg == pytest.approx(z, rel=1e-9, abs=1e-9)
            zc = o.golden(l, marg, 1e-3)  # the paper's epsilon
            assert zc <= z * (1 + 1e-12) + 1e-12 and zc >= z * (1 - 2e-2)
            if kstar > 0:
                prod, v, w = inst.segment(l)
                vt0 = inst.v0[l] + w.sum()
                D = vt0 + (v - w)[x > 0].sum()
                val, xg = o.fast_inner(l, marg, inst.lam[l] / D)
                assert val == pytest.approx(z, rel=1e-12)
                np.testing.assert_allclose(xg, x, rtol=1e-12, atol=1e-14)


# -- Section 3.2 equivalence, strong and weak duality -------------------------
@pytest.mark.parametrize("make", [tiny_mnl, small_gam])
def test_sblp_equals_cblp_and_strong_duality(make):
    """SBLP = CBLP (Section 3.2) under the GAM reading; the oracle's dual
    function at HiGHS's capacity duals equals the optimum; any y >= 0 bounds
    it from above (weak duality)."""
    inst = make()
    opt_s, ystar = sblp_highs(inst)
    opt_c = cblp_highs(inst)
    assert opt_s == pytest.approx(opt_c, rel=1e-7)
    o = Oracle(inst)
    assert o.dual(ystar) == pytest.approx(opt_s, rel=1e-7)
    for y in dual_points(inst, 6):
        assert o.dual(y) >= opt_s * (1 - 1e-9)


# -- a3: sales, consumption, revenue ----------------------------------------
@pytest.mark.parametrize("make", [tiny_mnl, small_gam])
def test_consumption_is_dual_gradient(make):
    """The dual function is piecewise linear with gradient c - A s(y)
    (Danskin); finite differences of Dual recover g, and the Lagrangian
    identity sum_l z_l = P - y^T g holds, i.e. sum_l z_l = sum_j m_j s_j (the
    form in which the GPU's dual step takes the iteration's sum of z)."""
    inst = make()
    o = Oracle(inst)
    A = dense_A(inst)
    for y in dual_points(inst, 3)[1:]:
        sw = o.sweep(y)
        np.testing.assert_allclose(sw["g"], A @ sw["s"], rtol=1e-12, atol=1e-12)
        assert sw["P"] == pytest.approx(float(inst.r @ sw["s"]), rel=1e-12)
        assert sw["zsum"] == pytest.approx(sw["P"] - float(y @ sw["g"]), rel=1e-10, abs=1e-9)
        assert sw["zsum"] == pytest.approx(float(o.margins(y) @ sw["s"]), rel=1e-10, abs=1e-9)
        D0 = o.dual(y)
        h = 1e-6 * max(1.0, float(np.mean(y)))
        for i in range(inst.m):
            e = np.zeros(inst.m); e[i] = h
            fd = (o.dual(y + e) - D0) / h
            assert fd == pytest.approx(inst.c[i] - sw["g"][i], rel=1e-4, abs=1e-4 * (1 + inst.c[i]))


# -- a4..a6: the run --------------------------------------------------------
def test_run_converges_to_lp_optimum_tiny():
    """Projected dual ascent (Algorithm 2, full batch) with averaging and
    restarts drives the dual bound at the averaged duals to the HiGHS optimum
    from above and the KKT residual to 1e-4 on the tiny capacitated MNL
    instance. With 40 segments the dual function is very non-smooth and a
    constant step leaves an O(tau) duality gap, so this instance's schedule
    halves the step at every restart (restart_tau_decay = 0.5, a restarted
    subgradient schedule); it converges at iteration 4544. Balancing tau at
    epoch-length restarts (restart_tau_balance = 0.5) converges too, later."""
    inst = tiny_mnl(0)
    opt, _ = sblp_highs(inst)
    o = Oracle(inst)
    run = o.run(Params(eval_every=64, restart_tau_decay=0.5, restart_tau_balance=0.0, kkt_tol=1e-4))
    ys = []
    for _ in range(80):
        st = run.step(64)
        ys.append(run.y.copy())
        if st["converged"]:
            break
    assert st["converged"] == 1 and st["kkt"] <= 1e-4, st
    assert st["t"] <= 80 * 64
    assert all(np.all(y >= 0) for y in ys)
    assert opt * (1 - 1e-12) <= st["dual_avg"] <= opt * (1 + 1e-4)
    assert o.dual(run.ybar) >= opt * (1 - 1e-12)
    balanced = o.run(Params(restart_tau_balance=0.5))
    for _ in range(300):
        st = balanced.step(64)
        if st["converged"]:
            break
    assert st["converged"] == 1 and st["kkt"] <= 1e-4, st
    assert opt * (1 - 1e-12) <= st["dual_avg"] <= opt * (1 + 3e-4)


@pytest.mark.slow
def test_run_converges_to_lp_optimum_gam():
    """Same on a GAM instance with many segments and the default constant step."""
    inst = mid_gam(1, L=3000, n=200, m=40)
    opt, _ = sblp_highs(inst)
    o = Oracle(inst)
    run = o.run(Params(eval_every=64, kkt_tol=1e-4, restart_tau_decay=0.7))
    for _ in range(60):
        st = run.step(64)
        if st["converged"]:
            break
    assert st["converged"] == 1, st
    assert st["dual_avg"] == pytest.approx(opt, rel=2e-4)


def test_balanced_restarts_reach_the_optimum_where_a_constant_step_stalls():
    """An instance of the batched family with few segments per product (1475
    segments, 4511 products): with the constant step the averaged duality gap
    stalls near 1e-3 (an O(tau) gap); balancing tau at the restarts the
    epoch-length rule forces reaches KKT <= 1e-4 and the HiGHS optimum."""
    from instances import batch_base
    inst = batch_base(4, 10)
    opt, _ = sblp_highs(inst)
    o = Oracle(inst)
    const = o.run(Params(restart_tau_balance=0.0))
    for _ in range(60):
        st = const.step(64)
    assert st["converged"] == 0 and st["gap"] > 3 * st["pinf"]
    run = o.run(Params(restart_tau_balance=0.5))
    for _ in range(300):
        st = run.step(64)
        if st["converged"]:
            break
    assert st["converged"] == 1, st
    assert st["dual_avg"] == pytest.approx(opt, rel=2e-4)
    assert o.dual(run.ybar) >= opt * (1 - 1e-12)


def test_regularised_step_shrinks_duals():
    """eq. stronglycvxupdate: with consumption equal to capacity the step
    reduces to y <- (1 - tau mu) y. Capacities are set to the consumption at a
    seeded y so that c - g = 0 there."""
    inst = small_gam()
    o = Oracle(inst)
    y0 = dual_points(inst, 2)[1]
    g = o.sweep(y0)["g"]
    inst2 = inst.with_capacity(g)
    o2 = Oracle(inst2)
    run = o2.run(Params(tau=0.05, mu=2.0, eval_every=0))
    run.y[:] = y0
    run.step(1)
    np.testing.assert_allclose(run.y, (1 - 0.05 * 2.0) * y0, rtol=1e-13, atol=1e-13)
    assert run.stats()["P"] == pytest.approx(float(inst.r @ o.sweep(y0)["s"]), rel=1e-12)


def test_step_sign_follows_overuse():
    """Projected ascent on the capacity prices (Algorithm 2): a resource used
    beyond capacity gets a higher price, an idle one is clipped at 0."""
    inst = small_gam()
    o = Oracle(inst)
    g0 = o.sweep(np.zeros(inst.m))["g"]
    run = o.run(Params(tau=0.01, eval_every=0))
    run.step(1)
    over = g0 > inst.c
    assert np.all(run.y[over] > 0)
    assert np.all(run.y[~over] == 0)
    np.testing.assert_allclose(run.y[over], 0.01 * (g0 - inst.c)[over], rtol=1e-13)


# -- a7: sampling -------------------------------------------------------------
def test_splitmix64_published_values():
    """SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: the first three
    outputs are e220a8397b1dcdaf, 6e789e6aa1b965f4, 06c45d188009454f. The k-th
    output is the hash of (k-1) * 0x9e3779b97f4a7c15."""
    gamma = 0x9E3779B97F4A7C15
    assert sample_hash(0, 0, 0) == 0xE220A8397B1DCDAF
    assert sample_hash(gamma, 0, 0) == 0x6E789E6AA1B965F4
    assert sample_hash((2 * gamma) % (1 << 64), 0, 0) == 0x06C45D188009454F


def test_sampled_run_keeps_stale_responses():
    """Bernoulli(p) sampling: about p L segments are re-solved per iteration
    (E[S_t] = p I), the aggregate runs over every segment's current response,
    and unsampled segments keep their last response."""
    inst = small_gam(L=2000, n=60, m=12)
    o = Oracle(inst)
    p = 0.3
    frac = np.mean([sample_hash(7, 1, l) < int(math.ldexp(p, 64)) for l in range(inst.L)])
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / inst.L)
    run = o.run(Params(tau=0.01, batch_frac=p, seed=7, eval_every=0))
    run.step(3)
    K = np.diff(inst.seg_ptr)
    s = np.bincount(inst.seg_prod, weights=run.x_cur, minlength=inst.n)
    np.testing.assert_allclose(run.s, s, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(run.g, dense_A(inst) @ s, rtol=1e-12, atol=1e-12)
    assert K.min() >= 3


# -- checker: every workload shape --------------------------------------------
def _wide_sets():
    return make_instance(n=60, m=10, L=200, kmin=33, kmax=40, gam=True, tightness=0.6, seed=8, name="wide_sets")


def _paper_shaped_small():
    from instances import paper_shaped
    return paper_shaped(3, L=100, n=100)


@pytest.mark.parametrize("make", [tiny_mnl, small_gam, lambda: with_zero_vt(small_gam()), _wide_sets,
                                  _paper_shaped_small],
                         ids=["tiny_mnl", "small_gam", "zero_vt", "wide_sets", "paper_shaped"])
def test_checker_holds_along_the_run(make):
    """Along a run on every workload shape: the duals and their averages stay
    >= 0, and the Lagrangian bound holds at the epoch average, since the
    averaged response is a convex combination of assortment points:
    Dual(y) >= Pbar + y^T (c - gbar) for every y >= 0 (weak duality)."""
    inst = make()
    o = Oracle(inst)
    run = o.run(Params())
    ys = dual_points(inst, 3)
    done = 0
    for t in (1, 10, 64, 130, 200):
        run.step(t - done)
        done = t
        st = run.stats()
        assert (run.y >= 0).all() and (run.ybar >= 0).all()
        if st["count"] == 0:
            continue
        pbar = st["sum_P"] / st["count"]
        for y in ys + [run.y, run.ybar]:
            d = o.dual(y)
            assert d >= pbar + float(y @ (inst.c - run.gbar)) - 1e-9 * (1.0 + abs(d)), (t, d)
