"""Pins of the oracle's recovery of assortment probabilities from sales
(Lemma recover, Section 4.4) and of its epoch-averaged sales x-bar, against
the closed-form choice probabilities, a hand-worked segment, and HiGHS on the
sales-based and the enumerated choice-based LP. CPU only."""
import numpy as np
import pytest

from instances import make_instance, mid_gam, tiny_mnl
from instances.gam import Instance
from oracle import Oracle, Params
from pins import cblp_highs, dense_A, gam_prob, sales_of, sblp_highs


def reconstruct(inst, alpha, order):
    """lam_l sum_r alpha_r pi_j(S_r) per nonzero, S_r = the top-r products."""
    out = np.zeros(inst.nnz)
    for l in range(inst.L):
        b, e = inst.seg_ptr[l], inst.seg_ptr[l + 1]
        prod, v, w = inst.segment(l)
        K = e - b
        al = alpha[b + l: b + l + K + 1]
        S = np.zeros(K, bool)
        for r in range(1, K + 1):
            S[order[b + r - 1]] = True
            out[b:e] += inst.lam[l] * al[r] * gam_prob(v, w, inst.v0[l], S)
    return out


def mixed_sales(inst, seed, parts=3):
    """Per segment, a random convex combination of `parts` random assortment points."""
    rng = np.random.default_rng(seed)
    x = np.zeros(inst.nnz)
    for l in range(inst.L):
        b, e = inst.seg_ptr[l], inst.seg_ptr[l + 1]
        wts = rng.dirichlet(np.ones(parts))
        for q in range(parts):
            S = rng.random(e - b) < 0.5
            x[b:e] += wts[q] * sales_of(inst, l, S)
    return x


def test_hand_worked_segment():
    """v = (1, 2, 1), v0 = 1, lam = 1 (MNL); half {A}, half {A, B}:
    x = (0.375, 0.25, 0); u = x / v ranks A, B, C; x0 = 0.375;
    alpha = (0, 0.5, 0.5, 0) for (empty, {A}, {A, B}, {A, B, C})."""
    inst = Instance(n=3, m=1, L=1, r=np.ones(3), c=np.ones(1), a_ptr=np.array([0, 1, 2, 3], np.int32),
                    a_idx=np.zeros(3, np.int32), a_val=None, seg_ptr=np.array([0, 3], np.int64),
                    seg_prod=np.array([0, 1, 2], np.int32), v=np.array([1.0, 2.0, 1.0]), w=None,
                    lam=np.array([1.0]), v0=np.array([1.0]))
    alpha, order = Oracle(inst).recover(np.array([0.375, 0.25, 0.0]))
    np.testing.assert_allclose(alpha, [0.0, 0.5, 0.5, 0.0], atol=1e-15)
    assert list(order) == [0, 1, 2]


@pytest.mark.parametrize("gam", [False, True])
def test_recovered_probabilities_reproduce_the_sales(gam):
    inst = make_instance(n=40, m=8, L=300, kmin=0, kmax=12, gam=gam, seed=21)
    x = mixed_sales(inst, 22)
    alpha, order = Oracle(inst).recover(x)
    assert alpha.min() >= -1e-12
    sums = np.array([alpha[inst.seg_ptr[l] + l: inst.seg_ptr[l + 1] + l + 1].sum() for l in range(inst.L)])
    np.testing.assert_allclose(sums, 1.0, atol=1e-12)
    np.testing.assert_allclose(reconstruct(inst, alpha, order), x, atol=1e-13)


def test_sblp_optimum_recovers_to_a_cblp_optimum():
    """HiGHS's SBLP optimum, mapped back, is a feasible CBLP point with the
    CBLP optimum's revenue (the two LPs have the same value)."""
    inst = tiny_mnl(0)
    opt_s, _, x = sblp_highs(inst, return_x=True)
    alpha, order = Oracle(inst).recover(np.maximum(x, 0.0))
    assert alpha.min() >= -1e-9
    xr = reconstruct(inst, alpha, order)
    np.testing.assert_allclose(xr, np.maximum(x, 0.0), atol=1e-9)
    revenue = float(inst.r[inst.seg_prod] @ xr)
    s = np.bincount(inst.seg_prod, weights=xr, minlength=inst.n)
    assert (dense_A(inst) @ s <= inst.c + 1e-8).all()
    opt_c = cblp_highs(inst)
    opt_c = opt_c[0] if isinstance(opt_c, tuple) else opt_c
    assert revenue == pytest.approx(opt_s, rel=1e-8)
    assert revenue == pytest.approx(opt_c, rel=1e-7)


def test_epoch_average_of_the_responses():
    """x-bar of an oracle run is SBLP-feasible per segment and aggregates to
    the averaged consumption g-bar."""
    inst = mid_gam(8, L=2000, n=120, m=24)
    run = Oracle(inst).run(Params(), track_x=True)
    run.step(150)
    xb = run.xbar
    w = inst.w if inst.w is not None else np.zeros(inst.nnz)
    vt = inst.v - w
    seg_of = np.repeat(np.arange(inst.L), np.diff(inst.seg_ptr))
    vt0 = inst.v0 + np.bincount(seg_of, weights=w, minlength=inst.L)
    x0 = inst.lam - np.bincount(seg_of, weights=vt / inst.v * xb, minlength=inst.L)
    assert (x0 >= -1e-12).all() and (xb >= 0).all()
    assert (xb / inst.v <= (x0 / vt0)[seg_of] + 1e-12).all()
    s = np.bincount(inst.seg_prod, weights=xb, minlength=inst.n)
    np.testing.assert_allclose(dense_A(inst) @ s, run.gbar, rtol=1e-11, atol=1e-12)
    alpha, _ = Oracle(inst).recover(xb)
    assert alpha.min() >= -1e-12
