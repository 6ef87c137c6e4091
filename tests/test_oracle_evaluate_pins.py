"""The oracle's KKT evaluation and restart rules against a hand-worked case (CPU only).

The paper forms no residuals (the Remark after Theorem 2 in Section 4.2
contrasts SPFOM with PDLP on exactly this point), so the averaging, the KKT
residual and the restart rules are the solver's own definition:

    ybar = sum_y / count,  gbar = sum_g / count,  Pbar = sum_P / count,
    pinf = ||(gbar - c)_+||_2 / (1 + ||c||_2),
    gap  = |Dual(ybar) - Pbar| / (1 + |Dual(ybar)| + |Pbar|),   KKT = max(pinf, gap);
    converged iff KKT <= kkt_tol; otherwise restart when KKT <= beta * KKT_anchor
    (progress) or count >= restart_artificial * t (epoch length): y <- ybar,
    sums cleared, KKT_anchor <- KKT, mu <- mu / 2, tau <- tau * decay, and for an
    epoch-length restart with balance b > 0, tau <- tau * clamp(sqrt(pinf / gap), b, 1 / b).

Every number below is worked by hand on an instance whose dual function has a
closed form, so a slip in a norm, a normalisation, a trigger or a clamp of
``orc_evaluate`` fails one of these tests.

Instance: products 0, 1, 2 with prices r = (4, 6, 10); resources 0, 1 with
capacities c = (3, 4), so ||c||_2 = 5; product 0 uses resource 0, product 1
resource 1, product 2 both. Three MNL segments, each considering one product:

    segment 0: product 0, v = 1, v0 = 1, lambda = 2  ->  z_0 = 2 m_0 / 2 = m_0
    segment 1: product 1, v = 1, v0 = 1, lambda = 2  ->  z_1 = m_1
    segment 2: product 2, v = 3, v0 = 1, lambda = 4  ->  z_2 = 4 * 3 m_2 / 4 = 3 m_2

(a single-product segment offers its product iff its margin is positive,
Section 3's choice probability v / (v0 + v)). At ybar = (1, 2) the margins are
m = (4 - 1, 6 - 2, 10 - 1 - 2) = (3, 4, 7), so sum_l z_l = 3 + 4 + 21 = 28,
c^T ybar = 3 + 8 = 11 and Dual(ybar) = 39.
"""
import math

import numpy as np
import pytest

from instances.gam import Instance
from oracle import Oracle, Params


def hand_instance() -> Instance:
    return Instance(
        n=3, m=2, L=3,
        r=np.array([4.0, 6.0, 10.0]), c=np.array([3.0, 4.0]),
        a_ptr=np.array([0, 1, 2, 4], np.int32), a_idx=np.array([0, 1, 0, 1], np.int32), a_val=None,
        seg_ptr=np.array([0, 1, 2, 3], np.int64), seg_prod=np.array([0, 1, 2], np.int32),
        v=np.array([1.0, 1.0, 3.0]), w=None, lam=np.array([2.0, 2.0, 4.0]), v0=np.array([1.0, 1.0, 1.0]),
        name="hand-worked")


def epoch(gbar, count=4, t=100, Pbar=35.0, anchor=1.0, mu=0.4, tau=0.5, **params):
    """An oracle run whose epoch holds `count` iterations with ybar = (1, 2),
    the given gbar and Pbar, after t iterations in all."""
    o = Oracle(hand_instance())
    run = o.run(Params(mu=mu, tau=tau, **params))
    run.y[:] = [7.0, 9.0]  # the current iterate: replaced by ybar at a restart
    run.sum_y[:] = np.array([1.0, 2.0]) * count
    run.sum_g[:] = np.asarray(gbar, np.float64) * count
    run.set_state(sum_P=Pbar * count, count=count, t=t, kkt_anchor=anchor, mu_cur=mu, tau_used=tau)
    return o, run


def test_dual_function_of_the_hand_instance():
    """The closed form above, as the oracle's dual function computes it."""
    o = Oracle(hand_instance())
    assert o.dual(np.array([1.0, 2.0])) == 39.0
    # a margin at or below zero drops its product: y = (5, 0) gives m = (-1, 6, 5)
    assert o.dual(np.array([5.0, 0.0])) == 15.0 + 0.0 + 6.0 + 15.0


def test_residuals_and_objective_pair():
    """gbar = (4, 5): both resources over by 1, pinf = sqrt(2) / 6; Pbar = 35,
    gap = |39 - 35| / (1 + 39 + 35) = 4 / 75; KKT = max = sqrt(2) / 6. No trigger
    fires (anchor 1: 0.2357 > 0.2 * 1; count 4 < 0.36 * 100), so the state stays."""
    o, run = epoch([4.0, 5.0])
    st = run.evaluate()
    assert st["dual_avg"] == 39.0 and st["primal_avg"] == 35.0
    assert st["pinf"] == pytest.approx(math.sqrt(2.0) / 6.0, rel=1e-15)
    assert st["gap"] == pytest.approx(4.0 / 75.0, rel=1e-15)
    assert st["kkt"] == st["pinf"]
    assert st["evals"] == 1 and st["restarts"] == 0 and st["converged"] == 0
    assert st["count"] == 4 and st["mu_cur"] == 0.4 and st["tau_used"] == 0.5 and st["kkt_anchor"] == 1.0
    assert list(run.y) == [7.0, 9.0] and list(run.sum_y) == [4.0, 8.0]


def test_only_overuse_counts_as_infeasibility():
    """gbar = (1, 5): resource 0 is under capacity by 2 (no contribution), resource 1
    over by 1: pinf = 1 / 6. The gap dominates when Pbar is low: Pbar = 10 gives
    gap = 29 / 50."""
    o, run = epoch([1.0, 5.0], Pbar=10.0)
    st = run.evaluate()
    assert st["pinf"] == pytest.approx(1.0 / 6.0, rel=1e-15)
    assert st["gap"] == pytest.approx(29.0 / 50.0, rel=1e-15)
    assert st["kkt"] == st["gap"]


def test_progress_restart():
    """Anchor 2: KKT = 0.2357 <= 0.2 * 2, a progress restart: y <- ybar = (1, 2), sums
    cleared, anchor <- KKT, mu halved, tau times the decay (0.5), and no balance
    factor even with b > 0 (the balance applies to epoch-length restarts only)."""
    o, run = epoch([4.0, 5.0], anchor=2.0, restart_tau_decay=0.5, restart_tau_balance=0.5)
    st = run.evaluate()
    assert st["restarts"] == 1 and st["converged"] == 0
    assert list(run.y) == [1.0, 2.0]
    assert not run.sum_y.any() and not run.sum_g.any() and st["sum_P"] == 0.0 and st["count"] == 0
    assert st["kkt_anchor"] == st["kkt"] == pytest.approx(math.sqrt(2.0) / 6.0, rel=1e-15)
    assert st["mu_cur"] == 0.2 and st["tau_used"] == 0.25


def test_epoch_length_restart_at_its_boundary():
    """count >= 0.36 t: with t = 25, 0.36 * 25 = 9 exactly. count = 8 keeps the epoch,
    count = 9 restarts it (anchor 1: KKT = 0.2357 > 0.2, no progress trigger)."""
    o, run = epoch([4.0, 5.0], count=8, t=25, restart_tau_balance=0.0)
    st = run.evaluate()
    assert st["restarts"] == 0 and st["count"] == 8
    o, run = epoch([4.0, 5.0], count=9, t=25, restart_tau_balance=0.0)
    st = run.evaluate()
    assert st["restarts"] == 1 and st["count"] == 0 and list(run.y) == [1.0, 2.0]
    assert st["mu_cur"] == 0.2 and st["tau_used"] == 0.5  # decay 1 (constant step), balance off


@pytest.mark.parametrize("gbar, factor", [
    ([4.0, 5.0], 2.0),                                     # sqrt((sqrt(2)/6) / (4/75)) = 2.10 -> upper bound 1/b
    ([3.1, 4.0], math.sqrt((0.1 / 6.0) / (4.0 / 75.0))),   # 0.559, inside [b, 1/b]
    ([3.05, 4.0], 0.5),                                    # sqrt((0.05/6) / (4/75)) = 0.395 -> lower bound b
])
def test_balance_clamp_on_epoch_length_restarts(gbar, factor):
    """An epoch-length restart with b = 0.5 scales tau by clamp(sqrt(pinf / gap), b, 1 / b)
    on top of the decay (0.8 here): tau = 0.5 * 0.8 * factor. gap = 4 / 75 in all
    three; anchor 0.1 keeps the progress trigger (KKT <= 0.02) off."""
    o, run = epoch(gbar, count=9, t=25, anchor=0.1, restart_tau_decay=0.8, restart_tau_balance=0.5)
    st = run.evaluate()
    assert st["restarts"] == 1
    assert st["tau_used"] == pytest.approx(0.5 * 0.8 * factor, rel=1e-13)


def test_balance_is_neutral_when_a_residual_is_zero():
    """gbar = (3, 4) meets the capacities exactly: pinf = 0, and the balance factor is 1."""
    o, run = epoch([3.0, 4.0], count=9, t=25, anchor=0.1, restart_tau_balance=0.5)
    st = run.evaluate()
    assert st["pinf"] == 0.0 and st["gap"] == pytest.approx(4.0 / 75.0, rel=1e-15)
    assert st["restarts"] == 1 and st["tau_used"] == 0.5


def test_convergence_stops_before_any_restart():
    """KKT <= kkt_tol: converged, and neither trigger restarts the epoch."""
    o, run = epoch([3.0, 4.0], count=9, t=25, Pbar=38.99, anchor=10.0, kkt_tol=1e-3)
    st = run.evaluate()
    # pinf = 0, gap = 0.01 / (1 + 39 + 38.99) = 1.266e-4
    assert st["gap"] == pytest.approx(0.01 / 78.99, rel=1e-9)
    assert st["converged"] == 1 and st["restarts"] == 0 and st["count"] == 9
    assert list(run.y) == [7.0, 9.0]
