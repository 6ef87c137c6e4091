"""Batched multi-period re-solves (paper_2602_22421_gb300.periods) against
one-at-a-time plain solves of the same problems (needs a GPU).

Every (period, instance) problem of the batched binary32 run, warm-started
from the previous period's bid prices, must reach KKT <= 1e-4 and the dual
objective the plain binary64 method reaches from y = 0 on the same capacities
and rates. Two points with KKT <= 1e-4 each lie within about 1e-4 of the
optimum, so their objectives are compared at 3e-4 relative.
"""
import numpy as np
import pytest

from instances import batch_base, period_rates

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def small_family(count=6):
    out = []
    for k in range(count):
        inst = batch_base(11, k)
        if inst.L > 20_000:  # keep the test quick: same distributions, fewer segments
            from instances import make_instance
            rng = np.random.default_rng([11, k, 1])
            inst = make_instance(n=inst.n, m=inst.m, L=int(rng.integers(1000, 20_000)), kmin=3, kmax=20,
                                 tightness=0.6, seed=int(rng.integers(1 << 40)))
        out.append(inst)
    return out


@pytest.mark.parametrize("precision", [32, 64])
def test_batched_periods_match_sequential_plain_solves(precision):
    from paper_2602_22421_gb300 import periods as PR
    insts = small_family()
    rho = period_rates(11, len(insts), 3)
    summary, path, per = PR.run_batched(insts, rho, periods=3, precision=precision, restart_tau_balance=0.5)
    # batches: binary32 tilings without staging or the slot-major copy; binary64: 1 or 2 (shared margins)
    choices = (1, 3, 5, 6, 7) if precision == 32 else (1, 2)
    assert summary["autotune_choice"] in choices
    assert all(r["converged"] == 1 for r in summary["records"])
    for c_k, lam_k in path:
        assert all((c >= 0).all() for c in c_k)
    # the inventory only decreases: a period's capacity times the periods left never exceeds the last one's
    left = [sum(float(c.sum()) for c in c_k) * (3 - k) for k, (c_k, _) in enumerate(path)]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(left, left[1:]))
    seq = PR.run_sequential(insts, path, restart_tau_balance=0.5)
    for r in seq:
        b, k = r["instance"], r["period"]
        st = per[k][b]
        assert r["converged"] == 1 and st["converged"] == 1 and st["kkt"] <= 1e-4
        assert st["dual_avg"] == pytest.approx(r["dual"], rel=3e-4), (b, k)
