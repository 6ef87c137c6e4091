"""Assortment recovery (spfom_recover) and the primal average x-bar
(spfom_xbar) against the oracle (needs a GPU). The recovery is per segment
and elementwise, so the values agree to 1e-12 (the prefix sums of D and of the
balance row run in a different order on the two sides)."""
import numpy as np
import pytest

from instances import make_instance, mid_gam
from oracle import Oracle, Params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def mixed(inst, seed):
    """SBLP-feasible sales: per segment a random convex combination of three
    assortment points (closed-form GAM sales)."""
    rng = np.random.default_rng(seed)
    w = inst.w if inst.w is not None else np.zeros(inst.nnz)
    x = np.zeros(inst.nnz)
    for l in range(inst.L):
        b, e = inst.seg_ptr[l], inst.seg_ptr[l + 1]
        for q, a in enumerate(rng.dirichlet(np.ones(3))):
            S = rng.random(e - b) < 0.5
            den = inst.v0[l] + inst.v[b:e][S].sum() + w[b:e][~S].sum()
            x[b:e] += a * np.where(S, inst.lam[l] * inst.v[b:e] / den, 0.0)
    return x


@pytest.mark.parametrize("inst", [make_instance(n=60, m=10, L=3001, kmin=0, kmax=32, gam=True, seed=31),
                                  mid_gam(32, L=4000, n=300, m=60)], ids=["ragged_k0_32", "mid"])
def test_recover_matches_oracle(inst):
    from paper_2602_22421_gb300 import Solver
    x = mixed(inst, 33)
    # ties: give some segments equal u values
    x[:64] = np.round(x[:64], 2)
    want_a, want_o = Oracle(inst).recover(x)
    with Solver(inst, device=0) as s:
        a, o = s.recover(x)
    np.testing.assert_allclose(a, want_a, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(o, want_o)


def test_xbar_tracks_the_oracle_and_recovers():
    from paper_2602_22421_gb300 import Solver
    inst = mid_gam(34, L=6000, n=300, m=60)
    run = Oracle(inst).run(Params(), track_x=True)
    with Solver(inst, device=0, track_xbar=1) as s:
        for t in (1, 63, 65, 130, 200):  # not right after an evaluation: a restart empties the epoch
            s.step(t - run.stats()["t"])
            run.step(t - run.stats()["t"])
            xb = s.xbar()
            ref = run.xbar
            scale = np.abs(ref).max()
            assert np.abs(xb - ref).max() <= 1e-6 * scale, t
        a, o = s.recover()
    want_a, want_o = Oracle(inst).recover(run.xbar)
    np.testing.assert_allclose(a, want_a, atol=1e-6)
    assert a.min() >= -1e-9


def test_xbar_needs_tracking():
    from paper_2602_22421_gb300 import Solver, SpfomError
    inst = mid_gam(35, L=500, n=50, m=10)
    with Solver(inst, device=0) as s:
        s.step(3)
        with pytest.raises(SpfomError):
            s.xbar()
    with pytest.raises(SpfomError):
        Solver(inst, device=0, track_xbar=1, precision=32)
