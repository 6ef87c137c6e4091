"""What the learned warm start gains (needs a GPU): a network trained by the
library's own kernels on the method's own solves of a small family of
instances starts held-out instances of that family closer to their optimum,
so the method reaches KKT <= 1e-4 in fewer iterations, at the same objective.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_trained_network_reduces_iterations_on_held_out_instances():
    """192 training instances of the warm-start family at 1e4..3e4 segments
    (the full evaluation uses 10^4; see the warm-start profile)."""
    from paper_2602_22421_gb300 import warmstart as W
    X, T, info = W.build_dataset(192, seed=W.TRAIN_SEED, chunk=64, L_lo=1e4, L_hi=3e4, workers=8, log=None)
    assert info["unconverged"] == 0 and X.shape == (192 * 400, 16)
    net = W.train(X, T, epochs=40, lr=1e-3, log=None)
    test = W.instances(W.TEST_SEED, range(12), L_lo=1e4, L_hi=3e4)
    recs = W.evaluate(net, test)
    s = W.summarize(recs)
    assert s["all_converged"] and s["max_kkt"] <= 1e-4
    assert s["max_objective_rel_diff"] <= 1e-4
    assert s["mode_counts"]["1"] >= 10  # the prediction is accepted and converges
    assert s["warm_mean_iters"] < 0.9 * s["cold_mean_iters"]
    net.close()
