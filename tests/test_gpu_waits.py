"""Bounded device waits that run out (needs a GPU).

Every wait on an mbarrier in the library's own kernels polls a bounded number
of times and then records an error that the host returns as SPFOM_ETIMEOUT;
nothing spins without a limit, and a block that gives up still lets the bulk
copies and tensor-core operations it issued finish before it leaves. These
tests set the limit to 0 polls (spfom_set_wait_limit,
spfom_mlp_set_wait_limit), so the first wait gives up at once, and check the
status, then that a fresh solver or network computes correct results on the
same device afterwards.
"""
import numpy as np
import pytest

from instances import mid_gam
from oracle import Oracle
from oracle import Params as OracleParams
from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_staged_segment_wait_gives_up_with_etimeout():
    from paper_2602_22421_gb300 import Solver
    from paper_2602_22421_gb300.spfom import ETIMEOUT, SpfomError
    inst = mid_gam(1, L=20_001, n=1000, m=200)
    with Solver(inst, device=0, precision=32, tiling=2) as s:
        s.set_wait_limit(0)
        with pytest.raises(SpfomError) as e:
            s.step(1)
        assert e.value.status == ETIMEOUT
    # a fresh solver on the same device: one binary32 iteration agrees with the FP64 oracle
    run = Oracle(inst).run(OracleParams())
    run.step(1)
    with Solver(inst, device=0, precision=32, tiling=2) as s:
        st = s.step(1)
        y = s.duals()
    assert st["iters"] == 1
    assert float(np.abs(y - run.y).max()) <= 1e-5 * max(1.0, float(np.abs(run.y).max()))


def test_tensor_core_product_wait_gives_up_with_etimeout():
    import torch
    from paper_2602_22421_gb300 import MLP
    from paper_2602_22421_gb300.spfom import ETIMEOUT, SpfomError
    rng = np.random.default_rng(3)
    X = rng.standard_normal((300, M.F)).astype(np.float32)
    p = M.glorot(3).astype(np.float32)
    x = torch.from_numpy(X).cuda()
    with MLP(0) as net:
        net.params = p
        net.set_wait_limit(0)
        with pytest.raises(SpfomError) as e:
            net.forward(x)
        assert e.value.status == ETIMEOUT
    with MLP(0) as net:
        net.params = p
        got = net.forward(x).cpu().numpy()
    want, _ = M.forward(p.astype(np.float64), X.astype(np.float64), rounding=True)
    assert float(np.linalg.norm(got - want) / np.linalg.norm(want)) <= 2e-3
