"""The allocation-free entry point spfom_sales_noalloc, through the C ABI.

It is meant for callers that cannot allocate device memory (code inside a
memory pool it does not own, or a host that must not allocate after start-up),
so the test hands it device buffers made beforehand and compares two calls in
a row against the solver's own segment pass at the same margins: the sales
summed per product and the sum of the segment values after one iteration from
y = 0. This file is collected last so that a failure here leaves every other
test already run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from instances import make_instance, mid_gam

pytestmark = pytest.mark.gpu

VALUE_RTOL = 1e-12  # per-value tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _device(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("make", [lambda: mid_gam(1, L=20_001, n=1000, m=200),
                                  lambda: make_instance(n=40, m=6, L=3000, kmin=0, kmax=32, gam=False, seed=4)],
                         ids=["gam", "mnl_max32"])
def test_noalloc_sales_match_the_solver_on_two_calls(make):
    torch = pytest.importorskip("torch")
    from paper_2602_22421_gb300 import VEC_MARGINS, VEC_S, Solver
    from paper_2602_22421_gb300.spfom import sales_noalloc
    inst = make()
    with Solver(inst, device=0, eval_every=0) as s:
        st = s.step(1)
        want_sales, want_z, marg = s.vector(VEC_S), st["z_sum"], s.vector(VEC_MARGINS)
    kmax = int(np.diff(inst.seg_ptr).max())
    d = {k: _device(torch, getattr(inst, k)) for k in ("seg_ptr", "seg_prod", "v", "lam", "v0")}
    dw = _device(torch, inst.w) if inst.w is not None else None
    dm = _device(torch, marg)
    sales = torch.full((inst.n,), -1.0, dtype=torch.float64, device="cuda")
    z = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        rc = sales_noalloc(inst.n, inst.L, kmax, d["seg_ptr"].data_ptr(), d["seg_prod"].data_ptr(),
                           d["v"].data_ptr(), None if dw is None else dw.data_ptr(), d["lam"].data_ptr(),
                           d["v0"].data_ptr(), dm.data_ptr(), sales.data_ptr(), z.data_ptr(), stream)
        assert rc == 0, f"call {call}: status {rc}"
        torch.cuda.synchronize()
        got = sales.cpu().numpy()
        np.testing.assert_allclose(got, want_sales, rtol=VALUE_RTOL, atol=VALUE_RTOL * np.abs(want_sales).max())
        assert z.item() == pytest.approx(want_z, rel=VALUE_RTOL)


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    from paper_2602_22421_gb300.spfom import NOALLOC_MAX_PRODUCTS, sales_noalloc
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    assert sales_noalloc(NOALLOC_MAX_PRODUCTS + 1, 1, 1, p, p, p, None, p, p, p, p, p) == 1
    assert sales_noalloc(10, 1, 33, p, p, p, None, p, p, p, p, p) == 1
