"""The allocation-free entry point spfom_sales_noalloc, through the C ABI.

It is meant for callers that cannot allocate device memory (code inside a
memory pool it does not own, or a host that must not allocate after start-up),
so the tests hand it device buffers made beforehand. They compare two calls in
a row against the solver's own segment pass at the same margins (the sales
summed per product and the sum of the segment values after one iteration from
y = 0), and against the FP64 oracle's sweep at seeded duals; they also cover a
stated max_set_size that is not a power of two, one that understates a set
(every output NaN), and empty instances. This file is collected last so that a
failure here leaves every other test already run; it also passes on its own in
a fresh process.
"""
import math

import numpy as np
import pytest

from instances import make_instance, mid_gam, seeded_duals

pytestmark = pytest.mark.gpu

VALUE_RTOL = 1e-12  # per-value tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _device(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _call(torch, inst, marg, max_set_size, sales, z):
    from paper_2602_22421_gb300.spfom import sales_noalloc
    d = {k: _device(torch, getattr(inst, k)) for k in ("seg_ptr", "seg_prod", "v", "lam", "v0")}
    dw = _device(torch, inst.w) if inst.w is not None else None
    dm = _device(torch, marg)
    stream = torch.cuda.current_stream().cuda_stream
    rc = sales_noalloc(inst.n, inst.L, max_set_size, d["seg_ptr"].data_ptr(), d["seg_prod"].data_ptr(),
                       d["v"].data_ptr(), None if dw is None else dw.data_ptr(), d["lam"].data_ptr(),
                       d["v0"].data_ptr(), dm.data_ptr(), sales.data_ptr(), z.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc


def _buffers(torch, n):
    return (torch.full((max(n, 1),), -1.0, dtype=torch.float64, device="cuda"),
            torch.full((1,), -1.0, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("make", [lambda: mid_gam(1, L=20_001, n=1000, m=200),
                                  lambda: make_instance(n=40, m=6, L=3000, kmin=0, kmax=32, gam=False, seed=4)],
                         ids=["gam", "mnl_max32"])
def test_noalloc_sales_match_the_solver_on_two_calls(make):
    torch = pytest.importorskip("torch")
    from paper_2602_22421_gb300 import VEC_MARGINS, VEC_S, Solver
    inst = make()
    with Solver(inst, device=0, eval_every=0) as s:
        st = s.step(1)
        want_sales, want_z, marg = s.vector(VEC_S), st["z_sum"], s.vector(VEC_MARGINS)
    kmax = int(np.diff(inst.seg_ptr).max())
    sales, z = _buffers(torch, inst.n)
    for call in range(2):
        assert _call(torch, inst, marg, kmax, sales, z) == 0, f"call {call}"
        got = sales.cpu().numpy()
        np.testing.assert_allclose(got, want_sales, rtol=VALUE_RTOL, atol=VALUE_RTOL * np.abs(want_sales).max())
        assert z.item() == pytest.approx(want_z, rel=VALUE_RTOL)


@pytest.mark.parametrize("slack", [0, 3], ids=["exact_max", "max_plus_3"])
def test_noalloc_sales_match_the_oracle_sweep(slack):
    """Sales and sum of z at seeded duals against Oracle.sweep (the oracle forms
    the margins too); max_set_size = the largest set (13, rounded up to 16
    lanes inside) or that plus 3 (16: the same lanes, another stated bound)."""
    torch = pytest.importorskip("torch")
    from oracle import Oracle
    inst = make_instance(n=300, m=60, L=5001, kmin=5, kmax=13, gam=True, tightness=0.6, seed=11)
    o = Oracle(inst)
    y = seeded_duals(inst.m, 21, float(np.mean(inst.r)) / 3.0)
    ref = o.sweep(y)
    marg = o.margins(y)
    kmax = int(np.diff(inst.seg_ptr).max())
    sales, z = _buffers(torch, inst.n)
    for call in range(2):
        assert _call(torch, inst, marg, kmax + slack, sales, z) == 0, f"call {call}"
        got = sales.cpu().numpy()
        np.testing.assert_allclose(got, ref["s"], rtol=VALUE_RTOL, atol=VALUE_RTOL * np.abs(ref["s"]).max())
        assert z.item() == pytest.approx(ref["zsum"], rel=VALUE_RTOL)


def test_noalloc_understated_max_set_size_gives_nan_then_recovers():
    """A stated bound of 5 with sets of up to 7 products: those segments are not
    solved and every output is NaN (not 5 rounded up to 8 lanes). The next call
    with the true bound clears the flag and matches the oracle."""
    torch = pytest.importorskip("torch")
    from oracle import Oracle
    inst = make_instance(n=50, m=10, L=700, kmin=3, kmax=7, gam=True, tightness=0.6, seed=12)
    assert int(np.diff(inst.seg_ptr).max()) == 7
    o = Oracle(inst)
    y = seeded_duals(inst.m, 22, float(np.mean(inst.r)) / 3.0)
    ref, marg = o.sweep(y), o.margins(y)
    sales, z = _buffers(torch, inst.n)
    assert _call(torch, inst, marg, 5, sales, z) == 0
    assert np.isnan(sales.cpu().numpy()).all() and math.isnan(z.item())
    assert _call(torch, inst, marg, 7, sales, z) == 0
    np.testing.assert_allclose(sales.cpu().numpy(), ref["s"], rtol=VALUE_RTOL,
                               atol=VALUE_RTOL * np.abs(ref["s"]).max())
    assert z.item() == pytest.approx(ref["zsum"], rel=VALUE_RTOL)


def test_noalloc_empty_instances():
    """L = 0: zero sales and z = 0. n = 0 with empty segments: z = 0 and NULL
    margins / sales / ids / attractions are accepted (max_set_size 0)."""
    torch = pytest.importorskip("torch")
    from paper_2602_22421_gb300.spfom import sales_noalloc
    stream = torch.cuda.current_stream().cuda_stream
    ptr0 = _device(torch, np.zeros(1, np.int64))
    marg = torch.ones(4, dtype=torch.float64, device="cuda")
    sales, z = _buffers(torch, 4)
    rc = sales_noalloc(4, 0, 3, ptr0.data_ptr(), None, None, None, None, None, marg.data_ptr(), sales.data_ptr(),
                       z.data_ptr(), stream)
    torch.cuda.synchronize()
    assert rc == 0 and not sales.cpu().numpy().any() and z.item() == 0.0
    ptr3 = _device(torch, np.zeros(4, np.int64))
    lam = torch.ones(3, dtype=torch.float64, device="cuda")
    rc = sales_noalloc(0, 3, 0, ptr3.data_ptr(), None, None, None, lam.data_ptr(), lam.data_ptr(), None, None,
                       z.data_ptr(), stream)
    torch.cuda.synchronize()
    assert rc == 0 and z.item() == 0.0


def test_noalloc_rejects_sizes_beyond_its_limits():
    torch = pytest.importorskip("torch")
    from paper_2602_22421_gb300.spfom import NOALLOC_MAX_PRODUCTS, sales_noalloc
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    assert sales_noalloc(NOALLOC_MAX_PRODUCTS + 1, 1, 1, p, p, p, None, p, p, p, p, p) == 1
    assert sales_noalloc(10, 1, 33, p, p, p, None, p, p, p, p, p) == 1
    assert sales_noalloc(10, 1, 4, p, None, p, None, p, p, p, p, p) == 1  # ids missing with sets allowed
