"""Pins of the warm-start oracle (oracle/mlp_oracle.py) against mathematics
that does not come from the oracle itself: BF16 rounding against torch's
conversion and hand-listed values, the gradient against central finite
differences, the forward pass against a network built to compute a closed
form, and the features against values worked out by hand on a 3-product
instance. CPU only.
"""
import math

import numpy as np
import pytest

from instances.gam import Instance
from oracle import Oracle
from oracle import mlp_oracle as M


def test_bf16_rounding_matches_hand_values_and_torch():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even significand
    vals = [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, 1 + 3 * 2 ** -9, -2.5, 0.0, 2 ** -130, 3.0e38]
    want = [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, 1 + 2 ** -7, -2.5, 0.0, 2 ** -130, None]
    got = M.bf16(vals)
    for g, w in zip(got, want):
        if w is not None:
            assert g == w
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).standard_normal(20000) * np.exp(np.random.default_rng(1).uniform(-20, 20, 20000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(x), ref)


def test_forward_of_a_network_built_for_a_closed_form():
    """W1 copies the 16 inputs into the first 16 units (ReLU keeps the positive
    parts), W2 sums them into unit 0, w3 reads unit 0: o = sum_k max(x_k, 0) + 1.5."""
    W1 = np.zeros((M.H, M.F))
    W1[np.arange(M.F), np.arange(M.F)] = 1.0
    W2 = np.zeros((M.H, M.H))
    W2[0, :M.F] = 1.0
    w3 = np.zeros(M.H)
    w3[0] = 1.0
    p = M.pack(W1, np.zeros(M.H), W2, np.zeros(M.H), w3, 1.5)
    X = np.random.default_rng(2).standard_normal((50, M.F))
    o, _ = M.forward(p, X, rounding=False)
    np.testing.assert_allclose(o, np.maximum(X, 0).sum(axis=1) + 1.5, rtol=1e-14)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    p = M.glorot(4)
    X = rng.standard_normal((20, M.F))
    t = rng.standard_normal(20)
    L, g = M.loss_grad(p, X, t, rounding=False)
    assert L == pytest.approx(M.loss(p, X, t, rounding=False), rel=1e-14)
    # coordinates from every parameter block: W1, b1, W2, b2, w3, b3
    offs = [0, M.H * M.F, M.H * M.F + M.H, M.H * M.F + M.H + M.H * M.H, M.PARAMS - M.H - 1, M.PARAMS - 1]
    sizes = [M.H * M.F, M.H, M.H * M.H, M.H, M.H, 1]
    idx = [o + int(rng.integers(s)) for o, s in zip(offs, sizes) for _ in range(6)]
    for k in idx:
        h = 1e-6 * (1.0 + abs(p[k]))
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (M.loss(pp, X, t, rounding=False) - M.loss(pm, X, t, rounding=False)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9), k


def test_rounded_gradient_stays_close_to_the_exact_one():
    """A sanity bound, not a parity tolerance: five BF16 rounding stages (unit
    roundoff 2^-9 each) with cancellation in the 256-term sums move the
    gradient by a few percent at most."""
    rng = np.random.default_rng(5)
    p = M.glorot(6)
    X = rng.standard_normal((300, M.F))
    t = rng.standard_normal(300)
    _, ge = M.loss_grad(p, X, t, rounding=False)
    _, gr = M.loss_grad(p, X, t, rounding=True)
    assert np.linalg.norm(gr - ge) <= 6e-2 * np.linalg.norm(ge)


def hand_instance(c=(0.5, 0.5)):
    """One MNL segment (lambda = 1, v0 = 1) over 3 products with v = 1 and prices
    10, 20, 30; product 0 uses resource 0, product 1 both, product 2 resource 1."""
    return Instance(n=3, m=2, L=1, r=np.array([10.0, 20.0, 30.0]), c=np.array(c, dtype=float),
                    a_ptr=np.array([0, 1, 3, 4], np.int32), a_idx=np.array([0, 0, 1, 1], np.int32), a_val=None,
                    seg_ptr=np.array([0, 3], np.int64), seg_prod=np.array([0, 1, 2], np.int32),
                    v=np.ones(3), w=None, lam=np.array([1.0]), v0=np.array([1.0]), name="hand")


def test_features_of_a_hand_worked_instance():
    inst = hand_instance()
    # at y = 0 the best assortment is {1, 2}: value (20 + 30) / (1 + 2) beats 30 / 2 and 60 / 4
    s0 = Oracle(inst).sweep(np.zeros(2))["s"]
    np.testing.assert_allclose(s0, [0.0, 1 / 3, 1 / 3], rtol=1e-15)
    f = M.features(inst, s0)
    want0 = [1.0, 2 / 3, 1.5, math.log(2 / 3), 1.0, 1.0, 0.0, 0.5, 1.0, 1.0, 4 / 3, 1.0, 0.0, 0, 0, 0]
    want1 = [1.0, 4 / 3, 0.75, math.log(4 / 3), 1.25, 1.5, 0.25, 1.0, 1.0, 1.0, 4 / 3, 1.0, 1.0, 0, 0, 0]
    np.testing.assert_allclose(f[0], want0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(f[1], want1, rtol=1e-12, atol=1e-12)


def test_features_are_invariant_to_the_units_of_price_and_capacity():
    from instances import mid_gam
    inst = mid_gam(2, L=400, n=60, m=12)
    s0 = Oracle(inst).sweep(np.zeros(inst.m))["s"]
    f = M.features(inst, s0)
    scaled = mid_gam(2, L=400, n=60, m=12)
    scaled.r = scaled.r * 7.0   # prices in other units: same best assortments, same sales
    scaled.c = scaled.c * 3.0   # capacities in other units, with the arrivals scaled alike
    scaled.lam = scaled.lam * 3.0
    s1 = Oracle(scaled).sweep(np.zeros(inst.m))["s"]
    np.testing.assert_allclose(s1, 3.0 * s0, rtol=1e-12)
    np.testing.assert_allclose(M.features(scaled, s1), f, rtol=1e-9, atol=1e-12)
