"""The warm-start network's tensor-core kernels and features against the CPU
oracle (oracle/mlp_oracle.py), through the C ABI (needs a GPU).

Tolerances. The kernels round inputs, weights, hidden activations and output
gradients to BF16 exactly where the oracle (rounding=True) does; what remains
is FP32 accumulation (K <= 256: about 256 * 2^-24 = 1.5e-5 relative) against
binary64, which moves a value across a BF16 rounding boundary for roughly
1.5e-5 / 2^-8 = 0.4% of the rounded elements, each such flip changing that
element by one BF16 unit (2^-8 relative). Normwise that is below
sqrt(0.004) * 2^-8 = 2.5e-4 per rounding stage; with up to five stages
compounding, outputs are held to 2e-3 and gradients to 5e-3 of their norm.
"""
import numpy as np
import pytest

from instances import mid_gam
from oracle import Oracle
from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu

OUT_RTOL = 2e-3
GRAD_RTOL = 5e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def tensors(X, t=None):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    return x if t is None else (x, torch.from_numpy(np.ascontiguousarray(t, np.float32)).cuda())


def nrel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def case(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, M.F)).astype(np.float32)
    X[:, 11] = 1.0
    t = rng.uniform(0.0, 2.0, rows).astype(np.float32)
    p = M.glorot(seed).astype(np.float32)
    return X, t, p


@pytest.mark.parametrize("rows", [1, 40, 300, 4099])
def test_forward_matches_oracle(rows):
    from paper_2602_22421_gb300 import MLP
    X, _, p = case(rows, 10 + rows)
    with MLP(0) as net:
        net.params = p
        np.testing.assert_array_equal(net.params, p)
        got = net.forward(tensors(X)).cpu().numpy()
    want, _ = M.forward(p.astype(np.float64), X.astype(np.float64), rounding=True)
    assert nrel(got, want) <= OUT_RTOL
    assert np.abs(got - want).max() <= 1e-2 * np.abs(want).max()


def _rounding_spread(q, dq, may_zero=None):
    """Largest |bf16(q') - bf16(q)| over q' in [q - dq, q + dq] (and q' = 0
    where may_zero): BF16 rounding is monotone, so the ends decide. An element
    whose interval holds no rounding boundary gets 0: both sides then round to
    the same BF16 value."""
    Q = M.bf16(q)
    lo, hi = q - dq, q + dq
    if may_zero is not None:
        lo = np.where(may_zero, np.minimum(lo, 0.0), lo)
        hi = np.where(may_zero, np.maximum(hi, 0.0), hi)
    return np.maximum(np.abs(M.bf16(hi) - Q), np.abs(M.bf16(lo) - Q))


def gradient_error_bounds(p, X, t):
    """Per-element bound on |GPU gradient - rounded-oracle gradient|, carried
    through the network to first order from the oracle's own intermediates.

    Both sides round the same operands to BF16 (so Xb, W1b, W2b, w3b agree);
    they differ by FP32 accumulation (at most K 2^-24 of the absolute sum of a
    length-K product) and where that difference carries a value across a BF16
    rounding boundary (_rounding_spread: 0 for the elements whose error
    interval holds no boundary, one BF16 unit or more for the rest). A ReLU
    whose pre-activation lies within its error bound of zero may switch its
    backward mask; that element's interval then reaches 0. Each gradient
    element is a sum over rows, and its bound is the sum of the bounds of its
    terms, so a cancelling sum keeps the bound of its terms and a few wrong
    elements inside a large block fail on their own."""
    W1, b1, W2, b2, w3, b3 = M.unpack(p)
    o, (Xb, W1b, W2b, w3b, h1, h2) = M.forward(p, X, rounding=True)
    R = len(o)
    g = lambda k: 1.01 * k * 2.0 ** -24
    aX, aW1, aW2, aw3 = np.abs(Xb), np.abs(W1b), np.abs(W2b), np.abs(w3b)
    z1 = Xb @ W1b.T + b1
    z2 = h1 @ W2b.T + b2
    dz1 = g(M.F + 1) * (aX @ aW1.T + np.abs(b1))
    dh1 = _rounding_spread(np.maximum(z1, 0.0), dz1)
    dz2 = dh1 @ aW2.T + g(M.H + 1) * (h1 @ aW2.T + np.abs(b2))
    dh2 = _rounding_spread(np.maximum(z2, 0.0), dz2)
    do = dh2 @ aw3 + g(M.H + 1) * (h2 @ aw3 + abs(b3))
    e = o - np.asarray(t, np.float64)
    q = 2.0 * e / R
    dO = M.bf16(q)
    ddO = _rounding_spread(q, 2.0 / R * do + 2.0 ** -23 * np.abs(q))
    aO = np.abs(dO)
    gw3 = dh2.T @ aO + h2.T @ ddO + g(R) * (h2.T @ aO)
    gb3 = ddO.sum() + g(R) * aO.sum()
    m2 = h2 > 0
    flip2 = np.abs(z2) <= dz2
    q2 = np.outer(dO, w3b) * m2
    dH2 = M.bf16(q2)
    aH2 = np.abs(dH2)
    ddH2 = _rounding_spread(q2, np.outer(ddO, aw3) * (m2 | flip2), may_zero=flip2)
    ddH2 = np.maximum(ddH2, np.outer(aO + ddO, aw3) * flip2)  # the mask may also switch on
    gW2 = ddH2.T @ h1 + aH2.T @ dh1 + g(R) * (aH2.T @ h1)
    gb2 = ddH2.sum(axis=0) + g(R) * aH2.sum(axis=0)
    m1 = h1 > 0
    flip1 = np.abs(z1) <= dz1
    pre = aH2 @ aW2
    q1 = (dH2 @ W2b) * m1
    dH1 = M.bf16(q1)
    aH1 = np.abs(dH1)
    ddH1 = _rounding_spread(q1, (ddH2 @ aW2 + g(M.H) * pre) * (m1 | flip1), may_zero=flip1)
    ddH1 = np.maximum(ddH1, (pre + ddH2 @ aW2) * flip1)
    gW1 = ddH1.T @ aX + g(R) * (aH1.T @ aX)
    gb1 = ddH1.sum(axis=0) + g(R) * aH1.sum(axis=0)
    return M.pack(gW1, gb1, gW2, gb2, gw3, gb3)


@pytest.mark.parametrize("rows", [40, 300, 2500])
def test_gradients_match_oracle(rows):
    """Every gradient element within twice its first-order error bound
    (gradient_error_bounds), and every parameter block within GRAD_RTOL of its
    norm."""
    from paper_2602_22421_gb300 import MLP
    X, t, p = case(rows, 20 + rows)
    with MLP(0) as net:
        net.params = p
        loss = net.loss_grad(*tensors(X, t))
        g = net.grads()
    L, gw = M.loss_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64), rounding=True)
    bound = gradient_error_bounds(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(L, rel=OUT_RTOL)
    blocks = {"W1": (0, M.H * M.F), "b1": (M.H * M.F, M.H), "W2": (M.H * M.F + M.H, M.H * M.H),
              "b2": (M.H * M.F + M.H + M.H * M.H, M.H), "w3": (M.PARAMS - M.H - 1, M.H), "b3": (M.PARAMS - 1, 1)}
    for name, (o, k) in blocks.items():
        err = np.abs(g[o:o + k].astype(np.float64) - gw[o:o + k])
        worst = int(np.argmax(err / (2.0 * bound[o:o + k] + 1e-30)))
        assert np.all(err <= 2.0 * bound[o:o + k] + 1e-30), \
            (name, worst, float(err[worst]), float(bound[o + worst]), float(gw[o + worst]))
        assert nrel(g[o:o + k], gw[o:o + k]) <= GRAD_RTOL, name


def test_adam_training_fits_a_smooth_target():
    """Training on the GPU by the network's own forward, backward and Adam
    kernels brings the loss of a smooth regression target down by 20x."""
    from paper_2602_22421_gb300 import MLP
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (8192, M.F)).astype(np.float32)
    t = (np.maximum(X[:, 0] + 0.5 * X[:, 1], 0) + 0.3 * X[:, 2] ** 2).astype(np.float32)
    x, tt = tensors(X, t)
    with MLP(0, seed=1) as net:
        first = net.loss_grad(x, tt)
        for _ in range(300):
            last = net.train_step(x, tt, 2e-3)
        p = net.params
    assert last <= first / 20
    # the trained parameters evaluate to the same loss on the oracle
    assert M.loss(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64)) == pytest.approx(
        net_loss_after(p, X, t), rel=2e-2)


def net_loss_after(p, X, t):
    from paper_2602_22421_gb300 import MLP
    with MLP(0) as net:
        net.params = p
        o = net.forward(tensors(X)).cpu().numpy().astype(np.float64)
    return float(np.mean((o - t) ** 2))


@pytest.mark.parametrize("inst", [mid_gam(3, L=3000, n=200, m=40), mid_gam(4, L=20_001, n=1500, m=300, kmin=10,
                                                                           kmax=30, tightness=0.4)],
                         ids=["small", "c5_like"])
def test_features_match_oracle(inst):
    from paper_2602_22421_gb300 import Solver
    s0 = Oracle(inst).sweep(np.zeros(inst.m))["s"]
    want = M.features(inst, s0)
    with Solver(inst, device=0) as s:
        got = s.features().cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6)


def test_warm_start_rejects_a_prediction_worse_than_zero():
    """Huge predicted prices have a worse dual objective than y = 0: the solve
    starts cold and matches the plain cold solve iteration for iteration."""
    from paper_2602_22421_gb300 import MLP, Solver
    inst = mid_gam(5, L=5000, n=300, m=60)
    p = np.zeros(M.PARAMS, np.float32)
    p[-1] = 1e3  # o = 1000 for every resource: y0 = 1000 mean(r)
    with Solver(inst, device=0) as s, MLP(0) as net:
        net.params = p
        cold = s.solve()
        warm, mode = s.solve_warm(net)
    assert mode == 0
    assert warm["converged"] == 1 and warm["iters"] == cold["iters"]
    assert warm["dual_avg"] == cold["dual_avg"]


def test_warm_start_near_the_optimum_and_the_budget_fallback():
    """Started from the optimal duals y* the solve converges in fewer
    iterations than from y = 0; spfom_solve_warm given a prediction it accepts
    but a 1-iteration budget falls back to the cold start."""
    from paper_2602_22421_gb300 import MLP, Solver
    inst = mid_gam(6, L=8000, n=400, m=80)
    with Solver(inst, device=0) as s:
        cold = s.solve()
        ystar = s.duals(averaged=True)
        hot = s.solve(ystar)
        assert hot["converged"] == 1 and hot["iters"] < cold["iters"]
        # a constant prediction equal to the mean optimal price: accepted when it
        # improves on y = 0; with a 1-iteration budget it cannot converge and falls back
        p = np.zeros(M.PARAMS, np.float32)
        p[-1] = float(np.mean(ystar) / np.mean(inst.r))
        with MLP(0) as net:
            net.params = p
            st, mode = s.solve_warm(net, warm_iters=1)
    assert st["converged"] == 1
    if mode != 0:
        assert mode == 2 and st["iters"] == cold["iters"]
