"""Seeded GAM choice-based LP instances.

Notation (products j, resources i, segments l) follows the sales-based LP of
Section 3.2 with the capacity row of Extension 2 (Section 5.2, eq. new_NRM_1):

* ``r[n]``            price of product j
* ``c[m]``            capacity of resource i
* ``A``               resource-by-product incidence, stored product-major:
                      product j uses resources ``a_idx[a_ptr[j]:a_ptr[j+1]]``
                      with coefficients ``a_val`` (``None`` = all ones)
* ``seg_ptr[L+1]``    CSR offsets of the segments' consideration sets
* ``seg_prod[nnz]``   product ids of each consideration set, ascending, distinct
* ``v[nnz]``          nominal attraction v_lj
* ``w[nnz]``          shadow attraction w_lj of the generalized attraction model
                      (Section 3, choice probability pi'); ``None`` = MNL (w = 0)
* ``lam[L]``          arrival rate lambda_l
* ``v0[L]``           no-purchase attraction v_l0

Only random draws and the instance arrays live here. Capacities are set from
the expected consumption when every product of each consideration set is
offered (``full_offer_demand``): the choice probability of Section 3 evaluated
at S = C_l, which needs no optimisation.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

_CHUNK = 1 << 20  # segments drawn per chunk; part of the recipe (fixes the RNG stream)


@dataclass
class Instance:
    n: int
    m: int
    L: int
    r: np.ndarray
    c: np.ndarray
    a_ptr: np.ndarray
    a_idx: np.ndarray
    a_val: Optional[np.ndarray]
    seg_ptr: np.ndarray
    seg_prod: np.ndarray
    v: np.ndarray
    w: Optional[np.ndarray]
    lam: np.ndarray
    v0: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.seg_ptr[-1])

    @property
    def nnzA(self) -> int:
        return int(self.a_ptr[-1])

    def nbytes(self) -> int:
        tot = 0
        for f in ("r", "c", "a_ptr", "a_idx", "a_val", "seg_ptr", "seg_prod", "v", "w", "lam", "v0"):
            a = getattr(self, f)
            if a is not None:
                tot += a.nbytes
        return tot

    def with_capacity(self, c: np.ndarray, name: str = "") -> "Instance":
        out = Instance(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        out.c = np.ascontiguousarray(c, dtype=np.float64)
        if name:
            out.name = name
        return out

    def segment(self, l: int):
        """(product ids, v, w) of segment l (w is zeros for MNL)."""
        b, e = int(self.seg_ptr[l]), int(self.seg_ptr[l + 1])
        w = self.w[b:e] if self.w is not None else np.zeros(e - b)
        return self.seg_prod[b:e], self.v[b:e], w


def _distinct_sorted(rng: np.random.Generator, n: int, K: np.ndarray) -> np.ndarray:
    """For each row l draw K[l] distinct uniform ids in [0, n), ascending.

    Sparse rows (4 * max K <= n) draw K ids and redraw a row whole when it
    repeats an id; dense rows rank n uniform keys and keep the first K. Both
    make every K-subset equally likely. Returns the rows concatenated."""
    L = K.size
    kmax = int(K.max()) if L else 0
    if kmax > n:
        raise ValueError("consideration set larger than the product count")
    col = np.arange(kmax)
    if 4 * kmax > n:
        out = np.argsort(rng.random((L, n)), axis=1)[:, :kmax]
        out = np.where(col[None, :] < K[:, None], out, n)
        out.sort(axis=1)
        return out[col[None, :] < K[:, None]].astype(np.int32)
    out = np.empty((L, kmax), dtype=np.int64)
    todo = np.arange(L)
    while todo.size:
        cand = rng.integers(0, n, size=(todo.size, kmax))
        pad = col[None, :] >= K[todo][:, None]
        cand = np.where(pad, n + col[None, :], cand)
        cand.sort(axis=1)
        dup = (np.diff(cand, axis=1) == 0).any(axis=1) if kmax > 1 else np.zeros(todo.size, bool)
        out[todo[~dup]] = cand[~dup]
        todo = todo[dup]
    return out[col[None, :] < K[:, None]].astype(np.int32)


def _draw(rng: np.random.Generator, dist, size):
    kind = dist[0]
    if kind == "const":
        return np.full(size, float(dist[1]))
    if kind == "uniform":
        return rng.uniform(dist[1], dist[2], size)
    if kind == "lognormal":
        return rng.lognormal(dist[1], dist[2], size)
    if kind == "exp":
        return rng.exponential(dist[1], size)
    raise ValueError(f"unknown distribution {dist}")


def full_offer_demand(inst: Instance) -> np.ndarray:
    """Expected consumption of each resource when each segment is offered its
    whole consideration set: d_i = sum_l lam_l sum_{j in C_l} a_ij v_lj /
    (v_l0 + sum_{k in C_l} v_lk). Products outside C_l have no attraction, so
    the shadow attractions do not enter (Section 3, pi' with S = C_l)."""
    K = np.diff(inst.seg_ptr)
    seg_of = np.repeat(np.arange(inst.L), K)
    den = inst.v0 + np.bincount(seg_of, weights=inst.v, minlength=inst.L)
    sales = np.bincount(inst.seg_prod, weights=inst.lam[seg_of] * inst.v / den[seg_of], minlength=inst.n)
    a_val = inst.a_val if inst.a_val is not None else np.ones(inst.nnzA)
    prod_of = np.repeat(np.arange(inst.n), np.diff(inst.a_ptr))
    return np.bincount(inst.a_idx, weights=a_val * sales[prod_of], minlength=inst.m)


def _segment_chunk(args):
    """Draws of one chunk of segments: product ids, v, theta, v0, lambda, from
    the chunk's own stream (seed, 1, chunk index)."""
    seed, ci, n, Kc, gam, v_dist, theta_dist, v0_dist, lam_dist = args
    rng = np.random.default_rng([seed, 1, ci])
    prod = _distinct_sorted(rng, n, Kc)
    v = _draw(rng, v_dist, int(Kc.sum()))
    w = np.repeat(_draw(rng, theta_dist, Kc.size), Kc) * v if gam else None
    v0 = _draw(rng, v0_dist, Kc.size)
    lam = _draw(rng, lam_dist, Kc.size)
    return prod, v, w, v0, lam


def make_instance(*, n: int, m: int, L: int, kmin: int, kmax: int, res_min: int = 1, res_max: int = 3,
                  gam: bool = True, v_dist=("uniform", 0.1, 1.0), theta_dist=("uniform", 0.0, 1.0),
                  v0_dist=("uniform", 0.5, 2.0), r_dist=("lognormal", 3.0, 0.5), lam_dist=("exp", 1.0),
                  tightness: Optional[float] = 0.6, c_dist=None, identity_A: bool = False,
                  seed: int = 1, name: str = "", workers: int = 1) -> Instance:
    """Draw one instance. The stream of `seed` draws the incidence, the prices,
    the set sizes and (last) capacities drawn directly; each chunk of 2^20
    segments draws its product ids, v, theta, v0 and lambda from its own stream
    (seed, 1, chunk), so chunks can be drawn in parallel (`workers` processes)
    with identical results. ``tightness=None`` makes capacities non-binding
    (1e30); ``c_dist`` draws capacities directly."""
    rng = np.random.default_rng(seed)
    # incidence: product j uses U{res_min..res_max} distinct resources
    if identity_A:
        if n != m:
            raise ValueError("identity incidence needs n == m")
        a_ptr = np.arange(n + 1, dtype=np.int32)
        a_idx = np.arange(n, dtype=np.int32)
    else:
        cnt = rng.integers(res_min, res_max + 1, size=n)
        a_idx = _distinct_sorted(rng, m, cnt)
        a_ptr = np.zeros(n + 1, dtype=np.int32)
        np.cumsum(cnt, out=a_ptr[1:])
    r = _draw(rng, r_dist, n)
    K = rng.integers(kmin, kmax + 1, size=L)
    seg_ptr = np.zeros(L + 1, dtype=np.int64)
    np.cumsum(K, out=seg_ptr[1:])
    nnz = int(seg_ptr[-1])
    seg_prod = np.empty(nnz, dtype=np.int32)
    v = np.empty(nnz)
    w = np.empty(nnz) if gam else None
    v0 = np.empty(L)
    lam = np.empty(L)
    starts = list(range(0, L, _CHUNK))
    jobs = [(seed, ci, n, K[s:min(L, s + _CHUNK)], gam, v_dist, theta_dist, v0_dist, lam_dist)
            for ci, s in enumerate(starts)]
    if workers > 1 and len(jobs) > 1:
        from concurrent.futures import ProcessPoolExecutor
        from multiprocessing import get_context
        with ProcessPoolExecutor(min(workers, len(jobs)), mp_context=get_context("spawn")) as pool:
            parts = list(pool.map(_segment_chunk, jobs))
    else:
        parts = [_segment_chunk(j) for j in jobs]
    for s, (pp, vv, ww, vv0, ll) in zip(starts, parts):
        e = min(L, s + _CHUNK)
        b0, b1 = int(seg_ptr[s]), int(seg_ptr[e])
        seg_prod[b0:b1] = pp
        v[b0:b1] = vv
        if gam:
            w[b0:b1] = ww
        v0[s:e] = vv0
        lam[s:e] = ll
    inst = Instance(n=n, m=m, L=L, r=r, c=np.zeros(m), a_ptr=a_ptr, a_idx=a_idx, a_val=None,
                    seg_ptr=seg_ptr, seg_prod=seg_prod, v=v, w=w, lam=lam, v0=v0, name=name)
    if c_dist is not None:
        inst.c = _draw(rng, c_dist, m)
    elif tightness is None:
        inst.c = np.full(m, 1e30)
    else:
        inst.c = tightness * full_offer_demand(inst)
    return inst


def tiny_mnl(seed: int = 0, capacity: str = "half") -> Instance:
    """Tiny plain CBLP: 12 products, 6 resources (1-2 per product), 40 segments
    with consideration sets of 4 products, MNL, v~U(0.1,1), v0=1,
    r~U(10,100), lambda~U(0.5,2); capacity 0.5 x demand, or non-binding."""
    return make_instance(n=12, m=6, L=40, kmin=4, kmax=4, res_min=1, res_max=2, gam=False,
                         v_dist=("uniform", 0.1, 1.0), v0_dist=("const", 1.0), r_dist=("uniform", 10.0, 100.0),
                         lam_dist=("uniform", 0.5, 2.0), tightness=None if capacity == "inf" else 0.5,
                         seed=seed, name=f"tiny_mnl(seed={seed},c={capacity})")


def mid_gam(seed: int = 1, L: int = 1_000_000, n: int = 10_000, m: int = 2000, kmin: int = 5, kmax: int = 15,
            tightness: Optional[float] = 0.6) -> Instance:
    """Mid GAM instance: 1e4 products, 2000 resources (1-3 per product), 1e6
    segments, |C_l|~U{5..15}; v~U(0.1,1), w=theta_l v with theta_l~U(0,1),
    v0~U(0.5,2), r~LogNormal(3,0.5), lambda~Exp(1), c = 0.6 x demand.
    Smaller L/n/m give parity-sized instances with the same distributions."""
    return make_instance(n=n, m=m, L=L, kmin=kmin, kmax=kmax, res_min=1, res_max=3, gam=True,
                         tightness=tightness, seed=seed, name=f"mid_gam(n={n},m={m},L={L},K={kmin}..{kmax},seed={seed})")


def huge_gam(seed: int = 2, L: int = 10_000_000, n: int = 100_000, m: int = 20_000, workers: int = 1) -> Instance:
    """Huge GAM instance: 1e5 products, 2e4 resources, 1e7 segments,
    |C_l|~U{10..30}, the mid instance's distributions, c = 0.4 x demand
    (chunks drawn by `workers` processes; the result does not depend on it)."""
    return make_instance(n=n, m=m, L=L, kmin=10, kmax=30, res_min=1, res_max=3, gam=True, tightness=0.4,
                         seed=seed, name=f"huge_gam(n={n},m={m},L={L},seed={seed})", workers=workers)


def paper_shaped(seed: int = 3, L: int = 100_000, n: int = 100) -> Instance:
    """Shape of the parallel-speedup study of Section 4.5: n = m = 100 with one
    resource per product, every segment considers all products, MNL, and
    c, r, v ~ U(0,1), lambda = 1."""
    return make_instance(n=n, m=n, L=L, kmin=n, kmax=n, gam=False, identity_A=True,
                         v_dist=("uniform", 0.0, 1.0), v0_dist=("uniform", 0.0, 1.0), r_dist=("uniform", 0.0, 1.0),
                         lam_dist=("const", 1.0), c_dist=("uniform", 0.0, 1.0), seed=seed,
                         name=f"paper_shaped(n={n},L={L},seed={seed})")


def batch_base(seed: int, k: int) -> Instance:
    """Base instance k of the batched multi-period family: n ~ U{200..5000},
    m = ceil(n / 5), L = floor(10^U(3, 5)), |C_l| ~ U{3..20}, the mid
    instance's distributions (c = 0.6 x demand of one period)."""
    rng = np.random.default_rng([seed, k])
    n = int(rng.integers(200, 5001))
    m = -(-n // 5)
    L = int(10.0 ** rng.uniform(3.0, 5.0))
    return make_instance(n=n, m=m, L=L, kmin=3, kmax=20, res_min=1, res_max=3, gam=True, tightness=0.6,
                         seed=int(rng.integers(1 << 62)), name=f"batch_base(seed={seed},k={k},n={n},L={L})")


def batch_family(seed: int = 4, count: int = 256) -> list:
    """The batched multi-period family: `count` base instances of uneven size."""
    return [batch_base(seed, k) for k in range(count)]


def period_rates(seed: int, count: int, periods: int = 16) -> np.ndarray:
    """Arrival-rate multipliers rho[period, instance] ~ U(0.5, 1.5)."""
    return np.random.default_rng([seed, 99]).uniform(0.5, 1.5, (periods, count))


def warm_family(seed: int, k: int, L_lo: float = 1e4, L_hi: float = 5e4) -> Instance:
    """Instance k of the learned-warm-start family: the huge instance's
    distributions (|C_l| ~ U{10..30}, c = 0.4 x demand) at reduced size,
    n = 2000 products, m = 400 resources, L = floor(10^U(log10 L_lo, log10 L_hi))."""
    rng = np.random.default_rng([seed, k, 5])
    L = int(10.0 ** rng.uniform(np.log10(L_lo), np.log10(L_hi)))
    return make_instance(n=2000, m=400, L=L, kmin=10, kmax=30, res_min=1, res_max=3, gam=True, tightness=0.4,
                         seed=int(rng.integers(1 << 62)), name=f"warm_family(seed={seed},k={k},L={L})")


def seeded_duals(m: int, seed: int, scale: float, frac_zero: float = 0.3) -> np.ndarray:
    """A seeded nonnegative dual vector: zero with probability frac_zero,
    else scale x U(0,1)."""
    rng = np.random.default_rng(seed)
    y = scale * rng.uniform(0.0, 1.0, m)
    y[rng.uniform(0.0, 1.0, m) < frac_zero] = 0.0
    return y
