"""Independent definitions the oracle is pinned to (test code only).

* ``brute_force_segment``: enumerate every assortment S of a segment's
  consideration set and evaluate lambda * sum_{j in S} m_j pi'_j(S) with the
  closed-form choice probability of the generalized attraction model
  (Section 3): pi'_j(S) = v_j / (v_0 + sum_{k in S} v_k + sum_{k not in S} w_k).
* ``sblp_highs``: the sales-based LP of Section 3.2 in its GAM form, solved by
  SciPy's HiGHS; returns the optimum and the capacity duals.
* ``cblp_highs``: the choice-based LP of Section 3.1 with every assortment
  enumerated, solved by HiGHS (tiny instances only).
"""
from __future__ import annotations

import itertools

import numpy as np


def dense_A(inst) -> np.ndarray:
    A = np.zeros((inst.m, inst.n))
    for j in range(inst.n):
        for p in range(inst.a_ptr[j], inst.a_ptr[j + 1]):
            A[inst.a_idx[p], j] += 1.0 if inst.a_val is None else inst.a_val[p]
    return A


def gam_prob(v, w, v0, S):
    """Choice probabilities of the items of S (mask) under pi' of Section 3."""
    den = v0 + v[S].sum() + w[~S].sum()
    return np.where(S, v / den, 0.0)


def brute_force_segment(inst, l: int, marg: np.ndarray):
    """max over all S of lam * sum_{j in S} m_j pi'_j(S); returns (value, best mask list)."""
    prod, v, w = inst.segment(l)
    K = len(prod)
    lam, v0 = inst.lam[l], inst.v0[l]
    m = marg[prod]
    best, arg = 0.0, [np.zeros(K, bool)]
    for bits in range(1, 1 << K):
        S = np.array([(bits >> k) & 1 == 1 for k in range(K)])
        val = lam * float((m * gam_prob(v, w, v0, S)).sum())
        if val > best * (1 + 1e-13) + 1e-300:
            best, arg = val, [S]
        elif abs(val - best) <= 1e-13 * max(1.0, abs(best)):
            arg.append(S)
    return best, arg


def sales_of(inst, l: int, S: np.ndarray) -> np.ndarray:
    prod, v, w = inst.segment(l)
    return inst.lam[l] * gam_prob(v, w, inst.v0[l], S)


def sblp_highs(inst, return_x: bool = False):
    """GAM sales-based LP: max sum r_j x_lj s.t. A x <= c; x_l0 + sum (vt/v) x_lj = lam_l;
    x_lj / v_lj <= x_l0 / vt_l0; x >= 0. Returns (OPT, capacity duals y*)."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    L, nnz, m = inst.L, inst.nnz, inst.m
    nv = nnz + L                      # x_lj (CSR order) then x_l0
    w = inst.w if inst.w is not None else np.zeros(nnz)
    vt = inst.v - w
    seg_of = np.repeat(np.arange(L), np.diff(inst.seg_ptr))
    vt0 = inst.v0 + np.bincount(seg_of, weights=w, minlength=L)
    cost = np.zeros(nv)
    cost[:nnz] = -inst.r[inst.seg_prod]
    A = dense_A(inst)
    # capacity rows
    rows, cols, vals = [], [], []
    for p in range(nnz):
        j = inst.seg_prod[p]
        for i in np.nonzero(A[:, j])[0]:
            rows.append(i); cols.append(p); vals.append(A[i, j])
    # scaling rows: x_lj / v_lj - x_l0 / vt_l0 <= 0
    for p in range(nnz):
        l = seg_of[p]
        rows += [m + p, m + p]; cols += [p, nnz + l]; vals += [1.0 / inst.v[p], -1.0 / vt0[l]]
    A_ub = coo_matrix((vals, (rows, cols)), shape=(m + nnz, nv)).tocsr()
    b_ub = np.concatenate([inst.c, np.zeros(nnz)])
    er, ec, ev = [], [], []
    for p in range(nnz):
        er.append(seg_of[p]); ec.append(p); ev.append(vt[p] / inst.v[p])
    for l in range(L):
        er.append(l); ec.append(nnz + l); ev.append(1.0)
    A_eq = coo_matrix((ev, (er, ec)), shape=(L, nv)).tocsr()
    res = linprog(cost, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=inst.lam, bounds=(0, None), method="highs")
    assert res.status == 0, res.message
    if return_x:
        return -res.fun, -res.ineqlin.marginals[:m], res.x[:nnz]
    return -res.fun, -res.ineqlin.marginals[:m]


def cblp_highs(inst):
    """Choice-based LP with every assortment of every segment enumerated."""
    from scipy.optimize import linprog
    A = dense_A(inst)
    cost, cap_cols, eq_rows = [], [], []
    for l in range(inst.L):
        prod, v, w = inst.segment(l)
        K = len(prod)
        for bits in range(1 << K):
            S = np.array([(bits >> k) & 1 == 1 for k in range(K)], dtype=bool)
            pi = gam_prob(v, w, inst.v0[l], S)
            cost.append(-float((inst.r[prod] * pi).sum()))
            cap_cols.append(A[:, prod] @ pi)
            eq_rows.append(l)
    nv = len(cost)
    A_ub = np.array(cap_cols).T
    A_eq = np.zeros((inst.L, nv))
    A_eq[eq_rows, np.arange(nv)] = 1.0
    res = linprog(np.array(cost), A_ub=A_ub, b_ub=inst.c, A_eq=A_eq, b_eq=inst.lam, bounds=(0, None),
                  method="highs")
    assert res.status == 0, res.message
    return -res.fun


def brute_force_all_products(inst, l: int, marg: np.ndarray) -> float:
    """Enumerate all 2^n assortments of the whole catalogue for segment l:
    products outside the consideration set have no attraction."""
    prod, v, w = inst.segment(l)
    vfull = np.zeros(inst.n); wfull = np.zeros(inst.n)
    vfull[prod] = v; wfull[prod] = w
    best = 0.0
    for bits in itertools.product([False, True], repeat=inst.n):
        S = np.array(bits)
        den = inst.v0[l] + vfull[S].sum() + wfull[~S].sum()
        best = max(best, inst.lam[l] * float((marg * np.where(S, vfull, 0.0)).sum()) / den)
    return best
