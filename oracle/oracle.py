"""Python access to the plain FP64 C oracle (``spfom_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline / reference leg use this module; the solver library
never imports it. It shares no code with the CUDA path: it reads instances from
the ``instances`` generator and nothing else.

The C source is compiled with ``-ffp-contract=off`` so that no multiply-add is
fused: the same bits come out on x86-64 and on AArch64 hosts.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spfom_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")

_f64p = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain gcc, no SIMD);
    ``omp=True``: the timing build ``liboracle_omp.so`` (segments over all
    host cores; another summation order, never used for parity)."""
    lib = LIB_OMP if omp else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC):
        return lib
    tmp = f"{lib}.{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", *(["-fopenmp"] if omp else []), "-o", tmp, SRC, "-lm"])
    os.replace(tmp, lib)
    return lib


class _Inst(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("L", C.c_int64),
                ("r", _f64p), ("c", _f64p), ("a_ptr", _i32p), ("a_idx", _i32p), ("a_val", _f64p),
                ("seg_ptr", _i64p), ("seg_prod", _i32p), ("v", _f64p), ("w", _f64p),
                ("lam", _f64p), ("v0", _f64p)]


class _Params(C.Structure):
    _fields_ = [("tau", C.c_double), ("tau0", C.c_double), ("mu", C.c_double), ("batch_frac", C.c_double),
                ("seed", C.c_uint64), ("eval_every", C.c_int64), ("restart_beta", C.c_double),
                ("restart_artificial", C.c_double), ("restart_tau_decay", C.c_double),
                ("restart_tau_balance", C.c_double), ("kkt_tol", C.c_double)]


class _State(C.Structure):
    _fields_ = [("y", _f64p), ("sum_y", _f64p), ("sum_g", _f64p), ("s", _f64p), ("g", _f64p), ("x_cur", _f64p),
                ("sum_x", _f64p), ("sum_P", C.c_double), ("count", C.c_int64), ("t", C.c_int64), ("restarts", C.c_int64),
                ("mu_cur", C.c_double), ("tau_used", C.c_double), ("kkt_anchor", C.c_double),
                ("z_sum", C.c_double), ("P", C.c_double), ("dual_iter", C.c_double),
                ("kkt", C.c_double), ("pinf", C.c_double), ("gap", C.c_double), ("dual_avg", C.c_double),
                ("primal_avg", C.c_double), ("evals", C.c_int64), ("converged", C.c_int32)]


_libs = {}


def lib(omp: bool = False):
    if omp not in _libs:
        h = C.CDLL(build(omp=omp))
        P = C.POINTER
        h.orc_margins.argtypes = [P(_Inst), _f64p, _f64p]
        h.orc_segment_solve.argtypes = [P(_Inst), C.c_int64, _f64p, _f64p, _i32p]
        h.orc_segment_solve.restype = C.c_double
        h.orc_fast_inner.argtypes = [P(_Inst), C.c_int64, _f64p, C.c_double, _f64p]
        h.orc_fast_inner.restype = C.c_double
        h.orc_segment_golden.argtypes = [P(_Inst), C.c_int64, _f64p, C.c_double]
        h.orc_segment_golden.restype = C.c_double
        h.orc_sweep.argtypes = [P(_Inst), _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        h.orc_dual.argtypes = [P(_Inst), _f64p]
        h.orc_dual.restype = C.c_double
        h.orc_sample_hash.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
        h.orc_sample_hash.restype = C.c_uint64
        h.orc_default_tau.argtypes = [P(_Inst), C.c_double]
        h.orc_default_tau.restype = C.c_double
        h.orc_state_init.argtypes = [P(_Inst), P(_Params), P(_State)]
        h.orc_run.argtypes = [P(_Inst), P(_Params), P(_State), C.c_int64]
        h.orc_run.restype = C.c_int
        h.orc_evaluate.argtypes = [P(_Inst), P(_Params), P(_State)]
        h.orc_evaluate.restype = None
        h.orc_recover.argtypes = [P(_Inst), _f64p, _f64p, _i32p]
        h.orc_recover.restype = None
        _libs[omp] = h
    return _libs[omp]


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


@dataclass
class Params:
    """Iteration parameters (same meaning as the library's spfom_params)."""
    tau: float = 0.0          # <= 0: tau0 * mean(r) / mean(c)
    tau0: float = 0.1         # step scale (Section 4.5 uses tau = 0.1 on U(0,1) data)
    mu: float = 0.0           # regulariser of eq. stronglycvxupdate
    batch_frac: float = 1.0   # Bernoulli(p) segment sampling; 1 = full batch
    seed: int = 0
    eval_every: int = 64
    restart_beta: float = 0.2
    restart_artificial: float = 0.36
    restart_tau_decay: float = 1.0
    restart_tau_balance: float = 0.0
    kkt_tol: float = 1e-4

    def _c(self) -> _Params:
        return _Params(self.tau, self.tau0, self.mu, self.batch_frac, self.seed, self.eval_every,
                       self.restart_beta, self.restart_artificial, self.restart_tau_decay,
                       self.restart_tau_balance, self.kkt_tol)


class Oracle:
    """FP64 oracle bound to one instance (arrays are kept alive here)."""

    def __init__(self, inst, omp: bool = False):
        """omp=True binds the all-core timing build (not for parity)."""
        self.inst = inst
        self._keep = dict(
            r=np.ascontiguousarray(inst.r, np.float64), c=np.ascontiguousarray(inst.c, np.float64),
            a_ptr=np.ascontiguousarray(inst.a_ptr, np.int32), a_idx=np.ascontiguousarray(inst.a_idx, np.int32),
            a_val=None if inst.a_val is None else np.ascontiguousarray(inst.a_val, np.float64),
            seg_ptr=np.ascontiguousarray(inst.seg_ptr, np.int64),
            seg_prod=np.ascontiguousarray(inst.seg_prod, np.int32),
            v=np.ascontiguousarray(inst.v, np.float64),
            w=None if inst.w is None else np.ascontiguousarray(inst.w, np.float64),
            lam=np.ascontiguousarray(inst.lam, np.float64), v0=np.ascontiguousarray(inst.v0, np.float64))
        k = self._keep
        self._c = _Inst(inst.n, inst.m, inst.L, _p(k["r"], _f64p), _p(k["c"], _f64p), _p(k["a_ptr"], _i32p),
                        _p(k["a_idx"], _i32p), _p(k["a_val"], _f64p), _p(k["seg_ptr"], _i64p),
                        _p(k["seg_prod"], _i32p), _p(k["v"], _f64p), _p(k["w"], _f64p), _p(k["lam"], _f64p),
                        _p(k["v0"], _f64p))
        self._lib = lib(omp)

    # --- a1 / a2 ---------------------------------------------------------
    def margins(self, y) -> np.ndarray:
        y = np.ascontiguousarray(y, np.float64)
        out = np.empty(self.inst.n)
        self._lib.orc_margins(C.byref(self._c), _p(y, _f64p), _p(out, _f64p))
        return out

    def segment_solve(self, l: int, marg):
        marg = np.ascontiguousarray(marg, np.float64)
        K = int(self.inst.seg_ptr[l + 1] - self.inst.seg_ptr[l])
        x = np.empty(max(K, 1))
        ks = C.c_int32(0)
        z = self._lib.orc_segment_solve(C.byref(self._c), l, _p(marg, _f64p), _p(x, _f64p), C.byref(ks))
        return z, x[:K], ks.value

    def fast_inner(self, l: int, marg, u: float):
        marg = np.ascontiguousarray(marg, np.float64)
        K = int(self.inst.seg_ptr[l + 1] - self.inst.seg_ptr[l])
        x = np.empty(max(K, 1))
        val = self._lib.orc_fast_inner(C.byref(self._c), l, _p(marg, _f64p), u, _p(x, _f64p))
        return val, x[:K]

    def golden(self, l: int, marg, eps: float) -> float:
        marg = np.ascontiguousarray(marg, np.float64)
        return self._lib.orc_segment_golden(C.byref(self._c), l, _p(marg, _f64p), eps)

    # --- a3 / dual ---------------------------------------------------------
    def sweep(self, y) -> dict:
        y = np.ascontiguousarray(y, np.float64)
        I = self.inst
        s, g, z = np.empty(I.n), np.empty(I.m), np.empty(I.L)
        P, zs = C.c_double(0), C.c_double(0)
        self._lib.orc_sweep(C.byref(self._c), _p(y, _f64p), _p(s, _f64p), _p(g, _f64p), C.byref(P),
                            C.byref(zs), _p(z, _f64p))
        return dict(s=s, g=g, P=P.value, zsum=zs.value, z=z)

    def dual(self, y) -> float:
        y = np.ascontiguousarray(y, np.float64)
        return self._lib.orc_dual(C.byref(self._c), _p(y, _f64p))

    def default_tau(self, tau0: float) -> float:
        return self._lib.orc_default_tau(C.byref(self._c), tau0)

    def run(self, params: Optional[Params] = None, y0=None, track_x: bool = False) -> "OracleRun":
        return OracleRun(self, params or Params(), y0, track_x)

    # --- f4 -------------------------------------------------------------------
    def recover(self, x):
        """Assortment probabilities (Lemma recover): (alpha [nnz + L], order [nnz])."""
        x = np.ascontiguousarray(x, np.float64)
        I = self.inst
        alpha = np.empty(I.nnz + I.L)
        order = np.empty(max(I.nnz, 1), np.int32)
        self._lib.orc_recover(C.byref(self._c), _p(x, _f64p), _p(alpha, _f64p), _p(order, _i32p))
        return alpha, order[:I.nnz]


def sample_hash(seed: int, t: int, l: int) -> int:
    return lib().orc_sample_hash(seed, t, l)


class OracleRun:
    """SPFOM run state on the oracle: ``step(k)`` advances k iterations."""

    def __init__(self, orc: Oracle, params: Params, y0=None, track_x: bool = False):
        I = orc.inst
        self.orc, self.params = orc, params
        self.y = np.zeros(I.m) if y0 is None else np.array(y0, np.float64)
        self.sum_y, self.sum_g = np.zeros(I.m), np.zeros(I.m)
        self.s, self.g = np.zeros(I.n), np.zeros(I.m)
        self.x_cur = np.zeros(I.nnz) if params.batch_frac < 1.0 else None
        self.sum_x = np.zeros(max(I.nnz, 1)) if track_x else None
        self._pc = params._c()
        self._st = _State(_p(self.y, _f64p), _p(self.sum_y, _f64p), _p(self.sum_g, _f64p), _p(self.s, _f64p),
                          _p(self.g, _f64p), _p(self.x_cur, _f64p), _p(self.sum_x, _f64p))
        orc._lib.orc_state_init(C.byref(orc._c), C.byref(self._pc), C.byref(self._st))
        if y0 is not None:  # orc_state_init leaves y alone
            self.y[:] = np.asarray(y0, np.float64)

    def step(self, iters: int) -> dict:
        rc = self.orc._lib.orc_run(C.byref(self.orc._c), C.byref(self._pc), C.byref(self._st), iters)
        if rc != 0:
            raise RuntimeError("oracle run failed")
        return self.stats()

    def evaluate(self) -> dict:
        """One KKT evaluation and restart test on the current epoch sums (what
        ``step`` runs every ``eval_every`` iterations); returns the stats."""
        self.orc._lib.orc_evaluate(C.byref(self.orc._c), C.byref(self._pc), C.byref(self._st))
        return self.stats()

    def set_state(self, **kw) -> None:
        """Overwrite scalar fields of the run state (sum_P, count, t, mu_cur,
        tau_used, kkt_anchor, ...); the arrays are the numpy views above."""
        for k, v in kw.items():
            if k in ("y", "sum_y", "sum_g", "s", "g", "x_cur", "sum_x") or not hasattr(self._st, k):
                raise KeyError(k)
            setattr(self._st, k, v)

    def stats(self) -> dict:
        st = self._st
        return {k: getattr(st, k) for k, _ in _State._fields_
                if k not in ("y", "sum_y", "sum_g", "s", "g", "x_cur", "sum_x")}

    @property
    def xbar(self) -> np.ndarray:
        """Epoch average of every segment's response, per nonzero (track_x runs)."""
        if self.sum_x is None:
            raise RuntimeError("run made without track_x")
        c = self._st.count
        return self.sum_x[:self.orc.inst.nnz] / c if c > 0 else np.full(self.orc.inst.nnz, math.nan)

    @property
    def ybar(self) -> np.ndarray:
        c = self._st.count
        return self.sum_y / c if c > 0 else self.y.copy()

    @property
    def gbar(self) -> np.ndarray:
        c = self._st.count
        return self.sum_g / c if c > 0 else np.full_like(self.sum_g, math.nan)
