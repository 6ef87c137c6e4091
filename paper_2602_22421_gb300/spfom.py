"""Python binding of libspfom.so (the C ABI of include/spfom.h and include/spfom_mlp.h).

Argument marshalling only: every step of the iteration runs in the library's
sm_103a kernels. The library must be built (``build.build()``); importing this
module on a machine without it raises instead of falling back to anything.
PyTorch, when present, only supplies the CUDA stream the ctx runs on.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libspfom.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, ENOTCONV, ENOTSUP = range(8)
VEC_Y, VEC_YBAR, VEC_SUM_Y, VEC_SUM_G, VEC_G, VEC_S, VEC_MARGINS = range(7)

# Every function the headers under include/ declare.
EXPORTS = ("spfom_default_params", "spfom_create", "spfom_load_instance", "spfom_reset", "spfom_step",
           "spfom_solve", "spfom_vector", "spfom_duals", "spfom_evaluate", "spfom_get_stats", "spfom_destroy",
           "spfom_last_error", "spfom_status_string", "spfom_sales_noalloc", "spfom_load_batch",
           "spfom_batch_stats", "spfom_update", "spfom_sales_at", "spfom_autotune", "spfom_set_wait_limit",
           "spfom_mlp_create", "spfom_mlp_set_wait_limit", "spfom_mlp_destroy", "spfom_mlp_set_params", "spfom_mlp_get_params",
           "spfom_mlp_get_grads", "spfom_mlp_forward", "spfom_mlp_loss_grad", "spfom_mlp_adam",
           "spfom_mlp_train_step", "spfom_features", "spfom_solve_warm", "spfom_xbar", "spfom_recover")

MLP_FEATURES, MLP_HIDDEN = 16, 256
MLP_PARAMS = 256 * 16 + 256 + 256 * 256 + 256 + 256 + 1

_f64p = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)


class Params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tau", C.c_double), ("tau0", C.c_double), ("mu", C.c_double),
                ("batch_frac", C.c_double), ("seed", C.c_uint64), ("eval_every", C.c_int64),
                ("restart_beta", C.c_double), ("restart_artificial", C.c_double),
                ("restart_tau_decay", C.c_double), ("restart_tau_balance", C.c_double), ("kkt_tol", C.c_double),
                ("max_iters", C.c_int64),
                ("device", C.c_int32), ("profile", C.c_int32), ("path", C.c_int32), ("pipeline", C.c_int32),
                ("graphs", C.c_int32),
                ("polish", C.c_int32), ("track_xbar", C.c_int32), ("tiling", C.c_int32),
                ("device_loop", C.c_int32), ("stream", C.c_void_p)]


class InstanceC(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("L", C.c_int64), ("r", _f64p), ("c", _f64p),
                ("a_ptr", _i32p), ("a_idx", _i32p), ("a_val", _f64p), ("seg_ptr", _i64p), ("seg_prod", _i32p),
                ("v", _f64p), ("w", _f64p), ("lam", _f64p), ("v0", _f64p)]


class DeviceSegments(C.Structure):
    _fields_ = [("n", C.c_int32), ("max_set_size", C.c_int32), ("L", C.c_int64), ("seg_ptr", C.c_void_p),
                ("seg_prod", C.c_void_p), ("v", C.c_void_p), ("w", C.c_void_p), ("lam", C.c_void_p),
                ("v0", C.c_void_p)]


NOALLOC_MAX_PRODUCTS = 131072


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int64), ("restarts", C.c_int64), ("evals", C.c_int64), ("epoch_iters", C.c_int64),
                ("converged", C.c_int32), ("pad_", C.c_int32), ("kkt", C.c_double), ("pinf", C.c_double),
                ("gap", C.c_double), ("dual_avg", C.c_double), ("primal_avg", C.c_double),
                ("dual_iter", C.c_double), ("z_sum", C.c_double), ("revenue", C.c_double),
                ("sum_revenue", C.c_double), ("tau", C.c_double), ("mu", C.c_double), ("seconds", C.c_double),
                ("seg_kernel_seconds", C.c_double), ("seg_kernel_launches", C.c_int64),
                ("kernel_launches", C.c_int64), ("fallback_segments", C.c_int64), ("fast_path", C.c_int32),
                ("iter_precision", C.c_int32), ("stall_iters", C.c_int64), ("stagnated", C.c_int32),
                ("pad2_", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}


class SpfomError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libspfom.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_2602_22421_gb300.build.build()")
        h = C.CDLL(LIB)
        P = C.POINTER
        h.spfom_default_params.argtypes = [P(Params)]
        h.spfom_default_params.restype = None
        h.spfom_create.argtypes = [P(Params), P(C.c_void_p)]
        h.spfom_load_instance.argtypes = [C.c_void_p, P(InstanceC)]
        h.spfom_reset.argtypes = [C.c_void_p, _f64p]
        h.spfom_step.argtypes = [C.c_void_p, C.c_int64, P(Stats)]
        h.spfom_solve.argtypes = [C.c_void_p, _f64p, P(Stats)]
        h.spfom_vector.argtypes = [C.c_void_p, C.c_int, _f64p]
        h.spfom_duals.argtypes = [C.c_void_p, C.c_int32, _f64p]
        h.spfom_evaluate.argtypes = [C.c_void_p, _f64p, _f64p, _f64p]
        h.spfom_get_stats.argtypes = [C.c_void_p, P(Stats)]
        h.spfom_destroy.argtypes = [C.c_void_p]
        h.spfom_destroy.restype = None
        h.spfom_last_error.argtypes = [C.c_void_p]
        h.spfom_last_error.restype = C.c_char_p
        h.spfom_status_string.argtypes = [C.c_int]
        h.spfom_status_string.restype = C.c_char_p
        h.spfom_sales_noalloc.argtypes = [P(DeviceSegments), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        h.spfom_sales_noalloc.restype = C.c_int
        h.spfom_load_batch.argtypes = [C.c_void_p, P(InstanceC), C.c_int32]
        h.spfom_batch_stats.argtypes = [C.c_void_p, P(Stats)]
        h.spfom_update.argtypes = [C.c_void_p, _f64p, _f64p]
        h.spfom_sales_at.argtypes = [C.c_void_p, _f64p, _f64p]
        h.spfom_autotune.argtypes = [C.c_void_p, C.c_int32, P(C.c_int32)]
        h.spfom_set_wait_limit.argtypes = [C.c_void_p, C.c_uint32]
        h.spfom_mlp_set_wait_limit.argtypes = [C.c_void_p, C.c_uint32]
        for f in ("spfom_load_batch", "spfom_batch_stats", "spfom_update", "spfom_sales_at", "spfom_autotune",
                  "spfom_set_wait_limit", "spfom_mlp_set_wait_limit"):
            getattr(h, f).restype = C.c_int
        _f32p = C.POINTER(C.c_float)
        h.spfom_mlp_create.argtypes = [C.c_int32, C.c_uint64, P(C.c_void_p)]
        h.spfom_mlp_destroy.argtypes = [C.c_void_p]
        h.spfom_mlp_destroy.restype = None
        h.spfom_mlp_set_params.argtypes = [C.c_void_p, _f32p]
        h.spfom_mlp_get_params.argtypes = [C.c_void_p, _f32p]
        h.spfom_mlp_get_grads.argtypes = [C.c_void_p, _f32p]
        h.spfom_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        h.spfom_mlp_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, _f64p, C.c_void_p]
        h.spfom_mlp_adam.argtypes = [C.c_void_p, C.c_float, C.c_void_p]
        h.spfom_mlp_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, _f64p,
                                           C.c_void_p]
        h.spfom_features.argtypes = [C.c_void_p, C.c_void_p]
        h.spfom_xbar.argtypes = [C.c_void_p, _f64p]
        h.spfom_recover.argtypes = [C.c_void_p, _f64p, _f64p, _i32p]
        h.spfom_xbar.restype = C.c_int
        h.spfom_recover.restype = C.c_int
        h.spfom_solve_warm.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, P(Stats), P(C.c_int32)]
        for f in ("spfom_mlp_create", "spfom_mlp_set_params", "spfom_mlp_get_params", "spfom_mlp_get_grads",
                  "spfom_mlp_forward", "spfom_mlp_loss_grad", "spfom_mlp_adam", "spfom_mlp_train_step",
                  "spfom_features", "spfom_solve_warm"):
            getattr(h, f).restype = C.c_int
        for f in ("spfom_create", "spfom_load_instance", "spfom_reset", "spfom_step", "spfom_solve", "spfom_vector",
                  "spfom_duals", "spfom_evaluate", "spfom_get_stats"):
            getattr(h, f).restype = C.c_int
        _lib = h
    return _lib


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


def default_params(**kw) -> Params:
    p = Params()
    lib().spfom_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def sales_noalloc(n, L, max_set_size, seg_ptr, seg_prod, v, w, lam, v0, margins, sales, z_sum, stream=None) -> int:
    """spfom_sales_noalloc on device pointers (ints, e.g. torch ``data_ptr()``);
    returns the status code. Allocates nothing."""
    d = DeviceSegments(n, max_set_size, L, seg_ptr, seg_prod, v, w or None, lam, v0)
    return lib().spfom_sales_noalloc(C.byref(d), margins, sales, z_sum, stream)


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


class InstanceArrays:
    """Contiguous host copies of an instance's arrays plus the C view of them."""

    def __init__(self, inst):
        self.keep = dict(
            r=np.ascontiguousarray(inst.r, np.float64), c=np.ascontiguousarray(inst.c, np.float64),
            a_ptr=np.ascontiguousarray(inst.a_ptr, np.int32), a_idx=np.ascontiguousarray(inst.a_idx, np.int32),
            a_val=None if inst.a_val is None else np.ascontiguousarray(inst.a_val, np.float64),
            seg_ptr=np.ascontiguousarray(inst.seg_ptr, np.int64),
            seg_prod=np.ascontiguousarray(inst.seg_prod, np.int32), v=np.ascontiguousarray(inst.v, np.float64),
            w=None if inst.w is None else np.ascontiguousarray(inst.w, np.float64),
            lam=np.ascontiguousarray(inst.lam, np.float64), v0=np.ascontiguousarray(inst.v0, np.float64))
        k = self.keep
        self.c = InstanceC(inst.n, inst.m, inst.L, _p(k["r"], _f64p), _p(k["c"], _f64p), _p(k["a_ptr"], _i32p),
                           _p(k["a_idx"], _i32p), _p(k["a_val"], _f64p), _p(k["seg_ptr"], _i64p),
                           _p(k["seg_prod"], _i32p), _p(k["v"], _f64p), _p(k["w"], _f64p), _p(k["lam"], _f64p),
                           _p(k["v0"], _f64p))

    def nbytes(self) -> int:
        return sum(a.nbytes for a in self.keep.values() if a is not None)


class Solver:
    """One spfom_ctx. ``Solver(inst, **params)`` creates it and loads ``inst``."""

    def __init__(self, inst=None, stream: Optional[int] = None, **params):
        self._lib = lib()
        p = default_params(**params)
        if p.stream is None:
            p.stream = stream if stream is not None else _current_stream()
        h = C.c_void_p()
        self._check(self._lib.spfom_create(C.byref(p), C.byref(h)), ctx=None)
        self._h = h
        self.params = p
        self.n = self.m = self.L = self.nnz = 0
        if inst is not None:
            self.load(inst)

    def _check(self, st: int, ctx="self"):
        if ctx == "self" and not getattr(self, "_h", None):
            raise SpfomError(ESTATE, "solver is closed")
        if st != OK:
            h = self._h if ctx == "self" else None
            msg = self._lib.spfom_last_error(h).decode() if h else self._lib.spfom_status_string(st).decode()
            raise SpfomError(st, msg)

    def load(self, inst):
        arrs = inst if isinstance(inst, InstanceArrays) else InstanceArrays(inst)
        self._check(self._lib.spfom_load_instance(self._h, C.byref(arrs.c)))
        self.n, self.m, self.L = arrs.c.n, arrs.c.m, arrs.c.L
        self.nnz = int(arrs.keep["seg_ptr"][-1])
        return self

    def load_batch(self, insts):
        """Load many instances as one batch (spfom_load_batch)."""
        arrs = [i if isinstance(i, InstanceArrays) else InstanceArrays(i) for i in insts]
        cs = (InstanceC * len(arrs))(*[a.c for a in arrs])
        self._keep_batch = arrs
        self._check(self._lib.spfom_load_batch(self._h, cs, len(arrs)))
        self.n = sum(a.c.n for a in arrs)
        self.m = sum(a.c.m for a in arrs)
        self.L = sum(a.c.L for a in arrs)
        self.nnz = sum(int(a.keep["seg_ptr"][-1]) for a in arrs)
        self.batch_sizes = [(a.c.n, a.c.m, a.c.L) for a in arrs]
        return self

    def batch_stats(self) -> list:
        out = (Stats * len(self.batch_sizes))()
        self._check(self._lib.spfom_batch_stats(self._h, out))
        return [o.as_dict() for o in out]

    def update(self, c=None, lam=None):
        c = None if c is None else np.ascontiguousarray(c, np.float64)
        lam = None if lam is None else np.ascontiguousarray(lam, np.float64)
        self._check(self._lib.spfom_update(self._h, _p(c, _f64p), _p(lam, _f64p)))

    def sales_at(self, y) -> np.ndarray:
        y = np.ascontiguousarray(y, np.float64)
        out = np.empty(max(self.n, 1))
        self._check(self._lib.spfom_sales_at(self._h, _p(y, _f64p), _p(out, _f64p)))
        return out[: self.n]

    def set_wait_limit(self, polls: int):
        """Polls before a bounded device wait gives up (spfom_set_wait_limit; testing aid)."""
        self._check(self._lib.spfom_set_wait_limit(self._h, int(polls)))

    def autotune(self, iters: int = 64) -> int:
        """Pick the fastest segment kernel for this instance (spfom_autotune)."""
        ch = C.c_int32(0)
        self._check(self._lib.spfom_autotune(self._h, int(iters), C.byref(ch)))
        return ch.value

    def xbar(self) -> np.ndarray:
        """Epoch-averaged responses per nonzero (spfom_xbar; needs track_xbar=1)."""
        out = np.empty(max(self.nnz, 1))
        self._check(self._lib.spfom_xbar(self._h, _p(out, _f64p)))
        return out[:self.nnz]

    def recover(self, x=None):
        """Assortment probabilities (spfom_recover): (alpha [nnz + L], order [nnz]);
        x None recovers from x-bar."""
        alpha = np.empty(max(self.nnz + self.L, 1))
        order = np.empty(max(self.nnz, 1), np.int32)
        xc = None if x is None else np.ascontiguousarray(x, np.float64)
        self._check(self._lib.spfom_recover(self._h, _p(xc, _f64p), _p(alpha, _f64p), _p(order, _i32p)))
        return alpha[:self.nnz + self.L], order[:self.nnz]

    def features(self, out=None):
        """Per-resource warm-start features (spfom_features) as a CUDA torch
        tensor [m, 16] (float32); ``out`` may supply it."""
        import torch
        if out is None:
            out = torch.empty((max(self.m, 1), MLP_FEATURES), dtype=torch.float32, device="cuda")
        self._check(self._lib.spfom_features(self._h, C.c_void_p(out.data_ptr())))
        return out[:self.m]

    def solve_warm(self, net: "MLP", warm_iters: int = 0):
        """spfom_solve_warm: (stats, mode) with mode 0 = prediction rejected
        (cold start), 1 = warm start converged, 2 = fell back to a cold start."""
        st, mode = Stats(), C.c_int32(-1)
        rc = self._lib.spfom_solve_warm(self._h, net._h, int(warm_iters), C.byref(st), C.byref(mode))
        if rc not in (OK, ENOTCONV):
            self._check(rc)
        return st.as_dict(), mode.value

    def reset(self, y0=None):
        y = None if y0 is None else np.ascontiguousarray(y0, np.float64)
        self._check(self._lib.spfom_reset(self._h, _p(y, _f64p)))

    def step(self, iters: int) -> dict:
        st = Stats()
        self._check(self._lib.spfom_step(self._h, int(iters), C.byref(st)))
        return st.as_dict()

    def solve(self, y0=None) -> dict:
        y = None if y0 is None else np.ascontiguousarray(y0, np.float64)
        st = Stats()
        rc = self._lib.spfom_solve(self._h, _p(y, _f64p), C.byref(st))
        if rc not in (OK, ENOTCONV):
            self._check(rc)
        return st.as_dict()

    def stats(self) -> dict:
        st = Stats()
        self._check(self._lib.spfom_get_stats(self._h, C.byref(st)))
        return st.as_dict()

    def vector(self, which: int) -> np.ndarray:
        size = self.n if which in (VEC_S, VEC_MARGINS) else self.m
        out = np.empty(max(size, 1))
        self._check(self._lib.spfom_vector(self._h, which, _p(out, _f64p)))
        return out[:size]

    def duals(self, averaged: bool = False) -> np.ndarray:
        out = np.empty(max(self.m, 1))
        self._check(self._lib.spfom_duals(self._h, 1 if averaged else 0, _p(out, _f64p)))
        return out[: self.m]

    def evaluate(self, y, per_segment: bool = False):
        y = np.ascontiguousarray(y, np.float64)
        z = np.empty(max(self.L, 1)) if per_segment else None
        d = C.c_double(0.0)
        self._check(self._lib.spfom_evaluate(self._h, _p(y, _f64p), _p(z, _f64p), C.byref(d)))
        return (d.value, z[: self.L]) if per_segment else d.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.spfom_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class MLP:
    """The warm-start network of include/spfom_mlp.h (spfom_mlp_*). Device
    arrays are CUDA torch tensors (float32, contiguous)."""

    def __init__(self, device: int = 0, seed: int = 0):
        self._lib = lib()
        h = C.c_void_p()
        st = self._lib.spfom_mlp_create(int(device), int(seed) & (2**64 - 1), C.byref(h))
        if st != OK:
            raise SpfomError(st, "spfom_mlp_create: " + self._lib.spfom_status_string(st).decode())
        self._h = h

    def _check(self, st: int, what: str):
        if not getattr(self, "_h", None):
            raise SpfomError(ESTATE, "network is closed")
        if st != OK:
            raise SpfomError(st, f"{what}: " + self._lib.spfom_status_string(st).decode())

    def set_wait_limit(self, polls: int):
        """Polls before a bounded copy wait of the tensor-core products gives up
        (spfom_mlp_set_wait_limit; testing aid)."""
        self._check(self._lib.spfom_mlp_set_wait_limit(self._h, int(polls)), "set_wait_limit")

    @staticmethod
    def _dev(t, rows, cols=None):
        import torch
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        assert t.shape[0] >= rows and (cols is None or (t.dim() == 2 and t.shape[1] == cols))
        return C.c_void_p(t.data_ptr())

    @property
    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        self._check(self._lib.spfom_mlp_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float))), "get_params")
        return out

    @params.setter
    def params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.shape == (MLP_PARAMS,)
        self._check(self._lib.spfom_mlp_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float))), "set_params")

    def grads(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        self._check(self._lib.spfom_mlp_get_grads(self._h, out.ctypes.data_as(C.POINTER(C.c_float))), "get_grads")
        return out

    def forward(self, x, out=None):
        import torch
        rows = int(x.shape[0])
        if out is None:
            out = torch.empty(max(rows, 1), dtype=torch.float32, device=x.device)
        self._check(self._lib.spfom_mlp_forward(self._h, self._dev(x, rows, MLP_FEATURES), rows,
                                                self._dev(out, rows), _current_stream()), "forward")
        return out[:rows]

    def loss_grad(self, x, t) -> float:
        rows, loss = int(x.shape[0]), C.c_double(0.0)
        self._check(self._lib.spfom_mlp_loss_grad(self._h, self._dev(x, rows, MLP_FEATURES), self._dev(t, rows), rows,
                                                  C.byref(loss), _current_stream()), "loss_grad")
        return loss.value

    def adam(self, lr: float):
        self._check(self._lib.spfom_mlp_adam(self._h, float(lr), _current_stream()), "adam")

    def train_step(self, x, t, lr: float) -> float:
        rows, loss = int(x.shape[0]), C.c_double(0.0)
        self._check(self._lib.spfom_mlp_train_step(self._h, self._dev(x, rows, MLP_FEATURES), self._dev(t, rows),
                                                   rows, float(lr), C.byref(loss), _current_stream()), "train_step")
        return loss.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.spfom_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
