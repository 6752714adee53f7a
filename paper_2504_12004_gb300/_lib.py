"""ctypes binding of libsbv.so: argument marshalling only.

Every function here converts torch tensors / numpy arrays into the plain
pointers and sizes of the C ABI in include/sbv.h and calls it.  No step of the
method runs in Python.  If the shared library has not been built, importing
the binding raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np
import torch

LIB_PATH = Path(__file__).resolve().parent / "libsbv.so"

SBV_OK, SBV_EINVAL, SBV_ENOTSPD, SBV_ENOMEM, SBV_ECUDA, SBV_ETIMEOUT, SBV_EUNSUPPORTED = range(7)
SBV_F64, SBV_F32 = 0, 1
SBV_PREC_FP64, SBV_PREC_MIXED, SBV_PREC_MIXED_BF16 = 0, 1, 2
PRECISIONS = {"fp64": SBV_PREC_FP64, "mixed": SBV_PREC_MIXED, "mixed_bf16": SBV_PREC_MIXED_BF16}
ERRNAMES = {1: "SBV_EINVAL", 2: "SBV_ENOTSPD", 3: "SBV_ENOMEM", 4: "SBV_ECUDA",
            5: "SBV_ETIMEOUT", 6: "SBV_EUNSUPPORTED"}

_lib = None


class MleOpts(C.Structure):
    """sbv_mle_opts"""
    _fields_ = [("max_evals", C.c_int32), ("fd_step", C.c_double), ("ftol", C.c_double),
                ("max_step", C.c_double), ("line_points", C.c_int32), ("precision", C.c_int32),
                ("nu2", C.c_int32), ("gradient", C.c_int32)]


class MleResult(C.Structure):
    """sbv_mle_result"""
    _fields_ = [("ll", C.c_double), ("evals", C.c_int32), ("calls", C.c_int32),
                ("iterations", C.c_int32), ("converged", C.c_int32), ("grad_evals", C.c_int32),
                ("proposals_won", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SurrogateOpts(C.Structure):
    """sbv_surrogate_opts"""
    _fields_ = [("exact_starts", C.c_int32), ("train_steps", C.c_int32), ("batch", C.c_int32),
                ("lr", C.c_float), ("ascent_starts", C.c_int32), ("ascent_iters", C.c_int32),
                ("candidates", C.c_int32), ("ascent_radius", C.c_double), ("seed", C.c_uint64),
                ("step_candidates", C.c_int32), ("step_radius", C.c_double),
                ("refit_every", C.c_int32)]


def mle_opts(max_evals=4000, fd_step=1e-3, ftol=1e-10, max_step=1.0, line_points=8,
             precision="mixed", nu2=5, gradient="differences") -> MleOpts:
    """gradient: "differences" (central, 2 (2 + d) rows) or "analytic" (sbv_loglik_grad, FP64)."""
    g = {"differences": 0, "analytic": 1}[gradient] if isinstance(gradient, str) else int(gradient)
    return MleOpts(max_evals, fd_step, ftol, max_step, line_points,
                   PRECISIONS[precision] if isinstance(precision, str) else int(precision), nu2, g)


def surrogate_opts(exact_starts=4, train_steps=4000, batch=512, lr=1e-3, ascent_starts=256,
                   ascent_iters=300, candidates=8, ascent_radius=1.0, seed=1, step_candidates=2,
                   step_radius=0.5, refit_every=10) -> SurrogateOpts:
    """candidates: restart proposals (0: none); step_candidates: proposals in every line search."""
    return SurrogateOpts(exact_starts, train_steps, batch, lr, ascent_starts, ascent_iters,
                         candidates, ascent_radius, seed, step_candidates, step_radius,
                         refit_every)

# (name, restype, argtypes) of every exported symbol
_P, _I32, _I64, _U64, _D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
SIGNATURES = {
    "sbv_version": (C.c_int, []),
    "sbv_create": (C.c_int, [C.POINTER(_P), C.c_int]),
    "sbv_destroy": (None, [_P]),
    "sbv_last_error": (C.c_char_p, [_P]),
    "sbv_blocking": (C.c_int, [_P, _P, C.c_int, _I64, _I32, _P, _I64, _I32, _U64,
                               _P, _P, _P, _P, _P, C.POINTER(_I64), _P]),
    "sbv_blocking_partitioned": (C.c_int, [_P, _P, C.c_int, _I64, _I32, _P, _I64, _I32, _U64, _I32,
                                           _P, _P, _P, _P, _P, C.POINTER(_I64), _P]),
    "sbv_knn": (C.c_int, [_P, _P, C.c_int, _I64, _I32, _P, _P, _P, _P, _P, _I64, _I32,
                          _P, _P, _P]),
    "sbv_loglik": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _P, _P, _P, _I64, _I32,
                             _I32, _P, _I32, _I32, _I32, _P, _P, _P, _P]),
    "sbv_loglik_grad": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _P, _P, _P, _I64, _I32,
                                  _I32, _P, _I32, _I32, _P, _P, _P, _P, _P, _P]),
    "sbv_sync_status": (C.c_int, [_P, _P]),
    "sbv_fp64_reruns": (C.c_int, [_P, _P, C.POINTER(_I64)]),
    "sbv_set_knn_mode": (C.c_int, [_P, _I32]),
    "sbv_predict": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _I64, _P, _I32, _P,
                              _I32, _I32, _P, _P, _P, _P, _P]),
    "sbv_predict_blocks": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _I64, _P, _I32, _P,
                                     _I32, _I32, _P, _P, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "sbv_loglik_fp64_noalloc": (C.c_int, [_P, C.c_int, _P, _I64, _I32, _P, _P, _P, _P, _I64,
                                          _I32, _I32, _P, _I32, _I32, _P, _P, _P, _P]),
    "sbv_loglik_graph_create": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _P, _P, _P, _I64,
                                          _I32, _I32, _I32, _I32, _I32, _P, _P, _P,
                                          C.POINTER(_P)]),
    "sbv_loglik_graph_launch": (C.c_int, [_P, _P, _P]),
    "sbv_loglik_graph_destroy": (None, [_P]),
    "sbv_autotune": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _P, _P, _P, _I64, _I32, _I32,
                               _P, _I32, _I32, _I32, C.POINTER(_I32), C.POINTER(_I32), _P]),
    "sbv_peak_probe": (C.c_int, [_P, _I32, C.POINTER(_D)]),
    "sbv_tuned_shape": (C.c_int, [_P, _I32, _I32, _I32, C.POINTER(_I32), C.POINTER(_I32),
                                  C.POINTER(_I32)]),
    "sbv_simulate": (C.c_int, [_P, _P, _P, _I64, _I32, _U64, _U64, _P, _P, _P, _P, _P, _P]),
    "sbv_matern": (C.c_int, [_P, _I32, _I32, _P, _I64, _P, _P]),
    "sbv_slabs": (C.c_int, [_P, _P, C.c_int, _I64, _I32, _P, _I32, _P, _P]),
    "sbv_predict_blocked": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _I64, _P, _I32, _I64,
                                      _I32, _U64, _P, _I32, _I32, _P, _P, _P, _P, _I64, _P, _P,
                                      _P, _P, _P, C.POINTER(_I64), _P]),
    "sbv_rac_plan": (C.c_int, [_U64, _I32, _P, _I64, _P, _P, _I64, _P]),
    "sbv_blocking_anchored": (C.c_int, [_P, _P, C.c_int, _I64, _I32, _P, _P, _I64, _I32,
                                        _P, _P, _P, _P, C.POINTER(_I64), _P]),
    "sbv_mlp_num_params": (_I64, [_I32]),
    "sbv_mlp_create": (C.c_int, [_P, _I32, _U64, C.POINTER(_P)]),
    "sbv_mlp_destroy": (None, [_P]),
    "sbv_mlp_set_params": (C.c_int, [_P, _P, _I64]),
    "sbv_mlp_get_params": (C.c_int, [_P, _P, _I64]),
    "sbv_mlp_grad": (C.c_int, [_P, _P, _P, _I64, _P, _P, _P]),
    "sbv_mlp_adam": (C.c_int, [_P, C.c_float, C.c_float, C.c_float, C.c_float, _P]),
    "sbv_mlp_train": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, C.c_float, _U64, C.POINTER(C.c_float),
                                _P]),
    "sbv_mlp_predict": (C.c_int, [_P, _P, _I64, _P, _P, _P]),
    "sbv_mle": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _P, _P, _P, _I64, _I32, _I32, _P, _P,
                          _P, _P, _P, _P, _P, _P, _I64, C.POINTER(_I64), _P]),
    "sbv_mle_multistart": (C.c_int, [_P, _P, C.c_int, _P, _I64, _I32, _P, _P, _P, _P, _I64, _I32,
                                     _I32, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _I64, _P, _P,
                                     _P]),
}


class SBVError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def load() -> C.CDLL:
    """Load libsbv.so (built by paper_2504_12004_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2504_12004_gb300.build` "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = C.CDLL(str(LIB_PATH))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return C.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    raise TypeError(type(t))


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _xdtype(X: torch.Tensor) -> int:
    if X.dtype == torch.float64:
        return SBV_F64
    if X.dtype == torch.float32:
        return SBV_F32
    raise TypeError(f"points must be float64 or float32, got {X.dtype}")


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _host_f64(a, name: str) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def rac_plan(seed: int, slab_counts, bc: int, bc_eff: int = 0):
    """Random choices of a partitioned blocking from the slab sizes alone
    (sbv_rac_plan): (quota per slab, anchor positions slab by slab, block
    rank for bc_eff blocks or None)."""
    lib = load()
    cnt = np.ascontiguousarray(np.asarray(slab_counts, dtype=np.int64))
    P = cnt.size
    quota = np.zeros(P, dtype=np.int64)
    rc = lib.sbv_rac_plan(int(seed) & 0xFFFFFFFFFFFFFFFF, P, _ptr(cnt), bc, _ptr(quota), None, 0, None)
    if rc != SBV_OK:
        raise SBVError(rc, "sbv_rac_plan: invalid arguments")
    pos = np.zeros(int(quota.sum()), dtype=np.int64)
    rank = np.zeros(bc_eff, dtype=np.int32) if bc_eff else None
    rc = lib.sbv_rac_plan(int(seed) & 0xFFFFFFFFFFFFFFFF, P, _ptr(cnt), bc, _ptr(quota), _ptr(pos),
                          bc_eff, _ptr(rank))
    if rc != SBV_OK:
        raise SBVError(rc, "sbv_rac_plan: invalid arguments")
    return quota, pos, rank


class Context:
    """An sbv_ctx on one CUDA device (owns the library's workspace)."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = device
        h = C.c_void_p()
        rc = self.lib.sbv_create(C.byref(h), device)
        if rc != SBV_OK:
            raise SBVError(rc, f"sbv_create(device={device}) failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.sbv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != SBV_OK:
            raise SBVError(rc, self.lib.sbv_last_error(self.h).decode())

    # ---- entry points -------------------------------------------------------
    def sbv_blocking(self, X, beta_scale, bc: int, kmeans_iters: int, seed: int, stream=None,
                     partitions: int = 1):
        X = _dev(X, None, "X")
        n, d = X.shape
        beta = _host_f64(beta_scale, "beta_scale")
        dev = X.device
        blk = torch.empty(n, dtype=torch.int32, device=dev)
        ptr = torch.empty(bc + 1, dtype=torch.int64, device=dev)
        pts = torch.empty(n, dtype=torch.int32, device=dev)
        rank = torch.empty(bc, dtype=torch.int32, device=dev)
        centres = torch.empty(bc, d, dtype=torch.float64, device=dev)
        bc_eff = C.c_int64(0)
        if partitions == 1:
            rc = self.lib.sbv_blocking(self.h, _ptr(X), _xdtype(X), n, d, _ptr(beta), bc,
                                       kmeans_iters, seed, _ptr(blk), _ptr(ptr), _ptr(pts),
                                       _ptr(rank), _ptr(centres), C.byref(bc_eff), _stream(stream))
        else:
            rc = self.lib.sbv_blocking_partitioned(self.h, _ptr(X), _xdtype(X), n, d, _ptr(beta), bc,
                                                   kmeans_iters, seed, partitions, _ptr(blk),
                                                   _ptr(ptr), _ptr(pts), _ptr(rank), _ptr(centres),
                                                   C.byref(bc_eff), _stream(stream))
        self._check(rc)
        k = bc_eff.value
        return dict(blk=blk, ptr=ptr[:k + 1].contiguous(), pts=pts, rank=rank[:k].contiguous(),
                    centres=centres[:k].contiguous(), bc_eff=k)

    def sbv_slabs(self, X, beta_scale, partitions: int, stream=None) -> torch.Tensor:
        """Slab of every point (Alg. 2 routing), int32 on the device."""
        X = _dev(X, None, "X")
        n, d = X.shape
        slab = torch.empty(n, dtype=torch.int32, device=X.device)
        if n:
            self._check(self.lib.sbv_slabs(self.h, _ptr(X), _xdtype(X), n, d,
                                           _ptr(_host_f64(beta_scale, "beta_scale")), partitions,
                                           _ptr(slab), _stream(stream)))
        return slab

    def sbv_blocking_anchored(self, X, beta_scale, anchors, kmeans_iters: int, stream=None):
        """RAC from the given anchors (host indices) plus Lloyd iterations on one
        partition; blocks in anchor order, no block order."""
        X = _dev(X, None, "X")
        n, d = X.shape
        a = np.ascontiguousarray(np.asarray(anchors, dtype=np.int64))
        k = a.size
        dev = X.device
        blk = torch.empty(n, dtype=torch.int32, device=dev)
        ptr = torch.empty(k + 1, dtype=torch.int64, device=dev)
        pts = torch.empty(n, dtype=torch.int32, device=dev)
        centres = torch.empty(k, d, dtype=torch.float64, device=dev)
        bc_eff = C.c_int64(0)
        self._check(self.lib.sbv_blocking_anchored(
            self.h, _ptr(X), _xdtype(X), n, d, _ptr(_host_f64(beta_scale, "beta_scale")), _ptr(a), k,
            kmeans_iters, _ptr(blk), _ptr(ptr), _ptr(pts), _ptr(centres), C.byref(bc_eff),
            _stream(stream)))
        e = bc_eff.value
        return dict(blk=blk, ptr=ptr[:e + 1].contiguous(), pts=pts, centres=centres[:e].contiguous(),
                    bc_eff=e)

    def sbv_set_knn_mode(self, mode: int):
        """0 automatic, 1 full scan, 2 pruned search (identical results)."""
        self._check(self.lib.sbv_set_knn_mode(self.h, mode))

    def sbv_knn(self, X, beta_scale, ptr, pts, rank, centres, m: int, stream=None):
        X = _dev(X, None, "X")
        n, d = X.shape
        bc = rank.numel()
        beta = _host_f64(beta_scale, "beta_scale")
        nbr = torch.empty(bc, max(m, 1), dtype=torch.int32, device=X.device)
        cnt = torch.empty(bc, dtype=torch.int32, device=X.device)
        rc = self.lib.sbv_knn(self.h, _ptr(X), _xdtype(X), n, d, _ptr(beta),
                              _ptr(_dev(ptr, torch.int64, "ptr")), _ptr(_dev(pts, torch.int32, "pts")),
                              _ptr(_dev(rank, torch.int32, "rank")),
                              _ptr(_dev(centres, torch.float64, "centres")), bc, m, _ptr(nbr),
                              _ptr(cnt), _stream(stream))
        self._check(rc)
        return nbr[:, :m], cnt

    def sbv_loglik(self, X, y, ptr, pts, nbr, cnt, theta, nu2: int = 5, precision="fp64",
                   ll=None, block_terms=None, status=None, stream=None, nmax: int = 0):
        """Enqueue the log-likelihood of every theta row; returns the device tensor ll (B).

        nmax: largest m_i + bs_i (see max_block_size); 0 lets the call read it
        from the device, which waits for the stream."""
        X = _dev(X, None, "X")
        n, d = X.shape
        bc = cnt.numel()
        m = nbr.shape[1] if nbr.dim() == 2 else 0
        th = _host_f64(theta, "theta").reshape(-1, 2 + d)
        B = th.shape[0]
        if ll is None:
            ll = torch.empty(B, dtype=torch.float64, device=X.device)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        nbr_c = _dev(nbr.contiguous() if nbr.stride(0) != m else nbr, torch.int32, "nbr")
        rc = self.lib.sbv_loglik(self.h, _ptr(X), _xdtype(X), _ptr(_dev(y, torch.float64, "y")), n, d,
                                 _ptr(_dev(ptr, torch.int64, "ptr")), _ptr(_dev(pts, torch.int32, "pts")),
                                 _ptr(nbr_c), _ptr(_dev(cnt, torch.int32, "cnt")), bc, m,
                                 int(nmax), _ptr(th), B, nu2, prec, _ptr(ll), _ptr(block_terms),
                                 _ptr(status), _stream(stream))
        self._check(rc)
        return ll

    def sbv_loglik_grad(self, X, y, ptr, pts, nbr, cnt, theta, nu2: int = 5, ll=None, grad=None,
                        block_terms=None, block_grads=None, status=None, stream=None, nmax: int = 0):
        """Enqueue the FP64 log-likelihood and its gradient in theta for every row;
        returns the device tensors (ll (B), grad (B x (2+d)))."""
        X = _dev(X, None, "X")
        n, d = X.shape
        bc = cnt.numel()
        m = nbr.shape[1] if nbr.dim() == 2 else 0
        th = _host_f64(theta, "theta").reshape(-1, 2 + d)
        B = th.shape[0]
        if ll is None:
            ll = torch.empty(B, dtype=torch.float64, device=X.device)
        if grad is None:
            grad = torch.empty(B, 2 + d, dtype=torch.float64, device=X.device)
        nbr_c = _dev(nbr.contiguous() if nbr.stride(0) != m else nbr, torch.int32, "nbr")
        rc = self.lib.sbv_loglik_grad(self.h, _ptr(X), _xdtype(X), _ptr(_dev(y, torch.float64, "y")),
                                      n, d, _ptr(_dev(ptr, torch.int64, "ptr")),
                                      _ptr(_dev(pts, torch.int32, "pts")), _ptr(nbr_c),
                                      _ptr(_dev(cnt, torch.int32, "cnt")), bc, m, int(nmax), _ptr(th),
                                      B, nu2, _ptr(ll), _ptr(grad), _ptr(block_terms),
                                      _ptr(block_grads), _ptr(status), _stream(stream))
        self._check(rc)
        return ll, grad

    def sbv_autotune(self, X, y, ptr, pts, nbr, cnt, theta, nu2: int = 5, precision="mixed",
                     nmax: int = 0, stream=None):
        """Time the block kernel's launch shapes on this structure; returns (threads, ctas_per_sm)."""
        X = _dev(X, None, "X")
        n, d = X.shape
        th = _host_f64(theta, "theta").reshape(-1, 2 + d)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        t, c = C.c_int32(0), C.c_int32(0)
        rc = self.lib.sbv_autotune(self.h, _ptr(X), _xdtype(X), _ptr(_dev(y, torch.float64, "y")), n, d,
                                   _ptr(_dev(ptr, torch.int64, "ptr")), _ptr(_dev(pts, torch.int32, "pts")),
                                   _ptr(_dev(nbr, torch.int32, "nbr")), _ptr(_dev(cnt, torch.int32, "cnt")),
                                   cnt.numel(), nbr.shape[1], int(nmax), _ptr(th), th.shape[0], nu2, prec,
                                   C.byref(t), C.byref(c), _stream(stream))
        self._check(rc)
        return t.value, c.value

    def sbv_tuned_shape(self, precision, nmax: int, d: int):
        """The autotuner's record: (threads, ctas_per_sm, tile)."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        t, c, w = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        self._check(self.lib.sbv_tuned_shape(self.h, prec, nmax, d, C.byref(t), C.byref(c),
                                             C.byref(w)))
        return t.value, c.value, w.value

    def sbv_peak_probe(self, kind: str = "fp64") -> float:
        """Measured FMA rate of the CUDA cores in TFLOP/s (kind "fp64" or "fp32")."""
        v = C.c_double(0.0)
        self._check(self.lib.sbv_peak_probe(self.h, {"fp64": 0, "fp32": 1}[kind], C.byref(v)))
        return v.value

    def sbv_loglik_graph_create(self, X, y, ptr, pts, nbr, cnt, B: int, nu2: int = 5,
                                precision="mixed", nmax: int = 0, block_terms=None, status=None):
        """Capture one evaluation as a CUDA graph; returns a LoglikGraph."""
        return LoglikGraph(self, X, y, ptr, pts, nbr, cnt, B, nu2, precision, nmax, block_terms,
                           status)

    def _structure(self, X, y, ptr, pts, nbr, cnt):
        X = _dev(X, None, "X")
        return (_ptr(X), _xdtype(X), _ptr(_dev(y, torch.float64, "y")), X.shape[0], X.shape[1],
                _ptr(_dev(ptr, torch.int64, "ptr")), _ptr(_dev(pts, torch.int32, "pts")),
                _ptr(_dev(nbr, torch.int32, "nbr")), _ptr(_dev(cnt, torch.int32, "cnt")),
                cnt.numel(), nbr.shape[1])

    def sbv_mle(self, X, y, ptr, pts, nbr, cnt, theta0, lower=None, upper=None, opts=None,
                nmax: int = 0, history: int = 0, stream=None):
        """BFGS maximum-likelihood estimate; returns (theta, MleResult[, (hist_u, hist_l)])."""
        st = self._structure(X, y, ptr, pts, nbr, cnt)
        d = st[4]
        th0 = _host_f64(theta0, "theta0").reshape(2 + d)
        lo = None if lower is None else _host_f64(lower, "lower").reshape(2 + d)
        hi = None if upper is None else _host_f64(upper, "upper").reshape(2 + d)
        out = np.empty(2 + d)
        res = MleResult()
        hu = np.empty((max(history, 1), 2 + d))
        hl = np.empty(max(history, 1))
        hlen = C.c_int64(0)
        rc = self.lib.sbv_mle(self.h, *st, int(nmax), _ptr(th0), _ptr(lo), _ptr(hi),
                              C.byref(opts) if opts is not None else None, _ptr(out), C.byref(res),
                              _ptr(hu) if history else None, _ptr(hl) if history else None, history,
                              C.byref(hlen) if history else None, _stream(stream))
        self._check(rc)
        if history:
            return out, res, (hu[:hlen.value], hl[:hlen.value])
        return out, res

    def sbv_mle_multistart(self, X, y, ptr, pts, nbr, cnt, starts, lower=None, upper=None,
                           opts=None, mlp=None, sopts=None, nmax: int = 0, stream=None,
                           prior=None):
        """MLE from every row of starts; returns (thetas, [MleResult]).  prior:
        (hist_u, hist_l) pairs of earlier runs (sbv_mle's history) that join
        the history before the first start."""
        st = self._structure(X, y, ptr, pts, nbr, cnt)
        d = st[4]
        S0 = _host_f64(starts, "starts").reshape(-1, 2 + d)
        lo = None if lower is None else _host_f64(lower, "lower").reshape(2 + d)
        hi = None if upper is None else _host_f64(upper, "upper").reshape(2 + d)
        pu = pl = None
        if prior is not None:
            pu = _host_f64(prior[0], "prior_u").reshape(-1, 2 + d)
            pl = _host_f64(prior[1], "prior_l").reshape(-1)
            if len(pl) != len(pu):
                raise ValueError("prior_u and prior_l differ in length")
        out = np.empty_like(S0)
        res = (MleResult * len(S0))()
        rc = self.lib.sbv_mle_multistart(self.h, *st, int(nmax), _ptr(S0), len(S0), _ptr(lo), _ptr(hi),
                                         C.byref(opts) if opts is not None else None,
                                         mlp.h if mlp is not None else None,
                                         C.byref(sopts) if sopts is not None else None,
                                         _ptr(pu), _ptr(pl), 0 if pl is None else len(pl),
                                         _ptr(out), C.cast(res, C.c_void_p), _stream(stream))
        self._check(rc)
        return out, [r for r in res]

    @staticmethod
    def max_block_size(ptr, cnt) -> int:
        """Largest m_i + bs_i, the nmax argument that spares sbv_loglik its device read."""
        return int((torch.diff(ptr).to(torch.int64) + cnt.to(torch.int64)).max().item())

    def sbv_sync_status(self, stream=None):
        self._check(self.lib.sbv_sync_status(self.h, _stream(stream)))

    def sbv_fp64_reruns(self, stream=None) -> int:
        """Items the mixed kernels handed to the FP64 kernels since the last sbv_sync_status."""
        c = C.c_int64(0)
        self._check(self.lib.sbv_fp64_reruns(self.h, _stream(stream), C.byref(c)))
        return c.value

    def sbv_predict(self, X, y, Xtest, beta_scale, m_pred: int, theta, nu2: int = 5,
                    precision="fp64", want_nbr=False, stream=None, blocks=None):
        """Predictive mean and variances; `blocks` (a dict from sbv_blocking on the
        same X) switches the neighbour search to sbv_predict_blocks."""
        X = _dev(X, None, "X")
        Xtest = _dev(Xtest, X.dtype, "Xtest")
        n, d = X.shape
        nt = Xtest.shape[0]
        beta = _host_f64(beta_scale, "beta_scale")
        th = _host_f64(theta, "theta").reshape(-1)
        dev = X.device
        mean = torch.empty(nt, dtype=torch.float64, device=dev)
        var = torch.empty(nt, dtype=torch.float64, device=dev)
        var_lat = torch.empty(nt, dtype=torch.float64, device=dev)
        nbr = torch.empty(nt, m_pred, dtype=torch.int32, device=dev) if want_nbr else None
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if blocks is None:
            rc = self.lib.sbv_predict(self.h, _ptr(X), _xdtype(X), _ptr(_dev(y, torch.float64, "y")),
                                      n, d, _ptr(Xtest), nt, _ptr(beta), m_pred, _ptr(th), nu2, prec,
                                      _ptr(mean), _ptr(var), _ptr(var_lat), _ptr(nbr), _stream(stream))
        else:
            b = blocks
            rc = self.lib.sbv_predict_blocks(
                self.h, _ptr(X), _xdtype(X), _ptr(_dev(y, torch.float64, "y")), n, d, _ptr(Xtest), nt,
                _ptr(beta), m_pred, _ptr(th), nu2, prec, _ptr(_dev(b["ptr"], torch.int64, "ptr")),
                _ptr(_dev(b["pts"], torch.int32, "pts")), _ptr(_dev(b["rank"], torch.int32, "rank")),
                _ptr(_dev(b["centres"], torch.float64, "centres")), b["rank"].numel(), _ptr(mean),
                _ptr(var), _ptr(var_lat), _ptr(nbr), _stream(stream))
        self._check(rc)
        return mean, var, var_lat, nbr

    def sbv_simulate(self, mean, var, ndraws: int = 1000, seed: int = 0, index_base: int = 0,
                     want_draws=False, stream=None):
        """Conditional simulation from predictive means and variances; returns
        (sample_mean, sample_var, ci_lo, ci_hi, draws or None)."""
        mean = _dev(mean, torch.float64, "mean")
        var = _dev(var, torch.float64, "var")
        if mean.shape != var.shape or mean.dim() != 1:
            raise ValueError("mean and var must be 1-d tensors of one length")
        nt = mean.numel()
        out = [torch.empty(nt, dtype=torch.float64, device=mean.device) for _ in range(4)]
        draws = (torch.empty(nt, int(ndraws), dtype=torch.float64, device=mean.device)
                 if want_draws else None)
        rc = self.lib.sbv_simulate(self.h, _ptr(mean), _ptr(var), nt, int(ndraws),
                                   int(seed) & 0xFFFFFFFFFFFFFFFF,
                                   int(index_base) & 0xFFFFFFFFFFFFFFFF, *[_ptr(t) for t in out],
                                   _ptr(draws), _stream(stream))
        self._check(rc)
        return (*out, draws)

    def sbv_matern(self, d2, nu2: int = 5, precision="fp64", stream=None):
        """Matern correlation M_nu(sqrt(d2)) through one precision's arithmetic."""
        d2 = _dev(d2, torch.float64, "d2")
        out = torch.empty_like(d2)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self._check(self.lib.sbv_matern(self.h, prec, nu2, _ptr(d2), d2.numel(), _ptr(out),
                                        _stream(stream)))
        return out

    def sbv_predict_blocked(self, X, y, Xtest, beta_scale, m_pred: int, bc_test: int, theta,
                            nu2: int = 5, precision="fp64", kmeans_iters: int = 10, seed: int = 0,
                            blocks=None, stream=None):
        """Block prediction: (mean, var, var_latent, test_block, nbr of the
        non-empty test blocks)."""
        X = _dev(X, None, "X")
        Xtest = _dev(Xtest, X.dtype, "Xtest")
        n, d = X.shape
        nt = Xtest.shape[0]
        dev = X.device
        mean = torch.empty(nt, dtype=torch.float64, device=dev)
        var = torch.empty(nt, dtype=torch.float64, device=dev)
        var_lat = torch.empty(nt, dtype=torch.float64, device=dev)
        tblk = torch.empty(nt, dtype=torch.int32, device=dev)
        nbr = torch.empty(bc_test, m_pred, dtype=torch.int32, device=dev)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        b = blocks or {}
        keff = C.c_int64(0)
        rc = self.lib.sbv_predict_blocked(
            self.h, _ptr(X), _xdtype(X), _ptr(_dev(y, torch.float64, "y")), n, d, _ptr(Xtest), nt,
            _ptr(_host_f64(beta_scale, "beta_scale")), m_pred, bc_test, kmeans_iters,
            int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(_host_f64(theta, "theta").reshape(-1)), nu2, prec,
            _ptr(b.get("ptr")), _ptr(b.get("pts")), _ptr(b.get("rank")), _ptr(b.get("centres")),
            b["rank"].numel() if b else 0, _ptr(mean), _ptr(var), _ptr(var_lat), _ptr(tblk),
            _ptr(nbr), C.byref(keff), _stream(stream))
        self._check(rc)
        return mean, var, var_lat, tblk, nbr[:keff.value]


class LoglikGraph:
    """One captured evaluation (sbv_loglik_graph_*): launch(theta) replays it.

    Holds references to every tensor the graph reads or writes, so they stay
    alive as long as the graph does."""

    def __init__(self, ctx: Context, X, y, ptr, pts, nbr, cnt, B, nu2, precision, nmax,
                 block_terms, status):
        self.ctx = ctx
        X = _dev(X, None, "X")
        n, d = X.shape
        self.d, self.B = d, B
        self.ll = torch.empty(B, dtype=torch.float64, device=X.device)
        self._keep = (X, y, ptr, pts, nbr, cnt, block_terms, status)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = C.c_void_p()
        rc = ctx.lib.sbv_loglik_graph_create(
            ctx.h, _ptr(X), _xdtype(X), _ptr(_dev(y, torch.float64, "y")), n, d,
            _ptr(_dev(ptr, torch.int64, "ptr")), _ptr(_dev(pts, torch.int32, "pts")),
            _ptr(_dev(nbr, torch.int32, "nbr")), _ptr(_dev(cnt, torch.int32, "cnt")), cnt.numel(),
            nbr.shape[1], int(nmax), B, nu2, prec, _ptr(self.ll), _ptr(block_terms), _ptr(status),
            C.byref(h))
        ctx._check(rc)
        self.h = h

    def launch(self, theta, stream=None):
        """Replay with new parameter rows (host, B x (2+d)); returns the device tensor ll."""
        th = _host_f64(theta, "theta").reshape(self.B, 2 + self.d)
        self.ctx._check(self.ctx.lib.sbv_loglik_graph_launch(self.h, _ptr(th), _stream(stream)))
        return self.ll

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.sbv_loglik_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The likelihood surrogate network (sbv_mlp_*): FP32 masters on the device."""

    def __init__(self, ctx: Context, in_dim: int, seed: int = 0):
        self.ctx = ctx
        self.in_dim = in_dim
        self.n_params = ctx.lib.sbv_mlp_num_params(in_dim)
        if self.n_params < 0:
            raise SBVError(SBV_EINVAL, f"in_dim={in_dim} out of range")
        h = C.c_void_p()
        ctx._check(ctx.lib.sbv_mlp_create(ctx.h, in_dim, seed, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.sbv_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        self.ctx._check(self.ctx.lib.sbv_mlp_get_params(self.h, _ptr(out), self.n_params))
        return out

    def set_params(self, params):
        v = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        self.ctx._check(self.ctx.lib.sbv_mlp_set_params(self.h, _ptr(v), v.size))

    def _rows(self, X):
        X = _dev(X, torch.float32, "X")
        if X.dim() != 2 or X.shape[1] != self.in_dim:
            raise ValueError(f"X must be K x {self.in_dim}")
        return X

    def grad(self, X, t, stream=None):
        """Returns (grads, loss) as device tensors."""
        X = self._rows(X)
        t = _dev(t, torch.float32, "t")
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        self.ctx._check(self.ctx.lib.sbv_mlp_grad(self.h, _ptr(X), _ptr(t), X.shape[0], _ptr(g),
                                                  _ptr(loss), _stream(stream)))
        return g, loss

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.ctx._check(self.ctx.lib.sbv_mlp_adam(self.h, lr, beta1, beta2, eps, _stream(stream)))

    def train(self, X, t, steps: int, batch: int, lr: float, seed: int = 0, stream=None) -> float:
        X = self._rows(X)
        t = _dev(t, torch.float32, "t")
        loss = C.c_float(0.0)
        self.ctx._check(self.ctx.lib.sbv_mlp_train(self.h, _ptr(X), _ptr(t), X.shape[0], steps, batch,
                                                   lr, seed, C.byref(loss), _stream(stream)))
        return loss.value

    def predict(self, X, want_grad=False, stream=None):
        X = self._rows(X)
        s = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        g = torch.empty(X.shape[0], self.in_dim, dtype=torch.float32, device=X.device) if want_grad else None
        self.ctx._check(self.ctx.lib.sbv_mlp_predict(self.h, _ptr(X), X.shape[0], _ptr(s), _ptr(g),
                                                     _stream(stream)))
        return (s, g) if want_grad else s
