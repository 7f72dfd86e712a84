"""Thin Python binding of libhrp.so (include/hrp.h), argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only turns torch
CUDA tensors into device pointers and streams into ``cudaStream_t`` handles.

Layout convention: the C ABI takes column-major matrices.  A column-major m x n
matrix with leading dimension ld is held here in a row-major torch tensor ``T`` of
shape (n, ld) with ``T[j, i] = M(i, j)``; ``colmajor()`` / ``from_colmajor()``
convert numpy arrays to and from that form.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhrp.so")

HRP_MAX_DEPTH = 16
PREC = {"F64": 0, "F32": 1, "F16": 2, "F8": 3}
PREC_NAME = {v: k for k, v in PREC.items()}
STATUS = {0: "HRP_OK", 1: "HRP_ERR_INVALID_ARG", 2: "HRP_ERR_NOT_SPD", 3: "HRP_ERR_NO_CONVERGENCE",
          4: "HRP_ERR_ALLOC", 5: "HRP_ERR_CUDA", 6: "HRP_ERR_TIMEOUT", 7: "HRP_ERR_UNSUPPORTED",
          8: "HRP_ERR_RANGE"}

EXPORTED = [
    "hrp_create", "hrp_destroy", "hrp_last_arg", "hrp_last_error", "hrp_status_string",
    "hrp_tree_parse", "hrp_tree_format", "hrp_potrf", "hrp_potrf_async", "hrp_potrf_host", "hrp_potrs",
    "hrp_posv", "hrp_backward_error", "hrp_set_timing", "hrp_get_timing", "hrp_last_launch_count",
    "hrp_potrs_noalloc", "hrp_potrf_batched", "hrp_potrs_batched", "hrp_posv_batched",
    "hrp_policy_features", "hrp_mlp_forward", "hrp_mlp_grad", "hrp_mlp_adam", "hrp_mlp_param_count",
    "hrp_policy_set", "hrp_policy_predict", "hrp_policy_tree", "hrp_last_policy_choice",
    "hrp_autotune_candidates", "hrp_autotune", "hrp_policy_load", "hrp_check", "hrp_set_wait_limit",
    "hrp_wait_selftest", "hrp_set_lookahead", "hrp_syrk", "hrp_trsm", "hrp_set_refinement",
    "hrp_last_inner_iterations", "hrp_autotune_orders", "hrp_set_batched_mode", "hrp_set_scaling",
    "hrp_set_fp32_split", "hrp_set_f8_gemm", "hrp_set_leaf_chain", "hrp_get_timeline", "hrp_policy_set_min_order",
]


class Tree(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("level", ctypes.c_int * HRP_MAX_DEPTH), ("leaf", ctypes.c_int),
                ("inner", ctypes.c_int), ("inner_size", ctypes.c_int), ("trsm_leaf", ctypes.c_int),
                ("syrk_leaf", ctypes.c_int), ("scale_block", ctypes.c_int), ("trsm_compute", ctypes.c_int),
                ("tile_occupancy", ctypes.c_int)]


class HrpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libhrp.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2601_08082_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, ip, dp, c_int, c_double = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), \
        ctypes.c_int, ctypes.c_double
    tp = ctypes.POINTER(Tree)
    L.hrp_create.argtypes = [ctypes.POINTER(vp), c_int]
    L.hrp_destroy.argtypes = [vp]
    L.hrp_last_arg.argtypes = [vp]
    L.hrp_last_error.argtypes = [vp]
    L.hrp_last_error.restype = ctypes.c_char_p
    L.hrp_status_string.argtypes = [c_int]
    L.hrp_status_string.restype = ctypes.c_char_p
    L.hrp_tree_parse.argtypes = [ctypes.c_char_p, c_int, tp]
    L.hrp_tree_format.argtypes = [tp, ctypes.c_char_p, ctypes.c_size_t]
    L.hrp_potrf.argtypes = [vp, tp, c_int, vp, c_int, ip, vp]
    L.hrp_potrf_async.argtypes = [vp, tp, c_int, vp, c_int, vp, vp]
    L.hrp_potrf_host.argtypes = [vp, tp, c_int, vp, c_int, vp, c_int, vp, vp]
    L.hrp_potrs.argtypes = [vp, c_int, c_int, vp, c_int, vp, c_int, vp]
    L.hrp_posv.argtypes = [vp, tp, c_int, c_int, vp, c_int, vp, c_int, vp, c_int, c_int, c_double, ip, dp, ip, ip, vp]
    L.hrp_backward_error.argtypes = [vp, c_int, vp, c_int, vp, c_int, dp, vp]
    L.hrp_set_timing.argtypes = [vp, c_int]
    L.hrp_set_lookahead.argtypes = [vp, c_int]
    L.hrp_set_batched_mode.argtypes = [vp, c_int]
    L.hrp_set_scaling.argtypes = [vp, c_int]
    L.hrp_set_fp32_split.argtypes = [vp, c_int]
    L.hrp_set_f8_gemm.argtypes = [vp, c_int]
    L.hrp_set_leaf_chain.argtypes = [vp, c_int]
    L.hrp_get_timeline.argtypes = [vp, vp, c_int]
    L.hrp_policy_set_min_order.argtypes = [vp, c_int]
    L.hrp_set_refinement.argtypes = [vp, c_int, c_int, c_double]
    L.hrp_last_inner_iterations.argtypes = [vp]
    L.hrp_last_inner_iterations.restype = ctypes.c_longlong
    L.hrp_syrk.argtypes = [vp, tp, c_int, c_int, vp, c_int, vp, c_int, vp]
    L.hrp_trsm.argtypes = [vp, tp, c_int, c_int, vp, c_int, vp, c_int, vp]
    L.hrp_get_timing.argtypes = [vp, dp, c_int]
    L.hrp_last_launch_count.argtypes = [vp]
    L.hrp_last_launch_count.restype = ctypes.c_longlong
    L.hrp_potrs_noalloc.argtypes = [c_int, c_int, vp, c_int, vp, c_int, vp]
    L.hrp_potrf_batched.argtypes = [vp, vp, c_int, vp, vp, vp, vp, vp]
    L.hrp_potrs_batched.argtypes = [vp, c_int, vp, vp, vp, c_int, vp, vp, vp]
    L.hrp_posv_batched.argtypes = [vp, vp, c_int, vp, vp, vp, c_int, vp, vp, vp, vp, c_int, c_double, ip, ip, dp,
                                   ip, vp]
    fp = ctypes.POINTER(ctypes.c_float)
    L.hrp_policy_features.argtypes = [vp, c_int, vp, c_int, c_int, fp, vp]
    L.hrp_mlp_forward.argtypes = [vp, vp, c_int, vp, vp, vp]
    L.hrp_mlp_grad.argtypes = [vp, vp, c_int, vp, vp, vp, vp, vp]
    L.hrp_mlp_adam.argtypes = [vp, vp, vp, vp, vp, c_int, ctypes.c_float, vp]
    L.hrp_mlp_param_count.argtypes = []
    L.hrp_policy_set.argtypes = [vp, fp, fp, fp]
    L.hrp_policy_predict.argtypes = [vp, fp, tp, ip]
    L.hrp_policy_load.argtypes = [vp, ctypes.c_char_p]
    L.hrp_check.argtypes = [vp, vp]
    L.hrp_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    L.hrp_wait_selftest.argtypes = [vp, ctypes.c_longlong, dp, vp]
    L.hrp_policy_tree.argtypes = [c_int, tp]
    L.hrp_last_policy_choice.argtypes = [vp]
    L.hrp_autotune_candidates.argtypes = [tp, vp, c_int]
    L.hrp_autotune.argtypes = [vp, tp, c_int, c_int, c_int, tp, fp, vp]
    L.hrp_autotune_orders.argtypes = [vp, tp, c_int, vp, c_int, vp]
    _lib = L
    return L


def tree_parse(spec: str, leaf: int = 128, trsm_leaf: int = 0, syrk_leaf: int = 0,
               trsm_fp64: bool = False, tile_occupancy: int = 0) -> Tree:
    t = Tree()
    st = load().hrp_tree_parse(spec.encode(), leaf, ctypes.byref(t))
    if st != 0:
        raise HrpError(st, f"bad tree spec {spec!r}")
    t.trsm_leaf = trsm_leaf
    t.syrk_leaf = syrk_leaf
    t.trsm_compute = 1 if trsm_fp64 else 0
    t.tile_occupancy = tile_occupancy
    return t


def tree_format(t: Tree) -> str:
    buf = ctypes.create_string_buffer(256)
    load().hrp_tree_format(ctypes.byref(t), buf, 256)
    return buf.value.decode()


def colmajor(a: np.ndarray):
    """numpy (m, n) -> torch CPU float64 tensor (n, m) holding the column-major matrix."""
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return torch.from_numpy(np.ascontiguousarray(a.T))


def from_colmajor(t, m: int | None = None) -> np.ndarray:
    """torch tensor (n, ld) column-major storage -> numpy (m, n)."""
    a = t.detach().cpu().numpy().T
    return a if m is None else a[:m]


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class Handle:
    """Owns an hrp_handle (workspace, streams' scratch) on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = load()
        self._h = ctypes.c_void_p()
        st = self._lib.hrp_create(ctypes.byref(self._h), device)
        if st != 0:
            raise HrpError(st, "hrp_create failed")
        self.device = device

    def close(self):
        if self._h:
            self._lib.hrp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, allow=()):
        if st != 0 and st not in allow:
            raise HrpError(st, self._lib.hrp_last_error(self._h).decode())
        return st

    def last_arg(self) -> int:
        return self._lib.hrp_last_arg(self._h)

    def launch_count(self) -> int:
        return self._lib.hrp_last_launch_count(self._h)

    def syrk(self, tree: Tree, A, C, stream=None) -> None:
        """C (n, ldc) column-major, lower triangle -= A A^T with A (k, lda) column-major n x k."""
        n, k = C.shape[0], A.shape[0]
        self._check(self._lib.hrp_syrk(self._h, ctypes.byref(tree), n, k, _ptr(A), A.shape[1], _ptr(C), C.shape[1],
                                       _stream(stream)))

    def trsm(self, tree: Tree, L, B, stream=None) -> None:
        """B (n, ldb) column-major m x n <- B L^{-T}, L (n, ldl) column-major lower."""
        n, m = L.shape[0], B.shape[1]
        self._check(self._lib.hrp_trsm(self._h, ctypes.byref(tree), m, n, _ptr(L), L.shape[1], _ptr(B), B.shape[1],
                                       _stream(stream)))

    def set_refinement(self, gmres: bool, restart: int = 20, inner_tol: float = 1e-8) -> None:
        """hrp_set_refinement: classical refinement, or GMRES-IR with this restart and tolerance."""
        self._check(self._lib.hrp_set_refinement(self._h, 1 if gmres else 0, restart, inner_tol))

    def inner_iterations(self) -> int:
        return self._lib.hrp_last_inner_iterations(self._h)

    def set_scaling(self, dynamic: bool) -> None:
        """hrp_set_scaling: two-sided power-of-two diagonal scaling before the recursion."""
        self._check(self._lib.hrp_set_scaling(self._h, 1 if dynamic else 0))

    def set_leaf_chain(self, mode: int) -> None:
        """hrp_set_leaf_chain: FP64 leaves in double-float arithmetic (1), in FP64 (0), or by
        tree (-1, default: double-float when the tree has a level below FP64)."""
        self._check(self._lib.hrp_set_leaf_chain(self._h, int(mode)))

    def set_f8_gemm(self, fp16_storage: bool) -> None:
        """hrp_set_f8_gemm: F8 levels by block-scaled E4M3 MMAs (False, default) or through
        FP16 storage on the FP16 GEMM (True)."""
        self._check(self._lib.hrp_set_f8_gemm(self._h, 1 if fp16_storage else 0))

    def set_fp32_split(self, on: bool) -> None:
        """hrp_set_fp32_split: FP32-level GEMMs by the TF32 split on tensor cores."""
        self._check(self._lib.hrp_set_fp32_split(self._h, 1 if on else 0))

    def set_batched_mode(self, persistent: bool) -> None:
        """hrp_set_batched_mode: one persistent launch (True) or one stream per system (False)."""
        self._check(self._lib.hrp_set_batched_mode(self._h, 1 if persistent else 0))

    def set_lookahead(self, enable: bool) -> None:
        self._check(self._lib.hrp_set_lookahead(self._h, 1 if enable else 0))

    # hrp_potrf: A is a column-major (n, lda) float64 CUDA tensor, overwritten with L
    def potrf(self, tree: Tree, A, n: int | None = None, stream=None, raise_not_spd: bool = False) -> int:
        n = A.shape[0] if n is None else n
        lda = A.shape[1]
        info = ctypes.c_int(0)
        st = self._lib.hrp_potrf(self._h, ctypes.byref(tree), n, _ptr(A), lda, ctypes.byref(info), _stream(stream))
        self._check(st, allow=() if raise_not_spd else (2,))
        return info.value

    def potrf_async(self, tree: Tree, A, d_info, n: int | None = None, stream=None) -> None:
        n = A.shape[0] if n is None else n
        st = self._lib.hrp_potrf_async(self._h, ctypes.byref(tree), n, _ptr(A), A.shape[1], _ptr(d_info),
                                       _stream(stream))
        self._check(st)

    def potrf_host(self, tree: Tree, hA, A, d_info, n: int | None = None, stream=None) -> None:
        """hrp_potrf_host: hA a column-major (n, ldha) float64 CPU tensor (page-locked for the
        overlap), A the column-major (n, lda) CUDA tensor that receives its lower triangle and L."""
        n = A.shape[0] if n is None else n
        st = self._lib.hrp_potrf_host(self._h, ctypes.byref(tree), n, _ptr(hA), hA.shape[1], _ptr(A), A.shape[1],
                                      _ptr(d_info), _stream(stream))
        self._check(st)

    # hrp_potrs: L (n, ldl) column-major factor, B (nrhs, ldb) column-major, overwritten with X
    def potrs(self, L, B, n: int | None = None, stream=None) -> None:
        n = L.shape[0] if n is None else n
        nrhs = B.shape[0]
        st = self._lib.hrp_potrs(self._h, n, nrhs, _ptr(L), L.shape[1], _ptr(B), B.shape[1], _stream(stream))
        self._check(st)

    def posv(self, tree, A, B, X, max_iter: int = 30, tol: float = 1e-12, n: int | None = None,
             stream=None, raise_errors: bool = False) -> dict:
        """tree=None: the learned policy chooses the tree (see policy_set)."""
        n = A.shape[0] if n is None else n
        nrhs = B.shape[0]
        iters, info, fb = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        resid = ctypes.c_double(0.0)
        tref = ctypes.byref(tree) if tree is not None else None
        st = self._lib.hrp_posv(self._h, tref, n, nrhs, _ptr(A), A.shape[1], _ptr(B), B.shape[1],
                                _ptr(X), X.shape[1], max_iter, tol, ctypes.byref(iters), ctypes.byref(resid),
                                ctypes.byref(info), ctypes.byref(fb), _stream(stream))
        self._check(st, allow=() if raise_errors else (2, 3))
        return {"status": st, "iters": iters.value, "resid": resid.value, "info": info.value,
                "used_fallback": fb.value}

    # batched: lists of column-major CUDA tensors; trees: one Tree or a list of Trees
    @staticmethod
    def _tree_array(trees, batch):
        """trees: one Tree, a list (None entries: the policy chooses) or None (policy for all)."""
        if trees is None:
            return None, ctypes.c_void_p(0)
        if isinstance(trees, Tree):
            trees = [trees] * batch
        keep = list(trees)
        arr = (ctypes.POINTER(Tree) * batch)(*[ctypes.pointer(t) if t is not None else ctypes.POINTER(Tree)()
                                               for t in keep])
        return (keep, arr), ctypes.cast(arr, ctypes.c_void_p)

    def potrf_batched(self, trees, As, d_info, stream=None) -> None:
        batch = len(As)
        keep, tptr = self._tree_array(trees, batch)
        n = (ctypes.c_int * batch)(*[A.shape[0] for A in As])
        lda = (ctypes.c_int * batch)(*[A.shape[1] for A in As])
        ptrs = (ctypes.c_void_p * batch)(*[A.data_ptr() for A in As])
        st = self._lib.hrp_potrf_batched(self._h, tptr, batch, n, ptrs, lda, _ptr(d_info), _stream(stream))
        self._check(st)

    def potrs_batched(self, Ls, Bs, stream=None) -> None:
        batch = len(Ls)
        n = (ctypes.c_int * batch)(*[L.shape[0] for L in Ls])
        ldl = (ctypes.c_int * batch)(*[L.shape[1] for L in Ls])
        lp = (ctypes.c_void_p * batch)(*[L.data_ptr() for L in Ls])
        nrhs = Bs[0].shape[0] if batch else 0
        ldb = (ctypes.c_int * batch)(*[B.shape[1] for B in Bs])
        bp = (ctypes.c_void_p * batch)(*[B.data_ptr() for B in Bs])
        st = self._lib.hrp_potrs_batched(self._h, batch, n, lp, ldl, nrhs, bp, ldb, _stream(stream))
        self._check(st)

    # ---- learned policy ----
    TIMING_CLASSES = ("leaf_potrf_fp64", "leaf_trsm", "gemm_f16_tcgen05", "gemm_simt", "other")

    def timing(self, tree, A, n: int | None = None) -> dict:
        """Factor A once with per-launch event timing; per kernel class: device ms,
        launches and the algorithmic flops those launches did (hrp_get_timing)."""
        n = A.shape[0] if n is None else n
        self._lib.hrp_set_timing(self._h, 1)
        try:
            self.potrf(tree, A, n=n)
            buf = (ctypes.c_double * 15)()
            if self._lib.hrp_get_timing(self._h, buf, 15) != 15:
                raise HrpError("hrp_get_timing returned fewer than 15 values")
        finally:
            self._lib.hrp_set_timing(self._h, 0)
        return {name: {"ms": buf[3 * c], "launches": int(buf[3 * c + 1]), "flops": buf[3 * c + 2]}
                for c, name in enumerate(self.TIMING_CLASSES)}

    def timeline(self) -> np.ndarray:
        """hrp_get_timeline after timing(): one row per launch (class, stream, start ms, end ms)."""
        cap = 4 * 200000
        buf = (ctypes.c_double * cap)()
        w = self._lib.hrp_get_timeline(self._h, buf, cap)
        return np.array(buf[:w], dtype=np.float64).reshape(-1, 4)

    def policy_features(self, A, lanczos_steps: int = 10, n: int | None = None, stream=None) -> np.ndarray:
        n = A.shape[0] if n is None else n
        f = (ctypes.c_float * 12)()
        st = self._lib.hrp_policy_features(self._h, n, _ptr(A), A.shape[1], lanczos_steps, f, _stream(stream))
        self._check(st)
        return np.array(f[:], dtype=np.float32)

    def mlp_forward(self, params, X, Z, stream=None) -> None:
        self._check(self._lib.hrp_mlp_forward(self._h, _ptr(params), X.shape[0], _ptr(X), _ptr(Z), _stream(stream)))

    def mlp_grad(self, params, X, y, grad, loss, stream=None) -> None:
        self._check(self._lib.hrp_mlp_grad(self._h, _ptr(params), X.shape[0], _ptr(X), _ptr(y), _ptr(grad),
                                           _ptr(loss), _stream(stream)))

    def mlp_adam(self, params, grad, m, v, step: int, lr: float, stream=None) -> None:
        self._check(self._lib.hrp_mlp_adam(self._h, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr,
                                           _stream(stream)))

    def policy_set(self, params, mean, scale) -> None:
        def fa(a):
            a = np.ascontiguousarray(a, dtype=np.float32)
            return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        (p, pp), (m, mp), (s, sp) = fa(params), fa(mean), fa(scale)
        self._check(self._lib.hrp_policy_set(self._h, pp, mp, sp))

    def policy_predict(self, feat) -> int:
        return self.policy_predict_tree(feat)[1]

    def policy_predict_tree(self, feat) -> tuple[Tree, int]:
        f = np.ascontiguousarray(feat, dtype=np.float32)
        idx = ctypes.c_int(-1)
        t = Tree()
        self._check(self._lib.hrp_policy_predict(self._h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                 ctypes.byref(t), ctypes.byref(idx)))
        return t, idx.value

    def policy_load(self, path: str) -> None:
        self._check(self._lib.hrp_policy_load(self._h, os.fsencode(path)))

    def policy_set_min_order(self, n_min: int) -> None:
        """hrp_policy_set_min_order: orders below n_min take the fallback tree, no features."""
        self._check(self._lib.hrp_policy_set_min_order(self._h, int(n_min)))

    def check(self, stream=None) -> int:
        """hrp_check: status of the device-side failures since the last synchronous call."""
        return self._lib.hrp_check(self._h, _stream(stream))

    def set_wait_limit(self, microseconds: int) -> None:
        self._check(self._lib.hrp_set_wait_limit(self._h, int(microseconds)))

    def wait_selftest(self, microseconds: int, stream=None) -> tuple[int, float]:
        """(status, microseconds the device waited) of a bounded wait on a flag nothing sets."""
        w = ctypes.c_double(0.0)
        st = self._lib.hrp_wait_selftest(self._h, int(microseconds), ctypes.byref(w), _stream(stream))
        return st, w.value

    def last_policy_choice(self) -> int:
        return self._lib.hrp_last_policy_choice(self._h)

    def posv_batched(self, trees, As, Bs, Xs, max_iter: int = 30, tol: float = 1e-12, stream=None) -> dict:
        batch = len(As)
        keep, tptr = self._tree_array(trees, batch)
        arr_i = lambda v: (ctypes.c_int * batch)(*v)
        arr_p = lambda ts: (ctypes.c_void_p * batch)(*[t.data_ptr() for t in ts])
        info, iters, fb = arr_i([0] * batch), arr_i([0] * batch), arr_i([0] * batch)
        resid = (ctypes.c_double * batch)()
        nrhs = Bs[0].shape[0] if batch else 1
        st = self._lib.hrp_posv_batched(self._h, tptr, batch,
                                        arr_i([A.shape[0] for A in As]), arr_p(As), arr_i([A.shape[1] for A in As]),
                                        nrhs, arr_p(Bs), arr_i([B.shape[1] for B in Bs]), arr_p(Xs),
                                        arr_i([X.shape[1] for X in Xs]), max_iter, tol, info, iters, resid, fb,
                                        _stream(stream))
        self._check(st, allow=(2, 3))
        return {"status": st, "info": list(info), "iters": list(iters), "resid": list(resid),
                "used_fallback": list(fb)}

    def autotune(self, tree: Tree, n: int, reps: int = 3, retune: bool = False, stream=None) -> tuple[Tree, float]:
        """(fastest valid candidate tree for order n, its median ms); see hrp_autotune."""
        out = Tree()
        ms = ctypes.c_float(0.0)
        st = self._lib.hrp_autotune(self._h, ctypes.byref(tree), n, reps, 1 if retune else 0, ctypes.byref(out),
                                    ctypes.byref(ms), _stream(stream))
        self._check(st)
        return out, float(ms.value)

    def autotune_orders(self, tree: Tree, orders, reps: int = 2, stream=None) -> None:
        """hrp_autotune_orders: tune each order; the batched calls then use the tuned cut-offs."""
        arr = (ctypes.c_int * len(orders))(*[int(o) for o in orders])
        self._check(self._lib.hrp_autotune_orders(self._h, ctypes.byref(tree), len(orders), arr, reps, _stream(stream)))

    def backward_error(self, A, L, n: int | None = None, stream=None) -> float:
        n = A.shape[0] if n is None else n
        out = ctypes.c_double(0.0)
        st = self._lib.hrp_backward_error(self._h, n, _ptr(A), A.shape[1], _ptr(L), L.shape[1], ctypes.byref(out),
                                          _stream(stream))
        self._check(st)
        return out.value


def autotune_candidates(tree: Tree) -> list[Tree]:
    """The autotuner's candidate trees for `tree` (host only): the given tree first."""
    L = load()
    cap = 32
    arr = (Tree * cap)()
    cnt = L.hrp_autotune_candidates(ctypes.byref(tree), ctypes.cast(arr, ctypes.c_void_p), cap)
    if cnt < 0:
        raise HrpError(1, "invalid tree")
    return [arr[i] for i in range(min(cnt, cap))]


def policy_tree(index: int) -> Tree:
    t = Tree()
    st = load().hrp_policy_tree(index, ctypes.byref(t))
    if st != 0:
        raise HrpError(st, f"no policy tree {index}")
    return t


def mlp_param_count() -> int:
    return load().hrp_mlp_param_count()
