"""Python front end of the C-ABI: a handle class over torch device tensors.

Vectors are torch complex128 tensors of shape (n,) or (n, nrhs); the library wants them
column-major, so an (n, nrhs) tensor is passed as the contiguous (nrhs, n) transpose.
Every computation runs in libd3m.so; this file only moves pointers.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, c_double, c_int32, c_void_p

import numpy as np

from . import _abi
from ._abi import check, load

PRECISIONS = {"fp64": _abi.D3M_FP64, "bf16x3": _abi.D3M_MIXED_BF16X3, "simt32": _abi.D3M_MIXED_SIMT32,
              "tf32": _abi.D3M_MIXED_TF32}


def _stream_ptr(stream=None) -> int:
    import torch
    if stream is None and not torch.cuda.is_available():
        return 0          # default stream; only host-side validation can run without a device
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _as_colmajor(B):
    """(n,) or (n, nrhs) -> contiguous (nrhs, n) complex128 tensor and nrhs."""
    import torch
    if B.dtype != torch.complex128:
        raise TypeError("right-hand sides must be complex128")
    # lazy conjugate / negative views would hand the raw (unconjugated) data to the library
    B = B.resolve_conj().resolve_neg()
    if B.dim() == 1:
        return B.contiguous().reshape(1, -1), 1, True
    return B.T.contiguous(), B.shape[1], False


def _options(precision, max_nrhs, refine_tol, refine_max_iter, timeout_ns, fp64_omega, debug_flags, graphs=False,
             prio_slack=None, seg_group=0, task_cost=None, pivot=False):
    opt = _abi.d3m_default_options()
    opt.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    opt.max_nrhs = max_nrhs
    opt.refine_tol = refine_tol
    opt.refine_max_iter = refine_max_iter
    if timeout_ns:
        opt.timeout_ns = timeout_ns
    opt.fp64_omega = int(fp64_omega)
    opt.debug_flags = debug_flags
    opt.graphs = int(graphs)
    if prio_slack is not None:
        opt.prio_slack = float(prio_slack)
    opt.seg_group = int(seg_group)
    if task_cost is not None:
        for q in range(6):
            opt.task_cost[q] = float(task_cost[q])
    opt.pivot = int(bool(pivot))
    return opt


class D3M:
    """One factorization handle (d3m_create ... d3m_destroy)."""

    def __init__(self, colptr, rowidx, m=None, blk_size=None, perm=None, precision="bf16x3",
                 max_nrhs: int = 32, refine_tol: float = 1e-12, refine_max_iter: int = 20,
                 timeout_ns: int = 0, fp64_omega: bool = False, debug_flags: int = 0, graphs: bool = False,
                 prio_slack=None, seg_group: int = 0, task_cost=None, pivot: bool = False, stream=None):
        lib = load()
        self._lib = lib
        self.h = c_void_p()
        pat, self._keep = _abi.make_pattern(colptr, rowidx, m, blk_size)
        opt = _options(precision, max_nrhs, refine_tol, refine_max_iter, timeout_ns, fp64_omega, debug_flags, graphs,
                       prio_slack, seg_group, task_cost, pivot)
        pp = None
        if perm is not None:
            self._perm = np.ascontiguousarray(perm, dtype=np.int32)
            pp = self._perm.ctypes.data_as(POINTER(c_int32))
        self.precision = precision
        self.stream = stream
        rc = lib.d3m_create(ctypes.byref(self.h), ctypes.byref(pat), pp, ctypes.byref(opt),
                            c_void_p(_stream_ptr(stream)))
        check(rc, None if not self.h else self.h)
        self.n = int(np.sum(blk_size)) if blk_size is not None else int(m) * (len(colptr) - 1)

    # -------------------------------------------------------------- C-ABI calls
    def factor(self, K):
        """K: complex128 lower blocks (torch tensor on the device, or pinned/host)."""
        if hasattr(K, "resolve_conj"):
            K = K.resolve_conj().resolve_neg().contiguous()
        ptr = K.data_ptr() if hasattr(K, "data_ptr") else K.ctypes.data
        return check(self._lib.d3m_factor(self.h, c_void_p(ptr), c_void_p(_stream_ptr(self.stream))), self.h)

    def solve(self, B, X=None, allow_not_converged: bool = False):
        import torch
        Bt, nrhs, vec = _as_colmajor(B)
        Xt = torch.empty_like(Bt) if X is None else X
        rc = self._lib.d3m_solve(self.h, c_void_p(Bt.data_ptr()), c_void_p(Xt.data_ptr()), nrhs,
                                 c_void_p(_stream_ptr(self.stream)))
        if not (allow_not_converged and rc == _abi.D3M_ERR_NOT_CONVERGED):
            check(rc, self.h)
        return Xt.reshape(-1) if vec else Xt.T

    def adjoint(self, G):
        import torch
        Gt, nrhs, vec = _as_colmajor(G)
        Lt = torch.empty_like(Gt)
        check(self._lib.d3m_adjoint(self.h, c_void_p(Gt.data_ptr()), c_void_p(Lt.data_ptr()), nrhs,
                                    c_void_p(_stream_ptr(self.stream))), self.h)
        return Lt.reshape(-1) if vec else Lt.T

    def grad_eps(self, Lam, X, dom_if, k2: float, noalloc: bool = False):
        """dJ/deps per domain; noalloc=True calls d3m_grad_eps_noalloc (no allocation inside)."""
        Lt, nrhs, _ = _as_colmajor(Lam)
        Xt, _, _ = _as_colmajor(X)
        ptr = np.zeros(len(dom_if) + 1, dtype=np.int32)
        for i, I in enumerate(dom_if):
            ptr[i + 1] = ptr[i] + len(I)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(I, dtype=np.int32) for I in dom_if])
                                    if len(dom_if) else np.zeros(0), dtype=np.int32)
        out = np.zeros(len(dom_if), dtype=np.float64)
        fn = self._lib.d3m_grad_eps_noalloc if noalloc else self._lib.d3m_grad_eps
        check(fn(self.h, c_void_p(Lt.data_ptr()), c_void_p(Xt.data_ptr()), nrhs,
                                     len(dom_if), ptr.ctypes.data_as(POINTER(c_int32)),
                                     flat.ctypes.data_as(POINTER(c_int32)), c_double(k2),
                                     out.ctypes.data_as(POINTER(c_double)),
                                     c_void_p(_stream_ptr(self.stream))), self.h)
        return out

    def grad_pattern(self, Lam, X, nvals: int):
        import torch
        Lt, nrhs, _ = _as_colmajor(Lam)
        Xt, _, _ = _as_colmajor(X)
        dK = torch.empty(nvals, dtype=torch.complex128, device=Lt.device)
        check(self._lib.d3m_grad_pattern(self.h, c_void_p(Lt.data_ptr()), c_void_p(Xt.data_ptr()), nrhs,
                                         c_void_p(dK.data_ptr()), c_void_p(_stream_ptr(self.stream))), self.h)
        return dK

    def factor_block(self, i: int, j: int, mi: int, mj: int) -> np.ndarray:
        out = np.zeros(mi * mj, dtype=np.complex128)
        check(self._lib.d3m_get_factor_block(self.h, i, j, c_void_p(out.ctypes.data),
                                             c_void_p(_stream_ptr(self.stream))), self.h)
        return out.reshape(mj, mi).T

    def pivots(self, j: int, mj: int) -> np.ndarray:
        out = np.zeros(mj, dtype=np.complex128)
        check(self._lib.d3m_get_pivots(self.h, j, c_void_p(out.ctypes.data), c_void_p(_stream_ptr(self.stream))),
              self.h)
        return out

    def pivot_blocks(self, j: int, mj: int):
        """(e, perm) of block column j: 2 x 2 sub-diagonals of D_j (c128) and the pivot order."""
        e = np.zeros(mj, dtype=np.complex128)
        perm = np.zeros(mj, dtype=np.int32)
        check(self._lib.d3m_get_pivot_blocks(self.h, j, c_void_p(e.ctypes.data), perm.ctypes.data_as(POINTER(c_int32)),
                                             c_void_p(_stream_ptr(self.stream))), self.h)
        return e, perm

    def trace(self) -> np.ndarray:
        """Task records of the last factorization (handle created with debug_flags=2):
        int64 [ntasks, 10] = start_ns, end_ns, sm_id, flags | tile << 8 | nk << 40, t1..t4, ready_ns,
        releaser (task id = row; flags 1 = diagonal tile, 4 = update task; nk = tile products)."""
        cnt = ctypes.c_int64()
        check(self._lib.d3m_get_trace(self.h, None, 0, ctypes.byref(cnt), c_void_p(_stream_ptr(self.stream))), self.h)
        out = np.zeros((cnt.value, 10), dtype=np.int64)
        check(self._lib.d3m_get_trace(self.h, c_void_p(out.ctypes.data), cnt.value, ctypes.byref(cnt),
                                      c_void_p(_stream_ptr(self.stream))), self.h)
        return out

    def info(self) -> dict:
        inf = _abi.d3m_info()
        check(self._lib.d3m_get_info(self.h, ctypes.byref(inf), c_void_p(_stream_ptr(self.stream))), self.h)
        return inf.as_dict()

    def last_error(self) -> str:
        return self._lib.d3m_last_error(self.h).decode()

    def close(self):
        if getattr(self, "h", None) and self.h:
            self._lib.d3m_destroy(self.h)
            self.h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class D3MBatch(D3M):
    """Many independent systems in one handle (d3m_create_batch): one persistent factorization
    launch for all of them and level-merged solve sweeps.  `instances` is a list of
    (colptr, rowidx, m_or_blk_size) tuples; `perms` a list of per-instance perms (or None).
    K, B and X are the instances' own arrays concatenated in instance order."""

    def __init__(self, instances, perms=None, precision="bf16x3", max_nrhs: int = 32, refine_tol: float = 1e-12,
                 refine_max_iter: int = 20, timeout_ns: int = 0, fp64_omega: bool = False, debug_flags: int = 0,
                 graphs: bool = False, task_cost=None, stream=None):
        lib = load()
        self._lib = lib
        self.h = c_void_p()
        count = len(instances)
        pats = (_abi.d3m_pattern * count)()
        self._keep = []
        self.sizes = []
        for i, (colptr, rowidx, msz) in enumerate(instances):
            if np.isscalar(msz):
                pat, keep = _abi.make_pattern(colptr, rowidx, int(msz), None)
                self.sizes.append(int(msz) * (len(colptr) - 1))
            else:
                pat, keep = _abi.make_pattern(colptr, rowidx, None, msz)
                self.sizes.append(int(np.sum(msz)))
            pats[i] = pat
            self._keep.append(keep)
        pp = None
        if perms is not None:
            self._perms = [None if q is None else np.ascontiguousarray(q, dtype=np.int32) for q in perms]
            pp = (POINTER(c_int32) * count)(*[
                ctypes.cast(None, POINTER(c_int32)) if q is None else q.ctypes.data_as(POINTER(c_int32))
                for q in self._perms])
        opt = _options(precision, max_nrhs, refine_tol, refine_max_iter, timeout_ns, fp64_omega, debug_flags, graphs,
                       task_cost=task_cost)
        self.precision = precision
        self.stream = stream
        rc = lib.d3m_create_batch(ctypes.byref(self.h), count, pats, pp, ctypes.byref(opt),
                                  c_void_p(_stream_ptr(stream)))
        check(rc, None if not self.h else self.h)
        self.count = count
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.n = int(self.offsets[-1])

    def instance_omega(self) -> np.ndarray:
        out = np.zeros(self.count, dtype=np.float64)
        check(self._lib.d3m_get_instance_omega(self.h, out.ctypes.data_as(POINTER(c_double)),
                                               c_void_p(_stream_ptr(self.stream))), self.h)
        return out
