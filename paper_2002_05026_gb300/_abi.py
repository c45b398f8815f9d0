"""ctypes binding of libd3m.so: the C-ABI of include/d3m.h, same names, marshalling only.

Loading fails loudly when the library has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libd3m.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "d3m.h")

D3M_OK = 0
D3M_ERR_INVALID = 1
D3M_ERR_OOM = 2
D3M_ERR_CUDA = 3
D3M_ERR_PIVOT = 4
D3M_ERR_NOT_CONVERGED = 5
D3M_ERR_TIMEOUT = 6
D3M_ERR_STATE = 7

D3M_FP64 = 0
D3M_MIXED_BF16X3 = 1
D3M_MIXED_SIMT32 = 2
D3M_MIXED_TF32 = 3

D3M_DEBUG_STALL_LAST_TASK = 1
D3M_DEBUG_TRACE = 2

ERROR_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "PIVOT", 5: "NOT_CONVERGED",
               6: "TIMEOUT", 7: "STATE"}


class d3m_pattern(ctypes.Structure):
    _fields_ = [("nblk", c_int32), ("m", c_int32), ("blk_size", POINTER(c_int32)),
                ("colptr", POINTER(c_int64)), ("rowidx", POINTER(c_int32))]


class d3m_options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("refine_max_iter", c_int32), ("refine_tol", c_double),
                ("timeout_ns", c_int64), ("tile", c_int32), ("max_nrhs", c_int32),
                ("fp64_omega", c_int32), ("debug_flags", c_int32), ("graphs", c_int32), ("seg_group", c_int32),
                ("prio_slack", c_double), ("refine_fwd_tol", c_double), ("task_cost", c_double * 6),
                ("pivot", c_int32)]


class d3m_info(ctypes.Structure):
    _fields_ = [("n", c_int64), ("nblk", c_int32), ("tile", c_int32), ("nnzb_K", c_int64),
                ("nblk_L_offdiag", c_int64), ("etree_depth", c_int32), ("max_col_height", c_int32),
                ("ntiles", c_int64), ("ntile_updates", c_int64), ("ndep_edges", c_int64),
                ("factor_flops", c_double), ("solve_flops_per_rhs", c_double),
                ("residual_flops_per_rhs", c_double), ("device_bytes", c_int64),
                ("status", c_int32), ("refine_iters", c_int32), ("omega", c_double),
                ("omega_first", c_double), ("min_abs_pivot", c_double), ("max_abs_pivot", c_double),
                ("factor_kernel_ms", c_double), ("solve_ms", c_double), ("residual_ms", c_double),
                ("kernel_launches", c_int64), ("factor_kernel_ms_total", c_double),
                ("residual_ms_total", c_double), ("sweep_ms_total", c_double),
                ("factor_kernel_calls", c_int64), ("residual_calls", c_int64), ("sweep_calls", c_int64),
                ("instances", c_int32), ("reserved0", c_int32), ("prio_tasks", c_int64),
                ("residual_bytes_fixed", c_double), ("residual_bytes_per_rhs", c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load() -> ctypes.CDLL:
    """Load the in-tree library (build it with paper_2002_05026_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libd3m.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    P = POINTER
    sig = {
        "d3m_default_options": (None, [P(d3m_options)]),
        "d3m_order_grid_nd": (c_int32, [c_int32, c_int32, c_int32, P(c_int32)]),
        "d3m_analyze": (c_int32, [P(d3m_pattern), P(c_int32), c_int32, P(d3m_info)]),
        "d3m_analyze_opts": (c_int32, [P(d3m_pattern), P(c_int32), P(d3m_options), P(d3m_info)]),
        "d3m_create": (c_int32, [P(c_void_p), P(d3m_pattern), P(c_int32), P(d3m_options), c_void_p]),
        "d3m_create_batch": (c_int32, [P(c_void_p), c_int32, P(d3m_pattern), P(P(c_int32)), P(d3m_options),
                                       c_void_p]),
        "d3m_get_instance_omega": (c_int32, [c_void_p, P(c_double), c_void_p]),
        "d3m_factor": (c_int32, [c_void_p, c_void_p, c_void_p]),
        "d3m_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
        "d3m_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
        "d3m_grad_eps": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, P(c_int32), P(c_int32),
                                   c_double, P(c_double), c_void_p]),
        "d3m_grad_eps_noalloc": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, P(c_int32),
                                           P(c_int32), c_double, P(c_double), c_void_p]),
        "d3m_grad_pattern": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
        "d3m_get_factor_block": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
        "d3m_get_pivots": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
        "d3m_get_pivot_blocks": (c_int32, [c_void_p, c_int32, c_void_p, P(c_int32), c_void_p]),
        "d3m_get_info": (c_int32, [c_void_p, P(d3m_info), c_void_p]),
        "d3m_get_trace": (c_int32, [c_void_p, c_void_p, c_int64, P(c_int64), c_void_p]),
        "d3m_last_error": (c_char_p, [c_void_p]),
        "d3m_destroy": (None, [c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def header_symbols() -> list:
    """Names of the functions declared in include/d3m.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(d3m_[a-z_]+)\s*\(", txt)))


class D3MError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, handle=None) -> int:
    if code != D3M_OK:
        msg = load().d3m_last_error(handle)
        raise D3MError(code, msg.decode() if msg else "")
    return code


# thin same-name wrappers ------------------------------------------------------------------
def d3m_default_options() -> d3m_options:
    o = d3m_options()
    load().d3m_default_options(ctypes.byref(o))
    return o


def d3m_order_grid_nd(nx: int, ny: int, nz: int):
    import numpy as np
    nif = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    perm = np.zeros(max(nif, 1), dtype=np.int32)
    check(load().d3m_order_grid_nd(nx, ny, nz, perm.ctypes.data_as(POINTER(c_int32))))
    return perm[:nif]


def make_pattern(colptr, rowidx, m=None, blk_size=None):
    """Build a d3m_pattern; returns (struct, keepalive arrays)."""
    import numpy as np
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    pat = d3m_pattern()
    pat.nblk = colptr.size - 1
    pat.m = int(m or 0)
    keep = [colptr, rowidx]
    if blk_size is not None:
        bs = np.ascontiguousarray(blk_size, dtype=np.int32)
        keep.append(bs)
        pat.blk_size = bs.ctypes.data_as(POINTER(c_int32))
    pat.colptr = colptr.ctypes.data_as(POINTER(c_int64))
    pat.rowidx = rowidx.ctypes.data_as(POINTER(c_int32))
    return pat, keep


def d3m_analyze_opts(colptr, rowidx, m=None, blk_size=None, perm=None, opt=None) -> dict:
    """Symbolic analysis with a handle's options (tile, priority model); opt: d3m_options or None."""
    import numpy as np
    pat, keep = make_pattern(colptr, rowidx, m, blk_size)
    pp = None
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.int32)
        pp = perm.ctypes.data_as(POINTER(c_int32))
    info = d3m_info()
    check(load().d3m_analyze_opts(ctypes.byref(pat), pp, ctypes.byref(opt) if opt is not None else None,
                                  ctypes.byref(info)))
    return info.as_dict()


def d3m_analyze(colptr, rowidx, m=None, blk_size=None, perm=None, tile: int = 128) -> dict:
    import numpy as np
    pat, keep = make_pattern(colptr, rowidx, m, blk_size)
    pp = None
    if perm is not None:
        perm = np.ascontiguousarray(perm, dtype=np.int32)
        pp = perm.ctypes.data_as(POINTER(c_int32))
    info = d3m_info()
    check(load().d3m_analyze(ctypes.byref(pat), pp, tile, ctypes.byref(info)))
    return info.as_dict()
