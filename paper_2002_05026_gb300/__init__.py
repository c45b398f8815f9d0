"""GB300 (sm_103a) D3M dual-system solver: block LDL^T factorization and solve of the reduced
complex-symmetric block-sparse matrix K, behind the C ABI of include/d3m.h (libd3m.so)."""
from ._abi import (D3M_FP64, D3M_MIXED_BF16X3, D3M_MIXED_SIMT32, D3M_MIXED_TF32, D3MError, d3m_analyze,  # noqa: F401
                   d3m_analyze_opts, d3m_default_options, d3m_order_grid_nd, header_symbols, load)
from .solver import D3M, D3MBatch  # noqa: F401

__all__ = ["D3M", "D3MBatch", "D3MError", "d3m_analyze", "d3m_analyze_opts", "d3m_order_grid_nd", "d3m_default_options", "load",
           "header_symbols", "D3M_FP64", "D3M_MIXED_BF16X3", "D3M_MIXED_SIMT32", "D3M_MIXED_TF32"]
