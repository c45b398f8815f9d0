"""d3m_grad_eps_noalloc: the epsilon gradient for callers that cannot allocate memory during the
call (an application whose own allocator owns the device memory and forbids library
allocations, or a device too full for late temporaries).  It must return what d3m_grad_eps
returns, through the C ABI, on repeated calls that reuse its fixed scratch array, and reject
inputs that would make its kernel read outside that array.  Kept in a file collected last."""
import ctypes

import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


def _dom_arrays(dom_if):
    ptr = np.zeros(len(dom_if) + 1, dtype=np.int32)
    for i, I in enumerate(dom_if):
        ptr[i + 1] = ptr[i] + len(I)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(I, dtype=np.int32) for I in dom_if]), dtype=np.int32)
    return ptr, flat


def _call(lib, h, fn, Lt, Xt, nrhs, ptr, flat, k2, stream, out=None):
    host = out is None
    if host:
        out = np.full(len(ptr) - 1, np.nan)
    optr = ctypes.cast(out.ctypes.data, ctypes.POINTER(ctypes.c_double)) if host else \
        ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double))
    rc = getattr(lib, fn)(h, ctypes.c_void_p(Lt.data_ptr()), ctypes.c_void_p(Xt.data_ptr()), nrhs, len(ptr) - 1,
                          ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          flat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.c_double(k2),
                          optr, ctypes.c_void_p(stream))
    return rc, out


def test_grad_eps_noalloc_matches_grad_eps():
    import torch
    from paper_2002_05026_gb300 import D3M, build
    build.build()
    g, m, k2, tau = (4, 3, 1), 24, 2.0, 0.05
    p = synth.make_problem(*g, m, k2, tau, 61)
    perm = O.nd_order(*g)
    s = D3M(p.colptr, p.rowidx, m=m, perm=perm, precision="bf16x3", max_nrhs=4)
    s.factor(torch.from_numpy(p.blocks).cuda())
    ptr, flat = _dom_arrays(p.dom_if)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                       # two calls in a row reuse the scratch array
        nrhs = 1 + call * 2
        b = torch.from_numpy(synth.rhs(70 + call, p.n, nrhs)).cuda()
        c = torch.from_numpy(synth.rhs(80 + call, p.n, nrhs)).cuda()
        x = s.solve(b)
        lam = s.adjoint(c)
        Lt, Xt = lam.T.contiguous(), x.T.contiguous()
        rc0, ref = _call(s._lib, s.h, "d3m_grad_eps", Lt, Xt, nrhs, ptr, flat, k2, stream)
        rc1, got = _call(s._lib, s.h, "d3m_grad_eps_noalloc", Lt, Xt, nrhs, ptr, flat, k2, stream)
        assert rc0 == 0 and rc1 == 0
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # a device output buffer gets the same values
    dev_out = torch.full((len(ptr) - 1,), float("nan"), dtype=torch.float64, device="cuda")
    rc2, _ = _call(s._lib, s.h, "d3m_grad_eps_noalloc", Lt, Xt, nrhs, ptr, flat, k2, stream, out=dev_out)
    assert rc2 == 0
    assert np.max(np.abs(dev_out.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    # exactly the largest domain count is accepted (extra domains with no interfaces get 0);
    # one more is rejected with D3M_ERR_INVALID, nothing launched
    ndom = len(ptr) - 1
    full = np.concatenate([ptr, np.full(16384 - ndom, ptr[-1], dtype=np.int32)]).astype(np.int32)
    rc3, got3 = _call(s._lib, s.h, "d3m_grad_eps_noalloc", Lt, Xt, nrhs, full, flat, k2, stream)
    assert rc3 == 0, s.last_error()
    assert np.max(np.abs(got3[:ndom] - ref)) <= 1e-12 * np.max(np.abs(ref)) and np.all(got3[ndom:] == 0.0)
    big = np.concatenate([full, full[-1:]]).astype(np.int32)
    rc, _ = _call(s._lib, s.h, "d3m_grad_eps_noalloc", Lt, Xt, nrhs, big, flat, k2, stream)
    assert rc == 1
    assert "scratch" in s.last_error()
    # a dom_ptr that decreases somewhere inside (its last entry still in range) is rejected
    bad = ptr.copy()
    bad[2], bad[3] = bad[3] + 1000, bad[3]
    assert bad[-1] == ptr[-1]
    rc, _ = _call(s._lib, s.h, "d3m_grad_eps_noalloc", Lt, Xt, nrhs, bad, flat, k2, stream)
    assert rc == 1 and "nondecreasing" in s.last_error()
    # a dom_if entry naming no interface is rejected
    badif = flat.copy()
    badif[len(badif) // 2] = p.nblk
    rc, _ = _call(s._lib, s.h, "d3m_grad_eps_noalloc", Lt, Xt, nrhs, ptr, badif, k2, stream)
    assert rc == 1 and "out of range" in s.last_error()
    # the valid call still works after the rejected ones
    rc4, got4 = _call(s._lib, s.h, "d3m_grad_eps_noalloc", Lt, Xt, nrhs, ptr, flat, k2, stream)
    assert rc4 == 0 and np.max(np.abs(got4 - ref)) <= 1e-12 * np.max(np.abs(ref))
