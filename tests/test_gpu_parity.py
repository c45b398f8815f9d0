"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars:
* plain FP64 path: factors (unique unpivoted L, D) entrywise and solutions to <= 1e-10
  relative error;
* mixed paths after FP64 refinement: relative forward error <= 1e-9 per column and normwise
  backward error omega <= 1e-12, omega recomputed by the oracle from the returned X;
* mixed-path factors are complex64 with split-BF16x3 products (about 2^-16 relative per
  product) or TF32 products (operands rounded to 11 significant bits, about 2^-11 relative per
  product), so they are compared with loose relative bounds (5e-3, 2e-2 for TF32) that still
  catch any structural error (wrong tile, sign, transpose or pivot).
"""
import numpy as np
import pytest

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2002_05026_gb300 import build
    build.build()
    return torch


def _setup(g, m, k2=1.0, tau=0.1, seed=101, perm="nd", real_g=False):
    from paper_2002_05026_gb300 import d3m_order_grid_nd
    p = synth.make_problem(*g, m, k2, tau, seed, real_g=real_g)
    if perm == "nd":
        pm = d3m_order_grid_nd(*g)
        assert pm.tolist() == O.nd_order(*g).tolist()
    else:
        pm = np.arange(p.nblk, dtype=np.int32)
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks, p.m)
    F = O.block_ldlt(O.permute_lower(Kb, pm), p.nblk, p.m)
    F.perm = pm
    return p, pm, Kb, F


def _run(torch, p, pm, precision, B, **kw):
    from paper_2002_05026_gb300 import D3M
    s = D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision=precision, max_nrhs=max(8, B.shape[1]), **kw)
    s.factor(torch.from_numpy(p.blocks_numpy()).cuda())
    X = s.solve(torch.from_numpy(np.ascontiguousarray(B)).cuda()).cpu().numpy()
    return s, X


def _factor_err(s, F, m):
    num = den = 0.0
    worst = 0.0
    for (i, j), Lo in F.L.items():
        Lg = s.factor_block(i, j, m, m)
        num += np.linalg.norm(Lg - Lo) ** 2
        den += np.linalg.norm(Lo) ** 2
        worst = max(worst, np.abs(Lg - Lo).max())
    dnum = dden = 0.0
    for j in range(F.nblk):
        d = s.pivots(j, m)
        dnum += np.linalg.norm(d - F.D[j]) ** 2
        dden += np.linalg.norm(F.D[j]) ** 2
    return np.sqrt(num / den), np.sqrt(dnum / dden), worst


def _fwd_err(X, Xo):
    return np.max(np.linalg.norm(X - Xo, axis=0) / np.linalg.norm(Xo, axis=0))


CASES = [((2, 2, 1), 64), ((2, 2, 1), 1), ((2, 2, 1), 2), ((3, 3, 1), 100), ((2, 2, 2), 16),
         ((1, 5, 1), 70), ((1, 2, 1), 64), ((3, 2, 1), 130), ((4, 4, 1), 64)]


@pytest.mark.parametrize("g,m", CASES)
def test_fp64_factor_and_solve(torch_cuda, g, m):
    p, pm, Kb, F = _setup(g, m, k2=1.0, tau=0.1, seed=7 + m)
    B = synth.rhs(3, p.n, 3)
    s, X = _run(torch_cuda, p, pm, "fp64", B)
    eL, eD, _ = _factor_err(s, F, m)
    assert eL <= 1e-10 and eD <= 1e-10, (eL, eD)
    Xo = O.block_solve(F, B)
    assert _fwd_err(X, Xo) <= 1e-10
    info = s.info()
    assert info["status"] == 0 and info["refine_iters"] == 1


def test_fp64_natural_order_and_omega(torch_cuda):
    p, pm, Kb, F = _setup((3, 3, 1), 40, perm="natural", seed=5)
    B = synth.rhs(4, p.n, 2)
    s, X = _run(torch_cuda, p, pm, "fp64", B, fp64_omega=True)
    eL, eD, _ = _factor_err(s, F, 40)
    assert eL <= 1e-10 and eD <= 1e-10
    om = O.omega(Kb, p.nblk, p.m, X, B)
    assert np.max(om) <= 1e-14
    # both at the rounding level: the device residual's floor is about 1e-15 of |K||x|
    assert s.info()["omega"] <= 1e-14


@pytest.mark.parametrize("precision", ["simt32", "bf16x3", "tf32"])
@pytest.mark.parametrize("g,m", [((2, 2, 1), 64), ((3, 3, 1), 100), ((2, 2, 2), 128), ((1, 3, 1), 1),
                                 ((4, 4, 1), 128), ((3, 2, 1), 200)])
def test_mixed_refined_solution(torch_cuda, precision, g, m):
    p, pm, Kb, F = _setup(g, m, k2=2.0, tau=0.05, seed=11 + m)
    B = synth.rhs(9, p.n, 4)
    s, X = _run(torch_cuda, p, pm, precision, B)
    Xo = O.block_solve(F, B)
    assert _fwd_err(X, Xo) <= 1e-9
    assert np.max(O.omega(Kb, p.nblk, p.m, X, B)) <= 1e-12
    info = s.info()
    assert info["status"] == 0 and info["omega"] <= 1e-12
    eL, eD, _ = _factor_err(s, F, m)
    bound = 2e-2 if precision == "tf32" else 5e-3
    assert eL <= bound and eD <= bound, (eL, eD)


def test_mixed_factor_accuracy_simt_vs_tc(torch_cuda):
    # the FP32 SIMT factor is at FP32 level; the split-BF16x3 factor within ~2^-16 * growth; the
    # TF32 factor within ~2^-11 * growth, and measurably less accurate than split-BF16x3 (each
    # engine really computes in its own precision)
    p, pm, Kb, F = _setup((3, 3, 1), 128, k2=2.0, tau=0.05, seed=3)
    B = synth.rhs(9, p.n, 1)
    s1, _ = _run(torch_cuda, p, pm, "simt32", B)
    s2, _ = _run(torch_cuda, p, pm, "bf16x3", B)
    s3, _ = _run(torch_cuda, p, pm, "tf32", B)
    e1 = _factor_err(s1, F, 128)[0]
    e2 = _factor_err(s2, F, 128)[0]
    e3 = _factor_err(s3, F, 128)[0]
    assert e1 <= 1e-5, e1
    assert e2 <= 2e-4, e2
    assert 5 * e2 <= e3 <= 5e-3, (e2, e3)


def test_decoupled_blocks(torch_cuda):
    from paper_2002_05026_gb300 import D3M
    m = 96
    singles = [synth.make_problem(2, 1, 1, m, 1.0, 0.1, 40 + s) for s in range(3)]
    colptr = np.arange(4, dtype=np.int64)
    rowidx = np.arange(3, dtype=np.int32)
    blocks = np.concatenate([q.blocks for q in singles])
    s = D3M(colptr, rowidx, m=m, precision="fp64")
    s.factor(torch_cuda.from_numpy(blocks).cuda())
    assert s.info()["nblk_L_offdiag"] == 0
    for k in range(3):
        L1, d1 = O.ldlt_unpivoted(singles[k].block(0))
        assert np.abs(s.factor_block(k, k, m, m) - L1).max() <= 1e-10
        assert np.abs(s.pivots(k, m) - d1).max() <= 1e-10 * np.abs(d1).max()


def test_real_g_variant(torch_cuda):
    p, pm, Kb, F = _setup((3, 3, 1), 64, k2=2.0, tau=0.05, seed=8, real_g=True)
    B = synth.rhs(2, p.n, 2)
    s, X = _run(torch_cuda, p, pm, "bf16x3", B)
    assert _fwd_err(X, O.block_solve(F, B)) <= 1e-9


def test_host_buffers(torch_cuda):
    # K and B from host memory, X returned to host memory
    from paper_2002_05026_gb300 import D3M
    p, pm, Kb, F = _setup((2, 2, 1), 64, seed=4)
    s = D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision="bf16x3")
    Kh = torch_cuda.from_numpy(p.blocks_numpy()).pin_memory()
    s.factor(Kh)
    B = synth.rhs(3, p.n, 2)
    Bh = torch_cuda.from_numpy(np.ascontiguousarray(B.T)).pin_memory()
    Xh = torch_cuda.empty_like(Bh).pin_memory()
    import ctypes
    rc = s._lib.d3m_solve(s.h, ctypes.c_void_p(Bh.data_ptr()), ctypes.c_void_p(Xh.data_ptr()), 2,
                          ctypes.c_void_p(torch_cuda.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch_cuda.cuda.synchronize()
    X = Xh.numpy().T
    assert _fwd_err(X, O.block_solve(F, B)) <= 1e-9


@pytest.mark.parametrize("prec", ["bf16x3", "tf32"])
def test_host_k_uploaded_during_factorization(torch_cuda, prec):
    # a page-locked host K is uploaded block by block while the factorization runs (tasks wait for
    # their block); a pageable one is copied first.  Both factor exactly like a device K: the same
    # arithmetic in the same order, so the solutions are bitwise equal.
    from paper_2002_05026_gb300 import D3M
    p, pm, Kb, F = _setup((3, 3, 1), 200, seed=6)
    B = synth.rhs(5, p.n, 3)
    Bd = torch_cuda.from_numpy(np.ascontiguousarray(B)).cuda()
    ref = D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision=prec, max_nrhs=3)
    ref.factor(torch_cuda.from_numpy(p.blocks_numpy()).cuda())
    Xref = ref.solve(Bd).cpu().numpy()
    ref.close()
    assert _fwd_err(Xref, O.block_solve(F, B)) <= 1e-9
    Kpage = torch_cuda.from_numpy(p.blocks_numpy())
    for Kh in (Kpage.pin_memory(), Kpage):
        s = D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision=prec, max_nrhs=3)
        for _ in range(2):                       # the second call uploads into the same buffer
            s.factor(Kh)
            X = s.solve(Bd).cpu().numpy()
            assert s.info()["status"] == 0
            assert np.array_equal(X, Xref)
        s.close()


def test_zero_pivot_reported(torch_cuda):
    from paper_2002_05026_gb300 import D3M, D3MError
    p, pm, Kb, F = _setup((2, 2, 1), 64, seed=4)
    K = p.blocks_numpy().copy()
    # first pivot of the elimination = entry (0, 0) of the diagonal block of interface perm[0]
    e = int(p.colptr[pm[0]])
    K[p.blk_off[e]] = 0.0
    for prec in ("fp64", "bf16x3"):
        s = D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision=prec)
        s.factor(torch_cuda.from_numpy(K).cuda())
        assert s.info()["status"] == 4          # D3M_ERR_PIVOT
        with pytest.raises(D3MError):
            s.solve(torch_cuda.from_numpy(synth.rhs(1, p.n, 1)).cuda())


def test_bounded_wait_timeout(torch_cuda):
    # one task gets an unmet dependency: the queue starves and every waiting block returns
    # D3M_ERR_TIMEOUT after the bounded wait; the context stays usable afterwards.
    from paper_2002_05026_gb300 import D3M
    p, pm, Kb, F = _setup((2, 2, 1), 64, seed=4)
    for prec in ("fp64", "bf16x3"):
        s = D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision=prec, timeout_ns=200_000_000, debug_flags=1)
        s.factor(torch_cuda.from_numpy(p.blocks_numpy()).cuda())
        assert s.info()["status"] == 6          # D3M_ERR_TIMEOUT
        s.close()
    B = synth.rhs(3, p.n, 1)
    s2, X = _run(torch_cuda, p, pm, "bf16x3", B)
    assert _fwd_err(X, O.block_solve(F, B)) <= 1e-9


def test_refactor_same_handle(torch_cuda):
    # a second factorization with the same handle (new K) resets the queue state
    from paper_2002_05026_gb300 import D3M
    p1, pm, Kb1, F1 = _setup((3, 3, 1), 64, seed=21)
    p2, _, Kb2, F2 = _setup((3, 3, 1), 64, seed=22)
    s = D3M(p1.colptr, p1.rowidx, m=64, perm=pm, precision="bf16x3")
    B = synth.rhs(3, p1.n, 2)
    for p, F in ((p1, F1), (p2, F2), (p1, F1)):
        s.factor(torch_cuda.from_numpy(p.blocks_numpy()).cuda())
        X = s.solve(torch_cuda.from_numpy(np.ascontiguousarray(B)).cuda()).cpu().numpy()
        assert _fwd_err(X, O.block_solve(F, B)) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "bf16x3", "tf32"])
def test_full_interface_size_many_rhs(torch_cuda, precision):
    # m = 512 as in the 8x8 and 6x6x6 workloads: the in-block chains span 4 (8) tiles of 128
    # (64) rows, i.e. 8 row strips per interface block, one cluster of 8 CTAs per block;
    # 11 right-hand sides = one group of 8 and a ragged group of 3
    p, pm, Kb, F = _setup((2, 2, 2), 512, k2=2.0, tau=0.05, seed=77)
    B = synth.rhs(5, p.n, 11)
    s, X = _run(torch_cuda, p, pm, precision, B)
    Xo = O.block_solve(F, B)
    assert _fwd_err(X, Xo) <= (1e-10 if precision == "fp64" else 1e-9)
    if precision != "fp64":
        assert np.max(O.omega(Kb, p.nblk, p.m, X, B)) <= 1e-12


def _omega_extended(Kb, nblk, m, X, B):
    # residual with extended-precision products and sums (80-bit on x86, 128-bit on aarch64)
    A = O.dense_from_lower(Kb, nblk, m).astype(np.clongdouble)
    R = B.astype(np.clongdouble) - A @ X.astype(np.clongdouble)
    kn = O.k_inf_norm(Kb, nblk, m)
    return (np.abs(R).max(axis=0) / (kn * np.abs(X).max(axis=0) + np.abs(B).max(axis=0))).astype(np.float64)


@pytest.mark.parametrize("precision", ["fp64", "bf16x3", "tf32"])
@pytest.mark.parametrize("g,m", [((3, 3, 1), 100), ((2, 2, 2), 128)])
def test_device_omega_matches_extended_precision(torch_cuda, precision, g, m):
    # the device residual (double-float products, FP64 accumulation) reports the backward
    # error of the returned X to within 2% at the 1e-13..1e-16 level, which a residual with
    # only FP32 accuracy (about 1e-7 relative) could not
    p, pm, Kb, F = _setup(g, m, k2=2.0, tau=0.05, seed=5 + m)
    B = synth.rhs(13, p.n, 4)
    s, X = _run(torch_cuda, p, pm, precision, B, fp64_omega=True)
    w_dev = s.info()["omega"]
    w_ext = np.max(_omega_extended(Kb, p.nblk, p.m, X, B))
    if precision == "fp64":
        # a plain FP64 solve sits at the rounding level of any FP64-class residual
        assert w_ext <= 1e-14 and w_dev <= 1e-14, (w_dev, w_ext)
    else:
        assert w_ext <= 1e-12
        assert w_dev == pytest.approx(w_ext, rel=0.02), (w_dev, w_ext)


@pytest.mark.parametrize("precision", ["fp64", "bf16x3"])
def test_device_k_read_in_place(torch_cuda, precision):
    # a device K is read in place by the factorization (and the norm/split of K); nothing reads
    # it afterwards, so overwriting it after d3m_factor (in stream order) leaves the solve intact
    from paper_2002_05026_gb300 import D3M
    torch = torch_cuda
    p, pm, Kb, F = _setup((3, 3, 1), 64, k2=2.0, tau=0.05, seed=31)
    B = synth.rhs(5, p.n, 3)
    s = D3M(p.colptr, p.rowidx, m=p.m, perm=pm, precision=precision, max_nrhs=8)
    Kd = torch.from_numpy(p.blocks_numpy()).cuda()
    s.factor(Kd)
    Kd.zero_()
    X = s.solve(torch.from_numpy(np.ascontiguousarray(B)).cuda()).cpu().numpy()
    s.close()
    assert _fwd_err(X, O.block_solve(F, B)) <= 1e-9
    if precision != "fp64":
        assert np.max(O.omega(Kb, p.nblk, p.m, X, B)) <= 1e-12
