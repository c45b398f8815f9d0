"""GPU parity of the pivoted variant: Bunch-Kaufman symmetric pivoting inside diagonal tiles
(the paper's sytrf, Sec. II) in the SIMT engines, against the oracle's block Bunch-Kaufman
factorization (oracle/ldlt_bk.py) on matrices where the unpivoted factorization breaks down.

Bars: FP64 pivot sequences equal to the oracle's, factors (Lt = P^T L, D with its 2 x 2 blocks)
entrywise to 1e-10 relative, solutions to 1e-10 and omega <= 1e-12; the complex64 SIMT engine
with pivoting plus FP64 refinement to omega <= 1e-12 and forward error <= 1e-9."""
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


def _zero_diag_problem(g, m, seed):
    # real-G recipe with k^2 = 1 and tau = 1e-4 (diagonal of K about 2 i tau plus noise), and the
    # diagonal of every diagonal block set to zero: the unpivoted factorization meets a zero
    # pivot at its first column, the symmetric indefinite one takes 2 x 2 pivots
    p = synth.make_problem(*g, m, 1.0, 1e-4, seed, real_g=True)
    blocks = p.blocks.copy()
    for gcol in range(p.nblk):
        e = int(p.colptr[gcol])                       # the diagonal block comes first in its column
        blk = blocks[e * m * m:(e + 1) * m * m].reshape(m, m)
        blk[np.diag_indices(m)] = 0.0
    p.blocks = blocks
    return p


def _oracle(p, perm):
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks, p.m)
    F = O.block_ldlt_bk(O.permute_lower(Kb, perm), p.nblk, p.m)
    F.perm = perm
    return Kb, F


@pytest.mark.parametrize("g,m", [((2, 2, 1), 64), ((3, 2, 1), 40)])
def test_fp64_pivoted_matches_oracle(torch_cuda, g, m):
    from paper_2002_05026_gb300 import D3M, D3MError
    torch = torch_cuda
    p = _zero_diag_problem(g, m, 3)
    perm = O.nd_order(*g)
    Kb, F = _oracle(p, perm)
    K = torch.from_numpy(p.blocks).cuda()
    B = synth.rhs(4, p.n, 3)
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    # unpivoted: zero pivot reported
    s0 = D3M(p.colptr, p.rowidx, m=m, perm=perm, precision="fp64")
    s0.factor(K)
    with pytest.raises(D3MError) as ei:
        s0.solve(Bd)
    assert ei.value.code == 4
    s0.close()
    # pivoted
    s = D3M(p.colptr, p.rowidx, m=m, perm=perm, precision="fp64", pivot=True, fp64_omega=True)
    s.factor(K)
    X = s.solve(Bd).cpu().numpy()
    assert np.max(O.omega(Kb, p.nblk, m, X, B)) <= 1e-12
    assert s.info()["omega"] <= 1e-12
    Xo = O.block_solve_bk(F, B)
    assert np.max(np.linalg.norm(X - Xo, axis=0) / np.linalg.norm(Xo, axis=0)) <= 1e-10
    two = 0
    for k in range(p.nblk):
        e, pv = s.pivot_blocks(k, m)
        assert pv.tolist() == F.piv[k].tolist(), k          # the same pivot decisions
        d = s.pivots(k, m)
        Dk = F.D[k]
        assert np.allclose(d, np.diag(Dk), rtol=0, atol=1e-10 * np.abs(Dk).max())
        assert np.allclose(e, np.append(np.diag(Dk, -1), 0.0), rtol=0, atol=1e-10 * np.abs(Dk).max())
        two += int(np.count_nonzero(e))
    assert two > 0                                           # 2 x 2 pivots were taken
    num = den = 0.0
    for (i, j), blk in F.Lt.items():
        Lg = s.factor_block(i, j, m, m)
        num += np.linalg.norm(Lg - blk) ** 2
        den += np.linalg.norm(blk) ** 2
    assert np.sqrt(num / den) <= 1e-10
    s.close()


def test_fp64_pivot_mode_without_pivots_is_unpivoted(torch_cuda):
    # on the benchmark recipe no pivot is needed: identity order, no 2 x 2 blocks, the same
    # factors as the unpivoted oracle
    from paper_2002_05026_gb300 import D3M
    torch = torch_cuda
    g, m = (2, 2, 1), 64
    p = synth.make_problem(*g, m, 2.0, 0.05, 9)
    perm = O.nd_order(*g)
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks, m)
    F0 = O.block_ldlt(O.permute_lower(Kb, perm), p.nblk, m)
    s = D3M(p.colptr, p.rowidx, m=m, perm=perm, precision="fp64", pivot=True)
    s.factor(torch.from_numpy(p.blocks).cuda())
    for k in range(p.nblk):
        e, pv = s.pivot_blocks(k, m)
        assert pv.tolist() == list(range(m)) and not np.any(e)
        assert np.allclose(s.pivots(k, m), F0.D[k], rtol=1e-10, atol=0)
    for (i, j), blk in F0.L.items():
        assert np.allclose(s.factor_block(i, j, m, m), blk, rtol=0, atol=1e-10)
    s.close()


def test_simt32_pivoted_refined(torch_cuda):
    from paper_2002_05026_gb300 import D3M
    torch = torch_cuda
    g, m = (2, 2, 1), 64
    p = _zero_diag_problem(g, m, 5)
    perm = O.nd_order(*g)
    Kb, F = _oracle(p, perm)
    B = synth.rhs(6, p.n, 2)
    s = D3M(p.colptr, p.rowidx, m=m, perm=perm, precision="simt32", pivot=True)
    s.factor(torch.from_numpy(p.blocks).cuda())
    X = s.solve(torch.from_numpy(np.ascontiguousarray(B)).cuda()).cpu().numpy()
    assert np.max(O.omega(Kb, p.nblk, m, X, B)) <= 1e-12
    Xo = O.block_solve_bk(F, B)
    assert np.max(np.linalg.norm(X - Xo, axis=0) / np.linalg.norm(Xo, axis=0)) <= 1e-9
    s.close()
