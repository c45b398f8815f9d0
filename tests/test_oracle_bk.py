"""Pins of the oracle's Bunch-Kaufman variant (Sec. II names sytrf, the symmetric indefinite
factorization with Bunch-Kaufman pivoting, as the dense kernel of the dual factorization).

Checked against what the definition fixes: reconstruction P A P^T = L D L^T, the dense LU
solution, hand-worked pivot decisions (a 2 x 2 pivot where both diagonal entries are small, a
swap where only the other diagonal entry is large), the multiplier bound of a 1 x 1 pivot,
the reduction to the unpivoted factorization when no pivot is needed, and, for the block
version with pivoting inside diagonal blocks, reconstruction and solution on a matrix where
the unpivoted factorization meets tiny pivots."""
import numpy as np
import pytest

import oracle as O
import synth


def _rand_sym(n, seed, diag_scale=1.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + A.T
    A[np.diag_indices(n)] *= diag_scale
    return A


@pytest.mark.parametrize("n,seed,ds", [(1, 1, 1.0), (2, 2, 1.0), (7, 3, 1.0), (40, 4, 1.0), (40, 5, 1e-3), (64, 6, 0.0)])
def test_bk_reconstruction_and_solve(n, seed, ds):
    A = _rand_sym(n, seed, ds)
    p, L, D, sz = O.ldlt_bk(A)
    assert sorted(p.tolist()) == list(range(n))
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.diag(L), 1)
    R = A[p][:, p] - L @ D @ L.T
    assert np.linalg.norm(R) <= 1e-13 * np.linalg.norm(A)
    # D: 1 x 1 and symmetric 2 x 2 blocks where sizes says so, zero elsewhere
    k = 0
    mask = np.zeros((n, n), dtype=bool)
    while k < n:
        s = int(sz[k])
        assert s in (1, 2)
        mask[k:k + s, k:k + s] = True
        k += s
    assert np.all(D[~mask] == 0) and np.allclose(D, D.T)
    b = np.random.default_rng(seed + 100).standard_normal((n, 2)) + 0j
    LU, pv = O.lu_factor_pp(A)
    x_lu = O.lu_solve_pp(LU, pv, b)
    y = np.linalg.solve(L, b[p])
    x = np.zeros_like(b)
    x[p] = np.linalg.solve(L.T, np.linalg.solve(D, y))
    assert np.linalg.norm(x - x_lu) <= 1e-10 * np.linalg.norm(x_lu)


def test_bk_two_by_two_when_both_diagonals_small():
    # |a_11| < alpha |a_21| and |a_22| < alpha |a_21|: one 2 x 2 pivot, the matrix itself
    A = np.array([[1e-3, 1.0 + 0.5j], [1.0 + 0.5j, 2e-3j]])
    p, L, D, sz = O.ldlt_bk(A)
    assert sz.tolist() == [2, 0] and p.tolist() == [0, 1]
    assert np.allclose(L, np.eye(2)) and np.allclose(D, A)


def test_bk_swap_when_other_diagonal_large():
    # column 0: |a_00| = 0.1 < alpha * lam (lam = 1 at row 2); row 2: sigma = 1, |a_22| = 5 >=
    # alpha sigma -> swap 0 and 2 and take a 1 x 1 pivot of 5
    A = np.array([[0.1, 0.0, 1.0], [0.0, 3.0, 0.0], [1.0, 0.0, 5.0]], dtype=complex)
    p, L, D, sz = O.ldlt_bk(A)
    assert p[0] == 2 and sz[0] == 1 and D[0, 0] == 5.0


def test_bk_bounds_growth_where_unpivoted_does_not():
    # a tiny leading diagonal entry: the unpivoted multipliers grow like 1 / eps, Bunch-Kaufman's
    # stay bounded (|l| <= 2 / alpha in the |Re| + |Im| measure for a pivot that passed the first
    # or third test) and its factor still reconstructs A
    A = _rand_sym(24, 13)
    A[0, 0] = 1e-12
    L0, d0 = O.ldlt_unpivoted(A)
    assert np.max(np.abs(L0)) > 1e6
    p, L, D, sz = O.ldlt_bk(A)
    assert np.max(np.abs(L.real) + np.abs(L.imag)) <= 30.0
    assert np.linalg.norm(A[p][:, p] - L @ D @ L.T) <= 1e-13 * np.linalg.norm(A)


def test_bk_reduces_to_unpivoted_when_dominant():
    # strongly diagonally dominant: every first test passes, no swaps, all 1 x 1: the unpivoted
    # factorization of the plain oracle
    A = _rand_sym(30, 12) * 0.01
    A[np.diag_indices(30)] += 5.0 + 1.0j
    p, L, D, sz = O.ldlt_bk(A)
    assert p.tolist() == list(range(30)) and np.all(sz == 1)
    L0, d0 = O.ldlt_unpivoted(A)
    assert np.allclose(L, L0, rtol=0, atol=1e-14) and np.allclose(np.diag(D), d0, rtol=0, atol=1e-13)


def _small_tau_problem(g, m, seed):
    # real G: M_i = G G^T - k^2 I + i tau I with G G^T's diagonal about 1, k^2 = 1: the diagonal of
    # K is about 2 i tau plus noise, far below its off-diagonal entries
    return synth.make_problem(*g, m, 1.0, 1e-4, seed, real_g=True)


@pytest.mark.parametrize("g,m", [((2, 2, 1), 12), ((3, 2, 1), 8)])
def test_block_bk_small_tau(g, m):
    p = _small_tau_problem(g, m, 5)
    perm = O.nd_order(*g)
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks, m)
    Kp = O.permute_lower(Kb, perm)
    F = O.block_ldlt_bk(Kp, p.nblk, m)
    F.perm = perm
    # reconstruction of P K P^T from the block factor
    N, n = p.nblk, p.n
    Lt = np.zeros((n, n), dtype=complex)
    Dd = np.zeros((n, n), dtype=complex)
    for (i, j), blk in F.Lt.items():
        Lt[i * m:(i + 1) * m, j * m:(j + 1) * m] = blk
    for k in range(N):
        Dd[k * m:(k + 1) * m, k * m:(k + 1) * m] = F.D[k]
    A = O.dense_from_lower(Kp, N, m)
    assert np.linalg.norm(A - Lt @ Dd @ Lt.T) <= 1e-12 * np.linalg.norm(A)
    # some block needed a swap or a 2 x 2 pivot
    assert any((F.piv[k] != np.arange(m)).any() or (F.sizes[k] == 2).any() for k in range(N))
    B = synth.rhs(3, n, 2)
    X = O.block_solve_bk(F, B)
    Ad = O.dense_from_lower(Kb, N, m)
    LU, pv = O.lu_factor_pp(Ad)
    Xlu = O.lu_solve_pp(LU, pv, B)
    assert np.linalg.norm(X - Xlu) <= 1e-10 * np.linalg.norm(Xlu)


def test_block_bk_equals_unpivoted_on_dominant_recipe():
    # the benchmark recipe (complex G, k^2 = 2) needs no pivoting: same factor as the plain oracle
    g, m = (2, 2, 1), 16
    p = synth.make_problem(*g, m, 2.0, 0.05, 7)
    perm = O.nd_order(*g)
    Kp = O.permute_lower(O.lower_blocks(p.colptr, p.rowidx, p.blocks, m), perm)
    F = O.block_ldlt_bk(Kp, p.nblk, m)
    F0 = O.block_ldlt(Kp, p.nblk, m)
    for k in range(p.nblk):
        assert (F.piv[k] == np.arange(m)).all() and (F.sizes[k] == 1).all()
        assert np.allclose(np.diag(F.D[k]), F0.D[k], rtol=1e-13, atol=0)
    for key, blk in F0.L.items():
        assert np.allclose(F.Lt[key], blk, rtol=0, atol=1e-13)
