"""Plain FP64 oracle of the pivoted variant: Bunch-Kaufman symmetric pivoting inside diagonal blocks.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): used by the tests; never by the library.

Sec. II of the paper weights the dual tasks with benchmarked GEMM, sytrf and triSolve times:
its dense diagonal-block factorization is the symmetric indefinite factorization with
Bunch-Kaufman partial pivoting (Bunch and Kaufman, "Some stable methods for calculating inertia
and solving symmetric linear systems", Math. Comp. 31, 1977).  The unpivoted factorization of
ldlt.py is the default reading; this module is the pivoted one, with the pivoting confined to
each diagonal block: the unknowns of one block are reordered among themselves, so the block
structure, the fill and the task graph stay those of the unpivoted factorization.

Definitions (complex symmetric, no conjugation anywhere):
* dense:  P A P^T = L D L^T, L unit lower triangular, D block diagonal with 1 x 1 and symmetric
  2 x 2 blocks; the pivot rule is Bunch-Kaufman's with alpha = (1 + sqrt(17)) / 8, magnitudes
  measured as |Re z| + |Im z| (the measure LAPACK's complex routines use);
* block:  with the diagonal block of column k factored as S_kk = Lt_kk D_k Lt_kk^T,
  Lt_kk = P_k^T L_kk (a row-permuted unit lower matrix), the off-diagonal blocks are
  Lt_jk = S_jk Lt_kk^{-T} D_k^{-1} and the Schur updates S_ij -= Lt_ik D_k Lt_jk^T, exactly the
  unpivoted block recursion with Lt_kk in place of L_kk and block-diagonal D_k;
* solve:  K = Lt D Lt^T: forward Lt y = b, diagonal D z = y, backward Lt^T x = z.
"""
from __future__ import annotations

import math

import numpy as np

from .ldlt import block_symbolic

ALPHA = (1.0 + math.sqrt(17.0)) / 8.0

__all__ = ["ALPHA", "cabs1", "ldlt_bk", "FactorBK", "block_ldlt_bk", "block_solve_bk"]


def cabs1(z) -> float:
    return float(abs(np.real(z)) + abs(np.imag(z)))


def ldlt_bk(A: np.ndarray):
    """Bunch-Kaufman factorization of a complex symmetric matrix: returns (perm, L, D, sizes)
    with A[perm][:, perm] = L D L^T; sizes[k] = 1 or 2 at the first column of each pivot block
    (0 at the second column of a 2 x 2 block).  At step k, with lam the largest off-diagonal
    magnitude in column k (at row r) and sigma the largest off-diagonal magnitude in row r of
    the remaining matrix:
      |a_kk| >= alpha lam                 -> 1 x 1 pivot a_kk;
      else |a_kk| sigma >= alpha lam^2    -> 1 x 1 pivot a_kk;
      else |a_rr| >= alpha sigma          -> swap k and r, 1 x 1 pivot;
      else                                -> swap k + 1 and r, 2 x 2 pivot on (k, k + 1)."""
    W = np.array(A, dtype=np.complex128, copy=True)
    n = W.shape[0]
    L = np.eye(n, dtype=np.complex128)
    D = np.zeros((n, n), dtype=np.complex128)
    perm = np.arange(n)
    sizes = np.zeros(n, dtype=np.int64)

    def swap(i, j, k):
        if i == j:
            return
        perm[[i, j]] = perm[[j, i]]
        W[[i, j], :] = W[[j, i], :]
        W[:, [i, j]] = W[:, [j, i]]
        L[[i, j], :k] = L[[j, i], :k]

    k = 0
    while k < n:
        akk = cabs1(W[k, k])
        if k + 1 < n:
            col = np.abs(W[k + 1:, k].real) + np.abs(W[k + 1:, k].imag)
            r = k + 1 + int(np.argmax(col))
            lam = float(col[r - k - 1])
        else:
            r, lam = k, 0.0
        s = 1
        if max(akk, lam) == 0.0:
            raise ZeroDivisionError(f"singular matrix at column {k}")
        if akk >= ALPHA * lam:
            pass
        else:
            row = np.concatenate([W[r, k:r], W[r + 1:, r]])       # row r of the remaining matrix, off the diagonal
            sigma = float(np.max(np.abs(row.real) + np.abs(row.imag)))
            if akk * sigma >= ALPHA * lam * lam:
                pass
            elif cabs1(W[r, r]) >= ALPHA * sigma:
                swap(k, r, k)
            else:
                swap(k + 1, r, k)
                s = 2
        if s == 1:
            d = W[k, k]
            D[k, k] = d
            sizes[k] = 1
            if k + 1 < n:
                l = W[k + 1:, k] / d
                W[k + 1:, k + 1:] -= np.outer(l, W[k, k + 1:])
                L[k + 1:, k] = l
        else:
            Dk = W[k:k + 2, k:k + 2].copy()
            D[k:k + 2, k:k + 2] = Dk
            sizes[k], sizes[k + 1] = 2, 0
            if k + 2 < n:
                C = W[k + 2:, k:k + 2]
                Lc = np.linalg.solve(Dk.T, C.T).T                 # C D_k^{-1}
                W[k + 2:, k + 2:] -= Lc @ C.T
                L[k + 2:, k:k + 2] = Lc
        k += s
    return perm, L, D, sizes


class FactorBK:
    """Block factor with pivoting inside diagonal blocks: Lt[(i, j)] (i > j: off-diagonal blocks;
    (k, k): Lt_kk = P_k^T L_kk), D[k] (m x m block diagonal), piv[k] (perm of block k), sizes[k]."""

    def __init__(self, Lt, D, piv, sizes, struct, perm, m):
        self.Lt, self.D, self.piv, self.sizes, self.struct = Lt, D, piv, sizes, struct
        self.perm, self.m = (None if perm is None else np.asarray(perm)), m

    @property
    def nblk(self):
        return len(self.D)


def block_ldlt_bk(Kp: dict, nblk: int, m: int) -> FactorBK:
    """Right-looking block LDL^T of the permuted lower blocks Kp with Bunch-Kaufman pivoting
    inside every diagonal block:
      FACTOR  S_kk[p][:, p] = L_kk D_k L_kk^T,  Lt_kk = P_k^T L_kk
      TRSM    Lt_jk = S_jk Lt_kk^{-T} D_k^{-1}                      for j in struct(k)
      UPDATE  S_ij -= Lt_ik D_k Lt_jk^T                            for i >= j in struct(k)."""
    S = {key: blk.copy() for key, blk in Kp.items()}
    struct, _parent = block_symbolic(nblk, Kp.keys())
    Lt, D, piv, sizes = {}, [None] * nblk, [None] * nblk, [None] * nblk
    for k in range(nblk):
        p, Lkk, Dk, sz = ldlt_bk(S.pop((k, k)))
        Ltk = np.zeros_like(Lkk)
        Ltk[p] = Lkk                                                   # P_k^T L_kk
        Lt[(k, k)], D[k], piv[k], sizes[k] = Ltk, Dk, p, sz
        for j in struct[k]:
            Sjk = S.pop((j, k))
            X = np.linalg.solve(Ltk, Sjk.T).T                          # S_jk Lt_kk^{-T}
            Lt[(j, k)] = np.linalg.solve(Dk, X.T).T                    # ... D_k^{-1} (D_k symmetric)
        for a, j in enumerate(struct[k]):
            Wjk = Lt[(j, k)] @ Dk                                      # Lt_jk D_k
            for i in struct[k][a:]:
                upd = Lt[(i, k)] @ Wjk.T
                if (i, j) in S:
                    S[(i, j)] -= upd
                else:
                    S[(i, j)] = -upd
    return FactorBK(Lt, D, piv, sizes, struct, None, m)


def block_solve_bk(F: FactorBK, B: np.ndarray) -> np.ndarray:
    """X = K^{-1} B with P K P^T = Lt D Lt^T (P: the block order F.perm); B in the original numbering."""
    m, N = F.m, F.nblk
    perm = F.perm
    B = np.asarray(B, dtype=np.complex128)
    if B.ndim == 1:
        B = B[:, None]
    Y = [B[perm[k] * m:(perm[k] + 1) * m, :].copy() for k in range(N)]
    for k in range(N):                                   # forward: Lt y = P b
        Y[k] = np.linalg.solve(F.Lt[(k, k)], Y[k])
        for i in F.struct[k]:
            Y[i] -= F.Lt[(i, k)] @ Y[k]
    Z = [np.linalg.solve(F.D[k], Y[k]) for k in range(N)]   # diagonal: D z = y
    for k in reversed(range(N)):                         # backward: Lt^T w = z
        for i in F.struct[k]:
            Z[k] -= F.Lt[(i, k)].T @ Z[i]
        Z[k] = np.linalg.solve(F.Lt[(k, k)].T, Z[k])
    X = np.zeros_like(B)
    for k in range(N):                                   # x = P^T w
        X[perm[k] * m:(perm[k] + 1) * m, :] = Z[k]
    return X
