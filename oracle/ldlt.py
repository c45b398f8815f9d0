"""Plain FP64 (complex128) oracle of the D3M factorization and solve of the dual matrix.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the bench's CPU baseline;
never by the library.  Plain numpy: every step is written out in the order of the method,
with library calls (matmul, triangular solve) only as single steps.

What it computes (paper Sec. I and II, the factorization and solve of the reduced matrix):
the reduced block-sparse matrix K (complex symmetric, K^T = K, not Hermitian) is put in a
nested-dissection interface order P, factored as  P K P^T = L D L^T  with L unit lower
triangular and D diagonal (scalar pivots, no pivoting; this pair is unique when all leading
principal minors are nonzero), and the system K X = B is solved by a forward sweep
(L y = P b), a diagonal step (z = D^{-1} y) and a backward sweep (L^T w = z, x = P^T w).
Per nonzero block the factorization does a dense update (GEMM), a dense triangular solve
and a dense factorization (Sec. II; the paper's BLAS names GEMM / triSolve / sytrf).

Readings where the paper is silent (all fixed here, nowhere else):
* ordering: geometric nested dissection over interfaces (function ``nd_order``);
* the diagonal-block factorization is unpivoted with scalar D (the paper's sytrf pivots;
  unpivoted LDL^T is the unique factor that the GPU path must reproduce entrywise);
* no conjugation anywhere (complex symmetric, not Hermitian);
* error metrics: normwise backward error omega per column (Rigal-Gaches) and relative
  forward error per column.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

__all__ = [
    "grid_interfaces", "nd_order", "lower_blocks", "permute_lower", "block_symbolic",
    "elimination_fill", "ldlt_unpivoted", "block_ldlt", "block_solve", "dense_from_lower",
    "lu_factor_pp", "lu_solve_pp", "residual", "omega", "adjoint_gradients",
    "pattern_gradient", "factor_flops", "Factor", "etree_depth", "k_inf_norm",
]


# --------------------------------------------------------------------------------------
# Topology and ordering
# --------------------------------------------------------------------------------------
def grid_interfaces(nx: int, ny: int, nz: int):
    """Interfaces of a domain grid as (domain coords (ix,iy,iz), axis), in global id order:
    domain order (ix slowest) then axis order x, y, z; an interface joins the domain with its
    +axis neighbour; outer boundary faces carry no unknowns."""
    out = []
    for ix in range(nx):
        for iy in range(ny):
            for iz in range(nz):
                for ax, ok in enumerate((ix + 1 < nx, iy + 1 < ny, iz + 1 < nz)):
                    if ok:
                        out.append(((ix, iy, iz), ax))
    return out


def nd_order(nx: int, ny: int, nz: int) -> np.ndarray:
    """Nested-dissection order of the interfaces of a domain grid, perm[new] = old.

    Reading of the method's interface ordering (the paper does not state one): split the
    current domain box along its longest extent (ties to the lower axis x < y < z) at
    mid = lo + floor(extent/2); the separator is the set of interfaces joining a domain at
    mid-1 to one at mid along that axis, ordered last in natural id order; recurse on the
    lower box then the upper box; a box whose extent is 1 in every axis, or which holds at
    most one interface, keeps its interfaces in natural order.
    """
    ifs = grid_interfaces(nx, ny, nz)

    def inside(c, lo, hi):
        return all(lo[a] <= c[a] < hi[a] for a in range(3))

    def rec(lo, hi):
        own = []
        for f, (c, ax) in enumerate(ifs):
            c2 = list(c)
            c2[ax] += 1
            if inside(c, lo, hi) and inside(c2, lo, hi):
                own.append(f)
        ext = [hi[a] - lo[a] for a in range(3)]
        if max(ext) <= 1 or len(own) <= 1:
            return own
        ax = int(np.argmax(ext))          # first maximum -> lowest axis on ties
        mid = lo[ax] + ext[ax] // 2
        sep = [f for f in own if ifs[f][1] == ax and ifs[f][0][ax] == mid - 1]
        lhi = list(hi)
        lhi[ax] = mid
        rlo = list(lo)
        rlo[ax] = mid
        return rec(lo, lhi) + rec(rlo, hi) + sep

    perm = rec([0, 0, 0], [nx, ny, nz])
    assert len(perm) == len(ifs)
    return np.asarray(perm, dtype=np.int32)


# --------------------------------------------------------------------------------------
# Block containers
# --------------------------------------------------------------------------------------
def lower_blocks(colptr, rowidx, flat, m: int):
    """Dict (row, col) -> m x m block from block-CSC lower storage (blocks column-major)."""
    out = {}
    e = 0
    for g in range(len(colptr) - 1):
        for e in range(colptr[g], colptr[g + 1]):
            f = int(rowidx[e])
            out[(f, g)] = np.asarray(flat[e * m * m:(e + 1) * m * m]).reshape(m, m).T.copy()
    return out


def permute_lower(Kb: dict, perm) -> dict:
    """Lower blocks of P K P^T: new block (i, j), i >= j, from old blocks (K symmetric)."""
    inv = np.empty(len(perm), dtype=np.int64)
    inv[np.asarray(perm)] = np.arange(len(perm))
    out = {}
    for (f, g), blk in Kb.items():
        i, j = int(inv[f]), int(inv[g])
        if i >= j:
            out[(i, j)] = blk.copy()
        else:
            out[(j, i)] = blk.T.copy()
    return out


def dense_from_lower(Kb: dict, nblk: int, m: int) -> np.ndarray:
    """Full dense symmetric matrix from lower blocks."""
    A = np.zeros((nblk * m, nblk * m), dtype=np.complex128)
    for (i, j), blk in Kb.items():
        A[i * m:(i + 1) * m, j * m:(j + 1) * m] = blk
        if i != j:
            A[j * m:(j + 1) * m, i * m:(i + 1) * m] = blk.T
    return A


# --------------------------------------------------------------------------------------
# Symbolic analysis (block level)
# --------------------------------------------------------------------------------------
def block_symbolic(nblk: int, keys):
    """Structure of the block factor by symbolic elimination: struct[k] = sorted rows i > k
    with L_ik != 0; parent[k] = min struct[k] (block elimination tree)."""
    rows = [set() for _ in range(nblk)]
    for (i, j) in keys:
        if i > j:
            rows[j].add(i)
    struct = [None] * nblk
    parent = [-1] * nblk
    for k in range(nblk):
        s = sorted(rows[k])
        struct[k] = s
        if s:
            p = s[0]
            parent[k] = p
            rows[p].update(x for x in s if x > p)
    return struct, parent


def elimination_fill(nblk: int, keys):
    """Fill by the graph elimination game (definition): eliminating vertex k joins all its
    not-yet-eliminated neighbours pairwise.  Returns struct lists like block_symbolic."""
    adj = [set() for _ in range(nblk)]
    for (i, j) in keys:
        if i != j:
            adj[i].add(j)
            adj[j].add(i)
    struct = []
    for k in range(nblk):
        nb = sorted(x for x in adj[k] if x > k)
        struct.append(nb)
        for a in nb:
            for b in nb:
                if a != b:
                    adj[a].add(b)
    return struct


def etree_depth(parent) -> int:
    depth = [1] * len(parent)
    for k in range(len(parent)):           # parents have larger ids
        if parent[k] >= 0:
            depth[parent[k]] = max(depth[parent[k]], depth[k] + 1)
    return max(depth) if depth else 0


def factor_flops(struct, m: int) -> float:
    """Algorithmic flops of the block factorization (complex MAC = 8 flops):
    N (4/3) m^3 (diagonal LDL^T) + n_L 4 m^3 (TRSM) + n_L 4 m^3 (diagonal-target updates)
    + n_off 8 m^3 (off-diagonal-target updates)."""
    nL = sum(len(s) for s in struct)
    noff = sum(len(s) * (len(s) - 1) // 2 for s in struct)
    N = len(struct)
    return N * (4.0 / 3.0) * m ** 3 + nL * 4.0 * m ** 3 + nL * 4.0 * m ** 3 + noff * 8.0 * m ** 3


# --------------------------------------------------------------------------------------
# Numeric factorization
# --------------------------------------------------------------------------------------
def ldlt_unpivoted(A: np.ndarray):
    """Scalar unpivoted LDL^T of a complex symmetric matrix (no conjugation), column by
    column:  d_c = A_cc - sum_{p<c} L_cp d_p L_cp ;
             L_rc = (A_rc - sum_{p<c} L_rp d_p L_cp) / d_c   (r > c).
    Returns (L unit lower, d)."""
    n = A.shape[0]
    L = np.eye(n, dtype=np.complex128)
    d = np.zeros(n, dtype=np.complex128)
    for c in range(n):
        w = d[:c] * L[c, :c]
        d[c] = A[c, c] - np.dot(L[c, :c], w)
        if c + 1 < n:
            L[c + 1:, c] = (A[c + 1:, c] - L[c + 1:, :c] @ w) / d[c]
    return L, d


class Factor:
    """Block factor of P K P^T: L[(i, j)] (i > j off-diagonal blocks; (k, k) unit lower
    diagonal blocks), D[k] (pivots of block column k), struct, perm."""

    def __init__(self, L, D, struct, perm, m):
        self.L, self.D, self.struct, self.perm, self.m = L, D, struct, np.asarray(perm), m

    @property
    def nblk(self):
        return len(self.D)

    def dense_L(self):
        n = self.nblk * self.m
        m = self.m
        out = np.zeros((n, n), dtype=np.complex128)
        for (i, j), blk in self.L.items():
            out[i * m:(i + 1) * m, j * m:(j + 1) * m] = blk
        return out

    def dense_D(self):
        return np.concatenate(self.D)


def block_ldlt(Kp: dict, nblk: int, m: int, ncols: int | None = None) -> Factor:
    """Right-looking block LDL^T of the permuted lower blocks Kp (new numbering).

    For block columns k = 0..N-1 (optionally only the first `ncols`):
      FACTOR  S_kk = L_kk D_k L_kk^T                      (unpivoted, scalar D)
      TRSM    L_jk = S_jk L_kk^{-T} D_k^{-1}   for j in struct(k)
      UPDATE  S_ij -= L_ik D_k L_jk^T          for i >= j in struct(k) (fill created)
    """
    S = {key: blk.copy() for key, blk in Kp.items()}
    struct, _parent = block_symbolic(nblk, Kp.keys())
    L = {}
    D = [None] * nblk
    last = nblk if ncols is None else ncols
    for k in range(last):
        Lkk, dk = ldlt_unpivoted(S.pop((k, k)))
        L[(k, k)] = Lkk
        D[k] = dk
        for j in struct[k]:
            Sjk = S.pop((j, k))
            # X L_kk^T = S_jk  <=>  L_kk X^T = S_jk^T
            Xt = sla.solve_triangular(Lkk, Sjk.T, lower=True, unit_diagonal=True)
            L[(j, k)] = Xt.T / dk[None, :]
        for a, j in enumerate(struct[k]):
            Wjk = L[(j, k)] * dk[None, :]          # L_jk D_k
            for i in struct[k][a:]:
                upd = L[(i, k)] @ Wjk.T
                if (i, j) in S:
                    S[(i, j)] -= upd
                else:
                    S[(i, j)] = -upd
    f = Factor(L, D, struct, None, m)
    f.S = S                                        # remaining Schur blocks (partial runs)
    return f


def block_solve(F: Factor, B: np.ndarray) -> np.ndarray:
    """X = K^{-1} B with P K P^T = L D L^T; B (n, nrhs) in the original numbering."""
    m, N = F.m, F.nblk
    perm = F.perm
    B = np.asarray(B, dtype=np.complex128)
    if B.ndim == 1:
        B = B[:, None]
    Y = [B[perm[k] * m:(perm[k] + 1) * m, :].copy() for k in range(N)]
    for k in range(N):                                   # forward: L y = P b
        Y[k] = sla.solve_triangular(F.L[(k, k)], Y[k], lower=True, unit_diagonal=True)
        for i in F.struct[k]:
            Y[i] -= F.L[(i, k)] @ Y[k]
    Z = [Y[k] / F.D[k][:, None] for k in range(N)]       # diagonal: z = D^{-1} y
    for k in reversed(range(N)):                         # backward: L^T w = z
        for i in F.struct[k]:
            Z[k] -= F.L[(i, k)].T @ Z[i]
        Z[k] = sla.solve_triangular(F.L[(k, k)].T, Z[k], lower=False, unit_diagonal=True)
    X = np.zeros_like(B)
    for k in range(N):                                   # x = P^T w
        X[perm[k] * m:(perm[k] + 1) * m, :] = Z[k]
    return X


# --------------------------------------------------------------------------------------
# Dense brute force: LU with partial pivoting (own code)
# --------------------------------------------------------------------------------------
def lu_factor_pp(A: np.ndarray):
    """Doolittle LU with partial (row) pivoting: P A = L U, packed in one array."""
    A = np.array(A, dtype=np.complex128)
    n = A.shape[0]
    piv = np.arange(n)
    for c in range(n):
        p = c + int(np.argmax(np.abs(A[c:, c])))
        if p != c:
            A[[c, p], :] = A[[p, c], :]
            piv[[c, p]] = piv[[p, c]]
        A[c + 1:, c] /= A[c, c]
        A[c + 1:, c + 1:] -= np.outer(A[c + 1:, c], A[c, c + 1:])
    return A, piv


def lu_solve_pp(LU, piv, B):
    B = np.asarray(B, dtype=np.complex128)
    X = B[piv].copy()
    n = LU.shape[0]
    for c in range(n):                                   # L y = P b (unit lower)
        X[c + 1:] -= np.outer(LU[c + 1:, c], X[c])
    for c in reversed(range(n)):                         # U x = y
        X[c] /= LU[c, c]
        X[:c] -= np.outer(LU[:c, c], X[c])
    return X


# --------------------------------------------------------------------------------------
# Residual, backward error, adjoint
# --------------------------------------------------------------------------------------
def residual(Kb: dict, m: int, X: np.ndarray, B: np.ndarray) -> np.ndarray:
    """r = b - K x with K given by its lower blocks (original numbering)."""
    R = np.array(B, dtype=np.complex128, copy=True)
    if R.ndim == 1:
        R = R[:, None]
        X = X[:, None]
    for (f, g), blk in Kb.items():
        R[f * m:(f + 1) * m] -= blk @ X[g * m:(g + 1) * m]
        if f != g:
            R[g * m:(g + 1) * m] -= blk.T @ X[f * m:(f + 1) * m]
    return R


def k_inf_norm(Kb: dict, nblk: int, m: int) -> float:
    """||K||_inf (max row sum of |K_uv|), using both triangles."""
    rows = np.zeros(nblk * m)
    for (f, g), blk in Kb.items():
        a = np.abs(blk)
        rows[f * m:(f + 1) * m] += a.sum(axis=1)
        if f != g:
            rows[g * m:(g + 1) * m] += a.sum(axis=0)
    return float(rows.max())


def omega(Kb: dict, nblk: int, m: int, X, B) -> np.ndarray:
    """Normwise backward error per column: ||b - Kx||_inf / (||K||_inf ||x||_inf + ||b||_inf)."""
    R = residual(Kb, m, X, B)
    X = X if X.ndim == 2 else X[:, None]
    B = B if B.ndim == 2 else B[:, None]
    kn = k_inf_norm(Kb, nblk, m)
    return np.abs(R).max(axis=0) / (kn * np.abs(X).max(axis=0) + np.abs(B).max(axis=0))


def adjoint_gradients(F: Factor, X: np.ndarray, C: np.ndarray, k2: float, dom_if, m: int):
    """For J = Re(sum_j c_j^T x_j) with K x = b:  lambda = K^{-1} c (same factors, K^T = K);
    dJ/deps_i = Re(k^2 sum_{u in unknowns of I(i)} lambda_u x_u) (dK/deps_i = -k^2 on the
    unknowns of I(i)); dJ/db in the Re + i Im convention = conj(lambda)."""
    Lam = block_solve(F, C)
    X = X if X.ndim == 2 else X[:, None]
    g = np.zeros(len(dom_if))
    for i, I in enumerate(dom_if):
        s = 0.0
        for f in I:
            s += np.sum(Lam[f * m:(f + 1) * m] * X[f * m:(f + 1) * m])
        g[i] = np.real(k2 * s)
    return Lam, g, np.conj(Lam)


def pattern_gradient(keys, m: int, Lam: np.ndarray, X: np.ndarray) -> dict:
    """dJ/dK on the stored lower blocks for J = Re(sum_j c_j^T x_j): the outer product -lambda x^T
    restricted to K's pattern; an off-diagonal stored block also stands for its transpose,
    so it collects -(lambda_f x_g^T + x_f lambda_g^T).  Summed over right-hand sides."""
    out = {}
    for (f, g) in keys:
        lf, lg = Lam[f * m:(f + 1) * m], Lam[g * m:(g + 1) * m]
        xf, xg = X[f * m:(f + 1) * m], X[g * m:(g + 1) * m]
        G = -(lf @ xg.T)
        if f != g:
            G -= xf @ lg.T
        out[(f, g)] = G
    return out
