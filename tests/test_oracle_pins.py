"""Pins of the CPU oracle against facts fixed by mathematics or by hand-worked examples.

Each test checks the oracle against something other than itself: an independent library
routine, a closed form, an invariant, a hand-derived case, or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(nx, ny, nz, m, k2=1.0, tau=0.1, seed=7, eps=None, real_g=False):
    p = synth.make_problem(nx, ny, nz, m, k2, tau, seed, eps=eps, real_g=real_g)
    Kb = O.lower_blocks(p.colptr, p.rowidx, p.blocks, p.m)
    return p, Kb


def _factor(p, Kb, perm=None):
    perm = O.nd_order(p.nx, p.ny, p.nz) if perm is None else np.asarray(perm)
    F = O.block_ldlt(O.permute_lower(Kb, perm), p.nblk, p.m)
    F.perm = perm
    return F


def _perm_index(perm, m):
    return np.concatenate([np.arange(perm[k] * m, (perm[k] + 1) * m) for k in range(len(perm))])


# ---------------------------------------------------------------- input generator pins
def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = synth.philox4x32_10([v[0]], [v[1]], [v[2]], [v[3]], v[4], v[5])
        assert [int(o[0]) for o in out] == v[6:10]


def test_normals_moments():
    z = synth.normal_rows(3, 1, 0, np.arange(400), 1000).ravel()
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_lower_pattern_closed_form():
    # two interfaces couple only through a shared domain, and two distinct interfaces share
    # at most one domain: #lower blocks = #interfaces + sum_i C(|I(i)|, 2)
    for g in [(2, 2, 1), (8, 8, 1), (6, 6, 6), (3, 4, 2)]:
        cp, ri = synth.lower_pattern(*g)
        deg = [len(I) for I in synth.domain_interfaces(*g)]
        nf = len(synth.interfaces(*g))
        assert cp.size - 1 == nf
        assert ri.size == nf + sum(d * (d - 1) // 2 for d in deg)
    # interface counts: (nx-1) ny nz + nx (ny-1) nz + nx ny (nz-1)
    assert len(synth.interfaces(8, 8, 1)) == 112
    assert len(synth.interfaces(6, 6, 6)) == 540


def test_oracle_interfaces_match_generator():
    for g in [(2, 2, 1), (3, 4, 2), (6, 6, 6)]:
        a = [(d, ax) for (d, ax, _e) in synth.interfaces(*g)]
        b = [(synth.domain_id(*g, *c), ax) for (c, ax) in O.grid_interfaces(*g)]
        assert a == b


def test_real_g_imaginary_part():
    # with real G, Im(M_i) = tau I, so Im(K) = 2 tau I exactly (each unknown in two domains)
    p, Kb = _problem(3, 3, 1, 4, tau=0.07, real_g=True)
    A = O.dense_from_lower(Kb, p.nblk, p.m)
    assert np.array_equal(A.imag, np.diag(np.full(p.n, 2 * 0.07)))


# ---------------------------------------------------------------- ordering
def test_nd_order_hand_examples():
    for line in open(os.path.join(GOLDEN, "nd_order_small.txt")):
        if line.startswith("#") or not line.strip():
            continue
        g, perm = line.split(":")
        g = tuple(int(t) for t in g.split())
        assert O.nd_order(*g).tolist() == [int(t) for t in perm.split()]


def test_nd_top_separator_8x8():
    # the last 8 interfaces are the x-interfaces between ix = 3 and ix = 4, natural order
    perm = O.nd_order(8, 8, 1)
    ifs = O.grid_interfaces(8, 8, 1)
    top = [f for f, (c, ax) in enumerate(ifs) if ax == 0 and c[0] == 3]
    assert perm[-8:].tolist() == top
    assert sorted(perm.tolist()) == list(range(112))


def test_nd_separator_property():
    # in ND order, an interface's block column never connects two different subtrees:
    # equivalently the elimination fill only connects ancestors, i.e. every struct(k)
    # lies on the etree path from k to the root.
    for g in [(8, 8, 1), (4, 4, 4), (5, 3, 2)]:
        perm = O.nd_order(*g)
        keys = _perm_keys(g, perm)
        st, par = O.block_symbolic(len(perm), keys)
        for k, s in enumerate(st):
            path, a = set(), par[k]
            while a >= 0:
                path.add(a)
                a = par[a]
            assert set(s) <= path


def _perm_keys(g, perm):
    cp, ri = synth.lower_pattern(*g)
    inv = np.empty(len(perm), dtype=int)
    inv[perm] = np.arange(len(perm))
    keys = []
    for c in range(cp.size - 1):
        for e in range(cp[c], cp[c + 1]):
            i, j = inv[ri[e]], inv[c]
            keys.append((max(i, j), min(i, j)))
    return keys


def test_symbolic_matches_elimination_game():
    for g in [(2, 2, 1), (8, 8, 1), (4, 4, 4), (6, 6, 6)]:
        perm = O.nd_order(*g)
        keys = _perm_keys(g, perm)
        st, _ = O.block_symbolic(len(perm), keys)
        assert st == O.elimination_fill(len(perm), keys)


def test_symbolic_hand_count_2x2():
    # 2x2 grid in ND order [f1, f3, f0, f2]: columns 0 and 1 couple to the separator {2, 3};
    # column 2 picks up fill (3,2) from both; 5 off-diagonal L blocks, etree 0,1 -> 2 -> 3.
    perm = O.nd_order(2, 2, 1)
    st, par = O.block_symbolic(4, _perm_keys((2, 2, 1), perm))
    assert st == [[2, 3], [2, 3], [3], []]
    assert par == [2, 2, 3, -1]
    assert O.factor_flops(st, 64) == pytest.approx(64 ** 3 * (4 * 4 / 3 + 5 * 4 + 5 * 4 + 2 * 8))


# ---------------------------------------------------------------- brute force
def test_dense_lu_matches_library_solve():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(60, 60)) + 1j * rng.normal(size=(60, 60))
    B = rng.normal(size=(60, 3)) + 1j * rng.normal(size=(60, 3))
    LU, piv = O.lu_factor_pp(A)
    X = O.lu_solve_pp(LU, piv, B)
    ref = np.linalg.solve(A, B)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("g,m", [((2, 2, 1), 8), ((3, 3, 1), 4), ((2, 2, 2), 3), ((1, 5, 1), 6)])
def test_block_solve_matches_dense_lu(g, m):
    p, Kb = _problem(*g, m, k2=1.3, tau=0.1, seed=11)
    F = _factor(p, Kb)
    B = synth.rhs(5, p.n, 3)
    X = O.block_solve(F, B)
    A = O.dense_from_lower(Kb, p.nblk, p.m)
    LU, piv = O.lu_factor_pp(A)
    ref = O.lu_solve_pp(LU, piv, B)
    assert np.max(np.linalg.norm(X - ref, axis=0) / np.linalg.norm(ref, axis=0)) < 1e-12
    assert np.max(O.omega(Kb, p.nblk, p.m, X, B)) < 1e-14


@pytest.mark.parametrize("g,m", [((2, 2, 1), 16), ((3, 3, 1), 5), ((2, 2, 2), 4)])
def test_reconstruction_and_symmetry(g, m):
    p, Kb = _problem(*g, m, seed=3)
    F = _factor(p, Kb)
    A = O.dense_from_lower(Kb, p.nblk, p.m)
    idx = _perm_index(F.perm, m)
    PA = A[np.ix_(idx, idx)]
    L, d = F.dense_L(), F.dense_D()
    R = L @ np.diag(d) @ L.T
    assert np.linalg.norm(PA - R) / np.linalg.norm(PA) < 1e-13
    assert np.linalg.norm(R - R.T) / np.linalg.norm(R) < 1e-15
    assert np.allclose(np.diag(L), 1.0) and np.count_nonzero(np.triu(L, 1)) == 0


def test_schur_blocks_symmetric():
    p, Kb = _problem(3, 3, 1, 6, seed=5)
    perm = O.nd_order(3, 3, 1)
    F = O.block_ldlt(O.permute_lower(Kb, perm), p.nblk, p.m, ncols=5)
    for (i, j), S in F.S.items():
        if i == j:
            assert np.linalg.norm(S - S.T) <= 1e-15 * np.linalg.norm(S)


def test_unpivoted_ldlt_small_closed_form():
    # 2x2 symmetric: d0 = a, l = b / a, d1 = c - b^2 / a  (no conjugation)
    a, b, c = 2 - 1j, 0.5 + 2j, -1 + 0.25j
    L, d = O.ldlt_unpivoted(np.array([[a, b], [b, c]]))
    assert d[0] == a and np.isclose(L[1, 0], b / a) and np.isclose(d[1], c - b * b / a)


# ---------------------------------------------------------------- structure pins
def test_decoupled_blocks_factor_independently():
    # several 2x1x1 problems (one interface each) on the diagonal: K is block diagonal,
    # L has no off-diagonal blocks, and every block's factor equals its stand-alone factor
    m = 12
    singles = [_problem(2, 1, 1, m, seed=40 + s)[1][(0, 0)] for s in range(4)]
    Kp = {(k, k): singles[k] for k in range(4)}
    F = O.block_ldlt(Kp, 4, m)
    assert all(i == j for (i, j) in F.L)
    for k in range(4):
        L1, d1 = O.ldlt_unpivoted(singles[k])
        assert np.array_equal(F.L[(k, k)], L1) and np.array_equal(F.D[k], d1)


def _chebyshev_u(N, x):
    u_prev, u = 1.0 + 0j, 2 * x
    if N == 0:
        return u_prev
    for _ in range(N - 1):
        u_prev, u = u, 2 * x * u - u_prev
    return u


def test_block_thomas_scalar_toeplitz():
    # m = 1 chain, natural order: tridiagonal complex-symmetric Toeplitz (a on the diagonal,
    # b off it).  No fill, and the pivots are ratios of leading minors:
    # det(T_k) = b^k U_k(a / 2b) (Chebyshev polynomials of the second kind).
    a, b, N = 2.5 + 0.3j, 0.9 - 0.4j, 9
    Kp = {(k, k): np.array([[a]]) for k in range(N)}
    Kp.update({(k + 1, k): np.array([[b]]) for k in range(N - 1)})
    F = O.block_ldlt(Kp, N, 1)
    assert all(i - j <= 1 for (i, j) in F.L)
    minors = [b ** k * _chebyshev_u(k, a / (2 * b)) for k in range(N + 1)]
    d = np.array([F.D[k][0] for k in range(N)])
    assert np.allclose(d, [minors[k + 1] / minors[k] for k in range(N)], rtol=1e-12)
    assert np.isclose(np.prod(d), minors[N], rtol=1e-11)


def test_block_thomas_scaled_identity():
    # K_kk = alpha I, K_{k+1,k} = beta I: the block pivots are d_k I with the scalar
    # recursion d_0 = alpha, d_k = alpha - beta^2 / d_{k-1}; L_{k+1,k} = (beta / d_k) I.
    alpha, beta, m, N = 3.0 - 0.5j, 1.1 + 0.2j, 5, 6
    Kp = {(k, k): alpha * np.eye(m) for k in range(N)}
    Kp.update({(k + 1, k): beta * np.eye(m) for k in range(N - 1)})
    F = O.block_ldlt(Kp, N, m)
    dk = alpha
    for k in range(N):
        assert np.allclose(F.D[k], dk, rtol=1e-14)
        if k + 1 < N:
            assert np.allclose(F.L[(k + 1, k)], (beta / dk) * np.eye(m), rtol=1e-14)
        dk = alpha - beta * beta / dk


def test_chain_natural_order_no_fill():
    g = (7, 1, 1)
    p, Kb = _problem(*g, 3, seed=2)
    perm = np.arange(p.nblk)
    F = _factor(p, Kb, perm)
    assert sum(len(s) for s in F.struct) == p.nblk - 1


# ---------------------------------------------------------------- adjoint pins
def test_duality_identity():
    p, Kb = _problem(3, 3, 1, 5, seed=9)
    F = _factor(p, Kb)
    b = synth.rhs(1, p.n, 1)
    c = synth.rhs(2, p.n, 1)
    x = O.block_solve(F, b)
    lam = O.block_solve(F, c)
    lhs, rhs_ = (c.T @ x).item(), (lam.T @ b).item()
    assert abs(lhs - rhs_) <= 1e-13 * abs(lhs)


def test_eps_gradient_central_differences():
    g, m, k2, tau = (3, 3, 1), 4, 2.0, 0.05
    ndom = 9
    eps = synth.domain_eps(17, ndom)
    b = synth.rhs(3, len(synth.interfaces(*g)) * m, 1)
    c = synth.sparse_adjoint_vector(4, b.shape[0], m, support_block=2)

    def J(e):
        p, Kb = _problem(*g, m, k2=k2, tau=tau, seed=21, eps=e)
        F = _factor(p, Kb)
        return np.real((c.T @ O.block_solve(F, b)).item()), p, F

    J0, p, F = J(eps)
    x = O.block_solve(F, b)
    _lam, grad, _gb = O.adjoint_gradients(F, x, c, k2, p.dom_if, m)
    h = 1e-6
    for i in range(ndom):
        e1, e2 = eps.copy(), eps.copy()
        e1[i] += h
        e2[i] -= h
        fd = (J(e1)[0] - J(e2)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-5 * max(abs(grad).max(), 1e-300)


def test_rhs_gradient_central_differences():
    p, Kb = _problem(2, 2, 1, 3, seed=6)
    F = _factor(p, Kb)
    b = synth.rhs(8, p.n, 1)
    c = synth.rhs(9, p.n, 1)
    x = O.block_solve(F, b)
    _lam, _g, gb = O.adjoint_gradients(F, x, c, 1.0, p.dom_if, p.m)
    h = 1e-6
    for u in [0, 3, 7, 11]:
        for unit, comp in ((1.0, np.real), (1j, np.imag)):
            bp, bm = b.copy(), b.copy()
            bp[u] += h * unit
            bm[u] -= h * unit
            fd = (np.real(c.T @ O.block_solve(F, bp)) - np.real(c.T @ O.block_solve(F, bm))).item() / (2 * h)
            assert abs(fd - comp(gb[u, 0])) <= 1e-5 * np.abs(gb).max()


def test_pattern_gradient_directional_derivative():
    p, Kb = _problem(2, 2, 1, 3, seed=12)
    b = synth.rhs(8, p.n, 2)
    c = synth.rhs(9, p.n, 2)
    perm = O.nd_order(2, 2, 1)

    def J(K):
        F = O.block_ldlt(O.permute_lower(K, perm), p.nblk, p.m)
        F.perm = perm
        return np.real(np.sum(c * O.block_solve(F, b))), F

    J0, F = J(Kb)
    x = O.block_solve(F, b)
    lam = O.block_solve(F, c)
    G = O.pattern_gradient(Kb.keys(), p.m, lam, x)
    rng = np.random.default_rng(0)
    dK = {k: rng.normal(size=v.shape) + 1j * rng.normal(size=v.shape) for k, v in Kb.items()}
    for k in dK:                                      # keep the diagonal blocks symmetric
        if k[0] == k[1]:
            dK[k] = dK[k] + dK[k].T
    h = 1e-6
    Jp = J({k: Kb[k] + h * dK[k] for k in Kb})[0]
    Jm = J({k: Kb[k] - h * dK[k] for k in Kb})[0]
    fd = (Jp - Jm) / (2 * h)
    # J is real-linear in dK: dJ = Re(sum <G, dK>) with the unconjugated pairing; the
    # diagonal stored block appears once, so its symmetric gradient pairs with dK directly
    pred = np.real(sum(np.sum(G[k] * dK[k]) for k in Kb))
    assert abs(fd - pred) <= 1e-6 * abs(pred)


def test_torch_philox_matches_definition():
    torch = pytest.importorskip("torch")
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        c = [torch.tensor([v[i]], dtype=torch.int64) for i in range(4)]
        out = synth._philox_torch(*c, v[4], v[5])
        assert [int(o[0]) for o in out] == v[6:10]
    a = synth.normal_rows(5, 1, 3, np.arange(64), 130)
    b = synth.normal_rows_torch(5, 1, 3, 64, 130, "cpu").numpy()
    assert np.abs(a - b).max() < 1e-13


def test_residual_and_omega_hand_worked():
    """r = b - K x and omega = ||r||inf / (||K||inf ||x||inf + ||b||inf) (reading R7) on a 4 x 4 K
    stored by its lower blocks (m = 2; K complex symmetric: the upper block is the TRANSPOSE of the
    stored lower one, not its conjugate).  Worked by hand:
        K = [[1, 0, 0,  0 ], [0, 1, 3i, 0], [0, 3i, 0.5, 0], [0, 0, 0, 0.5]],  ||K||inf = 4,
        x = e_2, b = (0, 3i, 0, 0):  K x = (0, 3i, 0.5, 0),  r = (0, 0, -0.5, 0),  omega = 0.5 / 7.
    A dropped mirror block gives omega 3/7, a conjugated one 6/7, an untransposed one 3/7, and a
    norm from the lower triangle alone 1/13."""
    I2 = np.eye(2, dtype=np.complex128)
    K10 = np.array([[0, 3j], [0, 0]], dtype=np.complex128)
    Kb = {(0, 0): I2, (1, 0): K10, (1, 1): 0.5 * I2}
    x = np.array([0, 0, 1, 0], dtype=np.complex128)[:, None]
    b = np.array([0, 3j, 0, 0], dtype=np.complex128)[:, None]
    r = O.residual(Kb, 2, x, b)
    assert np.array_equal(r[:, 0], np.array([0, 0, -0.5, 0], dtype=np.complex128))
    assert O.k_inf_norm(Kb, 2, 2) == 4.0
    assert O.omega(Kb, 2, 2, x, b)[0] == pytest.approx(0.5 / 7.0, rel=0, abs=1e-15)
    A = O.dense_from_lower(Kb, 2, 2)
    assert np.array_equal(A @ x[:, 0], np.array([0, 3j, 0.5, 0], dtype=np.complex128))
