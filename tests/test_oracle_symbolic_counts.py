"""Pins of the oracle's symbolic phase (Sec. II: the symbolic run of the sequential block
elimination that yields the task graph) to counts fixed outside the oracle.

* The structure counts of the benchmark workloads (the nested-dissection order of the domain
  grid, the interface-block pattern of K, the fill of the block factor) are compared with a
  count table worked out independently of this code: lower blocks of K, off-diagonal blocks of L
  after fill, elimination-tree depth, tallest column and the algorithmic factor flops.
* The elimination-tree depth is recomputed as the longest chain of the filled graph's
  elimination DAG (an edge k -> i for every fill-in row i of column k), and the off-diagonal
  block count from the update pairs of the graph elimination game, neither of which uses the
  parent recursion of ``block_symbolic`` or the closed-form sums of ``factor_flops``.
Only ``oracle`` and the input generator's pattern are used; the CUDA library is not loaded.
"""
import numpy as np
import pytest

import oracle as O
import synth


def _struct(nx, ny, nz):
    colptr, rowidx = synth.lower_pattern(nx, ny, nz)
    perm = O.nd_order(nx, ny, nz)
    N = colptr.size - 1
    inv = np.empty(N, dtype=np.int64)
    inv[perm] = np.arange(N)
    keys = []
    for g in range(N):
        for e in range(colptr[g], colptr[g + 1]):
            i, j = int(inv[rowidx[e]]), int(inv[g])
            keys.append((max(i, j), min(i, j)))
    st, par = O.block_symbolic(N, keys)
    return N, len(keys), keys, st, par


# (grid, m, N, lower blocks of K, off-diagonal L blocks, etree depth, tallest column, factor flops)
# (the flops as printed, to two or three significant digits)
TABLE = [
    ((2, 2, 1), 64, 4, 8, 5, 3, 2, "1.6e7"),
    ((8, 8, 1), 512, 112, 404, 760, 21, 11, "3.55e12"),
    ((6, 6, 6), 512, 540, 2772, 11576, 89, 53, "1.81e14"),
    ((8, 8, 1), 256, 112, 404, 760, 21, 11, "4.44e11"),
    ((2, 2, 1), 256, 4, 8, 5, 3, None, "1.0e9"),
    ((3, 3, 1), 256, 12, 34, 36, 8, None, "1.15e10"),
    ((4, 4, 1), 256, 24, 76, 92, 9, None, "3.33e10"),
    ((6, 6, 1), 256, 60, 208, 347, 17, None, "1.74e11"),
]


@pytest.mark.parametrize("g,m,N,nK,nL,depth,height,flops", TABLE)
def test_symbolic_counts_match_table(g, m, N, nK, nL, depth, height, flops):
    n, nkeys, _keys, st, par = _struct(*g)
    assert n == N
    assert nkeys == nK
    assert sum(len(s) for s in st) == nL
    assert O.etree_depth(par) == depth
    if height is not None:
        assert max(len(s) for s in st) == height
    # equal to the printed value within half a unit of its last digit
    mant, ex = flops.split("e")
    half_unit = 0.5 * 10.0 ** (int(ex) - (len(mant.split(".")[1]) if "." in mant else 0))
    assert abs(O.factor_flops(st, m) - float(flops)) <= half_unit


@pytest.mark.parametrize("g", [(2, 2, 1), (3, 3, 1), (8, 8, 1), (3, 3, 3), (4, 3, 2)])
def test_etree_depth_is_longest_elimination_chain(g):
    # depth of the elimination tree = number of columns on the longest path of the filled graph's
    # elimination DAG (every fill-in row of a column depends on it), by dynamic programming
    N, _nk, keys, _st, par = _struct(*g)
    fill = O.elimination_fill(N, keys)
    longest = [1] * N
    for k in range(N):
        for i in fill[k]:
            longest[i] = max(longest[i], longest[k] + 1)
    assert O.etree_depth(par) == max(longest)


@pytest.mark.parametrize("g,m", [((2, 2, 1), 64), ((3, 3, 1), 32), ((8, 8, 1), 512), ((3, 3, 3), 16)])
def test_factor_flops_from_elimination_game(g, m):
    # the elimination game eliminates column k against its d_k later neighbours: one diagonal
    # factorization, d_k triangular solves and d_k (d_k + 1) / 2 Schur updates of which d_k hit
    # diagonal blocks; flops per kind (complex multiply-add = 8): (4/3) m^3, 4 m^3, 4 m^3, 8 m^3
    N, _nk, keys, st, _par = _struct(*g)
    fill = O.elimination_fill(N, keys)
    flops = 0.0
    pairs = 0
    for k in range(N):
        d = len(fill[k])
        flops += (4.0 / 3.0) * m ** 3 + d * 4.0 * m ** 3
        for a in range(d):
            for b in range(a, d):
                flops += (4.0 if a == b else 8.0) * m ** 3
                pairs += 1
    assert O.factor_flops(st, m) == pytest.approx(flops, rel=1e-14)
    nL = sum(len(s) for s in st)
    assert pairs == nL + sum(len(s) * (len(s) - 1) // 2 for s in st)
