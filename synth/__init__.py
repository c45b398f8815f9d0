"""Seeded synthetic inputs for the D3M dual system (shared by the oracle, the tests and the bench).

This module only *makes inputs*.  It holds none of the factorization or solve arithmetic:
it draws random numbers, builds the per-domain dense blocks that stand in for the primal
reduction (the per-domain dual matrices of the paper's Sec. II, which need FEM meshes and are out of
scope), and adds them into the interface-block pattern of the reduced matrix K
(Fig. 1(b): one dense block per pair of interfaces that share a domain).

Conventions
-----------
* Domain grid nx x ny x nz, domain id d = (ix*ny + iy)*nz + iz (ix varies slowest).
* Interface f = (domain d, neighbour d + e_axis); enumerated in domain order, then axis
  order x, y, z.  Outer-boundary faces carry no dual unknowns.
* I(i) = interfaces of domain i sorted by global id; r_i = |I(i)| * m.
* M_i = G G^T - k^2 eps_i I + i tau I with G in C^{r_i x r_i}, G_ab = (N(0,1) + i N(0,1)) /
  sqrt(2 r_i) (transpose, not conjugate transpose).  With real_g=True, G is real with
  N(0,1)/sqrt(r_i) entries, so that Im(K) = 2 tau I exactly.
* K is stored as its lower block triangle in block-CSC order (diagonal block first in each
  column, rows ascending), each block m x m column-major, complex128.
* Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with the Box-Muller
  transform; the stream of one matrix row is keyed by (seed, tag) and counted by
  (j, row, domain, 0).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------------------
# Philox4x32-10 (counter-based RNG, published definition)
# --------------------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

TAG_G = 1
TAG_B = 2
TAG_C = 3
TAG_EPS = 4
TAG_BATCH = 5


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Ten Philox4x32 rounds on arrays of 32-bit counters (as uint64 arrays).

    Returns four uint64 arrays holding 32-bit outputs.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = c0 * _PHILOX_M0
        p1 = c2 * _PHILOX_M1
        hi0, lo0 = p0 >> _S32, p0 & _MASK32
        hi1, lo1 = p1 >> _S32, p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + _PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + _PHILOX_W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def _unit_open(x):
    """32-bit integer -> uniform double in (0, 1)."""
    return (x.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)


def normal_rows(seed: int, tag: int, domain: int, rows, count: int) -> np.ndarray:
    """Standard normals, `count` per row for each row id in `rows` -> (len(rows), count)."""
    rows = np.asarray(rows, dtype=np.uint64)
    nblk = (count + 3) // 4
    j = np.arange(nblk, dtype=np.uint64)
    c0 = np.broadcast_to(j[None, :], (rows.size, nblk))
    c1 = np.broadcast_to(rows[:, None], (rows.size, nblk))
    c2 = np.full((rows.size, nblk), domain, dtype=np.uint64)
    c3 = np.zeros((rows.size, nblk), dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(c0, c1, c2, c3, seed, tag)
    out = np.empty((rows.size, nblk, 4), dtype=np.float64)
    for (ua, ub, ia, ib) in ((x0, x1, 0, 1), (x2, x3, 2, 3)):
        rad = np.sqrt(-2.0 * np.log(_unit_open(ua)))
        ang = (2.0 * math.pi) * _unit_open(ub)
        out[:, :, ia] = rad * np.cos(ang)
        out[:, :, ib] = rad * np.sin(ang)
    return out.reshape(rows.size, nblk * 4)[:, :count]


def _philox_torch(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32-10 on torch int64 tensors holding 32-bit values.  The 32x32-bit products
    are formed as wrapping 64-bit products, whose high and low 32-bit halves are exact."""
    mask = 0xFFFFFFFF
    k0 = int(k0) & mask
    k1 = int(k1) & mask
    for _ in range(10):
        p0 = c0 * 0xD2511F53
        p1 = c2 * 0xCD9E8D57
        hi0, lo0 = (p0 >> 32) & mask, p0 & mask
        hi1, lo1 = (p1 >> 32) & mask, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _PHILOX_W0) & mask
        k1 = (k1 + _PHILOX_W1) & mask
    return c0, c1, c2, c3


def normal_rows_torch(seed: int, tag: int, domain: int, nrows: int, count: int, device):
    """Same stream as normal_rows for rows 0..nrows-1, computed with torch on `device`
    (equal to the numpy draw up to the rounding of log / sqrt / cos / sin)."""
    import torch
    nblk = (count + 3) // 4
    j = torch.arange(nblk, dtype=torch.int64, device=device)
    r = torch.arange(nrows, dtype=torch.int64, device=device)
    c0 = j[None, :].expand(nrows, nblk)
    c1 = r[:, None].expand(nrows, nblk)
    c2 = torch.full((nrows, nblk), domain, dtype=torch.int64, device=device)
    c3 = torch.zeros((nrows, nblk), dtype=torch.int64, device=device)
    x0, x1, x2, x3 = _philox_torch(c0, c1, c2, c3, seed, tag)
    out = torch.empty((nrows, nblk, 4), dtype=torch.float64, device=device)
    scale = 1.0 / 4294967296.0
    for (ua, ub, ia, ib) in ((x0, x1, 0, 1), (x2, x3, 2, 3)):
        rad = torch.sqrt(-2.0 * torch.log((ua.to(torch.float64) + 0.5) * scale))
        ang = (2.0 * math.pi) * ((ub.to(torch.float64) + 0.5) * scale)
        out[:, :, ia] = rad * torch.cos(ang)
        out[:, :, ib] = rad * torch.sin(ang)
    return out.reshape(nrows, nblk * 4)[:, :count]


def uniform01(seed: int, tag: int, ids) -> np.ndarray:
    """One uniform (0,1) double per id (counter (id, 0, 0, 0))."""
    ids = np.asarray(ids, dtype=np.uint64)
    z = np.zeros_like(ids)
    x0, _, _, _ = philox4x32_10(ids, z, z, z, seed, tag)
    return _unit_open(x0)


def complex_normal_rows(seed: int, tag: int, domain: int, rows, ncols: int) -> np.ndarray:
    """(N(0,1) + i N(0,1)) entries, row-major draw: entry c uses normals 2c (re), 2c+1 (im)."""
    z = normal_rows(seed, tag, domain, rows, 2 * ncols)
    return z[:, 0::2] + 1j * z[:, 1::2]


# --------------------------------------------------------------------------------------
# Domain grid topology
# --------------------------------------------------------------------------------------
def domain_id(nx, ny, nz, ix, iy, iz):
    return (ix * ny + iy) * nz + iz


def interfaces(nx: int, ny: int, nz: int):
    """List of (domain, axis, neighbour) in global interface order."""
    out = []
    for ix in range(nx):
        for iy in range(ny):
            for iz in range(nz):
                d = domain_id(nx, ny, nz, ix, iy, iz)
                if ix + 1 < nx:
                    out.append((d, 0, domain_id(nx, ny, nz, ix + 1, iy, iz)))
                if iy + 1 < ny:
                    out.append((d, 1, domain_id(nx, ny, nz, ix, iy + 1, iz)))
                if iz + 1 < nz:
                    out.append((d, 2, domain_id(nx, ny, nz, ix, iy, iz + 1)))
    return out


def domain_interfaces(nx: int, ny: int, nz: int):
    """I(i): sorted interface ids of every domain."""
    nd = nx * ny * nz
    lists = [[] for _ in range(nd)]
    for f, (d, _ax, e) in enumerate(interfaces(nx, ny, nz)):
        lists[d].append(f)
        lists[e].append(f)
    return [sorted(l) for l in lists]


def lower_pattern(nx: int, ny: int, nz: int):
    """Lower block-CSC pattern of K (diagonal included): (colptr int64, rowidx int32)."""
    nf = len(interfaces(nx, ny, nz))
    cols = [set([g]) for g in range(nf)]
    for I in domain_interfaces(nx, ny, nz):
        for a in I:
            for b in I:
                if a >= b:
                    cols[b].add(a)
    colptr = np.zeros(nf + 1, dtype=np.int64)
    rowidx = []
    for g in range(nf):
        rs = sorted(cols[g])
        rowidx.extend(rs)
        colptr[g + 1] = colptr[g] + len(rs)
    return colptr, np.asarray(rowidx, dtype=np.int32)


# --------------------------------------------------------------------------------------
# Problem assembly
# --------------------------------------------------------------------------------------
@dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    m: int
    k2: float
    tau: float
    seed: int
    eps: np.ndarray                    # per-domain epsilon_i
    colptr: np.ndarray                 # int64 [N+1]
    rowidx: np.ndarray                 # int32 [nnzb]
    blocks: object                     # complex128 flat array (numpy or torch), lower blocks
    blk_off: np.ndarray                # int64 [nnzb+1] element offsets into `blocks`
    dom_if: list = field(default_factory=list)   # I(i)
    real_g: bool = False

    @property
    def nblk(self) -> int:
        return self.colptr.size - 1

    @property
    def n(self) -> int:
        return self.nblk * self.m

    def block(self, e: int) -> np.ndarray:
        """Block e (CSC order) as an m x m numpy array (row, col)."""
        b = self.blocks[self.blk_off[e]:self.blk_off[e + 1]]
        if not isinstance(b, np.ndarray):
            b = b.cpu().numpy()
        return b.reshape(self.m, self.m).T

    def blocks_numpy(self) -> np.ndarray:
        b = self.blocks
        return b if isinstance(b, np.ndarray) else b.cpu().numpy()


def domain_G(seed: int, dom: int, r: int, real_g: bool = False) -> np.ndarray:
    rows = np.arange(r)
    if real_g:
        return normal_rows(seed, TAG_G, dom, rows, r) / math.sqrt(r)
    return complex_normal_rows(seed, TAG_G, dom, rows, r) / math.sqrt(2.0 * r)


def domain_eps(seed: int, ndom: int, lo: float = 1.0, hi: float = 4.0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, TAG_EPS, np.arange(ndom))


def make_problem(nx, ny, nz, m, k2, tau, seed, eps=None, real_g=False, device=None, domains=None) -> Problem:
    """Assemble K's lower blocks.  `device`: None for numpy, or a torch device ("cpu", "cuda")
    for the random draws and the G G^T products (the result is then a torch complex128
    tensor on that device).  `domains`: None for every domain, or a collection of domain ids
    whose blocks M_i alone are added (the others contribute nothing).  A block K_fg is then
    exact when every domain holding both f and g is listed (``interface_domains`` of g's
    column gives such a set), and partial otherwise."""
    dom_if = domain_interfaces(nx, ny, nz)
    ndom = nx * ny * nz
    colptr, rowidx = lower_pattern(nx, ny, nz)
    nf = colptr.size - 1
    if eps is None:
        eps = np.ones(ndom)
    eps = np.asarray(eps, dtype=np.float64)
    nnzb = rowidx.size
    blk_off = np.arange(nnzb + 1, dtype=np.int64) * (m * m)
    # (row, col) -> block index
    pos = {}
    for g in range(nf):
        for e in range(colptr[g], colptr[g + 1]):
            pos[(int(rowidx[e]), g)] = e
    use_torch = device is not None
    if use_torch:
        import torch
        blocks = torch.zeros(nnzb * m * m, dtype=torch.complex128, device=device)
    else:
        blocks = np.zeros(nnzb * m * m, dtype=np.complex128)
    for i in range(ndom):
        I = dom_if[i]
        r = len(I) * m
        if r == 0 or (domains is not None and i not in domains):
            continue
        sigma = -k2 * eps[i] + 1j * tau
        if use_torch:
            import torch
            z = normal_rows_torch(seed, TAG_G, i, r, r if real_g else 2 * r, device)
            if real_g:
                Gt = (z / math.sqrt(r)).to(torch.complex128)
            else:
                Gt = torch.complex(z[:, 0::2], z[:, 1::2]) / math.sqrt(2.0 * r)
            M = Gt @ Gt.T
            M.diagonal().add_(sigma)
        else:
            G = domain_G(seed, i, r, real_g).astype(np.complex128)
            M = G @ G.T
            M[np.diag_indices(r)] += sigma
        for a, f in enumerate(I):
            for b, g in enumerate(I):
                if f < g:
                    continue
                e = pos[(f, g)]
                sub = M[a * m:(a + 1) * m, b * m:(b + 1) * m]
                # column-major storage of block (f, g): flat index c*m + r  <=>  sub.T row-major
                if use_torch:
                    blocks[blk_off[e]:blk_off[e + 1]] += sub.T.contiguous().reshape(-1)
                else:
                    blocks[blk_off[e]:blk_off[e + 1]] += sub.T.reshape(-1)
    return Problem(nx, ny, nz, m, float(k2), float(tau), int(seed), eps, colptr, rowidx,
                   blocks, blk_off, dom_if, real_g)


def interface_domains(nx: int, ny: int, nz: int, ifaces) -> set:
    """The domains adjacent to the listed interfaces (each interface joins two domains).  Every
    K block K_fg with g in the list sums M_i over domains i containing g, so generating these
    domains makes the columns of the listed interfaces exact."""
    ifs = interfaces(nx, ny, nz)
    out = set()
    for f in ifaces:
        d, _ax, e = ifs[int(f)]
        out.add(d)
        out.add(e)
    return out


def rhs(seed: int, n: int, nrhs: int, tag: int = TAG_B) -> np.ndarray:
    """Complex N(0,1) right-hand sides, (N+iN)/sqrt(2), shape (n, nrhs), Fortran order."""
    z = complex_normal_rows(seed, tag, 0, np.arange(n), nrhs) / math.sqrt(2.0)
    return np.asfortranarray(z)


def sparse_adjoint_vector(seed: int, n: int, m: int, support_block: int, nrhs: int = 1) -> np.ndarray:
    """c ~ complex N(0,1) on the unknowns of one interface block, zero elsewhere."""
    c = np.zeros((n, nrhs), dtype=np.complex128, order="F")
    rows = np.arange(support_block * m, (support_block + 1) * m)
    c[rows, :] = complex_normal_rows(seed, TAG_C, 0, rows, nrhs) / math.sqrt(2.0)
    return c


# Named workloads (grid, m, k^2, tau, nrhs, seed)
WORKLOADS = {
    "grid2x2_m64": dict(nx=2, ny=2, nz=1, m=64, k2=1.0, tau=0.1, nrhs=1, seed=20260101),
    "grid8x8_m512": dict(nx=8, ny=8, nz=1, m=512, k2=2.0, tau=0.05, nrhs=8, seed=20260102),
    "grid6x6x6_m512": dict(nx=6, ny=6, nz=6, m=512, k2=4.0, tau=0.02, nrhs=32, seed=20260103),
    "grid4x4_m512": dict(nx=4, ny=4, nz=1, m=512, k2=2.0, tau=0.05, nrhs=8, seed=20260106),
    "adjoint8x8_m256": dict(nx=8, ny=8, nz=1, m=256, k2=2.0, tau=0.05, nrhs=1, seed=20260104),
}


def batch_instances(count: int, seed: int = 20260105):
    """Uneven instances: grid from {2x2,3x3,4x4,6x6}, m from {64,128,256},
    k^2 ~ U(0.5,4), tau ~ U(0.01,0.2), 4 RHS each; instance seed = seed + index."""
    grids = [(2, 2), (3, 3), (4, 4), (6, 6)]
    ms = [64, 128, 256]
    out = []
    ids = np.arange(count)
    u = [uniform01(seed, TAG_BATCH, ids * 4 + t) for t in range(4)]
    for i in range(count):
        g = grids[min(int(u[0][i] * 4), 3)]
        mm = ms[min(int(u[1][i] * 3), 2)]
        out.append(dict(nx=g[0], ny=g[1], nz=1, m=mm, k2=0.5 + 3.5 * u[2][i],
                        tau=0.01 + 0.19 * u[3][i], nrhs=4, seed=seed + i))
    return out
