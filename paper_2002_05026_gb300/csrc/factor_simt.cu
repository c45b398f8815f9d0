// Persistent block-DAG factorization with a SIMT tile engine (tile edge 64).
//
// R = double: the plain FP64 (complex128) path; R = float: complex64 factors without tensor
// cores (used as the SIMT reference of the mixed path).
//
// Each task works on one lower tile (I, J) of L (paper Sec. II: per nonzero block a task doing
// the dense update, the dense triangular solve and the dense factorization):
//   1. S = S_in - sum_{K in segment} L_IK (D_K L_JK^T)   (S_in = K_IJ or the tile's accumulator)
//   UPDATE task: store S in the accumulator and stop.  FINAL task:
//   2a. I == J: unpivoted LDL^T of S in shared memory (scalar pivots, no conjugation),
//       breakdown check |d| >= piv_tol * max|S|; store L_JJ, D_J and L_JJ^{-1} (for the solve)
//   2b. I != J: L_IJ = S L_JJ^{-T} D_J^{-1} by a column sweep (right-looking triangular solve).
// Pivot mode (p.pivot): the diagonal tile is factored with Bunch-Kaufman symmetric pivoting
// inside the tile (1 x 1 and 2 x 2 pivots; the paper's dense kernel is sytrf, Sec. II):
// S = Lt D Lt^T with Lt = P^T L (row-permuted unit lower) and D block diagonal (d, and e for the
// sub-diagonal of each 2 x 2 block); the tile stores Lt, Lt^{-1} = L^{-1} P, d, e and the
// permutation, and the off-diagonal tiles become L_IJ = S Lt^{-T} D^{-1}, a product with the
// stored inverse; W = L D of the updates takes the 2 x 2 blocks into account.  Everything else
// (the task graph, the update order, the solve's tile products) is unchanged.
// GB300 FP64 runs at a small fraction of FP32 throughput, so the FP64 path is bound by the
// DFMA rate: a simple register-blocked 64x64 complex tile product is enough to saturate it.
#include <cuda_runtime.h>

#include "device.cuh"

namespace d3m {

namespace {
constexpr int TB = 64;     // tile edge
constexpr int LDS = 65;    // padded shared-memory row stride (elements)
constexpr int NTHR = 256;
}  // namespace

// Bunch-Kaufman LDL^T of the 64 x 64 diagonal tile S held in sA (lower triangle used), pivots
// inside the tile, alpha = (1 + sqrt(17)) / 8, magnitudes |Re| + |Im|:
//   lam = max_{i > k} |S_ik| (row r); |S_kk| >= alpha lam -> 1 x 1 at k;
//   else sigma = max_{j != r} |S_rj| over the remaining matrix;
//        |S_kk| sigma >= alpha lam^2 -> 1 x 1 at k;  |S_rr| >= alpha sigma -> swap k, r, 1 x 1;
//        else swap k + 1, r and take the 2 x 2 pivot on (k, k + 1).
// Swaps are symmetric interchanges of the remaining matrix and of the rows of L computed so far.
// Stores Lt = P^T L, Lt^{-1} = L^{-1} P (via X = L^{-1} by columns), d, e (2 x 2 sub-diagonals)
// and the permutation; reports the smallest / largest pivot magnitude (|d|, or sqrt|det| of a
// 2 x 2 block) and the breakdown test against max|S| like the unpivoted path.
template <typename R>
__device__ __noinline__ void diag_tile_bk(const FactorParams& p, const TileTask& T, int task, typename CT<R>::C* sA,
                                          typename CT<R>::C* sB, typename CT<R>::C* s_col, typename CT<R>::C* s_d,
                                          typename CT<R>::C* s_tmp, R* s_red) {
  using C = typename CT<R>::C;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int s_perm[TB];
  __shared__ C s_e[TB];
  __shared__ int s_sel[3];                       // step size, index swapped with r (or -1), r
  __shared__ R s_val[NTHR / 32];
  __shared__ int s_idx[NTHR / 32];
  constexpr R ALPHA = (R)0.6403882032022076;     // (1 + sqrt(17)) / 8
  auto abs1 = [](C z) -> R { return fabs(z.x) + fabs(z.y); };
  auto at = [&](int i, int j) -> C& { return i >= j ? sA[i * LDS + j] : sA[j * LDS + i]; };
  // max |S| over the real lower triangle (breakdown scale)
  R mx = 0;
  for (int i = tid; i < TB * TB; i += NTHR) {
    const int r = i >> 6, c = i & 63;
    if (c <= r && r < T.rv) mx = fmax(mx, (R)sqrt(cabs2(sA[r * LDS + c])));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[warp] = mx;
  if (tid < TB) {
    s_perm[tid] = tid;
    s_e[tid] = CT<R>::make(0, 0);
  }
  __syncthreads();
  R smax = 0;
  for (int w = 0; w < NTHR / 32; ++w) smax = fmax(smax, s_red[w]);
  __syncthreads();
  // argmax of v over threads (ties to the lowest index): result in s_val[0], s_idx[0]
  auto argmax = [&](R v, int idx) {
    for (int o = 16; o > 0; o >>= 1) {
      const R v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
    }
    if (lane == 0) { s_val[warp] = v; s_idx[warp] = idx; }
    __syncthreads();
    if (tid == 0) {
      R bv = s_val[0];
      int bi = s_idx[0];
      for (int w = 1; w < NTHR / 32; ++w)
        if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bi)) { bv = s_val[w]; bi = s_idx[w]; }
      s_val[0] = bv;
      s_idx[0] = bi;
    }
    __syncthreads();
  };
  int k = 0;
  while (k < TB) {
    // lam, r: the largest magnitude below the diagonal in column k
    argmax((tid > k && tid < TB) ? abs1(sA[tid * LDS + k]) : (R)-1, tid);
    const R lam = fmax(s_val[0], (R)0);
    const int r = (s_val[0] >= 0) ? s_idx[0] : k;
    const R akk = abs1(sA[k * LDS + k]);
    __syncthreads();
    int step = 1, sw = -1;
    if (!(akk >= ALPHA * lam) && lam > 0) {
      // sigma: the largest off-diagonal magnitude of row r in the remaining matrix
      argmax((tid >= k && tid < TB && tid != r) ? abs1(at(r, tid)) : (R)-1, tid);
      const R sigma = fmax(s_val[0], (R)0);
      __syncthreads();
      if (akk * sigma >= ALPHA * lam * lam) {
      } else if (abs1(sA[r * LDS + r]) >= ALPHA * sigma) {
        sw = k;
      } else {
        sw = k + 1;
        step = 2;
      }
    }
    // symmetric interchange of sw and r (sw < r unless sw == r)
    if (sw >= 0 && sw != r) {
      const int a = sw, b = r;
      if (tid < TB) {
        const int t = tid;
        if (t < k) {                                       // rows of L computed so far
          const C v = sA[a * LDS + t];
          sA[a * LDS + t] = sA[b * LDS + t];
          sA[b * LDS + t] = v;
        } else if (t == a) {                               // diagonal entries
          const C v = sA[a * LDS + a];
          sA[a * LDS + a] = sA[b * LDS + b];
          sA[b * LDS + b] = v;
        } else if (t < a) {                                // k <= t < a: row a <-> row b
          const C v = sA[a * LDS + t];
          sA[a * LDS + t] = sA[b * LDS + t];
          sA[b * LDS + t] = v;
        } else if (t > a && t < b) {                       // column a below a <-> row b left of b
          const C v = sA[t * LDS + a];
          sA[t * LDS + a] = sA[b * LDS + t];
          sA[b * LDS + t] = v;
        } else if (t > b) {                                // column a <-> column b below b
          const C v = sA[t * LDS + a];
          sA[t * LDS + a] = sA[t * LDS + b];
          sA[t * LDS + b] = v;
        }
        if (t == 0) {
          const int pv = s_perm[a];
          s_perm[a] = s_perm[b];
          s_perm[b] = pv;
        }
      }
      __syncthreads();
    }
    if (step == 1) {
      if (tid < TB) {
        const C d = sA[k * LDS + k];
        if (tid > k) s_col[tid] = cdiv(sA[tid * LDS + k], d);
        s_tmp[tid] = sA[tid * LDS + k];                    // the column before scaling
        if (tid == k) s_d[k] = d;
      }
      __syncthreads();
      // trailing update of the lower triangle: S_rs -= l_r S_sk for r >= s > k
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int rr = i >> 6, ss = i & 63;
        if (ss > k && rr >= ss) sA[rr * LDS + ss] = cfms(s_col[rr], s_tmp[ss], sA[rr * LDS + ss]);
      }
      __syncthreads();
      if (tid > k && tid < TB) sA[tid * LDS + k] = s_col[tid];
    } else {
      // 2 x 2 pivot D_k = [[a11, a21], [a21, a22]]: [l1 l2] = [c1 c2] D_k^{-1}
      const C a11 = sA[k * LDS + k], a21 = sA[(k + 1) * LDS + k], a22 = sA[(k + 1) * LDS + k + 1];
      const C det = csub(cmul(a11, a22), cmul(a21, a21));
      if (tid < TB) {
        const C c1 = (tid > k + 1) ? sA[tid * LDS + k] : CT<R>::make(0, 0);
        const C c2 = (tid > k + 1) ? sA[tid * LDS + k + 1] : CT<R>::make(0, 0);
        s_tmp[tid] = c1;                                   // columns before scaling
        sB[tid] = c2;
        s_col[tid] = cdiv(csub(cmul(c1, a22), cmul(c2, a21)), det);
        sB[TB + tid] = cdiv(csub(cmul(c2, a11), cmul(c1, a21)), det);
        if (tid == k) {
          s_d[k] = a11;
          s_d[k + 1] = a22;
          s_e[k] = a21;
        }
      }
      __syncthreads();
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int rr = i >> 6, ss = i & 63;
        if (ss > k + 1 && rr >= ss) {
          C v = cfms(s_col[rr], s_tmp[ss], sA[rr * LDS + ss]);
          sA[rr * LDS + ss] = cfms(sB[TB + rr], sB[ss], v);
        }
      }
      __syncthreads();
      if (tid > k + 1 && tid < TB) {
        sA[tid * LDS + k] = s_col[tid];
        sA[tid * LDS + k + 1] = sB[TB + tid];
      }
      if (tid == 0) sA[(k + 1) * LDS + k] = CT<R>::make(0, 0);   // L is unit lower inside the block
    }
    __syncthreads();
    k += step;
  }
  // X = L^{-1} (unit lower), column j by thread j: x_i = [i == j] - sum_{j <= t < i} L_it x_t
  if (tid < TB) {
    const int j = tid;
    for (int i = 0; i < TB; ++i) {
      C v = CT<R>::make(i == j ? (R)1 : (R)0, 0);
      if (i > j)
        for (int t = j; t < i; ++t) v = cfms(sA[i * LDS + t], sB[t * LDS + j], v);
      sB[i * LDS + j] = (i >= j) ? v : CT<R>::make(0, 0);
    }
  }
  __syncthreads();
  // stores: Lt = P^T L (row perm[i] of Lt = row i of L), Lt^{-1} = L^{-1} P (column perm[b] of
  // Lt^{-1} = column b of X), d, e, perm
  C* Lg = reinterpret_cast<C*>(p.L) + (int64_t)T.tile * TB * TB;
  C* Li = reinterpret_cast<C*>(p.Linv) + (int64_t)T.col * TB * TB;
  for (int i = tid; i < TB * TB; i += NTHR) {
    const int r = i >> 6, c = i & 63;
    const C one = CT<R>::make(c == r ? (R)1 : (R)0, 0);
    Lg[(int64_t)s_perm[r] * TB + c] = (c < r) ? sA[r * LDS + c] : one;
    Li[(int64_t)r * TB + s_perm[c]] = sB[r * LDS + c];
  }
  if (tid < TB) {
    reinterpret_cast<C*>(p.D)[(int64_t)T.col * TB + tid] = s_d[tid];
    reinterpret_cast<C*>(p.E)[(int64_t)T.col * TB + tid] = s_e[tid];
    p.piv[(int64_t)T.col * TB + tid] = s_perm[tid];
  }
  // pivot magnitudes: |d| of 1 x 1 pivots, sqrt|det| of 2 x 2 blocks (real unknowns only)
  if (tid < 32) {
    R amin = (R)3.0e38, amax = 0;
    for (int c = tid; c < T.cv; c += 32) {
      const bool first2 = c + 1 < TB && (s_e[c].x != 0 || s_e[c].y != 0);
      const bool second2 = c > 0 && (s_e[c - 1].x != 0 || s_e[c - 1].y != 0);
      R a;
      if (first2) {
        const C det = csub(cmul(s_d[c], s_d[c + 1]), cmul(s_e[c], s_e[c]));
        a = (R)sqrt(sqrt(cabs2(det)));
      } else if (second2) {
        continue;
      } else {
        a = (R)sqrt(cabs2(s_d[c]));
      }
      amin = fmin(amin, a);
      amax = fmax(amax, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
      amin = fmin(amin, __shfl_xor_sync(0xffffffffu, amin, o));
      amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    if (tid == 0) {
      record_pivot_stats(p.ctl, (float)amin, (float)amax);
      if (!(amin >= (R)p.piv_tol * smax)) set_error(p.ctl, D3M_ERR_PIVOT, task);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(NTHR, 1) factor_simt_kernel(FactorParams p) {
  using C = typename CT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sA = reinterpret_cast<C*>(smem_raw);       // [64][65]
  C* sB = sA + TB * LDS;                         // [64][65]
  __shared__ C s_col[TB];
  __shared__ C s_d[TB];
  __shared__ C s_tmp[TB];
  __shared__ R s_red[NTHR / 32];
  __shared__ int s_task, s_pending;
  if (threadIdx.x == 0) s_pending = -1;          // read and written by thread 0 only

  C* Lg = reinterpret_cast<C*>(p.L);
  C* Linv = reinterpret_cast<C*>(p.Linv);
  C* Dg = reinterpret_cast<C*>(p.D);
  C* Sacc = reinterpret_cast<C*>(p.Sacc);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  for (;;) {
    const int task = sched_pop(p, &s_task, &s_pending);
    if (task < 0) break;
    const TileTask T = p.tasks[task];

    // ---------------------------------------------------------------- 1. Schur updates
    C acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = CT<R>::make(0, 0);
    for (int e = 0; e < T.nk; ++e) {
      const KEntry ke = p.klist[T.kl_off + e];
      const C* La = Lg + (int64_t)ke.a_tile * TB * TB;
      const C* Lb = Lg + (int64_t)ke.b_tile * TB * TB;
      const C* dK = Dg + (int64_t)ke.kcol * TB;
      const C* eK = p.E ? reinterpret_cast<const C*>(p.E) + (int64_t)ke.kcol * TB : nullptr;
      __syncthreads();
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int r = i >> 6, c = i & 63;
        sA[r * LDS + c] = ld_cg(La + i);
        C w = cmul(ld_cg(Lb + i), ld_cg(dK + c));              // W_JK = L_JK D_K
        if (eK) {                                               // 2 x 2 blocks of D_K
          if (c + 1 < TB) w = cfma(ld_cg(Lb + i + 1), ld_cg(eK + c), w);
          if (c > 0) w = cfma(ld_cg(Lb + i - 1), ld_cg(eK + c - 1), w);
        }
        sB[r * LDS + c] = w;
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < TB; ++k) {
        C a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sA[(ty + 16 * i) * LDS + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = sB[(tx + 16 * j) * LDS + k];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = cfma(a[i], bb[j], acc[i][j]);
      }
    }
    __syncthreads();
    C* Sa = (T.sidx >= 0) ? Sacc + (int64_t)T.sidx * TB * TB : nullptr;
    if (T.flags & TF_UPDATE) {
      // partial update: accumulator <- S_in - sum over this segment
      C kin[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = ty + 16 * i, c = tx + 16 * j;
          kin[i][j] = (T.flags & TF_S_IN) ? ld_cg(Sa + r * TB + c) : k_entry<R>(T, p.K, r, c);
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Sa[(ty + 16 * i) * TB + tx + 16 * j] = csub(kin[i][j], acc[i][j]);
      sched_complete(p, task);
      continue;
    }
    {
      C kin[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int r = ty + 16 * i, c = tx + 16 * j;
          kin[i][j] = (T.flags & TF_S_IN) ? ld_cg(Sa + r * TB + c) : k_entry<R>(T, p.K, r, c);
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sA[(ty + 16 * i) * LDS + tx + 16 * j] = csub(kin[i][j], acc[i][j]);
    }
    __syncthreads();

    if ((T.flags & TF_DIAG) && p.pivot) {
      // ------------------------------------------------------------ 2a'. diagonal tile, pivoted
      diag_tile_bk<R>(p, T, task, sA, sB, s_col, s_d, s_tmp, s_red);
    } else if (T.flags & TF_DIAG) {
      // ------------------------------------------------------------ 2a. diagonal tile
      // max |S| over the real lower triangle; the upper triangle is zeroed to hold X^T, X = L^{-1}
      R mx = 0;
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int r = i >> 6, c = i & 63;
        if (c <= r) {
          if (r < T.rv) mx = fmax(mx, (R)sqrt(cabs2(sA[r * LDS + c])));
        } else {
          sA[r * LDS + c] = CT<R>::make(0, 0);
        }
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((tid & 31) == 0) s_red[tid >> 5] = mx;
      __syncthreads();
      if (tid == 0) {
        R v = 0;
        for (int w = 0; w < NTHR / 32; ++w) v = fmax(v, s_red[w]);
        s_red[0] = v;
      }
      // unpivoted LDL^T fused with the inverse of L (see the tensor-core engine): at step c,
      // l_r = S[r][c] / d_c and u_s = column c (X[c][s] above the diagonal, 1 on it, S[s][c]
      // below); rank-1 update of every (r > c, s <= r), S below / X^T above the diagonal.
      {
        const int tr = tid >> 4, tcol = tid & 15;
        for (int c = 0; c < TB; ++c) {
          if (tid < TB) {
            const C d = sA[c * LDS + c];
            const C v = sA[tid * LDS + c];
            if (tid > c) s_col[tid] = cdiv(v, d);
            s_tmp[tid] = (tid == c) ? CT<R>::make(1, 0) : v;
            if (tid == c) s_d[c] = d;
          }
          __syncthreads();
          C lr[4], us[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            lr[a] = s_col[tr + 16 * a];
            us[a] = s_tmp[tcol + 16 * a];
          }
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int r = tr + 16 * a;
            if (r <= c) continue;
            C v[4];
            int off[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {          // all loads of the row first
              const int s = tcol + 16 * q;
              off[q] = (s > c) ? r * LDS + s : s * LDS + r;
              if (s <= r) v[q] = sA[off[q]];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (tcol + 16 * q <= r) sA[off[q]] = cfms(lr[a], us[q], v[q]);
          }
          __syncthreads();
          if (tid > c && tid < TB) sA[tid * LDS + c] = s_col[tid];
        }
        __syncthreads();
      }
      const R smax = s_red[0];
      // pivot checks on the real (non-padding) unknowns
      if (tid < 32) {
        R amin = (R)3.0e38, amax = 0;
        for (int c = tid; c < T.cv; c += 32) {
          const R a = (R)sqrt(cabs2(s_d[c]));
          amin = fmin(amin, a);
          amax = fmax(amax, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
          amin = fmin(amin, __shfl_xor_sync(0xffffffffu, amin, o));
          amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        }
        if (tid == 0) {
          record_pivot_stats(p.ctl, (float)amin, (float)amax);
          if (!(amin >= (R)p.piv_tol * smax)) set_error(p.ctl, D3M_ERR_PIVOT, task);
        }
      }
      // store L_JJ (unit lower), D_J, and L_JJ^{-1} (from the transposed upper storage)
      C* Lt = Lg + (int64_t)T.tile * TB * TB;
      C* Li = Linv + (int64_t)T.col * TB * TB;
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int r = i >> 6, c = i & 63;
        const C one = CT<R>::make(c == r ? (R)1 : (R)0, 0);
        Lt[i] = (c < r) ? sA[r * LDS + c] : one;
        Li[i] = (c < r) ? sA[c * LDS + r] : one;
      }
      if (tid < TB) Dg[(int64_t)T.col * TB + tid] = s_d[tid];
    } else if (p.pivot) {
      // ------------------------------------------------------------ 2b'. off-diagonal, pivot mode
      // L_IJ = (S Lt_JJ^{-T}) D_J^{-1}: product with the stored inverse, then the 1 x 1 / 2 x 2
      // blocks of D_J^{-1} on the columns
      const C* Li = Linv + (int64_t)T.col * TB * TB;
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int r = i >> 6, c = i & 63;
        sB[r * LDS + c] = ld_cg(Li + i);
      }
      if (tid < TB) {
        s_d[tid] = ld_cg(Dg + (int64_t)T.col * TB + tid);
        s_col[tid] = ld_cg(reinterpret_cast<const C*>(p.E) + (int64_t)T.col * TB + tid);
      }
      __syncthreads();
      C x[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) x[i][j] = CT<R>::make(0, 0);
#pragma unroll 4
      for (int k = 0; k < TB; ++k) {
        C a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sA[(ty + 16 * i) * LDS + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = sB[(tx + 16 * j) * LDS + k];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) x[i][j] = cfma(a[i], bb[j], x[i][j]);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sA[(ty + 16 * i) * LDS + tx + 16 * j] = x[i][j];
      __syncthreads();
      C* Lt = Lg + (int64_t)T.tile * TB * TB;
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int r = i >> 6, c = i & 63;
        const C* row = sA + r * LDS;
        C v;
        if (c + 1 < TB && (s_col[c].x != 0 || s_col[c].y != 0)) {
          // first column of a 2 x 2 block [[d_c, e], [e, d_c+1]]: [x_c x_c+1] D^{-1}
          const C e = s_col[c], d1 = s_d[c], d2 = s_d[c + 1];
          const C det = csub(cmul(d1, d2), cmul(e, e));
          v = cdiv(csub(cmul(row[c], d2), cmul(row[c + 1], e)), det);
        } else if (c > 0 && (s_col[c - 1].x != 0 || s_col[c - 1].y != 0)) {
          const C e = s_col[c - 1], d1 = s_d[c - 1], d2 = s_d[c];
          const C det = csub(cmul(d1, d2), cmul(e, e));
          v = cdiv(csub(cmul(row[c], d1), cmul(row[c - 1], e)), det);
        } else {
          v = cdiv(row[c], s_d[c]);
        }
        Lt[i] = v;
      }
    } else {
      // ------------------------------------------------------------ 2b. off-diagonal tile
      const C* Ld = Lg + (int64_t)T.diag * TB * TB;
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int r = i >> 6, c = i & 63;
        sB[r * LDS + c] = ld_cg(Ld + i);
      }
      if (tid < TB) s_d[tid] = ld_cg(Dg + (int64_t)T.col * TB + tid);
      __syncthreads();
      // X L_JJ^T = S: column c of X is final once columns < c are eliminated
      for (int c = 0; c < TB - 1; ++c) {
        const int w = TB - 1 - c;
        for (int i = tid; i < TB * w; i += NTHR) {
          const int r = i / w, cc = c + 1 + i % w;
          sA[r * LDS + cc] = cfms(sA[r * LDS + c], sB[cc * LDS + c], sA[r * LDS + cc]);
        }
        __syncthreads();
      }
      C* Lt = Lg + (int64_t)T.tile * TB * TB;
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int r = i >> 6, c = i & 63;
        Lt[i] = cdiv(sA[r * LDS + c], s_d[c]);
      }
    }
    sched_complete(p, task);
  }
}

int launch_factor_simt(const FactorParams& p, bool fp64, int nblocks, cudaStream_t st) {
  const size_t smem = (fp64 ? sizeof(double2) : sizeof(float2)) * 2 * TB * LDS;
  cudaError_t e;
  if (fp64) {
    e = cudaFuncSetAttribute(factor_simt_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    factor_simt_kernel<double><<<nblocks, NTHR, smem, st>>>(p);
  } else {
    e = cudaFuncSetAttribute(factor_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    factor_simt_kernel<float><<<nblocks, NTHR, smem, st>>>(p);
  }
  return (int)cudaGetLastError();
}

}  // namespace d3m
