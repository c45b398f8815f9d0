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
      __syncthreads();
      for (int i = tid; i < TB * TB; i += NTHR) {
        const int r = i >> 6, c = i & 63;
        sA[r * LDS + c] = ld_cg(La + i);
        sB[r * LDS + c] = cmul(ld_cg(Lb + i), ld_cg(dK + c));   // W_JK = L_JK D_K
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

    if (T.flags & TF_DIAG) {
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
