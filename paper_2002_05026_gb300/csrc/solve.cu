// Forward / diagonal / backward block sweeps (the solve that follows the block factorization of
// the dual system, Sec. II), the FP64 residual r = b - K x over the stored K
// (block SpMV, symmetric use of the lower blocks), the backward-error norms and the adjoint
// contractions.
//
// Sweeps are level-scheduled over the block elimination tree (all blocks of one level are
// independent): per level a gather kernel computes the off-block products of every tile
// (forward: L_IJ y_J into tile row I; backward: L_IJ^T w_I into tile column J) as partials,
// then a block kernel reduces them in a fixed order and runs the in-block tile chain with the
// stored inverses of the diagonal tiles.  Vectors are permuted and padded to the tile grid:
// Y[j * npad + row].
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "kernels.h"

namespace d3m {

namespace {
constexpr int GT = 256;   // threads of gather / block kernels
constexpr int ET = 256;   // threads of elementwise kernels
constexpr size_t SWEEP_SMEM_LIMIT = 220 * 1024;
constexpr uint64_t SWEEP_TIMEOUT_NS = 2000000000ull;   // bound on one staging wait
constexpr int HR = 64;    // rows of one staged half-tile

template <typename R>
__device__ __forceinline__ typename CT<R>::C czero() { return CT<R>::make(0, 0); }
}  // namespace

// Converged instances of a batched handle (done[instance] = 1) are skipped by every kernel of a
// refinement step: their x stays as it is and their rows are not swept again.
struct Mask {
  const int* done;           // [instances], nullptr = nothing masked
  const int32_t* tinst;      // [NT] instance of every tile row (permuted numbering)
  __device__ __forceinline__ bool off(int64_t tile) const { return done && done[tinst[tile]] != 0; }
};

// Programmatic dependent launch between the kernels of a sweep: a kernel lets its successor be
// scheduled at once (trigger) and does work that reads only data fixed before the solve (tiles of
// L, inverses, task lists) before it waits for its predecessor; everything else follows the wait.
// Every thread of every block waits before it exits, so completion stays transitive along the
// stream.  Launched without the attribute, both instructions are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------------------------ permutation + padding
template <typename R>
__global__ void permute_in_kernel(const double2* __restrict__ src, int64_t n,
                                  typename CT<R>::C* __restrict__ Y, int64_t npad,
                                  const int64_t* __restrict__ pad2orig, int nrhs, Mask mk, int b) {
  pdl_trigger();
  pdl_wait();
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= npad || mk.off(g / b)) return;
  const int64_t o = pad2orig[g];
  for (int j = 0; j < nrhs; ++j)
    Y[j * npad + g] = (o >= 0) ? CT<R>::from(src[j * n + o]) : CT<R>::make(0, 0);
}

// X (=, or += when accumulate) W in caller numbering; dmax[instance * ld + j] = max |W| of the
// step (float bits; the size of the correction drives the forward-error stopping test).
template <typename R>
__global__ void permute_out_kernel(const typename CT<R>::C* __restrict__ W, int64_t npad,
                                   double2* __restrict__ X, int64_t n,
                                   const int64_t* __restrict__ pad2orig, int nrhs, int accumulate, Mask mk, int b,
                                   unsigned* dmax, int ld) {
  pdl_trigger();
  pdl_wait();
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g - (threadIdx.x & 31) >= npad) return;              // whole warps past the end
  // a warp's 32 rows lie in one tile (tiles are >= 64 rows and warps 32-aligned)
  const bool act = g < npad && !mk.off(g / b) && pad2orig[g] >= 0;   // a converged instance keeps its x
  const int64_t o = act ? pad2orig[g] : 0;
  const int inst = (g < npad && mk.tinst) ? mk.tinst[g / b] : 0;
  for (int j = 0; j < nrhs; ++j) {
    float a = 0.f;
    if (act) {
      const typename CT<R>::C w = W[j * npad + g];
      double2 v = make_double2((double)w.x, (double)w.y);
      a = sqrtf((float)(v.x * v.x + v.y * v.y));
      if (accumulate) {
        const double2 x = X[j * n + o];
        v.x += x.x;
        v.y += x.y;
      }
      X[j * n + o] = v;
    }
    for (int s = 16; s > 0; s >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, s));
    if (dmax && (threadIdx.x & 31) == 0 && a > 0.f) atomicMax(dmax + inst * ld + j, __float_as_uint(a));
  }
}

// ------------------------------------------------------------------ bulk-copy staging
// A staged half tile is 64 rows of b elements in shared memory with a row stride of b elements
// + 16 bytes (rows stay 16-byte aligned for the bulk copies; the pad spreads rows over banks).
// Each row is one TMA bulk copy (cp.async.bulk, b * sizeof(C) = 1 KB) completing on an mbarrier.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <typename C>
__host__ __device__ constexpr int stage_ld(int b) { return b + (int)(16 / sizeof(C)); }

__device__ __forceinline__ void mbar_init_s(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait_s(uint64_t* bar, uint32_t parity, uint64_t deadline) {
  uint32_t ok = 0;
  while (true) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (globaltimer_ns() > deadline) return false;
  }
}

// Warp 0 issues the 64 row copies of rows [r0, r0 + 64) of a b x b row-major tile.
template <typename C>
__device__ __forceinline__ void stage_bulk(C* sL, const C* tile, int b, int r0, uint64_t* bar) {
  if (threadIdx.x >= 32) return;
  const uint32_t row_bytes = (uint32_t)(b * sizeof(C));
  const int ldl = stage_ld<C>(b);
  if (threadIdx.x == 0)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(HR * row_bytes)
                 : "memory");
  __syncwarp();
  for (int r = threadIdx.x; r < HR; r += 32)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sL + r * ldl)),
        "l"(tile + (int64_t)(r0 + r) * b), "r"(row_bytes), "r"(smem_addr(bar))
        : "memory");
}

// ------------------------------------------------------------------ register-blocked tile products
// 8 warps; each warp computes 8 outputs for all (<= 8) right-hand sides with the reduction
// index split over 4 lanes (summed with shuffles).  One tile element load feeds rc complex
// FMAs; vector rows use an odd stride so the 4 rows read by a warp fall in distinct banks.
constexpr int RCMAX = 8;

__host__ __device__ constexpr int vec_ld(int rc) { return rc | 1; }

template <typename C>
__device__ __forceinline__ C shfl_xor_c(C v, int o) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, o);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, o);
  return v;
}

template <typename C>
__device__ __forceinline__ void quad_reduce(C* acc) {
#pragma unroll
  for (int j = 0; j < RCMAX; ++j)
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, o);
      acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, o);
    }
}

// dst[r][j] (=, +=, or -= by MODE 0 / 1 / 2) sum_c M[r][c] V[c][j] for the 64 rows of a staged
// half tile M ([64][ldl]); V element (c, j) at V[c * ldv + j]; dst element (r, j) at dst[r * ldd + j].
template <typename R, int MODE>
__device__ __forceinline__ void rows_matvec(const typename CT<R>::C* M, int ldl, int b, const typename CT<R>::C* V,
                                            int ldv, int rc, typename CT<R>::C* dst, int ldd) {
  using C = typename CT<R>::C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = warp * 8 + (lane >> 2), cq = lane & 3;
  C acc[RCMAX];
#pragma unroll
  for (int j = 0; j < RCMAX; ++j) acc[j] = CT<R>::make(0, 0);
  const C* mrow = M + r * ldl;
#pragma unroll 4
  for (int c = cq; c < b; c += 4) {
    const C m = mrow[c];
    const C* v = V + c * ldv;
    C vv[RCMAX];
#pragma unroll
    for (int j = 0; j < RCMAX; ++j) vv[j] = (j < rc) ? v[j] : CT<R>::make(0, 0);
#pragma unroll
    for (int j = 0; j < RCMAX; ++j) acc[j] = cfma(m, vv[j], acc[j]);
  }
  quad_reduce(acc);
  if (cq == 0) {
#pragma unroll
    for (int j = 0; j < RCMAX; ++j)
      if (j < rc)
        dst[r * ldd + j] = MODE == 0 ? acc[j] : (MODE == 1 ? cadd(dst[r * ldd + j], acc[j]) : csub(dst[r * ldd + j], acc[j]));
  }
}

// rows_matvec on a dense [64][b] strip (one bulk copy): the 4 column classes of each of a warp's 8
// rows start at columns rotated by 4 per row, so every warp-wide load touches 32 consecutive
// columns (no bank conflicts); b is a power of two.
template <typename R, int MODE>
__device__ __forceinline__ void rows_matvec_dense(const typename CT<R>::C* M, int b, const typename CT<R>::C* V,
                                                  int ldv, int rc, typename CT<R>::C* dst, int ldd) {
  // warp w, lane l: rows rg + 16 a (rg = 2 w + l / 16, a < 4), columns l % 16 + 16 k, all right-hand
  // sides; the 16 column groups of a row are summed by a shuffle reduce-scatter (lane l % 16 ends
  // with values q = 2 (l % 16), 2 (l % 16) + 1 of q = a * 8 + j)
  using C = typename CT<R>::C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rg = 2 * warp + (lane >> 4), cg = lane & 15;
  C acc[4][RCMAX];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int j = 0; j < RCMAX; ++j) acc[a][j] = CT<R>::make(0, 0);
#pragma unroll 2
  for (int c = cg; c < b; c += 16) {
    C v[RCMAX];
#pragma unroll
    for (int j = 0; j < RCMAX; ++j) v[j] = (j < rc) ? V[c * ldv + j] : CT<R>::make(0, 0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const C m = M[(rg + 16 * a) * b + c];
#pragma unroll
      for (int j = 0; j < RCMAX; ++j) acc[a][j] = cfma(m, v[j], acc[a][j]);
    }
  }
  C* f = &acc[0][0];
#pragma unroll
  for (int o = 8, n = 32; o >= 1; o >>= 1, n >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int q = 0; q < n / 2; ++q) {
      const C lo = f[q], hi = f[q + n / 2];
      const C send = up ? lo : hi;
      C keep = up ? hi : lo;
      keep = cadd(keep, shfl_xor_c(send, o));
      f[q] = keep;
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = 2 * cg + u, a = q >> 3, j = q & 7;
    if (j < rc) {
      C* d = dst + (rg + 16 * a) * ldd + j;
      *d = MODE == 0 ? f[u] : (MODE == 1 ? cadd(*d, f[u]) : csub(*d, f[u]));
    }
  }
}

// dst[c][j] (=, +=, or -= by MODE 0 / 1 / 2) sum_{r < 64} M[r][c] V[r][j] for all b columns
// of a staged half tile.
template <typename R, int MODE>
__device__ __forceinline__ void cols_matvec(const typename CT<R>::C* M, int ldl, int b, const typename CT<R>::C* V,
                                            int ldv, int rc, typename CT<R>::C* dst, int ldd) {
  using C = typename CT<R>::C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rq = lane & 3;
  for (int c0 = 0; c0 < b; c0 += 64) {
    const int c = c0 + warp * 8 + (lane >> 2);
    C acc[RCMAX];
#pragma unroll
    for (int j = 0; j < RCMAX; ++j) acc[j] = CT<R>::make(0, 0);
#pragma unroll 4
    for (int r = rq; r < HR; r += 4) {
      const C m = M[r * ldl + c];
      const C* v = V + r * ldv;
      C vv[RCMAX];
#pragma unroll
      for (int j = 0; j < RCMAX; ++j) vv[j] = (j < rc) ? v[j] : CT<R>::make(0, 0);
#pragma unroll
      for (int j = 0; j < RCMAX; ++j) acc[j] = cfma(m, vv[j], acc[j]);
    }
    quad_reduce(acc);
    if (rq == 0) {
#pragma unroll
      for (int j = 0; j < RCMAX; ++j)
        if (j < rc)
          dst[c * ldd + j] = MODE == 0 ? acc[j] : (MODE == 1 ? cadd(dst[c * ldd + j], acc[j]) : csub(dst[c * ldd + j], acc[j]));
    }
  }
}

// ------------------------------------------------------------------ gather (off-block tiles)
// grid = (groups of the level * (b / 64) halves, ceil(nrhs / 8) rhs groups).  A block sums the
// products of its group's items (consecutive off-block tiles of one destination) for one
// 64-row half h of the tiles and up to 8 right-hand sides:
//   FWD: P[slot][h*64 + r][j] = sum_items sum_k L[h*64 + r][k] Y[src*b + k][j];
//   BWD: P[slot*nh + h][c][j] = sum_items sum_{r < 64} L[h*64 + r][c] W[src*b + h*64 + r][j].
// An item's tile half is contiguous (64 rows of a row-major tile) and comes in as ONE bulk copy
// into a dense [64][b] buffer; its source rows as one bulk copy per right-hand side.  Reads of the
// dense half stay conflict-free: forward, the 8 rows x 4 column classes of a warp start at
// columns rotated by 4 per row, so a warp touches 32 consecutive columns; backward, a thread owns
// one output column and the warp reads 32 consecutive columns of one row.  Items of a group are
// double buffered (the next loads while the current one is multiplied).
template <typename C>
__device__ __forceinline__ void stage_item(C* sT, C* sV, int ldv, const C* half, const C* Y, int64_t npad,
                                           int64_t y0, int vlen, int j0, int rc, int b, uint64_t* bar) {
  if (threadIdx.x >= 32) return;
  const uint32_t t_bytes = (uint32_t)(HR * b * sizeof(C)), v_bytes = (uint32_t)(vlen * sizeof(C));
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(t_bytes + rc * v_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(sT)),
        "l"(half), "r"(t_bytes), "r"(smem_addr(bar))
        : "memory");
  }
  __syncwarp();
  for (int j = threadIdx.x; j < rc; j += 32)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sV + j * ldv)),
        "l"(Y + (int64_t)(j0 + j) * npad + y0), "r"(v_bytes), "r"(smem_addr(bar))
        : "memory");
}

// Persistent gather: CTA c takes units u = c, c + grid, ... of the level (unit = one group's products
// for one 64-row half of its tiles, units of finished instances skipped); the tile halves and source
// rows of the next nstg - 1 items are in flight while one is multiplied.  Warp 0 issues the copies;
// it fetches the next unit's group and item at the top of an iteration (the loads overlap the
// products) and leaves each staged item's output slot in a small shared ring for the consumers.
constexpr int GMAXSTG = 4;
constexpr int GGT = 512;   // threads of a gather block (16 warps)

struct GatherMeta {
  int slot, h, end, more;   // partial slot, half, last item of its unit, another item follows
};

// The two halves of stage_item: the tile half (thread 0 also arms the barrier for both parts) and
// the source rows (lanes < rc of the issuing warp).
template <typename C>
__device__ __forceinline__ void stage_tile_only(C* sT, const C* half, int vlen, int rc, int b, uint64_t* bar) {
  if (threadIdx.x != 0) return;
  const uint32_t t_bytes = (uint32_t)(HR * b * sizeof(C)), v_bytes = (uint32_t)(vlen * sizeof(C));
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(t_bytes + rc * v_bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(sT)),
      "l"(half), "r"(t_bytes), "r"(smem_addr(bar))
      : "memory");
}
template <typename C>
__device__ __forceinline__ void stage_rows_only(C* sV, int ldv, const C* Y, int64_t npad, int64_t y0, int vlen, int j0,
                                                int rc, uint64_t* bar) {
  const uint32_t v_bytes = (uint32_t)(vlen * sizeof(C));
  for (int j = threadIdx.x; j < rc; j += 32)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(sV + j * ldv)),
        "l"(Y + (int64_t)(j0 + j) * npad + y0), "r"(v_bytes), "r"(smem_addr(bar))
        : "memory");
}

template <typename R, bool FWD>
__global__ void __launch_bounds__(GGT, 1) gather_kernel(const SolveGroup* __restrict__ groups,
                                                        const SolveItem* __restrict__ items,
                                                        const typename CT<R>::C* __restrict__ L,
                                                        const typename CT<R>::C* __restrict__ Y,
                                                        typename CT<R>::C* __restrict__ P, int64_t npad, int b,
                                                        int nrhs, int* status, Mask mk, int nunits, int nstg) {
  using C = typename CT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nh = b / HR;
  const int vlen = FWD ? b : HR;                         // source rows per right-hand side
  const int ldv = vlen + (int)(16 / sizeof(C));
  const int stg = HR * b + RCMAX * ldv;                  // elements of one stage buffer
  C* const sbase = reinterpret_cast<C*>(smem_raw);
  __shared__ __align__(8) uint64_t bars[GMAXSTG];
  __shared__ GatherMeta s_meta[GMAXSTG];
  const int j0 = blockIdx.y * RCMAX;
  const int rc = min(RCMAX, nrhs - j0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto skip = [&](int u) {                               // first active unit >= u (whole warps)
    if (!mk.done) return u;
    while (u < nunits) {
      const int cand = u + lane * (int)gridDim.x;        // 32 candidates per step
      const bool act = cand < nunits && !mk.off(groups[cand / nh].dst);
      const unsigned bal = __ballot_sync(0xffffffffu, act);
      if (bal) return u + (__ffs(bal) - 1) * (int)gridDim.x;
      u += 32 * (int)gridDim.x;
    }
    return u;
  };
  pdl_trigger();
  int pu = skip(blockIdx.x), pk = 0;                     // next unit / item to issue (warp 0)
  if (pu >= nunits) {                                    // uniform: nothing to do for this block
    pdl_wait();
    return;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < nstg; ++i) mbar_init_s(&bars[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // source rows past rc stay zero in every stage (the products run over all RCMAX rows)
  for (int i = threadIdx.x; i < nstg * (RCMAX - rc) * ldv; i += GGT) {
    const int st = i / ((RCMAX - rc) * ldv), e = i % ((RCMAX - rc) * ldv);
    sbase[(int64_t)st * stg + HR * b + rc * ldv + e] = CT<R>::make(0, 0);
  }
  __syncthreads();
  SolveGroup pg{};
  SolveItem pit{};
  auto fetch = [&]() {                                   // warp 0: group and item of (pu, pk)
    if (pu < nunits) {
      pg = groups[pu / nh];
      pit = items[pg.first + pk];
    }
  };
  // warp 0: (pu, pk) into `slot`, then advance; with rows == false only the tile half is copied
  // (the source rows follow with stage_rows once the predecessor has finished)
  int64_t y0s[GMAXSTG];
  auto issue = [&](int slot, bool rows) {
    const int h = pu % nh;
    const int64_t y0 = (int64_t)pit.src * b + (FWD ? 0 : h * HR);
    C* T = sbase + (int64_t)slot * stg;
    if (rows) {
      stage_item(T, T + HR * b, ldv, L + (int64_t)pit.tile * b * b + (int64_t)h * HR * b, Y, npad, y0, vlen, j0, rc,
                 b, &bars[slot]);
    } else {
      stage_tile_only(T, L + (int64_t)pit.tile * b * b + (int64_t)h * HR * b, vlen, rc, b, &bars[slot]);
      y0s[slot] = y0;
    }
    const bool end = (pk + 1 == pg.count);
    if (end) {
      pk = 0;
      pu = skip(pu + gridDim.x);
    } else {
      ++pk;
    }
    if (lane == 0) s_meta[slot] = GatherMeta{pg.slot, h, end ? 1 : 0, pu < nunits ? 1 : 0};
  };
  int inflight = 0;                                      // items issued, not yet consumed (warp 0)
  if (warp == 0) {
    for (int i = 0; i < nstg && pu < nunits; ++i, ++inflight) {
      fetch();
      issue(i, false);                                   // tiles of L are fixed during the solve
    }
  }
  pdl_wait();                                            // the source rows come from the predecessor
  if (warp == 0)
    for (int i = 0; i < inflight; ++i) {
      C* T = sbase + (int64_t)i * stg;
      stage_rows_only(T + HR * b, ldv, Y, npad, y0s[i], vlen, j0, rc, &bars[i]);
    }
  __syncthreads();                                       // s_meta of the first stages
  // forward: warp w, lane l -> rows rg + 32 i (rg = 2 w + l / 16, i < 2), columns l % 16 + 16 k, all
  //   right-hand sides; the 16 column groups of a row are summed by a shuffle reduce-scatter
  // backward: warp w -> rows 8 (w % 8) .. + 7 of the half and column half w / 8, lane l -> columns
  //   l + 32 k of that half; the 8 row groups are summed through shared memory in a fixed order
  constexpr int NA = 2;                                  // rows (forward) / column slots (backward) per thread
  C acc[NA][RCMAX];
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int j = 0; j < RCMAX; ++j) acc[a][j] = CT<R>::make(0, 0);
  const uint64_t deadline = globaltimer_ns() + SWEEP_TIMEOUT_NS;
  for (int it = 0;; ++it) {
    const int slot = it % nstg;
    const bool late = !mbar_wait_s(&bars[slot], (uint32_t)((it / nstg) & 1), deadline);
    if (__syncthreads_or(late)) {
      if (threadIdx.x == 0) {
        atomicExch(status, (int)D3M_ERR_TIMEOUT);
        // let the copies still in flight land before the block's shared memory is released
        for (int i = it; i < it + inflight; ++i)
          mbar_wait_s(&bars[i % nstg], (uint32_t)((i / nstg) & 1), globaltimer_ns() + SWEEP_TIMEOUT_NS);
      }
      __syncthreads();
      return;
    }
    const GatherMeta mt = s_meta[slot];
    --inflight;
    if (warp == 0) fetch();                              // loads overlap the products below
    const C* M = sbase + (int64_t)slot * stg;
    const C* V = M + HR * b;
    if (FWD) {
      const int rg = 2 * warp + (lane >> 4), cg = lane & 15;
#pragma unroll 2
      for (int c = cg; c < b; c += 16) {
        C v[RCMAX];
#pragma unroll
        for (int j = 0; j < RCMAX; ++j) v[j] = V[j * ldv + c];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
          const C m = M[(rg + 32 * a) * b + c];
#pragma unroll
          for (int j = 0; j < RCMAX; ++j) acc[a][j] = cfma(m, v[j], acc[a][j]);
        }
      }
    } else {
      const int rg8 = warp & 7, chalf = (warp >> 3) * (b / 2);
#pragma unroll 2
      for (int r = 8 * rg8; r < 8 * rg8 + 8; ++r) {
        C v[RCMAX];
#pragma unroll
        for (int j = 0; j < RCMAX; ++j) v[j] = V[j * ldv + r];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
          if (lane + 32 * a < b / 2) {
            const C m = M[r * b + chalf + lane + 32 * a];
#pragma unroll
            for (int j = 0; j < RCMAX; ++j) acc[a][j] = cfma(m, v[j], acc[a][j]);
          }
        }
      }
    }
    __syncthreads();                                     // the slot is consumed
    if (FWD) {
      if (warp == 0 && pu < nunits) {
        if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        issue(slot, true);
        ++inflight;
      }
      if (mt.end) {
        // reduce-scatter over the 16 lanes of a row group: value q = a * 8 + j; after the stage
        // with offset o a lane keeps the half selected by its bit o, so lane cg ends with q = cg
        C* f = &acc[0][0];
#pragma unroll
        for (int o = 8, n = 16; o >= 1; o >>= 1, n >>= 1) {
          const bool up = (lane & o) != 0;
#pragma unroll
          for (int q = 0; q < n / 2; ++q) {
            const C lo = f[q], hi = f[q + n / 2];
            const C send = up ? lo : hi;
            C keep = up ? hi : lo;
            keep = cadd(keep, shfl_xor_c(send, o));
            f[q] = keep;
          }
        }
        const int rg = 2 * warp + (lane >> 4), cg = lane & 15;
        const int a = cg >> 3, j = cg & 7;
        if (j < rc)
          P[(int64_t)mt.slot * nh * b * nrhs + (int64_t)(mt.h * HR + rg + 32 * a) * nrhs + j0 + j] = f[0];
#pragma unroll
        for (int a2 = 0; a2 < NA; ++a2)
#pragma unroll
          for (int j2 = 0; j2 < RCMAX; ++j2) acc[a2][j2] = CT<R>::make(0, 0);
      }
    } else {
      if (mt.end) {
        // sum the 8 row groups of every (column, rhs) in a fixed order, in the consumed slot
        C* red = sbase + (int64_t)slot * stg;            // [8][b][RCMAX], within the tile part
        const int rg8 = warp & 7, chalf = (warp >> 3) * (b / 2);
#pragma unroll
        for (int a = 0; a < NA; ++a) {
          const int c = chalf + lane + 32 * a;
          if (lane + 32 * a < b / 2)
#pragma unroll
            for (int j = 0; j < RCMAX; ++j) red[(rg8 * b + c) * RCMAX + j] = acc[a][j];
        }
        __syncthreads();
        C* out = P + ((int64_t)mt.slot * nh + mt.h) * b * nrhs + j0;
        for (int o = threadIdx.x; o < b * RCMAX; o += GGT) {
          const int c = o / RCMAX, j = o % RCMAX;
          C v = red[c * RCMAX + j];
#pragma unroll
          for (int w = 1; w < 8; ++w) v = cadd(v, red[(w * b + c) * RCMAX + j]);
          if (j < rc) out[(int64_t)c * nrhs + j] = v;
        }
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
          for (int j = 0; j < RCMAX; ++j) acc[a][j] = CT<R>::make(0, 0);
        __syncthreads();                                 // the slot is free again
      }
      if (warp == 0 && pu < nunits) {
        if (lane == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        issue(slot, true);
        ++inflight;
      }
    }
    if (!mt.more) break;
  }
}

// ------------------------------------------------------------------ in-block chains
struct BlockSweep {
  int* status;               // set to D3M_ERR_TIMEOUT if a bounded wait expires
  const int32_t* blocks;     // blocks of this level
  const int32_t* tstart;     // [N+1]
  const int64_t* tcolptr;    // [NT+1]
  const int64_t* slot_ptr;   // [NT] first | count << 32
  int64_t npad;
  int b, nrhs, rc;           // rhs handled per block (grid.y = ceil(nrhs / rc))
};

constexpr int MAXJOBS = 512;      // tile jobs of one block chain (nt (nt+1)/2 * b/64)
constexpr int MAXNT = 32;         // tiles per interface block

// Y(row) -= sum of the row's partials (fixed slot order) for every tile row of one level, after
// Y(row) /= D(row) when D is given (backward sweep: z = D^{-1} y first); one thread per (tile, row,
// rhs), rhs fastest (coalesced partial reads), 16 partial loads in flight per thread.
template <typename R>
__global__ void __launch_bounds__(ET) reduce_kernel(const int32_t* __restrict__ tiles, int ntl,
                                                    const int64_t* __restrict__ slot_ptr,
                                                    const typename CT<R>::C* __restrict__ P,
                                                    typename CT<R>::C* __restrict__ Y, int64_t npad, int b,
                                                    int nrhs, int nsub, const typename CT<R>::C* __restrict__ D,
                                                    Mask mk) {
  // a block takes 32 consecutive outputs (tile, row, rhs); warp w sums the partials w, w + 8, ...
  // of each (lanes = outputs, so the loads of a partial are contiguous), and the 8 sub-sums are
  // added in warp order: the summation order depends only on the partial count
  using C = typename CT<R>::C;
  constexpr int NW = ET / 32;
  __shared__ C s_sub[NW][32];
  pdl_trigger();
  pdl_wait();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t idx = blockIdx.x * (int64_t)32 + lane;
  const int j = (int)(idx % nrhs);
  const int64_t rest = idx / nrhs;
  const int row = (int)(rest % b);
  const int64_t tl = rest / b;
  bool live = tl < ntl;
  int I = 0;
  int64_t first = 0, cnt = 0;
  if (live) {
    I = tiles[tl];
    live = !mk.off(I);
  }
  if (live) {
    const int64_t sp = slot_ptr[I];
    first = sp & 0xffffffffLL;
    cnt = (sp >> 32) * nsub;
  }
  const int nh = b / HR;
  C acc = czero<R>();
  if (live && cnt > warp) {
    const C* pp = P + first * nh * (int64_t)b * nrhs + (int64_t)row * nrhs + j;
    const int64_t stride = (int64_t)b * nrhs * (nsub == 1 ? nh : 1);
    for (int64_t q0 = warp; q0 < cnt; q0 += 8 * NW) {
      C t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = (q0 + u * NW < cnt) ? pp[(q0 + u * NW) * stride] : czero<R>();
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = cadd(acc, t[u]);
    }
  }
  s_sub[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && live && (cnt > 0 || D)) {
    C* y = Y + (int64_t)j * npad + (int64_t)I * b + row;
    C v = *y;
    if (D) v = cdiv(v, D[(int64_t)I * b + row]);
    if (cnt) {
      C sum = s_sub[0][lane];
#pragma unroll
      for (int w = 1; w < NW; ++w) sum = cadd(sum, s_sub[w][lane]);
      v = csub(v, sum);
    }
    *y = v;
  }
}

// z = D^{-1} y over the whole padded vector (between the forward and backward sweeps)
template <typename R>
__global__ void diag_scale_kernel(typename CT<R>::C* __restrict__ Y, const typename CT<R>::C* __restrict__ D,
                                  int64_t npad, int nrhs) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= npad) return;
  const typename CT<R>::C d = D[g];
  for (int j = 0; j < nrhs; ++j) Y[(int64_t)j * npad + g] = cdiv(Y[(int64_t)j * npad + g], d);
}

// z = D^{-1} y with the 1 x 1 and 2 x 2 blocks of a pivoted factorization (E[g] != 0: rows g and
// g + 1 of one tile form the block [[D[g], E[g]], [E[g], D[g+1]]]; the first row's thread
// solves both)
template <typename R>
__global__ void diag_scale_bk_kernel(typename CT<R>::C* __restrict__ Y, const typename CT<R>::C* __restrict__ D,
                                     const typename CT<R>::C* __restrict__ E, int64_t npad, int nrhs, int b) {
  using C = typename CT<R>::C;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= npad) return;
  const int c = (int)(g % b);
  if (c > 0 && (E[g - 1].x != 0 || E[g - 1].y != 0)) return;   // second row of a 2 x 2 block
  if (c + 1 < b && (E[g].x != 0 || E[g].y != 0)) {
    const C d1 = D[g], d2 = D[g + 1], e = E[g];
    const C det = csub(cmul(d1, d2), cmul(e, e));
    for (int j = 0; j < nrhs; ++j) {
      const C y1 = Y[(int64_t)j * npad + g], y2 = Y[(int64_t)j * npad + g + 1];
      Y[(int64_t)j * npad + g] = cdiv(csub(cmul(d2, y1), cmul(e, y2)), det);
      Y[(int64_t)j * npad + g + 1] = cdiv(csub(cmul(d1, y2), cmul(e, y1)), det);
    }
    return;
  }
  const C d = D[g];
  for (int j = 0; j < nrhs; ++j) Y[(int64_t)j * npad + g] = cdiv(Y[(int64_t)j * npad + g], d);
}

// load one block's rows of Y into sv[row][rc]
template <typename C>
__device__ __forceinline__ void load_rows(const C* __restrict__ Y, int64_t npad, int64_t r0, int rows, int j0,
                                          int rc, int ldv, C* sv) {
  for (int i = threadIdx.x; i < rows * rc; i += GT) {
    const int row = i % rows, j = i / rows;
    sv[row * ldv + j] = Y[(int64_t)(j0 + j) * npad + r0 + row];
  }
}

// forward (partials already subtracted from Y):  y_t = Linv_tt r_t;  r_t' -= L_t't y_t  (Y keeps y: later
// levels gather L_IJ y_J; the diagonal step z = D^{-1} y is applied by the backward kernel).
// Tiles are staged with cp.async into two buffers: the next job's tile loads while the
// current one is used.
template <typename R>
__global__ void __launch_bounds__(GT) block_fwd_kernel(BlockSweep s, const typename CT<R>::C* __restrict__ L,
                                                       const typename CT<R>::C* __restrict__ Linv,
                                                       typename CT<R>::C* __restrict__ Y) {
  using C = typename CT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ const C* s_job[MAXJOBS];
  const int b = s.b, ldl = stage_ld<C>(b), nh = b / HR;
  __shared__ __align__(8) uint64_t bars[2];
  const int k = s.blocks[blockIdx.x];
  const int j0 = blockIdx.y * s.rc;
  const int rc = min(s.rc, s.nrhs - j0);
  const int ldv = vec_ld(s.rc);                // row stride of the running vectors
  const int t0 = s.tstart[k], nt = s.tstart[k + 1] - t0;
  const int rows = nt * b;
  C* sL0 = reinterpret_cast<C*>(smem_raw);     // [64][b+1] x 2
  C* sL1 = sL0 + HR * ldl;
  C* sv = sL1 + HR * ldl;                      // [rows][rc]  running r / y
  C* sy = sv + (int64_t)rows * ldv;           // [b][rc]     y_t
  // job list: for t: Linv_t halves, then L_{t', t} halves for t' > t
  // job table: for t, the halves of Linv_t, then of L_{t', t} for t' > t (tile ids of column
  // t0 + t inside the block are consecutive after its diagonal tile)
  __shared__ int64_t s_cp[MAXNT];
  if (threadIdx.x < nt) s_cp[threadIdx.x] = s.tcolptr[t0 + threadIdx.x];
  __syncthreads();
  int njobs = 0;
  for (int t = 0; t < nt; ++t) njobs += nh * (nt - t);
  for (int j = threadIdx.x; j < njobs; j += GT) {
    int t = 0, base = 0;
    while (base + nh * (nt - t) <= j) base += nh * (nt - t++);
    const int q = j - base, h = q % nh, tp = t + q / nh;   // tp == t: Linv_t
    s_job[j] = (tp == t) ? Linv + (int64_t)(t0 + t) * b * b + (int64_t)h * HR * b
                         : L + (s_cp[t] + (tp - t)) * (int64_t)b * b + (int64_t)h * HR * b;
  }
  if (threadIdx.x == 0) {
    mbar_init_s(&bars[0]);
    mbar_init_s(&bars[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  stage_bulk(sL0, s_job[0], b, 0, &bars[0]);
  uint32_t phase[2] = {0u, 0u};
  const uint64_t deadline = globaltimer_ns() + SWEEP_TIMEOUT_NS;
  load_rows(Y, s.npad, (int64_t)t0 * b, rows, j0, rc, ldv, sv);
  int job = 0;
  for (int t = 0; t < nt; ++t) {
    for (int q = 0; q < nh * (nt - t); ++q, ++job) {
      const int buf = job & 1;
      C* cur = buf ? sL1 : sL0;
      if (job + 1 < njobs) {
        // the other buffer was last read in the previous job (which ended with a barrier)
        if (threadIdx.x < 32) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        stage_bulk(buf ? sL0 : sL1, s_job[job + 1], b, 0, &bars[buf ^ 1]);
      }
      const bool late = !mbar_wait_s(&bars[buf], phase[buf], deadline);
      phase[buf] ^= 1u;
      if (__syncthreads_or(late)) {
        if (threadIdx.x == 0) atomicExch(s.status, (int)D3M_ERR_TIMEOUT);
        return;
      }
      const int h = q % nh;
      if (q < nh) {
        // y_t rows [h*64, h*64+64) = Linv_t[rows] r_t
        rows_matvec<R, 0>(cur, ldl, b, sv + (int64_t)t * b * ldv, ldv, rc, sy + h * HR * ldv, ldv);
        if (q == nh - 1) {
          __syncthreads();
          for (int i = threadIdx.x; i < b * rc; i += GT) {
            const int r = i % b, j = i / b;
            sv[(t * b + r) * ldv + j] = sy[r * ldv + j];
          }
        }
      } else {
        const int tp = t + 1 + (q - nh) / nh;
        rows_matvec<R, 2>(cur, ldl, b, sy, ldv, rc, sv + (int64_t)(tp * b + h * HR) * ldv, ldv);
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < rows * rc; i += GT) {
    const int row = i % rows, j = i / rows;
    Y[(int64_t)(j0 + j) * s.npad + (int64_t)t0 * b + row] = sv[row * ldv + j];
  }
}

// backward (Y holds D^{-1} y minus partials):  for t = nt-1..0: w_t = Linv_tt^T r_t;
// r_t' -= L_{t,t'}^T w_t (t' < t).  Same double-buffered staging as the forward kernel.
template <typename R>
__global__ void __launch_bounds__(GT) block_bwd_kernel(BlockSweep s, const typename CT<R>::C* __restrict__ L,
                                                       const typename CT<R>::C* __restrict__ Linv,
                                                       typename CT<R>::C* __restrict__ Y) {
  using C = typename CT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ const C* s_job[MAXJOBS];
  const int b = s.b, ldl = stage_ld<C>(b), nh = b / HR;
  __shared__ __align__(8) uint64_t bars[2];
  const int k = s.blocks[blockIdx.x];
  const int j0 = blockIdx.y * s.rc;
  const int rc = min(s.rc, s.nrhs - j0);
  const int ldv = vec_ld(s.rc);                // row stride of the running vectors
  const int t0 = s.tstart[k], nt = s.tstart[k + 1] - t0;
  const int rows = nt * b;
  C* sL0 = reinterpret_cast<C*>(smem_raw);
  C* sL1 = sL0 + HR * ldl;
  C* sv = sL1 + HR * ldl;
  C* sy = sv + (int64_t)rows * ldv;
  // job table: for t = nt-1..0, the halves of Linv_t, then of L_{t, t'} for t' < t
  __shared__ int64_t s_cp[MAXNT];
  if (threadIdx.x < nt) s_cp[threadIdx.x] = s.tcolptr[t0 + threadIdx.x];
  __syncthreads();
  int njobs = 0;
  for (int t = 0; t < nt; ++t) njobs += nh * (t + 1);
  for (int j = threadIdx.x; j < njobs; j += GT) {
    int t = nt - 1, base = 0;
    while (base + nh * (t + 1) <= j) base += nh * (t-- + 1);
    const int q = j - base, h = q % nh, k = q / nh;        // k == 0: Linv_t; else tile (t, k - 1)
    s_job[j] = (k == 0) ? Linv + (int64_t)(t0 + t) * b * b + (int64_t)h * HR * b
                        : L + (s_cp[k - 1] + (t - (k - 1))) * (int64_t)b * b + (int64_t)h * HR * b;
  }
  if (threadIdx.x == 0) {
    mbar_init_s(&bars[0]);
    mbar_init_s(&bars[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  stage_bulk(sL0, s_job[0], b, 0, &bars[0]);
  uint32_t phase[2] = {0u, 0u};
  const uint64_t deadline = globaltimer_ns() + SWEEP_TIMEOUT_NS;
  load_rows(Y, s.npad, (int64_t)t0 * b, rows, j0, rc, ldv, sv);
  int job = 0;
  for (int t = nt - 1; t >= 0; --t) {
    for (int i = threadIdx.x; i < b * ldv; i += GT) sy[i] = czero<R>();
    for (int q = 0; q < nh * (t + 1); ++q, ++job) {
      const int buf = job & 1;
      C* cur = buf ? sL1 : sL0;
      if (job + 1 < njobs) {
        // the other buffer was last read in the previous job (which ended with a barrier)
        if (threadIdx.x < 32) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        stage_bulk(buf ? sL0 : sL1, s_job[job + 1], b, 0, &bars[buf ^ 1]);
      }
      const bool late = !mbar_wait_s(&bars[buf], phase[buf], deadline);
      phase[buf] ^= 1u;
      if (__syncthreads_or(late)) {
        if (threadIdx.x == 0) atomicExch(s.status, (int)D3M_ERR_TIMEOUT);
        return;
      }
      const int h = q % nh;
      if (q < nh) {
        // w_t += Linv_t[rows of half h]^T r_t[rows of half h]
        cols_matvec<R, 1>(cur, ldl, b, sv + (int64_t)(t * b + h * HR) * ldv, ldv, rc, sy, ldv);
        if (q == nh - 1) {
          __syncthreads();
          for (int i = threadIdx.x; i < b * rc; i += GT) {
            const int r = i % b, j = i / b;
            sv[(t * b + r) * ldv + j] = sy[r * ldv + j];
          }
        }
      } else {
        // tile (t0+t, t0+tp): r_tp[c] -= sum_{r in half h} L[r][c] w_t[r]
        const int tp = (q - nh) / nh;
        cols_matvec<R, 2>(cur, ldl, b, sy + h * HR * ldv, ldv, rc, sv + (int64_t)tp * b * ldv, ldv);
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < rows * rc; i += GT) {
    const int row = i % rows, j = i / rows;
    Y[(int64_t)(j0 + j) * s.npad + (int64_t)t0 * b + row] = sv[row * ldv + j];
  }
}

// ------------------------------------------------------------------ cluster-cooperative block chains
// One thread-block cluster per (block, rhs group).  The block's rows are split into strips of 64
// rows (tile t, half h); strip s = t * nh + h is owned by CTA rank s % cl (local slot s / cl),
// which keeps its running vector in shared memory and streams only its own 64-row strips of L
// (forward: rows of the tiles (t', t); backward: 64-column strips of the tiles (t, t')).
// Step t of the chain: the owners of tile t read the full r_t from their partners' shared memory
// (DSMEM) and form their half of y_t = Linv_tt r_t (backward: w_t = Linv_tt^T r_t); after a
// cluster barrier every owner of a later tile reads the full y_t and updates its strip; a second
// barrier closes the step.  The gathered partials of the level are subtracted when the strips
// are loaded (and, backward, z = D^{-1} y is applied there), so a level needs no separate
// reduce or diagonal-scaling launch.
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// all threads of all CTAs of the cluster; release / acquire orders shared-memory writes
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// generic address of the same shared-memory location in CTA `rank` of the cluster
template <typename T>
__device__ __forceinline__ const T* cluster_map(const T* p, uint32_t rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(p), "r"(rank));
  return reinterpret_cast<const T*>(out);
}

// nrows row copies of rowlen elements (source row stride lds, shared row stride ldd) on one
// mbarrier; issued by warp 0.
template <typename C>
__device__ __forceinline__ void stage_rows(C* dst, int ldd, const C* src, int lds, int nrows, int rowlen,
                                           uint64_t* bar) {
  if (threadIdx.x >= 32) return;
  const uint32_t row_bytes = (uint32_t)(rowlen * sizeof(C));
  if (threadIdx.x == 0)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(nrows * row_bytes)
                 : "memory");
  __syncwarp();
  for (int r = threadIdx.x; r < nrows; r += 32)
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst + r * ldd)),
        "l"(src + (int64_t)r * lds), "r"(row_bytes), "r"(smem_addr(bar))
        : "memory");
}

// dst[c][j] (=, +=, or -= by MODE 0 / 1 / 2) sum_{r < nrows} M[r][c] V[r][j] for the 64 columns of
// a staged column strip
template <typename R, int MODE>
__device__ __forceinline__ void colstrip_matvec(const typename CT<R>::C* M, int ldm, int nrows,
                                                const typename CT<R>::C* V, int ldv, int rc,
                                                typename CT<R>::C* dst, int ldd) {
  using C = typename CT<R>::C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = warp * 8 + (lane >> 2), rq = lane & 3;
  C acc[RCMAX];
#pragma unroll
  for (int j = 0; j < RCMAX; ++j) acc[j] = CT<R>::make(0, 0);
#pragma unroll 4
  for (int r = rq; r < nrows; r += 4) {
    const C m = M[r * ldm + c];
    const C* v = V + r * ldv;
    C vv[RCMAX];
#pragma unroll
    for (int j = 0; j < RCMAX; ++j) vv[j] = (j < rc) ? v[j] : CT<R>::make(0, 0);
#pragma unroll
    for (int j = 0; j < RCMAX; ++j) acc[j] = cfma(m, vv[j], acc[j]);
  }
  quad_reduce(acc);
  if (rq == 0) {
#pragma unroll
    for (int j = 0; j < RCMAX; ++j)
      if (j < rc)
        dst[c * ldd + j] = MODE == 0 ? acc[j] : (MODE == 1 ? cadd(dst[c * ldd + j], acc[j]) : csub(dst[c * ldd + j], acc[j]));
  }
}

struct ChainSweep {
  int* status;               // set to D3M_ERR_TIMEOUT if a bounded wait expires
  const int32_t* blocks;     // blocks of this level
  const int32_t* tstart;     // [N+1]
  const int64_t* tcolptr;    // [NT+1]
  const int64_t* slot_ptr;   // [NT] first | count << 32 (partials of this direction)
  const void* P;             // partials of the level
  const void* D;             // pivots (backward)
  int64_t npad;
  int b, nrhs, rc;           // rhs per cluster (grid.y = ceil(nrhs / rc))
  int cl, nloc, stg;         // CTAs per cluster, strip slots per CTA, elements of one stage buffer
  int has_partials;
  int apply_d;               // backward: divide the loaded strips by D (else a reduce launch did)
  Mask mk;
  const void* Inv;           // off-diagonal tiles of the inverses of the diagonal blocks (INV mode)
  const int64_t* inv_off;    // [N] first tile of block k in Inv
  const void* InvT;          // transposed tiles Inv(c, a)^T, c >= a (diagonal included), INV mode
  const int64_t* invT_off;   // [N] first tile of block k in InvT
  int rrows;                 // rows of the largest block (INV mode: the whole r is gathered)
};

constexpr int CHAIN_MAXJ = 128;   // staged strips of one CTA
constexpr int CHAIN_MAXCL = 8;    // portable cluster size
constexpr int CHAIN_MAXLOC = 4;   // strips per CTA
constexpr int EXT_REDUCE = 12;    // partials per row above which a level gets a separate reduce launch

// INV mode: the diagonal block is applied as one product with its stored inverse,
//   y_J = L_JJ^{-1} r_J (forward),  w_J = L_JJ^{-T} r_J (backward),
// so every CTA only needs the whole r_J (one exchange through distributed shared memory) and
// its own strips of the inverse: no sequential steps and no barriers between them.
template <typename R, bool FWD, bool INV>
__global__ void __launch_bounds__(GT) chain_kernel(ChainSweep s, const typename CT<R>::C* __restrict__ L,
                                                   const typename CT<R>::C* __restrict__ Linv,
                                                   typename CT<R>::C* __restrict__ Y) {
  using C = typename CT<R>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ const C* s_job[CHAIN_MAXJ];
  __shared__ int64_t s_cp[MAXNT];
  __shared__ int s_nj;
  __shared__ __align__(8) uint64_t bars[2];
  const int b = s.b, nh = b / HR, CL = s.cl;
  const int rank = (int)cluster_ctarank();
  const int k = s.blocks[blockIdx.x / CL];
  const int j0 = blockIdx.y * s.rc;
  const int rc = min(s.rc, s.nrhs - j0);
  const int ldv = vec_ld(s.rc);
  const int t0 = s.tstart[k], nt = s.tstart[k + 1] - t0;
  pdl_trigger();
  if (s.mk.off(t0)) {                                 // every CTA of the cluster, before any barrier
    pdl_wait();
    return;
  }
  const int S = nt * nh;
  const int nloc = S > rank ? (S - rank + CL - 1) / CL : 0;
  const int ldst = FWD ? stage_ld<C>(b) : stage_ld<C>(HR);
  C* stg0 = reinterpret_cast<C*>(smem_raw);
  C* stg1 = stg0 + s.stg;
  C* sy = stg1 + s.stg;                              // [b][ldv]   gathered r_t or y_t
  C* rbuf = sy + (int64_t)b * ldv;                   // [nloc][64][ldv]  running strips
  C* obuf = rbuf + (int64_t)s.nloc * HR * ldv;       // [nloc][64][ldv]  solved strips
  C* sR = obuf + (int64_t)s.nloc * HR * ldv;         // INV: [rrows][ldv] the whole r_J
  const C* Inv = reinterpret_cast<const C*>(s.Inv);
  if (threadIdx.x < nt) s_cp[threadIdx.x] = s.tcolptr[t0 + threadIdx.x];
  __syncthreads();
  // staged strips in consumption order: per step, the strip of tile t first, then the updates
  // (INV: per local strip, its tiles of the inverse)
  if (threadIdx.x == 0 && INV) {
    int nj = 0;
    const int64_t ib = s.inv_off[k];
    const C* InvT = reinterpret_cast<const C*>(s.InvT);
    const int64_t ibt = s.invT_off[k];
    for (int l = 0; l < nloc; ++l) {
      const int sid = rank + l * CL, tq = sid / nh, h = sid % nh;
      const int64_t hoff = (int64_t)h * HR * b;       // row strip h (contiguous)
      for (int t = FWD ? 0 : tq; t < (FWD ? tq + 1 : nt); ++t) {
        // forward: tile (tq, t) of the inverse; backward: tile (tq, t) of the transposed inverse
        if (FWD) s_job[nj++] = (tq == t ? Linv + (int64_t)(t0 + tq) * b * b : Inv + (ib + tq * (tq - 1) / 2 + t) * (int64_t)b * b) + hoff;
        else s_job[nj++] = InvT + (ibt + t * (t + 1) / 2 + tq) * (int64_t)b * b + hoff;
      }
    }
    s_nj = nj;
    mbar_init_s(&bars[0]);
    mbar_init_s(&bars[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x == 0 && !INV) {
    int nj = 0;
    for (int q = 0; q < nt; ++q) {
      const int t = FWD ? q : nt - 1 - q;
      for (int pass = 0; pass < 2; ++pass)
        for (int l = 0; l < nloc; ++l) {
          const int sid = rank + l * CL, tp = sid / nh, h = sid % nh;
          const bool mine = pass == 0 ? tp == t : (FWD ? tp > t : tp < t);
          if (!mine) continue;
          const C* src;
          if (pass == 0) src = Linv + (int64_t)(t0 + t) * b * b + (FWD ? (int64_t)h * HR * b : (int64_t)h * HR);
          else if (FWD) src = L + (s_cp[t] + (tp - t)) * (int64_t)b * b + (int64_t)h * HR * b;
          else src = L + (s_cp[tp] + (t - tp)) * (int64_t)b * b + (int64_t)h * HR;
          s_job[nj++] = src;
        }
    }
    s_nj = nj;
    mbar_init_s(&bars[0]);
    mbar_init_s(&bars[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int nj = s_nj;
  auto stage = [&](int jb) {
    C* dst = (jb & 1) ? stg1 : stg0;
    if (INV) stage_rows(dst, HR * b, s_job[jb], HR * b, 1, HR * b, &bars[jb & 1]);   // one dense strip
    else if (FWD) stage_rows(dst, ldst, s_job[jb], b, HR, b, &bars[jb & 1]);
    else stage_rows(dst, ldst, s_job[jb], b, b, HR, &bars[jb & 1]);
  };
  if (nj > 0) stage(0);                                // tiles of L / the inverses: fixed during the solve
  pdl_wait();                                         // Y and the partials come from the predecessors
  // strips of r: Y rows (backward: D^{-1} y) minus the level's partials in fixed slot order
  {
    const C* P = reinterpret_cast<const C*>(s.P);
    const C* D = reinterpret_cast<const C*>(s.D);
    for (int l = 0; l < nloc; ++l) {
      const int sid = rank + l * CL, tp = sid / nh, h = sid % nh;
      const int I = t0 + tp;
      int64_t first = 0, cnt = 0;
      if (s.has_partials) {
        const int64_t sp = s.slot_ptr[I];
        first = sp & 0xffffffffLL;
        cnt = (sp >> 32) * (FWD ? 1 : nh);
      }
      const int64_t stride = (int64_t)b * s.nrhs * (FWD ? nh : 1);
      for (int i = threadIdx.x; i < HR * rc; i += GT) {
        const int j = i % rc, row = i / rc;
        const int64_t g = (int64_t)I * b + h * HR + row;
        C v = Y[(int64_t)(j0 + j) * s.npad + g];
        if (!FWD && s.apply_d) v = cdiv(v, D[g]);
        if (cnt) {
          // 16 independent loads in flight per thread; partial q goes to sub-sum q % 8 and the
          // sub-sums are added in order (the same order as reduce_kernel)
          const C* pp = P + first * nh * (int64_t)b * s.nrhs + (int64_t)(h * HR + row) * s.nrhs + (j0 + j);
          C sub[8];
#pragma unroll
          for (int w = 0; w < 8; ++w) sub[w] = czero<R>();
          for (int64_t q0 = 0; q0 < cnt; q0 += 16) {
            C t[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) t[u] = (q0 + u < cnt) ? pp[(q0 + u) * stride] : czero<R>();
#pragma unroll
            for (int u = 0; u < 16; ++u) sub[u & 7] = cadd(sub[u & 7], t[u]);
          }
          C acc = sub[0];
#pragma unroll
          for (int w = 1; w < 8; ++w) acc = cadd(acc, sub[w]);
          v = csub(v, acc);
        }
        rbuf[(l * HR + row) * ldv + j] = v;
      }
    }
  }
  uint32_t phase[2] = {0u, 0u};
  const uint64_t deadline = globaltimer_ns() + SWEEP_TIMEOUT_NS;
  bool bad = false;
  int job = 0;
  // wait for staged strip `job`, start the copy of the next one into the other buffer (its
  // previous reader finished before the barrier that ended that job)
  auto next_stage = [&]() -> const C* {
    const int buf = job & 1;
    if (!bad && job + 1 < nj) {
      if (threadIdx.x < 32) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      stage(job + 1);
    }
    const bool late = !bad && !mbar_wait_s(&bars[buf], phase[buf], deadline);
    phase[buf] ^= 1u;
    bad = __syncthreads_or(late || bad);
    ++job;
    return buf ? stg1 : stg0;
  };
  // full vector of tile t (b rows) from the owners' strip buffers
  auto gather_tile = [&](int t, const C* base) {
    for (int i = threadIdx.x; i < b * rc; i += GT) {
      const int j = i % rc, row = i / rc;
      const int sid = t * nh + row / HR;
      const C* src = cluster_map(base + (int64_t)(sid / CL) * HR * ldv, (uint32_t)(sid % CL));
      sy[row * ldv + j] = src[(row % HR) * ldv + j];
    }
  };
  __syncthreads();
  cluster_sync_all();                                 // every strip of r is loaded
  if constexpr (INV) {
    // the whole r_J from the owners' strips
    for (int i = threadIdx.x; i < nt * b * rc; i += GT) {
      const int j = i % rc, row = i / rc;
      const int sid = row / HR;
      const C* src = cluster_map(rbuf + (int64_t)(sid / CL) * HR * ldv, (uint32_t)(sid % CL));
      sR[row * ldv + j] = src[(row % HR) * ldv + j];
    }
    __syncthreads();
    for (int l = 0; l < nloc; ++l) {
      const int sid = rank + l * CL, tq = sid / nh, h = sid % nh;
      C* o = obuf + (int64_t)l * HR * ldv;
      const int n = FWD ? tq + 1 : nt - tq;
      for (int q = 0; q < n; ++q) {
        const C* M = next_stage();
        const C* V = sR + (int64_t)(FWD ? q : tq + q) * b * ldv;
        if (!bad) {
          if (q == 0) rows_matvec_dense<R, 0>(M, b, V, ldv, rc, o, ldv);
          else rows_matvec_dense<R, 1>(M, b, V, ldv, rc, o, ldv);
        }
        __syncthreads();
      }
      for (int i = threadIdx.x; i < HR * rc; i += GT) {
        const int row = i % HR, j = i / HR;
        Y[(int64_t)(j0 + j) * s.npad + (int64_t)(t0 + tq) * b + h * HR + row] = o[row * ldv + j];
      }
    }
    cluster_sync_all();                               // nobody reads this CTA's strips any more
  } else {
  for (int q = 0; q < nt; ++q) {
    const int t = FWD ? q : nt - 1 - q;
    // ---- the owners of tile t solve their halves
    bool own = false;
    for (int l = 0; l < nloc; ++l) own |= (rank + l * CL) / nh == t;
    if (own) {
      gather_tile(t, rbuf);
      __syncthreads();
      for (int l = 0; l < nloc; ++l) {
        const int sid = rank + l * CL, h = sid % nh;
        if (sid / nh != t) continue;
        const C* M = next_stage();
        C* o = obuf + (int64_t)l * HR * ldv;
        if (!bad) {
          if (FWD) rows_matvec<R, 0>(M, ldst, b, sy, ldv, rc, o, ldv);
          else colstrip_matvec<R, 0>(M, ldst, b, sy, ldv, rc, o, ldv);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < HR * rc; i += GT) {
          const int row = i % HR, j = i / HR;
          Y[(int64_t)(j0 + j) * s.npad + (int64_t)(t0 + t) * b + h * HR + row] = o[row * ldv + j];
        }
      }
    }
    cluster_sync_all();                               // y_t (w_t) is complete
    // ---- the owners of the remaining tiles apply it
    bool upd = false;
    for (int l = 0; l < nloc; ++l) {
      const int tp = (rank + l * CL) / nh;
      upd |= FWD ? tp > t : tp < t;
    }
    if (upd) {
      gather_tile(t, obuf);
      __syncthreads();
      for (int l = 0; l < nloc; ++l) {
        const int tp = (rank + l * CL) / nh;
        if (!(FWD ? tp > t : tp < t)) continue;
        const C* M = next_stage();
        C* r = rbuf + (int64_t)l * HR * ldv;
        if (!bad) {
          if (FWD) rows_matvec<R, 2>(M, ldst, b, sy, ldv, rc, r, ldv);
          else colstrip_matvec<R, 2>(M, ldst, b, sy, ldv, rc, r, ldv);
        }
        __syncthreads();
      }
    }
    cluster_sync_all();                               // the strips of tile t+1 (t-1) are final
  }
  }
  if (bad && threadIdx.x == 0) atomicExch(s.status, (int)D3M_ERR_TIMEOUT);
}

// ------------------------------------------------------------------ norms, omega, gradients
__global__ void vec_absmax_kernel(const double2* __restrict__ V, int64_t n, int nrhs, unsigned* out) {
  const int j = blockIdx.y;
  float a = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = V[(int64_t)j * n + i];
    const float x = (float)v.x, y = (float)v.y;
    a = fmaxf(a, sqrtf(x * x + y * y));
  }
  for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out + j, __float_as_uint(a));
}

// omega_(i,j) = |r|_(i,j) / (||K_i|| |x|_(i,j) + |b|_(i,j)) for instance i, column j (entry
// i * ld + j), recomputed for the instances still refining (a converged instance keeps the values
// of the step that converged it, and done[i] is set once all its columns meet tol);
// stat[0] = the largest over all instances.  One block of 256 threads.
// An instance is done when every column has omega <= tol and a small forward error: the last
// correction d_k is at most ftol of |x|, or, with the contraction rho = |d_k| / |d_(k-1)| < 1,
// the error left in x (about rho / (1 - rho) |d_k|) is (ftol <= 0 skips the forward test).
// stat[0] = the largest omega, stat[1] = instances not done.
__global__ void omega_kernel(const unsigned* rmax, const unsigned* xmax, const unsigned* bmax,
                             const unsigned* kmax, const unsigned* dmax, float* dprev, int ninst, int ld,
                             int nrhs, int* done, double tol, double ftol, double* omega, double* stat) {
  double w = 0.0, mu = 0.0;   // mu: how far the open instances are from both targets
  int open = 0;
  for (int i = threadIdx.x; i < ninst; i += blockDim.x) {
    double wi = 0.0, mui = 0.0;
    if (!done[i]) {
      const double kn = (double)__uint_as_float(kmax[i]);
      bool ok = true;
      for (int j = 0; j < nrhs; ++j) {
        const int q = i * ld + j;
        const double r = __uint_as_float(rmax[q]), x = __uint_as_float(xmax[q]), bb = __uint_as_float(bmax[q]);
        const double den = kn * x + bb;
        const double o = den > 0 ? r / den : (r > 0 ? 1.0 : 0.0);
        omega[q] = o;
        wi = fmax(wi, o);
        const double d = __uint_as_float(dmax[q]), dp = dprev[q];
        const double ratio = x > 0 ? d / x : (d > 0 ? 1.0 : 0.0);
        const double rho = dp > 0 ? d / dp : 1.0;
        const bool fwd = ftol <= 0 || ratio <= ftol || (rho < 1.0 && rho / (1.0 - rho) * ratio <= ftol);
        ok = ok && o <= tol && fwd;
        mui = fmax(mui, fmax(o / tol, ftol > 0 ? ratio / ftol : 0.0));
        dprev[q] = (float)d;
      }
      if (ok) done[i] = 1;
      else {
        ++open;
        mu = fmax(mu, mui);
      }
    } else {
      for (int j = 0; j < nrhs; ++j) wi = fmax(wi, omega[i * ld + j]);
    }
    w = fmax(w, wi);
  }
  __shared__ double s_w[256], s_mu[256];
  __shared__ int s_o[256];
  s_w[threadIdx.x] = w;
  s_mu[threadIdx.x] = mu;
  s_o[threadIdx.x] = open;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_w[threadIdx.x] = fmax(s_w[threadIdx.x], s_w[threadIdx.x + h]);
      s_mu[threadIdx.x] = fmax(s_mu[threadIdx.x], s_mu[threadIdx.x + h]);
      s_o[threadIdx.x] += s_o[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stat[0] = s_w[0];
    stat[1] = (double)s_o[0];
    stat[2] = s_mu[0];
  }
}

// per-interface complex contraction s_f = sum_j sum_u Lambda_uj X_uj (FP64)
__global__ void contract_kernel(const double2* __restrict__ Lam, const double2* __restrict__ X, int64_t n,
                                int nrhs, const int64_t* __restrict__ xoff_orig, const int32_t* __restrict__ m_orig,
                                double2* __restrict__ out) {
  const int f = blockIdx.x;
  const int mf = m_orig[f];
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < mf * nrhs; i += blockDim.x) {
    const int u = i % mf, j = i / mf;
    const int64_t o = (int64_t)j * n + xoff_orig[f] + u;
    acc = cfma(Lam[o], X[o], acc);
  }
  __shared__ double2 s[256];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] = cadd(s[threadIdx.x], s[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[f] = s[0];
}

// dK_fg(u, v) = -sum_j (Lam_f[u,j] X_g[v,j] + [f != g] X_f[u,j] Lam_g[v,j]), column-major block
__global__ void grad_pattern_kernel(const double2* __restrict__ Lam, const double2* __restrict__ X, int64_t n,
                                    int nrhs, const int64_t* __restrict__ colptr, const int32_t* __restrict__ rowidx,
                                    const int32_t* __restrict__ blk_col, const int64_t* __restrict__ kblk_off,
                                    const int64_t* __restrict__ xoff_orig, const int32_t* __restrict__ m_orig,
                                    double2* __restrict__ dK) {
  const int e = blockIdx.x;
  const int g = blk_col[e], f = rowidx[e];
  const int mf = m_orig[f], mg = m_orig[g];
  double2* out = dK + kblk_off[e];
  for (int64_t i = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)mf * mg;
       i += (int64_t)gridDim.y * blockDim.x) {
    const int u = (int)(i % mf), v = (int)(i / mf);
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < nrhs; ++j) {
      const int64_t of = (int64_t)j * n + xoff_orig[f] + u, og = (int64_t)j * n + xoff_orig[g] + v;
      acc = cfma(Lam[of], X[og], acc);
      if (f != g) acc = cfma(X[of], Lam[og], acc);
    }
    out[i] = make_double2(-acc.x, -acc.y);
  }
  (void)colptr;
}

// ------------------------------------------------------------------ launchers
// a kernel launch that may start before its predecessor in the stream has finished (the kernels
// of a sweep wait for it with pdl_wait before they touch its results)
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <typename R>
static int sweep_impl(SweepLaunch& a, cudaStream_t st) {
  using C = typename CT<R>::C;
  const int b = a.b;
  const int nthreads = 256;
  const int64_t gblocks = (a.npad + nthreads - 1) / nthreads;
  const C* L = (const C*)a.L;
  const C* Linv = (const C*)a.Linv;
  const C* D = (const C*)a.D;
  C* Y = (C*)a.Y;
  C* P = (C*)a.P;
  const int nh = b / HR;
  a.launches = 0;
  const Mask mk{a.done, a.tinst};
  launch_pdl(permute_in_kernel<R>, dim3((unsigned)gblocks), dim3(nthreads), 0, st, a.src, a.n, Y, a.npad, a.pad2orig, a.nrhs, mk, b);
  ++a.launches;
  // gather: persistent, one block per SM; a stage buffer holds a dense 64-row tile half and <= 8
  // source rows (padded by 16 bytes), as many stages as fit (<= GMAXSTG)
  const size_t gstage = sizeof(C) * ((size_t)HR * b + (size_t)RCMAX * (b + 16 / sizeof(C)));
  const int gstg = (int)std::max<size_t>(1, std::min<size_t>(GMAXSTG, SWEEP_SMEM_LIMIT / gstage));
  const size_t gsm = (size_t)gstg * gstage;
  const unsigned gy = (unsigned)((a.nrhs + RCMAX - 1) / RCMAX);
  cudaFuncSetAttribute(gather_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
  cudaFuncSetAttribute(gather_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
  int nsm = 0;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  auto launch_gather = [&](bool fwd, int64_t i0, int64_t i1) {
    if (a.tcmaps && sizeof(R) == 4) {
      // tensor-core gather (split-BF16x3 on L's operand planes): one unit per group
      launch_gather_tc(fwd, *a.tcmaps, (fwd ? a.fwd_groups : a.bwd_groups) + i0, fwd ? a.fwd_items : a.bwd_items,
                       Y, P, a.npad, a.nrhs, a.status, a.done, a.tinst, (int)(i1 - i0), nsm, st);
      return;
    }
    const int nunits = (int)((i1 - i0) * nh);
    const dim3 grid((unsigned)std::min<int64_t>(nunits, nsm), gy);
    if (fwd)
      launch_pdl(gather_kernel<R, true>, grid, dim3(GGT), gsm, st, a.fwd_groups + i0, a.fwd_items, L, Y, P, a.npad, b,
                 a.nrhs, a.status, mk, nunits, gstg);
    else
      launch_pdl(gather_kernel<R, false>, grid, dim3(GGT), gsm, st, a.bwd_groups + i0, a.bwd_items, L, Y, P, a.npad, b,
                 a.nrhs, a.status, mk, nunits, gstg);
  };
  // cluster chains: usable when every level's largest block fits CHAIN_MAXCL x CHAIN_MAXLOC strips
  const int crc = a.nrhs < RCMAX ? a.nrhs : RCMAX;
  const int cldv = vec_ld(crc);
  const int cstg = std::max(HR * stage_ld<C>(b), b * stage_ld<C>(HR));
  bool chain = a.lev_maxnt != nullptr;
  int max_loc = 1;
  for (int lv = 0; chain && lv < a.nlevels; ++lv) {
    const int S = a.lev_maxnt[lv] * nh;
    const int cl = std::min(CHAIN_MAXCL, S);
    const int nloc = (S + cl - 1) / cl;
    if (nloc > CHAIN_MAXLOC || a.lev_maxnt[lv] > MAXNT) chain = false;
    max_loc = std::max(max_loc, nloc);
  }
  // INV mode (inverses of the diagonal blocks were built with the factorization): the whole r_J
  // of the largest block is gathered into shared memory as well
  const bool inv = a.Inv != nullptr;
  const size_t rrows = inv ? (size_t)a.max_rows : 0;
  auto chain_smem = [&](int nloc) {
    return sizeof(C) * (2 * (size_t)cstg + (size_t)b * cldv + 2 * (size_t)nloc * HR * cldv + rrows * cldv);
  };
  if (chain && chain_smem(max_loc) > SWEEP_SMEM_LIMIT) chain = false;
  if (inv && !chain) return (int)cudaErrorInvalidConfiguration;   // the host enables INV only where it fits
  if (chain) {
    if (inv) {
      cudaFuncSetAttribute(chain_kernel<R, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chain_smem(max_loc));
      cudaFuncSetAttribute(chain_kernel<R, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chain_smem(max_loc));
    } else {
      cudaFuncSetAttribute(chain_kernel<R, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chain_smem(max_loc));
      cudaFuncSetAttribute(chain_kernel<R, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chain_smem(max_loc));
    }
    ChainSweep cs;
    cs.status = a.status;
    cs.tstart = a.tstart;
    cs.tcolptr = a.tcolptr;
    cs.P = P;
    cs.D = D;
    cs.npad = a.npad;
    cs.b = b;
    cs.nrhs = a.nrhs;
    cs.stg = cstg;
    cs.Inv = a.Inv;
    cs.inv_off = a.inv_off;
    cs.InvT = a.InvT;
    cs.invT_off = a.invT_off;
    cs.mk = mk;
    cs.rrows = (int)rrows;
    auto launch_chain = [&](int lv, bool fwd) -> cudaError_t {
      const int S = a.lev_maxnt[lv] * nh;
      cs.cl = std::min(CHAIN_MAXCL, S);
      cs.nloc = (S + cs.cl - 1) / cs.cl;
      cs.blocks = a.lev_blocks + a.lev_ptr[lv];
      const unsigned nb = (unsigned)(a.lev_ptr[lv + 1] - a.lev_ptr[lv]);
      cs.rc = crc;
      const unsigned ny = (unsigned)((a.nrhs + crc - 1) / crc);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(nb * (unsigned)cs.cl, ny, 1);
      cfg.blockDim = dim3(GT, 1, 1);
      cfg.dynamicSmemBytes = chain_smem(cs.nloc);
      cfg.stream = st;
      cudaLaunchAttribute attr[2];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)cs.cl;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[1].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 2;
      ++a.launches;
      if (inv)
        return fwd ? cudaLaunchKernelEx(&cfg, chain_kernel<R, true, true>, cs, L, Linv, Y)
                   : cudaLaunchKernelEx(&cfg, chain_kernel<R, false, true>, cs, L, Linv, Y);
      return fwd ? cudaLaunchKernelEx(&cfg, chain_kernel<R, true, false>, cs, L, Linv, Y)
                 : cudaLaunchKernelEx(&cfg, chain_kernel<R, false, false>, cs, L, Linv, Y);
    };
    for (int lv = 0; lv < a.nlevels; ++lv) {
      const int64_t i0 = a.fwd_group_ptr[lv], i1 = a.fwd_group_ptr[lv + 1];
      if (i1 > i0) {
        launch_gather(true, i0, i1);
        ++a.launches;
      }
      cs.slot_ptr = a.fwd_slot_ptr;
      cs.has_partials = i1 > i0;
      cs.apply_d = 0;
      if (i1 > i0 && a.lev_maxcnt_fwd[lv] > EXT_REDUCE) {
        // many partials per row: a wide reduce launch is cheaper than the cluster's strip loads
        const int64_t ntl = a.lev_tile_ptr[lv + 1] - a.lev_tile_ptr[lv];
        const int64_t nthr = ntl * b * a.nrhs;
        launch_pdl(reduce_kernel<R>, dim3((unsigned)((nthr + 31) / 32)), dim3(ET), 0, st, a.lev_tiles + a.lev_tile_ptr[lv], (int)ntl,
                                                                       a.fwd_slot_ptr, P, Y, a.npad, b, a.nrhs, 1, nullptr, mk);
        ++a.launches;
        cs.has_partials = 0;
      }
      cudaError_t e = launch_chain(lv, true);
      if (e != cudaSuccess) return (int)e;
    }
    const bool bk = a.E != nullptr;
    if (bk) {
      // pivoted factor: z = D^{-1} y with its 2 x 2 blocks as one pass between the sweeps
      diag_scale_bk_kernel<R><<<(unsigned)gblocks, nthreads, 0, st>>>(Y, D, (const C*)a.E, a.npad, a.nrhs, b);
      ++a.launches;
    }
    for (int lv = a.nlevels - 1; lv >= 0; --lv) {
      const int64_t i0 = a.bwd_group_ptr[lv], i1 = a.bwd_group_ptr[lv + 1];
      if (i1 > i0) {
        launch_gather(false, i0, i1);
        ++a.launches;
      }
      cs.slot_ptr = a.bwd_slot_ptr;
      cs.has_partials = i1 > i0;
      cs.apply_d = bk ? 0 : 1;
      if (i1 > i0 && a.lev_maxcnt_bwd[lv] > EXT_REDUCE) {
        const int64_t ntl = a.lev_tile_ptr[lv + 1] - a.lev_tile_ptr[lv];
        const int64_t nthr = ntl * b * a.nrhs;
        launch_pdl(reduce_kernel<R>, dim3((unsigned)((nthr + 31) / 32)), dim3(ET), 0, st, a.lev_tiles + a.lev_tile_ptr[lv], (int)ntl,
                                                                       a.bwd_slot_ptr, P, Y, a.npad, b, a.nrhs, nh, bk ? nullptr : D, mk);
        ++a.launches;
        cs.has_partials = 0;
        cs.apply_d = 0;
      }
      cudaError_t e = launch_chain(lv, false);
      if (e != cudaSuccess) return (int)e;
    }
    launch_pdl(permute_out_kernel<R>, dim3((unsigned)gblocks), dim3(nthreads), 0, st, Y, a.npad, a.dst, a.n, a.pad2orig, a.nrhs, a.accumulate, mk, b, a.dmax, a.ld_norm);
    ++a.launches;
    return (int)cudaGetLastError();
  }
  // single-CTA chains (blocks too large for one cluster)
  // rhs per block kernel: at most 8, fewer if the running vector would not fit in shared memory
  int rc = a.nrhs < 8 ? a.nrhs : 8;
  auto block_smem = [&](int r) {
    return sizeof(C) * (2 * (size_t)HR * stage_ld<C>(b) + ((size_t)a.max_rows + (size_t)b) * vec_ld(r));
  };
  while (rc > 1 && block_smem(rc) > SWEEP_SMEM_LIMIT) rc = (rc + 1) / 2;
  const size_t bsm = block_smem(rc);
  if (bsm > SWEEP_SMEM_LIMIT) return (int)cudaErrorInvalidConfiguration;
  cudaFuncSetAttribute(block_fwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm);
  cudaFuncSetAttribute(block_bwd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm);
  BlockSweep bs;
  bs.status = a.status;
  bs.tstart = a.tstart;
  bs.tcolptr = a.tcolptr;
  bs.npad = a.npad;
  bs.b = b;
  bs.nrhs = a.nrhs;
  bs.rc = rc;
  const unsigned ny = (unsigned)((a.nrhs + rc - 1) / rc);
  for (int lv = 0; lv < a.nlevels; ++lv) {
    const int64_t i0 = a.fwd_group_ptr[lv], i1 = a.fwd_group_ptr[lv + 1];
    const int64_t ntl = a.lev_tile_ptr[lv + 1] - a.lev_tile_ptr[lv];
    if (i1 > i0) {
      launch_gather(true, i0, i1);
      const int64_t nthr = ntl * b * a.nrhs;
      launch_pdl(reduce_kernel<R>, dim3((unsigned)((nthr + 31) / 32)), dim3(ET), 0, st, a.lev_tiles + a.lev_tile_ptr[lv], (int)ntl,
                                                                     a.fwd_slot_ptr, P, Y, a.npad, b, a.nrhs, 1, nullptr, mk);
      a.launches += 2;
    }
    bs.blocks = a.lev_blocks + a.lev_ptr[lv];
    bs.slot_ptr = a.fwd_slot_ptr;
    const unsigned nb = (unsigned)(a.lev_ptr[lv + 1] - a.lev_ptr[lv]);
    block_fwd_kernel<R><<<dim3(nb, ny), GT, bsm, st>>>(bs, L, Linv, Y);
    ++a.launches;
  }
  if (a.E) diag_scale_bk_kernel<R><<<(unsigned)gblocks, nthreads, 0, st>>>(Y, D, (const C*)a.E, a.npad, a.nrhs, b);
  else diag_scale_kernel<R><<<(unsigned)gblocks, nthreads, 0, st>>>(Y, D, a.npad, a.nrhs);
  ++a.launches;
  for (int lv = a.nlevels - 1; lv >= 0; --lv) {
    const int64_t i0 = a.bwd_group_ptr[lv], i1 = a.bwd_group_ptr[lv + 1];
    const int64_t ntl = a.lev_tile_ptr[lv + 1] - a.lev_tile_ptr[lv];
    if (i1 > i0) {
      launch_gather(false, i0, i1);
      const int64_t nthr = ntl * b * a.nrhs;
      launch_pdl(reduce_kernel<R>, dim3((unsigned)((nthr + 31) / 32)), dim3(ET), 0, st, a.lev_tiles + a.lev_tile_ptr[lv], (int)ntl,
                                                                     a.bwd_slot_ptr, P, Y, a.npad, b, a.nrhs, nh, nullptr, mk);
      a.launches += 2;
    }
    bs.blocks = a.lev_blocks + a.lev_ptr[lv];
    bs.slot_ptr = a.bwd_slot_ptr;
    const unsigned nb = (unsigned)(a.lev_ptr[lv + 1] - a.lev_ptr[lv]);
    block_bwd_kernel<R><<<dim3(nb, ny), GT, bsm, st>>>(bs, L, Linv, Y);
    ++a.launches;
  }
  launch_pdl(permute_out_kernel<R>, dim3((unsigned)gblocks), dim3(nthreads), 0, st, Y, a.npad, a.dst, a.n, a.pad2orig, a.nrhs, a.accumulate, mk, b, a.dmax, a.ld_norm);
  ++a.launches;
  return (int)cudaGetLastError();
}

int launch_sweep(SweepLaunch& a, bool fp64, cudaStream_t st) {
  return fp64 ? sweep_impl<double>(a, st) : sweep_impl<float>(a, st);
}

int launch_absmax(const double2* V, int64_t n, int nrhs, unsigned* out, cudaStream_t st) {
  const int64_t nb = (n + 255) / 256;
  vec_absmax_kernel<<<dim3((unsigned)(nb < 1024 ? nb : 1024), (unsigned)nrhs), 256, 0, st>>>(V, n, nrhs, out);
  return (int)cudaGetLastError();
}

int launch_omega(const unsigned* rmax, const unsigned* xmax, const unsigned* bmax, const unsigned* kmax,
                 const unsigned* dmax, float* dprev, int ninst, int ld, int nrhs, int* done, double tol, double ftol,
                 double* omega, double* stat, cudaStream_t st) {
  omega_kernel<<<1, 256, 0, st>>>(rmax, xmax, bmax, kmax, dmax, dprev, ninst, ld, nrhs, done, tol, ftol, omega, stat);
  return (int)cudaGetLastError();
}

int launch_contract(const double2* Lam, const double2* X, int64_t n, int nrhs, const int64_t* xoff_orig,
                    const int32_t* m_orig, int nblk, double2* out, cudaStream_t st) {
  contract_kernel<<<nblk, 256, 0, st>>>(Lam, X, n, nrhs, xoff_orig, m_orig, out);
  return (int)cudaGetLastError();
}

int launch_grad_pattern(const double2* Lam, const double2* X, int64_t n, int nrhs, const int64_t* colptr,
                        const int32_t* rowidx, const int32_t* blk_col, const int64_t* kblk_off,
                        const int64_t* xoff_orig, const int32_t* m_orig, int64_t nnzb, double2* dK, cudaStream_t st) {
  grad_pattern_kernel<<<dim3((unsigned)nnzb, 16), 256, 0, st>>>(Lam, X, n, nrhs, colptr, rowidx, blk_col, kblk_off,
                                                                 xoff_orig, m_orig, dK);
  return (int)cudaGetLastError();
}

}  // namespace d3m
