// FP64-accurate residual r = b - K x on the tcgen05 tensor cores (the refinement's residual:
// FP64 on the GPU only for r = b - K x and the solution update).
//
// Method: an exact-product splitting in the manner of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 2012), with the slices held as small integers in bf16:
//  * every stored block K_fg gets one scale 2^E (max |Re|, |Im| over the block < 2^E; the
//    diagonal entries of a diagonal block are left out of the block and applied in FP64); the
//    normalised entries k = K 2^-E are written as 9 balanced base-64 digits,
//        k ~ sum_{s=1..9} a_s 2^(-6 s),  a_1 in [-64, 64], a_s in [-32, 31] (s > 1),
//    each digit an integer that bf16 holds exactly (|k - sum| <= 2^-55);
//  * every block of x (block g, right-hand side j) gets its own scale 2^T and digits b_q the
//    same way;
//  * a digit product a_s b_q is an integer of at most 12 bits, so the tensor core's FP32
//    accumulation of all products of one level t = s + q over a block of up to 512 columns
//    (2 x 512 terms with the real embedding of the complex product, at most 9 digit pairs a
//    level) stays below 2^23.5 and is EXACT; the levels t = 2..10 (45 digit pairs) are kept;
//  * the nine exact level sums of a block are combined exactly in two 64-bit integers
//    (levels 2..6 and 7..10, aligned by their powers of 64), which are converted to FP64, scaled
//    by 2^(E + T) and accumulated in FP64; r = b - acc - diag(K) x.  A simulation of these steps
//    gives a residual error of 2-4e-17 of ||K|| ||x||, below that of a plain FP64 residual.
// Complex products use the real embedding along K: A = [a_r | a_i] (row u, 2 x 32 columns per
// chunk), B = [[b_r, b_i]; [-b_i, b_r]] (N = 2 NR output columns: Re of NR right-hand sides,
// then Im).  The digit planes of B are stacked, and so are the levels in TMEM, so that one MMA
// (N' = (9 - a) N <= 256 columns, split beyond) multiplies A digit a by every B digit it meets.
//
// Data (all bf16 digit planes of 128 or 64 rows x 32 columns = 64-byte rows, 64-byte swizzle on
// load): K digits per residual contribution (row tile, 32-column chunk, part r/i, digit), both
// orientations of an off-diagonal block stored (written once per factorization); x digits per
// block g (chunk, part, digit) and 64 rows (written per residual call).
//
// Kernel roles (320 threads): warp 0 issues the TMA loads (two 99 KB stages: 9 A planes of one
// part + 9 B planes), warp 1 issues the MMAs into 9 level accumulators in TMEM (9 x N <= 432
// columns, N = 2 NR <= 48: at most 24 right-hand sides a launch), warps 2..9 read the levels
// back after every block and accumulate.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "d3m.h"
#include "device.cuh"
#include "kernels.h"

namespace d3m {

namespace {

constexpr int RT_WARPS = 10;
constexpr int RT_THREADS = RT_WARPS * 32;
constexpr int ND = kResidDigits;                   // digits per value (levels kept: 0..ND-1)
constexpr int NRMAX = 24;                          // right-hand sides per launch (N = 2 NR <= 48)
constexpr uint32_t APLANE = 128 * 64;              // 8 KB: 128 rows x 32 bf16
constexpr uint32_t BPLANE_MAX = 2 * NRMAX * 64;    // 3 KB: up to 48 rows x 32 bf16
constexpr uint32_t A_STAGE = ND * APLANE;          // 72 KB
constexpr uint32_t B_STAGE = ND * BPLANE_MAX;      // 27 KB
constexpr uint32_t STG = A_STAGE + B_STAGE;        // 99 KB (a multiple of the 1 KB swizzle atom)
constexpr int NSTG = 2;
constexpr uint32_t RT_SMEM = NSTG * STG;            // 198 KB
static_assert(STG % 1024 == 0 && ND * 2 * NRMAX <= 512, "stage layout / TMEM columns");
constexpr int UNIT_KC = 16;                        // 32-column chunks per accumulation unit (512 columns)

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint64_t deadline) {
  while (!bar_try(bar, parity)) {
    if (globaltimer_ns() > deadline) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_3d(uint32_t dst, const void* map, int x, int y, int z, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
// K-major, 64-byte swizzle, 8-row groups 512 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// kind::f16, A and B bf16, D f32, K-major, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit_bar(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Balanced base-64 digits of a double relative to the scale 2^E (|x| < 2^E): x 2^-E ~
// sum_s d[s] 2^(-6 (s+1)), d[0] in [-64, 64], d[s] in [-32, 31].  Integer operations only: the
// 53-bit significand is aligned to a 54-bit fixed point (rounded), then peeled 6 bits at a time
// from the bottom.  Zeros, subnormals and values below 2^(E-55) give all-zero digits.
__device__ __forceinline__ void digits64(double x, int E, int* d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((u >> 52) & 0x7ff);
  long long F = 0;
  if (be != 0 && be != 0x7ff) {
    const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = be - 1021 - E;          // x 2^(54 - E) = mant 2^(be - 1075 + 54 - E)
    unsigned long long a;
    if (sh >= 0) a = mant << (sh > 1 ? 1 : sh);     // |x| < 2^E keeps sh <= 1 (|a| < 2^54)
    else if (sh > -64) a = (mant + (1ull << (-sh - 1))) >> (-sh);
    else a = 0;
    F = (u >> 63) ? -(long long)a : (long long)a;
  }
#pragma unroll
  for (int s = ND - 1; s >= 1; --s) {
    int v = (int)(F & 63);
    if (v >= 32) v -= 64;
    d[s] = v;
    F = (F - v) >> 6;
  }
  d[0] = (int)F;
}

// exponent E with |v| < 2^E for the largest magnitude v (as double bits); 0 for v = 0
__device__ __forceinline__ int scale_exp(unsigned long long maxbits) {
  const int be = (int)((maxbits >> 52) & 0x7ff);
  return be == 0 ? 0 : be - 1022;
}

__device__ __forceinline__ unsigned short bf16_of_int(int v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)v));   // |v| <= 64: exact
}

// ---------------------------------------------------------------- K digits
// (1) per stored block: max |Re|, |Im| (diagonal entries of a diagonal block excluded) as double
// bits, and the diagonal entries of the diagonal blocks (applied in FP64 by the residual)
__global__ void __launch_bounds__(256) kblock_max_kernel(ResidualTc p) {
  const int blk = blockIdx.x;
  const int f = p.blk_row[blk], g = p.blk_col[blk];
  const int mf = p.m_orig[f], mg = p.m_orig[g];
  const double2* Kb = p.K + p.kblk_off[blk];
  const int64_t tot = (int64_t)mf * mg;
  unsigned long long mx = 0;
  for (int64_t i = blockIdx.y * 256 + threadIdx.x; i < tot; i += 256 * gridDim.y) {
    const double2 v = __ldg(Kb + i);
    const int c = (int)(i / mf), u = (int)(i - (int64_t)c * mf);
    if (f == g && u == c) {
      p.Kdiag[p.xoff_orig[f] + u] = v;
      continue;
    }
    const double a = fmax(fabs(v.x), fabs(v.y));
    const unsigned long long ab = (unsigned long long)__double_as_longlong(a);
    mx = ab > mx ? ab : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(p.Kmax_bits + blk, mx);
}

// (2) digits of the stored blocks: one tile of 128 rows x 16 columns of a stored block K_fg
// (f >= g) per CTA (39 KB of shared memory: five CTAs per SM).  Every entry's 2 ND digits are
// extracted once, into shared memory (int8), and written to the planes of both residual
// contributions of the block: row block f (untransposed: planes of 128 rows u x 32 columns c, of
// which this CTA fills 16 columns) and, for f != g, row block g (transposed: planes of 128 rows c
// x 32 columns u, of which this CTA fills 16 rows).  K is read once, coalesced along u
// (column-major blocks).  Also adds |K| row sums (rows u) and column sums (rows c of the
// transposed use) into rowsum, for ||K||_inf.
constexpr int KD_U = 128, KD_C = 16, KD_LD = 136;   // tile rows, tile columns, padded byte row
constexpr size_t KD_SMEM = (size_t)2 * ND * KD_C * KD_LD;

__global__ void __launch_bounds__(256) kdigits_kernel(ResidualTc p) {
  extern __shared__ __align__(16) signed char sdig[];   // [2 ND][KD_C][KD_LD]
  __shared__ float s_cs[KD_C];
  const int blk = blockIdx.x, rt = blockIdx.y, ct = blockIdx.z;
  const int f = p.blk_row[blk], g = p.blk_col[blk];
  const int mf = p.m_orig[f], mg = p.m_orig[g];
  // the grid covers the largest blocks; a tile of columns past mg still runs while it lies in the
  // block's last 32-column chunk, so that every chunk's padding columns get zero digits
  if (rt * KD_U >= mf || ct * KD_C >= (mg + 31) / 32 * 32) return;
  const int E = scale_exp(p.Kmax_bits[blk]);
  const double2* Kb = p.K + p.kblk_off[blk];
  const bool diag = (f == g);
  const int tid = threadIdx.x, lane = tid & 31, ul = tid & 127, ch = tid >> 7;
  const int u = rt * KD_U + ul;
  if (tid < KD_C) s_cs[tid] = 0.f;
  __syncthreads();
  float rs = 0.f;
  for (int q = 0; q < KD_C / 2; ++q) {
    const int cl = ch + 2 * q, c = ct * KD_C + cl;
    double2 v = make_double2(0.0, 0.0);
    float a = 0.f;
    if (u < mf && c < mg) {
      v = __ldg(Kb + (int64_t)c * mf + u);
      const float fx = (float)v.x, fy = (float)v.y;
      a = sqrtf(fx * fx + fy * fy);
      if (diag && u == c) v = make_double2(0.0, 0.0);
    }
    rs += a;
    float cs = a;
    for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
    if (lane == 0) atomicAdd(&s_cs[cl], cs);
    int dr[ND], di[ND];
    digits64(v.x, E, dr);
    digits64(v.y, E, di);
#pragma unroll
    for (int s = 0; s < ND; ++s) {
      sdig[((0 * ND + s) * KD_C + cl) * KD_LD + ul] = (signed char)dr[s];
      sdig[((1 * ND + s) * KD_C + cl) * KD_LD + ul] = (signed char)di[s];
    }
  }
  if (u < mf) atomicAdd(p.rowsum + p.xoff_orig[f] + u, rs);
  __syncthreads();
  if (!diag && tid < KD_C && ct * KD_C + tid < mg) atomicAdd(p.rowsum + p.xoff_orig[g] + ct * KD_C + tid, s_cs[tid]);
  auto bf8 = [](const signed char* v8, int stride) {
    unsigned short h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = bf16_of_int((int)v8[q * stride]);
    return *reinterpret_cast<uint4*>(h);
  };
  // untransposed planes (row block f): 16-byte units (row r, 8 columns); the CTA's 16 columns
  // are units 2 (ct % 2) .. + 1 of chunk ct / 2
  {
    const int nkc = (mg + 31) / 32;
    const int kc = ct / 2, u0 = (ct & 1) * 2;
    unsigned short* base = p.kdig + ((int64_t)p.ks_plane[p.blk_eu[blk]] + (int64_t)rt * nkc * 2 * ND) * (128 * 32);
    for (int w = tid; w < 2 * ND * 128 * 2; w += 256) {
      const int j2 = w & 1, r = (w >> 1) & 127, pl = w >> 8;
      const uint4 val = bf8(sdig + ((int64_t)pl * KD_C + j2 * 8) * KD_LD + r, KD_LD);
      *reinterpret_cast<uint4*>(base + ((int64_t)kc * 2 * ND + pl) * (128 * 32) + r * 32 + (u0 + j2) * 8) = val;
    }
  }
  // transposed planes (row block g, source f): rows c (16 of the 128 of tile ct / 8), 32-column
  // chunks of u; a unit is 8 consecutive u of one c (consecutive shared bytes)
  if (!diag) {
    const int nkc = (mf + 31) / 32;
    unsigned short* base =
        p.kdig + ((int64_t)p.ks_plane[p.blk_et[blk]] + (int64_t)(ct / 8) * nkc * 2 * ND) * (128 * 32);
    const int r0 = (ct & 7) * KD_C;
    for (int w = tid; w < 2 * ND * 4 * KD_C * 4; w += 256) {
      const int j8 = w & 3, cl = (w >> 2) & (KD_C - 1), kcl = (w >> 6) & 3, pl = w >> 8;
      const int kc = rt * 4 + kcl;
      if (kc >= nkc) continue;
      const uint4 val = bf8(sdig + ((int64_t)pl * KD_C + cl) * KD_LD + kcl * 32 + j8 * 8, 1);
      *reinterpret_cast<uint4*>(base + ((int64_t)kc * 2 * ND + pl) * (128 * 32) + (r0 + cl) * 32 + j8 * 8) = val;
    }
  }
}

// (3) ||K_i||_inf = max row sum over the rows of instance i
__global__ void rowsum_max_kernel(const float* __restrict__ rowsum, const int64_t* __restrict__ xoff_orig,
                                  const int32_t* __restrict__ m_orig, const int32_t* __restrict__ inst, int nblk,
                                  unsigned* kmax) {
  const int f = blockIdx.x;
  float mx = 0.f;
  for (int u = threadIdx.x; u < m_orig[f]; u += blockDim.x) mx = fmaxf(mx, rowsum[xoff_orig[f] + u]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(kmax + inst[f], __float_as_uint(mx));
}

// ---------------------------------------------------------------- x digits (per residual call)
// Block g, right-hand sides j0 .. j0 + NR - 1: T_(g,j) from max |Re|, |Im| over the block's rows,
// then the B planes [chunk][part][digit] of N = 2 NR rows x 32 columns (rows beyond N unused):
//   part r: row j -> b_r(c, j), row NR + j -> b_i(c, j);  part i: row j -> -b_i, row NR + j -> b_r.
__global__ void __launch_bounds__(256) xdigits_kernel(ResidualTc p, const double2* __restrict__ X, int nrhs, int NR) {
  const int g = blockIdx.x, grp = blockIdx.y, j0 = grp * NR;
  if (p.done && p.done[p.inst[g]]) return;
  const int mg = p.m_orig[g];
  const int64_t xo = p.xoff_orig[g];
  __shared__ unsigned long long s_max[32];
  __shared__ int s_T[32];
  const int jl = threadIdx.x & 31, cl = threadIdx.x >> 5;   // column lane (j), 8 row lanes
  unsigned long long mx = 0;
  if (jl < NR && j0 + jl < nrhs)
    for (int c = cl; c < mg; c += 8) {
      const double2 v = X[(int64_t)(j0 + jl) * p.n + xo + c];
      const double a = fmax(fabs(v.x), fabs(v.y));
      const unsigned long long ab = (unsigned long long)__double_as_longlong(a);
      mx = ab > mx ? ab : mx;
    }
  if (threadIdx.x < 32) s_max[threadIdx.x] = 0;
  __syncthreads();
  atomicMax(&s_max[jl], mx);
  __syncthreads();
  if (threadIdx.x < 32) {
    s_T[threadIdx.x] = scale_exp(s_max[threadIdx.x]);
    if (threadIdx.x < NR) p.xT[((int64_t)grp * p.nblk + g) * 32 + threadIdx.x] = s_T[threadIdx.x];
  }
  __syncthreads();
  const int nkc = (mg + 31) / 32;
  const int N = 2 * NR;
  unsigned short* planes = p.xdig + ((int64_t)grp * p.xs_total + p.xs_plane[g]) * (64 * 32);
  // one thread per (chunk, row n, 8-column group): digits of 8 entries, 2 parts x 8 digits
  const int64_t jobs = (int64_t)nkc * N * 4;
  for (int64_t w = threadIdx.x; w < jobs; w += 256) {
    const int c8 = (int)(w & 3), n = (int)((w >> 2) % N);
    const int kc = (int)((w >> 2) / N);
    const int j = n < NR ? n : n - NR;
    const bool re_row = n < NR;
    unsigned short o[2][ND][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = kc * 32 + c8 * 8 + q;
      double2 v = make_double2(0.0, 0.0);
      if (c < mg && j0 + j < nrhs) v = X[(int64_t)(j0 + j) * p.n + xo + c];
      int dr[ND], di[ND];
      digits64(v.x, s_T[j], dr);
      digits64(v.y, s_T[j], di);
#pragma unroll
      for (int s = 0; s < ND; ++s) {
        // part r: Re rows take b_r, Im rows b_i; part i: Re rows take -b_i, Im rows b_r
        o[0][s][q] = bf16_of_int(re_row ? dr[s] : di[s]);
        o[1][s][q] = bf16_of_int(re_row ? -di[s] : dr[s]);
      }
    }
#pragma unroll
    for (int part = 0; part < 2; ++part)
#pragma unroll
      for (int s = 0; s < ND; ++s) {
        unsigned short* pl = planes + ((int64_t)(kc * 2 + part) * ND + s) * (64 * 32) + (int64_t)n * 32 + c8 * 8;
        *reinterpret_cast<uint4*>(pl) = *reinterpret_cast<uint4*>(&o[part][s][0]);
      }
  }
}

// ---------------------------------------------------------------- the residual kernel
__global__ void __launch_bounds__(RT_THREADS, 1)
    resid_tc_kernel(const ResidualTc p, const __grid_constant__ CUtensorMap mapA,
                    const __grid_constant__ CUtensorMap mapB, const double2* __restrict__ X,
                    const double2* __restrict__ B, double2* __restrict__ R, int nrhs, int NR, int ngrp) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_full[NSTG], bar_empty[NSTG], bar_accf, bar_acce;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the right-hand-side groups of one row tile are adjacent block indices, so they run together
  // and read the tile's K digits from L2 after the first one brought them in
  const int grp = blockIdx.x % ngrp, j0 = grp * NR;
  const int2 rtile = p.rtiles[blockIdx.x / ngrp];
  const int f = rtile.x, rt = rtile.y;
  if (p.done && p.done[p.inst[f]]) return;       // converged instance: r and its norms are kept
  const int mf = p.m_orig[f];
  const int N = 2 * NR;
  const int64_t e0 = p.res_ptr[f], e1 = p.res_ptr[f + 1];
  const uint64_t deadline = globaltimer_ns() + (uint64_t)p.timeout_ns;

  if (tid == 0) {
    for (int s = 0; s < NSTG; ++s) {
      bar_init(su32(&bar_full[s]), 1);
      bar_init(su32(&bar_empty[s]), 1);
    }
    bar_init(su32(&bar_accf), 1);
    bar_init(su32(&bar_acce), RT_WARPS - 2);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)), "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t bbytes = (uint32_t)N * 64;          // one B digit plane (N rows x 64 bytes)

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t e = e0; e < e1 && ok; ++e) {
        const int g = p.res_src[e];
        const int nkc = (p.m_orig[g] + 31) / 32;
        const int64_t abase = p.ks_plane[e] + (int64_t)rt * nkc * 2 * ND;
        const int64_t bbase = (int64_t)grp * p.xs_total + p.xs_plane[g];
        for (int kc = 0; kc < nkc && ok; ++kc)
          for (int part = 0; part < 2; ++part, ++it) {
            const uint32_t s = it % NSTG, use = it / NSTG;
            if (!bar_wait(su32(&bar_empty[s]), (use & 1) ^ 1, deadline)) { ok = false; break; }
            const uint32_t fb = su32(&bar_full[s]);
            bar_expect_tx(fb, A_STAGE + ND * bbytes);
            const uint32_t sa = su32(smem + s * STG);
            tma_3d(sa, &mapA, 0, 0, (int)(abase + (int64_t)(kc * 2 + part) * ND), fb);
            tma_3d(sa + A_STAGE, &mapB, 0, 0, (int)(bbase + (int64_t)(kc * 2 + part) * ND), fb);
          }
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t it = 0, unit = 0;
      bool ok = true;
      for (int64_t e = e0; e < e1 && ok; ++e) {
        const int g = p.res_src[e];
        const int nkc = (p.m_orig[g] + 31) / 32;
        for (int k0 = 0; k0 < nkc && ok; k0 += UNIT_KC, ++unit) {
          // the epilogue has read the previous unit's levels
          if (!bar_wait(su32(&bar_acce), (unit & 1) ^ 1, deadline)) { ok = false; break; }
          fence_after();
          const int k1 = min(nkc, k0 + UNIT_KC);
          for (int kc = k0; kc < k1 && ok; ++kc)
            for (int part = 0; part < 2; ++part, ++it) {
              const uint32_t s = it % NSTG, use = it / NSTG;
              if (!bar_wait(su32(&bar_full[s]), use & 1, deadline)) { ok = false; break; }
              fence_after();
              const uint32_t sa = su32(smem + s * STG), sb = sa + A_STAGE;
              const bool first = (kc == k0 && part == 0);
              // A digit da meets B digits 0 .. ND-1-da: those B planes are consecutive rows in
              // shared memory and the levels da .. ND-1 consecutive TMEM columns, so one MMA of
              // N' = (ND - da) N rows (split at 256) covers all of them
#pragma unroll
              for (int kk = 0; kk < 2; ++kk)
#pragma unroll
                for (int da = 0; da < ND; ++da) {
                  const int rows = (ND - da) * N;
                  // digit 0 of A opens every level of this unit (at kk = 0 of its first stage)
                  const uint32_t acc = (first && kk == 0 && da == 0) ? 0u : 1u;
                  for (int off = 0; off < rows; off += 256) {
                    const int nn = rows - off < 256 ? rows - off : 256;
                    mma_bf16(tmem + (uint32_t)(da * N + off), sdesc(sa + da * APLANE + kk * 32),
                             sdesc(sb + (uint32_t)off * 64 + kk * 32), idesc_bf16((uint32_t)nn), acc);
                  }
                }
              mma_commit_bar(su32(&bar_empty[s]));
            }
          mma_commit_bar(su32(&bar_accf));
        }
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (8 warps)
    const int quad = warp & 3, hpart = (warp - 2) >> 2;   // TMEM lanes 32 quad.., Re (0) / Im (1)
    const int row = quad * 32 + lane;
    const int u = rt * 128 + row;
    double acc[NRMAX];
#pragma unroll
    for (int j = 0; j < NRMAX; ++j) acc[j] = 0.0;
    uint32_t unit = 0;
    bool ok = true;
    for (int64_t e = e0; e < e1 && ok; ++e) {
      const int g = p.res_src[e];
      const int nkc = (p.m_orig[g] + 31) / 32;
      const int E = scale_exp(p.Kmax_bits[p.res_blk[e]]);
      const int* Tg = p.xT + ((int64_t)grp * p.nblk + g) * 32;
      for (int k0 = 0; k0 < nkc; k0 += UNIT_KC, ++unit) {
        if (!bar_wait(su32(&bar_accf), unit & 1, deadline)) { ok = false; break; }
        fence_after();
#pragma unroll
        for (int jb = 0; jb < NRMAX; jb += 8) {
          if (jb < NR) {
            // the level sums are exact integers below 2^23.5: levels 0..4 and 5..8 are combined
            // exactly in 64-bit integers aligned by powers of 64
            long long u1[8], u2[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) u1[q] = u2[q] = 0;
#pragma unroll
            for (int t = 0; t < ND; ++t) {
              float v[8];
              tmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(t * N + hpart * NR + jb), v);
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const long long iv = (long long)__float2int_rn(v[q]);
                if (t <= 4) u1[q] += iv << (6 * (4 - t));
                else u2[q] += iv << (6 * (8 - t));
              }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              // value = (u1 2^-36 + u2 2^-60) 2^(E + T): level t weighs 2^(-12 - 6 t)
              int ex = E + Tg[jb + q];
              ex = ex < -900 ? -900 : (ex > 900 ? 900 : ex);
              const double s1 = __longlong_as_double((long long)(ex - 36 + 1023) << 52);
              const double s2 = __longlong_as_double((long long)(ex - 60 + 1023) << 52);
              acc[jb + q] = fma((double)u1[q], s1, fma((double)u2[q], s2, acc[jb + q]));
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(su32(&bar_acce));
      }
    }
    if (!ok) atomicExch(&s_fail, 1);
    // r = b - acc - diag(K) x in FP64, and the maxima for omega
    const bool active = ok && u < mf;
    const int64_t xo = p.xoff_orig[f];
    const double2 kd = active ? p.Kdiag[xo + u] : make_double2(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < NRMAX; ++q) {
      const int j = j0 + q;
      if (active && q < NR && j < nrhs) {
        const int64_t o = (int64_t)j * p.n + xo + u;
        const double2 xv = X[o], bv = B[o];
        // this thread holds one part (Re or Im) of the block sums; the two parts of row u are
        // written by the two warps that share its TMEM lane quadrant
        if (hpart == 0) {
          const double dx = kd.x * xv.x - kd.y * xv.y;
          R[o].x = bv.x - acc[q] - dx;
        } else {
          const double dx = kd.x * xv.y + kd.y * xv.x;
          R[o].y = bv.y - acc[q] - dx;
        }
      }
    }
    // both parts are written: the norms are taken by the Re warps after a barrier among the
    // epilogue warps (named barrier 1, 256 threads)
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (hpart == 0) {
      for (int q = 0; q < NR; ++q) {
        const int j = j0 + q;
        float a = 0.f, x = 0.f, b = 0.f;
        if (active && j < nrhs) {
          const int64_t o = (int64_t)j * p.n + xo + u;
          const double2 r = R[o], xv = X[o], bv = B[o];
          const float rx = (float)r.x, ry = (float)r.y;
          a = sqrtf(rx * rx + ry * ry);
          const float xx = (float)xv.x, xy = (float)xv.y;
          x = sqrtf(xx * xx + xy * xy);
          const float bx = (float)bv.x, by = (float)bv.y;
          b = sqrtf(bx * bx + by * by);
        }
        for (int o = 16; o > 0; o >>= 1) {
          a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
          x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
          b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0 && j < nrhs) {
          const int qq = p.inst[f] * p.ld_norm + j0 + q;
          atomicMax(p.rmax + qq, __float_as_uint(a));
          atomicMax(p.xmax + qq, __float_as_uint(x));
          atomicMax(p.bmax + qq, __float_as_uint(b));
        }
      }
    }
  }

  __syncthreads();
  if (s_fail) {
    if (tid == 0) atomicExch(p.status, D3M_ERR_TIMEOUT);
    // give in-flight copies and MMAs time to land (bounded) before the memory is released
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 2000000ull) __nanosleep(1000);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
}

typedef CUresult (*EncodeTiledFn3)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

// Tensor maps of the digit planes: A (K digits): {32 columns, 128 rows, planes}, box {32, 128, ND};
// B (x digits): {32, 64, planes}, box {32, N, ND} for N = 16, 32, 48 (maps b[0..2]).
int resid_tc_make_maps(void* kdig, int64_t nplanes_a, void* xdig, int64_t nplanes_b, ResidTcMaps* out,
                       std::string& err) {
  static EncodeTiledFn3 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      err = "cuTensorMapEncodeTiled is not available from the driver";
      return 1;
    }
    encode = (EncodeTiledFn3)fn;
  }
  const cuuint32_t estr[3] = {1, 1, 1};
  {
    const cuuint64_t dim[3] = {32, 128, (cuuint64_t)nplanes_a};
    const cuuint64_t stride[2] = {64, 128 * 64};
    const cuuint32_t box[3] = {32, 128, (cuuint32_t)ND};
    CUtensorMap m;
    const CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, kdig, dim, stride, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      err = "cuTensorMapEncodeTiled (K digits) failed: " + std::to_string((int)r);
      return 1;
    }
    std::memcpy(out->a, &m, 128);
  }
  for (int k = 0; k < 3; ++k) {
    const cuuint64_t dim[3] = {32, 64, (cuuint64_t)nplanes_b};
    const cuuint64_t stride[2] = {64, 64 * 64};
    const cuuint32_t box[3] = {32, (cuuint32_t)(16 * (k + 1)), (cuuint32_t)ND};
    CUtensorMap m;
    const CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, xdig, dim, stride, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      err = "cuTensorMapEncodeTiled (x digits) failed: " + std::to_string((int)r);
      return 1;
    }
    std::memcpy(out->b[k], &m, 128);
  }
  return 0;
}

// digits of K (once per factorization, on the given stream), and ||K_i||_inf
int launch_kdigits(const ResidualTc& p, int nnzb, int nres, int max_rtiles, int nblk, cudaStream_t st) {
  cudaMemsetAsync(p.Kmax_bits, 0, (size_t)nnzb * sizeof(unsigned long long), st);
  cudaMemsetAsync(p.rowsum, 0, (size_t)p.n * sizeof(float), st);
  kblock_max_kernel<<<dim3((unsigned)nnzb, 8), 256, 0, st>>>(p);
  cudaFuncSetAttribute(kdigits_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KD_SMEM);
  kdigits_kernel<<<dim3((unsigned)nnzb, (unsigned)max_rtiles, (unsigned)(8 * max_rtiles)), 256, KD_SMEM, st>>>(p);
  rowsum_max_kernel<<<nblk, 128, 0, st>>>(p.rowsum, p.xoff_orig, p.m_orig, p.inst, nblk, p.kmax);
  return (int)cudaGetLastError();
}

// number of right-hand-side groups of one residual and their width NR (a multiple of 8, <= 24)
int resid_tc_groups(int nrhs, int* NR) {
  const int ng = (nrhs + NRMAX - 1) / NRMAX;
  const int per = (nrhs + ng - 1) / ng;
  *NR = (per + 7) / 8 * 8;
  return ng;
}

// r = b - K x for the right-hand sides [0, nrhs): the digits of x for every group, then one launch
// with the groups of a row tile as adjacent blocks
int launch_resid_tc(const ResidualTc& p, const ResidTcMaps& maps, const double2* X, const double2* B, double2* R,
                    int nrhs, int nrtiles, int nblk, cudaStream_t st, int64_t* launches) {
  const size_t smem = RT_SMEM + 1024;
  cudaError_t e = cudaFuncSetAttribute(resid_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int NR = 8;
  const int ng = resid_tc_groups(nrhs, &NR);
  CUtensorMap ma, mb;
  std::memcpy(&ma, maps.a, 128);
  std::memcpy(&mb, maps.b[NR / 8 - 1], 128);                     // box rows N = 2 NR = 16 (NR / 8)
  xdigits_kernel<<<dim3((unsigned)nblk, (unsigned)ng), 256, 0, st>>>(p, X, nrhs, NR);
  resid_tc_kernel<<<(unsigned)(nrtiles * ng), RT_THREADS, smem, st>>>(p, ma, mb, X, B, R, nrhs, NR, ng);
  *launches += 2;
  return (int)cudaGetLastError();
}

}  // namespace d3m
