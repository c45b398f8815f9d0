// Persistent block-DAG factorization with a tcgen05 tensor-core tile engine (tile edge 128).
//
// Arithmetic: complex64 factors.  Every product of the factorization (the Schur updates
// S_IJ -= L_IK D_K L_JK^T -- the paper's GEMM tasks, Sec. II -- and the triangular solve
// L_IJ = S_IJ (D_J^{-1} L_JJ^{-1})^T) runs on the 5th-generation tensor cores, in one of two
// engines (template parameter TF):
//  * split-BF16x3: a = a_hi + a_lo with a_hi = bf16(a), a_lo = bf16(a - a_hi); a*b ~ a_hi b_hi +
//    a_hi b_lo + a_lo b_hi, accumulated in FP32 in tensor memory (Henry, Tang, Heinecke,
//    "Leveraging the bfloat16 artificial intelligence datatype for higher-precision
//    computations", ARITH 2019);
//  * TF32: each operand rounded once to tf32 (10-bit mantissa, nearest), one kind::tf32 product,
//    FP32 accumulation; a third of the split products at half the bf16 rate, for a factor
//    accurate to about 2^-11 that the FP64 refinement then corrects.
// Complex products use the real embedding with B stored as two 128-row planes [B_r; B_i]: one
// M=128 x N=256 MMA of A_r over both planes adds [A_r B_r^T | A_r B_i^T] to a 256-column
// accumulator, and two M=128 x N=128 MMAs of A_i add -A_i B_i^T (the instruction's negate-B
// bit) to the real half and A_i B_r^T to the imaginary half: [Re | Im] of A B^T.
//
// Data movement: every finished L tile is written once, by its owner, as operand planes
// (opA: L_IJ; opB: W_IJ = L_IJ D_J, or T_J = D_J^{-1} L_JJ^{-1} for a diagonal tile), row-major
// with the K index contiguous: bf16 [hi_r, hi_i, lo_r, lo_i] / [hi, lo] x [W_r, W_i] (512 rows of
// 256 bytes), or tf32 [r, i] (256 rows of 512 bytes), 128 KB per tile either way; the TF32
// engine also writes bf16 split planes of every off-diagonal L tile (opS) for the solve.  TMA
// tiled loads (64-byte swizzle) stage K chunks of 64-byte rows (32 bf16 or 16 tf32 elements) into
// shared memory for the MMAs.  A paired update task (TF32 engine) stages one A chunk with the B
// chunks of two tiles (I, J) and (I, J + 1) and accumulates them in TMEM columns 0-255 and 256-511.
//
// Roles inside a 256-thread block: warp 0 lane 0 issues TMA loads, warp 1 lane 0 issues MMAs
// (and claims the block's next ready task while they run), all 8 warps run the epilogues (warp w
// reads TMEM lanes 32*(w%4).., columns half w/4), warp 2 releases a finished task's successors.
// Diagonal tiles are factored (unpivoted LDL^T) and inverted with SIMT FP32 in shared memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstring>

#include "device.cuh"
#include "kernels.h"

namespace d3m {

namespace {
constexpr int TB = 128;
constexpr int NTHR = 256;
constexpr uint32_t PLANE = TB * 64;             // 8 KB: one 128-row plane of one chunk (64-byte rows)

// Operand formats of the two engines.  A chunk is 64 bytes of every operand row (the 64-byte
// swizzle span): 32 bf16 or 16 tf32 elements of K.
template <bool TF> struct Eng;
template <> struct Eng<false> {                 // split-BF16x3
  static constexpr int KC = 32;                 // K elements per chunk
  static constexpr int NPA = 4, NPB = 4;        // planes per stage: A [hi_r, hi_i, lo_r, lo_i], B [hi, lo] x [r, i]
  static constexpr int NB = 1;                  // B operands per stage (no paired update tasks)
  static constexpr int NSTAGE = 3;              // GEMM pipeline depth (3 x 64 KB)
  static constexpr uint32_t ROWS = 512;         // operand rows of one tile in global memory
};
template <> struct Eng<true> {                  // TF32
  static constexpr int KC = 16;
  static constexpr int NPA = 2, NPB = 2;        // A [r, i], B [r, i]
  static constexpr int NB = 2;                  // B operands per stage: a paired task's two tiles
  static constexpr int NSTAGE = 4;              // 4 x 48 KB
  static constexpr uint32_t ROWS = 256;
};
template <bool TF> constexpr uint32_t stage_a() { return Eng<TF>::NPA * PLANE; }
template <bool TF> constexpr uint32_t stage_b() { return Eng<TF>::NPB * PLANE; }
template <bool TF> constexpr uint32_t stage_ab() { return stage_a<TF>() + stage_b<TF>(); }
template <bool TF> constexpr uint32_t stage_slot() { return stage_a<TF>() + Eng<TF>::NB * stage_b<TF>(); }
constexpr uint32_t SMEM_S = 0;                  // TRSM A operand: TB / KC chunks of stage_a (128 KB)
constexpr uint32_t SMEM_T = 128 * 1024;         // TRSM B stages (2 x stage_b)
constexpr uint32_t SMEM_BYTES = 192 * 1024;
static_assert(Eng<false>::NSTAGE * stage_slot<false>() <= SMEM_BYTES && SMEM_T + 2 * stage_b<false>() <= SMEM_BYTES, "smem");
static_assert(Eng<true>::NSTAGE * stage_slot<true>() <= SMEM_BYTES && SMEM_T + 2 * stage_b<true>() <= SMEM_BYTES, "smem");
static_assert((TB / Eng<false>::KC) * stage_a<false>() == SMEM_T && (TB / Eng<true>::KC) * stage_a<true>() == SMEM_T, "S");
constexpr int LDS = 129;                        // c64 diagonal tile row stride (elements)
constexpr uint32_t DIAG_AUX = 130 * 1024;       // d / column / scratch vectors of a diagonal task
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC1 = 0, ACC2 = 256;        // TMEM columns of the two accumulators

// instruction descriptors: D f32 (bits 4-5 = 1), A and B format (bits 7-9, 10-12: 1 = bf16 for
// kind::f16, 2 = tf32 for kind::tf32), both K-major, N >> 3 at bit 17, M >> 4 at bit 24 (M = 128,
// N = 256 or 128); bit 14 negates B
template <bool TF> constexpr uint32_t idesc(uint32_t n) {
  return (1u << 4) | ((TF ? 2u : 1u) << 7) | ((TF ? 2u : 1u) << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the deadline passed (the caller records a timeout).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t deadline) {
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() > deadline) return false;
  }
  return true;
}

// ------------------------------------------------------------------ TMA
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_prefetch_desc(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

// ------------------------------------------------------------------ tcgen05
// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512u >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)4 << 61;                 // 64-byte swizzle
  return d;
}
template <bool TF>
__device__ __forceinline__ void mma_tc(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accum, uint32_t idsc) {
  if constexpr (TF) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idsc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idsc), "r"(accum)
        : "memory");
  }
}
// [Re | Im] += A B^T for one operand pair: A planes a_r, a_i; B planes b (B_r) and b + PLANE (B_i)
// (accum = 0 on the very first product: the N = 256 MMA initialises every column)
template <bool TF>
__device__ __forceinline__ void cmma(uint32_t d, uint32_t a_r, uint32_t a_i, uint32_t b, uint32_t accum) {
  mma_tc<TF>(d, desc_sw64(a_r), desc_sw64(b), accum, idesc<TF>(256));                          // [A_r B_r | A_r B_i]
  mma_tc<TF>(d, desc_sw64(a_i), desc_sw64(b + PLANE), 1u, idesc<TF>(128) | (1u << 14));        // Re -= A_i B_i
  mma_tc<TF>(d + 128, desc_sw64(a_i), desc_sw64(b), 1u, idesc<TF>(128));                       // Im += A_i B_r
}
// All products of one staged chunk (64-byte rows; two MMA K-steps of 32 bytes each): A planes at
// a (stage layout of the engine), B planes at b.  first: the chunk starts the accumulation.
template <bool TF>
__device__ __forceinline__ void chunk_mma(uint32_t d, uint32_t a, uint32_t b, bool first) {
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const uint32_t ko = kk * 32;
    const uint32_t acc = (first && kk == 0) ? 0u : 1u;
    if constexpr (TF) {
      cmma<true>(d, a + ko, a + PLANE + ko, b + ko, acc);
    } else {
      const uint32_t a_hr = a + 0 * PLANE + ko, a_hi = a + 1 * PLANE + ko;
      const uint32_t a_lr = a + 2 * PLANE + ko, a_li = a + 3 * PLANE + ko;
      const uint32_t bh = b + ko, bl = b + 2 * PLANE + ko;
      // lo*hi and hi*lo first, then hi*hi
      cmma<false>(d, a_lr, a_li, bh, acc);
      cmma<false>(d, a_hr, a_hi, bl, 1u);
      cmma<false>(d, a_hr, a_hi, bh, 1u);
    }
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ------------------------------------------------------------------ bf16 split helpers
__device__ __forceinline__ void split2(float a, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(a);
  lo = __float2bfloat16_rn(a - __bfloat162float(hi));
}
// 8 values -> one 16-byte word of bf16 (hi or lo part)
__device__ __forceinline__ uint4 pack8(const __nv_bfloat16* v) {
  uint4 u;
  u.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
  u.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
  u.z = (uint32_t)__bfloat16_as_ushort(v[4]) | ((uint32_t)__bfloat16_as_ushort(v[5]) << 16);
  u.w = (uint32_t)__bfloat16_as_ushort(v[6]) | ((uint32_t)__bfloat16_as_ushort(v[7]) << 16);
  return u;
}

// Round to tf32 (nearest, ties away; the low 13 bits of the result are zero).
__device__ __forceinline__ uint32_t tf32_rn(float a) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(a));
  return u;
}
__device__ __forceinline__ uint4 pack4_tf32(const float* v) {
  return make_uint4(tf32_rn(v[0]), tf32_rn(v[1]), tf32_rn(v[2]), tf32_rn(v[3]));
}
// Write 16 K values of row r into a shared-memory K-major SW64 plane (one tf32 chunk).
__device__ __forceinline__ void store_smem_plane16_tf32(unsigned char* plane, int r, const float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t off = (uint32_t)r * 64u + ((uint32_t)(q ^ ((r >> 1) & 3)) << 4);
    *reinterpret_cast<uint4*>(plane + off) = pack4_tf32(v + 4 * q);
  }
}

// Write 32 K values of row r into a shared-memory K-major SW64 plane (one chunk) as hi/lo.
__device__ __forceinline__ void store_smem_plane32(unsigned char* plane_hi, unsigned char* plane_lo, int r,
                                                   const float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) split2(v[q * 8 + e], h[e], l[e]);
    const uint32_t off = (uint32_t)r * 64u + ((uint32_t)(q ^ ((r >> 1) & 3)) << 4);
    *reinterpret_cast<uint4*>(plane_hi + off) = pack8(h);
    *reinterpret_cast<uint4*>(plane_lo + off) = pack8(l);
  }
}

// Accumulator tile layout (TMEM-native): element (r, c) of the 128 x 128 complex tile is float2
// ((chunk * 16 + q) * 128 + r) * 2 + (c & 1) with chunk = c / 32, q = (c % 32) / 2, so the row-per-
// thread epilogue reads and writes 16-byte words that are contiguous across the 128 rows.
__device__ __forceinline__ float4* acc_slot(float2* Sa, int r, int c0) {
  return reinterpret_cast<float4*>(Sa) + (int64_t)(c0 >> 5) * 16 * TB + r;   // + q * TB
}

// 32 consecutive entries (row r, columns c0..c0+31) of the update's starting value: the tile's
// accumulator (Sa != nullptr) or K_IJ.  All loads are issued before any use.
__device__ __forceinline__ void load_s_in(const TileTask& T, const double2* K, float2* Sa, int r, int c0,
                                          float2* kin) {
  if (Sa) {
    const float4* s4 = acc_slot(Sa, r, c0);
    float4 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = ld_cg4(s4 + i * TB);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      kin[2 * i] = make_float2(v[i].x, v[i].y);
      kin[2 * i + 1] = make_float2(v[i].z, v[i].w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) kin[i] = k_entry<float>(T, K, r, c0 + i);
  }
}


// ---------------------------------------------------------------- diagonal tile: blocked LDL^T
// The diagonal tile S (128 x 128, complex symmetric, lower triangle in sS) is factored as
// S = L D L^T (unpivoted) and L is inverted, X = L^{-1}, in four panels of DW = 32 columns
// (right-looking on both).  Storage: sS holds L strictly below the diagonal and X transposed
// strictly above it (sS[c][r] = X[r][c]); d goes to s_d.  With block indices r, s, j and the
// current panel k:
//   diagonal block:  A_kk = L_kk D_k L_kk^T, X_kk = L_kk^{-1}           (two warps, registers)
//   panel below:     W_rk = A_rk X_kk^T (= L_rk D_k), L_rk = W_rk D_k^{-1}
//   trailing:        A_rs -= L_rk W_sk^T                                (r >= s > k)
//   inverse:         Z_rj += L_rk X_kj (r > k, j <= k);  X_rj = -X_rr Z_rj once X_rr exists
// (X_rj = -X_rr sum_{k=j}^{r-1} L_rk X_kj is the block form of L X = I).  Z_rj lives where X_rj
// ends up, in the upper triangle, which starts at zero.  The diagonal block of panel k + 1 is
// updated first, so that two warps factor it while the other six finish panel k's updates.
constexpr int DW = 32;          // panel width
constexpr int WT_LD = 96;       // row length of the W panel scratch (c-major: Wt[c][row - c1])
constexpr int XD_LD = DW + 1;   // row length of the dense copies of X_kk (two, by panel parity)

// The DW x DW diagonal block at (c0, c0), two warps: warp 0 factors it (lane i = row i), warp 1
// inverts L (lane j = column j of X) one phase of 8 columns behind, the two meeting at named
// barrier 1 after every phase.  Registers are shifted as the elimination advances (slot m holds
// column / row j + m at step j) so that all register indices are static and the loops stay
// rolled (straight-line code of this size would run out of the instruction cache).
template <int NM>
__device__ __forceinline__ void ldlt_phase(float2 (&a)[DW], int j0, float2* sS, float2* s_d, float2* colb, int c0,
                                           int lane) {
#pragma unroll 1
  for (int j = j0; j < j0 + 8; ++j) {
    // d_j = a_j[j]; l_i = a_i[j] / d_j; a_i[m] -= l_i a_m[j] for m > j.  Lanes m > j are the only
    // sources of a_m[j], so the unused entries above a lane's diagonal never reach a result.  The
    // column goes through a shared buffer (one broadcast load per entry), two buffers by step parity.
    const float2 cj = a[0];
    float2* cb = colb + (j & 1) * DW;
    cb[lane] = cj;
    __syncwarp();
    const float2 dj = cb[j];
    const float2 l = cdiv(cj, dj);
#pragma unroll
    for (int m = 1; m < NM; ++m) a[m - 1] = cfms(l, cb[(j + m) & 31], a[m]);
    a[NM - 1] = make_float2(0.f, 0.f);
    if (lane > j) sS[(c0 + lane) * LDS + c0 + j] = l;
    if (lane == j) s_d[c0 + j] = dj;
  }
}

template <int NM>
__device__ __forceinline__ void linv_phase(float2 (&x)[DW], int q0, float2* sS, float2* Xd, int c0, int lane) {
#pragma unroll 1
  for (int q = q0; q < q0 + 8; ++q) {
    // x holds rows q.. of column `lane` of X: X[q][lane] is final; X[m][lane] -= L[m][q] X[q][lane]
    const float2 xq = x[0];
    if (q > lane) sS[(c0 + lane) * LDS + c0 + q] = xq;      // X[q][lane] at sS[c0 + lane][c0 + q]
    Xd[q * XD_LD + lane] = xq;                               // dense copy, zeros and ones included
#pragma unroll
    for (int m = 1; m < NM; ++m) {
      const int row = min(q + m, DW - 1);                    // rows past the block feed unused slots
      x[m - 1] = cfms(sS[(c0 + row) * LDS + c0 + q], xq, x[m]);
    }
    x[NM - 1] = make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ void diag_block_2warps(float2* sS, float2* s_d, float2* Xd, int c0, int warp, int lane) {
  float2* colb = s_d + TB + DW * WT_LD + 2 * DW * XD_LD;   // [2][DW] column buffers of warp 0
  float2 v[DW];
  if (warp == 0) {
#pragma unroll
    for (int m = 0; m < DW; ++m) v[m] = (m <= lane) ? sS[(c0 + lane) * LDS + c0 + m] : make_float2(0.f, 0.f);
    ldlt_phase<32>(v, 0, sS, s_d, colb, c0, lane);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    ldlt_phase<24>(v, 8, sS, s_d, colb, c0, lane);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    ldlt_phase<16>(v, 16, sS, s_d, colb, c0, lane);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    ldlt_phase<8>(v, 24, sS, s_d, colb, c0, lane);
    asm volatile("bar.sync 1, 64;" ::: "memory");
  } else {
#pragma unroll
    for (int m = 0; m < DW; ++m) v[m] = make_float2(m == lane ? 1.f : 0.f, 0.f);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    linv_phase<32>(v, 0, sS, Xd, c0, lane);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    linv_phase<24>(v, 8, sS, Xd, c0, lane);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    linv_phase<16>(v, 16, sS, Xd, c0, lane);
    asm volatile("bar.sync 1, 64;" ::: "memory");
    linv_phase<8>(v, 24, sS, Xd, c0, lane);
  }
}


// All threads: W_rk, L_rk for the rows below panel k (k < 3) and X_kj = -X_kk Z_kj (j < k).
__device__ __forceinline__ void diag_panel_solve(float2* sS, const float2* s_d, float2* Wt, const float2* Xd, int k,
                                                 int tid) {
  const int c0 = DW * k, c1 = c0 + DW, nrb = 3 - k;
  // W: thread -> columns cg + 8 jj, rows c1 + rg + 32 ii
  const int cg = tid & 7, rg = tid >> 3;
  float2 w[3][4];
#pragma unroll
  for (int ii = 0; ii < 3; ++ii)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) w[ii][jj] = make_float2(0.f, 0.f);
  if (nrb > 0) {
#pragma unroll 4
    for (int q = 0; q < DW; ++q) {
      float2 xq[4], aq[3];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) xq[jj] = Xd[(cg + 8 * jj) * XD_LD + q];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) aq[ii] = ii < nrb ? sS[(c1 + rg + 32 * ii) * LDS + c0 + q] : make_float2(0.f, 0.f);
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) w[ii][jj] = cfma(aq[ii], xq[jj], w[ii][jj]);
    }
  }
  // X_kj: thread -> rows a = (tid >> 5) + 8 i, column b = tid & 31
  const int b = tid & 31, ar = tid >> 5;
  float2 xo[3][4];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) xo[j][i] = make_float2(0.f, 0.f);
  if (k > 0) {
#pragma unroll 4
    for (int q = 0; q < DW; ++q) {
      float2 xa[4], z[3];
#pragma unroll
      for (int i = 0; i < 4; ++i) xa[i] = Xd[(ar + 8 * i) * XD_LD + q];
#pragma unroll
      for (int j = 0; j < 3; ++j) z[j] = j < k ? sS[(DW * j + b) * LDS + c0 + q] : make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) xo[j][i] = cfma(xa[i], z[j], xo[j][i]);
    }
  }
  __syncthreads();   // every A_rk and Z_kj has been read
  if (nrb > 0) {
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int c = cg + 8 * jj;
      const float2 dinv = cdiv(make_float2(1.f, 0.f), s_d[c0 + c]);
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
        if (ii < nrb) {
          sS[(c1 + rg + 32 * ii) * LDS + c0 + c] = cmul(w[ii][jj], dinv);
          Wt[c * WT_LD + rg + 32 * ii] = w[ii][jj];
        }
    }
  }
#pragma unroll
  for (int j = 0; j < 3; ++j)
    if (j < k)
#pragma unroll
      for (int i = 0; i < 4; ++i) sS[(DW * j + b) * LDS + c0 + ar + 8 * i] = make_float2(-xo[j][i].x, -xo[j][i].y);
  __syncthreads();
}

// All threads: A_{k+1,k+1} -= L_{k+1,k} W_{k+1,k}^T (lower triangle).
__device__ __forceinline__ void diag_next_block(float2* sS, const float2* Wt, int k, int tid) {
  const int c0 = DW * k, c1 = c0 + DW;
  const int b = tid & 31, ar = tid >> 5;
  float2 acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int c = 0; c < DW; ++c) {
    const float2 wv = Wt[c * WT_LD + b];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = cfma(sS[(c1 + ar + 8 * i) * LDS + c0 + c], wv, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = ar + 8 * i;
    if (b <= a) {
      float2* o = sS + (c1 + a) * LDS + c1 + b;
      *o = csub(*o, acc[i]);
    }
  }
}

// Warps 2..7 (t = thread index among them): the rest of panel k's updates as 32 x 32 block jobs --
// trailing blocks (r, s), k < s <= r, other than (k+1, k+1), then Z blocks (r, j), r > k, j <= k.
// A job is two chunks of 32 threads; each thread owns rows aa + 8 i and columns bb + 8 q (i, q < 4).
__device__ __forceinline__ void diag_panel_update(float2* sS, const float2* Wt, const float2* Xd, int k, int t) {
  const int c0 = DW * k, c1 = c0 + DW;
  const int nT = (3 - k) * (4 - k) / 2 - 1, nZ = (3 - k) * (k + 1);
  const int nchunks = 2 * (nT + nZ);
  const int wi = t >> 5, lane = t & 31;
#pragma unroll 1
  for (int ch = wi; ch < nchunks; ch += 6) {
    const int job = ch >> 1;
    const int aa = (ch & 1) * 4 + (lane >> 3), bb = lane & 7;
    int rb, sb = 0, j = 0;
    const bool trailing = job < nT;
    if (trailing) {
      int e = job + 1;            // skip (k+1, k+1), the first pair in this order
      sb = k + 1;
      rb = k + 1;
      while (e > 0) {
        if (++rb > 3) { ++sb; rb = sb; }
        --e;
      }
    } else {
      const int e = job - nT;
      rb = k + 1 + e / (k + 1);
      j = e % (k + 1);
    }
    const float2* P0 = sS + (DW * rb + aa) * LDS + c0;
    float2 acc[4][4];
#pragma unroll
    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[ii][q] = make_float2(0.f, 0.f);
    // Q[c][b]: W_sk (trailing), X_kj from the upper triangle (j < k) or the dense X_kk (j = k)
    const float2* Q;
    int qs_c, qs_b;
    if (trailing) {
      Q = Wt + DW * sb - c1 + bb;
      qs_c = WT_LD;
      qs_b = 1;
    } else if (j < k) {
      Q = sS + (DW * j + bb) * LDS + c0;
      qs_c = 1;
      qs_b = LDS;
    } else {
      Q = Xd + bb;
      qs_c = XD_LD;
      qs_b = 1;
    }
#pragma unroll 2
    for (int c = 0; c < DW; ++c) {
      float2 pv[4], qv[4];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) pv[ii] = P0[8 * ii * LDS + c];
#pragma unroll
      for (int q = 0; q < 4; ++q) qv[q] = Q[c * qs_c + 8 * q * qs_b];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[ii][q] = cfma(pv[ii], qv[q], acc[ii][q]);
    }
    if (trailing) {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int a = aa + 8 * ii, b = bb + 8 * q;
          if (rb != sb || b <= a) {
            float2* o = sS + (DW * rb + a) * LDS + DW * sb + b;
            *o = csub(*o, acc[ii][q]);
          }
        }
    } else {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float2* o = sS + (DW * j + bb + 8 * q) * LDS + DW * rb + aa + 8 * ii;
          *o = make_float2(o->x + acc[ii][q].x, o->y + acc[ii][q].y);
        }
    }
  }
}

}  // namespace

template <bool TF>
__global__ void __launch_bounds__(NTHR, 1)
    factor_tc_kernel(const FactorParams p, const __grid_constant__ CUtensorMap mapA,
                     const __grid_constant__ CUtensorMap mapB) {
  constexpr int KC = Eng<TF>::KC, NSTAGE = Eng<TF>::NSTAGE, NCH = TB / KC;
  constexpr uint32_t STAGE_A = stage_a<TF>(), STAGE_B = stage_b<TF>(), STAGE = stage_ab<TF>();
  constexpr uint32_t SLOT = stage_slot<TF>();    // bytes between pipeline stages
  constexpr uint32_t ROWS = Eng<TF>::ROWS;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the dynamic region (swizzle atoms); pointer arithmetic on the shared
  // array keeps the accesses in the shared address space
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_tfull[2], bar_tempty[2], bar_acc, bar_acc2;
  __shared__ uint32_t s_tmem;
  __shared__ int s_task, s_pending;
  __shared__ int s_next[2];                      // task claimed ahead, by task parity (-1: none)
  if (threadIdx.x == 0) s_pending = -1;          // read and written by thread 0 only
  __shared__ float s_red[NTHR / 32];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float2* Lg = reinterpret_cast<float2*>(p.L);
  float2* Linv = reinterpret_cast<float2*>(p.Linv);
  float2* Dg = reinterpret_cast<float2*>(p.D);
  float2* Sacc = reinterpret_cast<float2*>(p.Sacc);
  unsigned char* opA = reinterpret_cast<unsigned char*>(p.opA);
  unsigned char* opB = reinterpret_cast<unsigned char*>(p.opB);

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&bar_tfull[s]), 1);
      mbar_init(smem_u32(&bar_tempty[s]), 1);
    }
    mbar_init(smem_u32(&bar_acc), 1);
    mbar_init(smem_u32(&bar_acc2), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    tma_prefetch_desc(&mapA);
    tma_prefetch_desc(&mapB);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  // pipeline counters (each kept by the thread that uses it)
  uint32_t g_load = 0, g_mma = 0, t_load = 0, t_mma = 0;
  uint32_t n_acc = 0, n_acc2 = 0;
  bool failed = false;

  // The MMA-issuing lane claims the block's next normal-lane task while the products of an
  // update or triangular-solve task run (sched_claim_normal), and warp 2 releases a finished
  // task's successors while warps 0 and 1 already issue the next task's loads and products, so
  // neither the queue round trips nor the release sit between two tasks.
  int tcount = 0;                    // tasks this block has run (parity selects s_next)
  int task = sched_pop(p, &s_task, &s_pending);
  while (task >= 0) {
    const TileTask T = p.tasks[task];
    if (tid == 32) s_next[tcount & 1] = -1;
    const uint64_t deadline = globaltimer_ns() + (uint64_t)p.timeout_ns;
    const int nchunk = T.nk * NCH;
    asm volatile("fence.proxy.async.global;" ::: "memory");
    // the tile's starting value (its accumulator, or K_IJ: up to 128 contiguous spans) is read
    // after the products; warps 2..5 prefetch it into L2 while they run
    if (warp >= 2 && warp < 6) {
      const int sp = tid - 64;
      if (T.flags & TF_S_IN) {
        if (sp < 8 && T.sidx >= 0)
          bulk_prefetch_l2(Sacc + (int64_t)T.sidx * TB * TB + sp * (TB * TB / 8), (uint32_t)(TB * TB / 8 * sizeof(float2)));
      } else if (T.k_off >= 0 && sp < (T.k_tr ? T.rv : T.cv)) {
        const int64_t base = T.k_tr ? (int64_t)(T.r0 + sp) * T.k_ld + T.c0 : (int64_t)(T.c0 + sp) * T.k_ld + T.r0;
        bulk_prefetch_l2(p.K + T.k_off + base, (uint32_t)((T.k_tr ? T.cv : T.rv) * sizeof(double2)));
      }
    }
    const bool pair = TF && (T.flags & TF_PAIR) != 0;   // a second tile (I, J + 1) shares the A operand
    if (pair && warp >= 6) {
      // the same for the second tile: its accumulator, or the spans of K_{I,J+1}
      const int sp = tid - 192;
      if (T.flags & TF_S_IN) {
        if (sp < 8 && T.sidx2 >= 0)
          bulk_prefetch_l2(Sacc + (int64_t)T.sidx2 * TB * TB + sp * (TB * TB / 8), (uint32_t)(TB * TB / 8 * sizeof(float2)));
      } else if (T.k_off >= 0) {
        for (int q = sp; q < (T.k_tr ? T.rv : T.cv2); q += 64) {
          const int64_t base = T.k_tr ? (int64_t)(T.r0 + q) * T.k_ld + T.c0_2 : (int64_t)(T.c0_2 + q) * T.k_ld + T.r0;
          bulk_prefetch_l2(p.K + T.k_off + base, (uint32_t)((T.k_tr ? T.cv2 : T.rv) * sizeof(double2)));
        }
      }
    }

    // ---------------------------------------------------------------- phase 1: Schur GEMM
    if (nchunk > 0) {
      if (warp == 0) {
        if (lane == 0) {
          for (int c = 0; c < nchunk && !failed; ++c) {
            const uint32_t s = g_load % NSTAGE, use = g_load / NSTAGE;
            if (!mbar_wait(smem_u32(&bar_empty[s]), (use & 1) ^ 1, deadline)) { failed = true; break; }
            const KEntry ke = p.klist[T.kl_off + c / NCH];
            const int x = (c % NCH) * KC;
            const uint32_t sb = smem_u32(smem + s * SLOT);
            const uint32_t fb = smem_u32(&bar_full[s]);
            mbar_expect_tx(fb, pair ? STAGE + STAGE_B : STAGE);
#pragma unroll
            for (int q = 0; q < Eng<TF>::NPA; ++q)
              tma_load_2d(sb + q * PLANE, &mapA, x, ke.a_tile * (int)ROWS + q * 128, fb);
#pragma unroll
            for (int q = 0; q < Eng<TF>::NPB; ++q)
              tma_load_2d(sb + STAGE_A + q * PLANE, &mapB, x, ke.b_tile * (int)ROWS + q * 128, fb);
            if (pair) {
#pragma unroll
              for (int q = 0; q < Eng<TF>::NPB; ++q)
                tma_load_2d(sb + STAGE + q * PLANE, &mapB, x, ke.b2_tile * (int)ROWS + q * 128, fb);
            }
            ++g_load;
          }
        }
        __syncwarp();
      } else if (warp == 1) {
        if (lane == 0) {
          for (int c = 0; c < nchunk && !failed; ++c) {
            const uint32_t s = g_mma % NSTAGE, use = g_mma / NSTAGE;
            if (!mbar_wait(smem_u32(&bar_full[s]), use & 1, deadline)) { failed = true; break; }
            tc_fence_after();
            const uint32_t sb = smem_u32(smem + s * SLOT);
            chunk_mma<TF>(tmem + ACC1, sb, sb + STAGE_A, c == 0);
            if (pair) chunk_mma<TF>(tmem + ACC2, sb, sb + STAGE, c == 0);
            mma_commit(smem_u32(&bar_empty[s]));
            ++g_mma;
          }
          mma_commit(smem_u32(&bar_acc));
          if (T.flags & TF_UPDATE) s_next[tcount & 1] = sched_claim_normal(p, &s_pending);
        }
        __syncwarp();
      }
      if (!mbar_wait(smem_u32(&bar_acc), n_acc & 1, deadline)) failed = true;
      ++n_acc;
      tc_fence_after();
    }
    if (__syncthreads_or(failed)) {
      if (tid == 0) set_error(p.ctl, D3M_ERR_TIMEOUT, task);
      break;
    }
    trace_mark(p, task, 0);

    const bool is_diag = (T.flags & TF_DIAG) != 0;
    const bool s_in = (T.flags & TF_S_IN) != 0;
    float2* Sa = (T.sidx >= 0) ? Sacc + (int64_t)T.sidx * TB * TB : nullptr;
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane;
    if (T.flags & TF_UPDATE) {
      // ------------------------------------------------------------ partial update task
      // (a paired task: the second tile from the accumulator at ACC2, with its own columns)
      if (!s_in) wait_k_block(p, T.kseq, task, deadline);
      for (int u = 0; u < (pair ? 2 : 1); ++u) {
        TileTask Tu = T;
        if (u) {
          Tu.tile = T.tile2;
          Tu.c0 = T.c0_2;
          Tu.cv = T.cv2;
          Tu.sidx = T.sidx2;
        }
        float2* Su = (Tu.sidx >= 0) ? Sacc + (int64_t)Tu.sidx * TB * TB : nullptr;
        const uint32_t acc = u ? ACC2 : ACC1;
        for (int pass = 0; pass < 2; ++pass) {
          const int c0 = half * 64 + pass * 32;
          float vr[32], vi[32];
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + acc + c0, vr);
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + acc + 128 + c0, vi);
          float4* slot = acc_slot(Su, r, c0);
          float2 kin[32];
          load_s_in(Tu, p.K, s_in ? Su : nullptr, r, c0, kin);   // all loads first
#pragma unroll
          for (int i = 0; i < 32; i += 2)
            slot[(i / 2) * TB] = make_float4(kin[i].x - vr[i], kin[i].y - vi[i], kin[i + 1].x - vr[i + 1], kin[i + 1].y - vi[i + 1]);
        }
      }
    } else {
      // ------------------------------------------------------------ final task
      if (!s_in) wait_k_block(p, T.kseq, task, deadline);
      // off-diagonal: prefetch the first two chunks of T_J (B operand of the TRSM product)
      if (!is_diag && tid == 0) {
        for (int c = 0; c < 2; ++c) {
          const uint32_t s = t_load & 1, use = t_load >> 1;
          if (!mbar_wait(smem_u32(&bar_tempty[s]), (use & 1) ^ 1, deadline)) { failed = true; break; }
          const uint32_t sb = smem_u32(smem + SMEM_T + s * STAGE_B);
          const uint32_t fb = smem_u32(&bar_tfull[s]);
          mbar_expect_tx(fb, STAGE_B);
#pragma unroll
          for (int q = 0; q < Eng<TF>::NPB; ++q)
            tma_load_2d(sb + q * PLANE, &mapB, c * KC, T.diag * (int)ROWS + q * 128, fb);
          ++t_load;
        }
      }

      // ---------------------------------------------------------------- phase 2: S = S_in - acc
      if (is_diag) {
        float2* sS = reinterpret_cast<float2*>(smem);   // [128][129]
        float2* s_d = reinterpret_cast<float2*>(smem + DIAG_AUX);
        for (int pass = 0; pass < 2; ++pass) {
          const int c0 = half * 64 + pass * 32;
          float vr[32], vi[32];
          if (nchunk > 0) {
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ACC1 + c0, vr);
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ACC1 + 128 + c0, vi);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) vr[i] = vi[i] = 0.f;
          }
          float2 kin[32];
          load_s_in(T, p.K, s_in ? Sa : nullptr, r, c0, kin);
#pragma unroll
          for (int i = 0; i < 32; ++i) sS[r * LDS + c0 + i] = make_float2(kin[i].x - vr[i], kin[i].y - vi[i]);
        }
        tc_fence_before();
        __syncthreads();
        trace_mark(p, task, 1);
        // max |S| over the real lower triangle (breakdown scale)
        float mx = 0.f;
        for (int i = tid; i < TB * TB; i += NTHR) {
          const int rr = i >> 7, cc = i & 127;
          if (cc <= rr && rr < T.rv) mx = fmaxf(mx, sqrtf(cabs2(sS[rr * LDS + cc])));
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_red[warp] = mx;
        __syncthreads();
        // Unpivoted LDL^T and X = L^{-1}, blocked in panels of DW columns (the diag_* functions)
        {
          // the upper triangle starts at zero (it accumulates the blocks of X)
          for (int i = tid; i < TB * TB; i += NTHR) {
            const int rr = i >> 7, cc = i & 127;
            if (cc > rr) sS[rr * LDS + cc] = make_float2(0.f, 0.f);
          }
          float2* Wt = s_d + TB;
          float2* Xd = Wt + DW * WT_LD;                 // [2][DW][XD_LD]
          __syncthreads();
          if (warp < 2) diag_block_2warps(sS, s_d, Xd, 0, warp, lane);
          __syncthreads();
#pragma unroll 1
          for (int k = 0; k < TB / DW; ++k) {
            float2* Xk = Xd + (k & 1) * DW * XD_LD;
            diag_panel_solve(sS, s_d, Wt, Xk, k, tid);
            if (k == TB / DW - 1) break;
            diag_next_block(sS, Wt, k, tid);
            __syncthreads();
            if (warp < 2) diag_block_2warps(sS, s_d, Xd + ((k + 1) & 1) * DW * XD_LD, DW * (k + 1), warp, lane);
            else diag_panel_update(sS, Wt, Xk, k, tid - 64);
            __syncthreads();
          }
          // D_J (L_JJ and L_JJ^{-1} in complex64 are written after the release, below)
          if (tid < TB) Dg[(int64_t)T.col * TB + tid] = s_d[tid];
        }
        trace_mark(p, task, 2);
        if (tid < 32) {
          float smax = 0.f;
          for (int w = 0; w < NTHR / 32; ++w) smax = fmaxf(smax, s_red[w]);
          float amin = 3.0e38f, amax = 0.f;
          for (int c = tid; c < T.cv; c += 32) {
            const float a = sqrtf(cabs2(s_d[c]));
            amin = fminf(amin, a);
            amax = fmaxf(amax, a);
          }
          for (int o = 16; o > 0; o >>= 1) {
            amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, o));
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
          }
          if (tid == 0) {
            record_pivot_stats(p.ctl, amin, amax);
            if (!(amin >= (float)p.piv_tol * smax)) set_error(p.ctl, D3M_ERR_PIVOT, task);
          }
        }
        // T_J = D^{-1} Linv as B planes
        {
          // T_J = D^{-1} L^{-1}: row n, columns k (X[n][k] = sS[k][n] for k < n); coalesced 16-byte
          // stores of the planes: bf16 [T_r, T_i] x [hi, lo] (16 threads per 256-byte plane row) or
          // tf32 [T_r, T_i] (32 threads per 512-byte plane row)
          uint4* Bt = reinterpret_cast<uint4*>(opB + (int64_t)T.tile * ROWS * TB * (TF ? 4 : 2));
          for (int it = tid; it < TB * 16; it += NTHR) {
            const int n = it >> 4, c8 = it & 15;
            const float2 dinv = cdiv(make_float2(1.f, 0.f), s_d[n]);
            float tr[8], ti[8];
#pragma unroll
            for (int k8 = 0; k8 < 8; ++k8) {
              const int k = c8 * 8 + k8;
              const float2 lv = (k < n) ? sS[k * LDS + n] : make_float2(k == n ? 1.f : 0.f, 0.f);
              const float2 tv = cmul(dinv, lv);
              tr[k8] = tv.x;
              ti[k8] = tv.y;
            }
            if constexpr (TF) {
              Bt[(0 * 128 + n) * 32 + 2 * c8] = pack4_tf32(tr);
              Bt[(0 * 128 + n) * 32 + 2 * c8 + 1] = pack4_tf32(tr + 4);
              Bt[(1 * 128 + n) * 32 + 2 * c8] = pack4_tf32(ti);
              Bt[(1 * 128 + n) * 32 + 2 * c8 + 1] = pack4_tf32(ti + 4);
            } else {
              __nv_bfloat16 h[2][8], lo[2][8];
#pragma unroll
              for (int k8 = 0; k8 < 8; ++k8) {
                split2(tr[k8], h[0][k8], lo[0][k8]);
                split2(ti[k8], h[1][k8], lo[1][k8]);
              }
#pragma unroll
              for (int pl = 0; pl < 2; ++pl) {
                Bt[((0 * 256 + pl * 128) + n) * 16 + c8] = pack8(h[pl]);
                Bt[((1 * 256 + pl * 128) + n) * 16 + c8] = pack8(lo[pl]);
              }
            }
          }
        }
        __syncthreads();
        trace_mark(p, task, 3);
      } else {
        // S planes for the TRSM product (A operand, SW64 K-major, 4 chunks)
        for (int pass = 0; pass < 2; ++pass) {
          const int c0 = half * 64 + pass * 32;
          float vr[32], vi[32];
          if (nchunk > 0) {
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ACC1 + c0, vr);
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ACC1 + 128 + c0, vi);
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) vr[i] = vi[i] = 0.f;
          }
          {
            float2 kin[32];
            load_s_in(T, p.K, s_in ? Sa : nullptr, r, c0, kin);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              vr[i] = kin[i].x - vr[i];
              vi[i] = kin[i].y - vi[i];
            }
          }
          if constexpr (TF) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              unsigned char* ch = smem + SMEM_S + (c0 / KC + hh) * STAGE_A;
              store_smem_plane16_tf32(ch + 0 * PLANE, r, vr + 16 * hh);
              store_smem_plane16_tf32(ch + 1 * PLANE, r, vi + 16 * hh);
            }
          } else {
            unsigned char* ch = smem + SMEM_S + (c0 / KC) * STAGE_A;
            store_smem_plane32(ch + 0 * PLANE, ch + 2 * PLANE, r, vr);
            store_smem_plane32(ch + 1 * PLANE, ch + 3 * PLANE, r, vi);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        trace_mark(p, task, 1);
        // ---------------------------------------------------------------- phase 3: TRSM product
        if (warp == 0) {
          if (lane == 0) {
            for (int c = 2; c < NCH && !failed; ++c) {
              const uint32_t s = t_load & 1, use = t_load >> 1;
              if (!mbar_wait(smem_u32(&bar_tempty[s]), (use & 1) ^ 1, deadline)) { failed = true; break; }
              const uint32_t sb = smem_u32(smem + SMEM_T + s * STAGE_B);
              const uint32_t fb = smem_u32(&bar_tfull[s]);
              mbar_expect_tx(fb, STAGE_B);
#pragma unroll
              for (int q = 0; q < Eng<TF>::NPB; ++q)
                tma_load_2d(sb + q * PLANE, &mapB, c * KC, T.diag * (int)ROWS + q * 128, fb);
              ++t_load;
            }
          }
          __syncwarp();
        } else if (warp == 1) {
          if (lane == 0) {
            tc_fence_after();
            for (int c = 0; c < NCH && !failed; ++c) {
              const uint32_t s = t_mma & 1, use = t_mma >> 1;
              if (!mbar_wait(smem_u32(&bar_tfull[s]), use & 1, deadline)) { failed = true; break; }
              tc_fence_after();
              const uint32_t ab = smem_u32(smem + SMEM_S + c * STAGE_A);
              const uint32_t tb = smem_u32(smem + SMEM_T + s * STAGE_B);
              chunk_mma<TF>(tmem + ACC2, ab, tb, c == 0);
              mma_commit(smem_u32(&bar_tempty[s]));
              ++t_mma;
            }
            mma_commit(smem_u32(&bar_acc2));
            s_next[tcount & 1] = sched_claim_normal(p, &s_pending);
          }
          __syncwarp();
        }
        if (!mbar_wait(smem_u32(&bar_acc2), n_acc2 & 1, deadline)) failed = true;
        ++n_acc2;
        tc_fence_after();
        if (__syncthreads_or(failed)) {
          if (tid == 0) set_error(p.ctl, D3M_ERR_TIMEOUT, task);
          break;
        }
        trace_mark(p, task, 2);
        // D_J into the (now idle) TRSM stage area; L_IJ (c64) staged row-major in [0, 128K) with the
        // 16-byte units of each 128-byte span XOR-swizzled by the row (conflict-free row writes)
        float2* s_d = reinterpret_cast<float2*>(smem + SMEM_T);
        if (tid < TB) s_d[tid] = ld_cg(Dg + (int64_t)T.col * TB + tid);
        float4* stg = reinterpret_cast<float4*>(smem);
        for (int pass = 0; pass < 2; ++pass) {
          const int c0 = half * 64 + pass * 32;
          float lr[32], li[32];
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ACC2 + c0, lr);
          tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ACC2 + 128 + c0, li);
#pragma unroll
          for (int i = 0; i < 32; i += 2) {
            const int u = (c0 + i) >> 1;
            stg[r * 64 + (u ^ (r & 7))] = make_float4(lr[i], li[i], lr[i + 1], li[i + 1]);
          }
        }
        __syncthreads();
        // ---------------------------------------------------------------- phase 4: store L_IJ
        // operand planes opA (L) and opB (W = L D_J), 16 bytes per thread; the complex64 copy of L
        // (read only by the solve sweeps) is written after the release, below
        uint4* A = reinterpret_cast<uint4*>(opA + (int64_t)T.tile * ROWS * TB * (TF ? 4 : 2));
        uint4* B = reinterpret_cast<uint4*>(opB + (int64_t)T.tile * ROWS * TB * (TF ? 4 : 2));
        for (int it = tid; it < TB * 16; it += NTHR) {
          const int rr = it >> 4, c8 = it & 15;   // row, group of 8 columns
          float2 l[8];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int u = c8 * 4 + k;
            const float4 v = stg[rr * 64 + (u ^ (rr & 7))];
            l[2 * k] = make_float2(v.x, v.y);
            l[2 * k + 1] = make_float2(v.z, v.w);
          }
          float pv[4][8];   // planes: L_r, L_i, W_r, W_i
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float2 w = cmul(l[k], s_d[c8 * 8 + k]);
            pv[0][k] = l[k].x;
            pv[1][k] = l[k].y;
            pv[2][k] = w.x;
            pv[3][k] = w.y;
          }
          if constexpr (TF) {
            // opA rows: plane * 128 + row (L_r, L_i); opB rows: the same for W; 32 uint4 per 512-byte row
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
              A[(pl * 128 + rr) * 32 + 2 * c8] = pack4_tf32(pv[pl]);
              A[(pl * 128 + rr) * 32 + 2 * c8 + 1] = pack4_tf32(pv[pl] + 4);
              B[(pl * 128 + rr) * 32 + 2 * c8] = pack4_tf32(pv[2 + pl]);
              B[(pl * 128 + rr) * 32 + 2 * c8 + 1] = pack4_tf32(pv[2 + pl] + 4);
            }
            if (p.opS) {
              // bf16 split planes of L for the solve's tensor-core products, in the layout of the
              // split-BF16x3 engine's opA (rows split * 256 + plane * 128 + row)
              __nv_bfloat16 h[2][8], lo[2][8];
#pragma unroll
              for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int k = 0; k < 8; ++k) split2(pv[q][k], h[q][k], lo[q][k]);
              uint4* Sp = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(p.opS) + (int64_t)T.tile * 512 * TB * 2);
              Sp[((0 * 256 + 0 * 128) + rr) * 16 + c8] = pack8(h[0]);
              Sp[((0 * 256 + 1 * 128) + rr) * 16 + c8] = pack8(h[1]);
              Sp[((1 * 256 + 0 * 128) + rr) * 16 + c8] = pack8(lo[0]);
              Sp[((1 * 256 + 1 * 128) + rr) * 16 + c8] = pack8(lo[1]);
            }
          } else {
            __nv_bfloat16 h[4][8], lo[4][8];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int k = 0; k < 8; ++k) split2(pv[q][k], h[q][k], lo[q][k]);
            // opA rows: split * 256 + plane * 128 + row; 16 uint4 per 256-byte row
            A[((0 * 256 + 0 * 128) + rr) * 16 + c8] = pack8(h[0]);
            A[((0 * 256 + 1 * 128) + rr) * 16 + c8] = pack8(h[1]);
            A[((1 * 256 + 0 * 128) + rr) * 16 + c8] = pack8(lo[0]);
            A[((1 * 256 + 1 * 128) + rr) * 16 + c8] = pack8(lo[1]);
            // opB rows: split * 256 + plane * 128 + row (planes W_r, W_i)
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
              B[((0 * 256 + pl * 128) + rr) * 16 + c8] = pack8(h[2 + pl]);
              B[((1 * 256 + pl * 128) + rr) * 16 + c8] = pack8(lo[2 + pl]);
            }
          }
        }
        __syncthreads();
        trace_mark(p, task, 3);
      }
    }

    // ---------------------------------------------------------------- completion
    tc_fence_before();
    asm volatile("fence.proxy.async.global;" ::: "memory");   // writes before other blocks' TMA reads
    __syncthreads();
    if (T.flags & TF_UPDATE) trace_mark(p, task, 3);
    const int next = s_next[tcount & 1];
    if (warp == 2) release_successors(p, task, lane);
    // Complex64 copies of the tile for the solve sweeps: no task of this factorization reads
    // them, so they are written after the successors are released (off the critical path).
    if (!(T.flags & TF_UPDATE)) {
      if (is_diag) {
        const float2* sS = reinterpret_cast<const float2*>(smem);
        float2* Lt = Lg + (int64_t)T.tile * TB * TB;
        float2* Li = Linv + (int64_t)T.col * TB * TB;
        for (int i = tid; i < TB * TB; i += NTHR) {
          const int rr = i >> 7, cc = i & 127;
          Lt[i] = (cc < rr) ? sS[rr * LDS + cc] : make_float2(cc == rr ? 1.f : 0.f, 0.f);
          Li[i] = (cc < rr) ? sS[cc * LDS + rr] : make_float2(cc == rr ? 1.f : 0.f, 0.f);
        }
      } else {
        const float4* stg = reinterpret_cast<const float4*>(smem);
        float4* Lt4 = reinterpret_cast<float4*>(Lg + (int64_t)T.tile * TB * TB);
        for (int e = tid; e < TB * 64; e += NTHR) {
          const int rr = e >> 6, u = e & 63;
          Lt4[e] = stg[rr * 64 + (u ^ (rr & 7))];
        }
      }
      __syncthreads();   // shared memory is read before the next task's loads overwrite it
    }
    ++tcount;
    task = next >= 0 ? next : sched_pop(p, &s_task, &s_pending);
  }

  // teardown: after a failed wait, give in-flight copies and MMAs time to land (bounded)
  if (failed || ld_volatile(&p.ctl->abort)) {
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 2000000ull) __nanosleep(1000);
  }
  // TMEM is released by the allocating warp
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int tc_make_maps(void* opA, void* opB, int64_t ntiles, bool tf32, TcMaps* out, std::string& err) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      err = "cuTensorMapEncodeTiled is not available from the driver";
      return 1;
    }
    encode = (EncodeTiledFn)fn;
  }
  static_assert(sizeof(CUtensorMap) == 128, "CUtensorMap size");
  // rows of 128 elements (256 bytes bf16, 512 bytes tf32); a box is one chunk (64 bytes) of 128 rows
  const int esz = tf32 ? 4 : 2;
  const cuuint64_t rows = (cuuint64_t)(tf32 ? Eng<true>::ROWS : Eng<false>::ROWS);
  const cuuint32_t box[2] = {(cuuint32_t)(64 / esz), (cuuint32_t)TB};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint64_t stride[1] = {(cuuint64_t)TB * esz};
  const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUtensorMap ma, mb;
  const cuuint64_t dim[2] = {(cuuint64_t)TB, (cuuint64_t)ntiles * rows};
  CUresult r1 = encode(&ma, dt, 2, opA, dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CUresult r2 = encode(&mb, dt, 2, opB, dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r1) + ", " + std::to_string((int)r2) + ")";
    return 1;
  }
  std::memcpy(out->a, &ma, 128);
  std::memcpy(out->b, &mb, 128);
  return 0;
}

int launch_factor_tc(const FactorParams& p, const TcMaps& maps, bool tf32, int nblocks, cudaStream_t st) {
  const size_t smem = SMEM_BYTES + 1024;   // + alignment slack
  auto kern = tf32 ? factor_tc_kernel<true> : factor_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  CUtensorMap ma, mb;
  std::memcpy(&ma, maps.a, 128);
  std::memcpy(&mb, maps.b, 128);
  kern<<<nblocks, NTHR, smem, st>>>(p, ma, mb);
  return (int)cudaGetLastError();
}

}  // namespace d3m
