// Off-block products of the solve sweeps on the tcgen05 tensor cores (mixed precision, tile 128).
//
// A sweep level gathers, for every destination tile, the products of the off-diagonal L tiles
// with the source vectors already solved (Sec. II: the solution phase runs over the same block
// tasks as the factorization):
//   forward   P[slot][r][j]   = sum_items sum_c L_IJ[r][c] y_J[c][j]      (destination row tile I)
//   backward  P[slot][0][c][j] = sum_items sum_r L_IJ[r][c] w_I[r][j]     (destination column tile J)
// in the partial layout of the SIMT gather (backward: the whole sum in sub-slot 0, zeros in the
// others), so the block chains that consume the partials are unchanged.
//
// Arithmetic: split-BF16x3 products (a = hi + lo; hi*hi + hi*lo + lo*hi) accumulated in FP32 in
// tensor memory, the same operands and accuracy as the factorization's tile engine.  The L tiles
// are read from the bf16 operand planes that the factorization wrote (hi_r, hi_i, lo_r, lo_i; row
// major, 128 x 128), K-major for the forward product and, for the backward product L^T, through
// the MMA's transposed-A (MN-major) mode with 32 x 32 boxes of the same planes.  The source
// vectors are split to bf16 hi/lo in shared memory by four builder warps: for a chunk of 32 source
// rows, B planes of N = 2 NR rows [Re | Im outputs] for the real part ([y_r; y_i]) and the
// imaginary part ([-y_i; y_r]) of A, so every MMA (M = 128, N = 2 NR) adds both parts of the
// complex product:  [Re | Im] += A_r [y_r | y_i] + A_i [-y_i | y_r].
//
// Roles (384 threads): warp 0 issues the TMA loads of the L planes, warp 1 the MMAs, warps 2..5
// write the partials (TMEM lanes 32 (w % 4) ..), warps 6..9 build the source planes.  Four
// 48 KB stages (one 32-row chunk of one item), two TMEM accumulators (the epilogue of one unit
// overlaps the next unit's products).
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

constexpr int GW = 10;                       // warps
constexpr int GTH = GW * 32;
constexpr int NBUILD = 4;                    // builder warps (6..9)
constexpr int GNST = 4;                      // stages
constexpr uint32_t GPLANE = 128 * 64;        // one A plane chunk: 128 rows x 64 bytes
constexpr uint32_t GA_STAGE = 4 * GPLANE;    // hi_r, hi_i, lo_r, lo_i: 32 KB
constexpr uint32_t GB_PLANE = 64 * 64;       // one B plane: up to 64 rows x 64 bytes
constexpr uint32_t GB_STAGE = 4 * GB_PLANE;  // [part r | part i] x [hi | lo]: 16 KB
constexpr uint32_t GSTG = GA_STAGE + GB_STAGE;
constexpr uint32_t GSMEM = GNST * GSTG;      // 192 KB
constexpr int GACC = 64;                     // TMEM columns of one accumulator (N <= 64)

__device__ __forceinline__ uint32_t su32g(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void gbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void gbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void gbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool gbar_wait(uint32_t bar, uint32_t parity, uint64_t deadline) {
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (globaltimer_ns() > deadline) return false;
  }
}
__device__ __forceinline__ void gtma_2d(uint32_t dst, const void* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// 64-byte swizzle descriptors.  K-major: 8-row groups 512 bytes apart (leading offset unused).
// MN-major (backward A = L^T): 32-element MN groups lbo bytes apart, 8-row K groups 512 apart.
__device__ __forceinline__ uint64_t gdesc(uint32_t saddr, uint32_t lbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// kind::f16, bf16 A and B, f32 D, M = 128, N; transpose_a: A is MN-major
__device__ __forceinline__ uint32_t gidesc(uint32_t n, bool transpose_a) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (transpose_a ? (1u << 15) : 0u) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}
__device__ __forceinline__ void gmma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void gcommit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void gfence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void gfence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void gtmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void gpdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void gpdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void gsplit(float a, unsigned short& hi, unsigned short& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(a);
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(__float2bfloat16_rn(a - __bfloat162float(h)));
}

}  // namespace

template <bool FWD>
__global__ void __launch_bounds__(GTH, 1)
    gather_tc_kernel(const SolveGroup* __restrict__ groups, const SolveItem* __restrict__ items,
                     const __grid_constant__ CUtensorMap mapK, const __grid_constant__ CUtensorMap mapT,
                     const float2* __restrict__ Y, float2* __restrict__ P, int64_t npad, int nrhs, int NR,
                     int* status, const int* __restrict__ done, const int32_t* __restrict__ tinst, int nunits) {
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  unsigned char* smem = gsm_raw + ((1024u - (su32g(gsm_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t a_full[GNST], b_full[GNST], s_empty[GNST], acc_full[2], acc_empty[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = 128, nh = 2;
  const int j0 = blockIdx.y * NR;
  const int N = 2 * NR;
  auto masked = [&](int u) { return done && done[tinst[groups[u].dst]] != 0; };
  gpdl_trigger();
  // the units of this block: u = blockIdx.x + k gridDim.x (every role walks the same list)
  int nmine = 0;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) nmine += masked(u) ? 0 : 1;
  if (nmine == 0) {
    gpdl_wait();
    return;
  }
  if (tid == 0) {
    for (int s = 0; s < GNST; ++s) {
      gbar_init(su32g(&a_full[s]), 1);
      gbar_init(su32g(&b_full[s]), NBUILD);
      gbar_init(su32g(&s_empty[s]), 1);
    }
    for (int s = 0; s < 2; ++s) {
      gbar_init(su32g(&acc_full[s]), 1);
      gbar_init(su32g(&acc_empty[s]), 4);
    }
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32g(&s_tmem)), "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  gfence_before();
  __syncthreads();
  gfence_after();
  const uint32_t tmem = s_tmem;
  const uint64_t deadline = globaltimer_ns() + 2000000000ull;

  if (warp == 0) {
    // ---------------------------------------------------------------- L planes (TMA)
    // the tiles of L are fixed during the solve: no wait for the predecessor kernel
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        if (masked(u)) continue;
        const SolveGroup g = groups[u];
        for (int q = 0; q < g.count && ok; ++q) {
          const int64_t row0 = (int64_t)items[g.first + q].tile * 512;   // opA rows of the tile
          for (int c = 0; c < 4; ++c, ++it) {
            const uint32_t s = it % GNST, use = it / GNST;
            if (!gbar_wait(su32g(&s_empty[s]), (use & 1) ^ 1, deadline)) { ok = false; break; }
            const uint32_t fb = su32g(&a_full[s]);
            gbar_expect_tx(fb, GA_STAGE);
            const uint32_t sa = su32g(smem + s * GSTG);
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) {
              // planes hi_r, hi_i, lo_r, lo_i at opA rows split * 256 + part * 128 (pl = 2 split + part)
              const int prow = (int)(row0 + (pl >> 1) * 256 + (pl & 1) * 128);
              if (FWD) {
                gtma_2d(sa + pl * GPLANE, &mapK, c * 32, prow, fb);          // rows r, columns c0..c0+31
              } else {
#pragma unroll
                for (int mc = 0; mc < 4; ++mc)                                // rows c0..c0+31, all columns
                  gtma_2d(sa + pl * GPLANE + mc * 2048, &mapT, mc * 32, prow + c * 32, fb);
              }
            }
          }
        }
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t it = 0, un = 0;
      bool ok = true;
      const uint32_t idesc = gidesc((uint32_t)N, !FWD);
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        if (masked(u)) continue;
        const SolveGroup g = groups[u];
        const uint32_t buf = un & 1, ause = un >> 1;
        if (!gbar_wait(su32g(&acc_empty[buf]), (ause & 1) ^ 1, deadline)) { ok = false; break; }
        gfence_after();
        const uint32_t d = tmem + buf * GACC;
        for (int q = 0; q < g.count && ok; ++q)
          for (int c = 0; c < 4; ++c, ++it) {
            const uint32_t s = it % GNST, use = it / GNST;
            if (!gbar_wait(su32g(&a_full[s]), use & 1, deadline) || !gbar_wait(su32g(&b_full[s]), use & 1, deadline)) {
              ok = false;
              break;
            }
            gfence_after();
            const uint32_t sa = su32g(smem + s * GSTG), sb = sa + GA_STAGE;
            const uint32_t bp = (uint32_t)N * 64;   // one B plane (N rows)
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              // K step of 16: K-major A advances 32 bytes in its rows, MN-major A 16 rows (1 KB)
              const uint32_t ako = FWD ? kk * 32 : kk * 1024;
              const uint32_t lbo = FWD ? 16 : 2048;
#pragma unroll
              for (int pr = 0; pr < 3; ++pr) {
                // split pairs (A, B): (lo, hi), (hi, lo), (hi, hi)
                const int sa_split = pr == 0 ? 1 : 0, sb_split = pr == 1 ? 1 : 0;
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                  const uint32_t acc = (q == 0 && c == 0 && kk == 0 && pr == 0 && part == 0) ? 0u : 1u;
                  const uint32_t a_addr = sa + (uint32_t)(sa_split * 2 + part) * GPLANE + ako;
                  const uint32_t b_addr = sb + (uint32_t)(part * 2 + sb_split) * bp + kk * 32;
                  gmma(d, gdesc(a_addr, lbo), gdesc(b_addr, 16), idesc, acc);
                }
              }
            }
            gcommit(su32g(&s_empty[s]));
          }
        gcommit(su32g(&acc_full[buf]));
        ++un;
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
    __syncwarp();
  } else if (warp < 6) {
    // ---------------------------------------------------------------- partials (epilogue)
    const int quad = warp & 3;
    const int row = quad * 32 + lane;           // TMEM lane: output row (forward) / column (backward)
    uint32_t un = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      if (masked(u)) continue;
      const SolveGroup g = groups[u];
      const uint32_t buf = un & 1, ause = un >> 1;
      if (!gbar_wait(su32g(&acc_full[buf]), ause & 1, deadline)) { ok = false; break; }
      gfence_after();
      float2* out = FWD ? P + (int64_t)g.slot * nh * b * nrhs + (int64_t)row * nrhs
                        : P + (int64_t)g.slot * nh * b * nrhs + (int64_t)row * nrhs;
      for (int jb = 0; jb < NR; jb += 8) {
        float re[8], im[8];
        gtmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + buf * GACC + jb, re);
        gtmem_ld8(tmem + ((uint32_t)(quad * 32) << 16) + buf * GACC + NR + jb, im);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (j0 + jb + q < nrhs) out[j0 + jb + q] = make_float2(re[q], im[q]);
      }
      if (!FWD) {
        // the other 64-row sub-slot of the backward partial holds zeros
        float2* z = P + ((int64_t)g.slot * nh + 1) * b * nrhs + (int64_t)row * nrhs;
        for (int q = 0; q < NR && j0 + q < nrhs; ++q) z[j0 + q] = make_float2(0.f, 0.f);
      }
      gfence_before();
      __syncwarp();
      if (lane == 0) gbar_arrive(su32g(&acc_empty[buf]));
      ++un;
    }
    if (!ok) atomicExch(&s_fail, 1);
  } else {
    // ---------------------------------------------------------------- source planes (4 warps)
    // the source rows come from the predecessor kernel (previous level)
    gpdl_wait();
    const int bt = tid - 6 * 32;                // 0..127
    uint32_t it = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      if (masked(u)) continue;
      const SolveGroup g = groups[u];
      for (int q = 0; q < g.count && ok; ++q) {
        const int64_t src0 = (int64_t)items[g.first + q].src * b;
        for (int c = 0; c < 4; ++c, ++it) {
          const uint32_t s = it % GNST, use = it / GNST;
          if (!gbar_wait(su32g(&s_empty[s]), (use & 1) ^ 1, deadline)) { ok = false; break; }
          unsigned char* sb = smem + s * GSTG + GA_STAGE;
          const uint32_t bp = (uint32_t)N * 64;
          // task = (right-hand side j < NR, 8-row group k8 < 4): 8 source values -> 8 planes' words
          for (int t = bt; t < NR * 4; t += 128) {
            const int j = t >> 2, k8 = t & 3;
            float yr[8], yi[8];
            if (j0 + j < nrhs) {
              const float4* src = reinterpret_cast<const float4*>(Y + (int64_t)(j0 + j) * npad + src0 + c * 32 + k8 * 8);
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float4 v = src[e];
                yr[2 * e] = v.x;
                yi[2 * e] = v.y;
                yr[2 * e + 1] = v.z;
                yi[2 * e + 1] = v.w;
              }
            } else {
#pragma unroll
              for (int e = 0; e < 8; ++e) yr[e] = yi[e] = 0.f;
            }
            unsigned short rh[8], rl[8], ih[8], il[8], nh_[8], nl[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              gsplit(yr[e], rh[e], rl[e]);
              gsplit(yi[e], ih[e], il[e]);
              nh_[e] = ih[e] ^ 0x8000u;                // -y_i: sign flip of both parts (exact)
              nl[e] = il[e] ^ 0x8000u;
            }
            // plane rows: Re outputs j, Im outputs NR + j; 16-byte unit k8 of a 64-byte row, swizzled
            auto put = [&](int plane, int rrow, const unsigned short* v) {
              const uint32_t off = (uint32_t)plane * bp + (uint32_t)rrow * 64u + ((uint32_t)(k8 ^ ((rrow >> 1) & 3)) << 4);
              *reinterpret_cast<uint4*>(sb + off) = *reinterpret_cast<const uint4*>(v);
            };
            // part r (A_r): [y_r | y_i]; part i (A_i): [-y_i | y_r]; planes part * 2 + split
            put(0, j, rh);
            put(0, NR + j, ih);
            put(1, j, rl);
            put(1, NR + j, il);
            put(2, j, nh_);
            put(2, NR + j, rh);
            put(3, j, nl);
            put(3, NR + j, rl);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
          __syncwarp();
          if (lane == 0) gbar_arrive(su32g(&b_full[s]));
        }
      }
    }
    if (!ok) atomicExch(&s_fail, 1);
  }

  if (warp < 6) gpdl_wait();                    // every thread waits before it exits
  __syncthreads();
  if (s_fail) {
    if (tid == 0) atomicExch(status, (int)D3M_ERR_TIMEOUT);
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 2000000ull) __nanosleep(1000);
  }
  gfence_before();
  __syncthreads();
  gfence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
}

// Tensor maps of the operand planes of L for the solve: box {32, 128} (forward, K-major) and
// {32, 32} (backward, read as MN-major blocks), both with the 64-byte swizzle.
int gather_tc_make_maps(void* opA, int64_t ntiles, GatherTcMaps* out, std::string& err) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      err = "cuTensorMapEncodeTiled is not available from the driver";
      return 1;
    }
    encode = (EncodeFn)fn;
  }
  const cuuint64_t dim[2] = {128, (cuuint64_t)ntiles * 512};
  const cuuint64_t stride[1] = {256};
  const cuuint32_t estr[2] = {1, 1};
  for (int k = 0; k < 2; ++k) {
    const cuuint32_t box[2] = {32, k == 0 ? 128u : 32u};
    CUtensorMap m;
    const CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, opA, dim, stride, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      err = "cuTensorMapEncodeTiled (solve operands) failed: " + std::to_string((int)r);
      return 1;
    }
    std::memcpy(k == 0 ? out->k : out->t, &m, 128);
  }
  return 0;
}

int launch_gather_tc(bool fwd, const GatherTcMaps& maps, const SolveGroup* groups, const SolveItem* items,
                     const void* Y, void* P, int64_t npad, int nrhs, int* status, const int* done,
                     const int32_t* tinst, int nunits, int nsm, cudaStream_t st) {
  const size_t smem = GSMEM + 1024;
  auto kern = fwd ? gather_tc_kernel<true> : gather_tc_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  CUtensorMap mk, mt;
  std::memcpy(&mk, maps.k, 128);
  std::memcpy(&mt, maps.t, 128);
  // right-hand sides in groups of at most 32 (N = 2 NR <= 64 TMEM columns per accumulator)
  const int ng = (nrhs + 31) / 32;
  const int per = (nrhs + ng - 1) / ng;
  const int NR = (per + 7) / 8 * 8;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nunits < nsm ? nunits : nsm), (unsigned)ng, 1);
  cfg.blockDim = dim3(GTH, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, groups, items, mk, mt, (const float2*)Y, (float2*)P, npad, nrhs, NR, status, done,
                         tinst, nunits);
  return (int)e;
}

}  // namespace d3m
