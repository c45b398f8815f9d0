// Inverses of the unit-lower diagonal blocks L_JJ (complex FP32), built once per factorization so
// that the solve applies every diagonal block as one product (y_J = L_JJ^{-1} r_J) instead of a
// sequential chain over its tiles.  With the tile inverses Linv_tt of the factorization:
//   Inv(t', t') = Linv_t't',   Inv(t, t') = -Linv_tt * sum_{s=t'}^{t-1} L(t, s) Inv(s, t')   (t > t').
// One thread block per (block J, tile column t') forms Inv(t, t') for t = t'+1, ..., nt-1 in order
// (each needs the ones above it in the same column).  Tiles are b x b, row-major, b in {64, 128}.
// Every tile is also stored transposed, InvT(t', t) = Inv(t, t')^T (t >= t', diagonal included),
// so that the backward solve streams contiguous row strips as well.
// Products: shared-memory staged FP32 SIMT GEMM, each of the 256 threads owning a TM x TM
// sub-tile (TM = b / 16).
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace d3m {

namespace {

constexpr int IT = 256;   // threads
constexpr int KC = 16;    // k-chunk of the staged products

// acc += A * Bm for b x b tiles in global memory (row-major, leading dimension b)
template <int B>
__device__ __forceinline__ void gemm_gg(const float2* __restrict__ A, const float2* __restrict__ Bm, float2* sA,
                                        float2* sB, float2 (&acc)[B / 16][B / 16]) {
  constexpr int TM = B / 16, LDA = B + 1;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int k0 = 0; k0 < B; k0 += KC) {
    __syncthreads();                                   // the previous chunk is consumed
    for (int i = threadIdx.x; i < B * KC; i += IT) {
      const int r = i / KC, kk = i % KC;
      sA[kk * LDA + r] = A[(int64_t)r * B + k0 + kk];  // transposed: (k, row)
    }
    for (int i = threadIdx.x; i < KC * B; i += IT) {
      const int kk = i / B, c = i % B;
      sB[kk * B + c] = Bm[(int64_t)(k0 + kk) * B + c];
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      float2 a[TM], bb[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = sA[kk * LDA + ty * TM + i];
#pragma unroll
      for (int j = 0; j < TM; ++j) bb[j] = sB[kk * B + tx * TM + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = cfma(a[i], bb[j], acc[i][j]);
    }
  }
}

// acc = A * C with A in global memory and C in shared memory ([B][B + 1])
template <int B>
__device__ __forceinline__ void gemm_gs(const float2* __restrict__ A, const float2* sC, float2* sA,
                                        float2 (&acc)[B / 16][B / 16]) {
  constexpr int TM = B / 16, LDA = B + 1;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int k0 = 0; k0 < B; k0 += KC) {
    __syncthreads();
    for (int i = threadIdx.x; i < B * KC; i += IT) {
      const int r = i / KC, kk = i % KC;
      sA[kk * LDA + r] = A[(int64_t)r * B + k0 + kk];
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      float2 a[TM], bb[TM];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = sA[kk * LDA + ty * TM + i];
#pragma unroll
      for (int j = 0; j < TM; ++j) bb[j] = sC[(k0 + kk) * LDA + tx * TM + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = cfma(a[i], bb[j], acc[i][j]);
    }
  }
}

template <int B>
__global__ void __launch_bounds__(IT) inv_build_kernel(const int2* __restrict__ work, const int32_t* __restrict__ tstart,
                                                       const int64_t* __restrict__ tcolptr,
                                                       const int64_t* __restrict__ inv_off,
                                                       const int64_t* __restrict__ invT_off,
                                                       const float2* __restrict__ L, const float2* __restrict__ Linv,
                                                       float2* __restrict__ Inv, float2* __restrict__ InvT) {
  constexpr int TM = B / 16, LDA = B + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sA = reinterpret_cast<float2*>(smem_raw);   // [KC][B + 1]
  float2* sB = sA + KC * LDA;                          // [KC][B]
  float2* sC = sB + KC * B;                            // [B][B + 1]
  const int2 wk = work[blockIdx.x];
  const int k = wk.x, tq = wk.y;
  const int t0 = tstart[k], nt = tstart[k + 1] - t0;
  const int64_t ib = inv_off[k], ibt = invT_off[k];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t tsz = (int64_t)B * B;
  {
    // InvT(tq, tq) = Linv_tq^T
    const float2* src = Linv + (int64_t)(t0 + tq) * tsz;
    float2* dst = InvT + (ibt + tq * (tq + 1) / 2 + tq) * tsz;
    for (int i = threadIdx.x; i < B * B; i += IT) {
      const int r = i / B, c = i % B;
      dst[(int64_t)c * B + r] = src[i];
    }
  }
  for (int t = tq + 1; t < nt; ++t) {
    float2 acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) acc[i][j] = make_float2(0.f, 0.f);
    // C = sum_s L(t, s) Inv(s, tq)
    for (int s = tq; s < t; ++s) {
      const float2* A = L + (tcolptr[t0 + s] + (t - s)) * tsz;
      const float2* Bm = (s == tq) ? Linv + (int64_t)(t0 + tq) * tsz : Inv + (ib + s * (s - 1) / 2 + tq) * tsz;
      gemm_gg<B>(A, Bm, sA, sB, acc);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) sC[(ty * TM + i) * LDA + tx * TM + j] = acc[i][j];
    // Inv(t, tq) = -Linv_tt C
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) acc[i][j] = make_float2(0.f, 0.f);
    gemm_gs<B>(Linv + (int64_t)(t0 + t) * tsz, sC, sA, acc);
    float2* out = Inv + (ib + t * (t - 1) / 2 + tq) * tsz;
    float2* outT = InvT + (ibt + t * (t + 1) / 2 + tq) * tsz;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        const float2 v = make_float2(-acc[i][j].x, -acc[i][j].y);
        out[(int64_t)(ty * TM + i) * B + tx * TM + j] = v;
        outT[(int64_t)(tx * TM + j) * B + ty * TM + i] = v;
      }
    __syncthreads();   // Inv(t, tq) is read back by this block for the next t
  }
}

}  // namespace

int launch_inv_build(const int2* work, int nwork, const int32_t* tstart, const int64_t* tcolptr,
                     const int64_t* inv_off, const int64_t* invT_off, const void* L, const void* Linv, void* Inv,
                     void* InvT, int b, cudaStream_t st) {
  if (nwork <= 0) return 0;
  const size_t smem = sizeof(float2) * ((size_t)KC * (b + 1) + (size_t)KC * b + (size_t)b * (b + 1));
  if (b == 128) {
    cudaFuncSetAttribute(inv_build_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    inv_build_kernel<128><<<nwork, IT, smem, st>>>(work, tstart, tcolptr, inv_off, invT_off, (const float2*)L,
                                                   (const float2*)Linv, (float2*)Inv, (float2*)InvT);
  } else if (b == 64) {
    cudaFuncSetAttribute(inv_build_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    inv_build_kernel<64><<<nwork, IT, smem, st>>>(work, tstart, tcolptr, inv_off, invT_off, (const float2*)L,
                                                  (const float2*)Linv, (float2*)Inv, (float2*)InvT);
  } else {
    return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace d3m
