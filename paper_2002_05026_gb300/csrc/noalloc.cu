// d3m_grad_eps_noalloc: the epsilon gradient with all temporary storage in a fixed static
// device array, for callers that must not allocate memory during the call (a host application
// whose own allocator owns the device memory and forbids allocations by libraries, or a device
// so full that a late cudaMalloc of temporaries could fail after the solves are done).
//
// The array g_noalloc_scratch lives in this file, is reserved on every device that loads the
// library, and keeps its contents between calls.  Host code must not use its name as a device
// address: the address is obtained once per device with cudaGetSymbolAddress.  The call copies
// the caller's index arrays from host memory and synchronizes the stream before it returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "d3m.h"
#include "kernels.h"

namespace {

constexpr int NA_MAX_IF = 16384;                 // interfaces
constexpr int NA_MAX_DOM = 16384;                // domains
constexpr int NA_MAX_DOMIF = 6 * NA_MAX_DOM;     // entries of dom_if
constexpr size_t NA_OFF_SUM = 0;                                          // double2 [NA_MAX_IF]
constexpr size_t NA_OFF_DPTR = NA_OFF_SUM + sizeof(double2) * NA_MAX_IF;   // int32 [NA_MAX_DOM + 1]
constexpr size_t NA_OFF_DIF = NA_OFF_DPTR + sizeof(int32_t) * (NA_MAX_DOM + 64);   // int32 [NA_MAX_DOMIF]
constexpr size_t NA_OFF_DJ = NA_OFF_DIF + sizeof(int32_t) * NA_MAX_DOMIF;  // double [NA_MAX_DOM]
constexpr size_t NA_BYTES = NA_OFF_DJ + sizeof(double) * NA_MAX_DOM;       // ~0.9 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};

// dJ[i] = k2 * sum over the interfaces f of domain i of Re(s_f), in list order
__global__ void domain_sum_kernel(const double2* __restrict__ sums, const int32_t* __restrict__ dom_ptr,
                                  const int32_t* __restrict__ dom_if, int ndom, double k2, double* __restrict__ dJ) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndom) return;
  double re = 0.0;
  for (int q = dom_ptr[i]; q < dom_ptr[i + 1]; ++q) re += sums[dom_if[q]].x;
  dJ[i] = k2 * re;
}

}  // namespace

namespace d3m {
// accessors to the handle (defined in api.cu)
int handle_geometry(d3m_handle h, int64_t* n, int32_t* nblk, const int64_t** xoff_orig, const int32_t** m_orig);
int handle_error(d3m_handle h, int code, const char* msg);
int handle_device(d3m_handle h);
}  // namespace d3m

extern "C" int d3m_grad_eps_noalloc(d3m_handle h, const void* Lambda, const void* X, int32_t nrhs, int32_t ndom,
                                    const int32_t* dom_ptr, const int32_t* dom_if, double k2, double* dJ_deps,
                                    void* stream) {
  using namespace d3m;
  if (!h) return D3M_ERR_INVALID;
  if (!Lambda || !X || !dom_ptr || !dom_if || !dJ_deps || nrhs < 1 || ndom < 0)
    return handle_error(h, D3M_ERR_INVALID, "bad argument to d3m_grad_eps_noalloc");
  int64_t n = 0;
  int32_t nblk = 0;
  const int64_t* xoff_orig = nullptr;
  const int32_t* m_orig = nullptr;
  handle_geometry(h, &n, &nblk, &xoff_orig, &m_orig);
  if (nblk > NA_MAX_IF || ndom > NA_MAX_DOM)
    return handle_error(h, D3M_ERR_INVALID,
                        "d3m_grad_eps_noalloc: sizes exceed its fixed scratch (interfaces <= 16384, domains <= "
                        "16384, domain-interface entries <= 98304)");
  // dom_ptr: starts at 0, nondecreasing (so every entry lies in [0, dom_ptr[ndom]]), and its
  // total fits the scratch; checked entry by entry before anything is copied or launched, so
  // the device kernel can only read the entries copied below
  if (dom_ptr[0] != 0) return handle_error(h, D3M_ERR_INVALID, "d3m_grad_eps_noalloc: dom_ptr[0] must be 0");
  for (int i = 0; i < ndom; ++i)
    if (dom_ptr[i + 1] < dom_ptr[i])
      return handle_error(h, D3M_ERR_INVALID, "d3m_grad_eps_noalloc: dom_ptr must be nondecreasing");
  if (dom_ptr[ndom] > NA_MAX_DOMIF)
    return handle_error(h, D3M_ERR_INVALID,
                        "d3m_grad_eps_noalloc: sizes exceed its fixed scratch (interfaces <= 16384, domains <= "
                        "16384, domain-interface entries <= 98304)");
  for (int q = 0; q < dom_ptr[ndom]; ++q)
    if (dom_if[q] < 0 || dom_if[q] >= nblk) return handle_error(h, D3M_ERR_INVALID, "dom_if entry out of range");
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, Lambda) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
      cudaPointerGetAttributes(&pa, X) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return handle_error(h, D3M_ERR_INVALID, "Lambda and X must be device memory");
  }
  // set-up, once per device, with that device current: the device address of the array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
    return handle_error(h, D3M_ERR_CUDA, "cudaGetDevice failed");
  if (dev != handle_device(h))
    return handle_error(h, D3M_ERR_INVALID,
                        "d3m_grad_eps_noalloc: the current device is not the device the handle was created on");
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return handle_error(h, D3M_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  unsigned char* base = g_scratch_ptr[dev];
  double2* sums = reinterpret_cast<double2*>(base + NA_OFF_SUM);
  int32_t* dptr = reinterpret_cast<int32_t*>(base + NA_OFF_DPTR);
  int32_t* dif = reinterpret_cast<int32_t*>(base + NA_OFF_DIF);
  double* dJ = reinterpret_cast<double*>(base + NA_OFF_DJ);
  cudaStream_t st = (cudaStream_t)stream;
  // every entry read below is written first in this call: nothing has to start at zero
  cudaError_t e = cudaMemcpyAsync(dptr, dom_ptr, sizeof(int32_t) * (ndom + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && dom_ptr[ndom] > 0)
    e = cudaMemcpyAsync(dif, dom_if, sizeof(int32_t) * dom_ptr[ndom], cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return handle_error(h, D3M_ERR_CUDA, cudaGetErrorString(e));
  int rc = launch_contract((const double2*)Lambda, (const double2*)X, n, nrhs, xoff_orig, m_orig, nblk, sums, st);
  if (rc) return handle_error(h, D3M_ERR_CUDA, "contract launch failed");
  if (ndom > 0) {
    domain_sum_kernel<<<(ndom + 127) / 128, 128, 0, st>>>(sums, dptr, dif, ndom, k2, dJ);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(dJ_deps, dJ, sizeof(double) * ndom, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return handle_error(h, D3M_ERR_CUDA, cudaGetErrorString(e));
  }
  return D3M_OK;
}
