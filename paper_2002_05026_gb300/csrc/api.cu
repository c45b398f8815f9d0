// C ABI of the D3M dual-system solver (declarations and contracts in include/d3m.h).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "d3m.h"
#include "device.cuh"
#include "kernels.h"
#include "symbolic.h"

using namespace d3m;

struct d3m_ctx {
  Symbolic S;
  d3m_options opt{};
  bool fp64 = true, tc = false, tf32 = false;
  int b = 64;
  int device = 0, nsm = 0;
  size_t csize = 16;                 // bytes of one factor element
  std::string err;
  std::vector<void*> allocs;
  int64_t dev_bytes = 0;
  bool factored = false;
  bool factor_checked = false;       // status of the last factorization already read
  int last_status = D3M_OK;
  int refine_iters = 0;
  double omega = NAN, omega_first = NAN;
  int omega_valid = 0;
  // device timing: event pairs recorded around launches, read by d3m_get_info
  enum { EV_FACTOR = 0, EV_RESID = 1, EV_SWEEP = 2, EV_SOLVE = 3, EV_KINDS = 4 };
  struct EvPair { cudaEvent_t a, b; int kind; };
  std::vector<cudaEvent_t> ev_pool;
  std::vector<EvPair> ev_pending;
  EvPair ev_open[EV_KINDS];
  double ev_total[EV_KINDS] = {0, 0, 0, 0};
  int64_t ev_calls[EV_KINDS] = {0, 0, 0, 0};
  double last_factor_ms = 0, last_solve_ms = 0, last_resid_ms = 0;
  int64_t launches = 0;
  // factor data
  double2* K = nullptr;
  TileTask* tasks = nullptr;
  KEntry* klist = nullptr;
  int32_t* ndeps = nullptr;
  int32_t* cnt = nullptr;
  int64_t* succ_ptr = nullptr;
  int32_t* succ = nullptr;
  int32_t* ready = nullptr;
  int32_t* init_ready = nullptr;
  int32_t* ready_hi = nullptr;       // priority lane
  int32_t* init_ready_hi = nullptr;
  Ctl* ctl = nullptr;
  Ctl* ctl0 = nullptr;               // initial queue state, copied into ctl by every factor call
  Ctl* h_ctl = nullptr;              // pinned copy of ctl after the factorization
  void* L = nullptr;
  void* Linv = nullptr;
  void* D = nullptr;
  void* opA = nullptr;
  void* opB = nullptr;
  void* opS = nullptr;               // TF32: bf16 split planes of L for the solve's tensor-core products
  void* Sacc = nullptr;
  void* E = nullptr;                 // pivot mode: sub-diagonals of the 2 x 2 pivot blocks [NT][b]
  int32_t* piv = nullptr;            // pivot mode: permutation of every diagonal tile [NT][b]
  int64_t* trace = nullptr;
  TcMaps maps;
  GatherTcMaps gmaps;                // L's operand planes for the tensor-core solve gathers
  bool gather_tc = false;
  // solve
  SolveItem* fwd_items = nullptr;
  SolveItem* bwd_items = nullptr;
  SolveGroup* fwd_groups = nullptr;
  SolveGroup* bwd_groups = nullptr;
  int64_t* fwd_slot = nullptr;
  int64_t* bwd_slot = nullptr;
  int32_t* lev_blocks = nullptr;
  std::vector<int64_t> lev_ptr;
  int32_t* lev_tiles = nullptr;
  std::vector<int64_t> lev_tile_ptr;
  std::vector<int32_t> lev_maxnt;    // most tiles of one block, per level
  std::vector<int32_t> lev_maxcnt_fwd, lev_maxcnt_bwd;   // most partials of one tile row / column
  int32_t* tstart = nullptr;
  int64_t* tcolptr = nullptr;
  int64_t* pad2orig = nullptr;
  void* Y = nullptr;
  void* P = nullptr;
  int max_rows = 0;
  // inverses of the diagonal blocks (mixed precision): the solve applies each diagonal block as
  // one product with its inverse
  bool use_inv = false;
  void* Inv = nullptr;
  int64_t* inv_off = nullptr;
  void* InvT = nullptr;
  int64_t* invT_off = nullptr;
  int2* inv_work = nullptr;
  int n_inv_work = 0;
  // refinement / residual
  double2* d_b = nullptr;
  double2* d_x = nullptr;
  double2* d_xbest = nullptr;
  double2* d_r = nullptr;
  int64_t* kblk_off = nullptr;
  int64_t* res_ptr = nullptr;
  int32_t* res_blk = nullptr;
  int32_t* res_src = nullptr;
  int32_t* res_tr = nullptr;
  int32_t* m_orig = nullptr;
  int64_t* xoff_orig = nullptr;
  unsigned* norms = nullptr;         // [3 * ninst * max_nrhs + ninst]: rmax, xmax, bmax, kmax
  double* omega_dev = nullptr;       // [ninst][max_nrhs]
  double* stat_dev = nullptr;        // [3]: max omega, instances still refining, their progress measure
  unsigned* dmax = nullptr;          // [ninst][max_nrhs] max |correction| of the step (float bits)
  float* dprev = nullptr;            // [ninst][max_nrhs] the same for the previous step
  int* sweep_status = nullptr;       // device: set by a sweep kernel whose bounded wait expired
  double* h_stat = nullptr;          // pinned [3]
  // gradients
  int32_t* rowidx = nullptr;
  int32_t* blk_col = nullptr;
  int64_t* colptr = nullptr;
  double2* contract = nullptr;
  // FP64-accurate residual on the tensor cores: digit planes of K (per factorization) and x
  ResidualTc rtc{};
  ResidTcMaps rtc_maps;
  std::vector<int2> rtile_host;      // (row block f, 128-row tile)
  int max_rtiles = 1;
  // batched handles: independent systems stored as one block-diagonal system
  int ninst = 1;
  std::vector<int32_t> inst_blk;     // [ninst+1] first block (caller numbering) of each instance
  int32_t* inst = nullptr;           // device [N]: instance of every block
  int32_t* tinst = nullptr;          // device [NT]: instance of every tile row (permuted numbering)
  int* done = nullptr;               // device [ninst]: 1 once an instance converged in this solve
  int last_nrhs = 0;                 // nrhs of the last solve (for the per-instance omega)
  // CUDA graphs (opt.graphs): launch sequences captured once on a private stream, replayed on
  // the caller's stream; keyed by what the captured pointers and sizes depend on
  cudaStream_t cap = nullptr;
  bool capturing = false;
  cudaStream_t side = nullptr;       // second stream of a factorization (norm and split of K)
  // upload of a host K while the factorization runs (tensor-core engines, page-locked K)
  cudaStream_t kup = nullptr;
  cudaEvent_t ev_kup0 = nullptr, ev_kup1 = nullptr;
  int32_t* k_arrived = nullptr;      // blocks uploaded so far, in the analysis' upload order
  bool kup_ok = false;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  struct Graph { const void* src; int nrhs, accumulate; cudaGraphExec_t exec; int64_t launches; };
  std::vector<Graph> g_factor, g_solve;
};

namespace {

thread_local std::string g_err;

int set_err(d3m_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  g_err = msg;
  return code;
}

#define CUDA_TRY(h, call)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return set_err(h, D3M_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

cudaEvent_t ev_get(d3m_ctx* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void ev_begin(d3m_ctx* h, int kind, cudaStream_t st) {
  if (h->capturing) return;          // captured work is timed around its graph launch
  d3m_ctx::EvPair& p = h->ev_open[kind];
  p.a = ev_get(h);
  p.b = ev_get(h);
  p.kind = kind;
  if (p.a) cudaEventRecord(p.a, st);
}

void ev_end(d3m_ctx* h, int kind, cudaStream_t st) {
  if (h->capturing) return;
  d3m_ctx::EvPair& p = h->ev_open[kind];
  if (!p.a || !p.b) return;
  cudaEventRecord(p.b, st);
  h->ev_pending.push_back(p);
  p.a = p.b = nullptr;
}

template <typename T>
T* dalloc(d3m_ctx* h, size_t count) {
  if (count == 0) count = 1;
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  h->allocs.push_back(p);
  h->dev_bytes += (int64_t)(count * sizeof(T));
  return (T*)p;
}

template <typename T>
int upload(d3m_ctx* h, T** dst, const std::vector<T>& v) {
  *dst = dalloc<T>(h, v.size());
  if (!*dst) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed (" + std::to_string(v.size() * sizeof(T)) + " bytes)");
  if (!v.empty()) CUDA_TRY(h, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return D3M_OK;
}

// page-locked (or registered) host memory, which the copy engines read asynchronously
static bool is_pinned_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

typedef CUresult (*WriteValue32Fn)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
static WriteValue32Fn write_value32() {
  static WriteValue32Fn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (WriteValue32Fn)f;
    cudaGetLastError();
  }
  return fn;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Replay (capturing on first use) the launch sequence `body` for key (src, nrhs, accumulate).
// The body enqueues on the stream it is given; h->launches counts its kernels once per replay.
template <typename F>
int graph_run(d3m_ctx* h, std::vector<d3m_ctx::Graph>& cache, const void* src, int nrhs, int accumulate,
              cudaStream_t st, F body) {
  d3m_ctx::Graph* g = nullptr;
  for (auto& c : cache)
    if (c.src == src && c.nrhs == nrhs && c.accumulate == accumulate) g = &c;
  if (!g) {
    if (!h->cap && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
      return set_err(h, D3M_ERR_CUDA, "cannot create the capture stream");
    const int64_t l0 = h->launches;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return set_err(h, D3M_ERR_CUDA, "cudaStreamBeginCapture failed");
    h->capturing = true;
    const int rc = body(h->cap);
    h->capturing = false;
    const cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (rc != D3M_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return set_err(h, D3M_ERR_CUDA, "graph capture failed");
    }
    cudaGraphDestroy(graph);
    if (cache.size() >= 8) {           // bounded cache: drop the oldest
      cudaGraphExecDestroy(cache.front().exec);
      cache.erase(cache.begin());
    }
    cache.push_back({src, nrhs, accumulate, exec, h->launches - l0});
    h->launches = l0;
    g = &cache.back();
  }
  CUDA_TRY(h, cudaGraphLaunch(g->exec, st));
  h->launches += g->launches;
  return D3M_OK;
}

void fill_structure(const Symbolic& S, d3m_info* info) {
  info->n = S.n;
  info->nblk = S.N;
  info->tile = S.b;
  info->nnzb_K = S.nnzb_K;
  info->nblk_L_offdiag = S.nL_off;
  info->etree_depth = S.depth;
  info->max_col_height = S.max_height;
  info->ntiles = S.tcolptr.empty() ? 0 : S.tcolptr.back();
  info->ntile_updates = S.n_tile_updates;
  info->ndep_edges = S.n_edges;
  info->factor_flops = S.factor_flops;
  info->solve_flops_per_rhs = S.solve_flops_rhs;
  info->residual_flops_per_rhs = S.residual_flops_rhs;
  info->prio_tasks = S.n_prio;
  info->residual_bytes_fixed = (double)S.kblk_off.back() * 16.0;
  info->residual_bytes_per_rhs = 3.0 * 16.0 * (double)S.n;
}

int factor_error(d3m_ctx* h) {
  const Ctl& c = *h->h_ctl;
  if (c.err == D3M_ERR_PIVOT)
    return set_err(h, D3M_ERR_PIVOT, "pivot below the breakdown threshold (task " + std::to_string(c.err_task) + ")");
  if (c.err == D3M_ERR_TIMEOUT)
    return set_err(h, D3M_ERR_TIMEOUT, "bounded device wait expired in the factorization queue");
  if (c.err != 0) return set_err(h, c.err, "factorization failed");
  if (c.done != (int64_t)h->S.tasks.size())
    return set_err(h, D3M_ERR_TIMEOUT, "factorization finished " + std::to_string(c.done) + " of " +
                                           std::to_string(h->S.tasks.size()) + " tasks");
  return D3M_OK;
}

}  // namespace

namespace d3m {
// handle accessors for entry points defined in other translation units
int handle_geometry(d3m_handle h, int64_t* n, int32_t* nblk, const int64_t** xoff_orig, const int32_t** m_orig) {
  *n = h->S.n;
  *nblk = h->S.N;
  *xoff_orig = h->xoff_orig;
  *m_orig = h->m_orig;
  return D3M_OK;
}
int handle_error(d3m_handle h, int code, const char* msg) { return set_err(h, code, msg); }
int handle_device(d3m_handle h) { return h->device; }
}  // namespace d3m

extern "C" {

void d3m_default_options(d3m_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = D3M_MIXED_BF16X3;
  o->refine_max_iter = 20;
  o->refine_tol = 1e-12;
  o->timeout_ns = 5000000000LL;
  o->tile = 0;
  o->max_nrhs = 32;
  o->fp64_omega = 0;
  o->debug_flags = 0;
  o->graphs = 0;
  o->prio_slack = 0.08;
  o->refine_fwd_tol = 1e-10;
}

int d3m_order_grid_nd(int32_t nx, int32_t ny, int32_t nz, int32_t* perm) {
  if (!perm) return set_err(nullptr, D3M_ERR_INVALID, "perm is NULL");
  std::vector<int32_t> p;
  int rc = order_grid_nd(nx, ny, nz, p);
  if (rc != D3M_OK) return set_err(nullptr, rc, "grid extents must be positive");
  std::copy(p.begin(), p.end(), perm);
  return D3M_OK;
}

int d3m_analyze(const d3m_pattern* pat, const int32_t* perm, int32_t tile, d3m_info* info) {
  if (!info) return set_err(nullptr, D3M_ERR_INVALID, "info is NULL");
  Symbolic S;
  std::string err;
  int rc = analyze(pat, perm, tile > 0 ? tile : 128, false, S, err);
  if (rc != D3M_OK) return set_err(nullptr, rc, err);
  std::memset(info, 0, sizeof(*info));
  fill_structure(S, info);
  info->omega = NAN;
  info->omega_first = NAN;
  return D3M_OK;
}

int d3m_analyze_opts(const d3m_pattern* pat, const int32_t* perm, const d3m_options* opt, d3m_info* info) {
  if (!info) return set_err(nullptr, D3M_ERR_INVALID, "info is NULL");
  d3m_options o;
  if (opt) o = *opt;
  else d3m_default_options(&o);
  const int prec = o.precision;
  if (prec != D3M_FP64 && prec != D3M_MIXED_BF16X3 && prec != D3M_MIXED_SIMT32 && prec != D3M_MIXED_TF32)
    return set_err(nullptr, D3M_ERR_INVALID, "unknown precision");
  const bool fp64 = prec == D3M_FP64, tc = prec == D3M_MIXED_BF16X3 || prec == D3M_MIXED_TF32;
  const int b = tc ? 128 : 64;
  if (o.tile != 0 && o.tile != b)
    return set_err(nullptr, D3M_ERR_INVALID, "tile must be 0 or " + std::to_string(b) + " for this precision");
  if (!(o.prio_slack >= 0)) o.prio_slack = 0.08;
  if (o.seg_group <= 0) o.seg_group = fp64 ? 1 : (prec == D3M_MIXED_TF32 ? 32 : 8);
  Symbolic S;
  std::string err;
  int rc = analyze(pat, perm, b, true, S, err, o.prio_slack, o.seg_group, o.task_cost, tc ? 16 : 1,
                   prec == D3M_MIXED_TF32);
  if (rc != D3M_OK) return set_err(nullptr, rc, err);
  std::memset(info, 0, sizeof(*info));
  fill_structure(S, info);
  info->omega = NAN;
  info->omega_first = NAN;
  return D3M_OK;
}

}  // extern "C"

// Shared by d3m_create and d3m_create_batch; inst_blk (batched handles) holds the first block
// of every instance in the caller's numbering.
static int create_impl(d3m_handle* out, const d3m_pattern* pat, const int32_t* perm, const d3m_options* opt,
                       const std::vector<int32_t>* inst_blk) {
  if (!out) return set_err(nullptr, D3M_ERR_INVALID, "out is NULL");
  *out = nullptr;
  d3m_ctx* h = new (std::nothrow) d3m_ctx();
  if (!h) return set_err(nullptr, D3M_ERR_OOM, "host allocation failed");
  if (inst_blk) h->inst_blk = *inst_blk;
  if (opt) h->opt = *opt;
  else d3m_default_options(&h->opt);
  const int prec = h->opt.precision;
  if (prec != D3M_FP64 && prec != D3M_MIXED_BF16X3 && prec != D3M_MIXED_SIMT32 && prec != D3M_MIXED_TF32) {
    delete h;
    return set_err(nullptr, D3M_ERR_INVALID, "unknown precision");
  }
  if (h->opt.max_nrhs <= 0) h->opt.max_nrhs = 32;
  if (h->opt.refine_max_iter <= 0) h->opt.refine_max_iter = 20;
  if (!(h->opt.refine_tol > 0)) h->opt.refine_tol = 1e-12;
  if (h->opt.timeout_ns <= 0) h->opt.timeout_ns = 5000000000LL;
  if (!(h->opt.prio_slack >= 0)) h->opt.prio_slack = 0.08;
  if (!(h->opt.refine_fwd_tol >= 0)) h->opt.refine_fwd_tol = 1e-10;
  h->fp64 = (prec == D3M_FP64);
  h->tc = (prec == D3M_MIXED_BF16X3 || prec == D3M_MIXED_TF32);
  h->tf32 = (prec == D3M_MIXED_TF32);
  h->b = h->tc ? 128 : 64;
  if (h->opt.tile != 0 && h->opt.tile != h->b) {
    delete h;
    return set_err(nullptr, D3M_ERR_INVALID, "tile must be 0 or " + std::to_string(h->tc ? 128 : 64) + " for this precision");
  }
  h->csize = h->fp64 ? sizeof(double2) : sizeof(float2);
  if (h->opt.pivot != 0 && h->opt.pivot != 1) {
    delete h;
    return set_err(nullptr, D3M_ERR_INVALID, "pivot must be 0 or 1");
  }
  if (h->opt.pivot && h->tc) {
    delete h;
    return set_err(nullptr, D3M_ERR_INVALID, "pivoting needs a SIMT engine (D3M_FP64 or D3M_MIXED_SIMT32)");
  }
  std::string err;
  // mixed precision: a tile's Schur updates from up to 8 source blocks form one update task (the
  // per-task epilogue through the accumulator dominates short segments), 32 with TF32 (its
  // factorization is bound by DRAM, and every segment boundary writes and reads back the tile's
  // accumulator); FP64 is DFMA bound and keeps one task per source block
  if (h->opt.seg_group <= 0) h->opt.seg_group = h->fp64 ? 1 : (h->tf32 ? 32 : 8);
  // the tensor-core gathers of the solve (split-BF16x3 products, both engines) sum up to 16 items of one
  // destination in tensor memory
  const int ggroup = h->tc ? 16 : 1;
  int rc = analyze(pat, perm, h->b, true, h->S, err, h->opt.prio_slack, h->opt.seg_group, h->opt.task_cost, ggroup,
                   h->tf32);
  if (rc != D3M_OK) {
    delete h;
    return set_err(nullptr, rc, err);
  }
  *out = h;
  const Symbolic& S = h->S;
  const int64_t ntiles = S.ntiles;
  const int64_t ntask = (int64_t)S.tasks.size();
  const int b = h->b;
  const int mr = h->opt.max_nrhs;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(h, D3M_ERR_CUDA, "no CUDA device");
  }
  int cc_major = 0, cc_minor = 0;
  cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, h->device);
  cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, h->device);
  if (cc_major != 10 || cc_minor != 3)
    return set_err(h, D3M_ERR_CUDA, "this library is built for sm_103a (GB300) only; device is sm_" +
                                        std::to_string(cc_major) + std::to_string(cc_minor));
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return set_err(h, D3M_ERR_CUDA, "cannot create the factorization's second stream");
  }
#define ALLOC(ptr, T, count)                                                                     \
  do {                                                                                           \
    ptr = dalloc<T>(h, (size_t)(count));                                                         \
    if (!ptr) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed for " #ptr);                    \
  } while (0)
#define UPLOAD(ptr, vec)                        \
  do {                                          \
    int rc_ = upload(h, &ptr, vec);             \
    if (rc_ != D3M_OK) return rc_;              \
  } while (0)
  // upload stream of a host K (tensor-core engines): its progress counter is written by stream
  // memory operations, which the persistent factorization polls; without them a host K is
  // copied before the factorization starts
  if (h->tc && write_value32()) {
    ALLOC(h->k_arrived, int32_t, 1);
    if (cudaStreamCreateWithFlags(&h->kup, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreateWithFlags(&h->ev_kup0, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&h->ev_kup1, cudaEventDisableTiming) == cudaSuccess &&
        write_value32()((CUstream)h->kup, (CUdeviceptr)h->k_arrived, 0u, 0u) == CUDA_SUCCESS &&
        cudaStreamSynchronize(h->kup) == cudaSuccess)
      h->kup_ok = true;
    cudaGetLastError();
  }
  // factorization (h->K, the copy target of a host K, is allocated by the first call that needs it)
  UPLOAD(h->tasks, S.tasks);
  UPLOAD(h->klist, S.klist);
  {
    std::vector<int32_t> nd = S.ndeps;
    if ((h->opt.debug_flags & D3M_DEBUG_STALL_LAST_TASK) && !nd.empty()) nd.back() += 1;
    UPLOAD(h->ndeps, nd);
  }
  ALLOC(h->cnt, int32_t, ntask);
  if (h->opt.debug_flags & D3M_DEBUG_TRACE) {
    ALLOC(h->trace, int64_t, 10 * ntask);
    CUDA_TRY(h, cudaMemset(h->trace, 0, 10 * ntask * sizeof(int64_t)));
  }
  UPLOAD(h->succ_ptr, S.succ_ptr);
  UPLOAD(h->succ, S.succ);
  ALLOC(h->ready, int32_t, ntask);
  UPLOAD(h->init_ready, S.init_ready);
  ALLOC(h->ready_hi, int32_t, std::max<int64_t>(1, S.n_prio));
  UPLOAD(h->init_ready_hi, S.init_ready_hi);
  ALLOC(h->ctl, Ctl, 1);
  ALLOC(h->ctl0, Ctl, 1);
  {
    Ctl c0;
    std::memset(&c0, 0, sizeof c0);
    c0.tail = (int32_t)S.init_ready.size();
    c0.tail_hi = (int32_t)S.init_ready_hi.size();
    c0.min_piv_bits = 0x7f7fffffu;   // FLT_MAX
    c0.max_piv_bits = 0u;
    CUDA_TRY(h, cudaMemcpy(h->ctl0, &c0, sizeof c0, cudaMemcpyHostToDevice));
  }
  CUDA_TRY(h, cudaMallocHost(&h->h_ctl, sizeof(Ctl)));
  std::memset(h->h_ctl, 0, sizeof(Ctl));
  h->L = dalloc<unsigned char>(h, (size_t)ntiles * b * b * h->csize);
  h->Linv = dalloc<unsigned char>(h, (size_t)S.NT * b * b * h->csize);
  h->D = dalloc<unsigned char>(h, (size_t)S.NT * b * h->csize);
  h->Sacc = dalloc<unsigned char>(h, (size_t)std::max<int64_t>(1, S.n_acc) * b * b * h->csize);
  if (!h->L || !h->Linv || !h->D || !h->Sacc) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed for the factor tiles");
  if (h->opt.pivot) {
    h->E = dalloc<unsigned char>(h, (size_t)S.NT * b * h->csize);
    h->piv = dalloc<int32_t>(h, (size_t)S.NT * b);
    if (!h->E || !h->piv) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed for the pivot blocks");
    CUDA_TRY(h, cudaMemset(h->E, 0, (size_t)S.NT * b * h->csize));
  }
  if (h->tc) {
    // operand planes, 8 bytes per complex element either way: bf16 A: [tile][2 splits][2 planes]
    // [b rows][b], B: [tile][2][2][b][b]; tf32 A and B: [tile][2 planes][b rows][b]
    h->opA = dalloc<unsigned char>(h, (size_t)ntiles * 4 * b * b * 2);
    h->opB = dalloc<unsigned char>(h, (size_t)ntiles * 4 * b * b * 2);
    if (!h->opA || !h->opB) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed for the tensor-core operands");
    std::string e2;
    if (tc_make_maps(h->opA, h->opB, ntiles, h->tf32, &h->maps, e2) != 0) return set_err(h, D3M_ERR_CUDA, e2);
    // the solve's off-block products run on the tensor cores from bf16 split planes of L: the
    // BF16x3 engine's own opA, or (TF32) a copy in that layout written beside the tf32 planes
    if (h->tf32) {
      h->opS = dalloc<unsigned char>(h, (size_t)ntiles * 4 * b * b * 2);
      if (!h->opS) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed for the solve operand planes");
    }
    if (gather_tc_make_maps(h->tf32 ? h->opS : h->opA, ntiles, &h->gmaps, e2) != 0) return set_err(h, D3M_ERR_CUDA, e2);
    h->gather_tc = true;
  }
  // solve
  UPLOAD(h->fwd_items, S.fwd_items);
  UPLOAD(h->bwd_items, S.bwd_items);
  UPLOAD(h->fwd_groups, S.fwd_groups);
  UPLOAD(h->bwd_groups, S.bwd_groups);
  UPLOAD(h->fwd_slot, S.fwd_slot_ptr);
  UPLOAD(h->bwd_slot, S.bwd_slot_ptr);
  {
    std::vector<int32_t> lb;
    h->lev_ptr.assign(1, 0);
    for (const auto& l : S.lev_blocks) {
      lb.insert(lb.end(), l.begin(), l.end());
      h->lev_ptr.push_back((int64_t)lb.size());
    }
    UPLOAD(h->lev_blocks, lb);
    std::vector<int32_t> lt;
    h->lev_tile_ptr.assign(1, 0);
    for (const auto& l : S.lev_blocks) {
      for (int k : l)
        for (int I = S.tstart[k]; I < S.tstart[k + 1]; ++I) lt.push_back(I);
      h->lev_tile_ptr.push_back((int64_t)lt.size());
    }
    UPLOAD(h->lev_tiles, lt);
    h->lev_maxnt.clear();
    for (const auto& l : S.lev_blocks) {
      int mx = 1;
      for (int k : l) mx = std::max(mx, S.ntile[k]);
      h->lev_maxnt.push_back(mx);
    }
    h->lev_maxcnt_fwd.clear();
    h->lev_maxcnt_bwd.clear();
    for (const auto& l : S.lev_blocks) {
      int64_t mf = 0, mb = 0;
      for (int k : l)
        for (int I = S.tstart[k]; I < S.tstart[k + 1]; ++I) {
          mf = std::max<int64_t>(mf, S.fwd_slot_ptr[I] >> 32);
          mb = std::max<int64_t>(mb, (S.bwd_slot_ptr[I] >> 32) * (b / 64));
        }
      h->lev_maxcnt_fwd.push_back((int32_t)mf);
      h->lev_maxcnt_bwd.push_back((int32_t)mb);
    }
    std::vector<int64_t> p2o(S.npad, -1);
    for (int k = 0; k < S.N; ++k)
      for (int u = 0; u < S.m[k]; ++u) p2o[S.xoff[k] + u] = S.xoff_orig[S.perm[k]] + u;
    UPLOAD(h->pad2orig, p2o);
    int mrows = 0, mnt = 0;
    for (int k = 0; k < S.N; ++k) {
      mrows = std::max(mrows, S.ntile[k] * b);
      mnt = std::max(mnt, S.ntile[k]);
    }
    h->max_rows = mrows;
    // the in-block sweep kernels keep one block's running vector (1 rhs at least) and two
    // staged half tiles in shared memory, and list at most 512 tile jobs per block
    const size_t need = h->csize * (2 * (size_t)64 * (b + 1) + (size_t)mrows + (size_t)b);
    if (need > 220 * 1024 || (int64_t)mnt * (mnt + 1) / 2 * (b / 64) > 512 || mnt > 32)
      return set_err(h, D3M_ERR_INVALID, "interface block too large for the solve kernels (m = " +
                                             std::to_string(mrows) + ")");
  }
  UPLOAD(h->tstart, S.tstart);
  UPLOAD(h->tcolptr, S.tcolptr);
  // mixed precision with blocks of at most 512 rows: build the diagonal blocks' inverses
  h->use_inv = !h->fp64 && h->max_rows <= 512;
  if (h->use_inv) {
    std::vector<int64_t> off(S.N, 0), offT(S.N, 0);
    std::vector<int2> work;
    int64_t ninv = 0, ninvT = 0;
    for (int k = 0; k < S.N; ++k) {
      const int nt = S.ntile[k];
      off[k] = ninv;
      offT[k] = ninvT;
      ninv += (int64_t)nt * (nt - 1) / 2;
      ninvT += (int64_t)nt * (nt + 1) / 2;
      for (int tq = 0; tq < nt; ++tq) work.push_back(make_int2(k, tq));
    }
    // longest columns first (tile products: sum over t > tq of t - tq + 1), so that the long
    // sequential columns start in the first wave and the short ones fill the gaps after them
    auto cost = [&](const int2& w) {
      const int nt = S.ntile[w.x];
      int64_t c = 0;
      for (int t = w.y + 1; t < nt; ++t) c += t - w.y + 1;
      return c;
    };
    std::stable_sort(work.begin(), work.end(), [&](const int2& a, const int2& c) { return cost(a) > cost(c); });
    UPLOAD(h->inv_off, off);
    UPLOAD(h->invT_off, offT);
    UPLOAD(h->inv_work, work);
    h->n_inv_work = (int)work.size();
    h->Inv = dalloc<unsigned char>(h, (size_t)std::max<int64_t>(1, ninv) * b * b * h->csize);
    h->InvT = dalloc<unsigned char>(h, (size_t)std::max<int64_t>(1, ninvT) * b * b * h->csize);
    if (!h->Inv || !h->InvT) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed for the block inverses");
  }
  h->Y = dalloc<unsigned char>(h, (size_t)S.npad * mr * h->csize);
  h->P = dalloc<unsigned char>(h, (size_t)std::max<int64_t>(1, S.max_level_groups) * (b / 64) * b * mr * h->csize);
  if (!h->Y || !h->P) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed for the solve workspace");
  // refinement + residual
  ALLOC(h->d_b, double2, S.n * mr);
  ALLOC(h->d_x, double2, S.n * mr);
  ALLOC(h->d_xbest, double2, S.n * mr);
  ALLOC(h->d_r, double2, S.n * mr);
  UPLOAD(h->kblk_off, S.kblk_off);
  UPLOAD(h->res_ptr, S.res_ptr);
  UPLOAD(h->res_blk, S.res_blk);
  UPLOAD(h->res_src, S.res_src);
  UPLOAD(h->res_tr, S.res_tr);
  {
    // residual digit planes: per contribution e of row block f from block g, ceil(m_f / 128) row
    // tiles x ceil(m_g / 32) chunks x 2 parts x 9 digits planes of 128 x 32 bf16; per block g,
    // ceil(m_g / 32) chunks x 2 x 9 planes of 64 x 32 bf16 for the digits of x
    const int64_t nres = (int64_t)S.res_blk.size();
    std::vector<int64_t> ksp(nres), xsp(S.N);
    std::vector<int32_t> rrow(nres), brow(S.nnzb_K), bcol(S.nnzb_K);
    int64_t pa = 0, pb = 0;
    for (int f = 0; f < S.N; ++f)
      for (int64_t e = S.res_ptr[f]; e < S.res_ptr[f + 1]; ++e) {
        ksp[e] = pa;
        rrow[e] = f;
        pa += (int64_t)((S.m_orig[f] + 127) / 128) * ((S.m_orig[S.res_src[e]] + 31) / 32) * 2 * kResidDigits;
      }
    for (int g = 0; g < S.N; ++g) {
      xsp[g] = pb;
      pb += (int64_t)((S.m_orig[g] + 31) / 32) * 2 * kResidDigits;
      for (int64_t q = S.colptr[g]; q < S.colptr[g + 1]; ++q) {
        brow[q] = S.rowidx[q];
        bcol[q] = g;
      }
      for (int r = 0; r < S.m_orig[g]; r += 128) h->rtile_host.push_back(make_int2(g, r / 128));
      h->max_rtiles = std::max(h->max_rtiles, (S.m_orig[g] + 127) / 128);
    }
    if (pa >= (int64_t)1 << 31 || pb >= (int64_t)1 << 31)
      return set_err(h, D3M_ERR_INVALID, "K too large for the residual's digit planes (2^31 planes)");
    ResidualTc& r = h->rtc;
    int64_t* d_ksp = nullptr;
    int64_t* d_xsp = nullptr;
    int32_t *d_rrow = nullptr, *d_brow = nullptr, *d_bcol = nullptr;
    int2* d_rt = nullptr;
    UPLOAD(d_ksp, ksp);
    UPLOAD(d_xsp, xsp);
    UPLOAD(d_rrow, rrow);
    UPLOAD(d_brow, brow);
    UPLOAD(d_bcol, bcol);
    UPLOAD(d_rt, h->rtile_host);
    {
      // the two residual contributions of every stored block (as stored, and transposed)
      std::vector<int32_t> eu(S.nnzb_K, -1), et(S.nnzb_K, -1);
      for (int64_t e = 0; e < nres; ++e) (S.res_tr[e] ? et : eu)[S.res_blk[e]] = (int32_t)e;
      int32_t *d_eu = nullptr, *d_et = nullptr;
      UPLOAD(d_eu, eu);
      UPLOAD(d_et, et);
      r.blk_eu = d_eu;
      r.blk_et = d_et;
    }
    r.ks_plane = d_ksp;
    r.xs_plane = d_xsp;
    r.res_row = d_rrow;
    r.blk_row = d_brow;
    r.blk_col = d_bcol;
    r.rtiles = d_rt;
    int nr_grp = 8;
    const int ngrp = resid_tc_groups(mr, &nr_grp);   // the most groups any nrhs <= max_nrhs uses
    r.xs_total = pb;
    r.nblk = S.N;
    ALLOC(r.kdig, unsigned short, pa * 128 * 32);
    ALLOC(r.xdig, unsigned short, pb * ngrp * 64 * 32);
    ALLOC(r.Kmax_bits, unsigned long long, S.nnzb_K);
    ALLOC(r.Kdiag, double2, S.n);
    ALLOC(r.rowsum, float, S.n);
    ALLOC(r.xT, int, (size_t)ngrp * S.N * 32);
    std::string e3;
    if (resid_tc_make_maps(r.kdig, pa, r.xdig, pb * ngrp, &h->rtc_maps, e3) != 0) return set_err(h, D3M_ERR_CUDA, e3);
  }
  UPLOAD(h->m_orig, S.m_orig);
  UPLOAD(h->xoff_orig, S.xoff_orig);
  {
    std::vector<int32_t> bc(S.nnzb_K);
    for (int g = 0; g < S.N; ++g)
      for (int64_t p = S.colptr[g]; p < S.colptr[g + 1]; ++p) bc[p] = g;
    UPLOAD(h->blk_col, bc);
  }
  UPLOAD(h->rowidx, S.rowidx);
  UPLOAD(h->colptr, S.colptr);
  {
    // instance of every block (caller numbering); one instance unless batched
    std::vector<int32_t> ib(S.N, 0);
    if (h->inst_blk.empty()) h->inst_blk = {0, S.N};
    h->ninst = (int)h->inst_blk.size() - 1;
    for (int i = 0; i < h->ninst; ++i)
      for (int f = h->inst_blk[i]; f < h->inst_blk[i + 1]; ++f) ib[f] = i;
    UPLOAD(h->inst, ib);
    std::vector<int32_t> ti(S.NT, 0);
    for (int I = 0; I < S.NT; ++I) ti[I] = ib[S.perm[S.tblk[I]]];
    UPLOAD(h->tinst, ti);
    ALLOC(h->done, int, h->ninst);
    CUDA_TRY(h, cudaMemset(h->done, 0, h->ninst * sizeof(int)));
  }
  ALLOC(h->norms, unsigned, 3 * (size_t)h->ninst * mr + h->ninst);
  ALLOC(h->omega_dev, double, (size_t)h->ninst * mr);
  ALLOC(h->stat_dev, double, 3);
  ALLOC(h->dmax, unsigned, (size_t)h->ninst * mr);
  ALLOC(h->dprev, float, (size_t)h->ninst * mr);
  ALLOC(h->sweep_status, int, 1);
  CUDA_TRY(h, cudaMemset(h->sweep_status, 0, sizeof(int)));
  ALLOC(h->contract, double2, S.N);
  CUDA_TRY(h, cudaMallocHost(&h->h_stat, 3 * sizeof(double)));
#undef ALLOC
#undef UPLOAD
  return D3M_OK;
}

extern "C" {

int d3m_create(d3m_handle* out, const d3m_pattern* pat, const int32_t* perm, const d3m_options* opt,
               void* stream) {
  (void)stream;
  return create_impl(out, pat, perm, opt, nullptr);
}

int d3m_create_batch(d3m_handle* out, int32_t count, const d3m_pattern* pats, const int32_t* const* perms,
                     const d3m_options* opt, void* stream) {
  (void)stream;
  if (!out) return set_err(nullptr, D3M_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (count < 1 || !pats) return set_err(nullptr, D3M_ERR_INVALID, "count must be >= 1 and pats non-NULL");
  // block-diagonal union: instance i's blocks follow those of instances < i
  std::vector<int32_t> bsz, rowidx, perm, inst_blk(1, 0);
  std::vector<int64_t> colptr(1, 0);
  for (int i = 0; i < count; ++i) {
    const d3m_pattern& q = pats[i];
    if (q.nblk < 1 || !q.colptr || !q.rowidx || (!q.blk_size && q.m < 1))
      return set_err(nullptr, D3M_ERR_INVALID, "instance " + std::to_string(i) + ": bad pattern");
    const int32_t off = inst_blk.back();
    const int64_t eoff = colptr.back();
    if (q.colptr[0] != 0 || q.colptr[q.nblk] < q.colptr[0])
      return set_err(nullptr, D3M_ERR_INVALID, "instance " + std::to_string(i) + ": bad colptr");
    for (int k = 0; k < q.nblk; ++k) {
      bsz.push_back(q.blk_size ? q.blk_size[k] : q.m);
      if (q.colptr[k + 1] < q.colptr[k])
        return set_err(nullptr, D3M_ERR_INVALID, "instance " + std::to_string(i) + ": bad colptr");
      colptr.push_back(eoff + q.colptr[k + 1]);
    }
    for (int64_t e = 0; e < q.colptr[q.nblk]; ++e) {
      const int32_t r = q.rowidx[e];
      // out-of-range rows are left for the symbolic analysis to reject, but must not alias
      // another instance's blocks
      rowidx.push_back(r >= 0 && r < q.nblk ? off + r : -1);
    }
    const int32_t* pi = perms ? perms[i] : nullptr;
    for (int k = 0; k < q.nblk; ++k) {
      const int32_t v = pi ? pi[k] : k;
      perm.push_back(v >= 0 && v < q.nblk ? off + v : -1);
    }
    inst_blk.push_back(off + q.nblk);
  }
  d3m_pattern u;
  u.nblk = inst_blk.back();
  u.m = 0;
  u.blk_size = bsz.data();
  u.colptr = colptr.data();
  u.rowidx = rowidx.data();
  return create_impl(out, &u, perm.data(), opt, &inst_blk);
}

int d3m_get_instance_omega(d3m_handle h, double* host_out, void* stream) {
  if (!h || !host_out) return set_err(h, D3M_ERR_INVALID, "handle or output is NULL");
  const int mr = h->opt.max_nrhs;
  std::vector<double> w((size_t)h->ninst * mr, NAN);
  CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)stream));
  if (h->omega_valid && h->last_nrhs > 0)
    CUDA_TRY(h, cudaMemcpy(w.data(), h->omega_dev, w.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int i = 0; i < h->ninst; ++i) {
    double o = h->omega_valid && h->last_nrhs > 0 ? 0.0 : NAN;
    for (int j = 0; j < h->last_nrhs && h->omega_valid; ++j) o = std::max(o, w[(size_t)i * mr + j]);
    host_out[i] = o;
  }
  return D3M_OK;
}

// parameters of the tensor-core residual (digit planes and geometry are fixed at create time)
static ResidualTc resid_params(d3m_ctx* h, const double2* K) {
  ResidualTc p = h->rtc;
  p.K = K;
  p.kblk_off = h->kblk_off;
  p.m_orig = h->m_orig;
  p.xoff_orig = h->xoff_orig;
  p.res_ptr = h->res_ptr;
  p.res_src = h->res_src;
  p.res_blk = h->res_blk;
  p.res_tr = h->res_tr;
  p.n = h->S.n;
  const int mr = h->opt.max_nrhs, ni = h->ninst;
  p.inst = h->inst;
  p.done = h->done;
  p.ld_norm = mr;
  p.rmax = h->norms;
  p.xmax = h->norms + (size_t)ni * mr;
  p.bmax = h->norms + 2 * (size_t)ni * mr;
  p.kmax = h->norms + 3 * (size_t)ni * mr;
  p.status = h->sweep_status;
  p.timeout_ns = h->opt.timeout_ns;
  return p;
}

// the launch sequence of one factorization (copy of K, queue reset, ||K_i||, persistent kernel,
// status read-back into pinned memory)
static int enqueue_factor(d3m_ctx* h, const void* Kin, bool kdev, cudaStream_t st) {
  const Symbolic& S = h->S;
  const int64_t ntiles = (int64_t)S.tasks.size();   // all tasks (final + update)
  const size_t kbytes = (size_t)S.kblk_off.back() * sizeof(double2);
  // a (16-byte aligned) device K is read in place by the two kernels that use it (the
  // factorization and the norm/split of K, both below); a host K is copied first
  const double2* Ksrc = h->K;
  // a page-locked host K is uploaded on a stream of its own in the analysis' order (the blocks of
  // the first columns to be eliminated first) while the factorization runs; a task that reads a
  // block waits for it
  const bool kup = !kdev && h->kup_ok && !h->capturing && is_pinned_host_ptr(Kin);
  if (kdev && ((uintptr_t)Kin & 15) == 0) Ksrc = static_cast<const double2*>(Kin);
  else if (!kup) CUDA_TRY(h, cudaMemcpyAsync(h->K, Kin, kbytes, kdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  if (kup) {
    CUDA_TRY(h, cudaMemsetAsync(h->k_arrived, 0, sizeof(int32_t), st));
    CUDA_TRY(h, cudaEventRecord(h->ev_kup0, st));
    CUDA_TRY(h, cudaStreamWaitEvent(h->kup, h->ev_kup0, 0));
    const double2* Kh = static_cast<const double2*>(Kin);
    for (size_t r = 0; r < S.kc_off.size(); ++r) {
      CUDA_TRY(h, cudaMemcpyAsync(h->K + S.kc_off[r], Kh + S.kc_off[r], (size_t)S.kc_len[r] * sizeof(double2),
                                  cudaMemcpyHostToDevice, h->kup));
      if (write_value32()((CUstream)h->kup, (CUdeviceptr)h->k_arrived, (cuuint32_t)S.kc_seq_end[r], 0u) != CUDA_SUCCESS)
        return set_err(h, D3M_ERR_CUDA, "cuStreamWriteValue32 failed during the upload of K");
    }
    CUDA_TRY(h, cudaEventRecord(h->ev_kup1, h->kup));
  }
  // reset the task graph state
  CUDA_TRY(h, cudaMemcpyAsync(h->cnt, h->ndeps, ntiles * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(h, cudaMemsetAsync(h->ready, 0xff, ntiles * sizeof(int32_t), st));
  const int n0 = (int)S.init_ready.size();
  if (n0 > 0) CUDA_TRY(h, cudaMemcpyAsync(h->ready, h->init_ready, n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(h, cudaMemsetAsync(h->ready_hi, 0xff, std::max<int64_t>(1, S.n_prio) * sizeof(int32_t), st));
  const int n0h = (int)S.init_ready_hi.size();
  if (n0h > 0)
    CUDA_TRY(h, cudaMemcpyAsync(h->ready_hi, h->init_ready_hi, n0h * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(h, cudaMemcpyAsync(h->ctl, h->ctl0, sizeof(Ctl), cudaMemcpyDeviceToDevice, st));
  int rc = 0;
  FactorParams p;
  p.tasks = h->tasks;
  p.klist = h->klist;
  p.cnt = h->cnt;
  p.succ_ptr = h->succ_ptr;
  p.succ = h->succ;
  p.ready = h->ready;
  p.ready_hi = h->ready_hi;
  p.n_norm = (int32_t)(ntiles - S.n_prio);
  p.ctl = h->ctl;
  p.ntasks = (int32_t)ntiles;
  p.b = h->b;
  p.K = Ksrc;
  p.L = h->L;
  p.Linv = h->Linv;
  p.D = h->D;
  p.opA = h->opA;
  p.opB = h->opB;
  p.opS = h->opS;
  p.k_arrived = kup ? h->k_arrived : nullptr;
  p.Sacc = h->Sacc;
  p.trace = h->trace;
  p.timeout_ns = h->opt.timeout_ns;
  p.piv_tol = 1e3 * (h->fp64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08);
  p.pivot = h->opt.pivot;
  p.E = h->E;
  p.piv = h->piv;
  if (h->trace) CUDA_TRY(h, cudaMemsetAsync(h->trace, 0xff, (size_t)10 * ntiles * sizeof(int64_t), st));
  ev_begin(h, d3m_ctx::EV_FACTOR, st);
  if (h->tc) rc = launch_factor_tc(p, h->maps, h->tf32, h->nsm, st);
  else rc = launch_factor_simt(p, h->fp64, h->nsm, st);
  if (rc) return set_err(h, D3M_ERR_CUDA, std::string("factor launch: ") + cudaGetErrorString((cudaError_t)rc));
  ev_end(h, d3m_ctx::EV_FACTOR, st);
  h->launches += 1;
  if (kup) CUDA_TRY(h, cudaStreamWaitEvent(st, h->ev_kup1, 0));   // the whole of K before the kernels below
  // ||K_i||_inf and the digit planes of K (for the residual) on a second stream, concurrently
  // with the block inverses: the persistent factorization holds every SM, the smaller kernels
  // share them
  CUDA_TRY(h, cudaEventRecord(h->ev_fork, st));
  CUDA_TRY(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  {
    ResidualTc rp = resid_params(h, Ksrc);
    CUDA_TRY(h, cudaMemsetAsync(rp.kmax, 0, h->ninst * sizeof(unsigned), h->side));
    rc = launch_kdigits(rp, (int)S.nnzb_K, (int)S.res_blk.size(), h->max_rtiles, S.N, h->side);
    if (rc) return set_err(h, D3M_ERR_CUDA, std::string("K digit launch: ") + cudaGetErrorString((cudaError_t)rc));
    h->launches += 3;
  }
  CUDA_TRY(h, cudaEventRecord(h->ev_join, h->side));
  if (h->use_inv && h->n_inv_work > 0) {
    rc = launch_inv_build(h->inv_work, h->n_inv_work, h->tstart, h->tcolptr, h->inv_off, h->invT_off, h->L, h->Linv,
                          h->Inv, h->InvT, h->b, st);
    if (rc) return set_err(h, D3M_ERR_CUDA, std::string("block inverse launch: ") + cudaGetErrorString((cudaError_t)rc));
    h->launches += 1;
  }
  CUDA_TRY(h, cudaStreamWaitEvent(st, h->ev_join, 0));
  CUDA_TRY(h, cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  return D3M_OK;
}

int d3m_factor(d3m_handle h, const void* Kin, void* stream) {
  if (!h) return set_err(nullptr, D3M_ERR_INVALID, "handle is NULL");
  if (!Kin) return set_err(h, D3M_ERR_INVALID, "K is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  const bool kdev = is_device_ptr(Kin);
  if ((!kdev || ((uintptr_t)Kin & 15) != 0) && !h->K) {
    // a host (or misaligned device) K is copied into a buffer of the handle, allocated on first use
    h->K = dalloc<double2>(h, (size_t)h->S.kblk_off.back());
    if (!h->K) return set_err(h, D3M_ERR_OOM, "cudaMalloc failed for the copy of K");
  }
  int rc;
  if (h->opt.graphs && kdev) {
    // whole sequence as one graph; the event pair then spans the copy of K and ||K|| as well
    ev_begin(h, d3m_ctx::EV_FACTOR, st);
    rc = graph_run(h, h->g_factor, Kin, 0, 0, st, [&](cudaStream_t cs) { return enqueue_factor(h, Kin, true, cs); });
    ev_end(h, d3m_ctx::EV_FACTOR, st);
  } else {
    rc = enqueue_factor(h, Kin, kdev, st);
  }
  if (rc != D3M_OK) return rc;
  h->factored = true;
  h->factor_checked = false;
  h->last_status = D3M_OK;
  return D3M_OK;
}

static int sweep(d3m_ctx* h, const double2* src, double2* dst, int nrhs, int accumulate, cudaStream_t st) {
  const Symbolic& S = h->S;
  SweepLaunch a;
  a.status = h->sweep_status;
  a.b = h->b;
  a.nrhs = nrhs;
  a.nlevels = S.nlevels;
  a.max_rows = h->max_rows;
  a.accumulate = accumulate;
  a.n = S.n;
  a.npad = S.npad;
  a.src = src;
  a.dst = dst;
  a.pad2orig = h->pad2orig;
  a.L = h->L;
  a.Linv = h->Linv;
  a.D = h->D;
  a.Y = h->Y;
  a.P = h->P;
  a.fwd_group_ptr = S.fwd_group_ptr.data();
  a.bwd_group_ptr = S.bwd_group_ptr.data();
  a.fwd_groups = h->fwd_groups;
  a.bwd_groups = h->bwd_groups;
  a.fwd_items = h->fwd_items;
  a.bwd_items = h->bwd_items;
  a.fwd_slot_ptr = h->fwd_slot;
  a.bwd_slot_ptr = h->bwd_slot;
  a.lev_blocks = h->lev_blocks;
  a.lev_ptr = h->lev_ptr.data();
  a.lev_tiles = h->lev_tiles;
  a.lev_tile_ptr = h->lev_tile_ptr.data();
  a.tstart = h->tstart;
  a.tcolptr = h->tcolptr;
  a.lev_maxnt = h->lev_maxnt.data();
  a.lev_maxcnt_fwd = h->lev_maxcnt_fwd.data();
  a.lev_maxcnt_bwd = h->lev_maxcnt_bwd.data();
  a.Inv = h->use_inv ? h->Inv : nullptr;
  a.inv_off = h->inv_off;
  a.InvT = h->InvT;
  a.invT_off = h->invT_off;
  a.done = h->done;
  a.tinst = h->tinst;
  a.dmax = h->dmax;
  a.ld_norm = h->opt.max_nrhs;
  a.tcmaps = h->gather_tc ? &h->gmaps : nullptr;
  a.E = h->E;
  a.nsm = h->nsm;
  ev_begin(h, d3m_ctx::EV_SWEEP, st);
  int rc = launch_sweep(a, h->fp64, st);
  if (rc) return set_err(h, D3M_ERR_CUDA, std::string("sweep launch: ") + cudaGetErrorString((cudaError_t)rc));
  ev_end(h, d3m_ctx::EV_SWEEP, st);
  h->launches += a.launches;
  return D3M_OK;
}

// r = b - K x and omega (device); returns D3M_OK or a launch error
static int residual_omega(d3m_ctx* h, const double2* X, const double2* B, int nrhs, cudaStream_t st) {
  const int mr = h->opt.max_nrhs, ni = h->ninst;
  CUDA_TRY(h, cudaMemsetAsync(h->norms, 0, 3 * (size_t)ni * mr * sizeof(unsigned), st));
  ResidualTc rp = resid_params(h, nullptr);
  ev_begin(h, d3m_ctx::EV_RESID, st);
  int64_t nl = 0;
  int rc = launch_resid_tc(rp, h->rtc_maps, X, B, h->d_r, nrhs, (int)h->rtile_host.size(), h->S.N, st, &nl);
  if (rc) return set_err(h, D3M_ERR_CUDA, std::string("residual launch: ") + cudaGetErrorString((cudaError_t)rc));
  ev_end(h, d3m_ctx::EV_RESID, st);
  h->launches += nl;
  rc = launch_omega(rp.rmax, rp.xmax, rp.bmax, rp.kmax, h->dmax, h->dprev, ni, mr, nrhs, h->done, h->opt.refine_tol,
                    h->opt.refine_fwd_tol, h->omega_dev, h->stat_dev, st);
  h->last_nrhs = nrhs;
  if (rc) return set_err(h, D3M_ERR_CUDA, std::string("omega launch: ") + cudaGetErrorString((cudaError_t)rc));
  h->launches += 2;
  return D3M_OK;
}

static int solve_impl(d3m_ctx* h, const void* Bin, void* Xout, int nrhs, cudaStream_t st) {
  if (!Bin || !Xout) return set_err(h, D3M_ERR_INVALID, "B or X is NULL");
  if (nrhs < 1 || nrhs > h->opt.max_nrhs)
    return set_err(h, D3M_ERR_INVALID, "nrhs out of range [1, max_nrhs]");
  if (!h->factored) return set_err(h, D3M_ERR_STATE, "solve before factor");
  if (!h->factor_checked) {
    // the first solve after a factorization reads its status (one synchronization)
    CUDA_TRY(h, cudaStreamSynchronize(st));
    h->factor_checked = true;
    int fe = factor_error(h);
    if (fe != D3M_OK) {
      h->last_status = fe;
      h->factored = false;
      return fe;
    }
  }
  const Symbolic& S = h->S;
  const size_t vbytes = (size_t)S.n * nrhs * sizeof(double2);
  const bool bdev = is_device_ptr(Bin), xdev = is_device_ptr(Xout);
  if (Bin == (const void*)Xout) return set_err(h, D3M_ERR_INVALID, "B and X may not alias");
  const bool graphs = h->opt.graphs != 0;
  const double2* B = (const double2*)Bin;
  if (!bdev || graphs) {
    // host B, or graph replay (captured launches read the library's own buffers)
    CUDA_TRY(h, cudaMemcpyAsync(h->d_b, Bin, vbytes, bdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    B = h->d_b;
  }
  double2* X = (xdev && !graphs) ? (double2*)Xout : h->d_x;
  h->omega = NAN;
  h->omega_first = NAN;
  h->omega_valid = 0;
  h->refine_iters = 0;
  CUDA_TRY(h, cudaMemsetAsync(h->done, 0, h->ninst * sizeof(int), st));   // every instance refines
  CUDA_TRY(h, cudaMemsetAsync(h->dprev, 0, (size_t)h->ninst * h->opt.max_nrhs * sizeof(float), st));
  ev_begin(h, d3m_ctx::EV_SOLVE, st);
  int status = D3M_OK;
  // one refinement step: x (+)= solve(src); r = b - K x and omega (FP64); omega -> pinned host
  auto step = [&](const double2* src, int acc, bool resid, cudaStream_t cs) -> int {
    CUDA_TRY(h, cudaMemsetAsync(h->dmax, 0, (size_t)h->ninst * h->opt.max_nrhs * sizeof(unsigned), cs));
    int rc = sweep(h, src, X, nrhs, acc, cs);
    if (rc) return rc;
    if (!resid) return D3M_OK;
    rc = residual_omega(h, X, B, nrhs, cs);
    if (rc) return rc;
    CUDA_TRY(h, cudaMemcpyAsync(h->h_stat, h->stat_dev, 3 * sizeof(double), cudaMemcpyDeviceToHost, cs));
    return D3M_OK;
  };
  auto run_step = [&](const double2* src, int acc, bool resid) -> int {
    if (!graphs) return step(src, acc, resid, st);
    return graph_run(h, h->g_solve, src, nrhs, acc | (resid ? 2 : 0), st,
                     [&](cudaStream_t cs) { return step(src, acc, resid, cs); });
  };
  if (h->fp64) {
    int rc = run_step(B, 0, h->opt.fp64_omega != 0);
    if (rc) return rc;
    h->refine_iters = 1;
    if (h->opt.fp64_omega) {
      CUDA_TRY(h, cudaStreamSynchronize(st));
      h->omega = h->omega_first = *h->h_stat;
      h->omega_valid = 1;
    }
  } else {
    int rc = 0;
    double best = INFINITY;
    std::vector<double> hist;
    const double2* src = B;
    for (int it = 0; it < h->opt.refine_max_iter; ++it) {
      rc = run_step(src, it > 0 ? 1 : 0, true);             // x (+)= solve(r); r = b - K x, omega
      if (rc) return rc;
      CUDA_TRY(h, cudaStreamSynchronize(st));
      const double w = h->h_stat[0];
      const bool all_done = h->h_stat[1] == 0.0;
      h->refine_iters = it + 1;
      if (it == 0) h->omega_first = w;
      hist.push_back(h->h_stat[2]);   // progress of the instances still open
      if (w < best) {
        best = w;
        if (w > h->opt.refine_tol)
          CUDA_TRY(h, cudaMemcpyAsync(h->d_xbest, X, vbytes, cudaMemcpyDeviceToDevice, st));
      }
      h->omega = w;
      h->omega_valid = 1;
      if (all_done) break;
      const size_t k = hist.size();
      const bool stagnated = (k >= 3 && !(hist[k - 1] <= 0.5 * hist[k - 3])) || !std::isfinite(w);
      if (stagnated || it + 1 == h->opt.refine_max_iter) {
        if (w > best) {
          CUDA_TRY(h, cudaMemcpyAsync(X, h->d_xbest, vbytes, cudaMemcpyDeviceToDevice, st));
          h->omega = best;
        }
        status = D3M_ERR_NOT_CONVERGED;
        set_err(h, status, "refinement did not reach the tolerance (omega " + std::to_string(h->omega) + ")");
        break;
      }
      src = h->d_r;
    }
  }
  ev_end(h, d3m_ctx::EV_SOLVE, st);
  if ((void*)X != Xout)
    CUDA_TRY(h, cudaMemcpyAsync(Xout, X, vbytes, xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  if (!h->fp64 || h->opt.fp64_omega) {
    // the refinement already synchronized: report an expired bounded wait of a sweep kernel
    int sw = 0;
    CUDA_TRY(h, cudaMemcpy(&sw, h->sweep_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (sw != 0) {
      h->last_status = sw;
      return set_err(h, sw, "bounded device wait expired in a solve sweep");
    }
  }
  h->last_status = status;
  return status;
}

int d3m_solve(d3m_handle h, const void* B, void* X, int32_t nrhs, void* stream) {
  if (!h) return set_err(nullptr, D3M_ERR_INVALID, "handle is NULL");
  return solve_impl(h, B, X, nrhs, (cudaStream_t)stream);
}

int d3m_adjoint(d3m_handle h, const void* G, void* Lambda, int32_t nrhs, void* stream) {
  if (!h) return set_err(nullptr, D3M_ERR_INVALID, "handle is NULL");
  // K^T = K: the adjoint system is solved with the same factors and refinement
  return solve_impl(h, G, Lambda, nrhs, (cudaStream_t)stream);
}

int d3m_grad_eps(d3m_handle h, const void* Lambda, const void* X, int32_t nrhs, int32_t ndom,
                 const int32_t* dom_ptr, const int32_t* dom_if, double k2, double* dJ, void* stream) {
  if (!h) return set_err(nullptr, D3M_ERR_INVALID, "handle is NULL");
  if (!Lambda || !X || !dom_ptr || !dom_if || !dJ || ndom < 0 || nrhs < 1)
    return set_err(h, D3M_ERR_INVALID, "bad argument to d3m_grad_eps");
  if (!is_device_ptr(Lambda) || !is_device_ptr(X)) return set_err(h, D3M_ERR_INVALID, "Lambda and X must be device memory");
  cudaStream_t st = (cudaStream_t)stream;
  const Symbolic& S = h->S;
  int rc = launch_contract((const double2*)Lambda, (const double2*)X, S.n, nrhs, h->xoff_orig, h->m_orig, S.N,
                           h->contract, st);
  if (rc) return set_err(h, D3M_ERR_CUDA, "contract launch failed");
  h->launches += 1;
  std::vector<double2> sf(S.N);
  CUDA_TRY(h, cudaMemcpyAsync(sf.data(), h->contract, S.N * sizeof(double2), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(h, cudaStreamSynchronize(st));
  for (int i = 0; i < ndom; ++i) {
    double re = 0.0;
    for (int q = dom_ptr[i]; q < dom_ptr[i + 1]; ++q) {
      const int f = dom_if[q];
      if (f < 0 || f >= S.N) return set_err(h, D3M_ERR_INVALID, "dom_if entry out of range");
      re += sf[f].x;
    }
    dJ[i] = k2 * re;   // Re(k2 * s) with real k2
  }
  return D3M_OK;
}

int d3m_grad_pattern(d3m_handle h, const void* Lambda, const void* X, int32_t nrhs, void* dK, void* stream) {
  if (!h) return set_err(nullptr, D3M_ERR_INVALID, "handle is NULL");
  if (!Lambda || !X || !dK || nrhs < 1) return set_err(h, D3M_ERR_INVALID, "bad argument to d3m_grad_pattern");
  if (!is_device_ptr(Lambda) || !is_device_ptr(X) || !is_device_ptr(dK))
    return set_err(h, D3M_ERR_INVALID, "Lambda, X and dK must be device memory");
  const Symbolic& S = h->S;
  int rc = launch_grad_pattern((const double2*)Lambda, (const double2*)X, S.n, nrhs, h->colptr, h->rowidx, h->blk_col,
                               h->kblk_off, h->xoff_orig, h->m_orig, S.nnzb_K, (double2*)dK, (cudaStream_t)stream);
  if (rc) return set_err(h, D3M_ERR_CUDA, "grad_pattern launch failed");
  h->launches += 1;
  return D3M_OK;
}

int d3m_get_factor_block(d3m_handle h, int32_t i, int32_t j, void* host_out, void* stream) {
  if (!h) return set_err(nullptr, D3M_ERR_INVALID, "handle is NULL");
  const Symbolic& S = h->S;
  if (!host_out || i < 0 || j < 0 || i >= S.N || j >= S.N || i < j) return set_err(h, D3M_ERR_INVALID, "bad block index");
  if (i != j && !std::binary_search(S.str[j].begin(), S.str[j].end(), i))
    return set_err(h, D3M_ERR_INVALID, "block not in the filled pattern");
  CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)stream));
  const int b = h->b, mi = S.m[i], mj = S.m[j];
  double2* out = (double2*)host_out;
  std::vector<unsigned char> tile((size_t)b * b * h->csize);
  for (int J = S.tstart[j]; J < S.tstart[j + 1]; ++J)
    for (int I = S.tstart[i]; I < S.tstart[i + 1]; ++I) {
      const int r0 = (I - S.tstart[i]) * b, c0 = (J - S.tstart[j]) * b;
      const int64_t t = (I >= J) ? S.tile_of(I, J) : -1;
      if (t < 0) {
        for (int c = c0; c < std::min(mj, c0 + b); ++c)
          for (int r = r0; r < std::min(mi, r0 + b); ++r) out[(int64_t)c * mi + r] = make_double2(0, 0);
        continue;
      }
      CUDA_TRY(h, cudaMemcpy(tile.data(), (unsigned char*)h->L + (size_t)t * b * b * h->csize, tile.size(),
                             cudaMemcpyDeviceToHost));
      for (int c = c0; c < std::min(mj, c0 + b); ++c)
        for (int r = r0; r < std::min(mi, r0 + b); ++r) {
          const size_t e = (size_t)(r - r0) * b + (c - c0);
          double2 v;
          if (h->fp64) v = ((double2*)tile.data())[e];
          else {
            const float2 f = ((float2*)tile.data())[e];
            v = make_double2(f.x, f.y);
          }
          out[(int64_t)c * mi + r] = v;
        }
    }
  return D3M_OK;
}

int d3m_get_pivots(d3m_handle h, int32_t j, void* host_out, void* stream) {
  if (!h) return set_err(nullptr, D3M_ERR_INVALID, "handle is NULL");
  const Symbolic& S = h->S;
  if (!host_out || j < 0 || j >= S.N) return set_err(h, D3M_ERR_INVALID, "bad block index");
  CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)stream));
  const int mj = S.m[j];
  std::vector<unsigned char> buf((size_t)mj * h->csize);
  CUDA_TRY(h, cudaMemcpy(buf.data(), (unsigned char*)h->D + (size_t)S.tstart[j] * h->b * h->csize, buf.size(),
                         cudaMemcpyDeviceToHost));
  double2* out = (double2*)host_out;
  for (int u = 0; u < mj; ++u) {
    if (h->fp64) out[u] = ((double2*)buf.data())[u];
    else {
      const float2 f = ((float2*)buf.data())[u];
      out[u] = make_double2(f.x, f.y);
    }
  }
  return D3M_OK;
}

int d3m_get_pivot_blocks(d3m_handle h, int32_t j, void* e_out, int32_t* perm_out, void* stream) {
  if (!h) return set_err(nullptr, D3M_ERR_INVALID, "handle is NULL");
  const Symbolic& S = h->S;
  if (j < 0 || j >= S.N) return set_err(h, D3M_ERR_INVALID, "bad block index");
  CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)stream));
  const int mj = S.m[j];
  std::vector<unsigned char> buf((size_t)mj * h->csize, 0);
  std::vector<int32_t> pv(mj);
  for (int u = 0; u < mj; ++u) pv[u] = u % h->b;
  if (h->E) {
    CUDA_TRY(h, cudaMemcpy(buf.data(), (unsigned char*)h->E + (size_t)S.tstart[j] * h->b * h->csize, buf.size(),
                           cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(pv.data(), h->piv + (size_t)S.tstart[j] * h->b, (size_t)mj * sizeof(int32_t),
                           cudaMemcpyDeviceToHost));
  }
  for (int u = 0; u < mj; ++u) {
    if (e_out) {
      double2* out = (double2*)e_out;
      if (h->fp64) out[u] = ((double2*)buf.data())[u];
      else {
        const float2 f = ((float2*)buf.data())[u];
        out[u] = make_double2(f.x, f.y);
      }
    }
    if (perm_out) perm_out[u] = (u / h->b) * h->b + pv[u];   // tile-local order + tile offset
  }
  return D3M_OK;
}

int d3m_get_trace(d3m_handle h, int64_t* host_out, int64_t cap, int64_t* count, void* stream) {
  if (!h || !count) return set_err(h, D3M_ERR_INVALID, "handle or count is NULL");
  if (!h->trace) return set_err(h, D3M_ERR_STATE, "tracing was not enabled at create (D3M_DEBUG_TRACE)");
  const int64_t n = (int64_t)h->S.tasks.size();
  *count = n;
  CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)stream));
  if (host_out && cap > 0) {
    const int64_t m = std::min(cap, n);
    CUDA_TRY(h, cudaMemcpy(host_out, h->trace, (size_t)m * 10 * sizeof(int64_t), cudaMemcpyDeviceToHost));
  }
  return D3M_OK;
}

int d3m_get_info(d3m_handle h, d3m_info* info, void* stream) {
  if (!h || !info) return set_err(h, D3M_ERR_INVALID, "handle or info is NULL");
  CUDA_TRY(h, cudaStreamSynchronize((cudaStream_t)stream));
  CUDA_TRY(h, cudaGetLastError());
  std::memset(info, 0, sizeof(*info));
  fill_structure(h->S, info);
  info->device_bytes = h->dev_bytes;
  info->instances = h->ninst;
  int st = h->last_status;
  {
    int sw = 0;
    CUDA_TRY(h, cudaMemcpy(&sw, h->sweep_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (sw != 0) st = sw;
  }
  if (h->factored) {
    int fe = factor_error(h);
    if (fe != D3M_OK) st = fe;
    info->min_abs_pivot = (double)([](unsigned u) { float f; std::memcpy(&f, &u, 4); return f; })(h->h_ctl->min_piv_bits);
    info->max_abs_pivot = (double)([](unsigned u) { float f; std::memcpy(&f, &u, 4); return f; })(h->h_ctl->max_piv_bits);
  }
  info->status = st;
  info->refine_iters = h->refine_iters;
  info->omega = h->omega_valid ? h->omega : NAN;
  info->omega_first = h->omega_valid ? h->omega_first : NAN;
  // fold the recorded event pairs into the totals; the last pair of a kind is the "last call"
  double tot[d3m_ctx::EV_KINDS] = {0, 0, 0, 0};
  int64_t cnt[d3m_ctx::EV_KINDS] = {0, 0, 0, 0};
  bool resid_seen = false;
  for (size_t e = 0; e < h->ev_pending.size(); ++e) {
    const auto& pr = h->ev_pending[e];
    float t = 0.f;
    CUDA_TRY(h, cudaEventElapsedTime(&t, pr.a, pr.b));
    tot[pr.kind] += t;
    cnt[pr.kind] += 1;
    if (pr.kind == d3m_ctx::EV_FACTOR) h->last_factor_ms = t;
    if (pr.kind == d3m_ctx::EV_SOLVE) {
      h->last_solve_ms = t;
      h->last_resid_ms = 0;
      resid_seen = true;
    }
    if (pr.kind == d3m_ctx::EV_RESID) {
      if (!resid_seen) h->last_resid_ms = 0;
      resid_seen = true;
      h->last_resid_ms += t;
    }
    h->ev_pool.push_back(pr.a);
    h->ev_pool.push_back(pr.b);
  }
  h->ev_pending.clear();
  info->factor_kernel_ms = h->last_factor_ms;
  info->solve_ms = h->last_solve_ms;
  info->residual_ms = h->last_resid_ms;
  info->kernel_launches = h->launches;
  info->factor_kernel_ms_total = tot[d3m_ctx::EV_FACTOR];
  info->residual_ms_total = tot[d3m_ctx::EV_RESID];
  info->sweep_ms_total = tot[d3m_ctx::EV_SWEEP];
  info->factor_kernel_calls = cnt[d3m_ctx::EV_FACTOR];
  info->residual_calls = cnt[d3m_ctx::EV_RESID];
  info->sweep_calls = cnt[d3m_ctx::EV_SWEEP];
  return D3M_OK;
}

const char* d3m_last_error(d3m_handle h) {
  if (h) return h->err.c_str();
  return g_err.c_str();
}

void d3m_destroy(d3m_handle h) {
  if (!h) return;
  for (auto& g : h->g_factor) cudaGraphExecDestroy(g.exec);
  if (h->side) cudaStreamSynchronize(h->side);   // work still running on the library's streams
  if (h->kup) cudaStreamSynchronize(h->kup);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->kup) cudaStreamDestroy(h->kup);
  if (h->ev_kup0) cudaEventDestroy(h->ev_kup0);
  if (h->ev_kup1) cudaEventDestroy(h->ev_kup1);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (auto& g : h->g_solve) cudaGraphExecDestroy(g.exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  if (h->h_stat) cudaFreeHost(h->h_stat);
  for (cudaEvent_t e : h->ev_pool)
    if (e) cudaEventDestroy(e);
  for (const auto& pr : h->ev_pending) {
    if (pr.a) cudaEventDestroy(pr.a);
    if (pr.b) cudaEventDestroy(pr.b);
  }
  for (const auto& pr : h->ev_open) {
    if (pr.a) cudaEventDestroy(pr.a);
    if (pr.b) cudaEventDestroy(pr.b);
  }
  delete h;
}

}  // extern "C"
