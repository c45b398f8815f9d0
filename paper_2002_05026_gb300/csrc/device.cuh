// Device-side helpers shared by the factorization kernels: complex arithmetic and the task
// queue of the persistent scheduler.
//
// Scheduler (replaces the paper's static list schedule, Sec. II, with a dynamic queue):
//   ready[]  : task ids in the order they became ready (slot s holds the s-th push, -1 = empty)
//   head     : next slot to claim (atomicAdd); tail: next slot to fill (atomicAdd)
//   cnt[t]   : unmet dependencies of task t; the producer that drops it to 0 pushes t.
// A block claims a slot, then waits (bounded by timeout_ns of %globaltimer, with backoff)
// until the slot is filled.  Every slot < ntasks is eventually filled while some block
// runs a task, so the only way a wait expires is a broken graph or an abort; then the block
// records D3M_ERR_TIMEOUT, raises `abort`, and returns.  A block that is still running a task
// may also take a task that is already pushed (sched_claim_normal), never one that is not, so
// it cannot wait on work that depends on its own.
// Memory order: data writes -> __syncthreads -> fence (release) -> atomicSub on successors;
// the pusher fences again before publishing the id; the consumer fences after reading it
// (acquire) and reads producer data with L1-bypassing loads or the TMA (async proxy).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "d3m.h"
#include "symbolic.h"

namespace d3m {

struct Ctl {
  int32_t head, tail, done, abort;
  int32_t err, err_task, head_hi, tail_hi;
  uint32_t min_piv_bits, max_piv_bits;  // |d| as float bits (non-negative => ordered as uint)
  int32_t pad2[6];
};

struct FactorParams {
  const TileTask* tasks;
  const KEntry* klist;
  int32_t* cnt;
  const int64_t* succ_ptr;
  const int32_t* succ;
  int32_t* ready;
  int32_t* ready_hi;     // priority lane (tasks flagged TF_PRIO)
  Ctl* ctl;
  int32_t ntasks;
  int32_t n_norm;        // tasks of the normal lane
  int32_t b;
  const double2* K;      // library copy of K (c128)
  void* L;               // [ntiles][b][b] complex (row-major tiles)
  void* Linv;            // [NT][b][b] inverse of the unit-lower diagonal tiles
  void* D;               // [NT][b] pivots
  void* opA;             // tensor-core operand planes (bf16) of L tiles
  void* opB;             // tensor-core operand planes (bf16) of W tiles / T_J
  void* opS;             // TF32 engine: bf16 split planes of the L tiles for the solve's products, or nullptr
  const int32_t* k_arrived;  // upload progress of a host K (stored blocks in upload order), or nullptr
  void* Sacc;            // [n_acc][b][b] partial Schur accumulators (complex, working precision)
  int64_t* trace;        // [ntasks][8] task records, or nullptr
  int64_t timeout_ns;
  double piv_tol;        // breakdown: |d| < piv_tol * max|S| of the diagonal tile
  int pivot;             // 1: Bunch-Kaufman pivoting inside diagonal tiles (SIMT engine)
  void* E;               // [NT][b] sub-diagonal entry of each 2 x 2 pivot block (pivot mode), 0 else
  int32_t* piv;          // [NT][b] permutation of each diagonal tile (pivot mode)
};

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  c.x = fma(a.x, b.x, c.x); c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y); c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  c.x = fmaf(a.x, b.x, c.x); c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y); c.y = fmaf(a.y, b.x, c.y);
  return c;
}
// acc - a*b
__device__ __forceinline__ double2 cfms(double2 a, double2 b, double2 c) {
  c.x = fma(-a.x, b.x, c.x); c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y); c.y = fma(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float2 cfms(float2 a, float2 b, float2 c) {
  c.x = fmaf(-a.x, b.x, c.x); c.x = fmaf(a.y, b.y, c.x);
  c.y = fmaf(-a.x, b.y, c.y); c.y = fmaf(-a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double s = 1.0 / (b.x * b.x + b.y * b.y);
  return make_double2((a.x * b.x + a.y * b.y) * s, (a.y * b.x - a.x * b.y) * s);
}
__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  float s = 1.0f / (b.x * b.x + b.y * b.y);
  return make_float2((a.x * b.x + a.y * b.y) * s, (a.y * b.x - a.x * b.y) * s);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float cabs2(float2 a) { return a.x * a.x + a.y * a.y; }

template <typename R> struct CT;
template <> struct CT<double> {
  using C = double2;
  static __device__ __forceinline__ C make(double x, double y) { return make_double2(x, y); }
  static __device__ __forceinline__ C from(double2 v) { return v; }
  static constexpr double u = 1.1102230246251565e-16;  // 2^-53
};
template <> struct CT<float> {
  using C = float2;
  static __device__ __forceinline__ C make(float x, float y) { return make_float2(x, y); }
  static __device__ __forceinline__ C from(double2 v) { return make_float2((float)v.x, (float)v.y); }
  static constexpr double u = 5.9604644775390625e-08;  // 2^-24
};

// L1-bypassing loads of data written by other blocks during the same launch
__device__ __forceinline__ double2 ld_cg(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_cg(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ float4 ld_cg4(const float4* p) { return __ldcg(p); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_volatile(const int32_t* p) { return *(const volatile int32_t*)p; }

__device__ __forceinline__ void set_error(Ctl* ctl, int code, int task) {
  if (atomicCAS(&ctl->err, 0, code) == 0) ctl->err_task = task;
  atomicExch(&ctl->abort, 1);
}

// ------------------------------------------------------------------ scheduler
__device__ __forceinline__ uint32_t sm_id() {
  uint32_t s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

// Trace record of one task: start (at pop or claim) and end (before its successors are released).
constexpr int TRACE_W = 10;
__device__ __forceinline__ void trace_begin(const FactorParams& p, int task) {
  if (p.trace && threadIdx.x == 0) p.trace[TRACE_W * (int64_t)task] = (int64_t)globaltimer_ns();
}
// phase mark k (0..3) of a task
__device__ __forceinline__ void trace_mark(const FactorParams& p, int task, int k) {
  if (p.trace && threadIdx.x == 0) p.trace[TRACE_W * (int64_t)task + 4 + k] = (int64_t)globaltimer_ns();
}

// Claim the next ready task for this block (all threads call; returns -1 when done/aborted).
// Two lanes: the priority lane is served first and claimed with a compare-and-swap only when a
// pushed task is there; the normal lane keeps one claimed slot per block (*s_pending, -1 when
// none), waited on between looks at the priority lane, so no block ever blocks on it alone.
// A block leaves when its normal slot is past the lane's end and every task has completed.
__device__ __forceinline__ int sched_pop(const FactorParams& p, int* s_task, int* s_pending) {
  if (threadIdx.x == 0) {
    int task = -1;
    int pend = *s_pending;
    if (pend < 0 && !ld_volatile(&p.ctl->abort)) pend = atomicAdd(&p.ctl->head, 1);
    const uint64_t t0 = globaltimer_ns();
    unsigned ns = 32;
    for (;;) {
      if (ld_volatile(&p.ctl->abort)) { task = -1; break; }
      const int hh = ld_volatile(&p.ctl->head_hi);
      if (hh < ld_volatile(&p.ctl->tail_hi)) {
        if (atomicCAS(&p.ctl->head_hi, hh, hh + 1) == hh) {
          // the pusher reserved slot hh before writing it
          for (;;) {
            task = ld_volatile(&p.ready_hi[hh]);
            if (task >= 0) break;
            if (ld_volatile(&p.ctl->abort) || globaltimer_ns() - t0 > (uint64_t)p.timeout_ns) {
              set_error(p.ctl, D3M_ERR_TIMEOUT, -1 - hh);
              task = -1;
              break;
            }
          }
          break;
        }
        continue;
      }
      if (pend < p.n_norm) {
        task = ld_volatile(&p.ready[pend]);
        if (task >= 0) {
          pend = -1;
          break;
        }
      } else if (ld_volatile(&p.ctl->done) >= p.ntasks) {
        task = -1;
        break;
      }
      if (globaltimer_ns() - t0 > (uint64_t)p.timeout_ns) {
        set_error(p.ctl, D3M_ERR_TIMEOUT, -1 - pend);
        task = -1;
        break;
      }
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
    }
    if (task >= 0) __threadfence();  // acquire: producer data is visible after this point
    *s_pending = pend;
    *s_task = task;
  }
  __syncthreads();
  const int t = *s_task;
  __syncthreads();
  if (t >= 0) trace_begin(p, t);
  return t;
}

// Non-blocking claim of a normal-lane task by ONE thread of a block that is still running a
// task (-1 if none is ready now).  The block's claimed slot (*s_pending) is taken if it has been
// filled; without one, a slot is claimed only when the lane holds a pushed task past its head
// (a pusher reserves a slot before writing it, so that wait is short; it is bounded all the
// same).  Priority-lane tasks are left to blocks that are free now.  The claimed task is ready,
// so it never depends on the caller's running task.
__device__ __forceinline__ int sched_claim_normal(const FactorParams& p, int* s_pending) {
  if (ld_volatile(&p.ctl->abort)) return -1;
  int pend = *s_pending;
  if (pend < 0) {
    const int h = ld_volatile(&p.ctl->head);
    if (h < ld_volatile(&p.ctl->tail) && atomicCAS(&p.ctl->head, h, h + 1) == h) pend = h;
    else return -1;
  }
  int task = -1;
  if (pend < p.n_norm) {
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
      task = ld_volatile(&p.ready[pend]);
      if (task >= 0) {
        pend = -1;
        break;
      }
      if (pend >= ld_volatile(&p.ctl->tail)) break;   // not pushed yet: the block keeps the slot
      if (ld_volatile(&p.ctl->abort) || globaltimer_ns() - t0 > (uint64_t)p.timeout_ns) {
        set_error(p.ctl, D3M_ERR_TIMEOUT, -1 - pend);
        task = -1;
        break;
      }
    }
  }
  *s_pending = pend;
  if (task >= 0) {
    __threadfence();  // acquire, as in sched_pop
    if (p.trace) p.trace[TRACE_W * (int64_t)task] = (int64_t)globaltimer_ns();
  }
  return task;
}

// Release the successors of `task`: one whole warp calls this (lane = its lane) after the
// block's writes of the task are ordered before it (proxy fence + block barrier).
__device__ __forceinline__ void release_successors(const FactorParams& p, int task, int lane) {
  if (p.trace && lane == 0) {
    const TileTask& T = p.tasks[task];
    p.trace[TRACE_W * (int64_t)task + 1] = (int64_t)globaltimer_ns();
    p.trace[TRACE_W * (int64_t)task + 2] = (int64_t)sm_id();
    p.trace[TRACE_W * (int64_t)task + 3] = (int64_t)T.flags | ((int64_t)T.tile << 8) | ((int64_t)T.nk << 40);
  }
  __threadfence();  // release: this block's tile writes before the counter updates
  const int64_t e0 = p.succ_ptr[task], e1 = p.succ_ptr[task + 1];
  for (int64_t e = e0 + lane; e < e1; e += 32) {
    const int s = p.succ[e];
    if (atomicSub(&p.cnt[s], 1) == 1) {
      if (p.trace) {
        p.trace[TRACE_W * (int64_t)s + 8] = (int64_t)globaltimer_ns();
        p.trace[TRACE_W * (int64_t)s + 9] = task;
      }
      __threadfence();
      if (p.tasks[s].flags & TF_PRIO) {
        const int pos = atomicAdd(&p.ctl->tail_hi, 1);
        atomicExch(&p.ready_hi[pos], s);
      } else {
        const int pos = atomicAdd(&p.ctl->tail, 1);
        atomicExch(&p.ready[pos], s);
      }
    }
  }
  if (lane == 0) atomicAdd(&p.ctl->done, 1);
}

// Release the successors of `task` (all threads call; warp 0 does the work).
__device__ __forceinline__ void sched_complete(const FactorParams& p, int task) {
  // writes of this thread become visible to later TMA (async-proxy) reads of other blocks
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) release_successors(p, task, threadIdx.x);
}

// A task that reads its stored K block while a host K is still being uploaded waits (bounded)
// until the block has arrived: the upload stream raises *k_arrived past the block's sequence
// number after its copy (all threads call; on expiry the factorization is aborted).
__device__ __forceinline__ void wait_k_block(const FactorParams& p, int kseq, int task, uint64_t deadline) {
  if (!p.k_arrived || kseq < 0) return;
  while (ld_volatile(p.k_arrived) <= kseq) {
    if (ld_volatile(&p.ctl->abort) || globaltimer_ns() > deadline) {
      set_error(p.ctl, D3M_ERR_TIMEOUT, task);
      return;
    }
    __nanosleep(256);
  }
  __threadfence();  // the block's data is read after the progress counter
}

__device__ __forceinline__ void record_pivot_stats(Ctl* ctl, float amin, float amax) {
  atomicMin(&ctl->min_piv_bits, __float_as_uint(amin));
  atomicMax(&ctl->max_piv_bits, __float_as_uint(amax));
}

// Entry (r, c) of the K tile of task T (padding: unit diagonal inside diagonal blocks).
template <typename R>
__device__ __forceinline__ typename CT<R>::C k_entry(const TileTask& T, const double2* K, int r, int c) {
  using C = typename CT<R>::C;
  if (r >= T.rv || c >= T.cv) {
    const bool one = (T.flags & TF_SAME_BLOCK) && (T.r0 + r == T.c0 + c);
    return CT<R>::make(one ? (R)1 : (R)0, (R)0);
  }
  if (T.k_off < 0) return CT<R>::make((R)0, (R)0);
  const int rr = T.r0 + r, cc = T.c0 + c;
  const int64_t idx = T.k_tr ? ((int64_t)rr * T.k_ld + cc) : ((int64_t)cc * T.k_ld + rr);
  return CT<R>::from(__ldg(K + T.k_off + idx));
}

}  // namespace d3m
