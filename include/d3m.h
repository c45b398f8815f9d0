/*
 * d3m.h -- C ABI of the GB300 (sm_103a) D3M dual-system solver.
 *
 * The library factors and solves the reduced block-sparse dual matrix K of the Direct
 * Domain Decomposition Method (D3M; Moshfegh, Makris, Vouvakis, "Parallel Direct Domain
 * Decomposition Methods (D3M) for Finite Elements", IEEE AP-S/URSI 2019):
 *   - Sec. I: the sparse FEM system is reduced to a block-sparse matrix K, which is solved
 *     with a block LDL^T factorization scheduled as a DAG of block tasks;
 *   - Sec. II: when K is factored and solved, each nonzero block of K is one task that
 *     performs its dense update, dense triangular solve and dense factorization; a symbolic
 *     run of the sequential algorithm yields the task graph (B-DAG); the dual tasks are
 *     weighted with GEMM, sytrf and triSolve timings;
 *   - Fig. 1(b)/(c): the sparsity of K and its task graph.
 * K is complex symmetric (K^T = K, not Hermitian) and indefinite.  The library computes
 * the unpivoted factorization P K P^T = L D L^T (L unit lower, D diagonal) and solves
 * K X = B by forward, diagonal and backward sweeps.
 *
 * Conventions shared by all calls
 *   - complex numbers are interleaved (re, im) pairs: "c128" = 2 x double, "c64" = 2 x float;
 *   - K is given by its LOWER block triangle in block-CSC order over the caller's (original)
 *     interface numbering: column g holds rows rowidx[colptr[g] .. colptr[g+1]-1], strictly
 *     ascending, the first one being g itself (diagonal block present); block (f, g) is an
 *     m_f x m_g dense block stored column-major with leading dimension m_f; blocks follow
 *     one another in that CSC order with no gaps;
 *   - right-hand sides and solutions are n x nrhs column-major with leading dimension n,
 *     n = sum_f m_f, rows in the caller's numbering;
 *   - every pointer may be host or device memory unless a call says otherwise; host buffers
 *     are copied by the library on the given stream;
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  No call synchronizes the
 *     stream except d3m_get_info / d3m_get_factor_block / d3m_get_pivots and the refinement
 *     loop inside d3m_solve, which reads one convergence word per iteration.
 *
 * Ownership: the caller owns every buffer it passes and the stream.  The library owns the
 * factors, the base-64 digit planes of K (kept for the FP64-accurate residual), a copy buffer for a host K
 * (allocated by the first d3m_factor that passes one), the task graph and its workspaces, from
 * d3m_create until d3m_destroy.  A handle is not thread-safe; use one per host thread.
 *
 * Errors: every int-returning call returns D3M_OK (0) or one of the D3M_ERR_* codes below;
 * d3m_last_error(h) gives a one-line text for the last failing call on h.
 */
#ifndef D3M_H
#define D3M_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct d3m_ctx* d3m_handle;

enum {
  D3M_OK = 0,
  D3M_ERR_INVALID = 1,        /* bad pattern, permutation, option or argument */
  D3M_ERR_OOM = 2,            /* device or host allocation failed */
  D3M_ERR_CUDA = 3,           /* a CUDA runtime call failed (text in d3m_last_error) */
  D3M_ERR_PIVOT = 4,          /* |d| below 1e3 * u * max|S_kk| in some diagonal block */
  D3M_ERR_NOT_CONVERGED = 5,  /* refinement hit its cap or stagnated; best x is written */
  D3M_ERR_TIMEOUT = 6,        /* a bounded device wait expired; the kernel returned */
  D3M_ERR_STATE = 7           /* call out of order (e.g. solve before factor) */
};

/* Arithmetic of the factorization (d3m_options.precision). */
enum {
  D3M_FP64 = 0,          /* complex128 factors, FP64 SIMT tile engine, no refinement */
  D3M_MIXED_BF16X3 = 1,  /* complex64 factors; Schur/TRSM products on tcgen05 tensor cores as
                            split-BF16x3 (a = a_hi + a_lo; hi*hi + hi*lo + lo*hi) with FP32
                            accumulation in TMEM; FP64 residual + iterative refinement */
  D3M_MIXED_SIMT32 = 2,  /* complex64 factors on an FP32 SIMT tile engine (no tensor cores);
                            FP64 residual + iterative refinement */
  D3M_MIXED_TF32 = 3     /* complex64 factors; Schur/TRSM products on tcgen05 tensor cores as one
                            kind::tf32 product (operands rounded to tf32, 10-bit mantissa) with
                            FP32 accumulation in TMEM, the source-block updates of tiles (I, J)
                            and (I, J+1) in one task sharing L_IK; the solve's products use bf16
                            split planes of L written beside the tf32 ones; FP64 residual +
                            iterative refinement */
};

typedef struct {
  int32_t nblk;             /* N, number of interface blocks */
  int32_t m;                /* uniform block size, used when blk_size == NULL */
  const int32_t* blk_size;  /* [N] per-block sizes m_f (host), or NULL */
  const int64_t* colptr;    /* [N+1] host, lower block-CSC column pointers */
  const int32_t* rowidx;    /* [colptr[N]] host, row block indices */
} d3m_pattern;

typedef struct {
  int32_t precision;        /* D3M_FP64 | D3M_MIXED_BF16X3 | D3M_MIXED_SIMT32 | D3M_MIXED_TF32 */
  int32_t refine_max_iter;  /* cap on refinement steps (default 20) */
  double refine_tol;        /* target normwise backward error omega (default 1e-12) */
  int64_t timeout_ns;       /* bound on any device-side wait (default 5 s) */
  int32_t tile;             /* tile edge; 0 = default (128 tensor-core, 64 SIMT) */
  int32_t max_nrhs;         /* largest nrhs a solve may use (default 32) */
  int32_t fp64_omega;       /* D3M_FP64 only: 1 = also compute omega after the solve
                               (one FP64 residual; default 0) */
  int32_t debug_flags;      /* D3M_DEBUG_* test hooks, 0 in normal use */
  int32_t graphs;           /* 1 = capture each launch sequence (factorization with K in device
                               memory; one refinement step of a solve) into a CUDA graph on
                               first use and replay it afterwards; default 0 */
  int32_t seg_group;        /* source blocks whose Schur updates of a tile form one update task
                               (0 = default: 32 with TF32, 8 in the other mixed modes, 1 in FP64; 1 = a task per
                               source block, the earliest start) */
  double prio_slack;        /* tasks whose estimated slack is within prio_slack x the critical
                               path are served first by the device scheduler (default 0.08;
                               0 = only the critical path itself) */
  double refine_fwd_tol;    /* mixed modes: refinement also requires, per column, that the last
                               correction d_k be <= refine_fwd_tol |x|, or that the error it
                               leaves, rho/(1-rho) |d_k| with rho = |d_k|/|d_(k-1)| < 1, be
                               (default 1e-10; 0 = backward error only) */
  double task_cost[6];      /* duration model of the scheduler's critical-path priority (the paper
                               weights its dual tasks with benchmarked GEMM / sytrf / triSolve
                               times, Sec. II): cost = base + per_k * nk, nk = tile products of
                               the task, for update tasks [0], [1], diagonal final tasks
                               (LDL^T + inverse) [2], [3] and off-diagonal final tasks
                               (triangular solve) [4], [5]; any common unit (e.g. measured ns,
                               see d3m_get_trace); all zero (default) = a built-in model */
  int32_t pivot;            /* 1 = Bunch-Kaufman symmetric pivoting (1 x 1 and 2 x 2 pivots, the
                               paper's sytrf, Sec. II) inside every diagonal tile: the tile is
                               factored as S = Lt D Lt^T, Lt = P^T L; the block structure and task
                               graph are unchanged.  SIMT engines only (D3M_FP64,
                               D3M_MIXED_SIMT32; D3M_ERR_INVALID otherwise).  0 (default) =
                               unpivoted, scalar D */
} d3m_options;

/* Test hook: upload the task graph with one extra unmet dependency on the last task, so the
 * device queue starves and every waiting block hits the bounded wait (-> D3M_ERR_TIMEOUT). */
#define D3M_DEBUG_STALL_LAST_TASK 1
/* Tracing: every factorization task records {start ns, end ns, SM id, task flags} from
 * %globaltimer into a device buffer (one record per task), read with d3m_get_trace. */
#define D3M_DEBUG_TRACE 2

typedef struct {
  int64_t n;                /* sum of block sizes */
  int32_t nblk;             /* N */
  int32_t tile;             /* tile edge b */
  int64_t nnzb_K;           /* stored lower blocks of K */
  int64_t nblk_L_offdiag;   /* off-diagonal blocks of L after fill */
  int32_t etree_depth;      /* depth of the block elimination tree */
  int32_t max_col_height;   /* max off-diagonal blocks in one column of L */
  int64_t ntiles;           /* lower tiles of L (tasks of the factorization DAG) */
  int64_t ntile_updates;    /* tile GEMM updates (K-list entries) */
  int64_t ndep_edges;       /* edges of the tile task graph */
  double factor_flops;      /* algorithmic flops of the block factorization (complex MAC = 8):
                               N (4/3) m^3 + n_L 4 m^3 (TRSM) + n_L 4 m^3 + n_off 8 m^3 (updates) */
  double solve_flops_per_rhs; /* 8 (2 nnz_offdiag(L) + sum m_k^2) + 6 n (forward + diagonal +
                                 backward sweeps, complex MAC = 8) */
  double residual_flops_per_rhs; /* 8 * entries of K (both triangles) */
  int64_t device_bytes;     /* device memory owned by the handle */
  /* last factor / solve (valid after d3m_get_info synchronizes) */
  int32_t status;           /* status of the last factor or solve */
  int32_t refine_iters;     /* solves done by the last d3m_solve / d3m_adjoint */
  double omega;             /* max over columns of the final backward error (NaN if not computed) */
  double omega_first;       /* backward error after the first (unrefined) solve */
  double min_abs_pivot;     /* min |d| over all pivots of the last factorization */
  double max_abs_pivot;     /* max |d| */
  double factor_kernel_ms;  /* device time of the last factorization kernel (CUDA events) */
  double solve_ms;          /* device time of the last d3m_solve / d3m_adjoint (events) */
  double residual_ms;       /* device time in FP64 residual kernels of that solve */
  int64_t kernel_launches;  /* kernels launched by this handle since d3m_create */
  /* device time summed over every launch since the previous d3m_get_info (CUDA events):
   * factorization kernels, FP64 residual kernels, and whole solve sweeps */
  double factor_kernel_ms_total;
  double residual_ms_total;
  double sweep_ms_total;
  int64_t factor_kernel_calls, residual_calls, sweep_calls;
  int32_t instances;        /* independent systems held by the handle (1 unless batched) */
  int32_t reserved0;
  int64_t prio_tasks;       /* tasks the device scheduler serves first: slack within 8% of the
                               estimated critical path of the task graph */
  /* algorithmic bytes of one FP64 residual r = b - K x: the stored lower blocks of K once in
   * c128 (residual_bytes_fixed) plus x and b read and r written in c128 per right-hand side */
  double residual_bytes_fixed;
  double residual_bytes_per_rhs;
} d3m_info;

/* Default options (precision D3M_MIXED_BF16X3). */
void d3m_default_options(d3m_options* opt);

/* Nested-dissection order of the interfaces of an nx x ny x nz domain grid (host only, no GPU).
 * Interfaces are numbered in domain order (domain id (ix*ny + iy)*nz + iz), then axis x, y, z,
 * one per pair of face neighbours.  The box is split along its longest extent (ties to the
 * lower axis) at lo + floor(extent/2); the interfaces across the cut are ordered last in
 * natural order; the lower half-box comes first; a box of extent 1 in every axis or with at
 * most one interface keeps natural order.  perm[new] = old, length = number of interfaces.
 * Returns D3M_ERR_INVALID for non-positive extents. */
int d3m_order_grid_nd(int32_t nx, int32_t ny, int32_t nz, int32_t* perm);

/* Symbolic analysis only (host, no GPU): fills the structural fields of `info` (n, nblk, tile,
 * nnzb_K, nblk_L_offdiag, etree_depth, max_col_height, ntiles, ntile_updates, ndep_edges,
 * factor_flops, solve_flops_per_rhs, residual_flops_per_rhs).  perm may be NULL (identity).
 * This is the paper's symbolic simulation that yields the task graph (Sec. II). */
int d3m_analyze(const d3m_pattern* pat, const int32_t* perm, int32_t tile, d3m_info* info);

/* Symbolic analysis with the options a handle would be created with (host, no GPU): the same
 * structural fields as d3m_analyze for the tile edge that opt->precision (or opt->tile) selects,
 * and prio_tasks, the tasks that the critical-path priority built from opt->task_cost (or the
 * built-in model), opt->prio_slack and opt->seg_group puts in the scheduler's priority lane.
 * opt NULL = defaults. */
int d3m_analyze_opts(const d3m_pattern* pat, const int32_t* perm, const d3m_options* opt, d3m_info* info);

/* Create a solver for one pattern: validates the pattern and perm (perm[new] = old, NULL =
 * identity), runs the symbolic analysis, builds the tile task graph and allocates every
 * device buffer on the current device.  `opt` NULL = defaults. */
int d3m_create(d3m_handle* out, const d3m_pattern* pat, const int32_t* perm,
               const d3m_options* opt, void* stream);

/* Batched solver: `count` independent systems (instances, e.g. frequency points or different
 * domain grids, each with its own pattern, block sizes and perms[i]; perms NULL or perms[i]
 * NULL = identity) held as ONE block-diagonal system.  Every later call works on all instances
 * at once: d3m_factor runs a single persistent launch whose device queue holds the task graphs
 * of all instances (they share no task, so they interleave freely and fill the GPU), and each
 * level of a solve sweep covers that level of every instance.  Layouts are the instances'
 * own, concatenated in instance order: K = the lower blocks of instance 0 in its pattern
 * order, then those of instance 1, ...; B and X are n x nrhs column-major with
 * n = sum n_i and instance i's unknowns at rows [sum_{j<i} n_j, ... + n_i) of every column
 * (so every instance takes the same nrhs).  Refinement stops when the backward error of EVERY
 * instance and column is <= refine_tol (omega is computed per instance, with ||K_i||, so a
 * badly scaled instance cannot hide behind another); d3m_get_instance_omega returns them.
 * Same errors as d3m_create, D3M_ERR_INVALID naming the first bad instance. */
int d3m_create_batch(d3m_handle* out, int32_t count, const d3m_pattern* pats,
                     const int32_t* const* perms, const d3m_options* opt, void* stream);

/* Backward error of every instance after the last d3m_solve / d3m_adjoint (max over its
 * columns; NaN if no omega was computed, e.g. D3M_FP64 without fp64_omega).  host_out has
 * d3m_info.instances entries.  Synchronizes `stream`. */
int d3m_get_instance_omega(d3m_handle h, double* host_out, void* stream);

/* Numeric factorization.  K: c128 lower blocks as described above (host or device).  A device
 * K (16-byte aligned) is read in place, in stream order: it must not change until the
 * factorization has completed on `stream` (nothing reads it afterwards).  A host K is copied
 * into the handle's buffer: a page-locked one (cudaHostAlloc / cudaHostRegister), with the
 * tensor-core engines, block by block in elimination order on a stream of the handle while the
 * factorization runs (a task waits for its block; the copy is complete before the kernels
 * that follow the factorization on `stream`), any other one before the factorization starts.
 * Either way the host buffer must stay unchanged until the factorization has completed on
 * `stream`.
 * One persistent kernel then factors K, its blocks pulling ready tile tasks from a device
 * queue with atomic dependency counters (Sec. II task model, Fig. 1(c)).
 * D3M_ERR_PIVOT if a pivot falls below the breakdown threshold, D3M_ERR_TIMEOUT if a device
 * wait expired.  Errors found on the device are returned by the next call that synchronizes
 * (d3m_get_info) and by d3m_solve. */
int d3m_factor(d3m_handle h, const void* K, void* stream);

/* Solve K X = B for nrhs columns (1 <= nrhs <= max_nrhs).  B, X: c128, n x nrhs column-major
 * (host or device; may not alias).  FP64 mode: one forward/diagonal/backward sweep.  Mixed
 * modes: x = 0, r = b; repeat { d = solve_c64(r); x += d (FP64); r = b - K x (FP64, block
 * SpMV over the stored K) } until, per instance, every column has omega <= refine_tol and an
 * estimated forward error <= refine_fwd_tol, or the cap; D3M_ERR_NOT_CONVERGED if the cap is hit
 * or the instances still open stop making progress (their largest omega / refine_tol and
 * correction / refine_fwd_tol fails to halve over two steps); X then holds the best iterate. */
int d3m_solve(d3m_handle h, const void* B, void* X, int32_t nrhs, void* stream);

/* Adjoint solve with the same factors: K^T Lambda = G, which is K Lambda = G since K^T = K.
 * Same refinement and layout as d3m_solve.  For J = Re(sum_j g_j^T x_j), Lambda gives
 * dJ/db = conj(Lambda) (PyTorch convention dJ/dRe + i dJ/dIm). */
int d3m_adjoint(d3m_handle h, const void* G, void* Lambda, int32_t nrhs, void* stream);

/* dJ/deps_i = Re(k2 * sum_j sum_{u in unknowns of I(i)} Lambda_uj X_uj) for every domain i,
 * where dK/deps_i = -k2 on the unknowns of the interfaces of domain i.  dom_ptr [ndom+1] and
 * dom_if (host int32) list each domain's interfaces (caller numbering).  Lambda, X: device
 * c128 n x nrhs.  dJ_deps: host double [ndom]; synchronizes the stream. */
int d3m_grad_eps(d3m_handle h, const void* Lambda, const void* X, int32_t nrhs,
                 int32_t ndom, const int32_t* dom_ptr, const int32_t* dom_if, double k2,
                 double* dJ_deps, void* stream);

/* Same result as d3m_grad_eps, for callers that cannot allocate memory while it runs: a host
 * application whose own allocator owns the device memory (a memory pool sized at start-up, a
 * framework that hands every free byte to its caching allocator) and forbids allocations by
 * libraries, or code running where the device is nearly full, so that a cudaMalloc of the
 * temporaries could fail after the expensive solves have already been done.  The paper has no
 * counterpart; this is an API convenience of this library.
 * It allocates nothing (no cudaMalloc / cudaFree / host allocation): its temporaries live in
 * one file-scope static device array of about 0.9 MB that every GPU loading the library keeps
 * until process exit.  Limits: at most 16384 interfaces, 16384 domains and 98304 dom_if
 * entries, else D3M_ERR_INVALID; dom_ptr must start at 0 and be nondecreasing, and every dom_if
 * entry must name an interface, else D3M_ERR_INVALID (checked on the host before anything is
 * copied or launched).  The handle's device must be the current device (D3M_ERR_INVALID
 * otherwise).  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress).  All calls share the array, so calls that overlap on the GPU (other
 * streams, other host threads) race; no entry of it needs to start at zero.  dom_ptr and
 * dom_if are copied from (pageable) host memory and the call synchronizes the stream before it
 * returns.  Lambda, X: device c128; dJ_deps: host or device double [ndom]. */
int d3m_grad_eps_noalloc(d3m_handle h, const void* Lambda, const void* X, int32_t nrhs,
                         int32_t ndom, const int32_t* dom_ptr, const int32_t* dom_if, double k2,
                         double* dJ_deps, void* stream);

/* Gradient of J = Re(sum_j g_j^T x_j) with respect to the stored lower blocks of K:
 * dJ/dK_fg = -(Lambda_f X_g^T + [f != g] X_f Lambda_g^T), summed over columns (the outer
 * product -Lambda X^T restricted to K's pattern; an off-diagonal stored block also stands
 * for its transpose).  Output dK: device c128 in K's block layout (unconjugated). */
int d3m_grad_pattern(d3m_handle h, const void* Lambda, const void* X, int32_t nrhs,
                     void* dK, void* stream);

/* Copy factor block L_ij (i >= j, NEW numbering; i == j gives the unit lower diagonal block)
 * to host memory as c128, m_i x m_j column-major.  Returns D3M_ERR_INVALID if (i, j) is not
 * in the filled pattern.  Synchronizes the stream. */
int d3m_get_factor_block(d3m_handle h, int32_t i, int32_t j, void* host_out, void* stream);

/* Copy the pivots D_j of block column j (NEW numbering) to host memory as c128 [m_j]. */
int d3m_get_pivots(d3m_handle h, int32_t j, void* host_out, void* stream);

/* Pivot data of block column j (NEW numbering) from a factorization with opt.pivot = 1, to host
 * memory: e_out (c128 [m_j], may be NULL) holds the sub-diagonal entry of every 2 x 2 pivot block
 * of D_j at its first row (0 elsewhere; d3m_get_pivots gives the diagonal), perm_out (int32
 * [m_j], may be NULL) the order of the block's unknowns after the pivoting inside its tiles
 * (pivot position i of the block holds its unknown perm_out[i]).  Without pivoting: zeros and
 * the identity.  Synchronizes the stream. */
int d3m_get_pivot_blocks(d3m_handle h, int32_t j, void* e_out, int32_t* perm_out, void* stream);

/* Task trace of the last factorization (handle created with D3M_DEBUG_TRACE): copies up to
 * `cap` records of 10 int64 each {start_ns, end_ns, sm_id, flags | (tile << 8) | (nk << 40), t1,
 * t2, t3, t4, ready_ns, releaser}, indexed by task id (flags: 1 diagonal tile, 4 update task;
 * nk: tile products of the task), to host memory and stores the number of tasks
 * in *count; t1..t4 are phase marks of the tensor-core engine (products done, S staged,
 * factor / triangular solve done, tile stored; -1 where a phase does not occur); ready_ns is
 * when the task's last dependency was released and releaser the task that released it (both
 * -1 for tasks ready at launch; every field is -1 before a task runs), so following releasers back from the last task to finish
 * gives the critical path as it ran.  Synchronizes the stream.
 * D3M_ERR_STATE if tracing was not enabled. */
int d3m_get_trace(d3m_handle h, int64_t* host_out, int64_t cap, int64_t* count, void* stream);

/* Synchronizes the stream, then fills `info` (structure + the last factor/solve results). */
int d3m_get_info(d3m_handle h, d3m_info* info, void* stream);

/* Text of the last error on h (static string if h is NULL).  Never NULL. */
const char* d3m_last_error(d3m_handle h);

/* Frees every library-owned buffer.  Safe on NULL. */
void d3m_destroy(d3m_handle h);

#ifdef __cplusplus
}
#endif
#endif /* D3M_H */
