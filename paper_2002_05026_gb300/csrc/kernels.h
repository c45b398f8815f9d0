// Launch interfaces of the device kernels (host side of the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "symbolic.h"

namespace d3m {

struct FactorParams;

struct SweepLaunch {
  int* status;                     // device word: D3M_ERR_TIMEOUT if a bounded wait expired
  int b, nrhs, nlevels, max_rows, accumulate;
  int64_t n, npad;
  const double2* src;              // right-hand side (caller numbering, c128)
  double2* dst;                    // solution (caller numbering, c128): = or += result
  const int64_t* pad2orig;         // [npad] original row of a padded row, -1 for padding
  const void* L;
  const void* Linv;
  const void* D;
  void* Y;                         // [nrhs][npad] work vector
  void* P;                         // partials
  const int64_t* fwd_group_ptr;    // host [nlevels+1]
  const int64_t* bwd_group_ptr;    // host [nlevels+1]
  const SolveGroup* fwd_groups;    // device
  const SolveGroup* bwd_groups;    // device
  const SolveItem* fwd_items;      // device
  const SolveItem* bwd_items;      // device
  const int64_t* fwd_slot_ptr;     // device [NT]
  const int64_t* bwd_slot_ptr;     // device [NT]
  const int32_t* lev_blocks;       // device, blocks grouped by level
  const int64_t* lev_ptr;          // host [nlevels+1]
  const int32_t* lev_tiles;        // device, tile indices of the blocks of each level
  const int64_t* lev_tile_ptr;     // host [nlevels+1]
  const int32_t* tstart;           // device [N+1]
  const int64_t* tcolptr;          // device [NT+1]
  const int32_t* lev_maxnt;        // host [nlevels]: most tiles of one block in the level
  const int32_t* lev_maxcnt_fwd;   // host [nlevels]: most forward partials of one tile row
  const int32_t* lev_maxcnt_bwd;   // host [nlevels]: most backward partials of one tile column
  const void* Inv;                 // off-diagonal tiles of the diagonal blocks' inverses, or nullptr
  const int* done;                 // device [instances]: converged instances are skipped, or nullptr
  const int32_t* tinst;            // device [NT]: instance of every tile row (permuted numbering)
  unsigned* dmax;                  // device [instances][ld_norm]: max |correction| of the step
  int ld_norm;
  const int64_t* inv_off;          // device [N]: first tile of block k in Inv
  const void* InvT;                // transposed inverse tiles (diagonal included)
  const int64_t* invT_off;         // device [N]: first tile of block k in InvT
  const struct GatherTcMaps* tcmaps;  // operand-plane maps for the tensor-core gathers, or nullptr
  const void* E;                   // pivot mode: sub-diagonals of the 2 x 2 blocks of D, or nullptr
  int nsm;
  int64_t launches;                // out: kernels launched by launch_sweep
};

// Tensor maps of L's bf16 operand planes for the tensor-core gathers of the solve (gather_tc.cu):
// k = box {32, 128} (forward, K-major), t = box {32, 32} (backward, MN-major blocks).
struct GatherTcMaps {
  alignas(64) unsigned char k[128];
  alignas(64) unsigned char t[128];
};
int gather_tc_make_maps(void* opA, int64_t ntiles, GatherTcMaps* out, std::string& err);
int launch_gather_tc(bool fwd, const GatherTcMaps& maps, const SolveGroup* groups, const SolveItem* items,
                     const void* Y, void* P, int64_t npad, int nrhs, int* status, const int* done,
                     const int32_t* tinst, int nunits, int nsm, cudaStream_t st);

// FP64-accurate residual on the tensor cores (resid_tc.cu): digit planes of K and x.
constexpr int kResidDigits = 9;       // base-64 digits per value; 2 x kResidDigits planes per chunk
struct ResidualTc {
  const double2* K;              // stored lower blocks (c128), read by the digit kernels only
  const int64_t* kblk_off;       // [nnzb+1]
  const int32_t* blk_row;        // [nnzb] row block f of every stored block (caller numbering)
  const int32_t* blk_col;        // [nnzb] column block g
  const int32_t* m_orig;         // [N]
  const int64_t* xoff_orig;      // [N]
  const int64_t* res_ptr;        // [N+1] residual contributions of every row block
  const int32_t* res_row;        // [contributions] row block f
  const int32_t* res_src;        // [contributions] source block g
  const int32_t* res_blk;        // [contributions] stored block
  const int32_t* res_tr;         // [contributions] 1: the stored block is used transposed
  const int32_t* blk_eu;         // [nnzb] residual contribution of the block as stored (row block f)
  const int32_t* blk_et;         // [nnzb] its transposed contribution (row block g), -1 for f == g
  const int64_t* ks_plane;       // [contributions] first K digit plane
  const int64_t* xs_plane;       // [N] first x digit plane of block g (within a group's planes)
  int64_t xs_total;              // x digit planes of one right-hand-side group
  int nblk;                      // N
  const int2* rtiles;            // [row tiles] (row block f, 128-row tile)
  unsigned short* kdig;          // K digit planes (bf16), 128 x 32 each
  unsigned short* xdig;          // x digit planes (bf16), 64 x 32 each
  unsigned long long* Kmax_bits; // [nnzb] max |Re|, |Im| of every stored block (double bits)
  double2* Kdiag;                // [n] diagonal entries of K (applied in FP64)
  float* rowsum;                 // [n] row sums of |K| (for ||K||_inf)
  int* xT;                       // [groups][N][32] scale exponents of the x blocks
  int64_t n;
  const int32_t* inst;           // [N] instance of every block
  const int* done;               // [instances] converged instances are skipped (or nullptr)
  int ld_norm;
  unsigned* rmax;                // [instances][ld_norm] max |r| as float bits
  unsigned* xmax;
  unsigned* bmax;
  unsigned* kmax;                // [instances] ||K_i||_inf
  int* status;                   // device word: D3M_ERR_TIMEOUT if a bounded wait expired
  int64_t timeout_ns;
};

struct ResidTcMaps {
  alignas(64) unsigned char a[128];
  alignas(64) unsigned char b[4][128];
};

int resid_tc_make_maps(void* kdig, int64_t nplanes_a, void* xdig, int64_t nplanes_b, ResidTcMaps* out,
                       std::string& err);
int launch_kdigits(const ResidualTc& p, int nnzb, int nres, int max_rtiles, int nblk, cudaStream_t st);
int resid_tc_groups(int nrhs, int* NR);
int launch_resid_tc(const ResidualTc& p, const ResidTcMaps& maps, const double2* X, const double2* B, double2* R,
                    int nrhs, int nrtiles, int nblk, cudaStream_t st, int64_t* launches);

// Tensor maps (CUtensorMap, 128 bytes each) of the tensor-core operand planes.
struct TcMaps {
  alignas(64) unsigned char a[128];
  alignas(64) unsigned char b[128];
};

int launch_factor_simt(const FactorParams& p, bool fp64, int nblocks, cudaStream_t st);
// tf32 = false: bf16 planes of the split-BF16x3 engine; true: tf32 planes
int tc_make_maps(void* opA, void* opB, int64_t ntiles, bool tf32, TcMaps* out, std::string& err);
int launch_factor_tc(const FactorParams& p, const TcMaps& maps, bool tf32, int nblocks, cudaStream_t st);
int launch_sweep(SweepLaunch& a, bool fp64, cudaStream_t st);
// Inverses of the unit-lower diagonal blocks (c64 tiles of edge b in {64, 128}), built from L and
// the inverses of the diagonal tiles: work = (block, tile column) pairs.
int launch_inv_build(const int2* work, int nwork, const int32_t* tstart, const int64_t* tcolptr,
                     const int64_t* inv_off, const int64_t* invT_off, const void* L, const void* Linv, void* Inv,
                     void* InvT, int b, cudaStream_t st);
int launch_absmax(const double2* V, int64_t n, int nrhs, unsigned* out, cudaStream_t st);
int launch_omega(const unsigned* rmax, const unsigned* xmax, const unsigned* bmax, const unsigned* kmax,
                 const unsigned* dmax, float* dprev, int ninst, int ld, int nrhs, int* done, double tol, double ftol,
                 double* omega, double* stat, cudaStream_t st);
int launch_contract(const double2* Lam, const double2* X, int64_t n, int nrhs, const int64_t* xoff_orig,
                    const int32_t* m_orig, int nblk, double2* out, cudaStream_t st);
int launch_grad_pattern(const double2* Lam, const double2* X, int64_t n, int nrhs, const int64_t* colptr,
                        const int32_t* rowidx, const int32_t* blk_col, const int64_t* kblk_off,
                        const int64_t* xoff_orig, const int32_t* m_orig, int64_t nnzb, double2* dK,
                        cudaStream_t st);

}  // namespace d3m
