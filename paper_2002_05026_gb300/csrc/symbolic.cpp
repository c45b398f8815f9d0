// Host symbolic analysis of the D3M dual matrix K (paper Sec. II: the task graph is produced
// by a symbolic simulation of the sequential algorithm; Fig. 1(c)).
//
// Block level: struct(k) of the block factor (block elimination tree + fill).
// Tile level: every block is cut into b x b tiles (padded to a multiple of b; the padding
// unknowns carry a unit diagonal and no coupling, which leaves the factor of the real
// unknowns unchanged).  One task per lower tile (I, J) of L accumulates its Schur updates
// S_IJ = K_IJ - sum_K L_IK D_K L_JK^T in a fixed K order, then either factors the diagonal
// tile (I == J) or applies the triangular solve L_IJ = S_IJ L_JJ^{-T} D_J^{-1}.
#include "symbolic.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>
#include <numeric>

namespace d3m {

int64_t Symbolic::tile_of(int I, int J) const {
  if (J < 0 || J >= NT) return -1;
  const int32_t* first = trow.data() + tcolptr[J];
  const int32_t* last = trow.data() + tcolptr[J + 1];
  const int32_t* it = std::lower_bound(first, last, I);
  if (it == last || *it != I) return -1;
  return tcolptr[J] + (it - first);
}

static int fail(std::string& err, const char* msg, long a = -1, long b = -1) {
  char buf[256];
  snprintf(buf, sizeof buf, msg, a, b);
  err = buf;
  return D3M_ERR_INVALID;
}

int analyze(const d3m_pattern* pat, const int32_t* perm_in, int b, bool build_tasks,
            Symbolic& s, std::string& err, double prio_slack, int seg_group, const double* task_cost,
            int gather_group, bool pair_updates) {
  if (seg_group < 1) seg_group = 1;
  if (!pat || !pat->colptr || !pat->rowidx) return fail(err, "pattern or its arrays are NULL");
  const int N = pat->nblk;
  if (N <= 0) return fail(err, "nblk must be positive (got %ld)", N);
  if (b <= 0 || b > 1024) return fail(err, "tile edge %ld out of range", b);
  s = Symbolic();
  s.N = N;
  s.b = b;
  // ---------------------------------------------------------------- validation
  s.m_orig.resize(N);
  for (int f = 0; f < N; ++f) {
    int mf = pat->blk_size ? pat->blk_size[f] : pat->m;
    if (mf <= 0) return fail(err, "block %ld has non-positive size %ld", f, mf);
    s.m_orig[f] = mf;
  }
  if (pat->colptr[0] != 0) return fail(err, "colptr[0] must be 0");
  s.colptr.assign(pat->colptr, pat->colptr + N + 1);
  for (int g = 0; g < N; ++g) {
    int64_t a = s.colptr[g], e = s.colptr[g + 1];
    if (e <= a) return fail(err, "column %ld has no diagonal block", g);
    if (pat->rowidx[a] != g) return fail(err, "column %ld does not start with its diagonal", g);
    for (int64_t p = a + 1; p < e; ++p) {
      int r = pat->rowidx[p];
      if (r <= pat->rowidx[p - 1] || r >= N)
        return fail(err, "column %ld: row indices must ascend within [col, N) (row %ld)", g, r);
    }
  }
  s.nnzb_K = s.colptr[N];
  s.rowidx.assign(pat->rowidx, pat->rowidx + s.nnzb_K);
  s.kblk_off.assign(s.nnzb_K + 1, 0);
  for (int g = 0; g < N; ++g)
    for (int64_t p = s.colptr[g]; p < s.colptr[g + 1]; ++p)
      s.kblk_off[p + 1] = s.kblk_off[p] + (int64_t)s.m_orig[s.rowidx[p]] * s.m_orig[g];
  s.perm.resize(N);
  s.inv.assign(N, -1);
  for (int k = 0; k < N; ++k) {
    int f = perm_in ? perm_in[k] : k;
    if (f < 0 || f >= N || s.inv[f] >= 0) return fail(err, "perm is not a permutation (entry %ld)", k);
    s.perm[k] = f;
    s.inv[f] = k;
  }
  // upload order of K: by the elimination position of the block's lower column, then of its row
  {
    std::vector<int64_t> ord(s.nnzb_K);
    std::vector<std::pair<int, int>> key(s.nnzb_K);
    for (int g = 0; g < N; ++g)
      for (int64_t e = s.colptr[g]; e < s.colptr[g + 1]; ++e) {
        const int a = s.inv[g], c = s.inv[s.rowidx[e]];
        key[e] = {std::min(a, c), std::max(a, c)};
      }
    std::iota(ord.begin(), ord.end(), (int64_t)0);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return key[x] < key[y]; });
    s.kseq.assign(s.nnzb_K, 0);
    s.kc_off.clear();
    s.kc_len.clear();
    s.kc_seq_end.clear();
    for (int64_t q = 0; q < s.nnzb_K; ++q) {
      const int64_t e = ord[q];
      s.kseq[e] = (int32_t)q;
      const int64_t off = s.kblk_off[e], len = s.kblk_off[e + 1] - s.kblk_off[e];
      if (!s.kc_off.empty() && s.kc_off.back() + s.kc_len.back() == off && s.kc_len.back() < ((int64_t)1 << 22)) {
        s.kc_len.back() += len;
        s.kc_seq_end.back() = (int32_t)(q + 1);
      } else {
        s.kc_off.push_back(off);
        s.kc_len.push_back(len);
        s.kc_seq_end.push_back((int32_t)(q + 1));
      }
    }
  }
  s.m.resize(N);
  for (int k = 0; k < N; ++k) s.m[k] = s.m_orig[s.perm[k]];
  s.xoff_orig.assign(N + 1, 0);
  for (int f = 0; f < N; ++f) s.xoff_orig[f + 1] = s.xoff_orig[f] + s.m_orig[f];
  s.n = s.xoff_orig[N];

  // ---------------------------------------------------------------- block symbolic factor
  std::vector<std::vector<int32_t>> rows(N);
  for (int g = 0; g < N; ++g)
    for (int64_t p = s.colptr[g] + 1; p < s.colptr[g + 1]; ++p) {
      int i = s.inv[s.rowidx[p]], j = s.inv[g];
      if (i < j) std::swap(i, j);
      rows[j].push_back(i);
    }
  s.str.assign(N, {});
  s.parent.assign(N, -1);
  for (int k = 0; k < N; ++k) {
    auto& r = rows[k];
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    s.str[k] = r;
    if (!r.empty()) {
      int p = r[0];
      s.parent[k] = p;
      rows[p].insert(rows[p].end(), r.begin() + 1, r.end());
    }
    std::vector<int32_t>().swap(r);
  }
  s.rowlist.assign(N, {});
  for (int k = 0; k < N; ++k)
    for (int i : s.str[k]) s.rowlist[i].push_back(k);
  s.level.assign(N, 0);
  for (int k = 0; k < N; ++k)
    if (s.parent[k] >= 0) s.level[s.parent[k]] = std::max(s.level[s.parent[k]], s.level[k] + 1);
  s.nlevels = 0;
  for (int k = 0; k < N; ++k) s.nlevels = std::max(s.nlevels, s.level[k] + 1);
  s.depth = s.nlevels;
  s.lev_blocks.assign(s.nlevels, {});
  for (int k = 0; k < N; ++k) s.lev_blocks[s.level[k]].push_back(k);
  s.max_height = 0;
  s.nL_off = 0;
  s.n_upd_off = 0;
  double F = 0, solve = 0;
  for (int k = 0; k < N; ++k) {
    const double mk = s.m[k];
    const auto& st = s.str[k];
    s.max_height = std::max<int>(s.max_height, (int)st.size());
    s.nL_off += (int64_t)st.size();
    s.n_upd_off += (int64_t)st.size() * (st.size() - 1) / 2;
    F += (4.0 / 3.0) * mk * mk * mk;                    // FACTOR k
    solve += 8.0 * mk * mk + 6.0 * mk;                 // two triangular sweeps + diagonal
    for (size_t a = 0; a < st.size(); ++a) {
      const double mj = s.m[st[a]];
      F += 4.0 * mj * mk * mk;                          // TRSM (j, k)
      F += 4.0 * mj * mj * mk;                          // UPDATE (j, j, k)
      solve += 16.0 * mj * mk;                          // L_jk in both sweeps
      for (size_t c = a + 1; c < st.size(); ++c) F += 8.0 * s.m[st[c]] * mj * mk;  // (i, j, k)
    }
  }
  s.factor_flops = F;
  s.solve_flops_rhs = solve;
  double kent = 0;
  for (int g = 0; g < N; ++g)
    for (int64_t p = s.colptr[g]; p < s.colptr[g + 1]; ++p)
      kent += (s.rowidx[p] == g ? 1.0 : 2.0) * s.m_orig[s.rowidx[p]] * s.m_orig[g];
  s.residual_flops_rhs = 8.0 * kent;

  // residual gather lists (caller numbering)
  {
    std::vector<std::vector<int32_t>> lb(N), ls(N), lt(N);
    for (int g = 0; g < N; ++g)
      for (int64_t p = s.colptr[g]; p < s.colptr[g + 1]; ++p) {
        int f = s.rowidx[p];
        lb[f].push_back((int32_t)p); ls[f].push_back(g); lt[f].push_back(0);
        if (f != g) { lb[g].push_back((int32_t)p); ls[g].push_back(f); lt[g].push_back(1); }
      }
    s.res_ptr.assign(N + 1, 0);
    for (int f = 0; f < N; ++f) {
      s.res_ptr[f + 1] = s.res_ptr[f] + (int64_t)lb[f].size();
      s.res_blk.insert(s.res_blk.end(), lb[f].begin(), lb[f].end());
      s.res_src.insert(s.res_src.end(), ls[f].begin(), ls[f].end());
      s.res_tr.insert(s.res_tr.end(), lt[f].begin(), lt[f].end());
    }
  }

  // ---------------------------------------------------------------- tiles
  s.ntile.resize(N);
  s.tstart.assign(N + 1, 0);
  for (int k = 0; k < N; ++k) {
    s.ntile[k] = (s.m[k] + b - 1) / b;
    s.tstart[k + 1] = s.tstart[k] + s.ntile[k];
  }
  s.NT = s.tstart[N];
  s.npad = (int64_t)s.NT * b;
  s.xoff.resize(N + 1);
  for (int k = 0; k <= N; ++k) s.xoff[k] = (int64_t)s.tstart[k] * b;
  s.tblk.resize(s.NT);
  for (int k = 0; k < N; ++k)
    for (int t = 0; t < s.ntile[k]; ++t) s.tblk[s.tstart[k] + t] = k;
  s.tcolptr.assign(s.NT + 1, 0);
  for (int J = 0; J < s.NT; ++J) {
    int q = s.tblk[J];
    int64_t cnt = s.tstart[q + 1] - J;
    for (int p : s.str[q]) cnt += s.ntile[p];
    s.tcolptr[J + 1] = s.tcolptr[J] + cnt;
  }
  s.trow.resize(s.tcolptr[s.NT]);
  for (int J = 0; J < s.NT; ++J) {
    int q = s.tblk[J];
    int64_t w = s.tcolptr[J];
    for (int I = J; I < s.tstart[q + 1]; ++I) s.trow[w++] = I;
    for (int p : s.str[q])
      for (int I = s.tstart[p]; I < s.tstart[p + 1]; ++I) s.trow[w++] = I;
  }
  s.diag_tile.resize(s.NT);
  for (int J = 0; J < s.NT; ++J) s.diag_tile[J] = (int32_t)s.tcolptr[J];
  const int64_t ntiles = s.tcolptr[s.NT];
  if (ntiles >= (int64_t)1 << 31) return fail(err, "too many tiles for 32-bit task ids");

  // counts of tile updates and task-graph edges (always computed)
  s.n_tile_updates = 0;
  s.n_edges = 0;
  for (int J = 0; J < s.NT; ++J) {
    int q = s.tblk[J];
    for (int64_t t = s.tcolptr[J]; t < s.tcolptr[J + 1]; ++t) {
      int I = s.trow[t], p = s.tblk[I];
      int64_t nk = J - s.tstart[q];
      int64_t ns = (nk >= 2) ? 2 : nk;
      const auto& rp = s.rowlist[p];
      const auto& rq = s.rowlist[q];
      if (p == q) {
        for (int k : rq) { nk += s.ntile[k]; ++ns; }
      } else {
        size_t a = 0, c = 0;
        while (a < rp.size() && c < rq.size()) {
          if (rp[a] < rq[c]) ++a;
          else if (rp[a] > rq[c]) ++c;
          else { nk += s.ntile[rp[a]]; ++ns; ++a; ++c; }
        }
      }
      s.n_tile_updates += nk;
      // segment sources, the chain of update tasks into the final task, and the diagonal tile
      // for a triangular solve (off-diagonal tiles give every segment to an update task)
      if (I == J) s.n_edges += nk + (ns > 1 ? ns - 1 : 0);
      else s.n_edges += 2 * nk + ns + 1;
    }
  }
  if (!build_tasks) return D3M_OK;

  // ---------------------------------------------------------------- tasks + K-lists
  // pass 1: K-lists (grouped by source block column) and segment counts per tile
  s.ntiles = ntiles;
  std::vector<int64_t> kl_ptr(ntiles + 1, 0);
  auto common_blocks = [&](int p, int q, std::vector<int32_t>& out) {
    out.clear();
    const auto& rp = s.rowlist[p];
    const auto& rq = s.rowlist[q];
    if (p == q) { out = rq; return; }
    std::set_intersection(rp.begin(), rp.end(), rq.begin(), rq.end(), std::back_inserter(out));
  };
  std::vector<int32_t> ks;
  std::vector<int32_t> nseg(ntiles, 0);
  std::vector<int32_t> nsrc(ntiles, 0);   // source-block segments (the ones that may be paired)
  for (int J = 0; J < s.NT; ++J) {
    int q = s.tblk[J];
    for (int64_t t = s.tcolptr[J]; t < s.tcolptr[J + 1]; ++t) {
      int I = s.trow[t], p = s.tblk[I];
      common_blocks(p, q, ks);
      int64_t nk = J - s.tstart[q];
      for (int k : ks) nk += s.ntile[k];
      kl_ptr[t + 1] = nk;
      // the in-block part is cut into [tstart, J-1) and [J-1, J): the last tile column K = J-1
      // becomes ready last (it is on the critical path), the others earlier; the source blocks
      // before it go seg_group to a segment
      const int nib = J - s.tstart[q];
      nsrc[t] = (int32_t)((ks.size() + seg_group - 1) / seg_group);
      nseg[t] = nsrc[t] + (nib >= 2 ? 2 : nib);
    }
  }
  for (int64_t t = 0; t < ntiles; ++t) kl_ptr[t + 1] += kl_ptr[t];
  s.klist.resize(kl_ptr[ntiles]);
  // update tasks per tile: off-diagonal tiles hand every segment to UPDATE tasks so that their
  // final task (staging + triangular solve) is all that waits for the diagonal tile; a diagonal
  // tile keeps its last segment in its final task
  std::vector<uint8_t> offd(ntiles, 0);
  for (int J = 0; J < s.NT; ++J)
    for (int64_t t = s.tcolptr[J]; t < s.tcolptr[J + 1]; ++t) offd[t] = (s.trow[t] != J);
  auto n_seg_upd = [&](int64_t t) -> int64_t { return offd[t] ? nseg[t] : std::max(0, nseg[t] - 1); };
  // pairs: leader (I, J) with J at an even offset in block q, follower (I, J + 1) in the same
  // block; both have the same source blocks, so the first nsrc segments coincide
  std::vector<int64_t> partner(ntiles, -1), leader_of(ntiles, -1);
  std::vector<int32_t> npair(ntiles, 0);
  if (pair_updates) {
    for (int J = 0; J + 1 < s.NT; ++J) {
      const int q = s.tblk[J];
      if ((J - s.tstart[q]) % 2 != 0 || J + 1 >= s.tstart[q + 1]) continue;
      for (int64_t t = s.tcolptr[J]; t < s.tcolptr[J + 1]; ++t) {
        const int I = s.trow[t];
        if (I < J + 1 || nsrc[t] == 0) continue;
        const int64_t t2 = s.tile_of(I, J + 1);
        if (t2 < 0) continue;
        const int np = (int)std::min<int64_t>(nsrc[t], std::min(n_seg_upd(t), n_seg_upd(t2)));
        if (np <= 0) continue;
        partner[t] = t2;
        leader_of[t2] = t;
        npair[t] = npair[t2] = np;
      }
    }
  }
  // update TASKS of a tile: a follower's paired segments run in its leader's tasks
  auto n_upd = [&](int64_t t) -> int64_t { return n_seg_upd(t) - (leader_of[t] >= 0 ? npair[t] : 0); };
  int64_t nupd = 0;
  for (int64_t t = 0; t < ntiles; ++t) nupd += n_upd(t);
  const int64_t ntask = ntiles + nupd;
  if (ntask >= (int64_t)1 << 31) return fail(err, "too many tasks for 32-bit task ids");
  s.tasks.resize(ntask);
  s.ndeps.assign(ntask, 0);
  s.n_acc = 0;
  // task ids: final task of tile t = t; update tasks numbered after the tiles, by tile
  std::vector<int64_t> upd_first(ntiles, -1);
  {
    int64_t nextu = ntiles;
    for (int64_t t = 0; t < ntiles; ++t)
      if (n_upd(t) > 0) { upd_first[t] = nextu; nextu += n_upd(t); }
  }
  // accumulator slots: every tile with at least one update segment
  std::vector<int32_t> sidx_of(ntiles, -1);
  for (int64_t t = 0; t < ntiles; ++t)
    if (n_seg_upd(t) > 0) sidx_of[t] = (int32_t)(s.n_acc++);
  // task id of update segment sg of tile t (paired segments of a follower: its leader's task)
  auto upd_id = [&](int64_t t, int sg) -> int64_t {
    if (leader_of[t] >= 0) return sg < npair[t] ? upd_first[leader_of[t]] + sg : upd_first[t] + (sg - npair[t]);
    return upd_first[t] + sg;
  };
  // dependencies per task id, then successor lists (CSR)
  std::vector<std::vector<int32_t>> tdeps(ntask);
  for (int J = 0; J < s.NT; ++J) {
    int q = s.tblk[J];
    for (int64_t t = s.tcolptr[J]; t < s.tcolptr[J + 1]; ++t) {
      int I = s.trow[t], p = s.tblk[I];
      common_blocks(p, q, ks);
      int64_t w = kl_ptr[t];
      // segment boundaries (offsets into this tile's K-list)
      std::vector<int64_t> sb;
      sb.push_back(w);
      auto push = [&](int K) {
        int64_t a = s.tile_of(I, K), bb = s.tile_of(J, K);
        const int64_t b2 = partner[t] >= 0 ? s.tile_of(J + 1, K) : -1;
        s.klist[w++] = KEntry{(int32_t)a, (int32_t)bb, K, (int32_t)b2};
      };
      for (size_t a = 0; a < ks.size(); ++a) {
        for (int K = s.tstart[ks[a]]; K < s.tstart[ks[a] + 1]; ++K) push(K);
        if ((a + 1) % seg_group == 0 || a + 1 == ks.size()) sb.push_back(w);
      }
      if (J - s.tstart[q] >= 2) {
        for (int K = s.tstart[q]; K < J - 1; ++K) push(K);
        sb.push_back(w);
      }
      if (J > s.tstart[q]) {
        push(J - 1);
        sb.push_back(w);
      }
      const int ns = (int)sb.size() - 1;           // == nseg[t]
      TileTask base;
      std::memset(&base, 0, sizeof base);
      base.tile = (int32_t)t;
      base.diag = s.diag_tile[J];
      base.col = J;
      base.r0 = (I - s.tstart[p]) * b;
      base.c0 = (J - s.tstart[q]) * b;
      base.rv = std::min(b, s.m[p] - base.r0);
      base.cv = std::min(b, s.m[q] - base.c0);
      int fp = s.perm[p], fq = s.perm[q];
      int scol = fq, srow = fp;
      base.k_tr = 0;
      if (fp < fq) { scol = fp; srow = fq; base.k_tr = 1; }
      base.k_off = -1;
      base.kseq = -1;
      base.k_ld = s.m_orig[srow];
      const int32_t* first = s.rowidx.data() + s.colptr[scol];
      const int32_t* last = s.rowidx.data() + s.colptr[scol + 1];
      const int32_t* it = std::lower_bound(first, last, srow);
      if (it != last && *it == srow) {
        base.k_off = s.kblk_off[s.colptr[scol] + (it - first)];
        base.kseq = s.kseq[s.colptr[scol] + (it - first)];
      }
      base.flags = (I == J ? TF_DIAG : 0) | (p == q ? TF_SAME_BLOCK : 0);
      const int nu = (int)n_seg_upd(t);             // update segments of this tile
      base.sidx = sidx_of[t];
      base.tile2 = -1;
      base.c0_2 = base.cv2 = 0;
      base.sidx2 = -1;
      auto seg_deps = [&](int sg, std::vector<int32_t>& d) {
        for (int64_t e = sb[sg]; e < sb[sg + 1]; ++e) {
          d.push_back(s.klist[e].a_tile);
          if (I != J) d.push_back(s.klist[e].b_tile);
        }
      };
      // update tasks: segments 0..nu-1, chained (a follower's first npair segments are its
      // leader's paired tasks, built there)
      const int sg0 = leader_of[t] >= 0 ? npair[t] : 0;
      for (int sg = sg0; sg < nu; ++sg) {
        const int64_t id = upd_id(t, sg);
        TileTask T = base;
        T.kl_off = sb[sg];
        T.nk = (int32_t)(sb[sg + 1] - sb[sg]);
        T.flags |= TF_UPDATE | (sg > 0 ? TF_S_IN : 0);
        auto& d = tdeps[id];
        seg_deps(sg, d);
        if (partner[t] >= 0 && sg < npair[t]) {
          // paired segment: the follower (I, J + 1) takes the same L_IK tiles and W_{J+1,K}
          const int64_t t2 = partner[t];
          T.flags |= TF_PAIR;
          T.tile2 = (int32_t)t2;
          T.c0_2 = (J + 1 - s.tstart[q]) * b;
          T.cv2 = std::min(b, s.m[q] - T.c0_2);
          T.sidx2 = sidx_of[t2];
          for (int64_t e = sb[sg]; e < sb[sg + 1]; ++e) {
            if (s.klist[e].b2_tile < 0) return fail(err, "internal: paired segment without tile (J+1, K)");
            d.push_back(s.klist[e].b2_tile);
          }
        }
        if (sg > 0) d.push_back((int32_t)upd_id(t, sg - 1));
        s.tasks[id] = T;
        s.ndeps[id] = (int32_t)d.size();
      }
      // final task: the remaining segment (diagonal tile only), then factor / triangular solve
      {
        TileTask T = base;
        const bool has_seg = nu < ns;
        T.kl_off = has_seg ? sb[nu] : kl_ptr[t];
        T.nk = has_seg ? (int32_t)(sb[nu + 1] - sb[nu]) : 0;
        if (nu > 0) T.flags |= TF_S_IN;
        s.tasks[t] = T;
        auto& d = tdeps[t];
        if (has_seg) seg_deps(nu, d);
        if (nu > 0) d.push_back((int32_t)upd_id(t, nu - 1));
        if (I != J) d.push_back(s.diag_tile[J]);
        s.ndeps[t] = (int32_t)d.size();
      }
    }
  }
  // successor lists
  std::vector<int64_t> scount(ntask + 1, 0);
  for (int64_t id = 0; id < ntask; ++id)
    for (int32_t d : tdeps[id]) scount[d + 1]++;
  for (int64_t id = 0; id < ntask; ++id) scount[id + 1] += scount[id];
  s.succ_ptr = scount;
  s.succ.resize(scount[ntask]);
  std::vector<int64_t> wpos(scount.begin(), scount.end() - 1);
  for (int64_t id = 0; id < ntask; ++id)
    for (int32_t d : tdeps[id]) s.succ[wpos[d]++] = (int32_t)id;
  std::vector<std::vector<int32_t>>().swap(tdeps);
  s.n_edges = (int64_t)s.succ.size();
  // Priority: an estimate of each task's duration (diagonal factorization + inverse,
  // triangular-solve final, update segment of nk tile products) gives the longest path from
  // the sources to a task's start (tl) and from its start to the end (bl); tasks whose slack
  // CP - tl - bl is within prio_slack * CP go to the priority lane, which the device
  // scheduler serves first, so the chain of diagonal factorizations does not queue behind
  // hundreds of ready updates.  The durations are the caller's measured model (the paper
  // weights its dual tasks with benchmarked GEMM, sytrf and triSolve times, Sec. II) or, without
  // one, a built-in model in microseconds of the tensor-core engine.
  {
    double cm[6] = {4.0, 3.0, 110.0, 3.0, 20.0, 3.0};
    if (task_cost) {
      bool any = false;
      for (int q = 0; q < 6; ++q) any = any || task_cost[q] > 0;
      if (any)
        for (int q = 0; q < 6; ++q) cm[q] = task_cost[q] > 0 ? task_cost[q] : 0.0;
    }
    std::vector<double> cost(ntask), tl(ntask, 0.0), bl(ntask, 0.0);
    for (int64_t id = 0; id < ntask; ++id) {
      const TileTask& T = s.tasks[id];
      const int k = (T.flags & TF_UPDATE) ? 0 : ((T.flags & TF_DIAG) ? 2 : 4);
      cost[id] = cm[k] + cm[k + 1] * T.nk * ((T.flags & TF_PAIR) ? 2 : 1);
    }
    std::vector<int32_t> indeg(s.ndeps.begin(), s.ndeps.end()), order;
    order.reserve(ntask);
    for (int64_t id = 0; id < ntask; ++id)
      if (indeg[id] == 0) order.push_back((int32_t)id);
    for (size_t q = 0; q < order.size(); ++q) {
      const int32_t t = order[q];
      for (int64_t e = s.succ_ptr[t]; e < s.succ_ptr[t + 1]; ++e) {
        const int32_t v = s.succ[e];
        tl[v] = std::max(tl[v], tl[t] + cost[t]);
        if (--indeg[v] == 0) order.push_back(v);
      }
    }
    if ((int64_t)order.size() != ntask) return fail(err, "internal: the task graph has a cycle");
    double cp = 0.0;
    for (int64_t q = (int64_t)order.size() - 1; q >= 0; --q) {
      const int32_t t = order[q];
      double m = 0.0;
      for (int64_t e = s.succ_ptr[t]; e < s.succ_ptr[t + 1]; ++e) m = std::max(m, bl[s.succ[e]]);
      bl[t] = cost[t] + m;
      cp = std::max(cp, tl[t] + bl[t]);
    }
    s.n_prio = 0;
    for (int64_t id = 0; id < ntask; ++id)
      if (cp - tl[id] - bl[id] <= prio_slack * cp) {
        s.tasks[id].flags |= TF_PRIO;
        ++s.n_prio;
      }
  }
  s.init_ready.clear();
  s.init_ready_hi.clear();
  for (int64_t id = 0; id < ntask; ++id)
    if (s.ndeps[id] == 0) (s.tasks[id].flags & TF_PRIO ? s.init_ready_hi : s.init_ready).push_back((int32_t)id);

  // ---------------------------------------------------------------- solve level sets
  s.fwd_item_ptr.assign(s.nlevels + 1, 0);
  s.bwd_item_ptr.assign(s.nlevels + 1, 0);
  s.fwd_slot_ptr.assign(s.NT + 1, 0);
  s.bwd_slot_ptr.assign(s.NT + 1, 0);
  s.fwd_items.clear();
  s.bwd_items.clear();
  s.max_level_items = 0;
  for (int lv = 0; lv < s.nlevels; ++lv) {
    int64_t f0 = (int64_t)s.fwd_items.size(), b0 = (int64_t)s.bwd_items.size();
    for (int k : s.lev_blocks[lv]) {
      for (int I = s.tstart[k]; I < s.tstart[k + 1]; ++I)       // forward: row I gathers
        for (int j : s.rowlist[k])
          for (int J = s.tstart[j]; J < s.tstart[j + 1]; ++J) {
            int32_t slot = (int32_t)(s.fwd_items.size() - f0);
            s.fwd_items.push_back(SolveItem{(int32_t)s.tile_of(I, J), J, I, slot});
          }
      for (int J = s.tstart[k]; J < s.tstart[k + 1]; ++J)       // backward: column J gathers
        for (int i : s.str[k])
          for (int I = s.tstart[i]; I < s.tstart[i + 1]; ++I) {
            int32_t slot = (int32_t)(s.bwd_items.size() - b0);
            s.bwd_items.push_back(SolveItem{(int32_t)s.tile_of(I, J), I, J, slot});
          }
    }
    s.fwd_item_ptr[lv + 1] = (int64_t)s.fwd_items.size();
    s.bwd_item_ptr[lv + 1] = (int64_t)s.bwd_items.size();
    s.max_level_items = std::max(s.max_level_items, s.fwd_item_ptr[lv + 1] - f0);
    s.max_level_items = std::max(s.max_level_items, s.bwd_item_ptr[lv + 1] - b0);
  }
  // Items of one destination are contiguous (pushed in a row).  A gather block sums the
  // products of up to G consecutive items of one destination into one partial slot; G grows
  // with the level's width so that wide levels write (and the chains read) fewer partials
  // while narrow levels keep one item per block.  slot_ptr[dst] = first slot of the level
  // (relative to its start) | number of slots << 32.  gather_group caps G: 1 for the SIMT
  // gathers (per-item latency dominates), more for the tensor-core gathers, whose items of one
  // group accumulate in tensor memory.
  const int nh = s.b / 64;
  // about two gather blocks per SM (SIMT); four groups per SM for the tensor-core gathers, whose
  // blocks are persistent over the level's groups
  const int64_t kGatherBlocks = gather_group > 1 ? 1216 : 304;
  const int64_t kGroupMax = std::max(1, gather_group);
  s.fwd_group_ptr.assign(s.nlevels + 1, 0);
  s.bwd_group_ptr.assign(s.nlevels + 1, 0);
  s.fwd_groups.clear();
  s.bwd_groups.clear();
  s.max_level_groups = 0;
  s.max_group = 1;
  for (int I = 0; I < s.NT; ++I) { s.fwd_slot_ptr[I] = 0; s.bwd_slot_ptr[I] = 0; }
  auto make_groups = [&](const std::vector<SolveItem>& items, int64_t i0, int64_t i1,
                         std::vector<SolveGroup>& groups, std::vector<int64_t>& slot_ptr) {
    const int64_t g0 = (int64_t)groups.size();
    const int64_t G = std::max<int64_t>(1, std::min<int64_t>(kGroupMax, (i1 - i0) * nh / kGatherBlocks));
    int64_t e = i0;
    while (e < i1) {
      const int d = items[e].dst;
      int64_t e1 = e;
      while (e1 < i1 && items[e1].dst == d) ++e1;
      const int64_t first_slot = (int64_t)groups.size() - g0;
      for (int64_t q = e; q < e1; q += G) {
        const int32_t cnt = (int32_t)std::min<int64_t>(G, e1 - q);
        groups.push_back(SolveGroup{(int32_t)q, cnt, (int32_t)((int64_t)groups.size() - g0), d});
        s.max_group = std::max(s.max_group, cnt);
      }
      const int64_t nslot = (int64_t)groups.size() - g0 - first_slot;
      slot_ptr[d] = first_slot | (nslot << 32);
      e = e1;
    }
    return (int64_t)groups.size() - g0;
  };
  for (int lv = 0; lv < s.nlevels; ++lv) {
    const int64_t nf = make_groups(s.fwd_items, s.fwd_item_ptr[lv], s.fwd_item_ptr[lv + 1], s.fwd_groups,
                                   s.fwd_slot_ptr);
    const int64_t nb = make_groups(s.bwd_items, s.bwd_item_ptr[lv], s.bwd_item_ptr[lv + 1], s.bwd_groups,
                                   s.bwd_slot_ptr);
    s.fwd_group_ptr[lv + 1] = (int64_t)s.fwd_groups.size();
    s.bwd_group_ptr[lv + 1] = (int64_t)s.bwd_groups.size();
    s.max_level_groups = std::max(s.max_level_groups, std::max(nf, nb));
  }
  return D3M_OK;
}

// ---------------------------------------------------------------- grid nested dissection
int order_grid_nd(int nx, int ny, int nz, std::vector<int32_t>& perm) {
  if (nx <= 0 || ny <= 0 || nz <= 0) return D3M_ERR_INVALID;
  struct If { int c[3]; int ax; };
  std::vector<If> ifs;
  for (int ix = 0; ix < nx; ++ix)
    for (int iy = 0; iy < ny; ++iy)
      for (int iz = 0; iz < nz; ++iz) {
        const int lim[3] = {nx, ny, nz};
        const int c[3] = {ix, iy, iz};
        for (int ax = 0; ax < 3; ++ax)
          if (c[ax] + 1 < lim[ax]) ifs.push_back(If{{ix, iy, iz}, ax});
      }
  perm.clear();
  std::function<void(const int*, const int*)> rec = [&](const int* lo, const int* hi) {
    std::vector<int32_t> own;
    for (size_t f = 0; f < ifs.size(); ++f) {
      bool in = true;
      for (int a = 0; a < 3; ++a) {
        int c0 = ifs[f].c[a], c1 = c0 + (ifs[f].ax == a ? 1 : 0);
        if (c0 < lo[a] || c1 >= hi[a]) { in = false; break; }
      }
      if (in) own.push_back((int32_t)f);
    }
    int ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    int ax = 0;
    for (int a = 1; a < 3; ++a)
      if (ext[a] > ext[ax]) ax = a;
    if (ext[ax] <= 1 || own.size() <= 1) {
      perm.insert(perm.end(), own.begin(), own.end());
      return;
    }
    int mid = lo[ax] + ext[ax] / 2;
    int lhi[3] = {hi[0], hi[1], hi[2]};
    int rlo[3] = {lo[0], lo[1], lo[2]};
    lhi[ax] = mid;
    rlo[ax] = mid;
    rec(lo, lhi);
    rec(rlo, hi);
    for (int32_t f : own)
      if (ifs[f].ax == ax && ifs[f].c[ax] == mid - 1) perm.push_back(f);
  };
  const int lo[3] = {0, 0, 0};
  const int hi[3] = {nx, ny, nz};
  rec(lo, hi);
  return perm.size() == ifs.size() ? D3M_OK : D3M_ERR_INVALID;
}

}  // namespace d3m
