// C ABI of libopf (declared in include/opf.h): set-up, power flow, reduced
// gradient and reduced Hessian.  Host orchestration only; all arithmetic of
// the path runs in the kernels of opf_kernels.cu.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "opf_internal.h"

using namespace opf;

static thread_local std::string g_err;

namespace opf {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace opf

#define FAIL(st, msg)  \
  do {                 \
    g_err = (msg);     \
    return (st);       \
  } while (0)

#define CK(call)                                                            \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      g_err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
      return OPF_ECUDA;                                                     \
    }                                                                       \
  } while (0)

template <class T>
static opf_status dalloc(opf_ctx* c, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    FAIL(OPF_ENOMEM, "device allocation failed");
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return OPF_OK;
}

template <class T>
static opf_status dupload(opf_ctx* c, T** p, const std::vector<T>& v) {
  opf_status st = dalloc(c, p, v.size());
  if (st) return st;
  if (!v.empty()) CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return OPF_OK;
}

#define TRY(x)                     \
  do {                             \
    opf_status s_ = (x);           \
    if (s_ != OPF_OK) return s_;   \
  } while (0)

static int find_pos(const Symbolic& s, int row, int col) {
  int lo = s.rp[row], hi = s.rp[row + 1] - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (s.ci[mid] < col) lo = mid + 1; else hi = mid;
  }
  return (s.ci[lo] == col) ? lo : -1;
}

static opf_status load_impl(opf_ctx* c, const opf_network_desc* d) {
  std::string why = build_hostnet(d, c->h);
  if (!why.empty()) FAIL(OPF_EINVAL, why);
  HostNet& h = c->h;
  Symbolic& s = c->s;
  build_symbolic(h, s);
  const int nb = h.nb, nl = h.nl, nx = h.nx, nnz = (int)s.ci.size();
  CK(cudaGetDevice(&c->device));
  CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));

  // pivot-order positions of the bus variables
  std::vector<int> pth(nb, -1), pvv(nb, -1);
  for (int i = 0; i < nb; i++) {
    if (h.xth[i] >= 0) pth[i] = s.iperm[h.xth[i]];
    if (h.xv[i] >= 0) pvv[i] = s.iperm[h.xv[i]];
  }
  // Jacobian slots (positions of the entries of G_x in the filled pattern)
  std::vector<int> slot_self(4 * (size_t)nb, -1), slot_adj(8 * (size_t)nl, -1);
  for (int i = 0; i < nb; i++) {
    if (h.type[i] == REF) continue;
    const bool pq = h.type[i] == PQ;
    slot_self[4 * i + 0] = find_pos(s, pth[i], pth[i]);
    if (pq) {
      slot_self[4 * i + 1] = find_pos(s, pth[i], pvv[i]);
      slot_self[4 * i + 2] = find_pos(s, pvv[i], pth[i]);
      slot_self[4 * i + 3] = find_pos(s, pvv[i], pvv[i]);
    }
    for (int k = h.adj_ptr[i]; k < h.adj_ptr[i + 1]; k++) {
      const int e = h.adj[k], l = e >> 1;
      const int o = (e & 1) ? h.f[l] : h.t[l];
      int* sl = &slot_adj[4 * (size_t)e];
      if (h.type[o] != REF) sl[0] = find_pos(s, pth[i], pth[o]);
      if (h.type[o] == PQ) sl[1] = find_pos(s, pth[i], pvv[o]);
      if (pq && h.type[o] != REF) sl[2] = find_pos(s, pvv[i], pth[o]);
      if (pq && h.type[o] == PQ) sl[3] = find_pos(s, pvv[i], pvv[o]);
      for (int q = 0; q < 4; q++)
        if (sl[q] == -1 && ((q == 0 && h.type[o] != REF) || (q == 1 && h.type[o] == PQ) ||
                            (q == 2 && pq && h.type[o] != REF) || (q == 3 && pq && h.type[o] == PQ)))
          FAIL(OPF_EINVAL, "internal: Jacobian entry outside the filled pattern");
    }
  }
  // transposition map
  std::vector<int> tmap(nnz);
  for (int i = 0; i < nx; i++)
    for (int p = s.rp[i]; p < s.rp[i + 1]; p++) tmap[p] = find_pos(s, s.ci[p], i);
  // columns of L: (row, position in row) sorted by row
  std::vector<int> lcnt(nx + 1, 0);
  for (int r = 0; r < nx; r++)
    for (int p = s.rp[r]; p < s.dp[r]; p++) lcnt[s.ci[p] + 1]++;
  for (int j = 0; j < nx; j++) lcnt[j + 1] += lcnt[j];
  std::vector<int> lcol_row(lcnt[nx]), lcol_pos(lcnt[nx]);
  {
    std::vector<int> fill(lcnt.begin(), lcnt.end() - 1);
    for (int r = 0; r < nx; r++)
      for (int p = s.rp[r]; p < s.dp[r]; p++) {
        const int j = s.ci[p];
        lcol_row[fill[j]] = r;
        lcol_pos[fill[j]++] = p;
      }
  }
  // level row lists and LU tasks
  auto level_lists = [&](const std::vector<int>& lev, int nlev, std::vector<int>& ptr, std::vector<int>& rows) {
    ptr.assign(nlev + 1, 0);
    for (int i = 0; i < nx; i++) ptr[lev[i] + 1]++;
    for (int k = 0; k < nlev; k++) ptr[k + 1] += ptr[k];
    rows.assign(nx, 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < nx; i++) rows[fill[lev[i]]++] = i;
  };
  std::vector<int> lrows_f, lrows_b;
  level_lists(s.lev_f, s.nlev_f, c->h_lev_ptr_f, lrows_f);
  level_lists(s.lev_b, s.nlev_b, c->h_lev_ptr_b, lrows_b);
  // dense trailing block [r0, nx): every row's upper part runs to the last column
  int r0 = nx - 1;
  while (r0 > 0 && s.rp[r0] - s.dp[r0 - 1] - 1 == nx - r0) r0--;
  // any suffix of a dense block is dense: keep at most kMaxDenseRows rows so the
  // packed triangle fits in shared memory (the rest join the level schedule)
  constexpr int kMaxDenseRows = 200;
  r0 = std::max(r0, nx - kMaxDenseRows);
  // bus of each pivot row; a block (theta and v of a PQ bus) never straddles r0
  std::vector<int> rowbus(nx);
  {
    std::vector<int> vbus(nx, -1);
    for (int b = 0; b < nb; b++) {
      if (h.xth[b] >= 0) vbus[h.xth[b]] = b;
      if (h.xv[b] >= 0) vbus[h.xv[b]] = b;
    }
    for (int r = 0; r < nx; r++) rowbus[r] = vbus[s.perm[r]];
  }
  if (r0 > 0 && r0 < nx && rowbus[r0 - 1] == rowbus[r0]) r0++;
  // sweep schedules of the other rows; rows of a level sorted by length (longest first)
  std::vector<int> sched_ptr_f, sched_rows_f, sched_ptr_b, sched_rows_b;
  {
    auto build = [&](const std::vector<int>& lev, bool fwd, std::vector<int>& ptr, std::vector<int>& rows) {
      int nlev = 0;
      for (int i = 0; i < r0; i++) nlev = std::max(nlev, lev[i] + 1);
      ptr.assign(nlev + 1, 0);
      for (int i = 0; i < r0; i++) ptr[lev[i] + 1]++;
      for (int k = 0; k < nlev; k++) ptr[k + 1] += ptr[k];
      rows.assign(r0, 0);
      std::vector<int> fill(ptr.begin(), ptr.end() - 1);
      for (int i = 0; i < r0; i++) rows[fill[lev[i]]++] = i;
      auto len = [&](int i) { return fwd ? s.dp[i] - s.rp[i] : s.rp[i + 1] - s.dp[i] - 1; };
      for (int k = 0; k < nlev; k++)
        std::stable_sort(rows.begin() + ptr[k], rows.begin() + ptr[k + 1],
                         [&](int a, int b) { return len(a) > len(b); });
    };
    std::vector<int> levb(nx, 0);
    for (int i = r0 - 1; i >= 0; i--) {
      int lv = 0;
      for (int p = s.dp[i] + 1; p < s.rp[i + 1]; p++)
        if (s.ci[p] < r0) lv = std::max(lv, levb[s.ci[p]] + 1);
      levb[i] = lv;
    }
    build(s.lev_f, true, sched_ptr_f, sched_rows_f);
    build(levb, false, sched_ptr_b, sched_rows_b);
  }
  // bus-block schedules of the rows below r0 (see DevNet::bmeta_f)
  std::vector<int> bsched_ptr_f, bsched_ptr_b;
  std::vector<int4> bmeta_f, bmeta_b;
  std::vector<int> bfirst;          // first pivot row of each block below r0
  std::vector<int> blev_f;          // forward level of each block
  {
    for (int r = 0; r < r0; r++)
      if (r == 0 || rowbus[r] != rowbus[r - 1]) bfirst.push_back(r);
    const int nbk = (int)bfirst.size();
    std::vector<int> bof(nx, -1);
    for (int k = 0; k < nbk; k++) {
      const int f = bfirst[k], e = (k + 1 < nbk) ? bfirst[k + 1] : r0;
      for (int r = f; r < e; r++) bof[r] = k;
    }
    auto bsize = [&](int k) { return ((k + 1 < nbk) ? bfirst[k + 1] : r0) - bfirst[k]; };
    // forward block levels (lower columns of the first row; the second row adds only the first)
    std::vector<int> lf(nbk, 0), lb(nbk, 0);
    for (int k = 0; k < nbk; k++) {
      const int f = bfirst[k];
      int lv = 0;
      for (int p = s.rp[f]; p < s.dp[f]; p++) lv = std::max(lv, lf[bof[s.ci[p]]] + 1);
      lf[k] = lv;
    }
    // backward block levels (upper columns below r0 of the last row)
    for (int k = nbk - 1; k >= 0; k--) {
      const int g = bfirst[k] + bsize(k) - 1;
      int lv = 0;
      for (int p = s.dp[g] + 1; p < s.rp[g + 1]; p++)
        if (s.ci[p] < r0) lv = std::max(lv, lb[bof[s.ci[p]]] + 1);
      lb[k] = lv;
    }
    auto rec = [&](int k, bool fwd) {
      const int f = bfirst[k], sz = bsize(k);
      if (fwd) return make_int4(f, s.rp[f], s.dp[f], sz == 2 ? s.rp[f + 1] - s.rp[f] : 0);
      const int g = f + sz - 1;
      return make_int4(g, s.dp[g] + 1, s.rp[g + 1], sz == 2 ? (s.dp[f] + 2) - (s.dp[g] + 1) : 0);
    };
    auto bbuild = [&](const std::vector<int>& lev, bool fwd, std::vector<int>& ptr, std::vector<int4>& meta) {
      int nlev = 0;
      for (int k = 0; k < nbk; k++) nlev = std::max(nlev, lev[k] + 1);
      ptr.assign(nlev + 1, 0);
      for (int k = 0; k < nbk; k++) ptr[lev[k] + 1]++;
      for (int l = 0; l < nlev; l++) ptr[l + 1] += ptr[l];
      std::vector<int> order(nbk), fill(ptr.begin(), ptr.end() - 1);
      for (int k = 0; k < nbk; k++) order[fill[lev[k]]++] = k;
      meta.resize(nbk);
      for (int k = 0; k < nbk; k++) meta[k] = rec(order[k], fwd);
      for (int l = 0; l < nlev; l++)
        std::stable_sort(meta.begin() + ptr[l], meta.begin() + ptr[l + 1],
                         [](const int4& a, const int4& b) { return a.z - a.y > b.z - b.y; });
    };
    bbuild(lf, true, bsched_ptr_f, bmeta_f);
    bbuild(lb, false, bsched_ptr_b, bmeta_b);
    blev_f = lf;
  }
  // LU tasks by bus block, grouped by block level: for block J (first pivot row
  // f, one or two rows) and each lower entry (r, f) of column f other than the
  // block's own second row, one task eliminates both columns of J from row r.
  // Record {position of A_rf, dp[f], rp[f + 1], dp[f + 1] or -1}; its Schur-update
  // targets are the positions in row r of the columns of f's upper entries past
  // the block.  A two-row block's second row is finished (L, U_vv and its U row
  // after eliminating f) by a finish record {dp[f], rp[f + 1], dp[f + 1], 0} in
  // the next level's launch, when no task reads it any more.
  std::vector<int4> btask, bfin;
  std::vector<int> btask_off(1, 0), task_map;
  c->h_task_ptr.assign(1, 0);
  c->h_fin_ptr.assign(1, 0);
  {
    const int nbk = (int)bfirst.size();
    int nl = 0;
    for (int k = 0; k < nbk; k++) nl = std::max(nl, blev_f[k] + 1);
    std::vector<std::vector<int>> at(nl);
    for (int k = 0; k < nbk; k++) at[blev_f[k]].push_back(k);
    for (int lv = 0; lv < nl; lv++) {
      for (int k : at[lv]) {
        const int f = bfirst[k], sz = ((k + 1 < nbk) ? bfirst[k + 1] : r0) - f;
        for (int q = lcnt[f]; q < lcnt[f + 1]; q++) {
          const int r = lcol_row[q];
          if (sz == 2 && r == f + 1) continue;
          btask.push_back(make_int4(lcol_pos[q], s.dp[f], s.rp[f + 1], sz == 2 ? s.dp[f + 1] : -1));
          for (int p = s.dp[f] + sz; p < s.rp[f + 1]; p++) task_map.push_back(find_pos(s, r, s.ci[p]));
          btask_off.push_back((int)task_map.size());
        }
        if (sz == 2) bfin.push_back(make_int4(s.dp[f], s.rp[f + 1], s.dp[f + 1], 0));
      }
      c->h_task_ptr.push_back((int)btask.size());
      c->h_fin_ptr.push_back((int)bfin.size());
    }
    // lanes per work item of each level launch (tasks of level lv, finish records
    // of level lv - 1): enough that the longest row takes at most four passes
    const int nlv = (int)c->h_task_ptr.size() - 1;
    c->h_lu_lanes.assign(nlv + 1, 32);
    for (int lv = 0; lv <= nlv; lv++) {
      int mx = 1;
      if (lv < nlv)
        for (int t = c->h_task_ptr[lv]; t < c->h_task_ptr[lv + 1]; t++) {
          const int4 r = btask[t];
          mx = std::max(mx, r.z - (r.y + (r.w >= 0 ? 2 : 1)));
        }
      if (lv > 0)
        for (int f = c->h_fin_ptr[lv - 1]; f < c->h_fin_ptr[lv]; f++) mx = std::max(mx, bfin[f].y - bfin[f].x - 2);
      int g = 1;
      while (g < 32 && 4 * g < mx) g *= 2;
      c->h_lu_lanes[lv] = g;
    }
  }
  // control buses: slack first, then PV
  std::vector<int> gn_bus, gn_of(nb, -1), ubus(h.nu, -1);
  gn_bus.push_back(h.ref);
  for (int i = 0; i < nb; i++)
    if (h.type[i] == PV) gn_bus.push_back(i);
  for (size_t k = 0; k < gn_bus.size(); k++) gn_of[gn_bus[k]] = (int)k;
  ubus[0] = h.ref;
  for (int i = 0; i < nb; i++)
    if (h.type[i] == PV) {
      ubus[h.uv[i]] = i;
      ubus[h.up[i]] = i;
    }

  // upload
  DevNet& n = c->dn;
  n.nb = nb;
  n.nl = nl;
  n.ng = h.ng;
  n.ref = h.ref;
  n.npv = h.npv;
  n.npq = h.npq;
  n.nx = nx;
  n.nu = h.nu;
  n.m = h.m;
  n.ngn = (int)gn_bus.size();
  n.nnz = nnz;
  n.nlev_f = (int)sched_ptr_f.size() - 1;
  n.nlev_b = (int)sched_ptr_b.size() - 1;
  n.r0 = r0;
  n.nroot = nx - r0;
  int* ip;
  double* dptr;
  TRY(dupload(c, &ip, h.f)); n.f = ip;
  TRY(dupload(c, &ip, h.t)); n.t = ip;
  TRY(dupload(c, &ip, h.gbus)); n.gbus = ip;
  TRY(dupload(c, &dptr, h.Y)); n.Y = dptr;
  TRY(dupload(c, &ip, h.type)); n.type = ip;
  TRY(dupload(c, &ip, h.gen_at)); n.gen_at = ip;
  TRY(dupload(c, &ip, h.pvpos)); n.pvpos = ip;
  TRY(dupload(c, &ip, h.pqpos)); n.pqpos = ip;
  TRY(dupload(c, &ip, h.xth)); n.xth = ip;
  TRY(dupload(c, &ip, h.xv)); n.xv = ip;
  TRY(dupload(c, &ip, h.uv)); n.uv = ip;
  TRY(dupload(c, &ip, h.up)); n.up = ip;
  TRY(dupload(c, &ip, pth)); n.pth = ip;
  TRY(dupload(c, &ip, pvv)); n.pvv = ip;
  TRY(dupload(c, &ip, h.adj_ptr)); n.adj_ptr = ip;
  TRY(dupload(c, &ip, h.adj)); n.adj = ip;
  {
    // buses by descending degree, then by the kind of bus (a generator's own
    // injection terms) and by their ends toward generator buses (last in each
    // adjacency list): four buses with the same key share a warp in the gathers
    std::vector<int> order(nb), gen_ends(nb, 0), slack_end(nb, 0);
    for (int i = 0; i < nb; i++) {
      order[i] = i;
      for (int k = h.adj_ptr[i]; k < h.adj_ptr[i + 1]; k++) {
        const int e = h.adj[k], l = e >> 1, o = (e & 1) ? h.f[l] : h.t[l];
        if (h.type[o] != PQ) gen_ends[i]++;
        if (o == h.ref) slack_end[i] = 1;
      }
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      const int da = h.adj_ptr[a + 1] - h.adj_ptr[a], db = h.adj_ptr[b + 1] - h.adj_ptr[b];
      if (da != db) return da > db;
      const int ca = gn_of[a] >= 0, cb = gn_of[b] >= 0;
      if (ca != cb) return ca > cb;
      if (gen_ends[a] != gen_ends[b]) return gen_ends[a] > gen_ends[b];
      return slack_end[a] > slack_end[b];
    });
    TRY(dupload(c, &ip, order)); n.bus_by_deg = ip;
  }
  TRY(dupload(c, &ip, gn_of)); n.gn_of = ip;
  TRY(dupload(c, &ip, gn_bus)); n.gn_bus = ip;
  {
    std::vector<int> order(gn_bus.size());
    for (size_t g = 0; g < order.size(); g++) order[g] = (int)g;
    auto deg = [&](int g) { return h.adj_ptr[gn_bus[g] + 1] - h.adj_ptr[gn_bus[g]]; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return deg(a) > deg(b); });
    TRY(dupload(c, &ip, order)); n.gn_by_deg = ip;
  }
  TRY(dupload(c, &dptr, h.c2)); n.c2 = dptr;
  TRY(dupload(c, &dptr, h.c1)); n.c1 = dptr;
  TRY(dupload(c, &c->c0, h.c0));
  TRY(dupload(c, &ip, s.rp)); n.rp = ip;
  TRY(dupload(c, &ip, s.ci)); n.ci = ip;
  TRY(dupload(c, &ip, s.dp)); n.dp = ip;
  TRY(dupload(c, &ip, s.perm)); n.perm = ip;
  {
    std::vector<int4> mf(sched_rows_f.size()), mb(sched_rows_b.size());
    for (size_t k = 0; k < mf.size(); k++) {
      const int i = sched_rows_f[k];
      mf[k] = make_int4(i, s.rp[i], s.dp[i], 0);
    }
    for (size_t k = 0; k < mb.size(); k++) {
      const int i = sched_rows_b[k];
      mb[k] = make_int4(i, s.dp[i] + 1, s.rp[i + 1], 0);
    }
    int4* q;
    TRY(dupload(c, &q, mf));
    n.lmeta_f = q;
    TRY(dupload(c, &q, mb));
    n.lmeta_b = q;
  }
  {
    int4* q4;
    TRY(dupload(c, &ip, bsched_ptr_f)); n.bptr_f = ip;
    TRY(dupload(c, &ip, bsched_ptr_b)); n.bptr_b = ip;
    TRY(dupload(c, &q4, bmeta_f)); n.bmeta_f = q4;
    TRY(dupload(c, &q4, bmeta_b)); n.bmeta_b = q4;
    n.nblev_f = (int)bsched_ptr_f.size() - 1;
    n.nblev_b = (int)bsched_ptr_b.size() - 1;
  }
  TRY(dupload(c, &ip, sched_ptr_f)); n.lev_ptr_f = ip;
  TRY(dupload(c, &ip, sched_rows_f)); n.lev_rows_f = ip;
  TRY(dupload(c, &ip, sched_ptr_b)); n.lev_ptr_b = ip;
  TRY(dupload(c, &ip, sched_rows_b)); n.lev_rows_b = ip;
  {
    std::vector<int4> busrec(nb), adjrec(2 * (size_t)nl);
    auto vslot = [&](int b) { return h.type[b] == opf::PQ ? pvv[b] : -2 - h.uv[b]; };
    for (int i = 0; i < nb; i++)
      busrec[i] = make_int4(vslot(i), h.type[i] == opf::REF ? -1 : pth[i], gn_of[i], h.up[i]);
    for (int q = 0; q < 2 * nl; q++) {
      const int e = h.adj[q], l = e >> 1, o = (e & 1) ? h.f[l] : h.t[l];
      adjrec[q] = make_int4(vslot(o), h.type[o] == opf::REF ? -1 : pth[o], gn_of[o], o == h.ref ? 1 : 0);
    }
    int4* q4;
    TRY(dupload(c, &q4, busrec));
    n.busrec = q4;
    TRY(dupload(c, &q4, adjrec));
    n.adjrec = q4;
  }
  TRY(dupload(c, &ip, slot_self)); n.slot_self = ip;
  TRY(dupload(c, &ip, slot_adj)); n.slot_adj = ip;
  TRY(dupload(c, &c->tmap, tmap));
  TRY(dupload(c, &c->lcol_row, lcol_row));
  {
    std::vector<int2> lc(lcol_row.size());
    for (size_t k = 0; k < lc.size(); k++) lc[k] = make_int2(lcol_row[k], lcol_pos[k]);
    int2* q2;
    TRY(dupload(c, &q2, lc));
    n.lcol = q2;
    TRY(dupload(c, &ip, lcnt));
    n.lcol_ptr = ip;
  }
  TRY(dupload(c, &c->lcol_pos, lcol_pos));
  TRY(dupload(c, &c->task_rec, btask));
  TRY(dupload(c, &c->task_off, btask_off));
  TRY(dupload(c, &c->fin_rec, bfin));
  TRY(dupload(c, &c->task_map, task_map));
  TRY(dupload(c, &c->ubus, ubus));
  {
    // elimination tree of L (parent of column j = first row below j with L_ij != 0)
    std::vector<int> par(nx, -1);
    for (int i = 0; i < nx; i++)
      for (int p = s.rp[i]; p < s.dp[i]; p++) {
        const int j = s.ci[p];
        if (par[j] < 0 || i < par[j]) par[j] = i;
      }
    TRY(dupload(c, &ip, par));
    n.eparent = ip;
    // full-Hessian column order: v_ref, then (v_k, p_k) of the PV buses in the
    // postorder of their theta rows, so that a tile's right-hand sides sit in
    // one subtree and the first triangular solve reaches few rows
    std::vector<int> kid_ptr(nx + 1, 0), kids(nx), post(nx, 0);
    for (int j = 0; j < nx; j++)
      if (par[j] >= 0) kid_ptr[par[j] + 1]++;
    for (int j = 0; j < nx; j++) kid_ptr[j + 1] += kid_ptr[j];
    {
      std::vector<int> fill(kid_ptr.begin(), kid_ptr.end() - 1);
      for (int j = 0; j < nx; j++)
        if (par[j] >= 0) kids[fill[par[j]]++] = j;
    }
    int cnt = 0;
    std::vector<std::pair<int, int>> stack;
    for (int r = nx - 1; r >= 0; r--) {
      if (par[r] >= 0) continue;
      stack.push_back({r, 0});
      while (!stack.empty()) {
        auto& top = stack.back();
        const int v = top.first, k = kid_ptr[v] + top.second;
        if (k < kid_ptr[v + 1]) {
          top.second++;
          stack.push_back({kids[k], 0});
        } else {
          post[v] = cnt++;
          stack.pop_back();
        }
      }
    }
    std::vector<int> pvb;
    for (int i = 0; i < nb; i++)
      if (h.type[i] == opf::PV) pvb.push_back(i);
    std::stable_sort(pvb.begin(), pvb.end(), [&](int a, int b) { return post[pth[a]] < post[pth[b]]; });
    std::vector<int> perm_cols;
    perm_cols.push_back(h.uv[h.ref]);
    for (int b : pvb) {
      perm_cols.push_back(h.uv[b]);
      perm_cols.push_back(h.up[b]);
    }
    // rows of the right-hand side -G_u e_j of each control (as the tile kernel scatters them)
    auto rhs_rows = [&](int j, std::vector<int>& out) {
      const int k = ubus[j];
      if (j >= 1 + h.npv) {
        out.push_back(pth[k]);
        return;
      }
      for (int q = h.adj_ptr[k]; q < h.adj_ptr[k + 1]; q++) {
        const int e = h.adj[q], l = e >> 1, o = (e & 1) ? h.f[l] : h.t[l];
        if (h.type[o] != opf::REF) out.push_back(pth[o]);
        if (h.type[o] == opf::PQ) out.push_back(pvv[o]);
      }
      if (h.type[k] == opf::PV) out.push_back(pth[k]);
    };
    // symmetric full Hessian: the position of each control in this order; per
    // pivot row the last position whose right-hand side reaches it (controls
    // taken from the last, so the first mark of a row is its largest; a walk
    // stops at a marked row, whose ancestors carry larger marks already); the
    // L^T sweep's backward levels with each level's blocks by descending mark
    // (stable: equal marks keep the longest-first order)
    std::vector<int> lt_mark;         // block marks, descending
    std::vector<long long> lt_ent;    // L^T entries of the blocks with the first k marks
    {
      std::vector<int> qpos(h.nu, 0), qrow(nx, -1), rr;
      for (int q = 0; q < h.nu; q++) qpos[perm_cols[q]] = q;
      for (int q = h.nu - 1; q >= 0; q--) {
        rr.clear();
        rhs_rows(perm_cols[q], rr);
        for (int r : rr)
          for (int x = r; x >= 0 && qrow[x] < 0; x = par[x]) qrow[x] = q;
      }
      std::vector<int4> meta_lt(bmeta_b.size());
      std::vector<int> q_lt(bmeta_b.size());
      std::vector<std::pair<int, int>> ord;
      for (size_t l = 0; l + 1 < bsched_ptr_b.size(); l++) {
        ord.clear();
        for (int k = bsched_ptr_b[l]; k < bsched_ptr_b[l + 1]; k++) {
          const int4 m = bmeta_b[k];
          ord.push_back({m.w != 0 ? std::max(qrow[m.x], qrow[m.x - 1]) : qrow[m.x], k});
        }
        std::stable_sort(ord.begin(), ord.end(),
                         [](const std::pair<int, int>& a, const std::pair<int, int>& b) { return a.first > b.first; });
        for (size_t i = 0; i < ord.size(); i++) {
          meta_lt[bsched_ptr_b[l] + i] = bmeta_b[ord[i].second];
          q_lt[bsched_ptr_b[l] + i] = ord[i].first;
        }
      }
      std::vector<std::pair<int, long long>> me;
      for (const int4& m : bmeta_b) {
        const int q = m.w != 0 ? std::max(qrow[m.x], qrow[m.x - 1]) : qrow[m.x];
        me.push_back({q, (long long)(m.z - m.y) * (m.w != 0 ? 2 : 1)});
      }
      std::sort(me.begin(), me.end(),
                [](const std::pair<int, long long>& a, const std::pair<int, long long>& b) { return a.first > b.first; });
      lt_ent.assign(1, 0);
      for (auto& e : me) {
        lt_mark.push_back(e.first);
        lt_ent.push_back(lt_ent.back() + e.second);
      }
      int4* q4p = nullptr;
      TRY(dupload(c, &q4p, meta_lt));
      n.bmeta_lt = q4p;
      TRY(dupload(c, &ip, q_lt));
      n.lt_q = ip;
      TRY(dupload(c, &ip, qpos));
      n.qpos = ip;
      TRY(dalloc(c, &c->tstart, h.nu));
    }
    // per block width: near-equal chunks of the order (as many tiles as a whole
    // number of waves over the SMs when that keeps tiles at least half full),
    // heaviest first by the reach of their first solve
    std::vector<int> stamp(nx, -1), rows;
    int stamp_id = 0;
    for (int lk = 0; lk < 6; lk++)
      for (int form = 0; form < 2; form++) {
        const int C = 1 << lk, nu = h.nu, T0 = (nu + C - 1) / C;
        int T = T0;
        if (form == 1 && T0 >= c->sm_count) {
          const int Tr = (T0 + c->sm_count - 1) / c->sm_count * c->sm_count;
          if (2 * nu >= Tr * C) T = Tr;
        }
        if (form == 1 && T == T0) {  // same tiling as the ceil form
          c->colmap[1][lk] = c->colmap[0][lk];
          c->coltiles[1][lk] = T0;
          continue;
        }
        std::vector<int> start(T + 1, 0);
        for (int t = 0; t < T; t++) start[t + 1] = start[t] + (form ? nu / T + (t < nu % T ? 1 : 0) : C);
        start[T] = nu;
        std::vector<std::pair<int, int>> cost(T);
        for (int t = 0; t < T; t++) {
          int reach = 0;
          rows.clear();
          for (int q = start[t]; q < start[t + 1]; q++) rhs_rows(perm_cols[q], rows);
          stamp_id++;
          for (int r : rows)
            for (int x = r; x >= 0 && stamp[x] != stamp_id; x = par[x]) {
              stamp[x] = stamp_id;
              reach++;
            }
          cost[t] = {-reach, t};
        }
        std::stable_sort(cost.begin(), cost.end());
        std::vector<int> map((size_t)T * C, -1);
        for (int t = 0; t < T; t++) {
          const int src = cost[t].second;
          for (int q = start[src]; q < start[src + 1]; q++) map[(size_t)t * C + (q - start[src])] = perm_cols[q];
        }
        TRY(dupload(c, &c->colmap[form][lk], map));
        c->coltiles[form][lk] = T;
      }
    // split tilings: k waves of full-width tiles, then at most one half-width
    // tile per SM for the remaining columns (every SM carries about the same
    // number of columns, with no idle lanes in the full-width tiles)
    for (int lk = 1; lk < 6; lk++) {
      const int C = 1 << lk, nu = h.nu, S = c->sm_count;
      const int waves = nu / (C * S);
      const int n1 = waves * S, rem = nu - n1 * C, n2 = (rem + C / 2 - 1) / (C / 2);
      if (waves < 1 || rem <= 0 || n2 > S) continue;
      // chunks of width w from q0, heaviest first by the work that varies between
      // tiles: the first solve's reach (rows x the mean entries of a row of L)
      // and the L^T entries a symmetric tile sweeps (the blocks marked at or
      // after its first position)
      const double row_ent = (double)(nnz - nx) / (2.0 * nx);
      auto order = [&](int q0, int w, int T) {
        std::vector<std::pair<double, int>> cost(T);
        for (int t = 0; t < T; t++) {
          int reach = 0;
          rows.clear();
          for (int q = q0 + t * w; q < std::min(nu, q0 + (t + 1) * w); q++) rhs_rows(perm_cols[q], rows);
          stamp_id++;
          for (int r : rows)
            for (int x = r; x >= 0 && stamp[x] != stamp_id; x = par[x]) {
              stamp[x] = stamp_id;
              reach++;
            }
          const int p = q0 + t * w;
          const size_t kept = std::upper_bound(lt_mark.begin(), lt_mark.end(), p, std::greater<int>()) -
                              lt_mark.begin();
          cost[t] = {-(reach * row_ent + (double)lt_ent[kept]), t};
        }
        std::stable_sort(cost.begin(), cost.end());
        std::vector<int> m((size_t)T * w, -1);
        for (int t = 0; t < T; t++) {
          const int src = cost[t].second;
          for (int q = q0 + src * w; q < std::min(nu, q0 + (src + 1) * w); q++)
            m[(size_t)t * w + (q - q0 - src * w)] = perm_cols[q];
        }
        return m;
      };
      std::vector<int> map = order(0, C, n1), m2 = order(n1 * C, C / 2, n2);
      map.insert(map.end(), m2.begin(), m2.end());
      TRY(dupload(c, &c->colmap_split[lk], map));
      c->split_n1[lk] = n1;
      c->split_n2[lk] = n2;
    }
  }
  TRY(dupload(c, &c->pd_nom, h.pd));
  TRY(dupload(c, &c->qd_nom, h.qd));
  TRY(dupload(c, &c->split_ctr, std::vector<int>(4 + kSplitMaxSm, 0)));
  // workspaces
  TRY(dalloc(c, &c->LU, nnz));
  TRY(dalloc(c, &c->T, nnz));
  TRY(dalloc(c, &c->invdiag, nx));
  TRY(dalloc(c, &c->x, nx));
  TRY(dalloc(c, &c->u, h.nu));
  TRY(dalloc(c, &c->pd, nb));
  TRY(dalloc(c, &c->qd, nb));
  TRY(dalloc(c, &c->vbus, nb));
  TRY(dalloc(c, &c->thbus, nb));
  TRY(dalloc(c, &c->g, nx));
  TRY(dalloc(c, &c->dvec, nx));
  TRY(dalloc(c, &c->yvec, nx));
  TRY(dalloc(c, &c->scal, 8));
  TRY(dalloc(c, &c->flags, 4));
  CK(cudaMemset(c->flags, 0, 4 * sizeof(int)));  // no error, default wait limits
  TRY(dalloc(c, &c->flows, 4 * (size_t)nl));
  TRY(dalloc(c, &c->Pbus, nb));
  TRY(dalloc(c, &c->Qbus, nb));
  TRY(dalloc(c, &c->cvec, h.m));
  TRY(dalloc(c, &c->phid, h.m));
  TRY(dalloc(c, &c->omega, h.m));
  TRY(dalloc(c, &c->dFx, nx));
  TRY(dalloc(c, &c->dFu, h.nu));
  TRY(dalloc(c, &c->lam, nx));
  TRY(dalloc(c, &c->dFx_w, nx));
  TRY(dalloc(c, &c->dFu_w, h.nu));
  TRY(dalloc(c, &c->lam_w, nx));
  TRY(dalloc(c, &c->btab, TAB_ROWS * (size_t)nl));
  TRY(dalloc(c, &c->busw, 8 * (size_t)nb));
  TRY(dalloc(c, &c->adjE, ADJ_W * 2 * (size_t)nl));
  TRY(dalloc(c, &c->busS, 4 * (size_t)nb));
  TRY(dalloc(c, &c->endflow, 20 * (size_t)nl));
  CK(cudaMallocHost(&c->h_scal, 8 * sizeof(double)));
  CK(cudaMallocHost(&c->h_flags, 4 * sizeof(int)));
  for (int k = 0; k < 4; k++) CK(cudaEventCreate(&c->ev[k]));
  TRY(setup_solve1(c));
  TRY(setup_sweep_streams(c, bsched_ptr_f, bmeta_f, bsched_ptr_b, bmeta_b));
  c->lu_dense_cluster = setup_lu_dense_cluster(c->dn.nroot);
  {
    // the trailing levels that the cluster's warps take in one pass each run
    // inside the cluster's launch (one cluster barrier per level)
    const int nlev = (int)c->h_task_ptr.size() - 1;
    std::vector<int4> lvrec(nlev + 1);
    for (int lv = 0; lv <= nlev; lv++) {
      lvrec[lv].x = lv < nlev ? c->h_task_ptr[lv] : 0;
      lvrec[lv].y = lv < nlev ? c->h_task_ptr[lv + 1] : 0;
      lvrec[lv].z = lv > 0 ? c->h_fin_ptr[lv - 1] : 0;
      lvrec[lv].w = lv > 0 ? c->h_fin_ptr[lv] : 0;
    }
    c->lu_tail_from = nlev + 1;
    if (c->lu_dense_cluster > 0) {
      const long warps = (long)c->lu_dense_cluster * kLuClusterThreads / 32;
      for (int lv = nlev; lv >= 0; lv--) {
        const long items = (lvrec[lv].y - lvrec[lv].x) + (lvrec[lv].w - lvrec[lv].z);
        const long per_warp = 32 / std::max(1, c->h_lu_lanes[lv]);
        if (items > warps * per_warp) break;
        c->lu_tail_from = lv;
      }
    }
    TRY(dupload(c, &c->lu_lvrec, lvrec));
    TRY(dupload(c, &c->lu_lanes, c->h_lu_lanes));
  }
  setup_hvp_smem();
  // the numeric refactorisation as one CUDA graph (captured once on a private stream)
  CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  {
    cudaStream_t user = c->stream;
    const long long l0 = c->launches;
    c->stream = c->cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      launch_lu_kernels(c);
      e = cudaStreamEndCapture(c->cap_stream, &graph);
    }
    c->stream = user;
    c->lu_graph_kernels = c->launches - l0;
    c->launches = l0;
    CK(e);
    e = cudaGraphInstantiate(&c->lu_exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
  }
  return OPF_OK;
}

static void free_impl(opf_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  if (c->scratch) cudaFree(c->scratch);
  if (c->stamps) cudaFree(c->stamps);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  for (int k = 0; k < 4; k++)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  free_step_work(c);
  if (c->batch_buf) cudaFree(c->batch_buf);
  if (c->lu_exec) cudaGraphExecDestroy(c->lu_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->worker) cudaStreamDestroy(c->worker);
  for (cudaEvent_t e : c->worker_ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

static void export_sym(const Symbolic& s, int* bus_order, int* perm, int* rowptr, int* colidx,
                       int* lev_f, int* lev_b) {
  if (bus_order) std::memcpy(bus_order, s.bus_order.data(), s.bus_order.size() * sizeof(int));
  if (perm) std::memcpy(perm, s.perm.data(), s.perm.size() * sizeof(int));
  if (rowptr) std::memcpy(rowptr, s.rp.data(), s.rp.size() * sizeof(int));
  if (colidx) std::memcpy(colidx, s.ci.data(), s.ci.size() * sizeof(int));
  if (lev_f) std::memcpy(lev_f, s.lev_f.data(), s.lev_f.size() * sizeof(int));
  if (lev_b) std::memcpy(lev_b, s.lev_b.data(), s.lev_b.size() * sizeof(int));
}

extern "C" {

opf_status opf_load_network(const opf_network_desc* desc, void* stream, opf_ctx** out) {
  if (!out) FAIL(OPF_EINVAL, "out is NULL");
  *out = nullptr;
  opf_ctx* c = new (std::nothrow) opf_ctx();
  if (!c) FAIL(OPF_ENOMEM, "host allocation failed");
  for (int k = 0; k < 4; k++) c->ev[k] = nullptr;
  c->stream = static_cast<cudaStream_t>(stream);
  opf_status st = load_impl(c, desc);
  if (st != OPF_OK) {
    std::string keep = g_err;
    free_impl(c);
    g_err = keep;
    return st;
  }
  *out = c;
  return OPF_OK;
}

void opf_free(opf_ctx* ctx) { free_impl(ctx); }

opf_status opf_set_stream(opf_ctx* c, void* stream) {
  if (!c) FAIL(OPF_EINVAL, "ctx is NULL");
  c->stream = static_cast<cudaStream_t>(stream);
  return OPF_OK;
}

opf_status opf_dims(const opf_ctx* c, int* nx, int* nu, int* m, int* npv, int* npq) {
  if (!c) FAIL(OPF_EINVAL, "ctx is NULL");
  if (nx) *nx = c->h.nx;
  if (nu) *nu = c->h.nu;
  if (m) *m = c->h.m;
  if (npv) *npv = c->h.npv;
  if (npq) *npq = c->h.npq;
  return OPF_OK;
}

opf_status opf_symbolic_sizes(const opf_ctx* c, int* nnz, int* nsb, int* nlf, int* nlb) {
  if (!c) FAIL(OPF_EINVAL, "ctx is NULL");
  if (nnz) *nnz = (int)c->s.ci.size();
  if (nsb) *nsb = (int)c->s.bus_order.size();
  if (nlf) *nlf = c->s.nlev_f;
  if (nlb) *nlb = c->s.nlev_b;
  return OPF_OK;
}

opf_status opf_symbolic_export(const opf_ctx* c, int* bus_order, int* perm, int* rowptr,
                               int* colidx, int* lev_f, int* lev_b) {
  if (!c) FAIL(OPF_EINVAL, "ctx is NULL");
  export_sym(c->s, bus_order, perm, rowptr, colidx, lev_f, lev_b);
  return OPF_OK;
}

}  // extern "C"

struct opf_symbolic {
  HostNet h;
  Symbolic s;
};

// Factorise the Jacobian of the converged state if opf_powerflow left it
// unfactorised (it does, so that a power flow whose factors nobody uses, such
// as a trial point followed by another power flow, skips the refactorisation).
opf_status opf::ensure_factors(opf_ctx* c) {
  if (!c->factors_stale) return OPF_OK;
  cudaStream_t st = c->stream;
  CK(cudaMemsetAsync(c->flags, 0, 2 * sizeof(int), st));
  launch_lu(c);
  CK(cudaMemcpyAsync(c->h_flags, c->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  c->factors_stale = false;
  if (c->h_flags[1]) {
    c->have_state = false;
    FAIL(OPF_ETIMEOUT, "a bounded wait of the LU refactorisation gave up");
  }
  if (c->h_flags[0]) {
    c->have_state = false;
    FAIL(OPF_ESINGULAR, "singular Jacobian at the power-flow solution");
  }
  return OPF_OK;
}

opf_status opf::check_al(const opf_ctx* c, const opf_al_params* p) {
  (void)c;
  if (!p || !p->sigma_c || !p->y || !p->s) FAIL(OPF_EINVAL, "AL parameters need sigma_c, y and s");
  if (!(p->rho >= 0.0) || !std::isfinite(p->sigma_f)) FAIL(OPF_EINVAL, "rho must be >= 0, sigma_f finite");
  return OPF_OK;
}

extern "C" {

opf_status opf_symbolic_analyze(const opf_network_desc* desc, opf_symbolic** out) {
  if (!out) FAIL(OPF_EINVAL, "out is NULL");
  *out = nullptr;
  opf_symbolic* sy = new (std::nothrow) opf_symbolic();
  if (!sy) FAIL(OPF_ENOMEM, "host allocation failed");
  std::string why = build_hostnet(desc, sy->h);
  if (!why.empty()) {
    delete sy;
    FAIL(OPF_EINVAL, why);
  }
  build_symbolic(sy->h, sy->s);
  *out = sy;
  return OPF_OK;
}

opf_status opf_symbolic_info(const opf_symbolic* sy, int* nx, int* nnz, int* nsb, int* nlf, int* nlb) {
  if (!sy) FAIL(OPF_EINVAL, "symbolic handle is NULL");
  if (nx) *nx = sy->h.nx;
  if (nnz) *nnz = (int)sy->s.ci.size();
  if (nsb) *nsb = (int)sy->s.bus_order.size();
  if (nlf) *nlf = sy->s.nlev_f;
  if (nlb) *nlb = sy->s.nlev_b;
  return OPF_OK;
}

opf_status opf_symbolic_get(const opf_symbolic* sy, int* bus_order, int* perm, int* rowptr,
                            int* colidx, int* lev_f, int* lev_b) {
  if (!sy) FAIL(OPF_EINVAL, "symbolic handle is NULL");
  export_sym(sy->s, bus_order, perm, rowptr, colidx, lev_f, lev_b);
  return OPF_OK;
}

void opf_symbolic_free(opf_symbolic* sy) { delete sy; }

opf_status opf_powerflow(opf_ctx* c, const double* u, const double* pd, const double* qd,
                         double* x_inout, const opf_pf_opts* opts, opf_pf_info* info) {
  if (!c || !u || !x_inout) FAIL(OPF_EINVAL, "ctx, u and x_inout are required");
  const double tol = opts ? opts->tol : 1e-10;
  const int max_it = opts ? opts->max_it : 20;
  if (!(tol > 0.0) || max_it < 0) FAIL(OPF_EINVAL, "tol must be > 0 and max_it >= 0");
  const int nx = c->h.nx, nb = c->h.nb;
  cudaStream_t st = c->stream;
  c->have_state = false;
  CK(cudaMemcpyAsync(c->u, u, c->h.nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(c->pd, pd ? pd : c->pd_nom, nb * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(c->qd, qd ? qd : c->qd_nom, nb * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(c->x, x_inout, nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
  opf_status result = OPF_ENOCONV;
  int it = 0;
  double res2 = NAN, resinf = NAN;
  c->factors_stale = false;
  CK(cudaMemsetAsync(c->flags, 0, 2 * sizeof(int), st));
  for (it = 0;; it++) {
    launch_unpack(c, c->x, c->u);
    CK(cudaMemsetAsync(c->LU, 0, c->dn.nnz * sizeof(double), st));
    CK(cudaMemsetAsync(c->scal, 0, 2 * sizeof(double), st));
    launch_pf_eval(c);
    CK(cudaMemcpyAsync(c->h_scal, c->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(c->h_flags, c->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    res2 = std::sqrt(c->h_scal[0]);
    resinf = c->h_scal[1];
    if (c->h_flags[1]) {  // the previous iteration's refactorisation
      result = OPF_ETIMEOUT;
      g_err = "a bounded wait of the LU refactorisation gave up";
      break;
    }
    if (c->h_flags[0]) {  // the previous iteration's refactorisation
      result = OPF_ESINGULAR;
      g_err = "zero or non-finite pivot in the LU refactorisation";
      break;
    }
    if (!std::isfinite(res2)) {
      result = OPF_ENOCONV;
      g_err = "non-finite power-flow residual";
      break;
    }
    if (res2 < tol) {
      // the Jacobian at the solution is in LU, factorised on first use
      result = OPF_OK;
      c->factors_stale = true;
      break;
    }
    if (it >= max_it) {
      result = OPF_ENOCONV;
      g_err = "Newton-Raphson reached max_it";
      break;
    }
    launch_lu(c);
    launch_solve1(c, c->g, c->dvec, false, 1.0);
    launch_axpy(c, c->x, c->dvec, -1.0, nx);
  }
  CK(cudaMemcpyAsync(x_inout, c->x, nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  if (info) {
    info->iterations = it;
    info->res2 = res2;
    info->resinf = resinf;
  }
  c->have_state = (result == OPF_OK);
  return result;
}

opf_status opf_reduced_gradient(opf_ctx* c, const opf_al_params* p, double* F, double* grad_u,
                                double* grad_s, double* cout, double* lambda, double* grad_pd,
                                double* grad_qd) {
  if (!c) FAIL(OPF_EINVAL, "ctx is NULL");
  if (!c->have_state) FAIL(OPF_ESTATE, "no converged power flow on this context");
  TRY(ensure_factors(c));
  TRY(check_al(c, p));
  cudaStream_t st = c->stream;
  launch_first_order(c, p, grad_s);
  if (F) CK(cudaMemcpyAsync(F, c->scal + 2, sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (grad_u) launch_grad_u(c, grad_u);
  if (cout) CK(cudaMemcpyAsync(cout, c->cvec, c->h.m * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (lambda) CK(cudaMemcpyAsync(lambda, c->lam, c->h.nx * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (grad_pd || grad_qd) launch_grad_load(c, p->sigma_f, grad_pd, grad_qd);
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  return OPF_OK;
}

static opf_status ensure_scratch(opf_ctx* c, size_t doubles) {
  if (c->scratch_bytes >= doubles * sizeof(double)) return OPF_OK;
  c->z_gen = -1;
  CK(cudaStreamSynchronize(c->stream));
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  if (cudaMalloc(&c->scratch, doubles * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->scratch = nullptr;
    FAIL(OPF_ENOMEM, "cannot allocate the Hessian workspace");
  }
  c->scratch_bytes = doubles * sizeof(double);
  return OPF_OK;
}

}  // extern "C"

// Zero multipliers, slacks and scalings [m] (first use): the AL inputs of the
// evaluations that need the branch tables but no multiplier (J alone, the
// generation cost's gradient).
opf_status opf::zero_params(opf_ctx* c, opf_al_params* q) {
  if (!c->zeros_m) {
    TRY(dalloc(c, &c->zeros_m, (size_t)std::max(c->h.m, 1)));
    CK(cudaMemsetAsync(c->zeros_m, 0, sizeof(double) * std::max(c->h.m, 1), c->stream));
  }
  *q = opf_al_params{0.0, 0.0, c->zeros_m, c->zeros_m, c->zeros_m, nullptr};
  return OPF_OK;
}

// The tiled Hessian and, with J, the reduced constraint Jacobian of the same
// columns (jac_only: J alone, the tiles stop after the first adjoint).
static opf_status hessian_impl(opf_ctx* c, const opf_al_params* p, const opf_hess_opts* o, double* H, double* J,
                               bool jac_only, opf_hess_info* info) {
  if (!c->have_state) FAIL(OPF_ESTATE, "no converged power flow on this context");
  TRY(ensure_factors(c));
  opf_al_params p0;
  if (!p && jac_only) {
    if (o && o->reuse_first_order) FAIL(OPF_EINVAL, "reuse_first_order needs the parameters");
    TRY(zero_params(c, &p0));
    p = &p0;
  }
  TRY(check_al(c, p));
  if (J && o && o->plain) FAIL(OPF_EINVAL, "the plain form does not compute J");
  const bool tuned = !(o && o->block_k) && c->tuned_k > 0;
  int C = (o && o->block_k) ? o->block_k : (tuned ? c->tuned_k : 8);
  if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16 && C != 32)
    FAIL(OPF_EINVAL, "block_k must be 1, 2, 4, 8, 16 or 32");
  const int nt = (o && o->threads) ? o->threads : (tuned ? c->tuned_threads : 256);
  if (nt != 128 && nt != 256 && nt != 512) FAIL(OPF_EINVAL, "threads must be 128, 256 or 512");
  c->hvp_threads = nt;
  const bool plain = o && o->plain;
  if (plain) C = 1;  // one direction per launch sequence
  const int nu = c->h.nu;
  const int col0 = o ? o->col_begin : 0;
  const int ncol = (o && o->col_count > 0) ? o->col_count : nu - col0;
  if (col0 < 0 || col0 >= nu || ncol < 1 || col0 + ncol > nu) FAIL(OPF_EINVAL, "column range outside [0, n_u)");
  int lk = 0;
  while ((1 << lk) < C) lk++;
  // the full Hessian at the default launch shape runs the split tiling when
  // the context has one for this width
  const bool split = !plain && !(o && o->grid > 0) && col0 == 0 && ncol == nu && nt == 256 &&
                     c->split_n1[lk] > 0;
  const int ntiles = plain ? ncol
                           : (split ? c->split_n1[lk] + c->split_n2[lk] : hvp_tiles(c, C, col0, col0 + ncol, true));
  int grid = plain ? 1 : ((o && o->grid > 0) ? o->grid : std::min(ntiles, hvp_occupancy(C, nt) * c->sm_count));
  grid = std::max(1, std::min(grid, ntiles));
  if (split) grid = ntiles;
  TRY(ensure_scratch(c, plain ? hvp_plain_scratch(c)
                              : (split ? hvp_split_scratch(c, C) : hvp_stride(c, C) * (size_t)grid)));
  cudaStream_t st = c->stream;
  const bool prof = info && o && o->phase_profile && !plain;
  if (prof) {
    if (c->stamps_cap < (size_t)ntiles) {
      CK(cudaStreamSynchronize(st));
      if (c->stamps) cudaFree(c->stamps);
      c->stamps = nullptr;
      c->stamps_cap = 0;
      if (cudaMalloc(&c->stamps, sizeof(unsigned long long) * 8 * (size_t)ntiles) != cudaSuccess) {
        cudaGetLastError();
        FAIL(OPF_ENOMEM, "cannot allocate the phase stamps");
      }
      c->stamps_cap = ntiles;
    }
    CK(cudaMemsetAsync(c->stamps, 0, sizeof(unsigned long long) * 8 * (size_t)ntiles, st));
    c->stamps_on = true;
  }
  CK(cudaEventRecord(c->ev[0], st));
  if (!(o && o->reuse_first_order)) {
    if (c->fo_reuse)
      launch_omega(c, p);
    else
      launch_first_order(c, p, nullptr);
  }
  launch_hess_prep(c, p->sigma_f);
  CK(cudaEventRecord(c->ev[1], st));
  int launches = 0;
  c->jac_out = J;
  c->jac_only = jac_only;
  const bool asym = info && o && o->asymmetry && col0 == 0 && ncol == nu && !jac_only;
  // the full Hessian by its symmetry: each tile keeps the rows at or after its
  // first column position, the mirror kernel completes H
  const bool sym = c->hess_sym && !plain && col0 == 0 && ncol == nu && !asym && !jac_only;
  c->sym_now = sym;
  if (plain) {
    c->z_gen = -1;
    launches = launch_hvp_plain(c, H, col0, col0 + ncol, c->scratch);
  } else if (split) {
    launch_hvp_split(c, C, H);
    launches = 1;
  } else {
    launch_hvp(c, C, H, grid, 0, 1, ntiles, col0, col0 + ncol);
    launches = 1;
  }
  if (sym) {
    launch_hess_mirror(c, H, nu);
    launches++;
  }
  c->sym_now = false;
  CK(cudaEventRecord(c->ev[2], st));
  c->stamps_on = false;
  c->jac_out = nullptr;
  c->jac_only = false;
  std::vector<unsigned long long> stamps;
  if (prof) {
    stamps.resize(8 * (size_t)ntiles);
    CK(cudaMemcpyAsync(stamps.data(), c->stamps, sizeof(unsigned long long) * stamps.size(),
                       cudaMemcpyDeviceToHost, st));
  }
  if (asym) {  // after the timed region
    CK(cudaMemsetAsync(c->scal + 4, 0, 2 * sizeof(double), st));
    launch_hess_asymmetry(c, H, nu, c->scal + 4);
    CK(cudaMemcpyAsync(c->h_scal + 4, c->scal + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  if (info) {
    info->block_k = C;
    info->grid = grid;
    info->tiles = ntiles;
    info->launches = launches;
    cudaEventElapsedTime(&info->ms_total, c->ev[0], c->ev[2]);
    cudaEventElapsedTime(&info->ms_hvp, c->ev[1], c->ev[2]);
    info->asymmetry = -1.0;
    if (asym)
      info->asymmetry = c->h_scal[5] > 0.0 ? std::sqrt(c->h_scal[4] / c->h_scal[5]) : 0.0;
    for (int k = 0; k < 5; k++) info->phase_ms[k] = 0.f;
    if (prof) {  // the HVP time apportioned to the phases by their share of the tiles' summed time
      double part[5] = {0, 0, 0, 0, 0}, tot = 0.0;
      for (int t = 0; t < ntiles; t++) {
        const unsigned long long* q = stamps.data() + 8 * (size_t)t;
        if (!(q[0] > 0 && q[5] >= q[0])) continue;
        for (int k = 0; k < 5; k++) part[k] += (double)(q[k + 1] - q[k]);
        tot += (double)(q[5] - q[0]);
      }
      if (tot > 0.0)
        for (int k = 0; k < 5; k++) info->phase_ms[k] = (float)(info->ms_hvp * part[k] / tot);
    }
  }
  return OPF_OK;
}

extern "C" {

opf_status opf_reduced_hessian(opf_ctx* c, const opf_al_params* p, const opf_hess_opts* o,
                               double* H, opf_hess_info* info) {
  if (!c || !H) FAIL(OPF_EINVAL, "ctx and H are required");
  return hessian_impl(c, p, o, H, nullptr, false, info);
}

opf_status opf_reduced_jacobian(opf_ctx* c, const opf_al_params* p, const opf_hess_opts* o, double* J,
                                double* H, opf_hess_info* info) {
  if (!c || !J) FAIL(OPF_EINVAL, "ctx and J are required");
  if (H && !p) FAIL(OPF_EINVAL, "the Hessian needs the AL parameters");
  return hessian_impl(c, p, o, H, J, H == nullptr, info);
}

opf_status opf_gradient_scaling(opf_ctx* c, double g_max, double s_min, const double* prior, double* J,
                                double* sigma_c, double* sigma_f) {
  if (!c || !J || !sigma_c) FAIL(OPF_EINVAL, "ctx, J and sigma_c are required");
  if (!(g_max > 0.0) || !std::isfinite(g_max) || !(s_min > 0.0 && s_min <= 1.0))
    FAIL(OPF_EINVAL, "g_max must be positive and finite, s_min in (0, 1]");
  if (!c->have_state) FAIL(OPF_ESTATE, "no converged power flow on this context");
  if (!c->gscale) TRY(dalloc(c, &c->gscale, (size_t)c->h.nu + 1));
  // the generation cost's reduced gradient: the AL functional with sigma_f = 1
  // and no multiplier or penalty term is the cost itself (Prop. 1)
  TRY(ensure_factors(c));
  opf_al_params p;
  TRY(zero_params(c, &p));
  p.sigma_f = 1.0;
  launch_first_order(c, &p, nullptr);
  launch_grad_u(c, c->gscale);
  opf_hess_opts o{};
  o.reuse_first_order = 1;
  TRY(hessian_impl(c, &p, &o, nullptr, J, true, nullptr));
  launch_grad_scaling(c, J, c->gscale, g_max, s_min, prior, sigma_c, c->gscale + c->h.nu);
  double sf = 1.0;
  CK(cudaMemcpyAsync(&sf, c->gscale + c->h.nu, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  if (sigma_f) *sigma_f = sf;
  return OPF_OK;
}

opf_status opf_hessian_autotune(opf_ctx* c, const opf_al_params* p, double* H, opf_hess_opts* best,
                                float* best_ms) {
  if (!c || !H) FAIL(OPF_EINVAL, "ctx and H are required");
  static const int cand[][2] = {{4, 128}, {4, 256}, {8, 128}, {8, 256}, {8, 512}, {16, 256}, {16, 512}, {32, 256}};
  float tbest = 0.f;
  int kb = 0, tb = 0;
  for (const auto& cd : cand) {
    opf_hess_opts o = {cd[0], 0, 0, 0, 0, cd[1], 0};
    opf_hess_info hi;
    TRY(opf_reduced_hessian(c, p, &o, H, &hi));
    TRY(opf_reduced_hessian(c, p, &o, H, &hi));
    if (kb == 0 || hi.ms_total < tbest) {
      tbest = hi.ms_total;
      kb = cd[0];
      tb = cd[1];
    }
  }
  c->tuned_k = kb;
  c->tuned_threads = tb;
  if (best) {
    *best = opf_hess_opts{kb, 0, 0, 0, 0, tb, 0};
  }
  if (best_ms) *best_ms = tbest;
  return OPF_OK;
}

opf_status opf_set_sweep_merge(opf_ctx* c, int lookahead, int narrow) {
  if (!c) FAIL(OPF_EINVAL, "ctx is required");
  return set_sweep_merge(c, lookahead, narrow);
}

opf_status opf_sweep_autotune(opf_ctx* c, int* lookahead, int* narrow, float* ms_pair, float* ms_all) {
  if (!c) FAIL(OPF_EINVAL, "ctx is required");
  if (!c->have_state) FAIL(OPF_ESTATE, "no converged power flow on this context");
  TRY(ensure_factors(c));
  if (!c->sw.ok) {  // level-record form: no schedule to choose
    if (lookahead) *lookahead = 0;
    if (narrow) *narrow = 0;
    if (ms_pair) *ms_pair = 0.f;
    if (ms_all)
      for (int k = 0; k < 8; k++) ms_all[k] = 0.f;
    return OPF_OK;
  }
  static const int cand[][2] = {{0, 0}, {1, 4}, {2, 4}, {4, 4}, {6, 4}, {8, 4}, {4, 2}, {4, 8}};
  cudaStream_t st = c->stream;
  float tbest = 0.f;
  int db = 0, wb = 0, ic = 0;
  for (const auto& cd : cand) {
    TRY(set_sweep_merge(c, cd[0], cd[1]));
    // one forward and one transposed solve per pair (the residual vector as input)
    launch_solve1(c, c->g, c->dvec, false, 1.0);
    launch_solve1(c, c->g, c->dvec, true, 1.0);
    float best = 0.f;
    for (int r = 0; r < 3; r++) {
      CK(cudaEventRecord(c->ev[0], st));
      launch_solve1(c, c->g, c->dvec, false, 1.0);
      launch_solve1(c, c->g, c->dvec, true, 1.0);
      CK(cudaEventRecord(c->ev[1], st));
      CK(cudaEventSynchronize(c->ev[1]));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
      if (r == 0 || ms < best) best = ms;
    }
    if (ms_all) ms_all[ic] = best;
    ic++;
    if (tbest == 0.f || best < tbest) {
      tbest = best;
      db = cd[0];
      wb = cd[1];
    }
  }
  TRY(set_sweep_merge(c, db, wb));
  CK(cudaGetLastError());
  if (lookahead) *lookahead = db;
  if (narrow) *narrow = wb;
  if (ms_pair) *ms_pair = tbest;
  return OPF_OK;
}

opf_status opf_reduced_hessian_batched(opf_ctx* const* ctxs, int n, const opf_al_params* params,
                                       double* const* H, const opf_hess_opts* o, opf_hess_info* info) {
  if (!ctxs || n < 1 || !params || !H) FAIL(OPF_EINVAL, "ctxs, params and H are required, n >= 1");
  opf_ctx* c0 = ctxs[0];
  if (!c0) FAIL(OPF_EINVAL, "null context");
  const int C = (o && o->block_k) ? o->block_k : 8;
  if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16 && C != 32)
    FAIL(OPF_EINVAL, "block_k must be 1, 2, 4, 8, 16 or 32");
  std::vector<int> order(n);
  size_t stride = 0;
  for (int k = 0; k < n; k++) {
    opf_ctx* c = ctxs[k];
    if (!c || !H[k]) FAIL(OPF_EINVAL, "null context or Hessian pointer in the batch");
    if (c->device != c0->device) FAIL(OPF_EINVAL, "all contexts of a batch must be on one device");
    if (!c->have_state) FAIL(OPF_ESTATE, "a context of the batch has no converged power flow");
    TRY(ensure_factors(c));
    TRY(check_al(c, &params[k]));
    stride = std::max(stride, hvp_stride(c, C));
    order[k] = k;
  }
  cudaStream_t st = c0->stream;
  CK(cudaEventRecord(c0->ev[0], st));
  // first-order quantities and branch tables per context, on the batch stream
  std::vector<HvpArgs> args(n);
  for (int k = 0; k < n; k++) {
    opf_ctx* c = ctxs[k];
    cudaStream_t keep = c->stream;
    c->stream = st;
    if (!(o && o->reuse_first_order)) launch_first_order(c, &params[k], nullptr);
    launch_hess_prep(c, params[k].sigma_f);
    c->stream = keep;
    c->sym_now = c->hess_sym;  // each Hessian by its symmetry, mirrored after the launch
    args[k] = make_hvp_args(c, C, H[k], 0, c->h.nu, false);
    c->sym_now = false;
  }
  // tile queue: contexts by decreasing factor size (longest processing time first)
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)ctxs[a]->dn.nnz * ctxs[a]->h.nu > (long long)ctxs[b]->dn.nnz * ctxs[b]->h.nu;
  });
  std::vector<int2> tiles;
  for (int k : order)
    for (int t = 0; t < args[k].ntiles; t++) tiles.push_back(make_int2(k, t));
  const int ntot = (int)tiles.size();
  const size_t bytes = n * sizeof(HvpArgs) + ntot * sizeof(int2) + 256;
  if (c0->batch_bytes < bytes) {
    CK(cudaStreamSynchronize(st));
    if (c0->batch_buf) cudaFree(c0->batch_buf);
    c0->batch_buf = nullptr;
    c0->batch_bytes = 0;
    if (cudaMalloc(&c0->batch_buf, bytes) != cudaSuccess) {
      cudaGetLastError();
      FAIL(OPF_ENOMEM, "cannot allocate the batch tables");
    }
    c0->batch_bytes = bytes;
  }
  char* base = static_cast<char*>(c0->batch_buf);
  HvpArgs* d_args = reinterpret_cast<HvpArgs*>(base);
  int2* d_tiles = reinterpret_cast<int2*>(base + n * sizeof(HvpArgs));
  int* d_counter = reinterpret_cast<int*>(base + n * sizeof(HvpArgs) + ntot * sizeof(int2));
  CK(cudaMemcpyAsync(d_args, args.data(), n * sizeof(HvpArgs), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d_tiles, tiles.data(), ntot * sizeof(int2), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d_counter, 0, sizeof(int), st));
  const int occ = std::max(1, hvp_batch_occupancy(C));
  int grid = (o && o->grid > 0) ? o->grid : occ * c0->sm_count;
  grid = std::max(1, std::min(grid, ntot));
  TRY(ensure_scratch(c0, stride * (size_t)grid));
  CK(cudaEventRecord(c0->ev[1], st));
  size_t smem = 0;
  for (int k = 0; k < n; k++) smem = std::max(smem, hvp_smem_bytes(args[k], C));
  c0->z_gen = -1;
  launch_hvp_batch(st, C, d_args, d_tiles, ntot, d_counter, c0->scratch, stride, grid, smem);
  c0->launches++;
  int launches = 1;
  for (int k = 0; k < n; k++) {
    if (!args[k].sym) continue;
    opf_ctx* c = ctxs[k];
    cudaStream_t keep = c->stream;
    c->stream = st;
    launch_hess_mirror(c, H[k], c->h.nu);
    c->stream = keep;
    launches++;
  }
  CK(cudaEventRecord(c0->ev[2], st));
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  if (info) {
    info->block_k = C;
    info->grid = grid;
    info->tiles = ntot;
    info->launches = launches;
    info->asymmetry = -1.0;
    for (int k = 0; k < 5; k++) info->phase_ms[k] = 0.f;
    cudaEventElapsedTime(&info->ms_total, c0->ev[0], c0->ev[2]);
    cudaEventElapsedTime(&info->ms_hvp, c0->ev[1], c0->ev[2]);
  }
  return OPF_OK;
}

opf_status opf_set_hessian_symmetry(opf_ctx* c, int on) {
  if (!c) FAIL(OPF_EINVAL, "ctx is required");
  c->hess_sym = on != 0;
  return OPF_OK;
}

opf_status opf_set_wait_limit(opf_ctx* c, int spins) {
  if (!c || spins < 0) FAIL(OPF_EINVAL, "ctx is NULL or spins < 0");
  CK(cudaMemcpyAsync(c->flags + 2, &spins, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->wait_limit = spins;
  return OPF_OK;
}

opf_status opf_launch_count(const opf_ctx* c, long long* launches) {
  if (!c || !launches) FAIL(OPF_EINVAL, "ctx and launches are required");
  *launches = c->launches;
  return OPF_OK;
}

const char* opf_status_str(int s) {
  switch (s) {
    case OPF_OK: return "ok";
    case OPF_EINVAL: return "invalid argument";
    case OPF_ENOMEM: return "out of memory";
    case OPF_ECUDA: return "CUDA error";
    case OPF_ENOCONV: return "Newton-Raphson did not converge";
    case OPF_ESINGULAR: return "singular Jacobian";
    case OPF_ENOTPD: return "matrix not positive definite";
    case OPF_ESTATE: return "no converged power-flow state";
    case OPF_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* opf_last_error(void) { return g_err.c_str(); }

}  // extern "C"
