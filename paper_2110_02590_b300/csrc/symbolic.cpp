// Host set-up of libopf: network validation, index maps (eq. statecontrol,
// Sec. II-B) and the symbolic analysis of G_x done once per topology (Sec. V-A,
// "Sparse linear system": the pattern of G_x is fixed by the network, so it is
// factorised symbolically once and only refactorised numerically afterwards).
//
// Pivot order: exact minimum degree on the graph of the state buses (all buses
// but the slack).  A bus weighs as many state variables as it has (1 for PV,
// 2 for PQ); its degree is the summed weight of its neighbours in the current
// elimination graph; the smallest degree is eliminated first, ties go to the
// smallest bus id.  The variables of a bus are consecutive pivots, theta
// before v.  Because both variables of a PQ bus couple to exactly the same
// buses, the filled pattern of the variable-level LU is the bus-level fill
// expanded into blocks.  No numerical pivoting: the pattern is symmetric and
// the values are not.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <queue>
#include <set>
#include <utility>

#include "opf_internal.h"

namespace opf {

std::string build_hostnet(const opf_network_desc* d, HostNet& h) {
  if (!d) return "null network description";
  if (d->n_bus < 2 || d->n_branch < 1 || d->n_gen < 1) return "need n_bus >= 2, n_branch >= 1, n_gen >= 1";
  if (d->ref_bus < 0 || d->ref_bus >= d->n_bus) return "ref_bus out of range";
  if (!d->pd || !d->qd || !d->br_from || !d->br_to || !d->br_r || !d->br_x || !d->br_b ||
      !d->br_tap || !d->gen_bus || !d->gen_c2 || !d->gen_c1)
    return "missing network array";
  h.nb = d->n_bus;
  h.nl = d->n_branch;
  h.ng = d->n_gen;
  h.ref = d->ref_bus;
  const int nb = h.nb, nl = h.nl, ng = h.ng;
  h.f.assign(d->br_from, d->br_from + nl);
  h.t.assign(d->br_to, d->br_to + nl);
  h.gbus.assign(d->gen_bus, d->gen_bus + ng);
  h.pd.assign(d->pd, d->pd + nb);
  h.qd.assign(d->qd, d->qd + nb);
  h.c2.assign(d->gen_c2, d->gen_c2 + ng);
  h.c1.assign(d->gen_c1, d->gen_c1 + ng);
  h.c0.assign(ng, 0.0);
  if (d->gen_c0) h.c0.assign(d->gen_c0, d->gen_c0 + ng);
  h.Y.assign(8 * (size_t)nl, 0.0);
  for (int l = 0; l < nl; l++) {
    if (h.f[l] < 0 || h.f[l] >= nb || h.t[l] < 0 || h.t[l] >= nb) return "branch end out of range";
    if (h.f[l] == h.t[l]) return "branch is a self-loop";
    double r = d->br_r[l], x = d->br_x[l], tau = d->br_tap[l];
    double den = r * r + x * x;
    if (!(den > 0.0)) return "branch with r = x = 0";
    if (!(tau > 0.0)) return "non-positive tap";
    // pi model: y = 1/(r + jx) = (r - jx)/|z|^2, tap on the from side
    double gs = r / den, bs = -x / den, bc = 0.5 * d->br_b[l];
    h.Y[0 * (size_t)nl + l] = gs / (tau * tau);
    h.Y[1 * (size_t)nl + l] = (bs + bc) / (tau * tau);
    h.Y[2 * (size_t)nl + l] = -gs / tau;
    h.Y[3 * (size_t)nl + l] = -bs / tau;
    h.Y[4 * (size_t)nl + l] = -gs / tau;
    h.Y[5 * (size_t)nl + l] = -bs / tau;
    h.Y[6 * (size_t)nl + l] = gs;
    h.Y[7 * (size_t)nl + l] = bs + bc;
  }
  h.gen_at.assign(nb, -1);
  h.type.assign(nb, PQ);
  for (int g = 0; g < ng; g++) {
    int b = h.gbus[g];
    if (b < 0 || b >= nb) return "generator bus out of range";
    if (h.gen_at[b] >= 0) return "two generators on one bus";
    h.gen_at[b] = g;
    h.type[b] = PV;
  }
  if (h.gen_at[h.ref] < 0) return "no generator on the reference bus";
  h.type[h.ref] = REF;
  h.pvpos.assign(nb, -1);
  h.pqpos.assign(nb, -1);
  h.npv = h.npq = 0;
  for (int i = 0; i < nb; i++) {
    if (h.type[i] == PV) h.pvpos[i] = h.npv++;
    if (h.type[i] == PQ) h.pqpos[i] = h.npq++;
  }
  h.nx = h.npv + 2 * h.npq;
  h.nu = 1 + 2 * h.npv;
  h.m = 2 * nl + h.npq + h.npv + 2;
  h.xth.assign(nb, -1);
  h.xv.assign(nb, -1);
  h.uv.assign(nb, -1);
  h.up.assign(nb, -1);
  for (int i = 0; i < nb; i++) {
    switch (h.type[i]) {
      case REF: h.uv[i] = 0; break;
      case PV:
        h.xth[i] = h.pvpos[i];
        h.uv[i] = 1 + h.pvpos[i];
        h.up[i] = 1 + h.npv + h.pvpos[i];
        break;
      default:
        h.xth[i] = h.npv + h.pqpos[i];
        h.xv[i] = h.npv + h.npq + h.pqpos[i];
    }
  }
  // incidence lists (entry = 2 * branch + side, side 0 = the bus is the from end)
  h.adj_ptr.assign(nb + 1, 0);
  for (int l = 0; l < nl; l++) {
    h.adj_ptr[h.f[l] + 1]++;
    h.adj_ptr[h.t[l] + 1]++;
  }
  for (int i = 0; i < nb; i++) h.adj_ptr[i + 1] += h.adj_ptr[i];
  h.adj.assign(2 * (size_t)nl, 0);
  std::vector<int> fill(h.adj_ptr.begin(), h.adj_ptr.end() - 1);
  for (int l = 0; l < nl; l++) {
    h.adj[fill[h.f[l]]++] = 2 * l;
    h.adj[fill[h.t[l]]++] = 2 * l + 1;
  }
  // within each bus, the ends whose other bus carries a generator come last (the
  // slack's last of all): the HVP gathers add Gauss-Newton terms for exactly those
  // ends, so buses with the same degree and the same count of such ends (which
  // the gathers take side by side) run those terms in step
  for (int b = 0; b < nb; b++) {
    auto key = [&](int e) {
      const int l = e >> 1, o = (e & 1) ? h.f[l] : h.t[l];
      return h.type[o] == PQ ? 0 : (h.type[o] == PV ? 1 : 2);
    };
    std::stable_sort(h.adj.begin() + h.adj_ptr[b], h.adj.begin() + h.adj_ptr[b + 1],
                     [&](int a, int c) { return key(a) < key(c); });
  }
  // every bus must reach the slack
  std::vector<char> seen(nb, 0);
  std::queue<int> q;
  q.push(h.ref);
  seen[h.ref] = 1;
  while (!q.empty()) {
    int b = q.front();
    q.pop();
    for (int k = h.adj_ptr[b]; k < h.adj_ptr[b + 1]; k++) {
      int l = h.adj[k] >> 1, o = (h.adj[k] & 1) ? h.f[l] : h.t[l];
      if (!seen[o]) {
        seen[o] = 1;
        q.push(o);
      }
    }
  }
  for (int i = 0; i < nb; i++)
    if (!seen[i]) return "a bus is not connected to the reference bus";
  return "";
}

void build_symbolic(const HostNet& h, Symbolic& s) {
  const int nb = h.nb, nx = h.nx;
  // bus graph of the state buses (distinct neighbours, sorted)
  std::vector<std::vector<int>> nbr(nb);
  for (int l = 0; l < h.nl; l++) {
    int a = h.f[l], b = h.t[l];
    if (a == h.ref || b == h.ref) continue;
    nbr[a].push_back(b);
    nbr[b].push_back(a);
  }
  for (auto& v : nbr) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  auto weight = [&](int b) { return h.type[b] == PQ ? 2 : 1; };
  std::vector<long long> deg(nb, 0);
  std::set<std::pair<long long, int>> queue;
  for (int b = 0; b < nb; b++) {
    if (b == h.ref) continue;
    long long d = 0;
    for (int o : nbr[b]) d += weight(o);
    deg[b] = d;
    queue.insert({d, b});
  }
  std::vector<std::vector<int>> elim_struct(nb);  // later buses adjacent at elimination
  s.bus_order.clear();
  std::vector<int> merged;
  while (!queue.empty()) {
    int p = queue.begin()->second;
    queue.erase(queue.begin());
    s.bus_order.push_back(p);
    std::vector<int> np = std::move(nbr[p]);
    nbr[p].clear();
    for (int q : np) {
      merged.clear();
      std::set_union(nbr[q].begin(), nbr[q].end(), np.begin(), np.end(), std::back_inserter(merged));
      merged.erase(std::remove_if(merged.begin(), merged.end(), [&](int z) { return z == q || z == p; }),
                   merged.end());
      nbr[q].swap(merged);
      long long d = 0;
      for (int o : nbr[q]) d += weight(o);
      queue.erase({deg[q], q});
      deg[q] = d;
      queue.insert({d, q});
    }
    elim_struct[p] = std::move(np);
  }
  // pivot order of the variables
  s.perm.clear();
  std::vector<int> first(nb, -1);
  for (int b : s.bus_order) {
    first[b] = (int)s.perm.size();
    s.perm.push_back(h.xth[b]);
    if (h.type[b] == PQ) s.perm.push_back(h.xv[b]);
  }
  s.iperm.assign(nx, -1);
  for (int k = 0; k < nx; k++) s.iperm[s.perm[k]] = k;
  // upper structure of each pivot column (= structure of column k of L)
  std::vector<std::vector<int>> upper(nx);
  for (int b : s.bus_order) {
    int w = weight(b), k0 = first[b];
    std::vector<int> below;
    for (int o : elim_struct[b])
      for (int r = 0; r < weight(o); r++) below.push_back(first[o] + r);
    std::sort(below.begin(), below.end());
    for (int c = 0; c < w; c++) {
      auto& u = upper[k0 + c];
      if (c == 0 && w == 2) u.push_back(k0 + 1);
      u.insert(u.end(), below.begin(), below.end());
    }
  }
  // lower structure = transpose; full rows = lower | diag | upper
  std::vector<int> lcount(nx, 0);
  for (int k = 0; k < nx; k++)
    for (int r : upper[k]) lcount[r]++;
  s.rp.assign(nx + 1, 0);
  for (int i = 0; i < nx; i++) s.rp[i + 1] = s.rp[i] + lcount[i] + 1 + (int)upper[i].size();
  s.ci.assign(s.rp[nx], 0);
  s.dp.assign(nx, 0);
  std::vector<int> pos(nx);
  for (int i = 0; i < nx; i++) pos[i] = s.rp[i];
  for (int k = 0; k < nx; k++)  // k ascending: lower parts come out sorted
    for (int r : upper[k]) s.ci[pos[r]++] = k;
  for (int i = 0; i < nx; i++) {
    s.dp[i] = pos[i];
    s.ci[pos[i]++] = i;
    for (int c : upper[i]) s.ci[pos[i]++] = c;
  }
  // level sets
  s.lev_f.assign(nx, 0);
  s.lev_b.assign(nx, 0);
  s.nlev_f = s.nlev_b = 0;
  for (int i = 0; i < nx; i++) {
    int lv = 0;
    for (int p = s.rp[i]; p < s.dp[i]; p++) lv = std::max(lv, s.lev_f[s.ci[p]] + 1);
    s.lev_f[i] = lv;
    s.nlev_f = std::max(s.nlev_f, lv + 1);
  }
  for (int i = nx - 1; i >= 0; i--) {
    int lv = 0;
    for (int p = s.dp[i] + 1; p < s.rp[i + 1]; p++) lv = std::max(lv, s.lev_b[s.ci[p]] + 1);
    s.lev_b[i] = lv;
    s.nlev_b = std::max(s.nlev_b, lv + 1);
  }
}

}  // namespace opf
