// Single-right-hand-side sweeps with the factor entries streamed through a
// shared-memory ring (the Newton updates of the power flow, Sec. III-A, and the
// adjoint solves of Prop. 1 and of the reduced-Newton step, Prop. 3).
//
// The level loop of a sweep is a chain of dependent steps: a level's rows can
// start only when the previous level's solution entries are written.  The
// factor entries themselves do not depend on the solution, so after each
// refactorisation they are gathered into one contiguous stream per (factor,
// direction), ordered level by level and cut into chunks at block boundaries.
// One 512-thread CTA holds the whole solution vector in shared memory and
// copies chunk c + 2 into a three-slot ring (cp.async, 16-byte pieces) while it
// computes chunk c, so the level chain reads shared memory only; between the
// two sweeps the dense trailing triangles pass through the ring.

#include <algorithm>
#include <cstring>
#include <vector>

#include "opf_internal.h"

namespace opf {
namespace {

constexpr int kSweepThreads = 512;
constexpr int kRing = 3;
constexpr int kHdr = 32;

inline int pad4(int e) { return (e + 3) & ~3; }
inline int rv_count(int nrec) { return (3 * nrec + 1) & ~1; }
constexpr int kMaxTasks = 2 * kSweepThreads / 32;  // warp tasks of a chunk (two passes of the CTA's warps)
inline size_t chunk_bytes(int nrec, int ent, int ntask) {
  return kHdr + 128 * (size_t)ntask + 16 * (size_t)nrec + 8 * (size_t)rv_count(nrec) + 20 * (size_t)pad4(ent);
}

// One block of a level in factor positions.
struct Rec {
  int lead, other;  // rows (other = -1: a single row)
  int q0, q1;       // the lead row's entries [q0, q1) (when pos is empty)
  int off;          // the second row's entry of position p is p + off
  int coup;         // position of the coupling entry (other >= 0; -1 with other >= 0: none, a partial sum)
  bool scale;       // multiply by 1 / U_rr of the rows (the sweep's diagonal)
  std::vector<int> pos;  // explicit entry positions of the lead row (replaces [q0, q1))
  int count() const { return pos.empty() ? q1 - q0 : (int)pos.size(); }
  int at(int t) const { return pos.empty() ? q0 + t : pos[t]; }
};

struct Built {
  std::vector<unsigned char> bytes;
  int tri_len = 0;            // bytes of the triangle segment at the start
  std::vector<int> off, len;  // chunks
  std::vector<int2> map;      // destination doubles relative to the stream start
};

// Lanes of a chunk.  Record r gets g_r lanes, the power of two that gives
// each lane at most k of its entries (at most 32); the groups are packed into
// warp tasks of 32 lanes in order, each at a multiple of its size.  The SM's FP64 unit takes one warp
// instruction per ~20 cycles whatever the number of active lanes, and one warp
// issues at most one per ~67 cycles, so the model counts warp FP64
// instructions: per task the most entries of a lane (twice when the task has a
// two-row block), one shuffle-add round per doubling of its largest group and
// the finishing operations, plus the latencies of a task's chain: ~60 cycles
// of shared-memory reads per pass of the entry loop, ~110 per shuffle round,
// ~300 to finish; task t runs on warp t mod 16.  k minimises the larger of
// the SM's FP64 time and the busiest warp's time.  Returns the lane map: per
// task and lane, record | lane in the group << 16 | log2 of the group << 21,
// or -1.
std::vector<int> plan_lanes(const std::vector<Rec>& L, size_t i, int nrec) {
  static const int ks[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 48, 64, 96, 128, 256};
  std::vector<int> best_map;
  long best = -1;
  for (int k : ks) {
    std::vector<int> map;
    std::vector<long> ins;
    int used = 32;  // lanes used in the current task
    int mx = 0, lgmax = 0;
    bool two = false;
    std::vector<long> lat;
    auto close = [&]() {
      if (map.empty()) return;
      ins.push_back((long)(two ? 2 : 1) * mx + lgmax + 3);
      lat.push_back(60L * (mx / 4 + mx % 4 + 1) + 110L * lgmax + 300);
    };
    for (int r = 0; r < nrec; r++) {
      const int len = L[i + r].count();
      int lg = 0;
      while (lg < 5 && (1 << lg) * k < len) lg++;
      const int g = 1 << lg;
      used = (used + g - 1) / g * g;  // a group sits at a multiple of its size (the shuffle reduction)
      if (used + g > 32) {
        close();
        map.resize(map.size() + 32, -1);
        used = 0;
        mx = 0;
        lgmax = 0;
        two = false;
      }
      for (int q = 0; q < g; q++) map[map.size() - 32 + used + q] = r | (q << 16) | (lg << 21);
      used += g;
      mx = std::max(mx, (len + g - 1) / g);
      lgmax = std::max(lgmax, lg);
      two = two || L[i + r].other >= 0;
    }
    close();
    const int ntask = (int)map.size() / 32;
    if (ntask > kMaxTasks) continue;
    constexpr int kWarps = kSweepThreads / 32;
    long warp_t[kWarps] = {}, total = 0;
    for (int t = 0; t < ntask; t++) {
      warp_t[t % kWarps] += 67 * ins[t] + lat[t];
      total += 20 * ins[t];
    }
    long cost = total;
    for (int w = 0; w < kWarps; w++) cost = std::max(cost, warp_t[w]);
    if (best < 0 || cost < best) {
      best = cost;
      best_map = map;
    }
  }
  return best_map;
}

// The trailing triangle segment: FWD the strictly lower part of the trailing
// block (row i, column j < i at i(i-1)/2 + j), else the strictly upper part
// (row i, column j > i at i(2s-i-1)/2 + j-i-1), then 1 / U_rr of its rows.
void build_tri(const Symbolic& s, int r0, int sr, bool fwd, bool use_t, Built& out) {
  const size_t ntri = (size_t)sr * (sr > 0 ? sr - 1 : 0) / 2;
  const size_t nt2 = (ntri + 1) & ~(size_t)1, ns2 = ((size_t)sr + 1) & ~(size_t)1;
  out.bytes.assign(8 * (nt2 + ns2), 0);
  auto code = [&](int p) { return 2 * p + (use_t ? 1 : 0); };
  size_t q = 0;
  if (fwd) {
    for (int i = 1; i < sr; i++)
      for (int j = 0; j < i; j++) out.map.push_back(make_int2((int)q++, code(s.dp[r0 + i] - (i - j))));
  } else {
    for (int i = 0; i + 1 < sr; i++)
      for (int j = i + 1; j < sr; j++) out.map.push_back(make_int2((int)q++, code(s.dp[r0 + i] + (j - i))));
  }
  for (int i = 0; i < sr; i++) out.map.push_back(make_int2((int)(nt2 + i), -1 - (r0 + i)));
}

// Level merging by look-ahead (lookahead = D > 0): a record of a narrow chunk
// t (at most `narrow` records) keeps only its late entries, those whose
// column is written by chunk t - 1; each other entry, whose column is written
// by a chunk q (or is final before the stream), is summed in one of the
// chunks max(q + 1, t - D) .. t - 1, spread so that each of those chunks takes
// about as many of the record's entries (one partial record per chunk and
// record: the same rows, no coupling, no scaling, its sum subtracted from the
// rows' right-hand side).  The rows of chunk t are read by no chunk before t
// and written by none but t and its partial records (each in its own chunk),
// so every partial sum lands before chunk t needs it, and the chain of a
// narrow level shrinks to its late entries while its earlier sums run beside
// the work of the chunks before it.  A partial record needs at least kMinMove
// entries and room in its chunk; otherwise its entries stay with the record.
constexpr int kMinMove = 4;

void lookahead_merge(std::vector<std::vector<Rec>>& ch, const Symbolic& s, int nx, int D, int narrow,
                     size_t slot) {
  if (D <= 0) return;
  const int nch = (int)ch.size();
  std::vector<int> prod(nx, -1);  // chunk writing each row (-1: final before the stream)
  std::vector<int> nrec(nch), ent(nch);
  for (int c = 0; c < nch; c++) {
    nrec[c] = (int)ch[c].size();
    ent[c] = 0;
    for (const Rec& R : ch[c]) {
      prod[R.lead] = c;
      if (R.other >= 0) prod[R.other] = c;
      ent[c] += R.count();
    }
  }
  std::vector<std::vector<Rec>> add(nch);  // partial records, appended after the pass
  for (int t = 1; t < nch; t++) {
    if ((int)ch[t].size() > narrow) continue;
    const int h0 = std::max(0, t - D);
    for (Rec& R : ch[t]) {
      std::vector<std::vector<int>> part(t - h0);
      std::vector<int> late;
      for (int k = 0; k < R.count(); k++) {
        const int p = R.at(k), lo = std::max(h0, prod[s.ci[p]] + 1);
        if (lo > t - 1) {
          late.push_back(p);
          continue;
        }
        int best = lo;  // the least loaded of the chunks that may take it
        for (int h = lo + 1; h < t; h++)
          if (part[h - h0].size() < part[best - h0].size()) best = h;
        part[best - h0].push_back(p);
      }
      for (int h = h0; h < t; h++) {
        std::vector<int>& v = part[h - h0];
        if (v.empty()) continue;
        if ((int)v.size() < kMinMove || nrec[h] + 1 > 32 * kMaxTasks ||
            chunk_bytes(nrec[h] + 1, ent[h] + (int)v.size(), kMaxTasks) > slot) {
          late.insert(late.end(), v.begin(), v.end());
          continue;
        }
        Rec P = R;
        P.coup = -1;
        P.scale = false;
        P.pos = v;
        add[h].push_back(P);
        nrec[h]++;
        ent[h] += (int)v.size();
      }
      if ((int)late.size() == R.count()) continue;  // nothing moved
      std::sort(late.begin(), late.end());
      R.pos = late;
      if (late.empty()) R.q1 = R.q0;  // no late entry: the record only finishes its rows
    }
  }
  for (int h = 0; h < nch; h++) ch[h].insert(ch[h].end(), add[h].begin(), add[h].end());
}

// Appends the levels, each cut into chunks of at most slot bytes (merged by
// look-ahead when D > 0); false if a block alone does not fit.
bool build_stream(const std::vector<std::vector<Rec>>& levels, const Symbolic& s, int nx, bool use_t, size_t slot,
                  int D, int narrow, Built& out) {
  auto code = [&](int p) { return 2 * p + (use_t ? 1 : 0); };
  const size_t first = out.off.size();
  // 1. chunks: each level cut at block boundaries
  std::vector<std::vector<Rec>> chunks;
  for (const auto& L : levels) {
    size_t i = 0;
    while (i < L.size()) {
      int nrec = 0, ent = 0;
      size_t j = i;
      while (j < L.size() && nrec < 32 * kMaxTasks) {
        const int e = L[j].count();
        if (chunk_bytes(nrec + 1, ent + e, kMaxTasks) > slot) break;
        nrec++;
        ent += e;
        j++;
      }
      if (nrec == 0) return false;
      chunks.emplace_back(L.begin() + i, L.begin() + j);
      i = j;
    }
  }
  // 2. level merging
  lookahead_merge(chunks, s, nx, D, narrow, slot);
  // 3. lanes and bytes of each chunk
  for (const auto& L : chunks) {
    const int nrec = (int)L.size();
    int ent = 0;
    for (const Rec& R : L) ent += R.count();
    const std::vector<int> lanes = plan_lanes(L, 0, nrec);
    const int ntask = (int)lanes.size() / 32;
    if (ntask == 0) return false;
    const size_t off = out.bytes.size(), len = chunk_bytes(nrec, ent, ntask);
    if (len > slot) return false;
    out.bytes.resize(off + len, 0);
    out.off.push_back((int)off);
    out.len.push_back((int)len);
    unsigned char* B = out.bytes.data() + off;
    const int E4 = pad4(ent), nrv = rv_count(nrec);
    const int hdr[8] = {nrec, ntask, E4, nrv, 0, 0, 0, 0};
    std::memcpy(B, hdr, sizeof(hdr));
    std::memcpy(B + kHdr, lanes.data(), 4 * lanes.size());
    const size_t o_rec = kHdr + 128 * (size_t)ntask, o_rv = o_rec + 16 * (size_t)nrec;
    const size_t o_ci = o_rv + 8 * (size_t)nrv;
    const size_t o_va = o_ci + 4 * (size_t)E4, o_vb = o_va + 8 * (size_t)E4;
    auto put_map = [&](size_t byte_off, int src) {
      out.map.push_back(make_int2((int)((off + byte_off) / 8), src));
    };
    int eoff = 0;
    for (int r = 0; r < nrec; r++) {
      const Rec& R = L[r];
      const int cnt = R.count();
      const int rec[4] = {R.lead, cnt, R.other, eoff};
      std::memcpy(B + o_rec + 16 * (size_t)r, rec, sizeof(rec));
      const double one = 1.0, zero = 0.0;
      if (R.other >= 0 && R.coup >= 0)
        put_map(o_rv + 8 * (size_t)(3 * r), code(R.coup));
      else
        std::memcpy(B + o_rv + 8 * (size_t)(3 * r), &zero, 8);
      if (R.scale)
        put_map(o_rv + 8 * (size_t)(3 * r + 1), -1 - R.lead);
      else
        std::memcpy(B + o_rv + 8 * (size_t)(3 * r + 1), &one, 8);
      if (R.scale && R.other >= 0)
        put_map(o_rv + 8 * (size_t)(3 * r + 2), -1 - R.other);
      else
        std::memcpy(B + o_rv + 8 * (size_t)(3 * r + 2), &one, 8);
      for (int t = 0; t < cnt; t++) {
        const int p = R.at(t), e = eoff + t;
        std::memcpy(B + o_ci + 4 * (size_t)e, &s.ci[p], 4);
        put_map(o_va + 8 * (size_t)e, code(p));
        if (R.other >= 0) put_map(o_vb + 8 * (size_t)e, code(p + R.off));
      }
      eoff += cnt;
    }
  }
  // each chunk names the chunk two places after it (the one it prefetches)
  const size_t nch = out.off.size();
  for (size_t c = first; c + 2 < nch; c++) {
    int* H = reinterpret_cast<int*>(out.bytes.data() + out.off[c]);
    H[4] = out.off[c + 2];
    H[5] = out.len[c + 2];
  }
  return true;
}

}  // namespace

template <bool TR>
__global__ void solve1s_kernel(DevNet n, SweepStream sf, SweepStream sb, const double* b, double* out,
                               double scale, int slot);

namespace {

// The four streams of one merge schedule: bytes, chunk table and gather map.
struct StreamSet {
  Built B[4];
  std::vector<unsigned char> all;
  std::vector<int2> map;
  std::vector<size_t> base;
  size_t maxlen = 16;
};

// Records of the level schedules: L (LU, forward, unit diagonal), U (LU,
// backward, scaled), U^T (T, forward, scaled), L^T (T, backward, unit
// diagonal).  The forward schedules end with the off-block part of the
// trailing rows (no scaling: the triangle applies it).
bool build_all(const opf_ctx* c, int D, int W, size_t slot, StreamSet& S) {
  const SweepStreams& sw = c->sw;
  const Symbolic& s = c->s;
  const int nx = c->dn.nx, r0 = c->dn.r0, sr = c->dn.nroot;
  std::vector<std::vector<Rec>> lev_f, lev_b;
  for (size_t l = 0; l + 1 < sw.h_bptr_f.size(); l++) {
    std::vector<Rec> L;
    for (int k = sw.h_bptr_f[l]; k < sw.h_bptr_f[l + 1]; k++) {
      const int4 m = sw.h_bmeta_f[k];
      L.push_back({m.x, m.w ? m.x + 1 : -1, m.y, m.z, m.w, m.w ? m.z + m.w : -1, true, {}});
    }
    lev_f.push_back(L);
  }
  {
    std::vector<Rec> L;
    for (int i = r0; i < nx; i++) {
      const int q1 = s.dp[i] - (i - r0);
      if (q1 > s.rp[i]) L.push_back({i, -1, s.rp[i], q1, 0, -1, false, {}});
    }
    std::stable_sort(L.begin(), L.end(), [](const Rec& a, const Rec& b) { return a.q1 - a.q0 > b.q1 - b.q0; });
    if (!L.empty()) lev_f.push_back(L);
  }
  for (size_t l = 0; l + 1 < sw.h_bptr_b.size(); l++) {
    std::vector<Rec> L;
    for (int k = sw.h_bptr_b[l]; k < sw.h_bptr_b[l + 1]; k++) {
      const int4 m = sw.h_bmeta_b[k];
      L.push_back({m.x, m.w ? m.x - 1 : -1, m.y, m.z, m.w, m.w ? m.y + m.w - 1 : -1, true, {}});
    }
    lev_b.push_back(L);
  }
  auto with_scale = [](const std::vector<std::vector<Rec>>& lv, bool on) {
    std::vector<std::vector<Rec>> out;
    for (const auto& L : lv) {
      std::vector<Rec> M;
      for (Rec r : L) {
        r.scale = r.scale && on;
        if (r.other < 0 && !r.scale && r.q1 == r.q0) continue;  // a unit-diagonal row with no entries
        M.push_back(r);
      }
      if (!M.empty()) out.push_back(M);
    }
    return out;
  };
  const std::vector<std::vector<Rec>> src[4] = {with_scale(lev_f, false), with_scale(lev_b, true),
                                                with_scale(lev_f, true), with_scale(lev_b, false)};
  for (int k = 0; k < 4; k++) {
    build_tri(s, r0, sr, k % 2 == 0, k >= 2, S.B[k]);
    S.B[k].tri_len = (int)S.B[k].bytes.size();
    if (!build_stream(src[k], s, nx, k >= 2, slot, D, W, S.B[k])) return false;
  }
  size_t total = 0;
  S.base.assign(4, 0);
  for (int k = 0; k < 4; k++) {
    S.base[k] = total;
    total += S.B[k].bytes.size();
    for (int l : S.B[k].len) S.maxlen = std::max(S.maxlen, (size_t)l);
  }
  S.all.assign(std::max<size_t>(total, 16), 0);
  for (int k = 0; k < 4; k++) {
    if (!S.B[k].bytes.empty()) std::memcpy(S.all.data() + S.base[k], S.B[k].bytes.data(), S.B[k].bytes.size());
    for (const int2& e : S.B[k].map) S.map.push_back(make_int2(e.x + (int)(S.base[k] / 8), e.y));
  }
  return true;
}

// Copies a built set into the context's stream buffers (in place: the LU
// graph's gather keeps its pointers and reads the entry count from the device).
opf_status upload_streams(opf_ctx* c, const StreamSet& S) {
  SweepStreams& sw = c->sw;
  if (S.all.size() > sw.cap_bytes || S.map.size() > sw.cap_map) {
    set_last_error("the merged sweep streams exceed the buffers allocated at load");
    return OPF_EINVAL;
  }
  const int nmap = (int)S.map.size();
  if (cudaMemcpy(sw.values, S.all.data(), S.all.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      (nmap > 0 && cudaMemcpy(sw.map, S.map.data(), S.map.size() * sizeof(int2), cudaMemcpyHostToDevice) !=
                       cudaSuccess) ||
      cudaMemcpy(sw.d_nmap, &nmap, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("cannot upload the single-RHS sweep streams");
    return OPF_ECUDA;
  }
  sw.nmap = nmap;
  for (int k = 0; k < 4; k++) {
    SweepStream& st = sw.s[k];
    st = SweepStream();
    st.base = reinterpret_cast<const unsigned char*>(sw.values) + S.base[k];
    st.tri_len = S.B[k].tri_len;
    st.nch = (int)S.B[k].off.size();
    if (st.nch > 0) {
      st.off0 = S.B[k].off[0];
      st.len0 = S.B[k].len[0];
    }
    if (st.nch > 1) {
      st.off1 = S.B[k].off[1];
      st.len1 = S.B[k].len[1];
    }
  }
  sw.slot = (int)std::max((S.maxlen + 15) / 16 * 16, (sw.tri_bytes + 31) / 32 * 16);
  sw.smem = (int)(sw.fixed + kRing * (size_t)sw.slot);
  return OPF_OK;
}

}  // namespace

opf_status setup_sweep_streams(opf_ctx* c, const std::vector<int>& bptr_f, const std::vector<int4>& bmeta_f,
                               const std::vector<int>& bptr_b, const std::vector<int4>& bmeta_b) {
  SweepStreams& sw = c->sw;
  sw = SweepStreams();
  const int nx = c->dn.nx, sr = c->dn.nroot;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  const size_t cap = (size_t)optin - 1024;
  const size_t ntri = (size_t)sr * (sr > 0 ? sr - 1 : 0) / 2;
  sw.fixed = 8 * (((size_t)nx + 1) & ~(size_t)1);
  sw.tri_bytes = 8 * ((ntri + 1) & ~(size_t)1) + 8 * (((size_t)sr + 1) & ~(size_t)1);
  if (sw.fixed + kRing * (size_t)4096 > cap) return OPF_OK;  // the solution does not fit: level-record form
  sw.max_slot = (cap - sw.fixed) / kRing / 16 * 16;
  if (sw.tri_bytes > 2 * sw.max_slot) return OPF_OK;  // the triangle segment must fit ring slots 1 and 2
  sw.h_bptr_f = bptr_f;
  sw.h_bmeta_f = bmeta_f;
  sw.h_bptr_b = bptr_b;
  sw.h_bmeta_b = bmeta_b;
  int D = kSweepLookahead, W = kSweepNarrow;
  StreamSet S;
  if (!build_all(c, D, W, sw.max_slot, S)) {
    S = StreamSet();
    D = W = 0;
    if (!build_all(c, 0, 0, sw.max_slot, S)) return OPF_OK;
  }
  // buffers with room for the other merge schedules (a merge adds records and
  // padding, never entries)
  sw.cap_bytes = S.all.size() + S.all.size() / 4 + 65536;
  sw.cap_map = S.map.size() + S.map.size() / 4 + 4096;
  void *dv = nullptr, *dm = nullptr, *dn = nullptr;
  if (cudaMalloc(&dv, sw.cap_bytes) != cudaSuccess || cudaMalloc(&dm, sw.cap_map * sizeof(int2)) != cudaSuccess ||
      cudaMalloc(&dn, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (dv) cudaFree(dv);
    if (dm) cudaFree(dm);
    set_last_error("cannot allocate the single-RHS sweep streams");
    return OPF_ENOMEM;
  }
  c->allocs.push_back(dv);
  c->allocs.push_back(dm);
  c->allocs.push_back(dn);
  sw.values = static_cast<double*>(dv);
  sw.map = static_cast<int2*>(dm);
  sw.d_nmap = static_cast<int*>(dn);
  if (opf_status rc = upload_streams(c, S)) return rc;
  if (cudaFuncSetAttribute(solve1s_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap) !=
          cudaSuccess ||
      cudaFuncSetAttribute(solve1s_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap) !=
          cudaSuccess) {
    cudaGetLastError();
    set_last_error("cannot raise the shared-memory limit of the streamed single-RHS sweep");
    return OPF_ECUDA;
  }
  sw.lookahead = D;
  sw.narrow = W;
  sw.ok = true;
  return OPF_OK;
}

opf_status set_sweep_merge(opf_ctx* c, int D, int W) {
  SweepStreams& sw = c->sw;
  if (D < 0 || W < 0 || (D > 0 && W < 1)) {
    set_last_error("lookahead must be >= 0 and narrow >= 1 with a lookahead");
    return OPF_EINVAL;
  }
  if (!sw.ok) return OPF_OK;  // level-record form: nothing to merge
  StreamSet S;
  if (!build_all(c, D, W, sw.max_slot, S)) {
    set_last_error("a merged chunk does not fit a ring slot");
    return OPF_EINVAL;
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {  // no solve still reads the old streams
    cudaGetLastError();
    set_last_error("stream synchronisation failed");
    return OPF_ECUDA;
  }
  if (opf_status rc = upload_streams(c, S)) return rc;
  sw.lookahead = D;
  sw.narrow = W;
  // the values of the new layout: gathered now from factors that are current,
  // else by the next refactorisation
  if (c->have_state && !c->factors_stale) launch_sweep_pack(c);
  return OPF_OK;
}

// ------------------------------------------------------------------ device

namespace {

__device__ __forceinline__ void ring_issue(unsigned char* dst, const unsigned char* src, int len) {
  for (int i = threadIdx.x * 16; i < len; i += blockDim.x * 16) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst + i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + i) : "memory");
  }
}
__device__ __forceinline__ void ring_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void ring_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One chunk.  Each warp task maps its lanes to records (lane map): lane li of
// a record's group of G lanes takes entries li, li + G, ... into one sum per
// row (the group's first lane starts from the right-hand side), the groups
// reduce by shuffles (both rows in one add per round: after the first round
// even lanes carry the lead row and odd lanes the second row), and the first
// lane finishes the block: the lead row, then the second row through the
// coupling entry.
template <bool DIAG>
__device__ __forceinline__ void sweep_chunk(const unsigned char* S, double* X) {
  const int* H = reinterpret_cast<const int*>(S);
  const int ntask = H[1], E4 = H[2], nrv = H[3], nrec = H[0];
  const int* lmap = H + 8;
  const int4* rec = reinterpret_cast<const int4*>(S + 32 + 128 * ntask);
  const double* rv = reinterpret_cast<const double*>(rec + nrec);
  const int* cix = reinterpret_cast<const int*>(rv + nrv);
  const double* va = reinterpret_cast<const double*>(cix + E4);
  const double* vb = va + E4;
  const int lane = threadIdx.x & 31, nwarps = (int)blockDim.x >> 5;
  for (int t = threadIdx.x >> 5; t < ntask; t += nwarps) {
    const int code = lmap[t * 32 + lane];
    const bool act = code >= 0;
    const int r = code & 0xffff, li = (code >> 16) & 31, lg = act ? (code >> 21) & 7 : 0, G = 1 << lg;
    const int4 m = act ? rec[r] : make_int4(0, 0, -1, 0);
    const bool two = m.z >= 0;
    const bool wtwo = __any_sync(0xffffffffu, two);
    const int wlg = __reduce_max_sync(0xffffffffu, (unsigned)lg);
    double a = (act && li == 0) ? X[m.x] : 0.0;
    double c = (two && li == 0) ? X[m.z] : 0.0;
    const int je = m.w + m.y;
    int j = m.w + li;
    if (wtwo) {
      for (; j + 3 * G < je; j += 4 * G) {  // the solution reads first, then the FMAs
        const int c0 = cix[j], c1 = cix[j + G], c2 = cix[j + 2 * G], c3 = cix[j + 3 * G];
        const double x0 = X[c0], x1 = X[c1], x2 = X[c2], x3 = X[c3];
        a = fma(-va[j], x0, a);
        c = fma(-vb[j], x0, c);
        a = fma(-va[j + G], x1, a);
        c = fma(-vb[j + G], x1, c);
        a = fma(-va[j + 2 * G], x2, a);
        c = fma(-vb[j + 2 * G], x2, c);
        a = fma(-va[j + 3 * G], x3, a);
        c = fma(-vb[j + 3 * G], x3, c);
      }
      for (; j < je; j += G) {
        const double x = X[cix[j]];
        a = fma(-va[j], x, a);
        c = fma(-vb[j], x, c);
      }
    } else {
      for (; j + 3 * G < je; j += 4 * G) {
        const int c0 = cix[j], c1 = cix[j + G], c2 = cix[j + 2 * G], c3 = cix[j + 3 * G];
        const double x0 = X[c0], x1 = X[c1], x2 = X[c2], x3 = X[c3];
        a = fma(-va[j], x0, a);
        a = fma(-va[j + G], x1, a);
        a = fma(-va[j + 2 * G], x2, a);
        a = fma(-va[j + 3 * G], x3, a);
      }
      for (; j < je; j += G) a = fma(-va[j], X[cix[j]], a);
    }
    if (wlg > 0) {
      if (wtwo) {
        const bool odd = li & 1;
        const double got = __shfl_xor_sync(0xffffffffu, odd ? a : c, 1);
        double v = (odd ? c : a) + (G >= 2 ? got : 0.0);
        for (int off = 2; off < (1 << wlg); off <<= 1) {
          const double p = __shfl_xor_sync(0xffffffffu, v, off);
          v += off < G ? p : 0.0;
        }
        const double cv = __shfl_down_sync(0xffffffffu, v, 1);
        if (G >= 2) {
          a = v;
          c = cv;
        }
      } else {
        for (int off = 1; off < (1 << wlg); off <<= 1) {
          const double p = __shfl_xor_sync(0xffffffffu, a, off);
          a += off < G ? p : 0.0;
        }
      }
    }
    if (act && li == 0) {
      const double v = DIAG ? a * rv[3 * r + 1] : a;
      X[m.x] = v;
      if (two) {
        const double w = fma(-rv[3 * r], v, c);
        X[m.z] = DIAG ? w * rv[3 * r + 2] : w;
      }
    }
  }
}

// All chunks of one stream; chunks 0 and 1 were issued by the caller as the
// two most recent commit groups.  On return every copy has landed and every
// thread is past the last chunk.
template <bool DIAG>
__device__ __forceinline__ void sweep_stream(const SweepStream& st, unsigned char* ring, int slot, double* X) {
  for (int c = 0; c < st.nch; c++) {
    ring_wait<1>();
    __syncthreads();
    const unsigned char* S = ring + (c % 3) * slot;
    if (c + 2 < st.nch) {
      const int* H = reinterpret_cast<const int*>(S);
      ring_issue(ring + ((c + 2) % 3) * slot, st.base + H[4], H[5]);
    }
    ring_commit();
    sweep_chunk<DIAG>(S, X);
  }
  ring_wait<0>();
  __syncthreads();
}

__device__ __forceinline__ void sweep_prefetch(const SweepStream& st, unsigned char* ring, int slot) {
  if (st.nch > 0) ring_issue(ring, st.base + st.off0, st.len0);
  ring_commit();
  if (st.nch > 1) ring_issue(ring + slot, st.base + st.off1, st.len1);
  ring_commit();
}

// Substitution through the staged trailing triangle (rows r0 .. r0 + s - 1), a
// column per step, then the diagonal scaling (DIAG); dinv holds 1 / U_rr of
// the trailing rows.
// Only the threads with a row to update form x_j: an FP64 instruction costs the
// pipe the same for a warp whatever its active lanes, so idle warps issue none.
template <bool FWD, bool DIAG>
__device__ __forceinline__ void tri_solve(int r0, int s, const double* tri, const double* dinv, double* X) {
  const int tid = threadIdx.x;
  if (FWD) {
    for (int j = 0; j < s - 1; j++) {
      if (tid < s - 1 - j) {
        const double xj = DIAG ? X[r0 + j] * dinv[j] : X[r0 + j];
        for (int i = j + 1 + tid; i < s; i += blockDim.x) X[r0 + i] -= tri[i * (i - 1) / 2 + j] * xj;
      }
      __syncthreads();
    }
  } else {
    for (int j = s - 1; j > 0; j--) {
      if (tid < j) {
        const double xj = DIAG ? X[r0 + j] * dinv[j] : X[r0 + j];
        for (int i = tid; i < j; i += blockDim.x) X[r0 + i] -= tri[i * (2 * s - i - 1) / 2 + (j - i - 1)] * xj;
      }
      __syncthreads();
    }
  }
  if (DIAG) {
    for (int i = threadIdx.x; i < s; i += blockDim.x) X[r0 + i] *= dinv[i];
  }
  __syncthreads();
}

}  // namespace

// out = G_x^{-1} (scale b) (TR = false: L then U from LU) or G_x^{-T} (scale b)
// (TR = true: U^T then L^T from T).  One CTA of 512 threads; dynamic shared
// memory: the solution (n_x doubles) and the ring.
template <bool TR>
__global__ void __launch_bounds__(kSweepThreads) solve1s_kernel(DevNet n, SweepStream sf, SweepStream sb, const double* b,
                                                      double* out, double scale, int slot) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int nx = n.nx, r0 = n.r0, s = n.nroot;
  const int ntri2 = (s * (s - 1) / 2 + 1) & ~1;
  double* X = reinterpret_cast<double*>(sm_raw);
  unsigned char* ring = sm_raw + 8 * ((nx + 1) & ~1);
  // between the two level sweeps the triangle segment occupies slots 1 and 2
  unsigned char* tseg = ring + slot;
  const double* tri = reinterpret_cast<const double*>(tseg);
  const double* dinv = tri + ntri2;
  sweep_prefetch(sf, ring, slot);
  {
    constexpr int U = 4;
    for (int i0 = threadIdx.x; i0 < nx; i0 += U * blockDim.x) {
      int p[U];
      double v[U];
#pragma unroll
      for (int k = 0; k < U; k++) {
        const int i = i0 + k * blockDim.x;
        p[k] = i < nx ? n.perm[i] : 0;
      }
#pragma unroll
      for (int k = 0; k < U; k++) v[k] = (i0 + k * (int)blockDim.x < nx) ? b[p[k]] : 0.0;
#pragma unroll
      for (int k = 0; k < U; k++)
        if (i0 + k * (int)blockDim.x < nx) X[i0 + k * blockDim.x] = scale * v[k];
    }
  }
  sweep_stream<TR>(sf, ring, slot, X);
  ring_issue(tseg, sf.base, sf.tri_len);
  ring_commit();
  if (sb.nch > 0) ring_issue(ring, sb.base + sb.off0, sb.len0);  // lands while the triangles run
  ring_commit();
  ring_wait<1>();
  __syncthreads();
  tri_solve<true, TR>(r0, s, tri, dinv, X);
  ring_issue(tseg, sb.base, sb.tri_len);
  ring_commit();
  ring_wait<0>();
  __syncthreads();
  tri_solve<false, !TR>(r0, s, tri, dinv, X);
  if (sb.nch > 1) ring_issue(ring + slot, sb.base + sb.off1, sb.len1);
  ring_commit();
  sweep_stream<!TR>(sb, ring, slot, X);
  {
    constexpr int U = 4;
    for (int i0 = threadIdx.x; i0 < nx; i0 += U * blockDim.x) {
      int p[U];
#pragma unroll
      for (int k = 0; k < U; k++) {
        const int i = i0 + k * blockDim.x;
        p[k] = i < nx ? n.perm[i] : 0;
      }
#pragma unroll
      for (int k = 0; k < U; k++)
        if (i0 + k * (int)blockDim.x < nx) out[p[k]] = X[i0 + k * blockDim.x];
    }
  }
}

__global__ void sweep_pack_kernel(const double* __restrict__ LU, const double* __restrict__ T,
                                  const double* __restrict__ invdiag, const int2* __restrict__ map,
                                  const int* __restrict__ nmap_dev, double* __restrict__ dst) {
  const int nmap = *nmap_dev;  // read at run time: a new merge schedule keeps the captured launch valid
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nmap; k += gridDim.x * blockDim.x) {
    const int2 e = map[k];
    dst[e.x] = e.y >= 0 ? ((e.y & 1) ? T[e.y >> 1] : LU[e.y >> 1]) : invdiag[-1 - e.y];
  }
}

void launch_sweep_pack(opf_ctx* c) {
  if (!c->sw.ok) return;
  c->launches++;
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((c->sw.cap_map + 255) / 256, 2 * (size_t)c->sm_count));
  sweep_pack_kernel<<<blocks, 256, 0, c->stream>>>(c->LU, c->T, c->invdiag, c->sw.map, c->sw.d_nmap,
                                                   c->sw.values);
}

void launch_solve1_streamed(opf_ctx* c, const double* b, double* out, bool transposed, double scale) {
  c->launches++;
  const SweepStreams& sw = c->sw;
  if (!transposed)
    solve1s_kernel<false><<<1, kSweepThreads, sw.smem, c->stream>>>(c->dn, sw.s[0], sw.s[1], b, out, scale, sw.slot);
  else
    solve1s_kernel<true><<<1, kSweepThreads, sw.smem, c->stream>>>(c->dn, sw.s[2], sw.s[3], b, out, scale, sw.slot);
}

}  // namespace opf
