// Device kernels of libopf (sm_103a, FP64).
//
// Layout: the factors of G_x live in one row-wise array on the filled pattern
// (pivot order): LU holds L (strictly lower, unit diagonal implied) and U
// (diagonal and upper); T holds the transposed values (T at (i,j) = LU at
// (j,i)) so that the forward and backward sweeps of both G_x and G_x^T read
// rows contiguously.  invdiag holds 1/U_ii so no sweep divides.
//
// The Hessian kernel gives each CTA a tile of Hessian columns and runs the
// whole adjoint-adjoint pipeline of Prop. 2 on it with no inter-CTA
// synchronisation: the columns of the Hessian are independent given the
// factors, so CTAs never wait on one another.  Within a CTA a warp holds
// 32/C rows x C columns; the C lanes of a row read the same factor entry
// (broadcast) and C consecutive right-hand-side values (one coalesced load).
#include <algorithm>
#include <cstdint>

#include "opf_internal.h"

namespace opf {

// ------------------------------------------------------------ branch flows

struct Flow {
  double P, Q, A, Bq, vs, vo;
  double dP[4], dQ[4];  // side-local order (v_s, v_o, theta_s, theta_o)
};

__device__ __forceinline__ void side_coeffs(const DevNet& n, int l, int s, double& Gss, double& Bss,
                                            double& Gso, double& Bso) {
  const int nl = n.nl;
  if (s == 0) {
    Gss = n.Y[l];
    Bss = n.Y[nl + l];
    Gso = n.Y[2 * nl + l];
    Bso = n.Y[3 * nl + l];
  } else {
    Gss = n.Y[6 * nl + l];
    Bss = n.Y[7 * nl + l];
    Gso = n.Y[4 * nl + l];
    Bso = n.Y[5 * nl + l];
  }
}

// Flow out of one end of a branch (pi model, polar form) and its gradient.
__device__ __forceinline__ void side_flow_sc(const DevNet& n, int l, int s, double vs, double vo, double sn,
                                             double cs, Flow& o);
__device__ __forceinline__ void side_flow(const DevNet& n, int l, int s, double vs, double vo,
                                          double ang, Flow& o) {
  double sn, cs;
  sincos(ang, &sn, &cs);
  side_flow_sc(n, l, s, vs, vo, sn, cs, o);
}

// side_flow with sin and cos of the angle difference given
__device__ __forceinline__ void side_flow_sc(const DevNet& n, int l, int s, double vs, double vo, double sn,
                                             double cs, Flow& o) {
  double Gss, Bss, Gso, Bso;
  side_coeffs(n, l, s, Gss, Bss, Gso, Bso);
  const double A = Gso * cs + Bso * sn;   // d A / d ang = -Bq
  const double Bq = Gso * sn - Bso * cs;  // d Bq / d ang = A
  const double vv = vs * vo;
  o.A = A;
  o.Bq = Bq;
  o.vs = vs;
  o.vo = vo;
  o.P = vs * vs * Gss + vv * A;
  o.Q = -vs * vs * Bss + vv * Bq;
  o.dP[0] = 2.0 * vs * Gss + vo * A;
  o.dP[1] = vs * A;
  o.dP[2] = -vv * Bq;
  o.dP[3] = vv * Bq;
  o.dQ[0] = -2.0 * vs * Bss + vo * Bq;
  o.dQ[1] = vs * Bq;
  o.dQ[2] = vv * A;
  o.dQ[3] = -vv * A;
}

__device__ __forceinline__ int other_end(const DevNet& n, int e) {
  const int l = e >> 1;
  return (e & 1) ? n.f[l] : n.t[l];
}

__global__ void unpack_kernel(DevNet n, const double* x, const double* u, double* vb, double* tb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n.nb) return;
  vb[i] = (n.type[i] == PQ) ? x[n.xv[i]] : u[n.uv[i]];
  tb[i] = (n.type[i] == REF) ? 0.0 : x[n.xth[i]];
}

// g and the values of G_x in the fixed pattern; one thread owns the rows of its bus.
// Branch terms of the power-flow residual and Jacobian, one thread per branch:
// one sincos serves both ends (the to side's angle is the negated from side's),
// and each end's ten terms {P, Q, dP/dv_s, dP/dth_s, dQ/dv_s, dQ/dth_s, dP/dth_o,
// dP/dv_o, dQ/dth_o, dQ/dv_o} go to ef[e] (e = 2 l + side), which the bus
// kernels (residual and Jacobian, first-order weights, control gradient) sum
// in adjacency order.
__global__ void pf_branch_kernel(DevNet n, const double* vb, const double* tb, double* ef) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n.nl) return;
  const int a = n.f[l], b = n.t[l];
  double sn, cs;
  sincos(tb[a] - tb[b], &sn, &cs);
#pragma unroll
  for (int s = 0; s < 2; s++) {
    const int i = s ? b : a, o = s ? a : b;
    Flow fl;
    side_flow_sc(n, l, s, vb[i], vb[o], s ? -sn : sn, cs, fl);
    double* r = ef + 10 * (size_t)(2 * l + s);
    r[0] = fl.P;
    r[1] = fl.Q;
    r[2] = fl.dP[0];
    r[3] = fl.dP[2];
    r[4] = fl.dQ[0];
    r[5] = fl.dQ[2];
    r[6] = fl.dP[3];
    r[7] = fl.dP[1];
    r[8] = fl.dQ[3];
    r[9] = fl.dQ[1];
  }
}

__global__ void pf_eval_kernel(DevNet n, const double* vb, const double* tb, const double* u,
                               const double* pd, const double* qd, double* g, double* LU,
                               double* scal, const double* ef) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double g2 = 0.0, gi = 0.0;
  if (i < n.nb && n.type[i] != REF) {
    const bool pq = n.type[i] == PQ;
    double P = 0, Q = 0, dPv = 0, dPt = 0, dQv = 0, dQt = 0;
    for (int k = n.adj_ptr[i]; k < n.adj_ptr[i + 1]; k++) {
      const int e = n.adj[k];
      const double* r = ef + 10 * (size_t)e;
      P += r[0];
      Q += r[1];
      dPv += r[2];
      dPt += r[3];
      dQv += r[4];
      dQt += r[5];
      const int* sl = n.slot_adj + 4 * (size_t)e;
      if (sl[0] >= 0) LU[sl[0]] += r[6];
      if (sl[1] >= 0) LU[sl[1]] += r[7];
      if (sl[2] >= 0) LU[sl[2]] += r[8];
      if (sl[3] >= 0) LU[sl[3]] += r[9];
    }
    const int* ss = n.slot_self + 4 * (size_t)i;
    LU[ss[0]] += dPt;
    if (ss[1] >= 0) LU[ss[1]] += dPv;
    if (ss[2] >= 0) LU[ss[2]] += dQt;
    if (ss[3] >= 0) LU[ss[3]] += dQv;
    const double pg = (n.type[i] == PV) ? u[n.up[i]] : 0.0;
    const double gp = P - pg + pd[i];
    g[n.xth[i]] = gp;
    g2 = gp * gp;
    gi = fabs(gp);
    if (pq) {
      const double gq = Q + qd[i];
      g[n.xv[i]] = gq;
      g2 += gq * gq;
      gi = fmax(gi, fabs(gq));
    }
  }
  // block reduction, then one atomic pair per block (same-address atomics serialise)
  __shared__ double r2[32], ri[32];
  for (int off = 16; off > 0; off >>= 1) {
    g2 += __shfl_down_sync(0xffffffffu, g2, off);
    gi = fmax(gi, __shfl_down_sync(0xffffffffu, gi, off));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    r2[wid] = g2;
    ri[wid] = gi;
  }
  __syncthreads();
  if (wid == 0) {
    g2 = lane < nw ? r2[lane] : 0.0;
    gi = lane < nw ? ri[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      g2 += __shfl_down_sync(0xffffffffu, g2, off);
      gi = fmax(gi, __shfl_down_sync(0xffffffffu, gi, off));
    }
    if (lane == 0) {
      atomicAdd(&scal[0], g2);
      // non-negative doubles order like their bit patterns
      atomicMax(reinterpret_cast<unsigned long long*>(&scal[1]), (unsigned long long)__double_as_longlong(gi));
    }
  }
}

// ------------------------------------------------------------ numeric LU

// One level of the right-looking LU on the fixed pattern, by bus blocks (one or
// two pivot rows f, f + 1 whose off-block patterns coincide).  Work items: the
// level's tasks (lu_task: eliminate the block's pivots from one row below it),
// then the finish records of the previous level's two-row blocks (lu_finish),
// which no task of this level reads.
__global__ void lu_level_kernel(double* LU, const int4* __restrict__ trec, const int* __restrict__ toff,
                                const int* __restrict__ map, int t0, int t1, const int4* __restrict__ frec,
                                int f0, int f1, int* flags, int G) {
  // G lanes per work item (a power of two set per level from its longest row):
  // short rows share a warp, so the per-item scalar FP64 work (the pivots'
  // divisions) is not repeated by 32 lanes for one item
  const int lane = threadIdx.x & 31, li = lane & (G - 1), ipw = 32 / G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int ntask = t1 - t0, nall = ntask + (f1 - f0);
  // the task records and targets are static: the first task's are read before
  // the wait for the previous level (programmatic dependent launch)
  const int wfirst = warp * ipw + lane / G;
  int4 tr_first = make_int4(0, 0, 0, 0);
  const int* tg_first = map;
  int tgt_first[LU_PRE] = {0, 0, 0, 0};
  if (wfirst < ntask) {
    tr_first = __ldg(trec + t0 + wfirst);
    tg_first = map + __ldg(toff + t0 + wfirst);
    lu_targets(tr_first, tg_first, li, G, tgt_first);
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the next level's grid may launch now (it waits for this one to finish)
  asm volatile("griddepcontrol.launch_dependents;");
  for (int base = warp * ipw; base < nall; base += nw * ipw) {
    const int w = base + lane / G;
    if (w < ntask) {
      if (w == wfirst) {
        lu_task<false>(LU, tr_first, tg_first, tgt_first, li, G, gmask, flags);
      } else {
        const int t = t0 + w;
        const int4 tr = __ldg(trec + t);
        const int* tg = map + __ldg(toff + t);
        int tgt[LU_PRE];
        lu_targets(tr, tg, li, G, tgt);
        lu_task<false>(LU, tr, tg, tgt, li, G, gmask, flags);
      }
    } else if (w < nall) {
      lu_finish<false>(LU, __ldg(frec + f0 + (w - ntask)), li, G, gmask);
    }
  }
}

// Dense LU of the trailing block [r0, r0 + s) (rows of it are contiguous in LU:
// row i holds columns r0 .. r0 + s - 1 from position dp[r0 + i] - i).  With
// smem, the block is factorised in shared memory (a warp per row of the
// trailing submatrix, lanes along the row).
__global__ void __launch_bounds__(1024) lu_dense_block_kernel(double* LU, const int* __restrict__ dp,
                                                              int r0, int s, int* flags, int smem) {
  extern __shared__ double A[];
  if (smem) {
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
      const int i = idx / s, j = idx - i * s;
      A[idx] = LU[dp[r0 + i] - i + j];
    }
    __syncthreads();
    // threads as 32 x (blockDim / 32): lane -> column, warp -> row
    const int tj = threadIdx.x & 31, ti = threadIdx.x >> 5, nti = blockDim.x >> 5;
    for (int k = 0; k < s - 1; k++) {
      const double ukk = A[k * s + k];
      if (threadIdx.x == 0 && (!(fabs(ukk) > 0.0) || !isfinite(ukk))) flags[0] = 1;
      const double inv = 1.0 / ukk;
      for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) A[i * s + k] *= inv;
      __syncthreads();
      for (int i = k + 1 + ti; i < s; i += nti) {
        const double l = A[i * s + k];
        for (int j = k + 1 + tj; j < s; j += 32) A[i * s + j] -= l * A[k * s + j];
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
      const int i = idx / s, j = idx - i * s;
      LU[dp[r0 + i] - i + j] = A[idx];
    }
    return;
  }
  for (int k = 0; k < s - 1; k++) {
    const int rk = r0 + k;
    const double ukk = LU[dp[rk]];
    if (threadIdx.x == 0 && (!(fabs(ukk) > 0.0) || !isfinite(ukk))) flags[0] = 1;
    const double inv = 1.0 / ukk;
    for (int i = k + 1 + threadIdx.x; i < s; i += blockDim.x) LU[dp[r0 + i] - (i - k)] *= inv;
    __syncthreads();
    const int w = s - 1 - k;
    for (int it = threadIdx.x; it < w * w; it += blockDim.x) {
      const int i = k + 1 + it / w, j = k + 1 + it % w, ri = r0 + i;
      LU[dp[ri] + (j - i)] -= LU[dp[ri] - (i - k)] * LU[dp[rk] + (j - k)];
    }
    __syncthreads();
  }
}
__global__ void lu_finish_kernel(const double* LU, double* T, double* invdiag, const int* tmap,
                                 const int* dp, int nx, int nnz, int* flags) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int i = tid; i < nx; i += nt) {
    const double d = LU[dp[i]];
    if (!(fabs(d) > 0.0) || !isfinite(d)) flags[0] = 1;
    invdiag[i] = 1.0 / d;
  }
  for (int p = tid; p < nnz; p += nt) T[p] = LU[tmap[p]];
}

// ------------------------------------------------------------ sweeps

// Rows [p0, p1) of V against the slab: s = X[i] - sum V[p] X[ci[p]] (two partial
// sums, eight then four loads in flight per lane group; a ragged tail of one to
// three entries is loaded in one batch, absent entries re-reading the first one).
template <int C>
__device__ __forceinline__ double row_dot(const DevNet& n, const double* __restrict__ V, const double* X,
                                          int i, int p0, int p1, int col) {
  double s0 = X[(size_t)i * C + col], s1 = 0.0;
  int p = p0;
  for (; p + 7 < p1; p += 8) {  // eight slab reads in flight
    int ci[8];
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) ci[k] = __ldg(n.ci + p + k);
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = X[(size_t)ci[k] * C + col];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      s0 -= V[p + k] * x[k];
      s1 -= V[p + k + 1] * x[k + 1];
    }
  }
  for (; p + 3 < p1; p += 4) {
    const int c0 = __ldg(n.ci + p), c1 = __ldg(n.ci + p + 1), c2 = __ldg(n.ci + p + 2), c3 = __ldg(n.ci + p + 3);
    const double v0 = V[p], v1 = V[p + 1], v2 = V[p + 2], v3 = V[p + 3];
    const double x0 = X[(size_t)c0 * C + col], x1 = X[(size_t)c1 * C + col];
    const double x2 = X[(size_t)c2 * C + col], x3 = X[(size_t)c3 * C + col];
    s0 -= v0 * x0;
    s1 -= v1 * x1;
    s0 -= v2 * x2;
    s1 -= v3 * x3;
  }
  const int r = p1 - p;
  if (r > 0) {
    const int q1 = p + (r > 1 ? 1 : 0), q2 = p + (r > 2 ? 2 : 0);
    const int c0 = __ldg(n.ci + p), c1 = __ldg(n.ci + q1), c2 = __ldg(n.ci + q2);
    const double v0 = V[p], v1 = V[q1], v2 = V[q2];
    const double x0 = X[(size_t)c0 * C + col], x1 = X[(size_t)c1 * C + col], x2 = X[(size_t)c2 * C + col];
    s0 -= v0 * x0;
    if (r > 1) s1 -= v1 * x1;
    if (r > 2) s0 -= v2 * x2;
  }
  return s0 + s1;
}

// row_dot over the columns set in the bit mask only (the slab is zero on the
// other columns).
template <int C>
__device__ __forceinline__ double row_dot_masked(const DevNet& n, const double* __restrict__ V, const double* X,
                                                 int i, int p0, int p1, int col, const unsigned* mask) {
  double s0 = X[(size_t)i * C + col], s1 = 0.0;
  int p = p0;
  for (; p + 1 < p1; p += 2) {
    const int c0 = __ldg(n.ci + p), c1 = __ldg(n.ci + p + 1);
    const bool b0 = (mask[c0 >> 5] >> (c0 & 31)) & 1u, b1 = (mask[c1 >> 5] >> (c1 & 31)) & 1u;
    if (b0) s0 -= V[p] * X[(size_t)c0 * C + col];
    if (b1) s1 -= V[p + 1] * X[(size_t)c1 * C + col];
  }
  if (p < p1) {
    const int c0 = __ldg(n.ci + p);
    if ((mask[c0 >> 5] >> (c0 & 31)) & 1u) s0 -= V[p] * X[(size_t)c0 * C + col];
  }
  return s0 + s1;
}

// Shared entries [q0, q1) of a bus block against the slab: a -= V[q] X[ci[q]] for
// the lead row and, for a two-row block, b -= V[q + off] X[ci[q]] for the other
// row (one index and one slab load for two products).
template <int C>
__device__ __forceinline__ void block_dot(const DevNet& n, const double* __restrict__ V, const double* X,
                                          int q0, int q1, int off, bool two, int col, double& a, double& b) {
  double a1 = 0.0, b1 = 0.0;
  int p = q0;
  for (; p + 7 < q1; p += 8) {  // eight slab reads in flight per lane
    int ci[8];
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) ci[k] = __ldg(n.ci + p + k);
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = X[(size_t)ci[k] * C + col];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      a -= V[p + k] * x[k];
      a1 -= V[p + k + 1] * x[k + 1];
    }
    if (two) {
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        b -= V[p + off + k] * x[k];
        b1 -= V[p + off + k + 1] * x[k + 1];
      }
    }
  }
  for (; p + 3 < q1; p += 4) {
    const int c0 = __ldg(n.ci + p), c1 = __ldg(n.ci + p + 1), c2 = __ldg(n.ci + p + 2), c3 = __ldg(n.ci + p + 3);
    const double x0 = X[(size_t)c0 * C + col], x1 = X[(size_t)c1 * C + col];
    const double x2 = X[(size_t)c2 * C + col], x3 = X[(size_t)c3 * C + col];
    a -= V[p] * x0;
    a1 -= V[p + 1] * x1;
    a -= V[p + 2] * x2;
    a1 -= V[p + 3] * x3;
    if (two) {
      b -= V[p + off] * x0;
      b1 -= V[p + off + 1] * x1;
      b -= V[p + off + 2] * x2;
      b1 -= V[p + off + 3] * x3;
    }
  }
  const int r = q1 - p;
  if (r > 0) {
    const int p1 = p + (r > 1 ? 1 : 0), p2 = p + (r > 2 ? 2 : 0);
    const int c0 = __ldg(n.ci + p), c1 = __ldg(n.ci + p1), c2 = __ldg(n.ci + p2);
    const double x0 = X[(size_t)c0 * C + col], x1 = X[(size_t)c1 * C + col], x2 = X[(size_t)c2 * C + col];
    a -= V[p] * x0;
    if (two) b -= V[p + off] * x0;
    if (r > 1) {
      a1 -= V[p1] * x1;
      if (two) b1 -= V[p1 + off] * x1;
    }
    if (r > 2) {
      a -= V[p2] * x2;
      if (two) b -= V[p2 + off] * x2;
    }
  }
  a += a1;
  b += b1;
}

// Dense trailing triangle of a sweep with each (row, column) value held in one
// thread's registers: thread t owns column t % C of rows t / C + m (blockDim / C),
// m < MR.  Step j: the owner of row j writes x_j (times 1/U_jj when DIAG) into
// its own slot of tb[s][C], one barrier, then every owner of a later (FWD) or
// earlier row subtracts its entry of V times that value.  The entries of V are
// loaded before the barrier, so their latency hides behind it; the slots are
// written once each, so one barrier per step suffices.  from_tb: the starting
// values are in tb (else in X); the results go to X, scaled by 1/U_ii when DIAG.
// Needs s C <= MR blockDim and tb holding s C doubles.
template <int C, bool FWD, bool DIAG, int MR>
__device__ __forceinline__ void tri_regs(const DevNet& n, const double* __restrict__ V,
                                         const double* __restrict__ invdiag, double* X, double* tb,
                                         bool from_tb) {
  const int r0 = n.r0, s = n.nroot;
  const int c = threadIdx.x % C, i0 = threadIdx.x / C, di = blockDim.x / C;
  double x[MR], dg[MR];
  int dpi[MR];
#pragma unroll
  for (int m = 0; m < MR; m++) {
    const int i = i0 + m * di;
    const bool own = i < s;
    x[m] = own ? (from_tb ? tb[i * C + c] : X[(size_t)(r0 + i) * C + c]) : 0.0;
    dpi[m] = own ? n.dp[r0 + i] : 0;
    dg[m] = (DIAG && own) ? invdiag[r0 + i] : 1.0;
  }
  for (int st = 0; st + 1 < s; st++) {
    const int j = FWD ? st : s - 1 - st;
    double v[MR];
#pragma unroll
    for (int m = 0; m < MR; m++) {
      const int i = i0 + m * di;
      const bool act = FWD ? (i > j && i < s) : (i < j);
      v[m] = act ? V[dpi[m] + (j - i)] : 0.0;  // entry (i, j): dp[i] + (j - i)
      if (i == j) tb[j * C + c] = x[m] * dg[m];
    }
    __syncthreads();
    const double xj = tb[j * C + c];
#pragma unroll
    for (int m = 0; m < MR; m++) {
      const int i = i0 + m * di;
      if (FWD ? (i > j && i < s) : (i < j)) x[m] = fma(-v[m], xj, x[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < MR; m++) {
    const int i = i0 + m * di;
    if (i < s) X[(size_t)(r0 + i) * C + c] = x[m] * dg[m];
  }
  __syncthreads();
}

// One triangular sweep over a CTA-private right-hand-side slab X[n_x][C].
// Rows outside the dense trailing block [r0, n_x) follow the level schedule
// (FWD: lower part of V, rows by ascending level; else the upper part).  The
// dense block is solved as a dense triangle, one column per step: after x_j is
// known every thread updates its (row, column) items below (FWD) or above it.
// DIAG: multiply each row by 1/U_ii once its sum is complete.  rmask (FWD
// only): the rows below r0 are already final and the slab is zero outside the
// rows set in the mask; only the trailing block remains.  lcnt (backward only):
// run the levels of the L^T ordering (DevNet::bmeta_lt), only the first
// lcnt[lv] blocks of level lv.  zmask (backward only): a row below r0 whose
// bit is clear starts from zero (its slab entries are not read: they were
// never written).
template <int C, bool FWD, bool DIAG>
__device__ __forceinline__ void sweep(const DevNet& n, const double* __restrict__ V,
                                      const double* __restrict__ invdiag, double* X,
                                      const unsigned* rmask = nullptr, double* tb = nullptr,
                                      const int* lcnt = nullptr, const unsigned* zmask = nullptr) {
  constexpr int RPW = 32 / C;
  constexpr int TRI_MR = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = lane % C;
  const int nslots = (blockDim.x >> 5) * RPW, myslot = warp * RPW + lane / C;
  const int r0 = n.r0, s = n.nroot;
  // a row's starting value
  auto start = [&](int r) -> double {
    if (!FWD && zmask && r < r0 && !((zmask[r >> 5] >> (r & 31)) & 1u)) return 0.0;
    return X[(size_t)r * C + col];
  };
  // the triangle in registers when the caller lends shared memory for it
  const bool treg = tb != nullptr && s * C <= TRI_MR * (int)blockDim.x;
  if (!FWD && treg) tri_regs<C, false, DIAG, TRI_MR>(n, V, invdiag, X, tb, false);
  if (!FWD && !treg) {  // dense upper triangle of the trailing block first
    for (int j = s - 1; j > 0; j--) {
      const int rj = r0 + j;
      const double dj = DIAG ? invdiag[rj] : 1.0;
      for (int it = threadIdx.x; it < j * C; it += blockDim.x) {
        const int i = it / C, c = it % C, ri = r0 + i;
        X[(size_t)ri * C + c] -= V[n.dp[ri] + (j - i)] * (X[(size_t)rj * C + c] * dj);
      }
      __syncthreads();
    }
    if (DIAG) {
      for (int it = threadIdx.x; it < s * C; it += blockDim.x) {
        const int i = it / C, c = it % C;
        X[(size_t)(r0 + i) * C + c] *= invdiag[r0 + i];
      }
      __syncthreads();
    }
  }
  // levels of bus blocks (one or two pivot rows each, see DevNet::bmeta_f)
  const int nlev = (FWD && rmask) ? 0 : (FWD ? n.nblev_f : n.nblev_b);
  const int* lptr = FWD ? n.bptr_f : n.bptr_b;
  const int4* lmeta = FWD ? n.bmeta_f : (lcnt ? n.bmeta_lt : n.bmeta_b);
  const int nwarps = blockDim.x >> 5, grp = lane / C;
  // the block's other row and its coupling entry (the diagonal block's off-diagonal)
  auto other_of = [](const int4& m) { return FWD ? m.x + 1 : m.x - 1; };
  auto coupling = [](const int4& m) { return FWD ? m.z + m.w : m.y + m.w - 1; };
  // narrow level (at most one block per warp): one warp per block, its lane
  // groups split the entries; else one lane group per block
  auto first_k = [&](int b, int e) { return (e - b <= nwarps && RPW > 1) ? b + warp : b + myslot; };
  const int4 none = make_int4(0, 0, 0, 0);
  // level lv: blocks [b, e) of [b, ef) (e < ef: a prefix, with lcnt)
  int b = nlev > 0 ? lptr[0] : 0, ef = nlev > 0 ? lptr[1] : 0;
  int e = (lcnt && nlev > 0) ? b + lcnt[0] : ef;
  int k0 = first_k(b, e);
  int4 mt = k0 < e ? __ldg(lmeta + k0) : none;
  for (int lv = 0; lv < nlev; lv++) {
    // the next level's bounds and this thread's first record of it do not
    // depend on the slab: load them before this level's work
    const int bn = ef, efn = (lv + 1 < nlev) ? lptr[lv + 2] : ef;
    const int en = (lcnt && lv + 1 < nlev) ? bn + lcnt[lv + 1] : efn;
    const int kn0 = first_k(bn, en);
    const int4 mtn = kn0 < en ? __ldg(lmeta + kn0) : none;
    if (e - b <= nwarps && RPW > 1) {
      for (int k = k0; k < e; k += nwarps) {
        const int4 m = (k == k0) ? mt : __ldg(lmeta + k);
        const bool two = m.w != 0;
        const int lead = m.x, oth = other_of(m), q1 = m.z, off = m.w;
        const double xl = start(lead), xo = two ? start(oth) : 0.0;
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
        int p = m.y + grp;
        for (; p + 3 * RPW < q1; p += 4 * RPW) {  // four slab reads in flight per lane
          const int c0 = __ldg(n.ci + p), c1 = __ldg(n.ci + p + RPW);
          const int c2 = __ldg(n.ci + p + 2 * RPW), c3 = __ldg(n.ci + p + 3 * RPW);
          const double x0 = X[(size_t)c0 * C + col], x1 = X[(size_t)c1 * C + col];
          const double x2 = X[(size_t)c2 * C + col], x3 = X[(size_t)c3 * C + col];
          a0 -= V[p] * x0;
          a1 -= V[p + RPW] * x1;
          a0 -= V[p + 2 * RPW] * x2;
          a1 -= V[p + 3 * RPW] * x3;
          if (two) {
            b0 -= V[p + off] * x0;
            b1 -= V[p + off + RPW] * x1;
            b0 -= V[p + off + 2 * RPW] * x2;
            b1 -= V[p + off + 3 * RPW] * x3;
          }
        }
        for (; p + RPW < q1; p += 2 * RPW) {
          const int c0 = __ldg(n.ci + p), c1 = __ldg(n.ci + p + RPW);
          const double x0 = X[(size_t)c0 * C + col], x1 = X[(size_t)c1 * C + col];
          a0 -= V[p] * x0;
          a1 -= V[p + RPW] * x1;
          if (two) {
            b0 -= V[p + off] * x0;
            b1 -= V[p + off + RPW] * x1;
          }
        }
        if (p < q1) {
          const double x0 = X[(size_t)__ldg(n.ci + p) * C + col];
          a0 -= V[p] * x0;
          if (two) b0 -= V[p + off] * x0;
        }
        double va = a0 + a1, vb = b0 + b1;
#pragma unroll
        for (int o = C; o < 32; o <<= 1) {
          va += __shfl_xor_sync(0xffffffffu, va, o);
          vb += __shfl_xor_sync(0xffffffffu, vb, o);
        }
        if (grp == 0) {
          va += xl;
          if (DIAG) va *= invdiag[lead];
          X[(size_t)lead * C + col] = va;
          if (two) {
            vb += xo;
            vb -= V[coupling(m)] * va;
            if (DIAG) vb *= invdiag[oth];
            X[(size_t)oth * C + col] = vb;
          }
        }
      }
    } else {
      for (int k = k0; k < e; k += nslots) {
        const int4 m = mt;
        if (k + nslots < e) mt = __ldg(lmeta + k + nslots);  // next block's record in flight
        const bool two = m.w != 0;
        if (!DIAG && !two && m.y == m.z) continue;           // one row, no entries: final
        const int lead = m.x, oth = other_of(m);
        double va = start(lead), vb = two ? start(oth) : 0.0;
        block_dot<C>(n, V, X, m.y, m.z, m.w, two, col, va, vb);
        if (DIAG) va *= invdiag[lead];
        X[(size_t)lead * C + col] = va;
        if (two) {
          vb -= V[coupling(m)] * va;
          if (DIAG) vb *= invdiag[oth];
          X[(size_t)oth * C + col] = vb;
        }
      }
    }
    __syncthreads();
    b = bn;
    e = en;
    ef = efn;
    k0 = kn0;
    mt = mtn;
  }
  if (FWD) {
    // off-block part of the trailing rows (columns < r0), all rows in parallel
    for (int k = myslot; k < s; k += nslots) {
      const int i = r0 + k;
      const double xi = rmask ? row_dot_masked<C>(n, V, X, i, n.rp[i], n.dp[i] - k, col, rmask)
                              : row_dot<C>(n, V, X, i, n.rp[i], n.dp[i] - k, col);
      if (treg) {
        tb[k * C + col] = xi;
      } else {
        X[(size_t)i * C + col] = xi;
      }
    }
    __syncthreads();
    if (treg) {
      tri_regs<C, true, DIAG, TRI_MR>(n, V, invdiag, X, tb, true);
      return;
    }
    // dense lower triangle
    for (int j = 0; j < s - 1; j++) {
      const int rj = r0 + j;
      const double dj = DIAG ? invdiag[rj] : 1.0;
      for (int it = threadIdx.x; it < (s - 1 - j) * C; it += blockDim.x) {
        const int i = j + 1 + it / C, c = it % C, ri = r0 + i;
        X[(size_t)ri * C + c] -= V[n.dp[ri] - (i - j)] * (X[(size_t)rj * C + c] * dj);
      }
      __syncthreads();
    }
    if (DIAG) {
      for (int it = threadIdx.x; it < s * C; it += blockDim.x) {
        const int i = it / C, c = it % C;
        X[(size_t)(r0 + i) * C + c] *= invdiag[r0 + i];
      }
      __syncthreads();
    }
  }
}

// Single-RHS sweep with the dense trailing triangle staged in shared memory:
// levels as in sweep<1>, then (FWD) the off-block part of the trailing rows and
// the triangle column by column reading the staged values, or (backward) the
// triangle first.  tri holds the strictly lower (FWD) or strictly upper part of
// the trailing block, packed by rows.
template <bool FWD, bool DIAG>
__device__ __forceinline__ void sweep1(const DevNet& n, const double* __restrict__ V,
                                       const double* __restrict__ invdiag, double* X, double* tri) {
  const int r0 = n.r0, s = n.nroot;
  // stage the triangle: FWD row i (1..s-1), column j < i at i(i-1)/2 + j;
  // backward row i (0..s-2), column j > i at (i(2s-i-1))/2 + (j-i-1)
  const int ntri = s * (s - 1) / 2;
  for (int q = threadIdx.x; q < ntri; q += blockDim.x) {
    if (FWD) {
      int i = (int)((1.0 + sqrt(1.0 + 8.0 * q)) * 0.5);
      while (i * (i - 1) / 2 > q) i--;
      while ((i + 1) * i / 2 <= q) i++;
      const int j = q - i * (i - 1) / 2;
      tri[q] = V[n.dp[r0 + i] - (i - j)];
    } else {
      int i = 0;
      // rows of the upper part have s-1, s-2, ... entries
      int lo = 0, hi = s - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mid * (2 * s - mid - 1) / 2 <= q) lo = mid; else hi = mid - 1;
      }
      i = lo;
      const int j = i + 1 + (q - i * (2 * s - i - 1) / 2);
      tri[q] = V[n.dp[r0 + i] + (j - i)];
    }
  }
  if (!FWD) {
    __syncthreads();
    for (int j = s - 1; j > 0; j--) {
      const double xj = X[r0 + j] * (DIAG ? invdiag[r0 + j] : 1.0);
      for (int i = threadIdx.x; i < j; i += blockDim.x)
        X[r0 + i] -= tri[i * (2 * s - i - 1) / 2 + (j - i - 1)] * xj;
      __syncthreads();
    }
    if (DIAG) {
      for (int i = threadIdx.x; i < s; i += blockDim.x) X[r0 + i] *= invdiag[r0 + i];
      __syncthreads();
    }
  }
  // levels of bus blocks below r0 (see DevNet::bmeta_f).  A level of cnt blocks
  // gives each block G lanes (the largest power of two <= min(32, threads / cnt)):
  // the lanes split the block's entries and reduce by shuffles.  The factor
  // data is static, so each level prefetches the next level's block record and
  // first entry before the barrier; only X reads stay on the chain.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nlev = FWD ? n.nblev_f : n.nblev_b;
  const int* lptr = FWD ? n.bptr_f : n.bptr_b;
  const int4* lmeta = FWD ? n.bmeta_f : n.bmeta_b;
  auto other_of = [](const int4& m) { return FWD ? m.x + 1 : m.x - 1; };
  auto coupling = [](const int4& m) { return FWD ? m.z + m.w : m.y + m.w - 1; };
  auto lanes_for = [&](int cnt) {
    int g = (int)blockDim.x / (cnt > 0 ? cnt : 1);
    g = g > 32 ? 32 : (g < 1 ? 1 : g);
    return 1 << (31 - __clz(g));
  };
  const int4 none = make_int4(0, 0, 0, 0);
  int4 mt = none;
  int pc = -1;
  double pva = 0.0, pvb = 0.0;
  auto fetch = [&](int lb, int le) {
    const int G = lanes_for(le - lb);
    const int k = lb + warp * (32 / G) + lane / G;
    mt = (k < le) ? lmeta[k] : none;
    const int p = mt.y + (lane & (G - 1));
    pc = (k < le && p < mt.z) ? n.ci[p] : -1;
    pva = (pc >= 0) ? V[p] : 0.0;
    pvb = (pc >= 0 && mt.w) ? V[p + mt.w] : 0.0;
  };
  int b = nlev > 0 ? lptr[0] : 0, e = nlev > 0 ? lptr[1] : 0;
  if (nlev > 0) fetch(b, e);
  for (int lv = 0; lv < nlev; lv++) {
    const int en = (lv + 1 < nlev) ? lptr[lv + 2] : e;
    const int G = lanes_for(e - b), gpw = 32 / G, ngroups = (int)blockDim.x / G, li = lane & (G - 1);
    for (int base = b + warp * gpw, first = 1; base < e; base += ngroups, first = 0) {
      const int k = base + lane / G;
      const bool act = k < e;
      const int4 m = act ? (first ? mt : lmeta[k]) : none;
      const bool two = m.w != 0;
      double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
      int p = m.y + li;
      if (first) {
        if (pc >= 0) {
          const double x = X[pc];
          a0 -= pva * x;
          b0 -= pvb * x;
        }
        p += G;
      }
      for (; p + G < m.z; p += 2 * G) {
        const int c0 = n.ci[p], c1 = n.ci[p + G];
        const double x0 = X[c0], x1 = X[c1];
        a0 -= V[p] * x0;
        a1 -= V[p + G] * x1;
        if (two) {
          b0 -= V[p + m.w] * x0;
          b1 -= V[p + m.w + G] * x1;
        }
      }
      if (p < m.z) {
        const double x0 = X[n.ci[p]];
        a0 -= V[p] * x0;
        if (two) b0 -= V[p + m.w] * x0;
      }
      double va = a0 + a1, vb = b0 + b1;
      for (int off = 1; off < G; off <<= 1) {
        va += __shfl_xor_sync(0xffffffffu, va, off);
        vb += __shfl_xor_sync(0xffffffffu, vb, off);
      }
      if (act && li == 0) {
        va += X[m.x];
        if (DIAG) va *= invdiag[m.x];
        X[m.x] = va;
        if (two) {
          const int o = other_of(m);
          vb += X[o] - V[coupling(m)] * va;
          if (DIAG) vb *= invdiag[o];
          X[o] = vb;
        }
      }
    }
    if (lv + 1 < nlev) fetch(e, en);
    __syncthreads();
    b = e;
    e = en;
  }
  if (FWD) {
    for (int k = warp; k < s; k += nwarps) {  // off-block part of the trailing rows, a warp per row
      const int i = r0 + k;
      const int p1 = n.dp[i] - k;
      double v = 0.0;
      for (int p = n.rp[i] + lane; p < p1; p += 32) v -= V[p] * X[n.ci[p]];
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) X[i] += v;
    }
    __syncthreads();
    for (int j = 0; j < s - 1; j++) {
      const double xj = X[r0 + j] * (DIAG ? invdiag[r0 + j] : 1.0);
      for (int i = j + 1 + threadIdx.x; i < s; i += blockDim.x) X[r0 + i] -= tri[i * (i - 1) / 2 + j] * xj;
      __syncthreads();
    }
    if (DIAG) {
      for (int i = threadIdx.x; i < s; i += blockDim.x) X[r0 + i] *= invdiag[r0 + i];
      __syncthreads();
    }
  }
  __syncthreads();
}

// Single right-hand side: out = G_x^{-1} (scale b) or G_x^{-T} (scale b).  One CTA.
// Dynamic shared memory: the packed dense triangle (s(s-1)/2 doubles) and, when
// use_smem, the right-hand side (n_x doubles) after it.
__global__ void __launch_bounds__(512) solve1_kernel(DevNet n, const double* LU, const double* T,
                                                       const double* invdiag, const double* b,
                                                       double* out, double* yg, int transposed,
                                                       double scale, int use_smem) {
  extern __shared__ double dsm[];
  double* tri = dsm;
  double* y = use_smem ? dsm + (n.nroot * (n.nroot - 1) / 2) : yg;
  for (int i = threadIdx.x; i < n.nx; i += blockDim.x) y[i] = scale * b[n.perm[i]];
  __syncthreads();
  if (!transposed) {
    sweep1<true, false>(n, LU, invdiag, y, tri);
    sweep1<false, true>(n, LU, invdiag, y, tri);
  } else {
    sweep1<true, true>(n, T, invdiag, y, tri);
    sweep1<false, false>(n, T, invdiag, y, tri);
  }
  for (int i = threadIdx.x; i < n.nx; i += blockDim.x) out[n.perm[i]] = y[i];
}

__global__ void axpy_kernel(double* x, const double* d, double a, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += a * d[i];
}

// ------------------------------------------------------------ gradient

__global__ void branch_flow_kernel(DevNet n, const double* vb, const double* tb, double* flows,
                                   double* c) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n.nl) return;
  const int a = n.f[l], b = n.t[l];
  Flow ff, ft;
  side_flow(n, l, 0, vb[a], vb[b], tb[a] - tb[b], ff);
  side_flow(n, l, 1, vb[b], vb[a], tb[b] - tb[a], ft);
  flows[l] = ff.P;
  flows[n.nl + l] = ff.Q;
  flows[2 * n.nl + l] = ft.P;
  flows[3 * n.nl + l] = ft.Q;
  c[l] = ff.P * ff.P + ff.Q * ff.Q;
  c[n.nl + l] = ft.P * ft.P + ft.Q * ft.Q;
}

__global__ void bus_inj_kernel(DevNet n, const double* vb, const double* flows, const double* pd,
                               const double* qd, double* Pb, double* Qb, double* c) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n.nb) return;
  double P = 0, Q = 0;
  for (int k = n.adj_ptr[i]; k < n.adj_ptr[i + 1]; k++) {
    const int e = n.adj[k], l = e >> 1, s = e & 1;
    P += flows[(2 * s) * n.nl + l];
    Q += flows[(2 * s + 1) * n.nl + l];
  }
  Pb[i] = P;
  Qb[i] = Q;
  const int o = 2 * n.nl;
  if (n.type[i] == PQ) c[o + n.pqpos[i]] = vb[i];
  else if (n.type[i] == REF) {
    c[o + n.npq] = P + pd[i];
    c[o + n.npq + 1] = Q + qd[i];
  } else c[o + n.npq + 2 + n.pvpos[i]] = Q + qd[i];
}

// phi'_i, grad_s, omega and the value of F (reduced into scal[2]).
__global__ void al_weights_kernel(DevNet n, const double* c, const double* sig, const double* y,
                                  const double* s, const double* om_in, double rho, double sigma_f,
                                  const double* Pb, const double* u, const double* pd,
                                  const double* c0, double* phid, double* gs, double* om,
                                  double* scal) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double part = 0.0;
  if (i < n.m) {
    const double r = c[i] - s[i], sg = sig[i];
    phid[i] = y[i] * sg + rho * sg * sg * r;
    if (gs) gs[i] = -phid[i];
    om[i] = om_in ? om_in[i] : rho * sg * sg;
    part = y[i] * sg * r + 0.5 * rho * sg * sg * r * r;
  }
  if (i < n.ng) {
    // cost of generator i (the slack takes p_ref = P_ref + pd_ref)
    const int b = n.gbus[i];
    const double p = (n.type[b] == REF) ? Pb[b] + pd[b] : u[n.up[b]];
    part += sigma_f * (n.c2[i] * p * p + n.c1[i] * p + c0[i]);
  }
  for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(&scal[2], part);
}

// First-order weights of F on the injections of bus b.
__device__ __forceinline__ void f_weights(const DevNet& n, int b, const double* phid,
                                          double sigma_f, double pref, double& wP, double& wQ) {
  const int orr = 2 * n.nl + n.npq;
  if (n.type[b] == REF) {
    const int g = n.gen_at[b];
    wP = phid[orr] + sigma_f * (2.0 * n.c2[g] * pref + n.c1[g]);
    wQ = phid[orr + 1];
  } else if (n.type[b] == PV) {
    wP = 0.0;
    wQ = phid[orr + 2 + n.pvpos[b]];
  } else {
    wP = 0.0;
    wQ = 0.0;
  }
}

// Partial derivatives of F w.r.t. (v_i, theta_i), gathered over the incident branches.
__global__ void dF_bus_kernel(DevNet n, const double* u, const double* phid, const double* Pb, const double* pd,
                              double sigma_f, double* dFx, double* dFu, const double* __restrict__ ef) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n.nb) return;
  const double pref = Pb[n.ref] + pd[n.ref];
  double wPi, wQi;
  f_weights(n, i, phid, sigma_f, pref, wPi, wQi);
  double dv = 0.0, dt = 0.0;
  for (int k = n.adj_ptr[i]; k < n.adj_ptr[i + 1]; k++) {
    const int e = n.adj[k], l = e >> 1, s = e & 1, o = other_end(n, e);
    const double* fi = ef + 10 * (size_t)e;        // this end
    const double* fo = ef + 10 * (size_t)(e ^ 1);  // the other end
    const double phi_i = phid[s * n.nl + l], phi_o = phid[(1 - s) * n.nl + l];
    double wPo, wQo;
    f_weights(n, o, phid, sigma_f, pref, wPo, wQo);
    const double ai = 2.0 * phi_i * fi[0] + wPi, bi = 2.0 * phi_i * fi[1] + wQi;
    const double ao = 2.0 * phi_o * fo[0] + wPo, bo = 2.0 * phi_o * fo[1] + wQo;
    dv += ai * fi[2] + bi * fi[4] + ao * fo[7] + bo * fo[9];
    dt += ai * fi[3] + bi * fi[5] + ao * fo[6] + bo * fo[8];
  }
  if (n.type[i] == PQ) dv += phid[2 * n.nl + n.pqpos[i]];
  if (n.type[i] != REF) dFx[n.xth[i]] = dt;
  if (n.type[i] == PQ) dFx[n.xv[i]] = dv;
  else dFu[n.uv[i]] = dv;
  if (n.type[i] == PV) {
    const int g = n.gen_at[i];
    const double p = u[n.up[i]];
    dFu[n.up[i]] = sigma_f * (2.0 * n.c2[g] * p + n.c1[g]);
  }
}

// grad_u = d_u F + G_u^T lambda, one thread per control bus (slack and PV).
__global__ void grad_u_kernel(DevNet n, const double* lam, const double* dFu, double* gu,
                              const double* __restrict__ ef) {
  int gidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (gidx >= n.ngn) return;
  const int k = n.gn_bus[gidx];
  double gv = dFu[n.uv[k]], selfP = 0.0;
  for (int q = n.adj_ptr[k]; q < n.adj_ptr[k + 1]; q++) {
    const int e = n.adj[q], o = other_end(n, e);
    const double* fo = ef + 10 * (size_t)(e ^ 1);  // the other end: its derivatives by v_k
    if (n.type[o] != REF) gv += lam[n.xth[o]] * fo[7];
    if (n.type[o] == PQ) gv += lam[n.xv[o]] * fo[9];
    if (n.type[k] == PV) selfP += ef[10 * (size_t)e + 2];
  }
  if (n.type[k] == PV) {
    gv += lam[n.xth[k]] * selfP;
    gu[n.up[k]] = dFu[n.up[k]] - lam[n.xth[k]];
  }
  gu[n.uv[k]] = gv;
}

__global__ void grad_load_kernel(DevNet n, const double* lam, const double* phid, const double* Pb,
                                 const double* pd, double sigma_f, double* gpd, double* gqd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n.nb) return;
  const int orr = 2 * n.nl + n.npq;
  if (n.type[i] == REF) {
    const int g = n.gen_at[i];
    const double pref = Pb[i] + pd[i];
    if (gpd) gpd[i] = sigma_f * (2.0 * n.c2[g] * pref + n.c1[g]) + phid[orr];
    if (gqd) gqd[i] = phid[orr + 1];
  } else {
    if (gpd) gpd[i] = lam[n.xth[i]];
    if (gqd) gqd[i] = (n.type[i] == PV) ? phid[orr + 2 + n.pvpos[i]] : lam[n.xv[i]];
  }
}

// ------------------------------------------------------------ Hessian tables

// Packed index of the symmetric 4x4 branch matrix, branch-local order (v_f, v_t, theta_f, theta_t).
__host__ __device__ __forceinline__ int pk(int a, int b) {
  if (a > b) {
    int t = a;
    a = b;
    b = t;
  }
  return a * 4 - (a * (a - 1)) / 2 + (b - a);
}

// Per branch: the 4x4 second derivative of l = F + lambda^T g restricted to the
// branch (injection weights, line-flow penalty curvature and omega-weighted
// Gauss-Newton term of the flows), and both ends' flow gradients.
__global__ void hess_prep_kernel(DevNet n, const double* vb, const double* tb, const double* lam,
                                 const double* phid, const double* om, const double* Pb,
                                 const double* pd, double sigma_f, double* tab) {
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n.nl) return;
  const int nl = n.nl, orr = 2 * nl + n.npq;
  const double pref = Pb[n.ref] + pd[n.ref];
  double M[10];
#pragma unroll
  for (int k = 0; k < 10; k++) M[k] = 0.0;
  for (int s = 0; s < 2; s++) {
    const int b = s ? n.t[l] : n.f[l], o = s ? n.f[l] : n.t[l];
    Flow F;
    side_flow(n, l, s, vb[b], vb[o], tb[b] - tb[o], F);
    double wP, wQ;
    if (n.type[b] == REF) {
      const int g = n.gen_at[b];
      wP = phid[orr] + sigma_f * (2.0 * n.c2[g] * pref + n.c1[g]);
      wQ = phid[orr + 1];
    } else if (n.type[b] == PV) {
      wP = lam[n.xth[b]];
      wQ = phid[orr + 2 + n.pvpos[b]];
    } else {
      wP = lam[n.xth[b]];
      wQ = lam[n.xv[b]];
    }
    const double ph = phid[s * nl + l], w2 = om[s * nl + l];
    const double aP = wP + 2.0 * ph * F.P, aQ = wQ + 2.0 * ph * F.Q;
    const double A = F.A, Bq = F.Bq, vs = F.vs, vo = F.vo, vv = vs * vo;
    double Gss, Bss, Gso, Bso;
    side_coeffs(n, l, s, Gss, Bss, Gso, Bso);
    const double hP[4][4] = {{2.0 * Gss, A, -vo * Bq, vo * Bq},
                             {A, 0.0, -vs * Bq, vs * Bq},
                             {-vo * Bq, -vs * Bq, -vv * A, vv * A},
                             {vo * Bq, vs * Bq, vv * A, -vv * A}};
    const double hQ[4][4] = {{-2.0 * Bss, Bq, vo * A, -vo * A},
                             {Bq, 0.0, vs * A, -vs * A},
                             {vo * A, vs * A, -vv * Bq, vv * Bq},
                             {-vo * A, -vs * A, vv * Bq, -vv * Bq}};
    double gh[4];
#pragma unroll
    for (int k = 0; k < 4; k++) gh[k] = 2.0 * (F.P * F.dP[k] + F.Q * F.dQ[k]);
    // side-local (v_s, v_o, th_s, th_o) -> branch-local (v_f, v_t, th_f, th_t)
    const int map[4] = {s, 1 - s, 2 + s, 3 - s};
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int c = a; c < 4; c++) {
        const double val = aP * hP[a][c] + aQ * hQ[a][c] +
                           2.0 * ph * (F.dP[a] * F.dP[c] + F.dQ[a] * F.dQ[c]) + w2 * gh[a] * gh[c];
        M[pk(map[a], map[c])] += val;
      }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      tab[(size_t)TAB_DP(s, map[k]) * nl + l] = F.dP[k];
      tab[(size_t)TAB_DQ(s, map[k]) * nl + l] = F.dQ[k];
      tab[(size_t)TAB_DS(s, map[k]) * nl + l] = gh[k];
    }
  }
#pragma unroll
  for (int k = 0; k < 10; k++) tab[(size_t)k * nl + l] = M[k];
}

// Bus weights: [0] kQ (omega of q_ref / q_pv), [1] kP (omega of p_ref plus the
// slack cost curvature 2 sigma_f c2), [2] omega of v_pq, [3] 2 sigma_f c2 of a PV unit.
__global__ void bus_weight_kernel(DevNet n, const double* om, double sigma_f, double* w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n.nb) return;
  const int orr = 2 * n.nl + n.npq, nb = n.nb;
  double kQ = 0, kP = 0, dv = 0, dpp = 0;
  if (n.type[i] == REF) {
    kQ = om[orr + 1];
    kP = om[orr] + 2.0 * sigma_f * n.c2[n.gen_at[i]];
  } else if (n.type[i] == PV) {
    kQ = om[orr + 2 + n.pvpos[i]];
    dpp = 2.0 * sigma_f * n.c2[n.gen_at[i]];
  } else {
    dv = om[2 * n.nl + n.pqpos[i]];
  }
  w[i] = kQ;
  w[nb + i] = kP;
  w[2 * nb + i] = dv;
  w[3 * nb + i] = dpp;
}

// Rows 4..7 of the bus weights: dQ_i/dv_i, dQ_i/dtheta_i, dP_i/dv_i, dP_i/dtheta_i
// (sums over the incident branch ends, from the branch table), and the
// per-adjacency coefficient records of the HVP gathers.
__global__ void bus_self_grad_kernel(DevNet n, const double* tab, double* w, double* adjE, double* busS) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n.nb) return;
  const int nl = n.nl, nb = n.nb;
  double qv = 0, qt = 0, pv = 0, pt = 0, svv = w[2 * nb + i], svt = 0, stt = 0;
  for (int q = n.adj_ptr[i]; q < n.adj_ptr[i + 1]; q++) {
    const int e = n.adj[q], l = e >> 1, s = e & 1, o = 1 - s;
    const double qss = tab[(size_t)TAB_DQ(s, s) * nl + l], qst = tab[(size_t)TAB_DQ(s, 2 + s) * nl + l];
    const double pss = tab[(size_t)TAB_DP(s, s) * nl + l], pst = tab[(size_t)TAB_DP(s, 2 + s) * nl + l];
    qv += qss;
    qt += qst;
    pv += pss;
    pt += pst;
    double E[ADJ_W];
    E[E_VV] = tab[(size_t)pk(s, s) * nl + l];
    E[E_VO] = tab[(size_t)pk(s, o) * nl + l];
    E[E_VT] = tab[(size_t)pk(s, 2 + s) * nl + l];
    E[E_TO] = tab[(size_t)pk(2 + s, o) * nl + l];
    E[E_TT] = tab[(size_t)pk(2 + s, 2 + s) * nl + l];
    E[E_QOV] = tab[(size_t)TAB_DQ(o, s) * nl + l];
    E[E_QOT] = tab[(size_t)TAB_DQ(o, 2 + s) * nl + l];
    E[E_POV] = tab[(size_t)TAB_DP(o, s) * nl + l];
    E[E_POT] = tab[(size_t)TAB_DP(o, 2 + s) * nl + l];
    E[E_QSV] = qss;
    E[E_QSO] = tab[(size_t)TAB_DQ(s, o) * nl + l];
    E[E_QST] = qst;
    E[E_PSV] = pss;
    E[E_PSO] = tab[(size_t)TAB_DP(s, o) * nl + l];
    E[E_PST] = pst;
    E[15] = 0.0;
    svv += E[E_VV];
    svt += E[E_VT];
    stt += E[E_TT];
    double2* dst = reinterpret_cast<double2*>(adjE + (size_t)q * ADJ_W);
#pragma unroll
    for (int k = 0; k < ADJ_W / 2; k++) dst[k] = make_double2(E[2 * k], E[2 * k + 1]);
  }
  w[4 * nb + i] = qv;
  w[5 * nb + i] = qt;
  w[6 * nb + i] = pv;
  w[7 * nb + i] = pt;
  reinterpret_cast<double4_32a*>(busS)[i] = make_double4_32a(svv, svt, stt, 0.0);
}

// ------------------------------------------------------------ HVP tiles



// Value of a direction slot (see DevNet::busrec) in column c (control j).
template <int C>
__device__ __forceinline__ double dslot(const double* Z, int z, int c, int j) {
  return z >= 0 ? Z[(size_t)z * C + c] : ((-2 - z) == j ? 1.0 : 0.0);
}

// N incident branch ends qb .. qb + N - 1 of a bus in the second-order gather:
// the other ends' terms of y = (grad^2 l)(z; w) (see hvp_tile, phase 4).  The
// callers split a bus's ends into groups of 4, 2 and 1, so no FP64 instruction
// is issued for an absent end.
template <int C, int N>
__device__ __forceinline__ void gather_ends(const DevNet& n, const double* Z, const double* __restrict__ E,
                                            const double* QD, const double* PD, int qb, int c, int j,
                                            double& yv, double& yt) {
  int4 ar[N];
  double vo[N], to[N];
#pragma unroll
  for (int u = 0; u < N; u++) ar[u] = n.adjrec[qb + u];
#pragma unroll
  for (int u = 0; u < N; u++) {
    vo[u] = dslot<C>(Z, ar[u].x, c, j);
    to[u] = ar[u].y >= 0 ? Z[(size_t)ar[u].y * C + c] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < N; u++) {
    const double2* e2 = reinterpret_cast<const double2*>(E + (size_t)(qb + u) * ADJ_W);
    const double2 e01 = e2[0], e23 = e2[1];  // (VO, VT), (TO, TT)
    yv = fma(e01.x, vo[u], fma(-e01.y, to[u], yv));  // chained FMAs, no DMUL/DADD
    yt = fma(e23.x, vo[u], fma(-e23.y, to[u], yt));
    if (ar[u].z >= 0) {  // Gauss-Newton terms of the other end's Q (and P at the slack)
      const double w = QD[(size_t)ar[u].z * C + c];
      const double2 e45 = e2[2];  // (QOV, QOT)
      yv += w * e45.x;
      yt += w * e45.y;
      if (ar[u].w) {
        const double w2 = PD[c];
        const double2 e67 = e2[3];  // (POV, POT)
        yv += w2 * e67.x;
        yt += w2 * e67.y;
      }
    }
  }
}

// N ends of a control bus for its Q (and, at the slack, P) directional
// derivatives (hvp_tile, phase 3); groups of 4, 2 and 1 as in gather_ends.
template <int C, int N>
__device__ __forceinline__ void qd_ends(const DevNet& n, const double* Z, const double* __restrict__ E, int qb,
                                        int c, int j, bool slack, double& qd, double& pdr) {
  int4 ar[N];
  double vo[N], to[N];
#pragma unroll
  for (int u = 0; u < N; u++) ar[u] = n.adjrec[qb + u];
#pragma unroll
  for (int u = 0; u < N; u++) {
    vo[u] = dslot<C>(Z, ar[u].x, c, j);
    to[u] = ar[u].y >= 0 ? Z[(size_t)ar[u].y * C + c] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < N; u++) {
    const double* e = E + (size_t)(qb + u) * ADJ_W;
    qd = fma(e[E_QSO], vo[u], fma(-e[E_QST], to[u], qd));  // chained FMAs, no DMUL/DADD
    if (slack) pdr = fma(e[E_PSO], vo[u], fma(-e[E_PST], to[u], pdr));
  }
}

// N ends of a control bus in H[:, tile] += G_u^T Psi (hvp_tile, phase 7).
template <int C, int N>
__device__ __forceinline__ void gu_ends(const DevNet& n, const double* R, const double* __restrict__ E, int qb,
                                        int c, double& gv) {
  int4 ar[N];
  double pt[N], pv[N];
#pragma unroll
  for (int u = 0; u < N; u++) ar[u] = n.adjrec[qb + u];
#pragma unroll
  for (int u = 0; u < N; u++) {
    pt[u] = ar[u].y >= 0 ? R[(size_t)ar[u].y * C + c] : 0.0;
    pv[u] = ar[u].x >= 0 ? R[(size_t)ar[u].x * C + c] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < N; u++) {
    const double* e = E + (size_t)(qb + u) * ADJ_W;
    gv = fma(pt[u], e[E_POV], fma(pv[u], e[E_QOV], gv));
  }
}

// One tile of C Hessian columns on one CTA: B = -G_u W, Z = G_x^{-1} B,
// second-order terms, Psi = G_x^{-T} R, H[:, tile] = T + G_u^T Psi (Prop. 2).
// Z is the CTA's workspace (2 n_x C + n_ctrl C + C doubles).
// Phase stamps of one tile (a.stamps non-null only in a profiling call): the
// global nanosecond timer at the tile's start and after phases (1), (2), (4),
// (6) and (7), read by thread 0 after the phase's last barrier.
__device__ __forceinline__ void hvp_stamp(const HvpArgs& a, int tile, int k) {
  if (a.stamps && threadIdx.x == 0) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    a.stamps[(size_t)tile * 8 + k] = t;
  }
}

// ZR: the slab already holds the tile's first adjoint (HvpArgs::zreuse; a
// separate instantiation, so the ordinary tile keeps its code unchanged)
template <int C, bool ZR = false>
__device__ __forceinline__ void hvp_tile(const HvpArgs& a, double* Z, int tile) {
  hvp_stamp(a, tile, 0);
  const DevNet& n = a.n;
  const int nb = n.nb, nu = n.nu;
  double* R = Z + (size_t)n.nx * C;
  double* QD = R + (size_t)n.nx * C;
  double* PD = QD + (size_t)n.ngn * C;
  const double* __restrict__ E = a.adjE;
  const double* __restrict__ bw = a.busw;
  // reach of the first triangular solve (dynamic shared memory): values of the
  // reached rows, bit mask over the rows below the trailing block with the
  // per-word prefix counts (the rank of a reached row), reached rows ascending
  extern __shared__ __align__(16) unsigned char hvp_dyn[];
  double* s_zs = reinterpret_cast<double*>(hvp_dyn);
  unsigned* s_mask = reinterpret_cast<unsigned*>(s_zs + (size_t)a.zs_cap * C);
  int* s_pre = reinterpret_cast<int*>(s_mask + a.rm_words);
  int* s_list = s_pre + a.rm_words;
  // the values region, free outside the first solve's reach phase, serves the
  // sweeps' dense trailing triangles
  double* s_tb = a.zs_cap >= n.nroot ? s_zs : nullptr;
  __shared__ int s_col[32];
  __shared__ int s_nl;
  __shared__ int s_qstart;
  __shared__ double s_part[2][16][32];  // per-warp partial row sums (<= 512 threads)
  const int r0 = n.r0, nwords = (r0 + 31) >> 5;
  const bool prune = nwords <= a.rm_words;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  {
    // column of each lane of the tile (NOCOL past the requested range)
    constexpr int NOCOL = -(1 << 30);
    if (threadIdx.x < C) {
      if (a.colmap) {
        const int j = a.colmap[tile * C + threadIdx.x];
        s_col[threadIdx.x] = j < 0 ? NOCOL : j;
      } else {
        const int pos = a.col0 + tile * C + threadIdx.x;
        s_col[threadIdx.x] = pos >= a.col_end ? NOCOL : pos;
      }
    }
    if (ZR) {  // the slab holds this tile's first adjoint from the previous launch
      __syncthreads();
      hvp_stamp(a, tile, 1);
      hvp_stamp(a, tile, 2);
    } else {
      // (0) right-hand side B = -G_u W, W = unit directions of the tile's columns:
      // first the rows it touches (marked), then, once the first solve's reach is
      // known, the slab is cleared on the reached rows and the trailing block only
      // (the U sweep starts the other rows from zero through the mask, so the slab
      // is neither cleared nor read there), then the values
      if (prune)
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) s_mask[w] = 0u;
      __syncthreads();
      auto rhs = [&](bool values) {
        // Z[r][c] = v (set) or -= v; without values, mark row r
        auto put = [&](int r, int c, double v, bool set) {
          if (values) {
            double& z = Z[(size_t)r * C + c];
            z = set ? v : z - v;
          } else if (prune && r < r0) {
            atomicOr(&s_mask[r >> 5], 1u << (r & 31));
          }
        };
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
          const int j = s_col[c];
          if (j < 0) continue;
          const int k = a.ubus[j];
          if (j >= 1 + n.npv) {  // p of a PV unit: dg/dp = -e_{P_k}
            put(n.pth[k], c, 1.0, true);
            continue;
          }
          for (int q = n.adj_ptr[k]; q < n.adj_ptr[k + 1]; q++) {
            const int4 ar = n.adjrec[q];
            if (ar.y >= 0) put(ar.y, c, values ? E[(size_t)q * ADJ_W + E_POV] : 0.0, false);
            if (ar.x >= 0) put(ar.x, c, values ? E[(size_t)q * ADJ_W + E_QOV] : 0.0, false);
          }
          if (n.type[k] == PV) put(n.pth[k], c, values ? bw[6 * nb + k] : 0.0, false);
        }
      };
      rhs(false);
      __syncthreads();
      // (1) Z = L^{-1} B.  The solution is nonzero only on the elimination-tree
      // ancestors of the right-hand side's rows: mark them, list them in
      // ascending order, and let one warp solve those rows one after another
      // (no block-wide barrier); the trailing block follows as usual.
      int nl = a.list_cap + 1;
      if (prune) {
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
          unsigned bits = s_mask[w];
          while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            int x = n.eparent[w * 32 + b];
            while (x >= 0 && x < r0) {  // parents increase: the walk ends
              const unsigned m = 1u << (x & 31);
              if (atomicOr(&s_mask[x >> 5], m) & m) break;  // the row's walk is someone else's
              x = n.eparent[x];
            }
          }
        }
        __syncthreads();
        if (warp == 0) {
          int base = 0;
          for (int w0 = 0; w0 < nwords; w0 += 32) {
            const int w = w0 + lane;
            const unsigned bits = w < nwords ? s_mask[w] : 0u;
            const int cnt = __popc(bits);
            int incl = cnt;
  #pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
              const int y = __shfl_up_sync(0xffffffffu, incl, off);
              if (lane >= off) incl += y;
            }
            int pos = base + incl - cnt;
            if (w < nwords) s_pre[w] = pos;
            unsigned bb = bits;
            while (bb) {
              const int b = __ffs(bb) - 1;
              bb &= bb - 1;
              if (pos < a.list_cap) s_list[pos] = w * 32 + b;
              pos++;
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
          }
          if (lane == 0) s_nl = base;
        }
        __syncthreads();
        nl = s_nl;
      }
      const bool reach = nl <= a.list_cap;  // the first solve and the U sweep see the reach only
      if (reach) {
        for (int idx = threadIdx.x; idx < nl * C; idx += blockDim.x) Z[(size_t)s_list[idx / C] * C + idx % C] = 0.0;
        for (size_t k = (size_t)r0 * C + threadIdx.x; k < (size_t)n.nx * C; k += blockDim.x) Z[k] = 0.0;
      } else {
        for (size_t k = threadIdx.x; k < (size_t)n.nx * C; k += blockDim.x) Z[k] = 0.0;
      }
      __syncthreads();
      rhs(true);
      __syncthreads();
      const int ngrp = blockDim.x / C, g = threadIdx.x / C, nwarp = blockDim.x >> 5;
      const double* __restrict__ Vl = a.LU;
      if (nl <= a.zs_cap) {
        // right-looking over the reached rows with their values in shared
        // memory: once row t is final, every lane group subtracts its column's
        // multiples from the later reached rows (all reached: ancestors of t),
        // one barrier per row; rows of the trailing block are left to it.
        const int col = threadIdx.x % C;
        for (int idx = threadIdx.x; idx < nl * C; idx += blockDim.x)
          s_zs[idx] = Z[(size_t)s_list[idx / C] * C + idx % C];
        int e0 = 0, e1 = 0;
        if (nl > 0) {
          e0 = n.lcol_ptr[s_list[0]];
          e1 = n.lcol_ptr[s_list[0] + 1];
        }
        __syncthreads();
        for (int t = 0; t < nl; t++) {
          int en0 = 0, en1 = 0;
          if (t + 1 < nl) {  // the next column's extent, in flight during this one
            const int in = s_list[t + 1];
            en0 = n.lcol_ptr[in];
            en1 = n.lcol_ptr[in + 1];
          }
          const double xt = s_zs[(size_t)t * C + col];
          for (int e = e0 + g; e < e1; e += ngrp) {
            const int2 rq = __ldg(n.lcol + e);
            if (rq.x < r0) {
              const int w = rq.x >> 5;
              const unsigned m = s_mask[w];
              const int pos = s_pre[w] + __popc(m & ((1u << (rq.x & 31)) - 1u));
              s_zs[(size_t)pos * C + col] -= Vl[rq.y] * xt;
            }
          }
          e0 = en0;
          e1 = en1;
          __syncthreads();
        }
        for (int idx = threadIdx.x; idx < nl * C; idx += blockDim.x)
          Z[(size_t)s_list[idx / C] * C + idx % C] = s_zs[idx];
      }
      if (nl > a.zs_cap && nl <= a.list_cap) {
        // the same with the reached values in the slab
        const int col = threadIdx.x % C;
        const double* __restrict__ V = Vl;
        int pn0 = 0, pn1 = 0;
        if (nl > 0) {
          pn0 = n.rp[s_list[0]];
          pn1 = n.dp[s_list[0]];
        }
        for (int t = 0; t < nl; t++) {
          const int i = s_list[t], p0 = pn0, p1 = pn1;
          if (t + 1 < nl) {  // the next row's extent, in flight during this row
            pn0 = n.rp[s_list[t + 1]];
            pn1 = n.dp[s_list[t + 1]];
          }
          double v0 = 0.0, v1 = 0.0;
          int p = p0 + g;
          for (; p + ngrp < p1; p += 2 * ngrp) {
            const int c0 = __ldg(n.ci + p), c1 = __ldg(n.ci + p + ngrp);
            const bool b0 = (s_mask[c0 >> 5] >> (c0 & 31)) & 1u, b1 = (s_mask[c1 >> 5] >> (c1 & 31)) & 1u;
            if (b0) v0 -= V[p] * Z[(size_t)c0 * C + col];
            if (b1) v1 -= V[p + ngrp] * Z[(size_t)c1 * C + col];
          }
          if (p < p1) {
            const int c0 = __ldg(n.ci + p);
            if ((s_mask[c0 >> 5] >> (c0 & 31)) & 1u) v0 -= V[p] * Z[(size_t)c0 * C + col];
          }
          double v = v0 + v1;
  #pragma unroll
          for (int off = C; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          if (lane < C) s_part[t & 1][warp][lane] = v;
          // the row's right-hand side, read before any warp overwrites it
          const double zi = lane < C ? Z[(size_t)i * C + lane] : 0.0;
          __syncthreads();
          if (lane < C) {
            double sum = zi;
            for (int w = 0; w < nwarp; w++) sum += s_part[t & 1][w][lane];
            Z[(size_t)i * C + lane] = sum;
          }
          __syncwarp();
        }
      }
      if (nl <= a.list_cap) {
        __syncthreads();
        sweep<C, true, false>(n, a.LU, a.invdiag, Z, s_mask, s_tb);
      } else {
        sweep<C, true, false>(n, a.LU, a.invdiag, Z, nullptr, s_tb);
      }
      hvp_stamp(a, tile, 1);
      // (2) U sweep
      sweep<C, false, true>(n, a.LU, a.invdiag, Z, nullptr, s_tb, nullptr, reach ? s_mask : nullptr);
      hvp_stamp(a, tile, 2);
    }
    // (2b) on request, the reduced constraint Jacobian of the tile's columns,
    // J W = d_x c Z + d_u c W (Sec. III-B), from the first adjoint Z just
    // computed: the |S|^2 rows of both branch ends and the PQ voltages here,
    // the generator P/Q rows in phase (3), which forms their directional
    // derivatives anyway.  Column fastest: the C lanes of a slab row read one
    // contiguous segment, and a warp's 32 / C consecutive branches give each
    // column one contiguous run of J.
    if (a.J) {
      const int nl = n.nl, m = n.m;
      for (int it = threadIdx.x; it < nl * C; it += blockDim.x) {
        const int l = it / C, c = it % C, j = s_col[c];
        if (j < 0) continue;
        const int4 bf = n.busrec[n.f[l]], bt = n.busrec[n.t[l]];
        // branch-local direction (v_f, v_t, theta_f, theta_t)
        const double d[4] = {dslot<C>(Z, bf.x, c, j), dslot<C>(Z, bt.x, c, j),
                             bf.y >= 0 ? Z[(size_t)bf.y * C + c] : 0.0, bt.y >= 0 ? Z[(size_t)bt.y * C + c] : 0.0};
        double* Jc = a.J + (size_t)j * m;
#pragma unroll
        for (int s = 0; s < 2; s++) {  // d|S_s|^2 . d, the end's gradient from the branch table
          double v = 0.0;
#pragma unroll
          for (int k = 0; k < 4; k++) v = fma(a.tab[(size_t)TAB_DS(s, k) * nl + l], d[k], v);
          Jc[(size_t)s * nl + l] = v;
        }
      }
      for (int it = threadIdx.x; it < nb * C; it += blockDim.x) {
        const int i = it / C, c = it % C, j = s_col[c];
        if (j < 0 || n.type[i] != PQ) continue;
        a.J[(size_t)j * m + 2 * nl + n.pqpos[i]] = Z[(size_t)n.busrec[i].x * C + c];
      }
    }
    // (3) directional derivatives of Q (slack and PV) and P (slack) for the
    // Gauss-Newton terms, stored pre-multiplied by their weights kQ, kP.  The
    // own-variable parts are the per-bus sums dQ_k/dv_k, dQ_k/dtheta_k, ...
    for (int it = threadIdx.x; it < n.ngn * C; it += blockDim.x) {  // buses by descending degree
      const int gi = n.gn_by_deg[it / C], c = it % C, k = n.gn_bus[gi], j = s_col[c];
      const int4 bk = n.busrec[k];
      const double vk = dslot<C>(Z, bk.x, c, j), tk = bk.y >= 0 ? Z[(size_t)bk.y * C + c] : 0.0;
      const bool slack = (k == n.ref);
      double qd = bw[4 * nb + k] * vk + bw[5 * nb + k] * tk, pdr = 0.0;
      if (slack) pdr = bw[6 * nb + k] * vk + bw[7 * nb + k] * tk;
      const int q1 = n.adj_ptr[k + 1];
      int qb = n.adj_ptr[k];
      for (; qb + 4 <= q1; qb += 4) qd_ends<C, 4>(n, Z, E, qb, c, j, slack, qd, pdr);
      if (qb + 2 <= q1) {
        qd_ends<C, 2>(n, Z, E, qb, c, j, slack, qd, pdr);
        qb += 2;
      }
      if (qb < q1) qd_ends<C, 1>(n, Z, E, qb, c, j, slack, qd, pdr);
      QD[(size_t)gi * C + c] = bw[k] * qd;
      if (slack) PD[c] = bw[nb + k] * pdr;
      if (a.J && j >= 0) {  // generator rows of J: p_ref, q_ref, q of a PV unit
        double* Jc = a.J + (size_t)j * n.m + 2 * n.nl + n.npq;
        if (slack) {
          Jc[0] = pdr;
          Jc[1] = qd;
        } else {
          Jc[2 + n.pvpos[k]] = qd;
        }
      }
    }
    __syncthreads();
    if (a.jac_only) {
      hvp_stamp(a, tile, 3);
      hvp_stamp(a, tile, 4);
      hvp_stamp(a, tile, 5);
      return;
    }
    // (4) y = (grad^2 l) (z; w) per bus; R = -y_x, H[u rows] = y_u.  The
    // own-variable coefficients are summed per bus (busS), so an incident
    // branch adds only its other end's terms.  Buses are taken by descending
    // degree, so the buses sharing a warp loop over the same number of entries.
    // The bus's static records (its slots, coefficients, entry range) are read
    // one item ahead, so an item waits for the slab only.
    const int nitem = nb * C;
    int i_n = 0, q0_n = 0, q1_n = 0;
    int4 bi_n = make_int4(-1, -1, -1, -1);
    double4_32a S_n = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    if ((int)threadIdx.x < nitem) {
      i_n = n.bus_by_deg[threadIdx.x / C];
      bi_n = n.busrec[i_n];
      S_n = reinterpret_cast<const double4_32a*>(a.busS)[i_n];
      q0_n = n.adj_ptr[i_n];
      q1_n = n.adj_ptr[i_n + 1];
    }
    for (int it = threadIdx.x; it < nitem; it += blockDim.x) {
      const int i = i_n, c = it % C, j = s_col[c];
      const int4 bi = bi_n;
      const double4_32a S = S_n;
      const int q1 = q1_n;
      int qb = q0_n;
      if (it + (int)blockDim.x < nitem) {
        i_n = n.bus_by_deg[(it + blockDim.x) / C];
        bi_n = n.busrec[i_n];
        S_n = reinterpret_cast<const double4_32a*>(a.busS)[i_n];
        q0_n = n.adj_ptr[i_n];
        q1_n = n.adj_ptr[i_n + 1];
      }
      const double vi = dslot<C>(Z, bi.x, c, j), ti = bi.y >= 0 ? Z[(size_t)bi.y * C + c] : 0.0;
      double yv = S.x * vi + S.y * ti, yt = S.y * vi + S.z * ti;
      for (; qb + 4 <= q1; qb += 4) gather_ends<C, 4>(n, Z, E, QD, PD, qb, c, j, yv, yt);
      if (qb + 2 <= q1) {
        gather_ends<C, 2>(n, Z, E, QD, PD, qb, c, j, yv, yt);
        qb += 2;
      }
      if (qb < q1) gather_ends<C, 1>(n, Z, E, QD, PD, qb, c, j, yv, yt);
      if (bi.z >= 0) {  // own injections: the gradients dQ_i, dP_i w.r.t. (v_i, theta_i) are per-bus sums
        const double w = QD[(size_t)bi.z * C + c];
        yv += w * bw[4 * nb + i];
        yt += w * bw[5 * nb + i];
        if (bi.y < 0) {
          const double w2 = PD[c];
          yv += w2 * bw[6 * nb + i];
          yt += w2 * bw[7 * nb + i];
        }
      }
      if (bi.y >= 0) R[(size_t)bi.y * C + c] = -yt;
      if (bi.x >= 0) {
        R[(size_t)bi.x * C + c] = -yv;
      } else if (j >= 0) {
        double* Hc = a.H + (size_t)j * nu;
        Hc[-2 - bi.x] = yv;
        if (bi.w >= 0) Hc[bi.w] = (bi.w == j) ? bw[3 * nb + i] : 0.0;
      }
    }
    __syncthreads();
    hvp_stamp(a, tile, 3);
    // symmetric Hessian: the tile's first column position qs; the tile keeps the
    // rows of the controls at positions >= qs, so Psi is needed on the blocks
    // whose lt_q >= qs only, a prefix of each level of the L^T ordering (its
    // length by binary search, one level per thread, into the reach prefix
    // words, free since phase (1))
    const int* lcnt = nullptr;
    int qs = 0;
    if (a.sym) {
      if (threadIdx.x == 0) {
        int q = 1 << 30;
        for (int c = 0; c < C; c++)
          if (s_col[c] >= 0) q = min(q, n.qpos[s_col[c]]);
        s_qstart = q;
      }
      __syncthreads();
      qs = s_qstart;
      if (n.nblev_b <= a.rm_words) {
        for (int lv = threadIdx.x; lv < n.nblev_b; lv += blockDim.x) {
          const int base = n.bptr_b[lv];
          int lo = base, hi = n.bptr_b[lv + 1];
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(n.lt_q + mid) >= qs)
              lo = mid + 1;
            else
              hi = mid;
          }
          s_pre[lv] = lo - base;
        }
        lcnt = s_pre;  // read after the U^T sweep's barriers
      }
      if ((int)threadIdx.x < C && s_col[threadIdx.x] >= 0) a.tstart[s_col[threadIdx.x]] = qs;
    }
    // (5)-(6) second second-order adjoint: U^T then L^T sweeps
    sweep<C, true, true>(n, a.T, a.invdiag, R, nullptr, s_tb);
    sweep<C, false, false>(n, a.T, a.invdiag, R, nullptr, s_tb, lcnt);
    hvp_stamp(a, tile, 4);
    // (7) H[:, tile] += G_u^T Psi (buses by descending degree)
    for (int it = threadIdx.x; it < n.ngn * C; it += blockDim.x) {
      const int gi = n.gn_by_deg[it / C], c = it % C, k = n.gn_bus[gi], j = s_col[c];
      if (j < 0) continue;
      const int4 bk = n.busrec[k];
      if (a.sym && n.qpos[-2 - bk.x] < qs && (bk.w < 0 || n.qpos[bk.w] < qs)) continue;  // rows mirrored
      double gv = 0.0;
      const int q1 = n.adj_ptr[k + 1];
      int qb = n.adj_ptr[k];
      for (; qb + 4 <= q1; qb += 4) gu_ends<C, 4>(n, R, E, qb, c, gv);
      if (qb + 2 <= q1) {
        gu_ends<C, 2>(n, R, E, qb, c, gv);
        qb += 2;
      }
      if (qb < q1) gu_ends<C, 1>(n, R, E, qb, c, gv);
      double* Hc = a.H + (size_t)j * nu;
      if (bk.w >= 0) {  // PV bus
        const double psi = R[(size_t)bk.y * C + c];
        gv += psi * bw[6 * nb + k];
        Hc[bk.w] -= psi;
      }
      Hc[-2 - bk.x] += gv;
    }
    __syncthreads();
    hvp_stamp(a, tile, 5);
  }
}

template <int C, int NT>
__global__ void __launch_bounds__(NT) hvp_tile_kernel(HvpArgs a) {
  double* Z = a.scratch + a.stride * blockIdx.x;
  for (int tile = a.first_tile + blockIdx.x * a.tile_step; tile < a.ntiles; tile += gridDim.x * a.tile_step)
    hvp_tile<C>(a, Z, tile);
}

// Split tiling: a1.ntiles tiles of width C and a2.ntiles of width C / 2 (each
// part with its own column map and workspace), one per CTA, all CTAs resident.
// The hardware's CTA-to-SM placement is not round robin (some SMs were given
// three of the first CTAs), so a CTA takes its tile by its rank on its SM: the
// first per_sm CTAs of an SM take a wide tile, the others a narrow one (an
// exhausted queue sends the CTA to the other).  The wide queue is ordered
// heaviest first; a CTA of even rank takes the heaviest remaining tile and one
// of odd rank the lightest, so the two wide tiles of an SM sum to about the
// mean (an SM's CTAs start together, in no fixed order across SMs).
// ctr: [0] wide claims, [1] narrow queue, [2] heavy end, [3] light end,
// [4 + smid] CTAs seen per SM; zero before the launch.
template <int C, int NT, bool ZR = false>
__global__ void __launch_bounds__(NT, 3) hvp_split_kernel(HvpArgs a1, HvpArgs a2, int per_sm, int* ctr) {
  __shared__ int s_pick;
  if (threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const int rank = smid < (unsigned)kSplitMaxSm ? atomicAdd(ctr + 4 + smid, 1) : 0;
    auto wide = [&]() -> int {  // a wide tile, or -1 when all are taken
      if (atomicAdd(ctr, 1) >= a1.ntiles) return -1;
      return (rank & 1) ? a1.ntiles - 1 - atomicAdd(ctr + 3, 1) : atomicAdd(ctr + 2, 1);
    };
    int kind = 1, t = -1;
    if (rank < per_sm) {
      t = wide();
      kind = 0;
    }
    if (t < 0) {
      kind = 1;
      t = atomicAdd(ctr + 1, 1);
      if (t >= a2.ntiles) {
        t = wide();
        kind = 0;
      }
    }
    s_pick = t < 0 ? -1 : ((t << 1) | kind);
  }
  __syncthreads();
  if (s_pick < 0) return;
  const int t = s_pick >> 1;
  if ((s_pick & 1) == 0) {
    if (t < a1.ntiles) hvp_tile<C, ZR>(a1, a1.scratch + a1.stride * t, t);
  } else {
    if (t < a2.ntiles) hvp_tile<C / 2, ZR>(a2, a2.scratch + a2.stride * t, t);
  }
}

// Persistent batched form: CTAs pull (context, tile) pairs from a queue (ordered
// largest network first) and run the same tile body with that context's
// arguments staged in shared memory.  No CTA waits on another.
template <int C>
__global__ void __launch_bounds__(256, 3) hvp_batch_kernel(const HvpArgs* __restrict__ args,
                                                        const int2* __restrict__ tiles, int ntot,
                                                        int* counter, double* scratch, size_t stride) {
  __shared__ HvpArgs sa;
  __shared__ int s_tile;
  double* Z = scratch + stride * blockIdx.x;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= ntot) break;
    const int2 ct = tiles[t];
    const int* src = reinterpret_cast<const int*>(args + ct.x);
    int* dst = reinterpret_cast<int*>(&sa);
    for (int k = threadIdx.x; k < (int)(sizeof(HvpArgs) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    hvp_tile<C>(sa, Z, ct.y);
  }
}

// ------------------------------------------------------------ plain form
// One Hessian column per launch sequence (the k = 1 baseline of the batched
// tiles, Sec. III-C computes the Hessian one HVP at a time in its plain form):
// the steps of hvp_tile with C = 1, each a device-wide launch, and the two
// solves on the streamed single-RHS sweeps (the library's fastest
// one-direction solve).  The solves take and return vectors in x order; the
// second-order gathers index pivot-order slots, so the vectors are permuted
// between them.

// B = -G_u e_j into the zeroed x-order vector bx (phase (0) of hvp_tile, one thread).
__global__ void plain_rhs_kernel(HvpArgs a, int j, double* bx) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const DevNet& n = a.n;
  const double* __restrict__ E = a.adjE;
  const int k = a.ubus[j];
  if (j >= 1 + n.npv) {  // p of a PV unit: dg/dp = -e_{P_k}
    bx[n.perm[n.pth[k]]] = 1.0;
    return;
  }
  for (int q = n.adj_ptr[k]; q < n.adj_ptr[k + 1]; q++) {
    const int4 ar = n.adjrec[q];
    if (ar.y >= 0) bx[n.perm[ar.y]] -= E[(size_t)q * ADJ_W + E_POV];
    if (ar.x >= 0) bx[n.perm[ar.x]] -= E[(size_t)q * ADJ_W + E_QOV];
  }
  if (n.type[k] == PV) bx[n.perm[n.pth[k]]] -= a.busw[6 * n.nb + k];
}

// to_pivot: dst[k] = src[perm[k]]; else dst[perm[k]] = src[k].
__global__ void plain_permute_kernel(const int* __restrict__ perm, const double* __restrict__ src,
                                     double* __restrict__ dst, int nx, int to_pivot) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nx; k += gridDim.x * blockDim.x) {
    if (to_pivot)
      dst[k] = src[perm[k]];
    else
      dst[perm[k]] = src[k];
  }
}

// Phase (3): directional derivatives of Q (and P at the slack) at the control buses.
__global__ void plain_qd_kernel(HvpArgs a, int j, const double* __restrict__ Z, double* QD, double* PD) {
  const DevNet& n = a.n;
  const int nb = n.nb;
  const double* __restrict__ E = a.adjE;
  const double* __restrict__ bw = a.busw;
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < n.ngn; gi += gridDim.x * blockDim.x) {
    const int k = n.gn_bus[gi];
    const int4 bk = n.busrec[k];
    const double vk = dslot<1>(Z, bk.x, 0, j), tk = bk.y >= 0 ? Z[bk.y] : 0.0;
    const bool slack = (k == n.ref);
    double qd = bw[4 * nb + k] * vk + bw[5 * nb + k] * tk, pdr = 0.0;
    if (slack) pdr = bw[6 * nb + k] * vk + bw[7 * nb + k] * tk;
    const int q1 = n.adj_ptr[k + 1];
    int qb = n.adj_ptr[k];
    for (; qb + 4 <= q1; qb += 4) qd_ends<1, 4>(n, Z, E, qb, 0, j, slack, qd, pdr);
    if (qb + 2 <= q1) {
      qd_ends<1, 2>(n, Z, E, qb, 0, j, slack, qd, pdr);
      qb += 2;
    }
    if (qb < q1) qd_ends<1, 1>(n, Z, E, qb, 0, j, slack, qd, pdr);
    QD[gi] = bw[k] * qd;
    if (slack) PD[0] = bw[nb + k] * pdr;
  }
}

// Phase (4): y = (grad^2 l)(z; w) per bus; R = -y_x (pivot order), H[u rows, j] = y_u.
__global__ void plain_gather_kernel(HvpArgs a, int j, const double* __restrict__ Z, const double* __restrict__ QD,
                                    const double* __restrict__ PD, double* R) {
  const DevNet& n = a.n;
  const int nb = n.nb;
  const double* __restrict__ E = a.adjE;
  const double* __restrict__ bw = a.busw;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
    const int4 bi = n.busrec[i];
    const double4_32a S = reinterpret_cast<const double4_32a*>(a.busS)[i];
    const double vi = dslot<1>(Z, bi.x, 0, j), ti = bi.y >= 0 ? Z[bi.y] : 0.0;
    double yv = S.x * vi + S.y * ti, yt = S.y * vi + S.z * ti;
    const int q1 = n.adj_ptr[i + 1];
    int qb = n.adj_ptr[i];
    for (; qb + 4 <= q1; qb += 4) gather_ends<1, 4>(n, Z, E, QD, PD, qb, 0, j, yv, yt);
    if (qb + 2 <= q1) {
      gather_ends<1, 2>(n, Z, E, QD, PD, qb, 0, j, yv, yt);
      qb += 2;
    }
    if (qb < q1) gather_ends<1, 1>(n, Z, E, QD, PD, qb, 0, j, yv, yt);
    if (bi.z >= 0) {
      const double w = QD[bi.z];
      yv += w * bw[4 * nb + i];
      yt += w * bw[5 * nb + i];
      if (bi.y < 0) {
        const double w2 = PD[0];
        yv += w2 * bw[6 * nb + i];
        yt += w2 * bw[7 * nb + i];
      }
    }
    if (bi.y >= 0) R[bi.y] = -yt;
    if (bi.x >= 0) {
      R[bi.x] = -yv;
    } else {
      double* Hc = a.H + (size_t)j * n.nu;
      Hc[-2 - bi.x] = yv;
      if (bi.w >= 0) Hc[bi.w] = (bi.w == j) ? bw[3 * nb + i] : 0.0;
    }
  }
}

// Phase (7): H[:, j] += G_u^T Psi (Psi in pivot order).
__global__ void plain_assemble_kernel(HvpArgs a, int j, const double* __restrict__ Psi) {
  const DevNet& n = a.n;
  const int nb = n.nb;
  const double* __restrict__ E = a.adjE;
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < n.ngn; gi += gridDim.x * blockDim.x) {
    const int k = n.gn_bus[gi];
    double gv = 0.0;
    const int q1 = n.adj_ptr[k + 1];
    int qb = n.adj_ptr[k];
    for (; qb + 4 <= q1; qb += 4) gu_ends<1, 4>(n, Psi, E, qb, 0, gv);
    if (qb + 2 <= q1) {
      gu_ends<1, 2>(n, Psi, E, qb, 0, gv);
      qb += 2;
    }
    if (qb < q1) gu_ends<1, 1>(n, Psi, E, qb, 0, gv);
    double* Hc = a.H + (size_t)j * n.nu;
    const int4 bk = n.busrec[k];
    if (bk.w >= 0) {  // PV bus
      const double psi = Psi[bk.y];
      gv += psi * a.busw[6 * nb + k];
      Hc[bk.w] -= psi;
    }
    Hc[-2 - bk.x] += gv;
  }
}

// ------------------------------------------------------------ launchers

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

void launch_unpack(opf_ctx* c, const double* x, const double* u) {
  c->launches++;
  unpack_kernel<<<nblk(c->dn.nb, 256), 256, 0, c->stream>>>(c->dn, x, u, c->vbus, c->thbus);
}

void launch_pf_eval(opf_ctx* c) {
  c->launches += 2;
  pf_branch_kernel<<<nblk(c->dn.nl, 128), 128, 0, c->stream>>>(c->dn, c->vbus, c->thbus, c->endflow);
  pf_eval_kernel<<<nblk(c->dn.nb, 256), 256, 0, c->stream>>>(c->dn, c->vbus, c->thbus, c->u, c->pd,
                                                               c->qd, c->g, c->LU, c->scal, c->endflow);
}

void launch_lu_kernels(opf_ctx* c) {
  const int nlev = (int)c->h_task_ptr.size() - 1;  // block levels of the non-trailing columns
  // level lv's tasks with the finish records of level lv - 1; one more launch
  // finishes the last level
  const int lv_end = c->lu_dense_cluster > 0 ? c->lu_tail_from : nlev + 1;
  for (int lv = 0; lv < lv_end; lv++) {
    const int t0 = lv < nlev ? c->h_task_ptr[lv] : 0, t1 = lv < nlev ? c->h_task_ptr[lv + 1] : 0;
    const int f0 = lv > 0 ? c->h_fin_ptr[lv - 1] : 0, f1 = lv > 0 ? c->h_fin_ptr[lv] : 0;
    const int items = (t1 - t0) + (f1 - f0);
    if (items == 0) continue;
    const int G = lv < (int)c->h_lu_lanes.size() ? c->h_lu_lanes[lv] : 32;
    const int blocks = std::min(nblk(nblk(items, 32 / G), 8), 4 * c->sm_count);
    c->launches++;
    // programmatic dependent launch: the next level's grid starts while this
    // one drains and waits in-kernel (griddepcontrol.wait) for its results
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(256);
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, lu_level_kernel, c->LU, (const int4*)c->task_rec, (const int*)c->task_off,
                       (const int*)c->task_map, t0, t1, (const int4*)c->fin_rec, f0, f1, c->flags, G);
  }
  c->launches++;
  const size_t dense_smem = sizeof(double) * (size_t)c->dn.nroot * c->dn.nroot;
  const int use_smem = dense_smem <= (size_t)kDenseLuSmem ? 1 : 0;
  if (c->lu_dense_cluster > 0) {
    LuTail tail;
    tail.task_rec = c->task_rec;
    tail.task_off = c->task_off;
    tail.task_map = c->task_map;
    tail.fin_rec = c->fin_rec;
    tail.lvrec = c->lu_lvrec;
    tail.lanes = c->lu_lanes;
    tail.lv0 = lv_end;
    tail.lv1 = nlev + 1;
    launch_lu_dense_cluster(c->stream, c->lu_dense_cluster, c->LU, c->dn.dp, c->dn.r0, c->dn.nroot, c->flags,
                            tail);
  } else
    lu_dense_block_kernel<<<1, 1024, use_smem ? dense_smem : 0, c->stream>>>(c->LU, c->dn.dp, c->dn.r0,
                                                                          c->dn.nroot, c->flags, use_smem);
  c->launches++;
  lu_finish_kernel<<<2 * c->sm_count, 256, 0, c->stream>>>(c->LU, c->T, c->invdiag, c->tmap, c->dn.dp,
                                                           c->dn.nx, c->dn.nnz, c->flags);
  launch_sweep_pack(c);
}

void launch_lu(opf_ctx* c) {
  cudaGraphLaunch(c->lu_exec, c->stream);
  c->launches += c->lu_graph_kernels;
  c->lu_gen++;  // new factors: first adjoints kept in the Hessian scratch are void
}

void launch_solve1(opf_ctx* c, const double* b, double* out, bool transposed, double scale) {
  if (c->sw.ok) {
    launch_solve1_streamed(c, b, out, transposed, scale);
    return;
  }
  c->launches++;
  solve1_kernel<<<1, 512, c->solve1_smem, c->stream>>>(c->dn, c->LU, c->T, c->invdiag, b, out, c->yvec,
                                                        transposed ? 1 : 0, scale, c->solve1_use_smem_rhs ? 1 : 0);
}

opf_status setup_solve1(opf_ctx* c) {
  cudaFuncSetAttribute(lu_dense_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseLuSmem);
  const size_t tri = sizeof(double) * (size_t)c->dn.nroot * (c->dn.nroot - 1) / 2;
  const size_t full = tri + sizeof(double) * (size_t)c->dn.nx;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  const size_t cap = (size_t)optin - 1024;
  // the attribute is per kernel, shared by every context: raise it to the device maximum once
  if (cudaFuncSetAttribute(solve1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("cannot raise the shared-memory limit of the single-RHS sweep");
    return OPF_ECUDA;
  }
  if (tri > cap) {
    set_last_error("dense trailing block too large for the single-RHS sweep");
    return OPF_EINVAL;
  }
  c->solve1_use_smem_rhs = full <= cap;
  c->solve1_smem = (int)(c->solve1_use_smem_rhs ? full : tri);
  return OPF_OK;
}

void launch_axpy(opf_ctx* c, double* x, const double* d, double a, int n) {
  c->launches++;
  axpy_kernel<<<nblk(n, 256), 256, 0, c->stream>>>(x, d, a, n);
}

void launch_first_order(opf_ctx* c, const opf_al_params* p, double* grad_s) {
  const DevNet& n = c->dn;
  cudaMemsetAsync(c->scal, 0, 8 * sizeof(double), c->stream);
  launch_unpack(c, c->x, c->u);
  c->launches += 2;
  pf_branch_kernel<<<nblk(n.nl, 128), 128, 0, c->stream>>>(n, c->vbus, c->thbus, c->endflow);
  branch_flow_kernel<<<nblk(n.nl, 256), 256, 0, c->stream>>>(n, c->vbus, c->thbus, c->flows, c->cvec);
  c->launches++;
  bus_inj_kernel<<<nblk(n.nb, 256), 256, 0, c->stream>>>(n, c->vbus, c->flows, c->pd, c->qd, c->Pbus,
                                                         c->Qbus, c->cvec);
  const int mm = std::max(n.m, n.ng);
  c->launches++;
  al_weights_kernel<<<nblk(mm, 256), 256, 0, c->stream>>>(
      n, c->cvec, p->sigma_c, p->y, p->s, p->omega, p->rho, p->sigma_f, c->Pbus, c->u, c->pd,
      c->c0, c->phid, grad_s, c->omega, c->scal);
  c->launches++;
  dF_bus_kernel<<<nblk(n.nb, 256), 256, 0, c->stream>>>(n, c->u, c->phid, c->Pbus, c->pd, p->sigma_f, c->dFx,
                                                        c->dFu, c->endflow);
  launch_solve1(c, c->dFx, c->lam, true, -1.0);
}

// F alone at the context's state (flows, constraint values and the AL sums;
// no adjoint solve), into F_out (device).
void launch_eval_F(opf_ctx* c, const opf_al_params* p, double* F_out) {
  const DevNet& n = c->dn;
  cudaMemsetAsync(c->scal + 2, 0, sizeof(double), c->stream);
  launch_unpack(c, c->x, c->u);
  branch_flow_kernel<<<nblk(n.nl, 256), 256, 0, c->stream>>>(n, c->vbus, c->thbus, c->flows, c->cvec);
  bus_inj_kernel<<<nblk(n.nb, 256), 256, 0, c->stream>>>(n, c->vbus, c->flows, c->pd, c->qd, c->Pbus,
                                                         c->Qbus, c->cvec);
  const int mm = std::max(n.m, n.ng);
  al_weights_kernel<<<nblk(mm, 256), 256, 0, c->stream>>>(
      n, c->cvec, p->sigma_c, p->y, p->s, p->omega, p->rho, p->sigma_f, c->Pbus, c->u, c->pd,
      c->c0, c->phid, nullptr, c->omega, c->scal);
  c->launches += 3;
  cudaMemcpyAsync(F_out, c->scal + 2, sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
}

// (in buffers of its own: the first-order adjoint lambda of the last Hessian or
// gradient stays valid)
void launch_weighted_grad(opf_ctx* c, const double* w, double* out) {
  const DevNet& n = c->dn;
  c->launches++;
  dF_bus_kernel<<<nblk(n.nb, 256), 256, 0, c->stream>>>(n, c->u, w, c->Pbus, c->pd, 0.0, c->dFx_w, c->dFu_w,
                                                        c->endflow);
  // d_u + G_u^T lambda = d_u + Z^T d_x from the Hessian's slabs when they hold its first adjoints
  if (launch_adjoint_from_slabs(c, c->dFx_w, c->dFu_w, out)) return;
  launch_solve1(c, c->dFx_w, c->lam_w, true, -1.0);
  c->launches++;
  grad_u_kernel<<<nblk(n.ngn, 128), 128, 0, c->stream>>>(n, c->lam_w, c->dFu_w, out, c->endflow);
}

// omega (and phi', unchanged when the first-order weights are) of p at the
// state of the last launch_first_order: its flows, constraint values and lambda
// stay.
void launch_omega(opf_ctx* c, const opf_al_params* p) {
  const DevNet& n = c->dn;
  const int mm = std::max(n.m, n.ng);
  cudaMemsetAsync(c->scal, 0, 8 * sizeof(double), c->stream);
  al_weights_kernel<<<nblk(mm, 256), 256, 0, c->stream>>>(
      n, c->cvec, p->sigma_c, p->y, p->s, p->omega, p->rho, p->sigma_f, c->Pbus, c->u, c->pd,
      c->c0, c->phid, nullptr, c->omega, c->scal);
  c->launches++;
}

void launch_grad_u(opf_ctx* c, double* gu) {
  c->launches++;
  grad_u_kernel<<<nblk(c->dn.ngn, 128), 128, 0, c->stream>>>(c->dn, c->lam, c->dFu, gu, c->endflow);
}

void launch_grad_load(opf_ctx* c, double sigma_f, double* gpd, double* gqd) {
  c->launches++;
  grad_load_kernel<<<nblk(c->dn.nb, 256), 256, 0, c->stream>>>(c->dn, c->lam, c->phid, c->Pbus, c->pd,
                                                               sigma_f, gpd, gqd);
}

void launch_hess_prep(opf_ctx* c, double sigma_f) {
  const DevNet& n = c->dn;
  c->launches++;
  hess_prep_kernel<<<nblk(n.nl, 128), 128, 0, c->stream>>>(n, c->vbus, c->thbus, c->lam, c->phid,
                                                           c->omega, c->Pbus, c->pd, sigma_f, c->btab);
  c->launches++;
  bus_weight_kernel<<<nblk(n.nb, 256), 256, 0, c->stream>>>(n, c->omega, sigma_f, c->busw);
  c->launches++;
  bus_self_grad_kernel<<<nblk(n.nb, 256), 256, 0, c->stream>>>(n, c->btab, c->busw, c->adjE, c->busS);
}

// ------------------------------------------------------------ gradient scaling
// The scale of a row whose largest derivative is mx: g_max / mx when mx
// exceeds g_max (floored at s_min), else 1 (Sec. IV-A, "Scaling").
__device__ __forceinline__ double grad_scale(double mx, double g_max, double s_min) {
  return mx > g_max ? fmax(s_min, g_max / mx) : 1.0;
}

// sig[i] from max_j |J[j m + i]| (J column-major m x nu).  Block (32, 8): the
// x threads take 32 consecutive rows (one coalesced 256-byte load per column),
// the y threads every 8th column; the eight partial maxima meet in shared memory.
// With a prior scale p_i (prior non-null) the rule applies to the row as
// written, p_i dc_i/du, and the result is p_i times its scale.
__global__ void __launch_bounds__(256) jac_row_scale_kernel(const double* __restrict__ J, int m, int nu,
                                                          double g_max, double s_min,
                                                          const double* __restrict__ prior, double* sig) {
  __shared__ double part[8][32];
  const int i = blockIdx.x * 32 + threadIdx.x;
  double mx = 0.0;
  if (i < m)
    for (int j = threadIdx.y; j < nu; j += 8) mx = fmax(mx, fabs(J[(size_t)j * m + i]));
  part[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && i < m) {
#pragma unroll
    for (int y = 1; y < 8; y++) mx = fmax(mx, part[y][threadIdx.x]);
    const double p = prior ? prior[i] : 1.0;
    sig[i] = p * grad_scale(p * mx, g_max, s_min);
  }
}

// out[0] = the scale of max_i |g[i]| (one block).
__global__ void __launch_bounds__(256) vec_scale_kernel(const double* __restrict__ g, int n, double g_max,
                                                      double s_min, double* out) {
  __shared__ double part[8];
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(g[i]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) mx = fmax(mx, part[w]);
    out[0] = grad_scale(fmax(mx, part[0]), g_max, s_min);
  }
}

void launch_grad_scaling(opf_ctx* c, const double* J, const double* gf, double g_max, double s_min,
                         const double* prior, double* sigma_c, double* sigma_f) {
  const int m = c->h.m, nu = c->h.nu;
  if (m > 0) {
    jac_row_scale_kernel<<<(m + 31) / 32, dim3(32, 8), 0, c->stream>>>(J, m, nu, g_max, s_min, prior, sigma_c);
    c->launches++;
  }
  vec_scale_kernel<<<1, 256, 0, c->stream>>>(gf, nu, g_max, s_min, sigma_f);
  c->launches++;
}

size_t hvp_stride(const opf_ctx* c, int C) {
  size_t s = 2 * (size_t)c->dn.nx * C + (size_t)c->dn.ngn * C + C;
  return (s + 31) & ~(size_t)31;
}

template <int C>
static void launch_hvp_t(opf_ctx* c, double* H, int grid, int first_tile, int tile_step, int ntiles,
                         int col0, int col_end) {
  HvpArgs a = make_hvp_args(c, C, H, col0, col_end, true);
  a.scratch = c->scratch;
  a.ntiles = ntiles;
  a.first_tile = first_tile;
  a.tile_step = tile_step;
  c->z_gen = -1;  // CTAs reuse their slabs across tiles
  const size_t sm = hvp_smem_bytes(a, C);
  if (c->hvp_threads == 512)
    hvp_tile_kernel<C, 512><<<grid, 512, sm, c->stream>>>(a);
  else if (c->hvp_threads == 128)
    hvp_tile_kernel<C, 128><<<grid, 128, sm, c->stream>>>(a);
  else
    hvp_tile_kernel<C, 256><<<grid, 256, sm, c->stream>>>(a);
  c->launches++;
}

template <int C>
static int hvp_occ_t(int nt) {
  int occ = 0;
  if (nt == 512)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hvp_tile_kernel<C, 512>, 512, hvp_smem_budget(C));
  else if (nt == 128)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hvp_tile_kernel<C, 128>, 128, hvp_smem_budget(C));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hvp_tile_kernel<C, 256>, 256, hvp_smem_budget(C));
  return std::max(occ, 1);
}

int hvp_occupancy(int C, int nt) {
  switch (C) {
    case 1: return hvp_occ_t<1>(nt);
    case 2: return hvp_occ_t<2>(nt);
    case 4: return hvp_occ_t<4>(nt);
    case 8: return hvp_occ_t<8>(nt);
    case 16: return hvp_occ_t<16>(nt);
    default: return hvp_occ_t<32>(nt);
  }
}

bool launch_hvp(opf_ctx* c, int C, double* H, int grid, int first_tile, int tile_step, int ntiles,
                int col0, int col_end) {
  switch (C) {
    case 1: launch_hvp_t<1>(c, H, grid, first_tile, tile_step, ntiles, col0, col_end); return true;
    case 2: launch_hvp_t<2>(c, H, grid, first_tile, tile_step, ntiles, col0, col_end); return true;
    case 4: launch_hvp_t<4>(c, H, grid, first_tile, tile_step, ntiles, col0, col_end); return true;
    case 8: launch_hvp_t<8>(c, H, grid, first_tile, tile_step, ntiles, col0, col_end); return true;
    case 16: launch_hvp_t<16>(c, H, grid, first_tile, tile_step, ntiles, col0, col_end); return true;
    case 32: launch_hvp_t<32>(c, H, grid, first_tile, tile_step, ntiles, col0, col_end); return true;
    default: return false;
  }
}

HvpArgs make_hvp_args(opf_ctx* c, int C, double* H, int col0, int col_end, bool balanced) {
  HvpArgs a;
  a.n = c->dn;
  a.LU = c->LU;
  a.T = c->T;
  a.invdiag = c->invdiag;
  a.tab = c->btab;
  a.busw = c->busw;
  a.adjE = c->adjE;
  a.busS = c->busS;
  a.ubus = c->ubus;
  // the full Hessian is tiled in the elimination-tree order of the controls
  const bool full = (col0 == 0 && col_end == c->h.nu);
  int lk = 0;
  while ((1 << lk) < C) lk++;
  a.colmap = full ? c->colmap[balanced ? 1 : 0][lk] : nullptr;
  a.H = H;
  a.J = c->jac_out;
  a.jac_only = c->jac_only ? 1 : 0;
  a.scratch = nullptr;
  a.stamps = c->stamps_on ? c->stamps : nullptr;
  a.stride = hvp_stride(c, C);
  a.ntiles = hvp_tiles(c, C, col0, col_end, balanced);
  a.first_tile = 0;
  a.tile_step = 1;
  a.col0 = col0;
  a.col_end = col_end;
  a.sym = (full && c->sym_now) ? 1 : 0;
  a.tstart = c->tstart;
  a.zreuse = 0;
  // shared-memory layout of the first solve's reach (no pruning when the mask
  // and list would take more than half of the budget)
  const int nwords = (c->dn.r0 + 31) / 32;
  a.rm_words = (nwords + 3) & ~3;
  a.list_cap = 2048;
  const long fixed = 8L * a.rm_words + 4L * a.list_cap;
  const int budget = hvp_smem_budget(C);
  if (fixed > budget / 2) {
    a.rm_words = 0;
    a.list_cap = 0;
    a.zs_cap = 0;
  } else {
    a.zs_cap = (int)std::min<long>(a.list_cap, (budget - fixed) / (8L * C));
  }
  return a;
}

size_t hvp_split_scratch(const opf_ctx* c, int C) {
  int lk = 0;
  while ((1 << lk) < C) lk++;
  return hvp_stride(c, C) * (size_t)c->split_n1[lk] + hvp_stride(c, C / 2) * (size_t)c->split_n2[lk];
}

template <int C>
static void launch_hvp_split_t(opf_ctx* c, double* H, int lk) {
  const int n1 = c->split_n1[lk], n2 = c->split_n2[lk];
  HvpArgs a1 = make_hvp_args(c, C, H, 0, c->h.nu, true);
  HvpArgs a2 = make_hvp_args(c, C / 2, H, 0, c->h.nu, true);
  a1.colmap = c->colmap_split[lk];
  a1.ntiles = n1;
  a1.scratch = c->scratch;
  a2.colmap = c->colmap_split[lk] + (size_t)n1 * C;
  a2.ntiles = n2;
  a2.scratch = c->scratch + a1.stride * (size_t)n1;
  if (a2.stamps) a2.stamps += (size_t)n1 * 8;
  a1.zreuse = a2.zreuse = (c->z_reuse && c->z_gen == c->lu_gen && c->z_C == C) ? 1 : 0;
  c->z_gen = c->lu_gen;
  c->z_C = C;
  const size_t sm = std::max(hvp_smem_bytes(a1, C), hvp_smem_bytes(a2, C / 2));
  const int per_sm = std::max(1, n1 / c->sm_count);
  cudaMemsetAsync(c->split_ctr, 0, sizeof(int) * (4 + kSplitMaxSm), c->stream);
  if (a1.zreuse)
    hvp_split_kernel<C, 256, true><<<n1 + n2, 256, sm, c->stream>>>(a1, a2, per_sm, c->split_ctr);
  else
    hvp_split_kernel<C, 256><<<n1 + n2, 256, sm, c->stream>>>(a1, a2, per_sm, c->split_ctr);
  c->launches++;
}

// z = (dx/du) d = sum over the tiles' columns j of Z_j d_j, from the first
// adjoints Z = G_x^{-1}(-G_u W) the last split Hessian launch left in its slabs
// (rows in the factor's pivot order, written to their state positions):
// the state direction of a control step without a triangular solve.
// blockIdx.y takes a range of tiles; the ranges meet in atomic sums (z zeroed
// by the caller).
__global__ void zd_slab_kernel(const double* __restrict__ S1, size_t st1, int n1, int C1,
                               const double* __restrict__ S2, size_t st2, int n2, int C2,
                               const int* __restrict__ colmap, const double* __restrict__ d,
                               const int* __restrict__ perm, int nx, int tiles_per_y, double* z) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nx) return;
  const int t0 = blockIdx.y * tiles_per_y, t1 = min(n1 + n2, t0 + tiles_per_y);
  double s = 0.0;
  for (int t = t0; t < t1; t++) {
    const bool wide = t < n1;
    const int C = wide ? C1 : C2;
    const double* Zt = wide ? S1 + st1 * t : S2 + st2 * (t - n1);
    const int* cm = wide ? colmap + (size_t)t * C1 : colmap + (size_t)n1 * C1 + (size_t)(t - n1) * C2;
    for (int c = 0; c < C; c++) {
      const int j = __ldg(cm + c);
      if (j >= 0) s = fma(Zt[(size_t)k * C + c], __ldg(d + j), s);
    }
  }
  atomicAdd(z + perm[k], s);
}

// out_j = base_j + sum_k Z_j[k] w[perm[k]] for every column j of the tiles whose
// first adjoints the last split Hessian launch left in its slabs: G_u^T lambda
// for lambda = -G_x^{-T} w without the transposed solve (Z = -G_x^{-1} G_u).
// One CTA per tile; each thread sums its rows for the tile's columns, then a
// block reduction.
template <int CMAX>
__global__ void __launch_bounds__(256) zt_slab_kernel(const double* __restrict__ S1, size_t st1, int n1, int C1,
                                                      const double* __restrict__ S2, size_t st2, int C2,
                                                      const int* __restrict__ colmap, const double* __restrict__ w,
                                                      const int* __restrict__ perm, int nx,
                                                      const double* __restrict__ base, double* out) {
  __shared__ double red[8][CMAX];
  const int t = blockIdx.x, wide = t < n1, C = wide ? C1 : C2;
  const double* Zt = wide ? S1 + st1 * t : S2 + st2 * (t - n1);
  const int* cm = wide ? colmap + (size_t)t * C1 : colmap + (size_t)n1 * C1 + (size_t)(t - n1) * C2;
  double acc[CMAX];
#pragma unroll
  for (int c = 0; c < CMAX; c++) acc[c] = 0.0;
  for (int k = threadIdx.x; k < nx; k += blockDim.x) {
    const double wk = __ldg(w + __ldg(perm + k));
#pragma unroll
    for (int c = 0; c < CMAX; c++)
      if (c < C) acc[c] = fma(Zt[(size_t)k * C + c], wk, acc[c]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < CMAX; c++) {
    double v = acc[c];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < C) {
    double v = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) v += red[q][threadIdx.x];
    const int j = __ldg(cm + threadIdx.x);
    if (j >= 0) out[j] = base[j] + v;
  }
}

bool launch_adjoint_from_slabs(opf_ctx* c, const double* w, const double* base, double* out) {
  if (c->z_gen != c->lu_gen || c->z_C < 2 || c->z_C > 16) return false;
  int lk = 0;
  while ((1 << lk) < c->z_C) lk++;
  const int n1 = c->split_n1[lk], n2 = c->split_n2[lk], C = c->z_C;
  if (n1 <= 0 || !c->colmap_split[lk]) return false;
  const size_t st1 = hvp_stride(c, C), st2 = hvp_stride(c, C / 2);
  const double* S2 = c->scratch + st1 * (size_t)n1;
  if (C <= 8)
    zt_slab_kernel<8><<<n1 + n2, 256, 0, c->stream>>>(c->scratch, st1, n1, C, S2, st2, C / 2, c->colmap_split[lk],
                                                      w, c->dn.perm, c->dn.nx, base, out);
  else
    zt_slab_kernel<16><<<n1 + n2, 256, 0, c->stream>>>(c->scratch, st1, n1, C, S2, st2, C / 2, c->colmap_split[lk],
                                                       w, c->dn.perm, c->dn.nx, base, out);
  c->launches++;
  return true;
}

bool launch_state_direction(opf_ctx* c, const double* d, double* z) {
  if (c->z_gen != c->lu_gen || c->z_C < 2) return false;
  int lk = 0;
  while ((1 << lk) < c->z_C) lk++;
  const int n1 = c->split_n1[lk], n2 = c->split_n2[lk], C = c->z_C;
  if (n1 <= 0 || !c->colmap_split[lk]) return false;
  const size_t st1 = hvp_stride(c, C), st2 = hvp_stride(c, C / 2);
  const int nx = c->dn.nx, per_y = 16;
  cudaMemsetAsync(z, 0, sizeof(double) * (size_t)nx, c->stream);
  const dim3 grid(nblk(nx, 256), nblk(n1 + n2, per_y));
  zd_slab_kernel<<<grid, 256, 0, c->stream>>>(c->scratch, st1, n1, C, c->scratch + st1 * (size_t)n1, st2, n2, C / 2,
                                             c->colmap_split[lk], d, c->dn.perm, nx, per_y, z);
  c->launches++;
  return true;
}

bool launch_hvp_split(opf_ctx* c, int C, double* H) {
  int lk = 0;
  while ((1 << lk) < C) lk++;
  if (c->split_n1[lk] <= 0) return false;
  switch (C) {
    case 2: launch_hvp_split_t<2>(c, H, lk); return true;
    case 4: launch_hvp_split_t<4>(c, H, lk); return true;
    case 8: launch_hvp_split_t<8>(c, H, lk); return true;
    case 16: launch_hvp_split_t<16>(c, H, lk); return true;
    case 32: launch_hvp_split_t<32>(c, H, lk); return true;
    default: return false;
  }
}

int hvp_smem_budget(int C) { return C <= 4 ? 34 * 1024 : HVP_DYN_SMEM; }

size_t hvp_smem_bytes(const HvpArgs& a, int C) {
  return 8 * (size_t)a.zs_cap * C + 8 * (size_t)a.rm_words + 4 * (size_t)a.list_cap;
}

template <int C>
static void setup_hvp_smem_t() {
  cudaFuncSetAttribute(hvp_tile_kernel<C, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, HVP_DYN_SMEM);
  cudaFuncSetAttribute(hvp_tile_kernel<C, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, HVP_DYN_SMEM);
  cudaFuncSetAttribute(hvp_tile_kernel<C, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, HVP_DYN_SMEM);
  cudaFuncSetAttribute(hvp_batch_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, HVP_DYN_SMEM);
  if (C >= 2) {
    cudaFuncSetAttribute(hvp_split_kernel<(C >= 2 ? C : 2), 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         HVP_DYN_SMEM);
    cudaFuncSetAttribute(hvp_split_kernel<(C >= 2 ? C : 2), 256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         HVP_DYN_SMEM);
  }
}

void setup_hvp_smem() {
  setup_hvp_smem_t<1>();
  setup_hvp_smem_t<2>();
  setup_hvp_smem_t<4>();
  setup_hvp_smem_t<8>();
  setup_hvp_smem_t<16>();
  setup_hvp_smem_t<32>();
}

int hvp_tiles(const opf_ctx* c, int C, int col0, int col_end, bool balanced) {
  int lk = 0;
  while ((1 << lk) < C) lk++;
  const int f = balanced ? 1 : 0;
  if (col0 == 0 && col_end == c->h.nu && c->coltiles[f][lk] > 0) return c->coltiles[f][lk];
  return (col_end - col0 + C - 1) / C;
}

template <int C>
static int batch_occ() {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hvp_batch_kernel<C>, 256, hvp_smem_budget(C));
  return occ;
}

int hvp_batch_occupancy(int C) {
  switch (C) {
    case 1: return batch_occ<1>();
    case 2: return batch_occ<2>();
    case 4: return batch_occ<4>();
    case 8: return batch_occ<8>();
    case 16: return batch_occ<16>();
    case 32: return batch_occ<32>();
    default: return 0;
  }
}

bool launch_hvp_batch(cudaStream_t st, int C, const HvpArgs* args, const int2* tiles, int ntot, int* counter,
                      double* scratch, size_t stride, int grid, size_t smem) {
  switch (C) {
    case 1: hvp_batch_kernel<1><<<grid, 256, smem, st>>>(args, tiles, ntot, counter, scratch, stride); return true;
    case 2: hvp_batch_kernel<2><<<grid, 256, smem, st>>>(args, tiles, ntot, counter, scratch, stride); return true;
    case 4: hvp_batch_kernel<4><<<grid, 256, smem, st>>>(args, tiles, ntot, counter, scratch, stride); return true;
    case 8: hvp_batch_kernel<8><<<grid, 256, smem, st>>>(args, tiles, ntot, counter, scratch, stride); return true;
    case 16: hvp_batch_kernel<16><<<grid, 256, smem, st>>>(args, tiles, ntot, counter, scratch, stride); return true;
    case 32: hvp_batch_kernel<32><<<grid, 256, smem, st>>>(args, tiles, ntot, counter, scratch, stride); return true;
    default: return false;
  }
}

// Same tile kernel with an explicitly given workspace (scratch of `grid` CTAs).
template <int C>
static void launch_hvp_scratch_t(opf_ctx* c, double* H, double* scratch, int grid, int ntiles, int col0,
                                 int col_end) {
  HvpArgs a = make_hvp_args(c, C, H, col0, col_end, true);
  a.scratch = scratch;
  a.ntiles = ntiles;
  hvp_tile_kernel<C, 256><<<grid, 256, hvp_smem_bytes(a, C), c->stream>>>(a);
  c->launches++;
}

bool launch_hvp_scratch(opf_ctx* c, int C, double* H, double* scratch, int grid, int ntiles, int col0,
                        int col_end) {
  switch (C) {
    case 1: launch_hvp_scratch_t<1>(c, H, scratch, grid, ntiles, col0, col_end); return true;
    case 2: launch_hvp_scratch_t<2>(c, H, scratch, grid, ntiles, col0, col_end); return true;
    case 4: launch_hvp_scratch_t<4>(c, H, scratch, grid, ntiles, col0, col_end); return true;
    case 8: launch_hvp_scratch_t<8>(c, H, scratch, grid, ntiles, col0, col_end); return true;
    case 16: launch_hvp_scratch_t<16>(c, H, scratch, grid, ntiles, col0, col_end); return true;
    case 32: launch_hvp_scratch_t<32>(c, H, scratch, grid, ntiles, col0, col_end); return true;
    default: return false;
  }
}

// Asymmetry of a computed Hessian (Sec. III-C assembles H column block by
// column block; in exact arithmetic it is symmetric): sums[0] += sum_ij (H_ij -
// H_ji)^2 and sums[1] += sum_ij H_ij^2 over one 32 x 32 tile per CTA, the tile
// and its mirror read through shared memory so both loads are coalesced
// (column-major H, leading dimension n).
__global__ void __launch_bounds__(256) hess_asym_kernel(const double* __restrict__ H, int n, double* sums) {
  __shared__ double A[32][33], B[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int i = bi * 32 + tx, j = bj * 32 + r;  // A[r][tx] = H(i, j); B[r][tx] = H(j', i') of the mirror
    A[r][tx] = (i < n && j < n) ? H[(size_t)j * n + i] : 0.0;
    const int i2 = bj * 32 + tx, j2 = bi * 32 + r;
    B[r][tx] = (i2 < n && j2 < n) ? H[(size_t)j2 * n + i2] : 0.0;
  }
  __syncthreads();
  double d2 = 0.0, h2 = 0.0;
  for (int r = ty; r < 32; r += 8) {
    const double a = A[r][tx];       // H(bi*32 + tx, bj*32 + r)
    const double b = B[tx][r];       // H(bj*32 + r, bi*32 + tx)
    d2 = fma(a - b, a - b, d2);
    h2 = fma(a, a, h2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    h2 += __shfl_xor_sync(0xffffffffu, h2, o);
  }
  if (tx == 0) {
    atomicAdd(sums, d2);
    atomicAdd(sums + 1, h2);
  }
}

void launch_hess_asymmetry(opf_ctx* c, const double* H, int n, double* sums) {
  const int nb = (n + 31) / 32;
  hess_asym_kernel<<<dim3(nb, nb), 256, 0, c->stream>>>(H, n, sums);
  c->launches++;
}

// Completion of a symmetric Hessian (HvpArgs::sym): the tile of column j kept
// the rows i with qpos[i] >= tstart[j]; the others take H(j, i), which the tile
// of column i kept (qpos[i] < tstart[j] <= qpos[j] and tstart[i] <= qpos[i]).
// One 32 x 32 tile per CTA, its mirror read through shared memory so both the
// loads and the stores coalesce (column-major H, leading dimension n).
__global__ void __launch_bounds__(256) hess_mirror_kernel(double* H, int n, const int* __restrict__ qpos,
                                                          const int* __restrict__ tstart) {
  __shared__ double B[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {  // B[r][tx] = H(bj*32 + tx, bi*32 + r)
    const int i2 = bj * 32 + tx, j2 = bi * 32 + r;
    B[r][tx] = (i2 < n && j2 < n) ? H[(size_t)j2 * n + i2] : 0.0;
  }
  __syncthreads();
  const int i = bi * 32 + tx;
  if (i >= n) return;
  const int qi = qpos[i];
  for (int r = ty; r < 32; r += 8) {
    const int j = bj * 32 + r;
    if (j < n && qi < tstart[j]) H[(size_t)j * n + i] = B[tx][r];  // H(i, j) = H(j, i)
  }
}

void launch_hess_mirror(opf_ctx* c, double* H, int n) {
  const int nb = (n + 31) / 32;
  hess_mirror_kernel<<<dim3(nb, nb), 256, 0, c->stream>>>(H, n, c->dn.qpos, c->tstart);
  c->launches++;
}

size_t hvp_plain_scratch(const opf_ctx* c) { return 4 * (size_t)c->dn.nx + (size_t)c->dn.ngn + 32; }

int launch_hvp_plain(opf_ctx* c, double* H, int col0, int col_end, double* work) {
  HvpArgs a = make_hvp_args(c, 1, H, col0, col_end, true);
  const int nx = c->dn.nx;
  double* bx = work;          // right-hand side, then R in x order
  double* zx = bx + nx;       // Z, then Psi in x order
  double* zp = zx + nx;       // Z, then Psi in pivot order
  double* rp = zp + nx;       // R in pivot order
  double* QD = rp + nx;
  double* PD = QD + c->dn.ngn;
  const int gb = std::max(1, std::min(nblk(nx, 256), 2 * c->sm_count));
  const int gn = std::max(1, nblk(c->dn.ngn, 128)), gbus = std::max(1, nblk(c->dn.nb, 128));
  const int* perm = c->dn.perm;
  int launches = 0;
  for (int j = col0; j < col_end; j++) {
    cudaMemsetAsync(bx, 0, sizeof(double) * nx, c->stream);
    plain_rhs_kernel<<<1, 32, 0, c->stream>>>(a, j, bx);
    launch_solve1(c, bx, zx, false, 1.0);
    plain_permute_kernel<<<gb, 256, 0, c->stream>>>(perm, zx, zp, nx, 1);
    plain_qd_kernel<<<gn, 128, 0, c->stream>>>(a, j, zp, QD, PD);
    plain_gather_kernel<<<gbus, 128, 0, c->stream>>>(a, j, zp, QD, PD, rp);
    plain_permute_kernel<<<gb, 256, 0, c->stream>>>(perm, rp, bx, nx, 0);
    launch_solve1(c, bx, zx, true, 1.0);
    plain_permute_kernel<<<gb, 256, 0, c->stream>>>(perm, zx, zp, nx, 1);
    plain_assemble_kernel<<<gn, 128, 0, c->stream>>>(a, j, zp);
    launches += 9;
  }
  c->launches += 7LL * (col_end - col0);  // the two solves count themselves
  return launches;
}

}  // namespace opf
