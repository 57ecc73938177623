// Reduced-Newton step of the augmented-Lagrangian subproblem (Prop. 3; entry
// point opf_al_step, declared in include/opf.h with the full formulas).
//
// Device pieces: the barrier/Sigma/omega terms, the reduced Jacobian products
// J^T v (weighted adjoint gradient) and J d (G_u d, one L/U solve, directional
// derivatives of c), a blocked FP64 Cholesky of S_uu (32-wide diagonal blocks,
// row-parallel triangular solves of the panel, 64x64-tiled symmetric rank-32
// updates), blocked dense triangular solves, the slack and dual steps and the
// fraction-to-the-boundary reductions.  The host drives the inertia correction
// and the trial power flows.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <vector>
#include <cmath>
#include <string>

#include "opf_internal.h"

using namespace opf;

namespace opf {

struct StepWork {
  int nu = 0, m = 0;
  double *S = nullptr, *L = nullptr;           // n_u x n_u column-major
  double *gu, *gs, *sig_u, *gpsi_u, *sig_s, *gpsi_s, *omega, *v, *r, *du, *ds, *Jtv, *Jdu;
  double *b, *z, *ut, *xt, *pd, *qd;
  double *strial, *lsv;                         // line search: trial s; [0] F, [1] barrier sum, [2] slope, [3] F_t, [4] barrier sum at the trial
  double *dz;                                   // 2 n_u + 2 m: zl_u, zu_u, zl_s, zu_s steps
  double* red;                                  // [2]: alpha_p, alpha_d (as ordered bits)
  double* Dinv;                                 // [ceil(n_u / 32)][32][32]: inverses of the factor's diagonal blocks
  int* oz_e = nullptr;                          // [n_u] row exponents of the emulated trailing update
  void* oz_d = nullptr;                         // 8 x 128 x (n_u rounded up to 128) bf16 digits of the emulated trailing update
  int* flag;
  double* h_red;
  double* h_ls = nullptr;  // pinned [8]: the line search's reductions
  int* h_flag;
  void* block = nullptr;
  cudaEvent_t ev[7] = {};  // phase boundaries of a step
  cudaStream_t aux = nullptr;       // the right-hand side J^T v runs here beside the Cholesky
  cudaEvent_t aux_go = nullptr, aux_done = nullptr;
  unsigned* trsv_flags = nullptr;  // [ceil(n_u / 32)] block flags of the dense solves (epochs)
  int* trsv_err = nullptr;         // a dense-solve wait timed out
  int* oz_err = nullptr;           // a wait of the tcgen05 emulated update timed out
  unsigned trsv_epoch = 0;
  // the factorisation's launch sequence as a CUDA graph, per trailing-update kind
  // (FP64, emulated), captured on first use for the wait limit and update engine
  // of that moment
  cudaGraphExec_t chol_exec[2] = {nullptr, nullptr};
  long long chol_lim[2] = {0, 0};
  int chol_engine[2] = {-1, -1};
  long long chol_kernels[2] = {0, 0};
  // tracking QP (opf_tracking_update): grad q, the linearisation point w_t and its
  // state, the KKT reductions and the constraint values at the new point
  void* qp_block = nullptr;
  double *gqu = nullptr, *gqs = nullptr, *u0 = nullptr, *s0 = nullptr, *x0 = nullptr, *kred = nullptr,
         *cv = nullptr, *h_kred = nullptr;
};

void free_step_work(opf_ctx* c) {
  if (!c->stepw) return;
  StepWork* w = c->stepw;
  if (w->block) cudaFree(w->block);
  if (w->aux_go) cudaEventDestroy(w->aux_go);
  if (w->aux_done) cudaEventDestroy(w->aux_done);
  if (w->aux) cudaStreamDestroy(w->aux);
  if (w->oz_e) cudaFree(w->oz_e);
  if (w->oz_d) cudaFree(w->oz_d);
  if (w->qp_block) cudaFree(w->qp_block);
  if (w->h_kred) cudaFreeHost(w->h_kred);
  if (w->h_red) cudaFreeHost(w->h_red);
  if (w->h_ls) cudaFreeHost(w->h_ls);
  if (w->h_flag) cudaFreeHost(w->h_flag);
  for (cudaEvent_t e : w->ev)
    if (e) cudaEventDestroy(e);
  for (cudaGraphExec_t g : w->chol_exec)
    if (g) cudaGraphExecDestroy(g);
  delete w;
  c->stepw = nullptr;
}

}  // namespace opf

namespace {

constexpr int NB = 32;   // panel width of the Cholesky
constexpr int GB = 128;  // columns per group: rank of one emulated trailing update

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------- Cholesky

// Diagonal block [k0, k0 + kb) and its inverse X = L_kk^{-1} in shared memory,
// one CTA of 16 warps in two roles.  Warp 0 carries the pivot chain in
// registers (lane i: row i of the current column): column j's pivot takes one
// reciprocal square root, the scaled column is published, and after the step's
// barrier warp 0 loads column j + 1 (updated by the other warps through column
// j - 1) and applies column j's rank-one term to it itself.  The other 15 warps
// lag one column: after barrier j they scale row j of X and apply column j to
// the columns from j + 2 on and to X (L_ic -= L_ij L_cj, X_ic -= L_ij X_jc),
// packed over their threads.  So the chain per column is rsqrt + two FP64 ops
// + one barrier.  X goes to Dinv (row-major), used by the panel solve below and
// by the dense triangular solves.
__global__ void __launch_bounds__(512) chol_diag_kernel(double* A, int n, int k0, int kb, int* flag,
                                                        double* Dinv) {
  __shared__ double T[NB][NB + 1], X[NB][NB + 1];
  __shared__ double s_r[NB];
  __shared__ unsigned short tbl[NB * (NB + 1) / 2];  // packed (row, column) offsets of a triangle
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  // what does not depend on the previous kernel runs before the wait for it
  for (int q = tid; q < NB * NB; q += nt) {
    const int i = q >> 5, c = q & 31;
    X[i][c] = (i == c) ? 1.0 : 0.0;
  }
  for (int e = tid; e < NB * (NB + 1) / 2; e += nt) {
    int ri = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while (ri * (ri + 1) / 2 > e) ri--;
    while ((ri + 1) * (ri + 2) / 2 <= e) ri++;
    tbl[e] = (unsigned short)((ri << 8) | (e - ri * (ri + 1) / 2));
  }
  if (tid == 0) s_bad = 0;
  pdl_wait();
  if (*flag) return;
  for (int q = tid; q < NB * NB; q += nt) {  // lanes along a column of A (coalesced)
    const int i = q & 31, c = q >> 5;
    T[i][c] = (i < kb && c <= i) ? A[(size_t)(k0 + c) * n + k0 + i] : 0.0;
  }
  __syncthreads();
  if (warp == 0) {
    double col = T[lane][0];
    for (int j = 0; j < kb; j++) {
      double a = __shfl_sync(0xffffffffu, col, j);
      const bool bad = !(a > 0.0) || !isfinite(a);
      double r = rsqrt(a);
      if (bad) {
        a = 1.0;
        r = 1.0;
      }
      const double l = (lane == j) ? a * r : col * r;
      if (lane >= j && lane < kb) T[lane][j] = l;
      if (lane == 0) {
        s_r[j] = r;
        if (bad) s_bad = 1;
      }
      __syncthreads();  // column j published; the other warps' column j - 1 applied
      if (j + 1 < kb) {
        const double lj1 = __shfl_sync(0xffffffffu, l, j + 1);
        col = fma(-l, lj1, T[lane][j + 1]);
      }
    }
  } else {
    const int bt = tid - 32, nbt = nt - 32;
    for (int j = 0; j < kb; j++) {
      __syncthreads();
      if (warp == 1 && lane <= j) X[j][lane] *= s_r[j];
      asm volatile("bar.sync 1, %0;" ::"r"(nbt) : "memory");
      const int m2 = kb - 2 - j;  // columns j + 2 .. kb - 1 of the trailing triangle
      const int nT = m2 > 0 ? m2 * (m2 + 1) / 2 : 0, nX = (kb - 1 - j) * (j + 1);
      for (int e = bt; e < nT + nX; e += nbt) {
        if (e < nT) {
          const int t = tbl[e], ii = j + 2 + (t >> 8), cc = j + 2 + (t & 255);
          T[ii][cc] = fma(-T[ii][j], T[cc][j], T[ii][cc]);
        } else {
          const int e2 = e - nT, ri = e2 / (j + 1), cc = e2 - ri * (j + 1), ii = j + 1 + ri;
          X[ii][cc] = fma(-T[ii][j], X[j][cc], X[ii][cc]);
        }
      }
    }
  }
  __syncthreads();  // the last column's updates
  if (tid == 0 && s_bad) *flag = 1;
  for (int q = tid; q < NB * NB; q += nt) {
    const int i = q >> 5, c = q & 31;
    Dinv[(size_t)(k0 / NB) * NB * NB + q] = (i < kb && c <= i) ? X[i][c] : 0.0;
    const int ia = q & 31, ca = q >> 5;  // lanes along a column of A
    if (ia < kb && ca <= ia) A[(size_t)(k0 + ca) * n + k0 + ia] = T[ia][ca];
  }
  pdl_trigger();
}

// Panel below the diagonal block: X21 = A21 L_kk^{-T} = A21 Dinv^T as a small
// GEMM (blockDim / 16 rows x 32 columns per CTA, at most 16 rows), written in
// place.  Dinv is lower triangular, so column c takes the terms t <= c only;
// thread (row, c) also owns column 31 - c, and the two runs of term pairs add
// up to 17 for every thread, so a warp issues 34 FMAs per thread instead of 64
// (the FP64 pipe issues whole warp instructions).  Each column keeps the even
// and the odd terms in separate sums, in increasing t, as the full product would.
__global__ void __launch_bounds__(256) chol_trsm_kernel(double* A, int n, int k0, int kb, const int* flag,
                                                        const double* __restrict__ Dinv) {
  pdl_wait();
  if (*flag) return;
  __shared__ double M[NB][NB + 1];  // M[c][t] = (L_kk^{-1})_ct
  __shared__ double P[16][NB + 1];  // P[r][t] = A21[row r][t]
  const double* D = Dinv + (size_t)(k0 / NB) * NB * NB;
  const int rows = blockDim.x >> 4, row0 = k0 + kb + blockIdx.x * rows;
  for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) M[q >> 5][q & 31] = D[q];
  for (int q = threadIdx.x; q < rows * NB; q += blockDim.x) {
    const int r = q % rows, tt = q / rows, g = row0 + r;
    P[r][tt] = (tt < kb && g < n) ? A[(size_t)(k0 + tt) * n + g] : 0.0;
  }
  __syncthreads();
  const int r = threadIdx.x >> 4, c0 = threadIdx.x & 15, c1 = NB - 1 - c0;
  const int n0 = (c0 + 2) >> 1;  // term pairs of column c0; column c1 takes the other 17 - n0
  double e0 = 0.0, o0 = 0.0, e1 = 0.0, o1 = 0.0;
#pragma unroll
  for (int q = 0; q < 17; q++) {
    const bool first = q < n0;
    const int tt = first ? 2 * q : 2 * (q - n0), c = first ? c0 : c1;
    double e = first ? e0 : e1, o = first ? o0 : o1;
    e = fma(P[r][tt], M[c][tt], e);
    o = fma(P[r][tt + 1], M[c][tt + 1], o);
    if (first) {
      e0 = e;
      o0 = o;
    } else {
      e1 = e;
      o1 = o;
    }
  }
  const int g = row0 + r;
  if (g < n) {
    if (c0 < kb) A[(size_t)(k0 + c0) * n + g] = e0 + o0;
    if (c1 < kb) A[(size_t)(k0 + c1) * n + g] = e1 + o1;
  }
  pdl_trigger();
}

// trailing lower triangle -= P P^T, P = A[r0:, k0:k0+kb]; one TS x TS tile per CTA
// (16 x 16 threads, (TS/16)^2 outputs each).  The tiles are laid from the
// origin r0 = k0 + kb + off: first_col = 1, the first tile column only; 2, a
// grid of tile columns x tile rows (blockIdx.x, blockIdx.y; tiles above the
// diagonal skipped); else every tile bj <= bi of the triangle.  Columns at or
// past col_end are left alone.
template <int TS>
__global__ void __launch_bounds__(256) chol_syrk_kernel(double* A, int n, int k0, int kb, const int* flag,
                                                        int first_col, int off, int col_end) {
  pdl_wait();
  if (*flag) return;
  constexpr int R = TS / 16;
  const int r0 = k0 + kb + off;  // origin of the tiled triangle
  int bi, bj;
  if (first_col == 2) {  // rectangle of tile rows x tile columns, upper tiles skipped
    bi = blockIdx.y;
    bj = blockIdx.x;
    if (bi < bj) return;
  } else if (first_col) {
    bi = blockIdx.x;
    bj = 0;
  } else {
    const int t = blockIdx.x;
    bi = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((bi + 1) * (bi + 2) / 2 <= t) bi++;
    while (bi * (bi + 1) / 2 > t) bi--;
    bj = t - bi * (bi + 1) / 2;
  }
  __shared__ double Pa[TS][NB + 1], Pb[TS][NB + 1];
  for (int q = threadIdx.x; q < TS * NB; q += blockDim.x) {
    const int rr = q % TS, k = q / TS;
    const int ga = r0 + bi * TS + rr, gb = r0 + bj * TS + rr;
    Pa[rr][k] = (k < kb && ga < n) ? A[(size_t)(k0 + k) * n + ga] : 0.0;
    Pb[rr][k] = (k < kb && gb < n) ? A[(size_t)(k0 + k) * n + gb] : 0.0;
  }
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  double acc[R][R] = {};
  for (int k = 0; k < kb; k++) {
    double a[R], b[R];
#pragma unroll
    for (int q = 0; q < R; q++) {
      a[q] = Pa[ty * R + q][k];
      b[q] = Pb[tx * R + q][k];
    }
#pragma unroll
    for (int p = 0; p < R; p++)
#pragma unroll
      for (int q = 0; q < R; q++) acc[p][q] += a[p] * b[q];
  }
#pragma unroll
  for (int p = 0; p < R; p++)
#pragma unroll
    for (int q = 0; q < R; q++) {
      const int gi = r0 + bi * TS + ty * R + p, gj = r0 + bj * TS + tx * R + q;
      if (gi < n && gj <= gi && gj < col_end) A[(size_t)gj * n + gi] -= acc[p][q];
    }
  pdl_trigger();
}

// ---------------------------------------------------------------- dense triangular solves

// Dense triangular solve with the Cholesky factor in one cooperative launch
// per direction (forward L y = b, backward L^T x = y; b is overwritten with the
// solution).  L is lower, column-major with leading dimension n, and its
// transpose is copied into the strict upper triangle (chol_upper_copy_kernel),
// so both directions read the off-diagonal block (row block i, column block k)
// at (32 k + c) n + 32 i + lane: lanes along rows, coalesced.  Row block i
// (32 rows) belongs to CTA i mod gridDim.x, which takes its blocks in solve
// order.  Block i depends on the finished blocks k < i (forward) or k > i
// (backward); the neighbour i -+ 1, the last to finish, is split over the 8
// warps (4 columns each), the others go whole to the warps in turn, earliest
// finished first.  Each
// warp loads its tile before it waits for the block's flag; then it reads the
// block's solution and accumulates.  The diagonal block's inverse (prefetched,
// 4 columns per warp) gives the block's solution, which warp 0 publishes with
// the call's epoch (store, fence, release flag).  Every wait is bounded: on
// timeout the kernel sets err and stops waiting (the result is then void).
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void wait_block(const unsigned* flag, unsigned epoch, int* err, int lane,
                                           long long lim) {
  long long spins = 0;
  while (ld_acquire_u32(flag) != epoch) {
    if (++spins > lim || *(volatile int*)err) {
      if (lane == 0) atomicExch(err, 1);
      break;
    }
    __nanosleep(32);
  }
}

// L^T into the strict upper triangle, 32 x 32 tiles through shared memory.
__global__ void chol_upper_copy_kernel(double* A, int n) {
  __shared__ double T[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // tile of rows bi, columns bj of L (bi > bj)
  if (bi <= bj) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += blockDim.x >> 5) {
    const int row = bi * 32 + tx, col = bj * 32 + r;
    T[r][tx] = (row < n && col < n) ? A[(size_t)col * n + row] : 0.0;  // L(row, col)
  }
  __syncthreads();
  for (int r = ty; r < 32; r += blockDim.x >> 5) {
    const int col = bi * 32 + r, row = bj * 32 + tx;  // upper position (row, col) holds L(col, row)
    if (row < n && col < n) A[(size_t)col * n + row] = T[tx][r];
  }
}

template <bool FWD>
__global__ void __launch_bounds__(256) chol_trsv_kernel(const double* __restrict__ L, int n,
                                                        const double* __restrict__ Dinv, double* b,
                                                        unsigned* flags, unsigned epoch, int* err,
                                                        long long lim) {
  __shared__ double part[8][32];
  __shared__ double accs[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = (n + 31) >> 5;
  for (int q = blockIdx.x; q < nb; q += gridDim.x) {
    const int i = FWD ? q : nb - 1 - q;
    const int row = i * 32 + lane;
    const bool live = row < n;
    const double* D = Dinv + (size_t)i * 1024;
    double dv[4];
#pragma unroll
    for (int cc = 0; cc < 4; cc++) {
      const int c = 4 * warp + cc;
      dv[cc] = FWD ? D[lane * 32 + c] : D[c * 32 + lane];
    }
    const double bi = live ? b[row] : 0.0;
    double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0;
    // whole blocks, the earliest finished first: forward 0 .. i - 2, backward
    // nb - 1 down to i + 2
    const int nwhole = FWD ? i - 1 : nb - i - 2;
    for (int m = warp; m < nwhole; m += 8) {
      const int k = FWD ? m : nb - 1 - m;
      const int col0 = k * 32, kc = min(32, n - col0);
      double t[32];
#pragma unroll
      for (int c = 0; c < 32; c++) t[c] = (live && c < kc) ? L[(size_t)(col0 + c) * n + row] : 0.0;
      wait_block(flags + k, epoch, err, lane, lim);
      const double xk = (col0 + lane < n) ? __ldcg(b + col0 + lane) : 0.0;
#pragma unroll
      for (int c = 0; c < 32; c += 4) {
        p0 = fma(t[c], __shfl_sync(0xffffffffu, xk, c), p0);
        p1 = fma(t[c + 1], __shfl_sync(0xffffffffu, xk, c + 1), p1);
        p2 = fma(t[c + 2], __shfl_sync(0xffffffffu, xk, c + 2), p2);
        p3 = fma(t[c + 3], __shfl_sync(0xffffffffu, xk, c + 3), p3);
      }
    }
    // the neighbour block, 4 columns per warp
    if (FWD ? i > 0 : i < nb - 1) {
      const int k = FWD ? i - 1 : i + 1, col0 = k * 32, kc = min(32, n - col0);
      double t4[4];
#pragma unroll
      for (int cc = 0; cc < 4; cc++) {
        const int c = 4 * warp + cc;
        t4[cc] = (live && c < kc) ? L[(size_t)(col0 + c) * n + row] : 0.0;
      }
      wait_block(flags + k, epoch, err, lane, lim);
      const double xk = (col0 + lane < n) ? __ldcg(b + col0 + lane) : 0.0;
      p0 = fma(t4[0], __shfl_sync(0xffffffffu, xk, 4 * warp), p0);
      p1 = fma(t4[1], __shfl_sync(0xffffffffu, xk, 4 * warp + 1), p1);
      p2 = fma(t4[2], __shfl_sync(0xffffffffu, xk, 4 * warp + 2), p2);
      p3 = fma(t4[3], __shfl_sync(0xffffffffu, xk, 4 * warp + 3), p3);
    }
    part[warp][lane] = (p0 + p1) + (p2 + p3);
    __syncthreads();
    if (warp == 0)
      accs[lane] = bi - (((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
                         ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane])));
    __syncthreads();
    // x_i = L_ii^{-1} acc (forward) or L_ii^{-T} acc (backward), 4 columns per warp
    part[warp][lane] = fma(dv[0], accs[4 * warp], dv[1] * accs[4 * warp + 1]) +
                       fma(dv[2], accs[4 * warp + 2], dv[3] * accs[4 * warp + 3]);
    __syncthreads();
    if (warp == 0) {
      const double x = ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
                       ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane]));
      if (live) b[row] = x;
      __syncwarp();  // orders the warp's stores before lane 0's release
      if (lane == 0) st_release_u32(flags + i, epoch);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- step kernels

// S <- (S + S^T) / 2 + diag(sig_u) on the lower triangle (the factorisation reads
// no other part), 32 x 32 tile pairs through shared memory so both reads coalesce.
__global__ void sym_diag_kernel(double* S, int n, const double* sig_u) {
  __shared__ double T[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;  // tile of rows bi, columns bj (bi >= bj)
  if (bi < bj) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += blockDim.x >> 5) {  // T[c][tx] = S(row bj*32 + tx, col bi*32 + c)
    const int row = bj * 32 + tx, col = bi * 32 + r;
    T[r][tx] = (row < n && col < n) ? S[(size_t)col * n + row] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += blockDim.x >> 5) {  // element (row bi*32 + tx, col bj*32 + r)
    const int row = bi * 32 + tx, col = bj * 32 + r;
    if (row < n && col <= row) {
      double* p = S + (size_t)col * n + row;
      *p = (row == col) ? *p + sig_u[row] : 0.5 * (*p + T[tx][r]);
    }
  }
}

// L = S + delta I on the lower triangle (the factorisation reads no other part;
// the dense solves' transposed copy fills the strict upper triangle later).
__global__ void add_diag_kernel(double* L, const double* S, int n, double delta) {
  const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || i < j) return;
  L[(size_t)j * n + i] = S[(size_t)j * n + i] + ((i == j) ? delta : 0.0);
}

// Sigma, grad psi, omega and v = rho D^2 (rho D^2 + Sigma_s)^{-1} grad_s psi
__global__ void step_prep_kernel(int nu, int m, const double* u, const double* ulo, const double* uhi,
                                 const double* zlu, const double* zuu, const double* s, const double* slo,
                                 const double* shi, const double* zls, const double* zus, const double* gu,
                                 const double* gs, const double* sigc, double rho, double mu, double* sig_u,
                                 double* gpsi_u, double* sig_s, double* gpsi_s, double* omega, double* v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) {
    const double dl = u[i] - ulo[i], dh = uhi[i] - u[i];
    sig_u[i] = zlu[i] / dl + zuu[i] / dh;
    gpsi_u[i] = gu[i] - mu / dl + mu / dh;
  }
  if (i < m) {
    const double dl = s[i] - slo[i], dh = shi[i] - s[i];
    const double sg = zls[i] / dl + zus[i] / dh;
    const double gp = gs[i] - mu / dl + mu / dh;
    const double rd2 = rho * sigc[i] * sigc[i];
    sig_s[i] = sg;
    gpsi_s[i] = gp;
    omega[i] = rd2 * sg / (rd2 + sg);
    v[i] = rd2 / (rd2 + sg) * gp;
  }
}

__global__ void step_sigma_kernel(int nu, int m, const double* u, const double* ulo, const double* uhi,
                                  const double* zlu, const double* zuu, const double* s, const double* slo,
                                  const double* shi, const double* zls, const double* zus, const double* sigc,
                                  double rho, double* sig_u, double* sig_s, double* omega) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) sig_u[i] = zlu[i] / (u[i] - ulo[i]) + zuu[i] / (uhi[i] - u[i]);
  if (i < m) {
    const double sg = zls[i] / (s[i] - slo[i]) + zus[i] / (shi[i] - s[i]);
    const double rd2 = rho * sigc[i] * sigc[i];
    sig_s[i] = sg;
    omega[i] = rd2 * sg / (rd2 + sg);
  }
}

__global__ void neg_sum_kernel(int n, const double* a, const double* b, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = -a[i] - b[i];
}

// G_u d into x order (rows P_i, Q_i), from the branch table at the current state
__global__ void gu_times_kernel(DevNet n, const double* tab, const double* d, double* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n.nb || n.type[i] == REF) return;
  const int nl = n.nl;
  double ap = 0.0, aq = 0.0, selfp = 0.0;
  for (int q = n.adj_ptr[i]; q < n.adj_ptr[i + 1]; q++) {
    const int e = n.adj[q], l = e >> 1, s = e & 1;
    const int o = s ? n.f[l] : n.t[l];
    if (n.type[o] != PQ) {
      const double dv = d[n.uv[o]];
      ap += tab[(size_t)TAB_DP(s, 1 - s) * nl + l] * dv;
      aq += tab[(size_t)TAB_DQ(s, 1 - s) * nl + l] * dv;
    }
    selfp += tab[(size_t)TAB_DP(s, s) * nl + l];
  }
  if (n.type[i] == PV) ap += selfp * d[n.uv[i]] - d[n.up[i]];
  b[n.xth[i]] = ap;
  if (n.type[i] == PQ) b[n.xv[i]] = aq;
}

__device__ __forceinline__ void dir_at(const DevNet& n, const double* z, const double* du, int b, double& vd,
                                       double& td) {
  vd = (n.type[b] == PQ) ? z[n.xv[b]] : du[n.uv[b]];
  td = (n.type[b] == REF) ? 0.0 : z[n.xth[b]];
}

// J d = d_u c d + d_x c z: line flows per branch
__global__ void jvp_branch_kernel(DevNet n, const double* tab, const double* flows, const double* z,
                                  const double* du, double* jd) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n.nl) return;
  const int nl = n.nl;
  double d[4];
  dir_at(n, z, du, n.f[l], d[0], d[2]);
  dir_at(n, z, du, n.t[l], d[1], d[3]);
  for (int s = 0; s < 2; s++) {
    double pdot = 0.0, qdot = 0.0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      pdot += tab[(size_t)TAB_DP(s, k) * nl + l] * d[k];
      qdot += tab[(size_t)TAB_DQ(s, k) * nl + l] * d[k];
    }
    jd[s * nl + l] = 2.0 * (flows[(2 * s) * nl + l] * pdot + flows[(2 * s + 1) * nl + l] * qdot);
  }
}

// J d: voltage, slack P/Q and PV Q rows per bus
__global__ void jvp_bus_kernel(DevNet n, const double* tab, const double* z, const double* du, double* jd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n.nb) return;
  const int nl = n.nl, o_v = 2 * nl, o_r = 2 * nl + n.npq;
  if (n.type[i] == PQ) {
    jd[o_v + n.pqpos[i]] = z[n.xv[i]];
    return;
  }
  double pdot = 0.0, qdot = 0.0;
  for (int q = n.adj_ptr[i]; q < n.adj_ptr[i + 1]; q++) {
    const int e = n.adj[q], l = e >> 1, s = e & 1;
    double d[4];
    dir_at(n, z, du, n.f[l], d[0], d[2]);
    dir_at(n, z, du, n.t[l], d[1], d[3]);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      pdot += tab[(size_t)TAB_DP(s, k) * nl + l] * d[k];
      qdot += tab[(size_t)TAB_DQ(s, k) * nl + l] * d[k];
    }
  }
  if (n.type[i] == REF) {
    jd[o_r] = pdot;
    jd[o_r + 1] = qdot;
  } else {
    jd[o_r + 2 + n.pvpos[i]] = qdot;
  }
}

__device__ __forceinline__ void atomic_min_pos(double* a, double v) {
  atomicMin(reinterpret_cast<unsigned long long*>(a), (unsigned long long)__double_as_longlong(v));
}

// d_s, dual steps and the fraction-to-the-boundary step lengths (reduced into red[0..1])
__global__ void step_finish_kernel(int nu, int m, const double* u, const double* du, const double* ulo,
                                   const double* uhi, const double* zlu, const double* zuu, const double* s,
                                   const double* slo, const double* shi, const double* zls, const double* zus,
                                   const double* gpsi_s, const double* sig_s, const double* jdu,
                                   const double* sigc, double rho, double mu, double tau, double* ds,
                                   double* dz, double* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double ap = 1.0, ad = 1.0;
  if (i < nu) {
    const double dl = u[i] - ulo[i], dh = uhi[i] - u[i], d = du[i];
    const double dzl = mu / dl - zlu[i] - zlu[i] / dl * d;
    const double dzh = mu / dh - zuu[i] + zuu[i] / dh * d;
    dz[i] = dzl;
    dz[nu + i] = dzh;
    if (d < 0) ap = fmin(ap, -tau * dl / d);
    if (d > 0) ap = fmin(ap, tau * dh / d);
    if (dzl < 0) ad = fmin(ad, -tau * zlu[i] / dzl);
    if (dzh < 0) ad = fmin(ad, -tau * zuu[i] / dzh);
  }
  if (i < m) {
    const double rd2 = rho * sigc[i] * sigc[i];
    const double d = (-gpsi_s[i] + rd2 * jdu[i]) / (rd2 + sig_s[i]);
    ds[i] = d;
    const double dl = s[i] - slo[i], dh = shi[i] - s[i];
    const double dzl = mu / dl - zls[i] - zls[i] / dl * d;
    const double dzh = mu / dh - zus[i] + zus[i] / dh * d;
    dz[2 * nu + i] = dzl;
    dz[2 * nu + m + i] = dzh;
    if (d < 0) ap = fmin(ap, -tau * dl / d);
    if (d > 0) ap = fmin(ap, tau * dh / d);
    if (dzl < 0) ad = fmin(ad, -tau * zls[i] / dzl);
    if (dzh < 0) ad = fmin(ad, -tau * zus[i] / dzh);
  }
  for (int off = 16; off > 0; off >>= 1) {
    ap = fmin(ap, __shfl_down_sync(0xffffffffu, ap, off));
    ad = fmin(ad, __shfl_down_sync(0xffffffffu, ad, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_min_pos(&red[0], ap);
    atomic_min_pos(&red[1], ad);
  }
}

__global__ void axpy2_kernel(int n, const double* x, const double* d, double a, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[i] + a * d[i];
}

__global__ void update_kernel(int nu, int m, double* u, const double* du, double* s, const double* ds,
                              double* zlu, double* zuu, double* zls, double* zus, const double* dz, double ap,
                              double ad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) {
    u[i] += ap * du[i];
    zlu[i] += ad * dz[i];
    zuu[i] += ad * dz[nu + i];
  }
  if (i < m) {
    s[i] += ap * ds[i];
    zls[i] += ad * dz[2 * nu + i];
    zus[i] += ad * dz[2 * nu + m + i];
  }
}

// Line-search terms: out[0] += sum log(w - w_lo) + log(w_hi - w) over w = (u, s)
// (the barrier is -mu times it), and, when gu is given, out[1] += grad psi^T d.
__global__ void ls_terms_kernel(int nu, int m, const double* u, const double* s, const double* ulo,
                                const double* uhi, const double* slo, const double* shi, const double* gu,
                                const double* du, const double* gs, const double* ds, double* out) {
  double b = 0.0, sl = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nu + m; i += gridDim.x * blockDim.x) {
    if (i < nu) {
      b += log(u[i] - ulo[i]) + log(uhi[i] - u[i]);
      if (gu) sl += gu[i] * du[i];
    } else {
      const int k = i - nu;
      b += log(s[k] - slo[k]) + log(shi[k] - s[k]);
      if (gu) sl += gs[k] * ds[k];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    b += __shfl_xor_sync(0xffffffffu, b, o);
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, b);
    if (gu) atomicAdd(out + 1, sl);
  }
}

// QP gradient after a step of the tracking QP (Sec. IV-C): the Hessian is
// constant, and the Newton system (H + Sigma) d = -grad psi gives H d =
// -grad psi - Sigma d, so grad q <- grad q + alpha (-grad psi - Sigma d).
__global__ void qp_grad_update_kernel(int nu, int m, double* gqu, double* gqs, const double* gpsi_u,
                                      const double* gpsi_s, const double* sig_u, const double* sig_s,
                                      const double* du, const double* ds, double alpha) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) gqu[i] += alpha * (-gpsi_u[i] - sig_u[i] * du[i]);
  if (i < m) gqs[i] += alpha * (-gpsi_s[i] - sig_s[i] * ds[i]);
}

// out[i] += a (x[i] - x0[i])  (the u-block regularisation delta enters grad q as delta (u - u_t))
__global__ void add_scaled_diff_kernel(int n, double* out, double a, const double* x, const double* x0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += a * (x[i] - x0[i]);
}

// w <- w0 + alpha (w - w0)  (a shortened tracking step)
__global__ void shrink_kernel(int n, double* w, const double* w0, double alpha) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = w0[i] + alpha * (w[i] - w0[i]);
}

#define SCK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
      return OPF_ECUDA;                                                             \
    }                                                                               \
  } while (0)

opf_status alloc_step(opf_ctx* c) {
  if (c->stepw) return OPF_OK;
  const int nu = c->h.nu, m = c->h.m, nx = c->h.nx, nb = c->h.nb;
  StepWork* w = new StepWork();
  w->nu = nu;
  w->m = m;
  const size_t sizes[] = {(size_t)nu * nu, (size_t)nu * nu, (size_t)nu, (size_t)m, (size_t)nu, (size_t)nu,
                          (size_t)m, (size_t)m, (size_t)m, (size_t)m, (size_t)nu, (size_t)nu, (size_t)m,
                          (size_t)nu, (size_t)m, (size_t)nx, (size_t)nx, (size_t)nu, (size_t)nx, (size_t)nb,
                          (size_t)nb, 2 * (size_t)nu + 2 * (size_t)m, 2, ((size_t)nu + 31) / 32 * 1024,
                          (size_t)m, 8};
  double** ptrs[] = {&w->S, &w->L, &w->gu, &w->gs, &w->sig_u, &w->gpsi_u, &w->sig_s, &w->gpsi_s, &w->omega,
                     &w->v, &w->r, &w->du, &w->ds, &w->Jtv, &w->Jdu, &w->b, &w->z, &w->ut, &w->xt,
                     &w->pd, &w->qd, &w->dz, &w->red, &w->Dinv, &w->strial, &w->lsv};
  const int np = sizeof(sizes) / sizeof(sizes[0]);
  size_t total = 0;
  for (int k = 0; k < np; k++) total += (sizes[k] + 31) & ~(size_t)31;
  total += 32 + (size_t)nu / 32 + 16;  // flag, dense-solve error and block flags (ints)
  if (cudaMalloc(&w->block, total * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    delete w;
    set_last_error("cannot allocate the reduced-Newton step workspace");
    return OPF_ENOMEM;
  }
  double* p = static_cast<double*>(w->block);
  for (int k = 0; k < np; k++) {
    *ptrs[k] = p;
    p += (sizes[k] + 31) & ~(size_t)31;
  }
  w->flag = reinterpret_cast<int*>(p);
  w->trsv_err = w->flag + 1;
  w->oz_err = w->flag + 2;
  w->trsv_flags = reinterpret_cast<unsigned*>(w->flag + 8);
  if (cudaMemset(w->flag, 0, (8 + (size_t)nu / 32 + 1) * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(w->block);
    delete w;
    set_last_error("cannot initialise the reduced-Newton step workspace");
    return OPF_ECUDA;
  }
  if (cudaMallocHost(&w->h_red, 2 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&w->h_ls, 8 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&w->h_flag, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    c->stepw = w;
    free_step_work(c);
    set_last_error("cannot allocate pinned step buffers");
    return OPF_ENOMEM;
  }
  if (cudaMalloc(&w->oz_e, sizeof(int) * (size_t)nu) != cudaSuccess ||
      cudaMalloc(&w->oz_d, (size_t)2 * 8 * GB * (size_t)oz_rows_tiled(nu)) != cudaSuccess) {
    cudaGetLastError();
    c->stepw = w;
    free_step_work(c);
    set_last_error("cannot allocate the emulated-update workspace");
    return OPF_ENOMEM;
  }
  {
    const opf_status so = setup_oz();
    if (so != OPF_OK) {
      c->stepw = w;
      free_step_work(c);
      return so;
    }
  }
  if (cudaStreamCreateWithFlags(&w->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->aux_go, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&w->aux_done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    c->stepw = w;
    free_step_work(c);
    set_last_error("cannot create the step's second stream");
    return OPF_ECUDA;
  }
  c->stepw = w;
  return OPF_OK;
}

// Blocked Cholesky in groups of GB = 128 columns.  Inside a group, 32-wide
// panels run right-looking in FP64 (diagonal block with its inverse, panel
// solve, update of the group's remaining columns); after the group, the rest of
// the trailing triangle takes the group's rank-128 update at once, emulated on
// the tensor cores (launch_oz_update: exact digit products, FP64 sums), or,
// with emulate false, as four rank-32 FP64 updates (chol_syrk_kernel over the
// whole trailing triangle, one per panel of the group).
opf_status launch_cholesky(opf_ctx* c, StepWork* w, double* A, int n, int* flag, bool emulate) {
  cudaStream_t s1 = c->stream;
  for (int c0 = 0; c0 < n; c0 += GB) {
    const int c1 = std::min(n, c0 + GB);
    for (int k0 = c0; k0 < c1; k0 += NB) {
      const int kb = std::min(NB, n - k0);
      SCK(launch_pdl(chol_diag_kernel, dim3(1), dim3(512), 0, s1, A, n, k0, kb, flag, w->Dinv));
      c->launches++;
      const int rest = n - k0 - kb;
      if (rest <= 0) break;
      {  // 8-row CTAs when they leave the busiest SM fewer rows than 16-row ones
        const int sm = std::max(1, c->sm_count);
        const int rows = ((nblk(rest, 8) + sm - 1) / sm) * 8 < ((nblk(rest, 16) + sm - 1) / sm) * 16 ? 8 : 16;
        SCK(launch_pdl(chol_trsm_kernel, dim3(nblk(rest, rows)), dim3(16 * rows), 0, s1, A, n, k0, kb, flag,
                       w->Dinv));
      }
      c->launches++;
      if (k0 + kb < c1) {  // the group's remaining columns, all rows below
        // a 32 x 32 tile is ~1,000 warp FP64 instructions (~10 us of one SM's
        // FP64 pipe); 16 x 16 tiles when they leave the busiest SM less work
        const long long t32 = (long long)nblk(c1 - k0 - kb, 32) * nblk(rest, 32);
        const long long t16 = (long long)nblk(c1 - k0 - kb, 16) * nblk(rest, 16);
        const int sm = std::max(1, c->sm_count);
        if ((t16 + sm - 1) / sm < 4 * ((t32 + sm - 1) / sm)) {
          const dim3 grid(nblk(c1 - k0 - kb, 16), nblk(rest, 16));
          SCK(launch_pdl(chol_syrk_kernel<16>, grid, dim3(256), 0, s1, A, n, k0, kb, flag, 2, 0, c1));
        } else {
          const dim3 grid(nblk(c1 - k0 - kb, 32), nblk(rest, 32));
          SCK(launch_pdl(chol_syrk_kernel<32>, grid, dim3(256), 0, s1, A, n, k0, kb, flag, 2, 0, c1));
        }
        c->launches++;
      }
    }
    if (c1 < n) {
      if (emulate) {
        OzEngine eng;
        eng.engine = c->oz_engine;
        eng.err = w->oz_err;
        eng.lim = c->wait_limit > 0 ? (long long)c->wait_limit : (1ll << 24);
        eng.sm_count = c->sm_count;
        launch_oz_update(s1, A, n, c0, c1 - c0, c1, w->oz_e, w->oz_d, flag, eng);
        c->launches += 2;
      } else {
        const int tiles = (n - c1 + 31) / 32;
        for (int k0 = c0; k0 < c1; k0 += NB) {
          const int kb = std::min(NB, c1 - k0);
          SCK(launch_pdl(chol_syrk_kernel<32>, dim3(tiles * (tiles + 1) / 2), dim3(256), 0, s1, A, n, k0, kb, flag,
                         0, c1 - k0 - kb, n));
          c->launches++;
        }
      }
    }
  }
  return OPF_OK;
}

// launch_cholesky on w->L as one graph launch (about three hundred kernels on
// the 9.2k grid), captured on the context's capture stream at first use and
// again when the wait limit or the update engine has changed since.
opf_status launch_cholesky_graph(opf_ctx* c, StepWork* w, int n, bool emulate) {
  const int e = emulate ? 1 : 0;
  const long long lim = c->wait_limit > 0 ? (long long)c->wait_limit : (1ll << 24);
  if (!w->chol_exec[e] || w->chol_lim[e] != lim || w->chol_engine[e] != c->oz_engine) {
    if (w->chol_exec[e]) {
      SCK(cudaStreamSynchronize(c->stream));
      cudaGraphExecDestroy(w->chol_exec[e]);
      w->chol_exec[e] = nullptr;
    }
    cudaStream_t user = c->stream;
    const long long l0 = c->launches;
    c->stream = c->cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    opf_status rc = OPF_OK;
    if (err == cudaSuccess) {
      rc = launch_cholesky(c, w, w->L, n, w->flag, emulate);
      err = cudaStreamEndCapture(c->cap_stream, &graph);
    }
    c->stream = user;
    w->chol_kernels[e] = c->launches - l0;
    c->launches = l0;
    if (rc != OPF_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    SCK(err);
    err = cudaGraphInstantiate(&w->chol_exec[e], graph, 0);
    cudaGraphDestroy(graph);
    SCK(err);
    w->chol_lim[e] = lim;
    w->chol_engine[e] = c->oz_engine;
  }
  SCK(cudaGraphLaunch(w->chol_exec[e], c->stream));
  c->launches += w->chol_kernels[e];
  return OPF_OK;
}

// L = S + delta I factorised in place in w->L; ok: no pivot was non-positive.
// Mode 1 (the default) emulates the trailing updates on the tensor cores.
// Mode 0 also factorises S + delta I again with FP64 trailing updates when a
// pivot fails, before the caller raises delta: the emulation errs by up to
// ~5 K u max_k|P_rk| max_k|P_ck| per element (relative to the rows' largest
// panel entries), where an FP64 update errs by ~K u sum_k |P_rk P_ck|, so on a
// Schur complement whose rows span many decades a pivot the FP64 update keeps
// positive could fail.  Mode 2: FP64 only.  fp64_runs counts the FP64
// factorisations.
opf_status factor_shifted(opf_ctx* c, StepWork* w, int nu, double delta, bool& ok, int& fp64_runs) {
  cudaStream_t stream = c->stream;
  auto run = [&](bool emulate) -> opf_status {
    add_diag_kernel<<<dim3(nblk(nu, 256), nu), 256, 0, stream>>>(w->L, w->S, nu, delta);
    SCK(cudaMemsetAsync(w->flag, 0, sizeof(int), stream));
    c->launches++;
    const opf_status rc = launch_cholesky_graph(c, w, nu, emulate);
    if (rc) return rc;
    if (!emulate) fp64_runs++;
    SCK(cudaMemcpyAsync(w->h_flag, w->flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, stream));
    SCK(cudaStreamSynchronize(stream));
    if (w->h_flag[2]) {  // a wait of the emulated update gave up: the factor is void
      SCK(cudaMemsetAsync(w->oz_err, 0, sizeof(int), stream));
      set_last_error("emulated Cholesky update: a bounded wait for the tensor cores gave up");
      return OPF_ETIMEOUT;
    }
    ok = !w->h_flag[0];
    return OPF_OK;
  };
  const opf_status rc = run(c->chol_mode != 2);
  if (rc || ok || c->chol_mode != 0) return rc;
  return run(false);
}

// Inertia correction: the first delta of the sequence delta_0 = d0, delta_t =
// d0 10^t (d0 > 0) or 1e-8 10^(t - 1) (d0 = 0), t <= max_raises, for which
// factor_shifted succeeds; L then holds that factorisation.  S + delta I
// positive definite implies it for every larger delta, so success is monotone
// in t and a bisection finds the same t as trying them in turn: the first
// nlinear candidates in turn, then bisection over the rest.  Callers take all
// of them in turn from a carried-over delta (which usually succeeds at once or
// after a raise or two, where a bisection over 24 candidates would cost more)
// and bisect after delta = 0 from a fresh start (the 9.2k grid then needs
// t = 17: 6 factorisations instead of 18).  raises = t; OPF_ENOTPD (with msg)
// when no candidate succeeds.
opf_status inertia_search(opf_ctx* c, StepWork* w, int nu, double d0, int max_raises, int nlinear,
                          const char* msg, double& delta, int& raises, int& factorisations, int& fp64_runs) {
  auto delta_at = [&](int t) {
    if (t == 0) return d0;
    return d0 > 0.0 ? d0 * std::pow(10.0, (double)t) : 1e-8 * std::pow(10.0, (double)(t - 1));
  };
  int last = -1;
  auto attempt = [&](int t, bool& ok) -> opf_status {
    ok = false;
    last = t;
    factorisations++;
    return factor_shifted(c, w, nu, delta_at(t), ok, fp64_runs);
  };
  int t_ok = -1, lo = -1;
  for (int t = 0; t < std::min(nlinear, max_raises + 1); t++) {
    bool ok = false;
    const opf_status rc = attempt(t, ok);
    if (rc) return rc;
    if (ok) {
      t_ok = t;
      break;
    }
    lo = t;
  }
  if (t_ok < 0) {
    int hi = max_raises + 1;  // past the last candidate: fails
    while (hi - lo > 1) {
      const int mid = lo + (hi - lo) / 2;
      bool ok = false;
      const opf_status rc = attempt(mid, ok);
      if (rc) return rc;
      if (ok) {
        hi = mid;
      } else {
        lo = mid;
      }
    }
    t_ok = hi;
    // L holds the last factorisation computed: redo the chosen one if that was
    // a failure; should the redo fail (success not monotone after all), go on in turn
    while (t_ok <= max_raises && last != t_ok) {
      bool ok = false;
      const opf_status rc = attempt(t_ok, ok);
      if (rc) return rc;
      if (!ok) t_ok++;
    }
    if (t_ok > max_raises) {
      set_last_error(msg);
      return OPF_ENOTPD;
    }
  }
  delta = delta_at(t_ok);
  raises = t_ok;
  return OPF_OK;
}

opf_status launch_chol_solve(opf_ctx* c, StepWork* w, double* A, int n, double* b) {
  const int nb = (n + 31) / 32;  // Dinv holds the diagonal blocks' inverses from the factorisation
  chol_upper_copy_kernel<<<dim3(nb, nb), 256, 0, c->stream>>>(A, n);
  c->launches++;
  int occ = 0;
  SCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chol_trsv_kernel<true>, 256, 0));
  const int grid = std::max(1, std::min(nb, occ * c->sm_count));
  for (int dir = 0; dir < 2; dir++) {
    unsigned epoch = ++w->trsv_epoch;
    const double* Dv = w->Dinv;
    long long lim = c->wait_limit > 0 ? (long long)c->wait_limit : (1ll << 24);
    void* args[] = {(void*)&A, (void*)&n, (void*)&Dv, (void*)&b, (void*)&w->trsv_flags, (void*)&epoch,
                    (void*)&w->trsv_err, (void*)&lim};
    SCK(cudaLaunchCooperativeKernel(dir == 0 ? (const void*)chol_trsv_kernel<true> : (const void*)chol_trsv_kernel<false>,
                                    dim3(grid), dim3(256), args, 0, c->stream));
    c->launches++;
  }
  return OPF_OK;
}

}  // namespace

namespace {

// The part of a reduced-Newton step before its Hessian: Sigma, the Schur
// weights omega, the first-order quantities with omega (gradient), grad psi and
// v.  *ps receives the parameters of the step's Schur Hessian.
opf_status step_begin(opf_ctx* c, const opf_al_params* p, opf_al_state* st, opf_al_params* ps_out) {
  if (!c || !p || !st) {
    set_last_error("ctx, params and state are required");
    return OPF_EINVAL;
  }
  if (!c->have_state) {
    set_last_error("no converged power flow on this context");
    return OPF_ESTATE;
  }
  {
    const opf_status fs = ensure_factors(c);
    if (fs != OPF_OK) return fs;
  }
  if (!p->sigma_c || !p->y || !st->u || !st->s || !st->zl_u || !st->zu_u || !st->zl_s || !st->zu_s ||
      !st->u_lo || !st->u_hi || !st->s_lo || !st->s_hi || !st->x || !(st->mu >= 0.0) || !(p->rho > 0.0)) {
    set_last_error("opf_al_step needs every state array, mu >= 0 and rho > 0");
    return OPF_EINVAL;
  }
  opf_status rc = alloc_step(c);
  if (rc) return rc;
  StepWork* w = c->stepw;
  const int nu = c->h.nu, m = c->h.m;
  cudaStream_t stream = c->stream;
  // phase boundaries: start, first order, Hessian, Schur rhs, Cholesky, solves, end of step (trial PF)
  cudaEvent_t* ev = w->ev;
  if (!ev[0])
    for (int k = 0; k < 7; k++) SCK(cudaEventCreate(&ev[k]));
  SCK(cudaEventRecord(ev[0], stream));
  // Sigma and the Schur weights omega (state only)
  step_sigma_kernel<<<nblk(std::max(nu, m), 256), 256, 0, stream>>>(
      nu, m, st->u, st->u_lo, st->u_hi, st->zl_u, st->zu_u, st->s, st->s_lo, st->s_hi, st->zl_s, st->zu_s,
      p->sigma_c, p->rho, w->sig_u, w->sig_s, w->omega);
  c->launches++;
  // first-order quantities once, with omega: grad_u, grad_s = -phi' (the gradient does not depend on omega)
  opf_al_params ps = *p;
  ps.s = st->s;
  ps.omega = w->omega;
  rc = opf_reduced_gradient(c, &ps, w->lsv, w->gu, w->gs, nullptr, nullptr, nullptr, nullptr);
  if (rc) return rc;
  SCK(cudaEventRecord(ev[1], stream));
  step_prep_kernel<<<nblk(std::max(nu, m), 256), 256, 0, stream>>>(
      nu, m, st->u, st->u_lo, st->u_hi, st->zl_u, st->zu_u, st->s, st->s_lo, st->s_hi, st->zl_s, st->zu_s,
      w->gu, w->gs, p->sigma_c, p->rho, st->mu, w->sig_u, w->gpsi_u, w->sig_s, w->gpsi_s, w->omega, w->v);
  c->launches++;
  *ps_out = ps;
  return OPF_OK;
}

// The part of a reduced-Newton step after its Hessian (in the step workspace's
// S): the Schur system, its Cholesky with the inertia correction, the solves,
// the slack and dual steps, the fraction to the boundary, the trial power flows
// and the update.  ms_hessian: the Hessian's device time, for info.
opf_status step_end(opf_ctx* c, const opf_al_params* p, opf_al_state* st, const opf_step_opts* o,
                    opf_step_info* info, double* du_out, double* ds_out, float ms_hessian) {
  StepWork* w = c->stepw;
  opf_status rc = OPF_OK;
  const int nu = c->h.nu, m = c->h.m, nx = c->h.nx, nb = c->h.nb;
  const int max_halvings = (o && o->max_halvings) ? o->max_halvings : 10;
  const int max_inertia = (o && o->max_inertia) ? o->max_inertia : 24;
  cudaStream_t stream = c->stream;
  cudaEvent_t* ev = w->ev;
  cudaEvent_t e0 = ev[0], e1 = ev[5];
  sym_diag_kernel<<<dim3(nblk(nu, 32), nblk(nu, 32)), 256, 0, stream>>>(w->S, nu, w->sig_u);
  c->launches++;
  // r = -grad_u psi - J^T v on the second stream, beside the Cholesky (it reads
  // the state and v, and writes the adjoint buffers, which the factorisation
  // does not touch); the solves below wait for it
  SCK(cudaEventRecord(w->aux_go, stream));
  SCK(cudaStreamWaitEvent(w->aux, w->aux_go, 0));
  c->stream = w->aux;
  launch_weighted_grad(c, w->v, w->Jtv);
  neg_sum_kernel<<<nblk(nu, 256), 256, 0, w->aux>>>(nu, w->gpsi_u, w->Jtv, w->r);
  c->launches++;
  c->stream = stream;
  SCK(cudaEventRecord(w->aux_done, w->aux));
  SCK(cudaEventRecord(ev[3], stream));
  // Cholesky with inertia correction (inertia_search)
  const double delta0 = (o && o->delta_start > 0.0) ? o->delta_start : 0.0;
  double delta = 0.0;
  int tries = 0, fp64_runs = 0, factorisations = 0;
  rc = inertia_search(c, w, nu, delta0, max_inertia, delta0 > 0.0 ? max_inertia + 1 : 1,
                      "S_uu not positive definite after the inertia corrections", delta, tries, factorisations,
                      fp64_runs);
  if (rc) {
    cudaStreamWaitEvent(stream, w->aux_done, 0);  // no work of this call outlives it
    return rc;
  }
  SCK(cudaStreamWaitEvent(stream, w->aux_done, 0));
  SCK(cudaEventRecord(ev[4], stream));
  SCK(cudaMemcpyAsync(w->du, w->r, nu * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  rc = launch_chol_solve(c, w, w->L, nu, w->du);
  if (rc) return rc;
  // J d_u: z = -G_x^{-1} G_u d_u, then the directional derivatives of c
  // (from the Hessian's first adjoints when its slabs still hold them)
  if (!launch_state_direction(c, w->du, w->z)) {
    gu_times_kernel<<<nblk(nb, 256), 256, 0, stream>>>(c->dn, c->btab, w->du, w->b);
    c->launches++;
    launch_solve1(c, w->b, w->z, false, -1.0);
  }
  jvp_branch_kernel<<<nblk(c->dn.nl, 256), 256, 0, stream>>>(c->dn, c->btab, c->flows, w->z, w->du, w->Jdu);
  jvp_bus_kernel<<<nblk(nb, 256), 256, 0, stream>>>(c->dn, c->btab, w->z, w->du, w->Jdu);
  c->launches += 2;
  // d_s, dual steps, fraction to the boundary
  const double tau = std::max(0.99, 1.0 - st->mu);
  const double one = 1.0;
  SCK(cudaMemcpyAsync(w->red, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
  SCK(cudaMemcpyAsync(w->red + 1, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
  step_finish_kernel<<<nblk(std::max(nu, m), 256), 256, 0, stream>>>(
      nu, m, st->u, w->du, st->u_lo, st->u_hi, st->zl_u, st->zu_u, st->s, st->s_lo, st->s_hi, st->zl_s,
      st->zu_s, w->gpsi_s, w->sig_s, w->Jdu, p->sigma_c, p->rho, st->mu, tau, w->ds, w->dz, w->red);
  c->launches++;
  SCK(cudaMemcpyAsync(w->h_red, w->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
  SCK(cudaMemcpyAsync(w->h_flag, w->trsv_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  SCK(cudaStreamSynchronize(stream));
  SCK(cudaGetLastError());
  if (*w->h_flag) {
    SCK(cudaMemsetAsync(w->trsv_err, 0, sizeof(int), stream));  // the next call starts clean
    set_last_error("dense triangular solve: a bounded block wait gave up");
    return OPF_ETIMEOUT;
  }
  double ap = w->h_red[0];
  const double ad = w->h_red[1];
  SCK(cudaEventRecord(e1, stream));
  // trial power flows with halving (loads kept from the current state)
  SCK(cudaMemcpyAsync(w->pd, c->pd, nb * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  SCK(cudaMemcpyAsync(w->qd, c->qd, nb * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  int halvings = 0;
  opf_pf_info pfi = {0, 0.0, 0.0};
  const bool ls = o && o->line_search;
  const int glg = std::max(1, std::min(nblk(nu + m, 256), 4 * c->sm_count));
  double psi0 = 0.0, slope = 0.0;
  if (ls) {  // psi at the current point and its slope along the step
    SCK(cudaMemsetAsync(w->lsv + 1, 0, 2 * sizeof(double), stream));
    ls_terms_kernel<<<glg, 256, 0, stream>>>(nu, m, st->u, st->s, st->u_lo, st->u_hi, st->s_lo, st->s_hi,
                                             w->gpsi_u, w->du, w->gpsi_s, w->ds, w->lsv + 1);
    c->launches++;
    SCK(cudaMemcpyAsync(w->h_ls, w->lsv, 3 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    SCK(cudaStreamSynchronize(stream));
    psi0 = w->h_ls[0] - st->mu * w->h_ls[1];
    slope = w->h_ls[2];
  }
  opf_al_params pt = *p;  // the AL at the trial point's slacks
  pt.s = w->strial;
  pt.omega = nullptr;
  for (;;) {
    axpy2_kernel<<<nblk(nu, 256), 256, 0, stream>>>(nu, st->u, w->du, ap, w->ut);
    // first-order predictor of the new state: x + alpha z, z = dx/du d_u (from J d_u)
    axpy2_kernel<<<nblk(nx, 256), 256, 0, stream>>>(nx, st->x, w->z, ap, w->xt);
    c->launches += 2;
    opf_status prc = opf_powerflow(c, w->ut, w->pd, w->qd, w->xt, nullptr, &pfi);
    if (prc == OPF_OK) {
      if (!ls || halvings >= max_halvings) break;
      // Armijo on the barrier function psi_mu = F + barrier at the trial point
      axpy2_kernel<<<nblk(m, 256), 256, 0, stream>>>(m, st->s, w->ds, ap, w->strial);
      c->launches++;
      launch_eval_F(c, &pt, w->lsv + 3);
      SCK(cudaMemsetAsync(w->lsv + 4, 0, sizeof(double), stream));
      ls_terms_kernel<<<glg, 256, 0, stream>>>(nu, m, w->ut, w->strial, st->u_lo, st->u_hi, st->s_lo, st->s_hi,
                                               nullptr, nullptr, nullptr, nullptr, w->lsv + 4);
      c->launches++;
      SCK(cudaMemcpyAsync(w->h_ls + 3, w->lsv + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
      SCK(cudaStreamSynchronize(stream));
      if (w->h_ls[3] - st->mu * w->h_ls[4] <= psi0 + 1e-4 * ap * slope) break;
    } else {
      if (prc != OPF_ENOCONV && prc != OPF_ESINGULAR) return prc;
      if (halvings >= max_halvings) {
        set_last_error("no trial control with a converged power flow after the halvings");
        return OPF_ENOCONV;
      }
    }
    ap *= 0.5;
    halvings++;
  }
  if (du_out) SCK(cudaMemcpyAsync(du_out, w->du, nu * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  if (ds_out) SCK(cudaMemcpyAsync(ds_out, w->ds, m * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  update_kernel<<<nblk(std::max(nu, m), 256), 256, 0, stream>>>(nu, m, st->u, w->du, st->s, w->ds, st->zl_u,
                                                                st->zu_u, st->zl_s, st->zu_s, w->dz, ap, ad);
  c->launches++;
  SCK(cudaMemcpyAsync(st->x, w->xt, nx * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  SCK(cudaEventRecord(ev[6], stream));
  SCK(cudaStreamSynchronize(stream));
  SCK(cudaGetLastError());
  if (info) {
    float t[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 6; k++) cudaEventElapsedTime(&t[k], ev[k], ev[k + 1]);
    info->ms_first_order = t[0];
    info->ms_rhs = t[2];
    info->ms_cholesky = t[3];
    info->ms_solve = t[4];
    info->ms_trial = t[5];
    info->alpha_p = ap;
    info->alpha_d = ad;
    info->delta = delta;
    info->halvings = halvings;
    info->inertia_tries = tries;
    info->cholesky_fp64 = fp64_runs;
    info->factorisations = factorisations;
    info->pf_iterations = pfi.iterations;
    info->ms_hessian = ms_hessian;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    info->ms_total = ms;
    info->du_inf = info->ds_inf = 0.0;
  }
  return OPF_OK;
}

}  // namespace

extern "C" opf_status opf_al_step(opf_ctx* c, const opf_al_params* p, opf_al_state* st,
                                  const opf_step_opts* o, opf_step_info* info, double* du_out,
                                  double* ds_out) {
  opf_al_params ps;
  opf_status rc = step_begin(c, p, st, &ps);
  if (rc) return rc;
  StepWork* w = c->stepw;
  const int block_k = o ? o->block_k : 0;
  // S_uu = H(omega) + Sigma_u (symmetrised), on the first-order quantities just evaluated
  opf_hess_opts ho = {block_k, 0, 0, 0, 0, 0, 1};
  opf_hess_info hi;
  rc = opf_reduced_hessian(c, &ps, &ho, w->S, &hi);
  if (rc) return rc;
  SCK(cudaEventRecord(w->ev[2], c->stream));
  return step_end(c, p, st, o, info, du_out, ds_out, hi.ms_total);
}

// ---------------------------------------------------------------- tracking QP

namespace {

opf_status alloc_qp(opf_ctx* c, StepWork* w) {
  if (w->qp_block) return OPF_OK;
  const size_t nu = c->h.nu, m = c->h.m, nx = c->h.nx;
  const size_t n = 2 * (nu + 32) + 3 * (m + 32) + nx + 32 + 8;
  if (cudaMalloc(&w->qp_block, n * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&w->h_kred, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (w->qp_block) cudaFree(w->qp_block);
    w->qp_block = nullptr;
    set_last_error("cannot allocate the tracking QP workspace");
    return OPF_ENOMEM;
  }
  double* q = static_cast<double*>(w->qp_block);
  auto take = [&](size_t k) {
    double* r = q;
    q += (k + 31) & ~(size_t)31;
    return r;
  };
  w->gqu = take(nu);
  w->u0 = take(nu);
  w->gqs = take(m);
  w->s0 = take(m);
  w->cv = take(m);
  w->x0 = take(nx);
  w->kred = take(8);
  return OPF_OK;
}

}  // namespace

extern "C" opf_status opf_tracking_update(opf_ctx* c, const opf_al_params* p, double* y, opf_al_state* st,
                                          const opf_qp_opts* o, opf_qp_info* info) {
  if (!c || !p || !y || !st || !p->sigma_c || !st->u || !st->s || !st->zl_u || !st->zu_u || !st->zl_s ||
      !st->zu_s || !st->u_lo || !st->u_hi || !st->s_lo || !st->s_hi || !st->x) {
    set_last_error("ctx, params (with sigma_c), y and every state array are required");
    return OPF_EINVAL;
  }
  if (!c->have_state) {
    set_last_error("no converged power flow on this context");
    return OPF_ESTATE;
  }
  if (!(p->rho > 0.0) || !(st->mu > 0.0)) {
    set_last_error("opf_tracking_update needs rho > 0 and mu > 0");
    return OPF_EINVAL;
  }
  {
    const opf_status fs = ensure_factors(c);
    if (fs != OPF_OK) return fs;
  }
  opf_status rc = alloc_step(c);
  if (rc) return rc;
  StepWork* w = c->stepw;
  rc = alloc_qp(c, w);
  if (rc) return rc;
  const int nu = c->h.nu, m = c->h.m, nx = c->h.nx, nb = c->h.nb;
  const int max_it = (o && o->max_it > 0) ? o->max_it : 50;
  const double tol = (o && o->tol > 0.0) ? o->tol : 1e-6;
  const int block_k = o ? o->block_k : 0;
  const int max_halvings = (o && o->max_halvings) ? o->max_halvings : 10;
  const int max_inertia = (o && o->max_inertia) ? o->max_inertia : 24;
  cudaStream_t stream = c->stream;
  cudaEvent_t* ev = w->ev;
  if (!ev[0])
    for (int k = 0; k < 7; k++) SCK(cudaEventCreate(&ev[k]));
  SCK(cudaEventRecord(ev[0], stream));
  const int gb = nblk(std::max(nu, m), 256);
  // the linearisation point w_t, its state, and g_t = grad L_rho(w_t; y) = grad q(0)
  opf_al_params pt = *p;
  pt.y = y;
  pt.s = st->s;
  pt.omega = nullptr;
  rc = opf_reduced_gradient(c, &pt, nullptr, w->gqu, w->gqs, nullptr, nullptr, nullptr, nullptr);
  if (rc) return rc;
  SCK(cudaMemcpyAsync(w->u0, st->u, nu * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  SCK(cudaMemcpyAsync(w->s0, st->s, m * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  SCK(cudaMemcpyAsync(w->x0, st->x, nx * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  pt.s = w->s0;  // the Hessian's first-order weights stay those of w_t
  // every Hessian of this QP is taken at w_t: after the first, the tiles start
  // from the first adjoints their slabs kept (the factors do not change until
  // the trial power flows after the iterations)
  // and the same state and first-order weights (pt: y, s_t): after the first,
  // the Hessian entry refreshes omega only (launch_omega)
  struct ZReuseOff {
    opf_ctx* c;
    ~ZReuseOff() { c->z_reuse = c->fo_reuse = false; }
  } z_reuse_off{c};
  double mu = st->mu, delta = (o && o->delta_start > 0.0) ? o->delta_start : 0.0;
  double e_mu = 0.0, e_0 = 0.0, ap = 0.0, ad = 0.0, kkt_first = 0.0, ap_min = 1.0;
  float ms_hess = 0.f, ms_chol = 0.f;
  int it = 0, increases = 0, fp64_runs = 0;
  // convexity: the smallest delta of {delta_start or 0, 1e-8, 1e-7, ...} with H_uu + delta I
  // positive definite (H_uu = H(0), no Gauss-Newton weights), so that the QP is convex
  // (skipped with inertia_only: delta then grows only where an iteration's S needs it)
  if (!(o && o->inertia_only)) {
    SCK(cudaMemsetAsync(w->omega, 0, m * sizeof(double), stream));
    SCK(cudaMemsetAsync(w->sig_u, 0, nu * sizeof(double), stream));
    opf_al_params p0 = pt;
    p0.omega = w->omega;
    opf_hess_opts ho = {block_k, 0, 0, 0, 0, 0, 0};
    opf_hess_info hi;
    rc = opf_reduced_hessian(c, &p0, &ho, w->S, &hi);
    if (rc) return rc;
    c->z_reuse = c->fo_reuse = true;
    ms_hess += hi.ms_total;
    sym_diag_kernel<<<dim3(nblk(nu, 32), nblk(nu, 32)), 256, 0, stream>>>(w->S, nu, w->sig_u);
    c->launches++;
    SCK(cudaEventRecord(ev[1], stream));
    int raises = 0, nfac = 0;
    rc = inertia_search(c, w, nu, delta, max_inertia, delta > 0.0 ? max_inertia + 1 : 1,
                        "tracking QP: H_uu not positive definite after the inertia corrections", delta, raises, nfac,
                        fp64_runs);
    if (rc) return rc;
    increases += raises;
    SCK(cudaEventRecord(ev[2], stream));
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[1], ev[2]);
    ms_chol += t;
  }
  const double delta_convex = delta;
  for (it = 0;; it++) {
    SCK(cudaMemsetAsync(w->kred, 0, 4 * sizeof(double), stream));
    launch_al_kkt(c, w->gqu, w->gqs, st, nullptr, nullptr, mu, w->kred);
    SCK(cudaMemcpyAsync(w->h_kred, w->kred, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    SCK(cudaStreamSynchronize(stream));
    e_mu = std::max(w->h_kred[0], w->h_kred[1]);
    e_0 = std::max(w->h_kred[0], w->h_kred[2]);
    if (it == 0) kkt_first = e_0;
    if (e_0 <= tol || it == max_it) break;
    if (e_mu <= 10.0 * mu) mu = std::max(tol / 10.0, std::min(0.2 * mu, std::pow(mu, 1.5)));
    step_prep_kernel<<<gb, 256, 0, stream>>>(nu, m, st->u, st->u_lo, st->u_hi, st->zl_u, st->zu_u, st->s, st->s_lo,
                                             st->s_hi, st->zl_s, st->zu_s, w->gqu, w->gqs, p->sigma_c, p->rho, mu,
                                             w->sig_u, w->gpsi_u, w->sig_s, w->gpsi_s, w->omega, w->v);
    c->launches++;
    // S = H(omega) + Sigma_u at the fixed linearisation point (eq. schur_matrix)
    opf_al_params ps = pt;
    ps.omega = w->omega;
    opf_hess_opts ho = {block_k, 0, 0, 0, 0, 0, 0};
    opf_hess_info hi;
    rc = opf_reduced_hessian(c, &ps, &ho, w->S, &hi);
    if (rc) return rc;
    c->z_reuse = c->fo_reuse = true;
    ms_hess += hi.ms_total;
    sym_diag_kernel<<<dim3(nblk(nu, 32), nblk(nu, 32)), 256, 0, stream>>>(w->S, nu, w->sig_u);
    // r = -grad_u psi - J^T v
    launch_weighted_grad(c, w->v, w->Jtv);
    neg_sum_kernel<<<nblk(nu, 256), 256, 0, stream>>>(nu, w->gpsi_u, w->Jtv, w->r);
    c->launches += 2;
    // Cholesky; the QP's u-block regularisation delta only grows
    SCK(cudaEventRecord(ev[1], stream));
    const double d_old = delta;
    {
      int raises = 0, nfac = 0;
      rc = inertia_search(c, w, nu, delta, max_inertia, delta > 0.0 ? max_inertia + 1 : 1,
                          "tracking QP: S_uu not positive definite after the inertia corrections", delta, raises,
                          nfac, fp64_runs);
      if (rc) return rc;
      increases += raises;
    }
    SCK(cudaEventRecord(ev[2], stream));
    {
      float t = 0.f;
      cudaEventSynchronize(ev[2]);
      cudaEventElapsedTime(&t, ev[1], ev[2]);
      ms_chol += t;
    }
    if (delta != d_old) {  // the QP's Hessian gained (delta - d_old) I on the u-block
      const double dd = delta - d_old;
      add_scaled_diff_kernel<<<nblk(nu, 256), 256, 0, stream>>>(nu, w->gqu, dd, st->u, w->u0);
      add_scaled_diff_kernel<<<nblk(nu, 256), 256, 0, stream>>>(nu, w->gpsi_u, dd, st->u, w->u0);
      add_scaled_diff_kernel<<<nblk(nu, 256), 256, 0, stream>>>(nu, w->r, -dd, st->u, w->u0);
      c->launches += 3;
    }
    SCK(cudaMemcpyAsync(w->du, w->r, nu * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    rc = launch_chol_solve(c, w, w->L, nu, w->du);
    if (rc) return rc;
    // J d_u
    if (!launch_state_direction(c, w->du, w->z)) {
      gu_times_kernel<<<nblk(nb, 256), 256, 0, stream>>>(c->dn, c->btab, w->du, w->b);
      c->launches++;
      launch_solve1(c, w->b, w->z, false, -1.0);
    }
    jvp_branch_kernel<<<nblk(c->dn.nl, 256), 256, 0, stream>>>(c->dn, c->btab, c->flows, w->z, w->du, w->Jdu);
    jvp_bus_kernel<<<nblk(nb, 256), 256, 0, stream>>>(c->dn, c->btab, w->z, w->du, w->Jdu);
    c->launches += 2;
    const double tau = std::max(0.99, 1.0 - mu);
    const double one = 1.0;
    SCK(cudaMemcpyAsync(w->red, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
    SCK(cudaMemcpyAsync(w->red + 1, &one, sizeof(double), cudaMemcpyHostToDevice, stream));
    step_finish_kernel<<<gb, 256, 0, stream>>>(nu, m, st->u, w->du, st->u_lo, st->u_hi, st->zl_u, st->zu_u, st->s,
                                               st->s_lo, st->s_hi, st->zl_s, st->zu_s, w->gpsi_s, w->sig_s, w->Jdu,
                                               p->sigma_c, p->rho, mu, tau, w->ds, w->dz, w->red);
    c->launches++;
    SCK(cudaMemcpyAsync(w->h_red, w->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    SCK(cudaMemcpyAsync(w->h_flag, w->trsv_err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    SCK(cudaStreamSynchronize(stream));
    if (*w->h_flag) {
      SCK(cudaMemsetAsync(w->trsv_err, 0, sizeof(int), stream));
      set_last_error("dense triangular solve: a bounded block wait gave up");
      return OPF_ETIMEOUT;
    }
    ap = w->h_red[0];
    ad = w->h_red[1];
    ap_min = std::min(ap_min, ap);
    update_kernel<<<gb, 256, 0, stream>>>(nu, m, st->u, w->du, st->s, w->ds, st->zl_u, st->zu_u, st->zl_s, st->zu_s,
                                          w->dz, ap, ad);
    qp_grad_update_kernel<<<gb, 256, 0, stream>>>(nu, m, w->gqu, w->gqs, w->gpsi_u, w->gpsi_s, w->sig_u, w->sig_s,
                                                  w->du, w->ds, ap);
    c->launches += 2;
  }
  SCK(cudaEventRecord(ev[3], stream));
  // w_{t+1}: the power flow at the QP's controls (loads of the current state), the
  // step toward it halved until it converges
  SCK(cudaMemcpyAsync(w->pd, c->pd, nb * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  SCK(cudaMemcpyAsync(w->qd, c->qd, nb * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  int halvings = 0;
  opf_pf_info pfi = {0, 0.0, 0.0};
  for (;;) {
    SCK(cudaMemcpyAsync(w->xt, w->x0, nx * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    const opf_status prc = opf_powerflow(c, st->u, w->pd, w->qd, w->xt, nullptr, &pfi);
    if (prc == OPF_OK) break;
    if (prc != OPF_ENOCONV && prc != OPF_ESINGULAR) return prc;
    if (halvings >= max_halvings) {
      set_last_error("tracking update: no control toward the QP solution with a converged power flow");
      return OPF_ENOCONV;
    }
    shrink_kernel<<<nblk(nu, 256), 256, 0, stream>>>(nu, st->u, w->u0, 0.5);
    shrink_kernel<<<nblk(m, 256), 256, 0, stream>>>(m, st->s, w->s0, 0.5);
    c->launches += 2;
    halvings++;
  }
  SCK(cudaMemcpyAsync(st->x, w->xt, nx * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  // y_{t+1} = y_t + rho D_c (c_t(u_{t+1}) - s_{t+1})
  opf_al_params pn = *p;
  pn.y = y;
  pn.s = st->s;
  pn.omega = nullptr;
  rc = opf_reduced_gradient(c, &pn, nullptr, nullptr, nullptr, w->cv, nullptr, nullptr, nullptr);
  if (rc) return rc;
  launch_al_dual_update(c, y, p->rho, p->sigma_c, w->cv, st->s);
  SCK(cudaEventRecord(ev[4], stream));
  SCK(cudaStreamSynchronize(stream));
  SCK(cudaGetLastError());
  st->mu = mu;
  if (info) {
    info->qp_iterations = it;
    info->halvings = halvings;
    info->pf_iterations = pfi.iterations;
    info->inertia_increases = increases;
    info->cholesky_fp64 = fp64_runs;
    info->delta = delta;
    info->delta_convex = delta_convex;
    info->kkt = e_0;
    info->kkt_first = kkt_first;
    info->alpha_p_min = ap_min;
    info->mu = mu;
    info->alpha_p = ap;
    info->ms_hessian = ms_hess;
    info->ms_cholesky = ms_chol;
    cudaEventElapsedTime(&info->ms_total, ev[0], ev[4]);
    cudaEventElapsedTime(&info->ms_qp, ev[0], ev[3]);
  }
  return OPF_OK;
}

// ---------------------------------------------------------------- batched steps

extern "C" opf_status opf_al_step_batched(opf_ctx* const* ctxs, int n, const opf_al_params* params,
                                          opf_al_state* states, const double* const* pd,
                                          const double* const* qd, const opf_step_opts* o,
                                          opf_step_info* infos, opf_status* status, opf_batch_info* binfo) {
  if (!ctxs || n < 1 || !params || !states) {
    set_last_error("ctxs, params and states are required, n >= 1");
    return OPF_EINVAL;
  }
  for (int k = 0; k < n; k++) {
    if (!ctxs[k]) {
      set_last_error("null context in the batch");
      return OPF_EINVAL;
    }
    if (ctxs[k]->device != ctxs[0]->device) {
      set_last_error("all contexts of a batch must be on one device");
      return OPF_EINVAL;
    }
    for (int j = 0; j < k; j++)
      if (ctxs[j] == ctxs[k]) {
        set_last_error("a context appears twice in the batch");
        return OPF_EINVAL;
      }
  }
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  // every context works on a stream of its own during the call (contexts created on
  // one stream would otherwise serialise the host threads' work): it starts after
  // the work already on the context's stream, and that stream waits for it at the end
  std::vector<cudaStream_t> caller(n);
  for (int k = 0; k < n; k++) {
    opf_ctx* c = ctxs[k];
    if (!c->worker) {
      if (cudaStreamCreateWithFlags(&c->worker, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->worker_ev[0], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->worker_ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cannot create a context's worker stream");
        return OPF_ECUDA;
      }
    }
    caller[k] = c->stream;
    SCK(cudaEventRecord(c->worker_ev[0], c->stream));
    SCK(cudaStreamWaitEvent(c->worker, c->worker_ev[0], 0));
    c->stream = c->worker;
  }
  auto restore = [&]() {
    for (int k = 0; k < n; k++) {
      opf_ctx* c = ctxs[k];
      cudaEventRecord(c->worker_ev[1], c->worker);
      cudaStreamWaitEvent(caller[k], c->worker_ev[1], 0);
      c->stream = caller[k];
    }
  };
  // contexts by decreasing work (longest processing time first) for the host threads
  std::vector<int> order(n);
  for (int k = 0; k < n; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)ctxs[a]->dn.nnz * ctxs[a]->h.nu > (long long)ctxs[b]->dn.nnz * ctxs[b]->h.nu;
  });
  std::vector<opf_status> st(n, OPF_OK);
  std::vector<std::string> msg(n);
  std::vector<opf_al_params> ps(n);
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nthreads = (int)std::min<unsigned>((unsigned)n, std::min(hw, 32u));
  const int dev = ctxs[0]->device;
  // run f(k) for every context on nthreads host threads, largest first; each
  // context's work is ordered on its own stream, so the GPU overlaps them
  auto parallel = [&](auto&& f) {
    std::atomic<int> next(0);
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; t++)
      pool.emplace_back([&]() {
        cudaSetDevice(dev);
        for (int i = next++; i < n; i = next++) {
          const int k = order[i];
          if (st[k] != OPF_OK) continue;
          st[k] = f(k);
          if (st[k] != OPF_OK) msg[k] = opf_last_error();
        }
      });
    for (auto& th : pool) th.join();
  };
  // (A) power flow at the snapshot's loads, then the step up to its Hessian
  parallel([&](int k) -> opf_status {
    opf_ctx* c = ctxs[k];
    opf_al_state* s = &states[k];
    if (pd && pd[k]) {
      opf_pf_info pfi;
      const opf_status r = opf_powerflow(c, s->u, pd[k], qd ? qd[k] : nullptr, s->x, nullptr, &pfi);
      if (r) return r;
    }
    const opf_status r = step_begin(c, &params[k], s, &ps[k]);
    if (r) return r;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? OPF_OK : OPF_ECUDA;
  });
  const auto t1 = clk::now();
  // (B) every live context's Schur Hessian in one persistent launch
  std::vector<opf_ctx*> live;
  std::vector<opf_al_params> lp;
  std::vector<double*> lh;
  for (int k : order)
    if (st[k] == OPF_OK) {
      live.push_back(ctxs[k]);
      lp.push_back(ps[k]);
      lh.push_back(ctxs[k]->stepw->S);
    }
  float ms_hess = 0.f;
  opf_hess_info hi = {};
  if (!live.empty()) {
    opf_hess_opts ho = {o ? o->block_k : 0, 0, 0, 0, 0, 0, 1};
    const opf_status r = opf_reduced_hessian_batched(live.data(), (int)live.size(), lp.data(), lh.data(), &ho, &hi);
    if (r) {
      restore();
      return r;
    }
    ms_hess = hi.ms_total;
    for (opf_ctx* c : live) cudaEventRecord(c->stepw->ev[2], c->stream);
  }
  const auto t2 = clk::now();
  // (C) Cholesky, solves, fraction to the boundary, trial power flows, update
  parallel([&](int k) -> opf_status {
    return step_end(ctxs[k], &params[k], &states[k], o, infos ? &infos[k] : nullptr, nullptr, nullptr, ms_hess);
  });
  const auto t3 = clk::now();
  restore();
  opf_status first = OPF_OK;
  int failed = 0;
  for (int k = 0; k < n; k++) {
    if (status) status[k] = st[k];
    if (st[k] != OPF_OK) {
      failed++;
      if (first == OPF_OK) {
        first = st[k];
        set_last_error("context " + std::to_string(k) + ": " + msg[k]);
      }
    }
  }
  if (binfo) {
    auto ms = [](clk::time_point a, clk::time_point b) {
      return (float)std::chrono::duration<double, std::milli>(b - a).count();
    };
    binfo->ms_powerflow_first_order = ms(t0, t1);
    binfo->ms_hessians = ms(t1, t2);
    binfo->ms_steps = ms(t2, t3);
    binfo->ms_total = ms(t0, t3);
    binfo->hessian_tiles = hi.tiles;
    binfo->host_threads = nthreads;
    binfo->failed = failed;
  }
  return first;
}

extern "C" opf_status opf_set_cholesky_mode(opf_ctx* c, int mode) {
  if (!c || mode < 0 || mode > 2) {
    set_last_error("ctx is required and mode must be 0, 1 or 2");
    return OPF_EINVAL;
  }
  c->chol_mode = mode;
  return OPF_OK;
}

extern "C" opf_status opf_set_update_engine(opf_ctx* c, int engine) {
  if (!c || engine < 0 || engine > 2) {
    set_last_error("ctx is required and engine must be 0 (tcgen05 for large updates), 1 (mma.sync) or 2 (tcgen05)");
    return OPF_EINVAL;
  }
  c->oz_engine = engine;
  return OPF_OK;
}
