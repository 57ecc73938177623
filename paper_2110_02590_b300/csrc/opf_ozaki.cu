// FP64 rank-K updates of a lower triangle, C -= P P^T, emulated exactly on the
// bf16 tensor cores (the trailing updates of the Schur-complement Cholesky in
// the reduced-Newton step, Prop. 3).
//
// Ozaki splitting: every row r of P (K <= 128 columns) is written in fixed
// point against its own power of two, |P_rk| < 2^E_r, as eight signed 7-bit
// digits, P_rk = sum_s d_s(r, k) 2^(E_r - 7 (s + 1)) + tail, |tail| < 2^(E_r - 56).
// The digits are integers of magnitude <= 127, exact in bf16, and a product
// of two is below 2^14, so for each level t = s + s' (eight levels, at most
// eight digit pairs each) the sum over the K <= 128 columns stays below 2^24:
// the tensor core's FP32 accumulation is exact in any order.  The FP64 result
// is then sum_t 2^(E_r + E_c - 14 - 7 t) acc_t, summed in FP64.  Levels t >= 8
// (at most 7 digit pairs at level 8, each further level 2^-7 smaller) and the
// digit tails (below 2^(E_r - 56)) are dropped: each of the K products errs by
// less than 9.1 2^(E_r + E_c - 56) < 4.6 u max_k|P_rk| max_k|P_ck| (u = 2^-53,
// 2^E_r <= 2 max_k|P_rk|), so an element of the update errs by less than
// 5 K u max_k|P_rk| max_k|P_ck| before the final FP64 roundings.  The bound is
// relative to the rows' largest entries, not to sum_k |P_rk P_ck| as an FP64
// dot product's: the small entries of a row with a wide dynamic range lose
// relative accuracy.
//
// The digits are computed with integer shifts of the FP64 bit patterns (no
// rounding step), and the tensor-core work is 36 digit pairs per output: the
// B300's bf16 rate (~1.1 PFLOP/s for mma.sync in registers) against its FP64
// rate (~1 TFLOP/s) makes this ~10-30 times faster than FP64 FMAs.

#include <cuda_bf16.h>

#include <algorithm>

#include <cstdint>

#include "opf_internal.h"

namespace opf {

namespace {

constexpr int OZ_S = 8;       // digits per value
constexpr int OZ_TILE = 64;   // output tile (rows and columns)
constexpr int OZ_KC = 32;     // columns staged per pass
constexpr int OZ_PAD = 40;    // bf16 per staged row (32 + 8: conflict-free fragment loads)

// |x| < 2^E for x != 0: the exponent of the bit above the leading one
__device__ __forceinline__ int exp_bound(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const int ef = (int)(b >> 52);
  if (ef) return ef - 1022;
  return (64 - __clzll((long long)b)) - 1074;  // subnormal
}

// floor(|x| 2^(56 - E)) for |x| < 2^E, from the bit pattern
__device__ __forceinline__ unsigned long long fixed56(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const int ef = (int)(b >> 52);
  const unsigned long long mant = (b & 0x000fffffffffffffull) | (ef ? (1ull << 52) : 0ull);
  const int ex = ef ? ef - 1075 : -1074;  // |x| = mant 2^ex
  const int sh = ex + 56 - E;
  if (sh >= 0) return mant << sh;
  return (-sh >= 64) ? 0ull : (mant >> (-sh));
}

}  // namespace

// Digits of P = A[r0 : r0 + M, c0 : c0 + K] (column-major A, leading dimension
// n): E[r] and D[s][r][k] (bf16, row-major, K per row).  One CTA per 32 rows,
// its 32 warps over the columns; the digits pass through shared memory so that both
// the reads (along rows) and the writes (along columns) coalesce.
__global__ void __launch_bounds__(1024) oz_slice_kernel(const double* __restrict__ A, int n, int c0, int K, int r0,
                                                      int M, int* __restrict__ E, __nv_bfloat16* __restrict__ D,
                                                      const int* flag) {
  pdl_wait();
  if (*flag) return;
  __shared__ int emax_s[32][32];
  __shared__ __nv_bfloat16 dig[OZ_S][32][33];  // [digit][column in the pass][row]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  const bool live = r < M;
  int em = -4096;
  const int nw = blockDim.x >> 5;
  for (int k = w; k < K; k += nw) {
    const double x = live ? A[(size_t)(c0 + k) * n + r0 + r] : 0.0;
    if (x != 0.0) em = max(em, exp_bound(x));
  }
  emax_s[w][lane] = em;
  __syncthreads();
  if (w == 0) {
    int m = emax_s[0][lane];
    for (int q = 1; q < nw; q++) m = max(m, emax_s[q][lane]);
    if (live) E[r] = m;
    emax_s[0][lane] = m;
  }
  __syncthreads();
  const int er = emax_s[0][lane];
  for (int kt = 0; kt < K; kt += 32) {
    for (int kk = w; kk < 32; kk += nw) {
      const int k = kt + kk;
      const double x = (live && k < K) ? A[(size_t)(c0 + k) * n + r0 + r] : 0.0;
      const unsigned long long q = (x != 0.0) ? fixed56(x, er) : 0ull;
      const bool neg = x < 0.0;
#pragma unroll
      for (int s = 0; s < OZ_S; s++) {
        const int d = (int)((q >> (49 - 7 * s)) & 127ull);
        dig[s][kk][lane] = __int2bfloat16_rn(neg ? -d : d);
      }
    }
    __syncthreads();
    for (int q = w; q < OZ_S * 32; q += nw) {
      const int s = q >> 5, rr = q & 31, row = blockIdx.x * 32 + rr;
      if (row < M && kt + lane < K) D[((size_t)s * M + row) * K + kt + lane] = dig[s][lane][rr];
    }
    __syncthreads();
  }
  pdl_trigger();
}

namespace {

__device__ __forceinline__ void mma_bf16(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void ldsm_x4(unsigned* r, const unsigned short* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void cp16(unsigned short* dst, const void* src, bool in) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = in ? 16 : 0;  // zero fill past the last row
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(sz) : "memory");
}

constexpr int OZ_STAGE = 2 * OZ_S * OZ_TILE * OZ_PAD;  // bf16 per pipeline stage (tiles A and B)

// Digits [0, NSL) of 64 rows from row0, columns [kt, kt + 32), into one stage.
template <int NSL>
__device__ __forceinline__ void oz_issue(unsigned short* S, const __nv_bfloat16* __restrict__ D, int M, int K,
                                         int rowA, int rowB, int kt) {
  constexpr int pieces = 2 * NSL * OZ_TILE * 4;  // 16-byte pieces (4 per staged row)
  for (int q = threadIdx.x; q < pieces; q += blockDim.x) {
    const int half = q / (NSL * OZ_TILE * 4), rem = q - half * NSL * OZ_TILE * 4;
    const int s = rem / (OZ_TILE * 4), rem2 = rem - s * OZ_TILE * 4, rr = rem2 >> 2, pc = rem2 & 3;
    const int row = (half ? rowB : rowA) + rr;
    const bool in = row < M;
    const __nv_bfloat16* src = D + ((size_t)s * M + (in ? row : 0)) * K + kt + pc * 8;
    cp16(S + ((size_t)(half * OZ_S + s) * OZ_TILE + rr) * OZ_PAD + pc * 8, src, in);
  }
}

}  // namespace

// One 64 x 64 tile: all eight levels in one pass over the K columns (two
// cp.async stages of all eight digit planes of both row blocks).  Warps 4 x 4,
// each 16 x 16 outputs as one m16 x two n8 tiles: per 16 columns a warp holds
// the eight digits' B fragments in registers, then takes each A digit once and
// issues its pairs (digit i with digits j <= 7 - i) into acc[i + j].  The
// FP32 level sums are exact integers; levels 0-3 and 4-7 fold into exact
// 64-bit integers, which convert to FP64 exactly and meet in one FMA.
__device__ __forceinline__ void oz_tile(double* A, int n, int r0, int M, int K, const __nv_bfloat16* __restrict__ D,
                                        const int* __restrict__ E, unsigned short* sm, int bi, int bj) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wr = warp >> 2, wc = warp & 3;
  const int g = lane >> 2, tq = lane & 3;
  const int rowA = bi * OZ_TILE, rowB = bj * OZ_TILE;
  float acc[OZ_S][2][4];
#pragma unroll
  for (int l = 0; l < OZ_S; l++)
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
      for (int v = 0; v < 4; v++) acc[l][q][v] = 0.f;
  const int nch = K / OZ_KC;
  oz_issue<OZ_S>(sm, D, M, K, rowA, rowB, 0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int c = 0; c < nch; c++) {
    if (c + 1 < nch) oz_issue<OZ_S>(sm + ((c + 1) & 1) * OZ_STAGE, D, M, K, rowA, rowB, (c + 1) * OZ_KC);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    const unsigned short* SA = sm + (c & 1) * OZ_STAGE;
    const unsigned short* SB = SA + OZ_S * OZ_TILE * OZ_PAD;
#pragma unroll
    for (int ks = 0; ks < OZ_KC; ks += 16) {
      unsigned b[OZ_S][4];  // per digit: columns wc*16 + [0, 8) and [8, 16), k halves
#pragma unroll
      for (int j = 0; j < OZ_S; j++)
        ldsm_x4(b[j], SB + ((size_t)j * OZ_TILE + wc * 16 + (lane & 7) + ((lane >> 4) << 3)) * OZ_PAD + ks +
                          ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int i = 0; i < OZ_S; i++) {
        unsigned a[4];
        ldsm_x4(a, SA + ((size_t)i * OZ_TILE + wr * 16 + (lane & 15)) * OZ_PAD + ks + (lane >> 4) * 8);
#pragma unroll
        for (int j = 0; j + i < OZ_S; j++) {
          mma_bf16(acc[i + j][0], a, &b[j][0]);
          mma_bf16(acc[i + j][1], a, &b[j][2]);
        }
      }
    }
    __syncthreads();
  }
  const double s28 = __longlong_as_double((long long)(1023 - 28) << 52);  // 2^-28: levels 4-7 against 0-3
#pragma unroll
  for (int q = 0; q < 2; q++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const int lr = rowA + wr * 16 + g + (v >= 2 ? 8 : 0);
      const int lc = rowB + wc * 16 + q * 8 + 2 * tq + (v & 1);
      if (lr < M && lc <= lr) {
        long long hi = 0, lo = 0;  // sum_l acc[l] 2^(7 (3 - l)), sum_l acc[4 + l] 2^(7 (3 - l))
#pragma unroll
        for (int l = 0; l < 4; l++) {
          hi += (long long)__float2int_rz(acc[l][q][v]) * (1ll << (7 * (3 - l)));
          lo += (long long)__float2int_rz(acc[4 + l][q][v]) * (1ll << (7 * (3 - l)));
        }
        const double sum = fma((double)lo, s28, (double)hi);  // x 2^21
        const int e = E[lr] + E[lc] - 35;
        const double sc = (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52)
                                                    : ldexp(1.0, e);
        double* p = A + (size_t)(r0 + lc) * n + r0 + lr;
        *p = fma(-sum, sc, *p);
      }
    }
}

// The tiles of one launch: strip = 0, the lower triangle of tile rows and
// columns from toff on; strip = 1, tile columns toff and toff + 1 (the next
// 128 columns), every row tile at or below them.  CTAs loop over the tiles.
__global__ void __launch_bounds__(512, 1) oz_syrk_kernel(double* A, int n, int r0, int M, int K,
                                                     const __nv_bfloat16* __restrict__ D, const int* __restrict__ E,
                                                     const int* flag, int strip, int toff, int ntiles) {
  pdl_wait();
  if (*flag) return;
  extern __shared__ __align__(16) unsigned short oz_sm[];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    int bi, bj;
    if (strip) {  // (0, 0), then (1, 0), (1, 1), (2, 0), (2, 1), ...
      bi = t == 0 ? 0 : (t + 1) >> 1;
      bj = t == 0 ? 0 : (t + 1) & 1;
    } else {
      bi = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
      while (bi * (bi + 1) / 2 > t) bi--;
      while ((bi + 1) * (bi + 2) / 2 <= t) bi++;
      bj = t - bi * (bi + 1) / 2;
    }
    oz_tile(A, n, r0, M, K, D, E, oz_sm, bi + toff, bj + toff);
  }
  pdl_trigger();
}

size_t oz_syrk_smem() { return 2 * sizeof(unsigned short) * (size_t)OZ_STAGE; }

opf_status setup_oz() {
  if (cudaFuncSetAttribute(oz_syrk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_syrk_smem()) !=
      cudaSuccess) {
    cudaGetLastError();
    set_last_error("cannot raise the shared-memory limit of the emulated FP64 update");
    return OPF_ECUDA;
  }
  return OPF_OK;
}

// Digits of P = A[r0 : n, c0 : c0 + K] (K <= 128, a multiple of 32) into E
// (n - r0 ints) and D (8 (n - r0) K bf16).
void launch_oz_slice(cudaStream_t st, const double* A, int n, int c0, int K, int r0, int* E, void* D,
                     const int* flag) {
  const int M = n - r0;
  if (M <= 0 || K <= 0) return;
  launch_pdl(oz_slice_kernel, dim3((M + 31) / 32), dim3(1024), 0, st, A, n, c0, K, r0, M, E,
             static_cast<__nv_bfloat16*>(D), flag);
}

// A[r0 :, r0 :] (lower) -= P P^T from the digits: part = 0 the whole triangle,
// 1 the first 128 columns (all rows below), 2 the columns after them; grid 0
// takes one CTA per tile, else at most grid CTAs.
void launch_oz_syrk(cudaStream_t st, double* A, int n, int K, int r0, const int* E, const void* D, const int* flag,
                    int part, int grid) {
  const int M = n - r0;
  if (M <= 0 || K <= 0) return;
  const int nt = (M + OZ_TILE - 1) / OZ_TILE;
  int ntiles = 0, strip = 0, toff = 0;
  if (part == 0) {
    ntiles = nt * (nt + 1) / 2;
  } else if (part == 1) {
    strip = 1;
    ntiles = 2 * nt - 1;
  } else {
    toff = 2;
    ntiles = nt > 2 ? (nt - 2) * (nt - 1) / 2 : 0;
  }
  if (ntiles <= 0) return;
  const int g = grid > 0 ? std::min(grid, ntiles) : ntiles;
  launch_pdl(oz_syrk_kernel, dim3(g), dim3(512), oz_syrk_smem(), st, A, n, r0, M, K,
             static_cast<const __nv_bfloat16*>(D), E, flag, strip, toff, ntiles);
}

void launch_oz_update(cudaStream_t st, double* A, int n, int c0, int K, int r0, int* E, void* D, const int* flag) {
  launch_oz_slice(st, A, n, c0, K, r0, E, D, flag);
  launch_oz_syrk(st, A, n, K, r0, E, D, flag, 0, 0);
}

}  // namespace opf
