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
// B300's bf16 tensor rate (~1.8 PFLOP/s with tcgen05, ~1.1 with mma.sync in
// registers) against its FP64 rate (~1.2 TFLOP/s) makes this ~10-30 times
// faster than FP64 FMAs.  Two engines run the tile products: the tcgen05
// kernel (default; level sums in tensor memory, digits staged by bulk copies)
// and the warp-level mma.sync kernel; both sum the same exact integers and
// round the same way, so their results are bit-identical.

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
// n): E[r] and the eight bf16 digit planes.  Row-major layout (tiled = false):
// D[s][r][k], K per row, M rows.  Core-matrix layout (tiled = true), the one
// the tcgen05 kernel stages with bulk copies: for each 16 columns of K (kc)
// and digit s, a block of Mp rows (M rounded up to 128, the extra rows zero)
// of 16 digits in 8-row x 8-column core matrices of 128 bytes, the two core
// matrices of an 8-row group side by side (element (r, k) at ((kc 8 + s) Mp +
// (r / 8) 8) 16 + ((k / 8) mod 2) 64 + (r mod 8) 8 + k mod 8), so 128 or 64
// consecutive rows of one plane and kc are one contiguous run.  One CTA per 32
// rows, its 32 warps over the columns; the digits pass through shared memory
// so that the reads (along rows) coalesce and every thread writes 16 bytes.
__global__ void __launch_bounds__(1024) oz_slice_kernel(const double* __restrict__ A, int n, int c0, int K, int r0,
                                                      int M, int Mp, bool tiled, int* __restrict__ E,
                                                      __nv_bfloat16* __restrict__ D, const int* flag) {
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
  const int rows_out = tiled ? Mp : M;
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
    // one 16-byte piece (8 digits of one row and plane) per item: 8 planes x 32 rows x 4 groups
    for (int it = threadIdx.x; it < OZ_S * 32 * 4; it += blockDim.x) {
      const int g = it & 3, rr = (it >> 2) & 31, s = it >> 7;
      const int row = blockIdx.x * 32 + rr, k0 = kt + g * 8;
      if (row >= rows_out || k0 >= K) continue;
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; e++) v[e] = dig[s][g * 8 + e][rr];
      const size_t idx = tiled ? (((size_t)(k0 >> 4) * OZ_S + s) * Mp + (row >> 3) * 8) * 16 + ((k0 >> 3) & 1) * 64 +
                                     (row & 7) * 8
                               : ((size_t)s * M + row) * K + k0;
      *reinterpret_cast<uint4*>(D + idx) = *reinterpret_cast<const uint4*>(v);
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

// ---------------------------------------------------------------------------
// The same update on the fifth-generation tensor cores (tcgen05): 128 x 64
// output tiles whose eight level sums live in tensor memory (TMEM) as eight
// 128-lane x 64-column FP32 accumulators -- all 512 columns of the SM's TMEM,
// so one CTA per SM, persistent over the tiles.  Warp-specialised:
//   warp 0, the producer: per job (tile, 16 columns of K) 16 bulk copies
//     (cp.async.bulk, the TMA engine) of the digit planes, in the core-matrix
//     layout oz_slice writes, into one of four shared-memory stages, completed
//     on the stage's `full` mbarrier by byte count;
//   warp 1, the MMA issuer (it also allocates and frees the TMEM): per job the
//     36 digit-pair MMAs (M = 128, N = 64, K = 16, bf16, FP32 accumulation:
//     exact, as above), committed to the stage's `empty` mbarrier, and after a
//     tile's last job to `accf`; before a tile's first MMA it waits on `acce`;
//   warps 4-11, the epilogue: each reads TMEM lanes 32 (w mod 4) .. + 31 and
//     half of the columns with tcgen05.ld, folds the levels exactly as the
//     warp-level kernel does (so both engines give bit-identical results),
//     updates A and arrives on `acce`.
// The shared-memory operands use the no-swizzle K-major canonical layout: 8-row
// x 16-byte core matrices, neighbours along K 128 bytes apart, 8-row groups 256
// bytes apart.  Every wait is bounded: a wait that gives up sets `abort` (every
// other wait loop watches it) and *err; after all roles stop, the copies and
// MMAs already issued are drained with a limit of their own, far above their
// duration, before the TMEM is freed.

namespace {

constexpr int TC_M = 128;                              // output rows per tile (TMEM lanes)
constexpr int TC_N = 64;                               // output columns per tile
constexpr int TC_KC = 16;                              // K per job: one MMA step
constexpr int TC_NST = 4;                              // shared-memory stages
constexpr int TC_PLANE_A = TC_M * TC_KC * 2;           // bytes of one digit plane of the row block
constexpr int TC_PLANE_B = TC_N * TC_KC * 2;           // ... of the column block
constexpr int TC_STAGE = OZ_S * (TC_PLANE_A + TC_PLANE_B);
constexpr int TC_COLS = OZ_S * TC_N;                   // TMEM columns: the eight level accumulators
constexpr int TC_EPI_WARPS = 8;                        // warps 4 .. 11
constexpr int TC_THREADS = 32 * (4 + TC_EPI_WARPS);
constexpr long long TC_DRAIN = 1ll << 26;             // polls of the drain after an abort
// instruction descriptor (kind::f16): FP32 accumulator, bf16 A and B, both
// K-major, N / 8 at bit 17, M / 16 at bit 24
constexpr unsigned TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(TC_N >> 3) << 17) |
                              ((unsigned)(TC_M >> 4) << 24);

// shared-memory matrix descriptor: no swizzle, K-major core matrices, leading
// (K) byte offset 128, stride (row-group) byte offset 256, descriptor version 1
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr) {
  return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)(128 >> 4) << 16) |
         ((unsigned long long)(256 >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long ad, unsigned long long bd, bool acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(TC_IDESC), "r"((unsigned)acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ bool tc_try(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Poll for the mbarrier phase of this parity, at most lim times.
__device__ __forceinline__ bool tc_poll(unsigned bar, unsigned parity, long long lim) {
  for (long long it = 0; it < lim; it++)
    if (tc_try(bar, parity)) return true;
  return false;
}

// Wait for the mbarrier phase of this parity; false when `lim` polls pass or
// another role has aborted.
__device__ __forceinline__ bool tc_wait(unsigned bar, unsigned parity, long long lim, volatile int* abort_) {
  for (long long it = 0; it < lim; it++) {
    if (tc_try(bar, parity)) return true;
    if (*abort_) return false;
  }
  return false;
}

__device__ __forceinline__ void tc_ld16(unsigned* r, unsigned taddr) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// The update of one element in integer arithmetic: with X = hi 2^28 + lo (exact,
// |X| < 2^76 as a 128-bit two's-complement pair), returns u = RN(X) 2^(e - 28)
// (X rounded once to 53 bits, ties to even), which is what the warp-level
// kernel's fma(lo, 2^-28, hi) times 2^e gives; ok is false when u would leave
// the normal range (the caller then uses that FP64 formula).  Branch-free, so
// the elements of a chunk interleave; one FP64 operation per element is left
// (old - u) where the FP64 formula takes four.
__device__ __forceinline__ double tc_fold(long long hi, long long lo, int e, bool& ok) {
  unsigned long long xl = (unsigned long long)hi << 28;
  long long xh = hi >> 36;
  const unsigned long long l2 = xl + (unsigned long long)lo;
  xh += (long long)(l2 < xl) - (long long)(lo < 0);
  xl = l2;
  const bool neg = xh < 0;
  const unsigned long long nl = ~xl + 1ull;
  const long long nh = ~xh + (long long)(nl == 0ull);
  xl = neg ? nl : xl;
  xh = neg ? nh : xh;
  const bool zero = (xl | (unsigned long long)xh) == 0ull;
  const int nb = xh ? 128 - __clzll(xh) : 64 - __clzll((long long)xl);  // bit length of |X|
  int sh = nb - 53;
  // sh <= 0: exact, m = |X| 2^-sh; 1 <= sh <= 23: the dropped bits round to nearest even
  const int ls = max(-sh, 0), rs = min(max(sh, 1), 63);
  const unsigned long long rem = xl & ((1ull << rs) - 1ull), half = 1ull << (rs - 1);
  unsigned long long mr = (xl >> rs) | ((unsigned long long)xh << (64 - rs));
  mr += (rem > half || (rem == half && (mr & 1ull))) ? 1ull : 0ull;
  const bool carry = mr == (1ull << 53);
  mr = carry ? (mr >> 1) : mr;
  const unsigned long long m = sh > 0 ? mr : (xl << min(ls, 63));
  sh = sh > 0 ? sh + (int)carry : sh;
  const int biased = sh + e - 28 + 52 + 1023;
  ok = zero || (biased >= 1 && biased <= 2046);
  const double u = __longlong_as_double((long long)((neg ? (1ull << 63) : 0ull) |
                                                    ((unsigned long long)(biased & 2047) << 52) |
                                                    (m & ((1ull << 52) - 1ull))));
  return zero ? 0.0 : u;
}

// (row tile, column tile) of tile t: row tile bi holds column tiles 0 ..
// min(2 bi + 1, nct - 1) (the lower triangle in 128 x 64 tiles)
__device__ __forceinline__ void tc_tile_of(int t, int nct, int& bi, int& bj) {
  bi = 0;
  for (;;) {
    const int cnt = min(2 * bi + 2, nct);
    if (t < cnt) break;
    t -= cnt;
    bi++;
  }
  bj = t;
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS, 1) oz_syrk_tc_kernel(double* A, int n, int r0, int M, int Mp, int K,
                                                                   const __nv_bfloat16* __restrict__ D,
                                                                   const int* __restrict__ E, const int* flag,
                                                                   int* err, long long lim, int ntiles, int nct) {
  pdl_wait();
  if (*flag) return;
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  __shared__ __align__(8) unsigned long long bars[2 * TC_NST + 2];  // full[4], empty[4], accf, acce
  __shared__ unsigned tslot;
  __shared__ volatile int abort_;
  __shared__ int last_load, last_mma, last_taken;  // jobs: copied, committed, consumed by the MMAs
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned base = ((unsigned)__cvta_generic_to_shared(tc_sm) + 1023u) & ~1023u;
  const unsigned b0 = (unsigned)__cvta_generic_to_shared(&bars[0]);
  auto full = [&](int s) { return b0 + 8u * (unsigned)s; };
  auto empty = [&](int s) { return b0 + 8u * (unsigned)(TC_NST + s); };
  const unsigned accf = b0 + 8u * (2 * TC_NST), acce = accf + 8u;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(&tslot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * TC_NST + 1; s++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0 + 8u * (unsigned)s) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acce), "r"(TC_EPI_WARPS) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_ = 0;
    last_load = last_mma = last_taken = -1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tslot;
  const int nch = K / TC_KC;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int njobs = my_tiles * nch;
  auto tile_rows = [&](int lt, int& rowA, int& rowB) {
    int bi, bj;
    tc_tile_of((int)blockIdx.x + lt * (int)gridDim.x, nct, bi, bj);
    rowA = bi * TC_M;
    rowB = bj * TC_N;
  };
  auto fail = [&]() {
    abort_ = 1;
    atomicExch(err, 1);
  };

  if (warp == 0) {  // producer
    for (int j = 0; j < njobs; j++) {
      const int s = j % TC_NST;
      bool ok = true;
      if (lane == 0) {
        if (j >= TC_NST) ok = tc_wait(empty(s), (unsigned)(((j - TC_NST) / TC_NST) & 1), lim, &abort_);
        if (ok) {
          int ra, rb;
          tile_rows(j / nch, ra, rb);
          const int kc = j % nch;
          const unsigned st = base + (unsigned)s * TC_STAGE;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(s)), "r"(TC_STAGE)
                       : "memory");
#pragma unroll 1
          for (int pl = 0; pl < OZ_S; pl++) {
            const __nv_bfloat16* pa = D + (((size_t)kc * OZ_S + pl) * Mp + ra) * TC_KC;
            const __nv_bfloat16* pb = D + (((size_t)kc * OZ_S + pl) * Mp + rb) * TC_KC;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    st + (unsigned)(pl * TC_PLANE_A)),
                "l"(pa), "r"(TC_PLANE_A), "r"(full(s))
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    st + (unsigned)(OZ_S * TC_PLANE_A + pl * TC_PLANE_B)),
                "l"(pb), "r"(TC_PLANE_B), "r"(full(s))
                : "memory");
          }
          last_load = j;
        } else {
          fail();
        }
      }
      if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
    }
  } else if (warp == 1) {  // MMA issuer
    for (int j = 0; j < njobs; j++) {
      const int s = j % TC_NST, lt = j / nch, c = j % nch;
      bool ok = true;
      if (lane == 0) {
        if (c == 0 && lt > 0) ok = tc_wait(acce, (unsigned)((lt - 1) & 1), lim, &abort_);  // accumulators read
        if (ok) ok = tc_wait(full(s), (unsigned)((j / TC_NST) & 1), lim, &abort_);       // operands landed
        if (ok) {
          last_taken = j;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned sa = base + (unsigned)s * TC_STAGE, sb = sa + OZ_S * TC_PLANE_A;
#pragma unroll
          for (int i = 0; i < OZ_S; i++) {
            const unsigned long long ad = tc_desc(sa + i * TC_PLANE_A);
#pragma unroll
            for (int jj = 0; jj + i < OZ_S; jj++)
              tc_mma(tmem + (unsigned)((i + jj) * TC_N), ad, tc_desc(sb + jj * TC_PLANE_B), c > 0 || i > 0);
          }
          tc_commit(empty(s));
          if (c == nch - 1) tc_commit(accf);
          last_mma = j;
        } else {
          fail();
        }
      }
      if (!__shfl_sync(0xffffffffu, (int)ok, 0)) break;
    }
  } else if (warp >= 4) {  // epilogue
    const int q = warp & 3, h = (warp - 4) >> 2;
    const double s28 = __longlong_as_double((long long)(1023 - 28) << 52);  // 2^-28: levels 4-7 against 0-3
    for (int lt = 0; lt < my_tiles; lt++) {
      const bool ok = __all_sync(0xffffffffu, tc_wait(accf, (unsigned)(lt & 1), lim, &abort_));
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int ra, rb;
      tile_rows(lt, ra, rb);
      const int lr = ra + q * 32 + lane;
      const int er = lr < M ? E[lr] : 0;
      // the exponents of this warp's 32 columns, one load per lane (broadcast by shuffles)
      const int ecol = rb + h * 32 + lane < M ? E[rb + h * 32 + lane] : 0;
      // (1) both 16-column chunks out of TMEM: the levels folded into exact
      // integers and rounded to the subtrahends u (the FP64 formula where they
      // leave the normal range); then the accumulators are released, so the
      // next tile's MMAs run while (2) updates A
      double u[2][16];
      unsigned fb[2] = {0u, 0u};
#pragma unroll
      for (int cc = 0; cc < 2; cc++) {
        const int col0 = h * 32 + cc * 16;
        // hi = (acc0 2^7 + acc1) 2^14 + (acc2 2^7 + acc3), lo likewise from levels
        // 4-7: a pair folds exactly in 32-bit integers, since level t holds t + 1
        // digit pairs over K <= 128 columns (|acc_t| <= (t + 1) 128 127^2), so
        // |acc_t 2^7 + acc_t+1| < 1.87e9 < 2^31
        long long hi[16], lo[16];
#pragma unroll
        for (int l = 0; l < OZ_S; l += 2) {
          unsigned v0[16], v1[16];
          tc_ld16(v0, tmem + ((unsigned)(q * 32) << 16) + (unsigned)(l * TC_N + col0));
          tc_ld16(v1, tmem + ((unsigned)(q * 32) << 16) + (unsigned)((l + 1) * TC_N + col0));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int k = 0; k < 16; k++) {
            const int pr = __float2int_rz(__uint_as_float(v0[k])) * 128 + __float2int_rz(__uint_as_float(v1[k]));
            if (l == 0) hi[k] = (long long)pr * (1ll << 14);
            if (l == 2) hi[k] += pr;
            if (l == 4) lo[k] = (long long)pr * (1ll << 14);
            if (l == 6) lo[k] += pr;
          }
        }
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int lc = rb + col0 + k;
          const int ec = __shfl_sync(0xffffffffu, ecol, cc * 16 + k);
          bool ok;
          u[cc][k] = tc_fold(hi[k], lo[k], er + ec - 35, ok);
          fb[cc] |= (lr < M && lc <= lr && !ok) ? (1u << k) : 0u;
        }
        if (fb[cc]) {  // rare: a subnormal or out-of-range subtrahend
#pragma unroll
          for (int k = 0; k < 16; k++)
            if ((fb[cc] >> k) & 1u) u[cc][k] = fma((double)lo[k], s28, (double)hi[k]);  // x 2^21
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(acce) : "memory");
      // (2) the old values of a chunk first (independent loads), then its updates
#pragma unroll
      for (int cc = 0; cc < 2; cc++) {
        const int col0 = h * 32 + cc * 16;
        double old[16];
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int lc = rb + col0 + k;
          old[k] = (lr < M && lc <= lr) ? A[(size_t)(r0 + lc) * n + r0 + lr] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int lc = rb + col0 + k;
          if (lr < M && lc <= lr) {
            double r = old[k] - u[cc][k];
            if ((fb[cc] >> k) & 1u) {  // rare: a subnormal or out-of-range subtrahend
              const int e = er + E[lc] - 35;
              const double scl = (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52)
                                                           : ldexp(1.0, e);
              r = fma(-u[cc][k], scl, old[k]);
            }
            A[(size_t)(r0 + lc) * n + r0 + lr] = r;
          }
        }
      }
    }
  }
  __syncthreads();
  if (abort_ && threadIdx.x == 32) {
    // drain: the MMAs already committed and the copies not yet consumed
    // complete before the TMEM and the shared memory are released
    if (last_mma >= 0) tc_poll(empty(last_mma % TC_NST), (unsigned)((last_mma / TC_NST) & 1), TC_DRAIN);
    for (int j = last_taken + 1; j <= last_load; j++)
      tc_poll(full(j % TC_NST), (unsigned)((j / TC_NST) & 1), TC_DRAIN);
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
  }
  pdl_trigger();
}

size_t oz_syrk_smem() { return 2 * sizeof(unsigned short) * (size_t)OZ_STAGE; }
size_t oz_syrk_tc_smem() { return (size_t)TC_NST * TC_STAGE + 1024; }

opf_status setup_oz() {
  if (cudaFuncSetAttribute(oz_syrk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_syrk_smem()) !=
          cudaSuccess ||
      cudaFuncSetAttribute(oz_syrk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)oz_syrk_tc_smem()) != cudaSuccess) {
    cudaGetLastError();
    set_last_error("cannot raise the shared-memory limit of the emulated FP64 update");
    return OPF_ECUDA;
  }
  return OPF_OK;
}

// Digits of P = A[r0 : n, c0 : c0 + K] (K <= 128, a multiple of 32) into E
// (n - r0 ints) and D (8 (n - r0) K bf16).
void launch_oz_slice(cudaStream_t st, const double* A, int n, int c0, int K, int r0, int* E, void* D,
                     const int* flag, bool tiled) {
  const int M = n - r0;
  if (M <= 0 || K <= 0) return;
  const int Mp = oz_rows_tiled(M);
  launch_pdl(oz_slice_kernel, dim3(((tiled ? Mp : M) + 31) / 32), dim3(1024), 0, st, A, n, c0, K, r0, M, Mp, tiled,
             E, static_cast<__nv_bfloat16*>(D), flag);
}

// A[r0 :, r0 :] (lower) -= P P^T from the digits, with the warp-level MMAs:
// part = 0 the whole triangle, 1 the first 128 columns (all rows below), 2 the
// columns after them; grid 0 takes one CTA per tile, else at most grid CTAs.
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

// The same update on the tcgen05 tensor cores from the core-matrix digits: 128 x
// 64 tiles of the lower triangle, one persistent CTA per SM (at most sm_count).
void launch_oz_syrk_tc(cudaStream_t st, double* A, int n, int K, int r0, const int* E, const void* D,
                       const int* flag, int* err, long long lim, int sm_count) {
  const int M = n - r0;
  if (M <= 0 || K <= 0) return;
  const int nrt = (M + TC_M - 1) / TC_M, nct = (M + TC_N - 1) / TC_N;
  int ntiles = 0;
  for (int bi = 0; bi < nrt; bi++) ntiles += std::min(2 * bi + 2, nct);
  const int g = std::max(1, std::min(ntiles, sm_count));
  launch_pdl(oz_syrk_tc_kernel, dim3(g), dim3(TC_THREADS), oz_syrk_tc_smem(), st, A, n, r0, M, oz_rows_tiled(M), K,
             static_cast<const __nv_bfloat16*>(D), E, flag, err, lim, ntiles, nct);
}

void launch_oz_update(cudaStream_t st, double* A, int n, int c0, int K, int r0, int* E, void* D, const int* flag,
                      const OzEngine& eng) {
  const int M = n - r0;
  const int nrt = (M + TC_M - 1) / TC_M, nct = (M + TC_N - 1) / TC_N;
  int ntiles = 0;
  for (int bi = 0; bi < nrt; bi++) ntiles += std::min(2 * bi + 2, nct);
  const bool tc = eng.engine == 2 || (eng.engine == 0 && ntiles >= OZ_TC_MIN_TILES);
  launch_oz_slice(st, A, n, c0, K, r0, E, D, flag, tc);
  if (tc)
    launch_oz_syrk_tc(st, A, n, K, r0, E, D, flag, eng.err, eng.lim, eng.sm_count);
  else
    launch_oz_syrk(st, A, n, K, r0, E, D, flag, 0, 0);
}

}  // namespace opf
