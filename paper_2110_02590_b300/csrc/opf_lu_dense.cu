// Dense LU (no pivoting, like the rest of the refactorisation) of the trailing
// block [r0, r0 + s) of the power-flow Jacobian's factor (Sec. III-A: the
// Newton-Raphson step needs G_x factorised at every iterate), spread over one
// thread-block cluster.
//
// The block is the root separator: its rows are mutually dense and it comes
// last, after every sparse level.  One CTA has ~1/1.6 FP64 lane-operations per
// cycle, so a single CTA spends most of its time waiting for the FP64 unit;
// the cluster divides the rank-one updates among K SMs.  CTA q owns the rows
// i = q (mod K) in its shared memory.  Step k: the owner of row k + 1 applies
// row k to it first, forms 1 / U_{k+1,k+1}, and writes row k + 1 with that
// reciprocal into every CTA's copy of the pivot rows (distributed shared
// memory, one slot per row, so no slot is ever reused), then raises each
// CTA's flag for step k + 1 with release semantics at cluster scope; the other
// rows follow.  A CTA waits for a step's flag by polling its own shared memory
// (acquire); each wait is bounded (flags[2] spins, else 2^22) and, on timeout,
// sets the timeout flag flags[1] and goes on, so that every CTA still reaches
// the final cluster barrier (the factor is then void and the call reports
// OPF_ETIMEOUT).

#include "opf_internal.h"

namespace opf {

namespace {

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_map(const void* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st_f64(unsigned addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void cl_release_u32(unsigned addr, unsigned v) {
  asm volatile("st.release.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned cl_acquire_u32(const unsigned* p) {
  unsigned v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.acquire.cluster.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

}  // namespace

// Dynamic shared memory per CTA: own rows [nr][s], pivot rows [s][s] and their
// reciprocals [s] (doubles), then the step flags [s] (u32); nr = ceil(s / K).
// Before the trailing block, the cluster runs the last, narrow levels of the
// sparse LU (tail): their work items are spread over all warps of the cluster
// as in one level launch, the factor is read through L2 (lu_ld<true>), and a
// cluster barrier (release / acquire) separates the levels, in place of a
// kernel boundary each.
__global__ void __launch_bounds__(kLuClusterThreads, 1)
    lu_dense_cluster_kernel(double* LU, const int* __restrict__ dp, int r0, int s, int* flags, LuTail tail) {
  extern __shared__ __align__(16) double dsm[];
  const int K = (int)cl_size(), q = (int)cl_rank();
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tail.lv0 < tail.lv1) {
    const int lane = tid & 31;
    const int warp = (q * nt + tid) >> 5, nw = (K * nt) >> 5;
    for (int lv = tail.lv0; lv < tail.lv1; lv++) {
      const int4 rg = __ldg(tail.lvrec + lv);  // {t0, t1, f0, f1}
      const int G = __ldg(tail.lanes + lv), li = lane & (G - 1), ipw = 32 / G;
      const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
      const int ntask = rg.y - rg.x, nall = ntask + (rg.w - rg.z);
      for (int base = warp * ipw; base < nall; base += nw * ipw) {
        const int w = base + lane / G;
        if (w < ntask) {
          const int t = rg.x + w;
          const int4 tr = __ldg(tail.task_rec + t);
          const int* tg = tail.task_map + __ldg(tail.task_off + t);
          int tgt[LU_PRE];
          lu_targets(tr, tg, li, G, tgt);
          lu_task<true>(LU, tr, tg, tgt, li, G, gmask, flags);
        } else if (w < nall) {
          lu_finish<true>(LU, __ldg(tail.fin_rec + rg.z + (w - ntask)), li, G, gmask);
        }
      }
      cl_sync();
    }
  }
  const long long lim = flags[2] > 0 ? (long long)flags[2] : (1ll << 22);
  const int nr = (s + K - 1) / K;
  double* mine = dsm;                    // row q + K t at mine[t * s]
  double* piv = mine + (size_t)nr * s;   // row k at piv[k * s]
  double* pinv = piv + (size_t)s * s;    // 1 / U_kk
  unsigned* flag = reinterpret_cast<unsigned*>(pinv + s);
  for (int e = tid; e < nr * s; e += nt) {
    const int t = e / s, j = e - t * s, i = q + K * t;
    mine[e] = (i < s) ? __ldcg(LU + dp[r0 + i] - i + j) : 0.0;
  }
  for (int k = tid; k < s; k += nt) flag[k] = 0u;
  __syncthreads();
  cl_sync();  // every CTA's flags are clear before any remote write
  // row k (owned here) with its reciprocal into every CTA's pivot slot k, then the flags
  auto publish = [&](int k) {
    const double* row = mine + (size_t)(k / K) * s;
    if (tid < K) {  // one thread per destination: the reciprocal
      const double u = row[k];
      if (tid == 0 && (!(fabs(u) > 0.0) || !isfinite(u))) flags[0] = 1;
      cl_st_f64(cl_map(pinv + k, tid), 1.0 / u);
    }
    const int w = s - k;
    for (int e = tid; e < K * w; e += nt) {
      const int p = e / w, j = k + (e - p * w);
      cl_st_f64(cl_map(piv + (size_t)k * s + j, p), row[j]);
    }
    __syncthreads();
    // the release store orders this CTA's writes above (ordered before it by the barrier)
    if (tid < K) cl_release_u32(cl_map(flag + k, tid), (unsigned)(k + 1));
  };
  if (q == 0 && s > 0) publish(0);
  for (int k = 0; k + 1 < s; k++) {
    // wait for row k
    if (tid == 0) {
      long long spins = 0;
      while (cl_acquire_u32(flag + k) != (unsigned)(k + 1)) {
        if (++spins > lim) {
          atomicExch(flags + 1, 1);
          break;
        }
      }
    }
    __syncthreads();
    const double* pk = piv + (size_t)k * s;
    const double ik = pinv[k];
    // the next pivot row first, then its publication
    if ((k + 1) % K == q) {
      double* row = mine + (size_t)((k + 1) / K) * s;
      const double l = row[k] * ik;
      for (int j = k + 1 + tid; j < s; j += nt) row[j] = fma(-l, pk[j], row[j]);
      __syncthreads();
      if (tid == 0) row[k] = l;
      publish(k + 1);
    }
    // the other rows below k: multipliers, then the rank-one update
    const int t0 = (k + 1 - q + K - 1) / K;  // first own row index i > k (i = q + K t)
    for (int t = t0 + tid; t < nr; t += nt) {
      const int i = q + K * t;
      if (i > k + 1 && i < s) mine[(size_t)t * s + k] *= ik;
    }
    __syncthreads();
    const int w = s - k - 1;
    int rows = nr - t0;
    if (rows > 0) {
      for (int e = tid; e < rows * w; e += nt) {
        const int tt = t0 + e / w, j = k + 1 + (e - (e / w) * w), i = q + K * tt;
        if (i > k + 1 && i < s) {
          double* a = mine + (size_t)tt * s;
          a[j] = fma(-a[k], pk[j], a[j]);
        }
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nr * s; e += nt) {
    const int t = e / s, j = e - t * s, i = q + K * t;
    if (i < s) LU[dp[r0 + i] - i + j] = mine[e];
  }
  cl_sync();  // no CTA leaves while others may still write into its shared memory
}

size_t lu_dense_cluster_smem(int s, int K) {
  const size_t nr = (size_t)(s + K - 1) / K;
  return sizeof(double) * (nr * s + (size_t)s * s + s) + sizeof(unsigned) * (size_t)s;
}

// Largest cluster (16, else 8) whose CTAs fit the block; 0 keeps the one-CTA kernel.
int setup_lu_dense_cluster(int s) {
  if (s < 32) return 0;
  cudaFuncSetAttribute(lu_dense_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int K : {16, 8}) {
    const size_t smem = lu_dense_cluster_smem(s, K);
    if (smem > 200 * 1024) continue;
    if (cudaFuncSetAttribute(lu_dense_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(K);
    cfg.blockDim = dim3(kLuClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclu = 0;
    if (cudaOccupancyMaxActiveClusters(&nclu, lu_dense_cluster_kernel, &cfg) == cudaSuccess && nclu > 0) return K;
    cudaGetLastError();
  }
  return 0;
}

void launch_lu_dense_cluster(cudaStream_t st, int K, double* LU, const int* dp, int r0, int s, int* flags,
                             const LuTail& tail) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = K;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(K);
  cfg.blockDim = dim3(kLuClusterThreads);
  cfg.dynamicSmemBytes = lu_dense_cluster_smem(s, K);
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, lu_dense_cluster_kernel, LU, dp, r0, s, flags, tail);
}

}  // namespace opf
