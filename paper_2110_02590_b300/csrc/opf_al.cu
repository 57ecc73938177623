// Static OPF: the augmented-Lagrangian outer loop (Sec. IV-B "Static OPF
// algorithm"; entry point opf_al_solve, declared in include/opf.h with the
// readings it takes).  Each outer iteration solves the AL subproblem for fixed
// rho and y by reduced-Newton barrier steps (opf_al_step), warm-started from
// the previous primal-dual point, then updates y <- y + rho D_c (c - s) and
// rho.  The loop is host code; the KKT errors, the primal infeasibility and
// the multiplier update are device reductions and kernels.
#include <algorithm>
#include <cmath>
#include <string>

#include "opf_internal.h"

using namespace opf;

namespace opf {

__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

// red[0] = max |grad L - z_lo + z_hi| over u and s, red[1] = max complementarity
// error |(w - w_lo) z_lo - mu|, |(w_hi - w) z_hi - mu| at mu, red[2] the same at
// mu = 0, red[3] = max |sigma_c (c - s)| (c may be null: 0) (NaN entries count as infinite).
__global__ void al_kkt_kernel(int nu, int m, const double* __restrict__ gu, const double* __restrict__ gs,
                              const double* __restrict__ u, const double* __restrict__ ulo,
                              const double* __restrict__ uhi, const double* __restrict__ zlu,
                              const double* __restrict__ zuu, const double* __restrict__ s,
                              const double* __restrict__ slo, const double* __restrict__ shi,
                              const double* __restrict__ zls, const double* __restrict__ zus,
                              const double* __restrict__ c, const double* __restrict__ sig, double mu,
                              double* red) {
  double e[4] = {0.0, 0.0, 0.0, 0.0};
  auto acc = [&](int k, double v) {
    v = fabs(v);
    if (!(v <= e[k])) e[k] = isnan(v) ? INFINITY : v;
  };
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nu + m; i += gridDim.x * blockDim.x) {
    double g, w, lo, hi, zl, zu;
    if (i < nu) {
      g = gu[i], w = u[i], lo = ulo[i], hi = uhi[i], zl = zlu[i], zu = zuu[i];
    } else {
      const int k = i - nu;
      g = gs[k], w = s[k], lo = slo[k], hi = shi[k], zl = zls[k], zu = zus[k];
      if (c) acc(3, sig[k] * (c[k] - w));
    }
    acc(0, g - zl + zu);
    const double cl = (w - lo) * zl, ch = (hi - w) * zu;
    acc(1, cl - mu);
    acc(1, ch - mu);
    acc(2, cl);
    acc(2, ch);
  }
#pragma unroll
  for (int k = 0; k < 4; k++)
    for (int o = 16; o > 0; o >>= 1) e[k] = fmax(e[k], __shfl_xor_sync(0xffffffffu, e[k], o));
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < 4; k++) atomic_max_nonneg(red + k, e[k]);
}

// y <- y + rho sigma_c (c - s)  (the multiplier update of the scaled AL, Sec. IV-A/IV-B)
__global__ void al_dual_update_kernel(int m, double* y, double rho, const double* __restrict__ sig,
                                      const double* __restrict__ c, const double* __restrict__ s) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
    y[k] += rho * sig[k] * (c[k] - s[k]);
}

void launch_al_kkt(opf_ctx* c, const double* gu, const double* gs, const opf_al_state* st, const double* cv,
                   const double* sig, double mu, double* red) {
  const int nu = c->h.nu, m = c->h.m;
  const int grid = std::max(1, std::min((nu + m + 255) / 256, 4 * c->sm_count));
  al_kkt_kernel<<<grid, 256, 0, c->stream>>>(nu, m, gu, gs, st->u, st->u_lo, st->u_hi, st->zl_u, st->zu_u, st->s,
                                             st->s_lo, st->s_hi, st->zl_s, st->zu_s, cv, sig, mu, red);
  c->launches++;
}

void launch_al_dual_update(opf_ctx* c, double* y, double rho, const double* sig, const double* cv,
                           const double* s) {
  const int m = c->h.m;
  al_dual_update_kernel<<<std::max(1, std::min((m + 255) / 256, 4 * c->sm_count)), 256, 0, c->stream>>>(
      m, y, rho, sig, cv, s);
  c->launches++;
}

}  // namespace opf

namespace {

struct AlWork {
  double *gu = nullptr, *gs = nullptr, *c = nullptr, *F = nullptr, *red = nullptr;
  double* h_red = nullptr;  // pinned [5]: the four maxima and F
};

#define ACK(call)                                                           \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));  \
      return OPF_ECUDA;                                                     \
    }                                                                       \
  } while (0)

// Gradient, c and F at the context's converged state, then the KKT errors:
// out[0] = E_mu, out[1] = E_0, out[2] = primal infeasibility, out[3] = F.
opf_status al_errors(opf_ctx* c, const opf_al_params* p, const opf_al_state* st, double mu, AlWork& w,
                     double out[4]) {
  opf_status rc = opf_reduced_gradient(c, p, w.F, w.gu, w.gs, w.c, nullptr, nullptr, nullptr);
  if (rc) return rc;
  cudaStream_t stream = c->stream;
  ACK(cudaMemsetAsync(w.red, 0, 4 * sizeof(double), stream));
  launch_al_kkt(c, w.gu, w.gs, st, w.c, p->sigma_c, mu, w.red);
  ACK(cudaMemcpyAsync(w.h_red, w.red, 4 * sizeof(double), cudaMemcpyDeviceToHost, stream));
  ACK(cudaMemcpyAsync(w.h_red + 4, w.F, sizeof(double), cudaMemcpyDeviceToHost, stream));
  ACK(cudaStreamSynchronize(stream));
  ACK(cudaGetLastError());
  out[0] = std::max(w.h_red[0], w.h_red[1]);
  out[1] = std::max(w.h_red[0], w.h_red[2]);
  out[2] = w.h_red[3];
  out[3] = w.h_red[4];
  return OPF_OK;
}

}  // namespace

extern "C" opf_status opf_al_solve(opf_ctx* c, const opf_al_params* p, double* y, opf_al_state* st,
                                   const opf_al_opts* o, opf_al_info* info, double* history) {
  if (!c || !p || !y || !st || !p->sigma_c) {
    set_last_error("ctx, params (with sigma_c), y and state are required");
    return OPF_EINVAL;
  }
  if (!c->have_state) {
    set_last_error("no converged power flow on this context");
    return OPF_ESTATE;
  }
  if (!(p->rho > 0.0) || !(st->mu > 0.0)) {
    set_last_error("opf_al_solve needs rho > 0 and mu > 0");
    return OPF_EINVAL;
  }
  const int max_outer = (o && o->max_outer > 0) ? o->max_outer : 20;
  const int max_inner = (o && o->max_inner > 0) ? o->max_inner : 30;
  const double eta_p = (o && o->eta_primal > 0.0) ? o->eta_primal : 1e-5;
  const double eta_d = (o && o->eta_dual > 0.0) ? o->eta_dual : 1e-4;
  const double rho_max = (o && o->rho_max > 0.0) ? o->rho_max : 1e6;
  const int block_k = o ? o->block_k : 0;
  const double gmax = o ? o->scaling_gmax : 0.0;
  if (!(gmax >= 0.0) || !std::isfinite(gmax)) {
    set_last_error("scaling_gmax must be >= 0 and finite");
    return OPF_EINVAL;
  }
  const int nu = c->h.nu, m = c->h.m;
  AlWork w;
  void* block = nullptr;
  const size_t nd = (size_t)nu + 3 * (size_t)m + 8;
  if (cudaMalloc(&block, nd * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&w.h_red, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (block) cudaFree(block);
    set_last_error("cannot allocate the outer loop's workspace");
    return OPF_ENOMEM;
  }
  double* q = static_cast<double*>(block);
  w.gu = q;
  w.gs = q + nu;
  w.c = q + nu + m;
  w.red = q + nu + 2 * (size_t)m;
  w.F = w.red + 4;
  double* sig_scaled = w.F + 4;  // [m]
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);

  opf_status rc = OPF_OK;
  // the problem's scales: the caller's, or scaled by its gradients at the start
  const double* sigma_c = p->sigma_c;
  double sigma_f = p->sigma_f;
  if (gmax > 0.0) {
    void* J = nullptr;
    if (cudaMalloc(&J, sizeof(double) * (size_t)m * (size_t)nu) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("cannot allocate the Jacobian of the gradient scaling");
      rc = OPF_ENOMEM;
    } else {
      rc = opf_gradient_scaling(c, gmax, 1e-8, p->sigma_c, static_cast<double*>(J), sig_scaled, &sigma_f);
      cudaFree(J);
      sigma_c = sig_scaled;
    }
  }
  if (rc == OPF_OK && o && o->sigma_c_used)
    if (cudaMemcpyAsync(o->sigma_c_used, sigma_c, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess) {
      cudaGetLastError();
      set_last_error("cannot copy the constraint scales");
      rc = OPF_ECUDA;
    }
  double rho = p->rho, mu = st->mu, prev_eta = INFINITY, delta = 0.0;
  double E[4] = {0, 0, 0, 0};
  int outer = 0, steps_total = 0, converged = 0;
  opf_step_info si;
  for (int k = 0; k < max_outer && rc == OPF_OK; k++) {
    const double omega_k = std::max(eta_d, std::pow(10.0, -(double)(k + 1)));
    opf_al_params pk = *p;
    pk.sigma_c = sigma_c;
    pk.sigma_f = sigma_f;
    pk.y = y;
    pk.rho = rho;
    pk.s = st->s;
    pk.omega = nullptr;
    int steps = 0;
    for (int j = 0; j <= max_inner; j++) {
      rc = al_errors(c, &pk, st, mu, w, E);
      if (rc) break;
      if (E[1] <= omega_k || j == max_inner) break;
      if (E[0] <= 10.0 * mu) mu = std::max(eta_d / 10.0, std::min(0.2 * mu, std::pow(mu, 1.5)));
      st->mu = mu;
      opf_step_opts so = {block_k, 0, 0, delta >= 1e-7 ? delta / 10.0 : 0.0, 1};
      rc = opf_al_step(c, &pk, st, &so, &si, nullptr, nullptr);
      if (rc) break;
      delta = si.delta;
      steps++;
    }
    if (rc) break;
    steps_total += steps;
    outer = k + 1;
    if (history) {
      double* h = history + 8 * (size_t)k;
      h[0] = steps;
      h[1] = mu;
      h[2] = rho;
      h[3] = E[2];
      h[4] = E[1];
      h[5] = E[3];
      h[6] = delta;
      h[7] = 0.0;
    }
    if (E[2] <= eta_p && E[1] <= eta_d) {
      converged = 1;
      break;
    }
    launch_al_dual_update(c, y, rho, sigma_c, w.c, st->s);
    if (E[2] > 0.25 * prev_eta) rho = std::min(10.0 * rho, rho_max);
    prev_eta = E[2];
  }
  st->mu = mu;
  cudaEventRecord(e1, c->stream);
  cudaError_t ce = cudaStreamSynchronize(c->stream);
  if (rc == OPF_OK && ce != cudaSuccess) {
    set_last_error(std::string("opf_al_solve: ") + cudaGetErrorString(ce));
    rc = OPF_ECUDA;
  }
  if (info) {
    info->outer = outer;
    info->steps = steps_total;
    info->converged = converged;
    info->primal_inf = E[2];
    info->dual_inf = E[1];
    info->F = E[3];
    info->rho = rho;
    info->mu = mu;
    info->sigma_f = sigma_f;
    info->ms_total = 0.f;
    cudaEventElapsedTime(&info->ms_total, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(block);
  cudaFreeHost(w.h_red);
  return rc;
}
