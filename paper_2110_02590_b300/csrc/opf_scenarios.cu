// Scenario batches of one network: the power flow and the reduced objective
// (and, on request, its adjoint gradient, Prop. 1) for many load scenarios,
// spread over a pool of contexts of that network.  Each context works on its
// own stream, driven by its own host thread, so the GPU overlaps the
// scenarios' latency-bound power flows and solves (a 2,000-bus power flow
// leaves most of the GPU idle).  Used by the autograd objective's forward and
// backward passes (the backward pass restarts each scenario from the state the
// forward pass returned, x0 == x_out).
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "opf_internal.h"

using namespace opf;

extern "C" opf_status opf_objective_batched(opf_ctx* const* ctxs, int nctx, int n, const opf_al_params* p,
                                            const double* u, const double* pd, const double* qd,
                                            const double* s, const double* x0, double* x_out, double* F,
                                            double* grad_u, double* grad_pd, double* grad_qd, double* grad_s,
                                            opf_status* status) {
  if (!ctxs || nctx < 1 || n < 0 || !p || !u || !s || !x0) {
    set_last_error("ctxs, p, u, s and x0 are required, nctx >= 1, n >= 0");
    return OPF_EINVAL;
  }
  const opf_ctx* c0 = ctxs[0];
  for (int k = 0; k < nctx; k++) {
    const opf_ctx* c = ctxs[k];
    if (!c || c->device != c0->device || c->h.nb != c0->h.nb || c->h.nx != c0->h.nx || c->h.nu != c0->h.nu ||
        c->h.m != c0->h.m) {
      set_last_error("the contexts of a scenario batch must be of one network on one device");
      return OPF_EINVAL;
    }
    for (int j = 0; j < k; j++)
      if (ctxs[j] == c) {
        set_last_error("a context appears twice in the pool");
        return OPF_EINVAL;
      }
  }
  const size_t nu = c0->h.nu, nb = c0->h.nb, nx = c0->h.nx, m = c0->h.m;
  // x0 == x_out: every scenario starts from its own row of x_out
  const bool own_start = x_out && x0 == x_out;
  std::vector<opf_status> st(n, OPF_OK);
  std::vector<std::string> msg(n);
  std::atomic<int> next(0);
  const int dev = c0->device;
  auto work = [&](int w) {
    cudaSetDevice(dev);
    opf_ctx* c = ctxs[w];
    double* x = nullptr;
    if (!x_out && cudaMalloc(&x, nx * sizeof(double)) != cudaSuccess) {  // one state per worker
      cudaGetLastError();
      for (int k = next++; k < n; k = next++) {
        st[k] = OPF_ENOMEM;
        msg[k] = "cannot allocate a worker's state";
      }
      return;
    }
    for (int k = next++; k < n; k = next++) {
      double* xk = x_out ? x_out + k * nx : x;
      opf_status r = OPF_OK;
      if (!own_start)
        r = cudaMemcpyAsync(xk, x0, nx * sizeof(double), cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess
                ? OPF_OK
                : OPF_ECUDA;
      if (r == OPF_OK)
        r = opf_powerflow(c, u + k * nu, pd ? pd + k * nb : nullptr, qd ? qd + k * nb : nullptr, xk, nullptr,
                          nullptr);
      if (r == OPF_OK) {
        opf_al_params pk = *p;
        pk.s = s + k * m;
        pk.omega = nullptr;
        r = opf_reduced_gradient(c, &pk, F ? F + k : nullptr, grad_u ? grad_u + k * nu : nullptr,
                                 grad_s ? grad_s + k * m : nullptr, nullptr, nullptr,
                                 grad_pd ? grad_pd + k * nb : nullptr, grad_qd ? grad_qd + k * nb : nullptr);
      }
      st[k] = r;
      if (r != OPF_OK) msg[k] = opf_last_error();
    }
    if (x) cudaFree(x);
  };
  const int nw = std::min(nctx, std::max(n, 1));
  std::vector<std::thread> pool;
  for (int w = 1; w < nw; w++) pool.emplace_back(work, w);
  work(0);
  for (auto& t : pool) t.join();
  opf_status first = OPF_OK;
  for (int k = 0; k < n; k++) {
    if (status) status[k] = st[k];
    if (st[k] != OPF_OK && first == OPF_OK) {
      first = st[k];
      set_last_error("scenario " + std::to_string(k) + ": " + msg[k]);
    }
  }
  return first;
}
