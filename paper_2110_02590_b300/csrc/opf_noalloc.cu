// Reduced Hessian without any device allocation.
//
// opf_reduced_hessian sizes its per-tile workspace on the first call and
// allocates it with cudaMalloc.  Some callers cannot allow that: a real-time
// control loop that must not stall on the allocator (cudaMalloc can
// synchronise the whole device and its latency is unbounded), or a host
// process whose device-memory budget is fixed once at start-up.
// opf_reduced_hessian_noalloc computes the same Hessian with the same tile
// kernel, but its workspace is the fixed array below, so the call itself
// allocates nothing.
#include <algorithm>
#include <mutex>
#include <string>

#include "opf_internal.h"

using namespace opf;

namespace {

constexpr size_t kScratchBytes = (size_t)OPF_NOALLOC_SCRATCH_BYTES;
constexpr size_t kScratchDoubles = kScratchBytes / sizeof(double);
constexpr int kMaxDevices = 64;

// One workspace per GPU that loads the library, held until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {};

// Device address of the array on `device` (looked up once per device, with that
// device current).  In host code the array's name is only a stand-in symbol.
opf_status scratch_for_device(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_last_error("device ordinal out of range for the static workspace table");
    return OPF_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[device]) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) {
      set_last_error("cudaGetDevice failed");
      return OPF_ECUDA;
    }
    if (prev != device && cudaSetDevice(device) != cudaSuccess) {
      set_last_error("cudaSetDevice failed");
      return OPF_ECUDA;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess || !p) {
      set_last_error(std::string("cudaGetSymbolAddress of the static workspace failed: ") +
                     cudaGetErrorString(e));
      return OPF_ECUDA;
    }
    g_dev_ptr[device] = static_cast<double*>(p);
  }
  *out = g_dev_ptr[device];
  return OPF_OK;
}

}  // namespace

extern "C" opf_status opf_reduced_hessian_noalloc(opf_ctx* c, const opf_al_params* p,
                                                  const opf_hess_opts* o, double* H,
                                                  opf_hess_info* info) {
  if (!c || !H) {
    set_last_error("ctx and H are required");
    return OPF_EINVAL;
  }
  if (o && (o->plain || o->threads || o->reuse_first_order)) {
    set_last_error("opf_reduced_hessian_noalloc supports block_k, grid and the column range only "
                   "(plain, threads and reuse_first_order must be 0)");
    return OPF_EINVAL;
  }
  const int C = (o && o->block_k) ? o->block_k : 8;
  if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16 && C != 32) {
    set_last_error("block_k must be 1, 2, 4, 8, 16 or 32");
    return OPF_EINVAL;
  }
  const int nu = c->h.nu;
  const int col0 = o ? o->col_begin : 0;
  const int ncol = (o && o->col_count > 0) ? o->col_count : nu - col0;
  if (col0 < 0 || col0 >= nu || ncol < 1 || col0 + ncol > nu) {
    set_last_error("column range outside [0, n_u)");
    return OPF_EINVAL;
  }
  // the size limit depends on the network and block_k only
  const size_t stride = hvp_stride(c, C);
  if (stride > kScratchDoubles) {
    set_last_error("one tile of this network needs " + std::to_string(stride * sizeof(double)) +
                   " bytes of workspace, more than the " + std::to_string(kScratchBytes) +
                   "-byte static workspace; use a smaller block_k or opf_reduced_hessian");
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
  {
    const opf_status ps = check_al(c, p);
    if (ps != OPF_OK) return ps;
  }
  double* scratch = nullptr;
  opf_status st = scratch_for_device(c->device, &scratch);
  if (st != OPF_OK) return st;
  const int ntiles = hvp_tiles(c, C, col0, col0 + ncol, true);
  int grid = (o && o->grid > 0) ? o->grid : ntiles;
  grid = std::min(grid, (int)(kScratchDoubles / stride));
  grid = std::max(1, std::min(grid, ntiles));
  cudaEventRecord(c->ev[0], c->stream);
  launch_first_order(c, p, nullptr);
  launch_hess_prep(c, p->sigma_f);
  cudaEventRecord(c->ev[1], c->stream);
  launch_hvp_scratch(c, C, H, scratch, grid, ntiles, col0, col0 + ncol);
  cudaEventRecord(c->ev[2], c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("opf_reduced_hessian_noalloc: ") + cudaGetErrorString(e));
    return OPF_ECUDA;
  }
  if (info) {
    info->block_k = C;
    info->grid = grid;
    info->tiles = ntiles;
    info->launches = 1;
    info->asymmetry = -1.0;
    for (int k = 0; k < 5; k++) info->phase_ms[k] = 0.f;
    cudaEventElapsedTime(&info->ms_total, c->ev[0], c->ev[2]);
    cudaEventElapsedTime(&info->ms_hvp, c->ev[1], c->ev[2]);
  }
  return OPF_OK;
}
