// Internal declarations of libopf: the context, the host symbolic analysis and
// the kernel launchers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/opf.h"

namespace opf {

// Per-branch Hessian table rows (each row holds n_l doubles): 0..9 the packed
// symmetric 4x4 second derivative in branch-local order (v_f, v_t, theta_f,
// theta_t); 10+4s+k = dP of end s w.r.t. local variable k; 18+4s+k = dQ;
// 26+4s+k = d|S_s|^2 = 2 (P_s dP_s + Q_s dQ_s), the gradient of the end's
// flow constraint (the rows of the reduced Jacobian).
#define TAB_DP(s, k) (10 + 4 * (s) + (k))
#define TAB_DQ(s, k) (18 + 4 * (s) + (k))
#define TAB_DS(s, k) (26 + 4 * (s) + (k))
#define TAB_ROWS 34

// Per-adjacency coefficient record (bus i at end s of branch l, o the other
// end), ADJ_W doubles.  The branch functions depend on the angles only through
// theta_s - theta_o, so every theta_o derivative is the negated theta_s one.
// E_VO, E_VT, E_TO, E_TT: second derivatives of l in the rows of v_s / theta_s
// against v_o / theta_s; E_QO*, E_PO*: dQ_o, dP_o w.r.t. (v_s, theta_s);
// E_QS*, E_PS*: dQ_s, dP_s w.r.t. (v_s, v_o, theta_s); E_VV: d2l/dv_s^2.
#define ADJ_W 16
enum AdjField { E_VO = 0, E_VT = 1, E_TO = 2, E_TT = 3, E_QOV = 4, E_QOT = 5, E_POV = 6, E_POT = 7,
                E_QSV = 8, E_QSO = 9, E_QST = 10, E_PSV = 11, E_PSO = 12, E_PST = 13, E_VV = 14 };

enum BusType { REF = 0, PV = 1, PQ = 2 };

// Host-side network with index maps (eq. statecontrol).
struct HostNet {
  int nb = 0, nl = 0, ng = 0, ref = 0, npv = 0, npq = 0, nx = 0, nu = 0, m = 0;
  std::vector<int> f, t, gbus;
  std::vector<double> Y;  // 8 * nl: Gff, Bff, Gft, Bft, Gtf, Btf, Gtt, Btt (blocks of nl)
  std::vector<double> pd, qd, c2, c1, c0;
  std::vector<int> type, gen_at, pvpos, pqpos, xth, xv, uv, up;
  std::vector<int> adj_ptr, adj;  // bus -> incident entries, entry = 2 * branch + side
};

// Symbolic analysis of G_x (pivot order, filled pattern, level sets).
struct Symbolic {
  std::vector<int> bus_order, perm, iperm;
  std::vector<int> rp, ci, dp;     // row-wise filled pattern, pivot order
  std::vector<int> lev_f, lev_b;   // level of each row (forward / backward)
  int nlev_f = 0, nlev_b = 0;
};

// Returns an empty string on success, else the reason.
std::string build_hostnet(const opf_network_desc* d, HostNet& h);
void build_symbolic(const HostNet& h, Symbolic& s);

// Device views passed to kernels (plain pointers).
struct DevNet {
  int nb, nl, ng, ref, npv, npq, nx, nu, m, ngn, nnz;
  const int *f, *t, *gbus;
  const double* Y;
  const int *type, *gen_at, *pvpos, *pqpos, *xth, *xv, *uv, *up;
  const int *pth, *pvv;            // pivot-order index of theta / v of each bus (-1)
  const int *adj_ptr, *adj;
  const int* bus_by_deg;           // [nb] buses by descending degree (ties: ascending id)
  const int* gn_of;                // per bus: index among ref + PV buses (-1)
  const int* gn_bus;               // [ngn]
  const int* gn_by_deg;            // [ngn] indices into gn_bus by descending degree of the bus
  const double *c2, *c1;
  // LU pattern
  const int *rp, *ci, *dp, *perm;
  // execution schedule of the sweeps: level lists of the rows outside the dense
  // trailing block [r0, nx) (which is solved as a dense triangle)
  const int *lev_ptr_f, *lev_rows_f, *lev_ptr_b, *lev_rows_b;
  const int4 *lmeta_f, *lmeta_b;   // per scheduled row: {row, first entry, end entry, 0}
  int nlev_f, nlev_b;
  // bus-block schedules of the multi-column sweeps: the one or two pivot rows of a
  // bus (theta, v of a PQ bus are consecutive and share their off-block pattern)
  // are solved together.  Record {lead row, first shared entry, end, offset}: the
  // lead row's entries [q0, q1) and the other row's entries at q + offset
  // (offset 0: a one-row block).  Forward: other = lead + 1, coupling entry
  // q1 + offset; backward: other = lead - 1, coupling entry q0 + offset - 1.
  const int *bptr_f, *bptr_b;
  const int4 *bmeta_f, *bmeta_b;
  int nblev_f, nblev_b;
  // the backward levels again for the L^T sweep of a symmetric Hessian tile:
  // each level's blocks by descending lt_q (then length), where lt_q of a block
  // is the last position, in the full-Hessian column order, of a control whose
  // right-hand-side rows have one of the block's rows as an elimination-tree
  // ancestor; a tile whose first column position is p needs Psi exactly on the
  // blocks with lt_q >= p, a prefix of every level (qpos: the position of each
  // control in that order)
  const int4* bmeta_lt;
  const int *lt_q, *qpos;
  int r0, nroot;
  const int* slot_self;            // [4 * nb]: P-theta, P-v, Q-theta, Q-v
  const int* slot_adj;             // [4 * 2 nl]
  // direction records of the HVP gathers.  A direction slot z >= 0 is the
  // pivot-order row holding the value; z <= -2 encodes a control unit vector
  // (the value is 1 in the column of control -2 - z, else 0); -1 means none.
  const int* eparent;              // [nx] elimination-tree parent of each pivot row (-1 at a root)
  const int* lcol_ptr;             // [nx + 1] columns of L (CSC): entries lcol_ptr[j] ..
  const int2* lcol;                // per entry {row, position in LU}, rows ascending
  const int4* busrec;              // [nb]: {v slot, theta slot, control-bus index or -1, up or -1}
  const int4* adjrec;              // [2 nl], adjacency order: the other end's {v slot, theta slot,
                                   //   control-bus index or -1, 1 if it is the slack}
};

// Arguments of the HVP tile kernels (one network, one Hessian).
struct HvpArgs {
  DevNet n;
  const double *LU, *T, *invdiag, *tab, *busw;
  const double* adjE;  // [2 nl][ADJ_W] per-adjacency coefficients
  const double* busS;  // [nb] x 4 per-bus coefficient sums
  const int* ubus;  // bus of each control
  const int* colmap;  // null: tile position p is column col0 + p; else column colmap[p] (-1: none)
  double* H;
  double* J;            // null, or the reduced constraint Jacobian [n_u][m] (column j at J + j m)
  int jac_only;         // 1: the tiles stop after J (H untouched, may be null)
  double* scratch;
  unsigned long long* stamps;  // null, or [tiles][8] phase stamps per tile (hvp_stamp)
  size_t stride;    // doubles of scratch per CTA
  int ntiles, first_tile, tile_step;
  int col0, col_end;  // columns computed: col0 .. col_end - 1
  // dynamic shared memory of the tile (hvp_smem_bytes): reached-row values
  // [zs_cap][C], reach mask and its word prefix [rm_words] each, reach list [list_cap]
  int zs_cap, rm_words, list_cap;
  // symmetric full Hessian: a tile computes only the rows of the controls at or
  // after its first column position (pruning the L^T sweep to their Psi rows)
  // and records that position per column in tstart; a mirror kernel fills the
  // rest from the transposed entries
  int sym;
  int* tstart;
  // 1: each tile's slab already holds its first adjoint Z from the previous
  // launch with the same tiling and factors (one tile per CTA, each with its
  // own slab): phases (0)-(2) are skipped.  Z = G_x^{-1} G_u W does not depend
  // on the second-order weights, so a QP's Hessians at one linearisation
  // point share it.
  int zreuse;
};

// Shared memory of the trailing dense block's LU (the whole block; larger blocks
// are factorised in global memory).
constexpr int kDenseLuSmem = 200 * 1024;

// Dynamic shared memory of the HVP tile kernels (bytes; opted in at load).
constexpr int HVP_DYN_SMEM = 56 * 1024;
constexpr int kSplitMaxSm = 1024;  // SM ids the split launch counts CTAs for
size_t hvp_smem_bytes(const HvpArgs& a, int C);
int hvp_smem_budget(int C);  // dynamic shared memory a tile of width C may use (<= HVP_DYN_SMEM)
void setup_hvp_smem();

// kernel launchers (opf_kernels.cu)
void launch_unpack(opf_ctx* c, const double* x, const double* u);
void launch_pf_eval(opf_ctx* c);
void launch_lu(opf_ctx* c);          // replays the captured refactorisation graph
void launch_lu_kernels(opf_ctx* c);  // the kernel sequence itself (captured at load)
void launch_solve1(opf_ctx* c, const double* b, double* out, bool transposed, double scale);
opf_status setup_solve1(opf_ctx* c);  // shared-memory size of the single-RHS sweep
void launch_axpy(opf_ctx* c, double* x, const double* d, double a, int n);
void launch_first_order(opf_ctx* c, const opf_al_params* p, double* grad_s);
void launch_eval_F(opf_ctx* c, const opf_al_params* p, double* F_out);  // F only, into device F_out
void launch_grad_u(opf_ctx* c, double* gu);
// sigma_c [m] and sigma_f [1] (device) of the gradient-based scaling from J
// (m x n_u column-major), the cost gradient gf [n_u] and an optional prior [m]
void launch_grad_scaling(opf_ctx* c, const double* J, const double* gf, double g_max, double s_min,
                         const double* prior, double* sigma_c, double* sigma_f);
void launch_grad_load(opf_ctx* c, double sigma_f, double* gpd, double* gqd);
void launch_hess_prep(opf_ctx* c, double sigma_f);
size_t hvp_stride(const opf_ctx* c, int C);
// sums[0] += ||H - H^T||_F^2, sums[1] += ||H||_F^2 (H: n x n column-major)
void launch_hess_asymmetry(opf_ctx* c, const double* H, int n, double* sums);
void launch_hess_mirror(opf_ctx* c, double* H, int n);  // completes a symmetric Hessian (HvpArgs::sym)
bool launch_hvp(opf_ctx* c, int C, double* H, int grid, int first_tile, int tile_step, int ntiles,
                int col0, int col_end);
bool launch_hvp_scratch(opf_ctx* c, int C, double* H, double* scratch, int grid, int ntiles, int col0,
                        int col_end);
void set_last_error(const std::string& msg);  // message returned by opf_last_error
opf_status ensure_factors(opf_ctx* c);  // factorise the converged state's Jacobian if still pending
opf_status check_al(const opf_ctx* c, const opf_al_params* p);  // AL inputs present, rho >= 0, sigma_f finite
opf_status zero_params(opf_ctx* c, opf_al_params* q);  // sigma_f = rho = 0, zero [m] arrays
// balanced: the single-network launch (tiles in whole waves over the SMs)
HvpArgs make_hvp_args(opf_ctx* c, int C, double* H, int col0, int col_end, bool balanced);
int hvp_tiles(const opf_ctx* c, int C, int col0, int col_end, bool balanced);  // tiles of a column range
// The full Hessian as split_n1 tiles of width C and split_n2 of width C / 2 in
// one launch (false when the context has no split tiling at this width).
bool launch_hvp_split(opf_ctx* c, int C, double* H);
size_t hvp_split_scratch(const opf_ctx* c, int C);  // doubles of workspace it needs
// z [n_x] = (dx/du) d from the first adjoints the last split Hessian launch left
// in its slabs (valid while the factors and the slabs are those of that launch);
// false (nothing launched) when they are not
bool launch_state_direction(opf_ctx* c, const double* d, double* z);
// out [n_u] = base + G_u^T lambda with lambda = -G_x^{-T} w [n_x], from the same
// slabs (false, nothing launched, when they do not hold the first adjoints)
bool launch_adjoint_from_slabs(opf_ctx* c, const double* w, const double* base, double* out);
// The plain form: Hessian columns col0 .. col_end - 1 one at a time, each a
// sequence of device-wide launches around two streamed single-RHS solves;
// work holds hvp_plain_scratch doubles.  Returns the kernels launched.
size_t hvp_plain_scratch(const opf_ctx* c);
int launch_hvp_plain(opf_ctx* c, double* H, int col0, int col_end, double* work);
int hvp_batch_occupancy(int C);  // resident CTAs per SM of the batched tile kernel
int hvp_occupancy(int C, int nt);  // resident CTAs per SM of hvp_tile_kernel<C, nt>
bool launch_hvp_batch(cudaStream_t st, int C, const HvpArgs* args, const int2* tiles, int ntot, int* counter,
                      double* scratch, size_t stride, int grid, size_t smem);
// J^T w for the reduced constraint Jacobian: the adjoint gradient with first-order
// weights w and no cost (sigma_f = 0); needs the flows of the current state.
void launch_weighted_grad(opf_ctx* c, const double* w, double* out);
void launch_omega(opf_ctx* c, const opf_al_params* p);  // omega (and phi') alone, from the last first order
struct StepWork;
void free_step_work(opf_ctx* c);
// KKT errors of a barrier subproblem at st with gradient (gu, gs) (opf_al.cu):
// red[0..3] (zeroed by the caller) = max |g - z_lo + z_hi|, max complementarity
// error at mu, at 0, and max |sigma_c (c - s)| (0 when cv is null).
void launch_al_kkt(opf_ctx* c, const double* gu, const double* gs, const opf_al_state* st, const double* cv,
                   const double* sig, double mu, double* red);
// y += rho sigma_c (c - s)
void launch_al_dual_update(opf_ctx* c, double* y, double rho, const double* sig, const double* cv,
                           const double* s);

#ifdef __CUDACC__
// Programmatic dependent launch: a kernel launched by launch_pdl may start while
// the previous kernel on its stream drains; it must call pdl_wait() before it
// reads anything that kernel writes, and calls pdl_trigger() once its own work
// is issued (exiting counts as the trigger).  (The LU level kernel triggers
// right after its wait instead: its grids are one wave, so the next level's CTAs
// may sit resident early; for the Cholesky kernels, whose grids take the whole
// GPU, an early trigger made the factorisation ~0.2 ms slower.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// 1 / u by the Newton-Raphson iteration for the reciprocal, r <- r + r (1 - u r)
// (each step squares the relative error), from the hardware's approximate FP64
// reciprocal: two steps reach full double precision for normal u (equal to
// IEEE 1 / u except for u just below a power of two (every mantissa bit set),
// where the result is one unit in the last place off; subnormal and zero u give NaN, which the pivot checks catch,
// and so does a subnormal result).  It issues
// one MUFU and four DFMA where the IEEE division issues a longer FP64 sequence,
// which matters where many warps each divide once (the FP64 pipe runs one warp
// instruction per ~20 cycles whatever the active lanes).
__device__ __forceinline__ double recip_nr(double u) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(u));
  double e = fma(-u, r, 1.0);
  r = fma(r, e, r);
  e = fma(-u, r, 1.0);
  return fma(r, e, r);
}

// Work items of the right-looking LU by bus blocks (one level's tasks, and the
// finish records of the previous level's two-row blocks), each on a lane group
// of G lanes (li: lane in the group; gmask: the group's lanes).  CG: the factor
// is read past L1 (a launch that runs several levels, where other CTAs' updates
// of one level land in L2 before the next).
template <bool CG>
__device__ __forceinline__ double lu_ld(const double* p) {
  if (CG) return __ldcg(p);
  return *p;
}
// Task {position of A_rf, dp[f], rp[f + 1], dp[f + 1] or -1}: for row r below the
// block, l_f = A_rf / U_ff and, for a two-row block, l_v = (A_r,f+1 - l_f U_f,f+1)
// / U_vv with the block's own U_vv = A_vv - (A_vf / U_ff) U_f,f+1 formed on the
// fly; then every column c of row f past the block gets A_rc -= l_f U_fc +
// l_v (A_vc - L_vf U_fc) at its precomputed target tg[c - first] (atomics: the
// tasks of a level may share targets).  The lane groups are sized so that a
// lane takes at most LU_PRE columns: their entries and targets are read in the
// same round as the pivots (nothing the task writes aliases them), so the task
// waits for L2 once instead of once per column step.
constexpr int LU_PRE = 4;
// The task's first LU_PRE targets per lane (static: a launch may read them
// before it waits for the previous level).
__device__ __forceinline__ void lu_targets(const int4 tr, const int* __restrict__ tg, int li, int G,
                                           int (&tgt)[LU_PRE]) {
  const int q0 = tr.y + (tr.w >= 0 ? 2 : 1);
#pragma unroll
  for (int k = 0; k < LU_PRE; k++) {
    const int q = q0 + li + k * G;
    tgt[k] = q < tr.z ? __ldg(tg + (q - q0)) : 0;
  }
}
template <bool CG>
__device__ __forceinline__ void lu_task(double* LU, const int4 tr, const int* __restrict__ tg,
                                        const int (&tgt)[LU_PRE], int li, int G, unsigned gmask, int* flags) {
  const bool two = tr.w >= 0;
  const int q0 = tr.y + (two ? 2 : 1), qv = tr.w + 1;
  double ufc[LU_PRE], avc[LU_PRE];
#pragma unroll
  for (int k = 0; k < LU_PRE; k++) {
    const int q = q0 + li + k * G;
    const bool in = q < tr.z;
    ufc[k] = in ? lu_ld<CG>(LU + q) : 0.0;
    avc[k] = (in && two) ? lu_ld<CG>(LU + qv + (q - q0)) : 0.0;
  }
  const double uff = lu_ld<CG>(LU + tr.y);
  const double inv_ff = recip_nr(uff);
  const double arf = lu_ld<CG>(LU + tr.x);
  const double lf = arf * inv_ff;
  double lv = 0.0, lvf = 0.0;
  if (two) {
    // l_v = (A_rv - l_f U_fv) / (A_vv - L_vf U_fv), both scaled by U_ff so that
    // its reciprocal runs beside 1 / U_ff instead of after it
    const double ufv = lu_ld<CG>(LU + tr.y + 1), avf = lu_ld<CG>(LU + tr.w - 1);
    const double avv = lu_ld<CG>(LU + tr.w), arv = lu_ld<CG>(LU + tr.x + 1);
    lvf = avf * inv_ff;
    lv = fma(arv, uff, -arf * ufv) * recip_nr(fma(avv, uff, -avf * ufv));
  }
  __syncwarp(gmask);
  if (li == 0) {
    LU[tr.x] = lf;
    if (two) LU[tr.x + 1] = lv;
    if (!(fabs(uff) > 0.0) || !isfinite(lf) || !isfinite(lv)) flags[0] = 1;
  }
#pragma unroll
  for (int k = 0; k < LU_PRE; k++) {
    if (q0 + li + k * G < tr.z) {
      double d = lf * ufc[k];
      if (two) d += lv * (avc[k] - lvf * ufc[k]);
      atomicAdd(&LU[tgt[k]], -d);
    }
  }
  for (int q = q0 + li + LU_PRE * G; q < tr.z; q += G) {  // wider rows than the lane sizing gives
    const double u = lu_ld<CG>(LU + q);
    double d = lf * u;
    if (two) d += lv * (lu_ld<CG>(LU + qv + (q - q0)) - lvf * u);
    atomicAdd(&LU[tg[q - q0]], -d);
  }
}
// Finish record {dp[f], rp[f + 1], dp[f + 1]} of a two-row block: L_vf, U_vv and
// the second row's upper entries after eliminating f (no task reads them any
// more); the row entries are read in the pivots' round as in lu_task.
template <bool CG>
__device__ __forceinline__ void lu_finish(double* LU, const int4 fr, int li, int G, unsigned gmask) {
  const int p0 = fr.x + 2, w0 = fr.z + 1;
  double uq[LU_PRE], vq[LU_PRE];
#pragma unroll
  for (int k = 0; k < LU_PRE; k++) {
    const int q = p0 + li + k * G;
    const bool in = q < fr.y;
    uq[k] = in ? lu_ld<CG>(LU + q) : 0.0;
    vq[k] = in ? lu_ld<CG>(LU + w0 + (q - p0)) : 0.0;
  }
  const double uff = lu_ld<CG>(LU + fr.x);
  const double lvf = lu_ld<CG>(LU + fr.z - 1) * recip_nr(uff);
  const double ufv = lu_ld<CG>(LU + fr.x + 1);
  const double avv = lu_ld<CG>(LU + fr.z);
#pragma unroll
  for (int k = 0; k < LU_PRE; k++) {
    const int q = p0 + li + k * G;
    if (q < fr.y) LU[w0 + (q - p0)] = vq[k] - lvf * uq[k];
  }
  for (int q = p0 + li + LU_PRE * G; q < fr.y; q += G)
    LU[w0 + (q - p0)] = lu_ld<CG>(LU + w0 + (q - p0)) - lvf * lu_ld<CG>(LU + q);
  __syncwarp(gmask);
  if (li == 0) {
    LU[fr.z - 1] = lvf;
    LU[fr.z] = avv - lvf * ufv;
  }
}
#endif

// Level-packed single-RHS sweeps (opf_sweep.cu).  The factor entries a sweep
// reads are copied after each refactorisation into one contiguous stream per
// (factor, direction): first the dense trailing triangle (packed by rows) and
// 1 / U_rr of the trailing rows, then the levels, cut into chunks at block
// boundaries so that each chunk fits a shared-memory ring slot.  Chunk c holds
// a 32-byte header {records, warp tasks, padded entries, padded record values,
// offset and length of chunk c + 2}, per warp task the record and group lane
// of each of its 32 lanes, the records {lead row, entries, second row or -1,
// first entry}, per record {coupling, scale of the lead row, scale of the
// second row}, and the entries' columns, lead-row values and second-row values.
struct SweepStream {
  const unsigned char* base = nullptr;  // device bytes of the stream
  int tri_len = 0;                      // bytes of the trailing-triangle segment at the start
  int nch = 0;                          // chunks
  int off0 = 0, len0 = 0, off1 = 0, len1 = 0;  // the first two chunks (bytes)
};
struct SweepStreams {
  bool ok = false;       // false: the sweep keeps the level-record form (sweep1)
  int slot = 0;          // ring slot bytes
  int smem = 0;          // dynamic shared bytes of the streamed solve
  SweepStream s[4];      // L of LU (forward), U of LU (backward), U^T from T (forward), L^T from T (backward)
  int2* map = nullptr;   // {destination double, source}: source 2p (LU) / 2p + 1 (T), or -1 - row (1 / U_rr)
  int nmap = 0;
  int* d_nmap = nullptr;     // nmap on the device (read by the captured gather)
  double* values = nullptr;  // the streams' bytes, as doubles for the gather
  size_t cap_bytes = 0, cap_map = 0;  // capacity of values (bytes) and map (entries)
  size_t fixed = 0, tri_bytes = 0, max_slot = 0;  // solution bytes, triangle segment, largest ring slot
  int lookahead = 0, narrow = 0;  // level-merge schedule of the streams (set_sweep_merge)
  std::vector<int> h_bptr_f, h_bptr_b;  // the bus-block level schedules the streams are built from
  std::vector<int4> h_bmeta_f, h_bmeta_b;
};
// Default level-merge schedule of the streamed sweeps: look-ahead distance in
// chunks and the largest chunk (records) that is merged.
constexpr int kSweepLookahead = 4;
constexpr int kSweepNarrow = 4;
// FP64 rank-K update of a lower triangle emulated on bf16 tensor cores
// (opf_ozaki.cu): A[r0 :, r0 :] -= P P^T with P = A[r0 : n, c0 : c0 + K],
// K <= 128 a multiple of 32; E: n - r0 ints, D: 8 (n - r0) K bf16 workspace.
// Dense LU of the trailing block on one thread-block cluster (opf_lu_dense.cu):
// the cluster size for a block of s rows (0: the one-CTA kernel), and the launch.
// The cluster also runs the last sparse levels [lv0, nlev] first (lvrec: per
// level {t0, t1, f0, f1} task and finish ranges, lanes: lane-group width), one
// cluster barrier per level instead of one launch.
constexpr int kLuClusterThreads = 256;
int setup_lu_dense_cluster(int s);
struct LuTail {
  const int4* task_rec = nullptr;
  const int* task_off = nullptr;
  const int* task_map = nullptr;
  const int4* fin_rec = nullptr;
  const int4* lvrec = nullptr;  // indexed by level
  const int* lanes = nullptr;   // indexed by level
  int lv0 = 0, lv1 = 0;         // levels [lv0, lv1) run in the cluster
};
void launch_lu_dense_cluster(cudaStream_t st, int K, double* LU, const int* dp, int r0, int s, int* flags,
                             const LuTail& tail);

opf_status setup_oz();
// Which tensor-core engine runs the emulated update: 0 the tcgen05 kernel (TMEM
// accumulators; its bounded mbarrier waits record a timeout in *err, polling at
// most lim times) for updates of at least OZ_TC_MIN_TILES 128 x 64 tiles and the
// warp-level mma.sync kernel for smaller ones (whose latency the 128-row tiles
// do not hide); 1 mma.sync only; 2 tcgen05 only.
constexpr int OZ_TC_MIN_TILES = 80;
struct OzEngine {
  int engine = 0;
  int* err = nullptr;
  long long lim = 1ll << 24;
  int sm_count = 148;
};
void launch_oz_update(cudaStream_t st, double* A, int n, int c0, int K, int r0, int* E, void* D, const int* flag,
                      const OzEngine& eng);
// the halves of launch_oz_update: digits, then the tiles of one part (0 all,
// 1 the first 128 columns, 2 the rest) on at most grid CTAs (0: one per tile)
// with the warp-level MMAs, or the whole triangle with tcgen05
void launch_oz_slice(cudaStream_t st, const double* A, int n, int c0, int K, int r0, int* E, void* D,
                     const int* flag, bool tiled);
// rows of the core-matrix digit layout of an M-row panel (M rounded up to 128);
// the digit workspace holds 8 oz_rows_tiled(M) K bf16
inline int oz_rows_tiled(int M) { return (M + 127) / 128 * 128; }
void launch_oz_syrk(cudaStream_t st, double* A, int n, int K, int r0, const int* E, const void* D, const int* flag,
                    int part, int grid);
void launch_oz_syrk_tc(cudaStream_t st, double* A, int n, int K, int r0, const int* E, const void* D,
                       const int* flag, int* err, long long lim, int sm_count);

opf_status setup_sweep_streams(opf_ctx* c, const std::vector<int>& bptr_f, const std::vector<int4>& bmeta_f,
                               const std::vector<int>& bptr_b, const std::vector<int4>& bmeta_b);
void launch_sweep_pack(opf_ctx* c);  // after a refactorisation (captured in the LU graph)
opf_status set_sweep_merge(opf_ctx* c, int lookahead, int narrow);  // rebuild the streams in place
void launch_solve1_streamed(opf_ctx* c, const double* b, double* out, bool transposed, double scale);

}  // namespace opf

struct opf_ctx {
  opf::HostNet h;
  opf::Symbolic s;
  opf::DevNet dn;
  cudaStream_t stream = nullptr;
  int device = 0, sm_count = 0;
  std::vector<void*> allocs;

  // device: LU values and schedules
  double *LU = nullptr, *T = nullptr, *invdiag = nullptr;
  int* tmap = nullptr;
  int *lcol_pos = nullptr;        // per lower entry (CSC order): position of L_rj in row r
  int *lcol_row = nullptr;
  // LU by bus blocks (see load_impl): task records, target offsets and targets,
  // finish records of two-row blocks; per block level the task and finish ranges
  int4* task_rec = nullptr;
  int* task_off = nullptr;
  int* task_map = nullptr;
  int4* fin_rec = nullptr;
  std::vector<int> h_task_ptr, h_fin_ptr;
  std::vector<int> h_lu_lanes;      // per launch of the LU levels: lanes per work item
  int4* lu_lvrec = nullptr;         // per launch {t0, t1, f0, f1}
  int* lu_lanes = nullptr;          // h_lu_lanes on the device
  int lu_tail_from = 0;             // first level launch run inside the dense block's cluster
  std::vector<int> h_lev_ptr_f, h_lev_ptr_b;

  // device: state of the last converged power flow
  double *x = nullptr, *u = nullptr, *pd = nullptr, *qd = nullptr;
  double *pd_nom = nullptr, *qd_nom = nullptr, *c0 = nullptr;
  int* ubus = nullptr;            // bus of each control (v_ref, v_pv, p_pv)
  // full-Hessian tilings, per block width C = 1 << k and form f (0: ceil(n_u / C)
  // tiles, for the batched launch; 1: whole waves over the SMs when the tiles
  // stay at least half full): colmap[f][k] holds coltiles[f][k] x C columns
  // (-1 = idle lane), heaviest tiles first
  int* colmap[2][6] = {};
  int coltiles[2][6] = {};
  // split tiling of the full Hessian at width C = 1 << k: split_n1[k] tiles of
  // width C (whole waves over the SMs) then split_n2[k] <= SMs tiles of width
  // C / 2 for the rest; colmap_split[k] holds n1 x C then n2 x C/2 columns
  int* colmap_split[6] = {};
  int split_n1[6] = {}, split_n2[6] = {};
  int* split_ctr = nullptr;  // the split launch's tile queues and per-SM CTA counts (4 + kSplitMaxSm)
  int* tstart = nullptr;     // [n_u] first column position of each column's tile (symmetric Hessian)
  double *vbus = nullptr, *thbus = nullptr;
  double *g = nullptr, *dvec = nullptr, *yvec = nullptr;
  double* scal = nullptr;         // [8] reductions: |g|^2, |g|_inf bits, F, ...
  int* flags = nullptr;           // [4] set by kernels: [0] bad pivot, [1] a bounded wait gave up;
                                  // [2] spin limit of the bounded waits (0: each kernel's default)
  int wait_limit = 0;             // host copy of flags[2] (opf_set_wait_limit)
  double* h_scal = nullptr;       // pinned host mirror of scal
  int* h_flags = nullptr;         // pinned host mirror of flags
  bool have_state = false;
  bool factors_stale = false;     // LU holds the unfactorised Jacobian of the converged state

  // gradient / Hessian workspaces
  double *flows = nullptr;        // [4 nl]: Pf, Qf, Pt, Qt
  double *Pbus = nullptr, *Qbus = nullptr;
  double *cvec = nullptr, *phid = nullptr, *omega = nullptr;
  double *dFx = nullptr, *dFu = nullptr, *lam = nullptr;
  double *dFx_w = nullptr, *dFu_w = nullptr, *lam_w = nullptr;  // launch_weighted_grad's own
  double *btab = nullptr;         // [TAB_ROWS nl] per-branch Hessian table
  double *busw = nullptr;         // [8 nb]: kQ, kP, diag v, diag p, dQi/dvi, dQi/dthi, dPi/dvi, dPi/dthi
  double* adjE = nullptr;         // [2 nl][ADJ_W] per-adjacency coefficients of the HVP gathers
  double* busS = nullptr;         // [nb] x 4: per-bus sums of E_VV (+ omega of v_pq), E_VT, E_TT, 0
  double* endflow = nullptr;      // [2 nl][10] branch-end terms of the power-flow residual and Jacobian
  int hvp_threads = 256;          // threads per HVP tile CTA
  int solve1_smem = 0;            // dynamic shared bytes of the single-RHS sweep
  bool solve1_use_smem_rhs = false;  // the right-hand side also lives in shared memory
  double* scratch = nullptr;      // HVP per-CTA slabs
  unsigned long long* stamps = nullptr;  // phase stamps of a profiling Hessian call
  size_t stamps_cap = 0;          // tiles the stamps array holds
  bool stamps_on = false;         // the HVP launches of this call record phase stamps
  double* jac_out = nullptr;      // the HVP launches of this call also write J columns here
  bool jac_only = false;          // ... and stop after them (opf_reduced_jacobian without H)
  double* zeros_m = nullptr;      // [m] zeros: AL inputs of the multiplier-free evaluations (first use)
  double* gscale = nullptr;       // [n_u + 1]: cost gradient and sigma_f of opf_gradient_scaling (first use)
  size_t scratch_bytes = 0;
  cudaEvent_t ev[4];
  long long launches = 0;         // kernels launched by this context
  opf::StepWork* stepw = nullptr;  // reduced-Newton step workspace (first opf_al_step)
  int tuned_k = 0, tuned_threads = 0;  // opf_hessian_autotune's choice (0 = none)
  int chol_mode = 1;               // dense Cholesky trailing updates (opf_set_cholesky_mode)
  bool hess_sym = true;            // full Hessians by symmetry (opf_set_hessian_symmetry)
  bool sym_now = false;            // set for the duration of one such launch
  // first-adjoint reuse across split Hessian launches (HvpArgs::zreuse): allowed
  // by the caller (z_reuse), valid while the factors (lu_gen) and the tile width
  // are those of the last split launch (z_gen, z_C); other users of the
  // scratch clear z_gen
  bool z_reuse = false;
  long long lu_gen = 0, z_gen = -1;
  int z_C = 0;
  // set by a caller whose Hessians share the state and first-order weights and
  // differ in omega only (the tracking QP): the Hessian entry refreshes omega
  // and keeps c, phi', lambda of the previous call
  bool fo_reuse = false;
  int oz_engine = 0;               // emulated updates: 0 tcgen05 for large ones, 1 mma.sync, 2 tcgen05 (opf_set_update_engine)
  void* batch_buf = nullptr;       // batched-Hessian argument and tile tables (grown on demand)
  size_t batch_bytes = 0;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t worker = nullptr;   // the context's own stream inside a batched call (created on first use)
  cudaEvent_t worker_ev[2] = {};   // ordering between the caller's stream and the worker stream
  cudaGraphExec_t lu_exec = nullptr;
  long long lu_graph_kernels = 0;
  opf::SweepStreams sw;            // level-packed single-RHS sweep streams
  int lu_dense_cluster = 0;        // CTAs of the trailing block's cluster LU (0: one CTA)
};
