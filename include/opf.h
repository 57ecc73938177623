/*
 * opf.h -- C ABI of the B300 reduced-space OPF library (libopf.so).
 *
 * Method: feasible reduced-space optimal power flow (Pacaud, Maldonado,
 * Shin, Schanen, Anitescu, arXiv 2110.02590).  The library evaluates, on one
 * GPU and in FP64, the hot path of the method:
 *   - the Newton-Raphson power flow that keeps every iterate on g(x,u) = 0
 *     (eq. projection:newtonraphson, Sec. III-A), with a numeric LU
 *     refactorisation of G_x = dg/dx on a sparsity pattern fixed at load;
 *   - the reduced gradient of the scaled augmented Lagrangian by the adjoint
 *     method (Prop. 1, Sec. III-B; eq. gradient_auglag, Sec. IV-A);
 *   - the dense reduced Hessian from batched adjoint-adjoint Hessian-vector
 *     products (Prop. 2, Sec. III-B; Sec. III-C "Reduced Hessian").
 *
 * Notation and layouts (all FP64, per unit):
 *   buses 0..n_bus-1; ref_bus carries exactly one generator; the PV buses are
 *   the other generator buses and the PQ buses the rest, both in ascending id;
 *   u = (v_ref, v_pv, p_pv), n_u = 1 + 2 n_pv          (eq. statecontrol)
 *   x = (theta_pv, theta_pq, v_pq), n_x = n_pv + 2 n_pq
 *   g = (P_pv - p_pv + pd_pv, P_pq + pd_pq, Q_pq + qd_pq), P,Q = injections
 *   c = (|S_f|^2 per branch, |S_t|^2 per branch, v_pq, p_ref, q_ref, q_pv),
 *       m = 2 n_branch + n_pq + n_pv + 2                  (Sec. II-B, IV-A)
 *   F = sigma_f f + sum_i [ y_i sigma_i (c_i - s_i) + rho/2 sigma_i^2 (c_i - s_i)^2 ]
 *       (scaled augmented Lagrangian, Sec. IV-A "Scaling"), f = generation cost.
 *   Branches use the pi model: series y = 1/(r + jx), tap on the from side,
 *   charging b/2 at each end.
 *
 * Conventions: every call is ordered on the context's CUDA stream; pointers
 * are device pointers owned by the caller unless marked (host); outputs that
 * are host structs are valid when the call returns (the call synchronises
 * the stream).  No call throws or aborts: failures return an opf_status.
 * The library never falls back to the CPU.
 */
#ifndef OPF_H
#define OPF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OPF_OK = 0,
  OPF_EINVAL = 1,     /* bad argument or network (message: opf_last_error) */
  OPF_ENOMEM = 2,     /* device or host allocation failed */
  OPF_ECUDA = 3,      /* a CUDA runtime call failed */
  OPF_ENOCONV = 4,    /* Newton-Raphson hit max_it or produced a non-finite residual */
  OPF_ESINGULAR = 5,  /* a zero or non-finite pivot in the LU refactorisation */
  OPF_ENOTPD = 6,     /* dense Cholesky failed after the inertia corrections */
  OPF_ESTATE = 7,     /* gradient/Hessian requested without a converged power flow */
  OPF_ETIMEOUT = 8    /* a bounded device-side wait gave up (opf_set_wait_limit) */
} opf_status;

typedef struct opf_ctx opf_ctx;

/* Network description (all arrays host, copied at load). */
typedef struct {
  int n_bus, n_branch, n_gen, ref_bus;
  const double *pd, *qd;               /* nominal loads [n_bus] */
  const double *vmin, *vmax;           /* voltage bounds [n_bus] */
  const int *br_from, *br_to;          /* branch ends [n_branch] */
  const double *br_r, *br_x, *br_b;    /* series r, x, total charging b [n_branch] */
  const double *br_tap, *br_rate;      /* off-nominal tap (1 = line), MVA rating [n_branch] */
  const int *gen_bus;                  /* one generator per bus at most [n_gen] */
  const double *gen_c2, *gen_c1, *gen_c0;  /* cost c2 p^2 + c1 p + c0, p in p.u. [n_gen] */
  const double *gen_pmin, *gen_pmax, *gen_qmin, *gen_qmax;  /* [n_gen] */
  double base_mva;
} opf_network_desc;

/*
 * opf_load_network: validate the network, build the index maps (eq.
 * statecontrol), run the symbolic analysis of G_x once (exact minimum degree
 * on the bus graph, filled pattern, level sets; Sec. V-A "Sparse linear
 * system": the pattern is fixed by the topology), upload everything and
 * allocate all workspaces.  `stream` is a cudaStream_t (NULL = legacy
 * default stream).  Errors: OPF_EINVAL (branch end out of range or a
 * self-loop, r = x = 0, two generators on a bus, no generator on ref_bus,
 * a state bus not connected to the slack), OPF_ENOMEM, OPF_ECUDA.
 * On success *out owns all device memory until opf_free.
 */
opf_status opf_load_network(const opf_network_desc* desc, void* stream, opf_ctx** out);
void opf_free(opf_ctx* ctx);
opf_status opf_set_stream(opf_ctx* ctx, void* stream);

/* Sizes (host outputs; any pointer may be NULL). */
opf_status opf_dims(const opf_ctx* ctx, int* nx, int* nu, int* m, int* npv, int* npq);

/*
 * Symbolic analysis export, for bit-exact comparison (host outputs).
 * opf_symbolic_sizes: nnz of the filled pattern (L + U + diagonal), number of
 * state buses (n_bus - 1), number of forward and backward levels.
 * opf_symbolic_export: bus_order[n_state_bus] (elimination order of the
 * buses), perm[n_x] (perm[k] = x index of the k-th pivot; the variables of a
 * bus are consecutive, theta before v), rowptr[n_x+1] and colidx[nnz] (row-wise
 * filled pattern in pivot order, sorted), lev_f[n_x] (level of row k of L:
 * 1 + the largest level among its off-diagonal columns, 0 if none), lev_b[n_x]
 * (the same for the rows of U, counted from the last row).
 */
opf_status opf_symbolic_sizes(const opf_ctx* ctx, int* nnz, int* n_state_bus, int* n_lev_f,
                              int* n_lev_b);
opf_status opf_symbolic_export(const opf_ctx* ctx, int* bus_order, int* perm, int* rowptr,
                               int* colidx, int* lev_f, int* lev_b);

/*
 * Host-only symbolic analysis (no GPU needed): the same ordering, filled
 * pattern and level sets that opf_load_network computes, for callers that
 * want to inspect or compare the integer structures.  Export layout as for
 * opf_symbolic_export.  Errors: OPF_EINVAL (invalid network).
 */
typedef struct opf_symbolic opf_symbolic;
opf_status opf_symbolic_analyze(const opf_network_desc* desc, opf_symbolic** out);
opf_status opf_symbolic_info(const opf_symbolic* sym, int* nx, int* nnz, int* n_state_bus,
                             int* n_lev_f, int* n_lev_b);
opf_status opf_symbolic_get(const opf_symbolic* sym, int* bus_order, int* perm, int* rowptr,
                            int* colidx, int* lev_f, int* lev_b);
void opf_symbolic_free(opf_symbolic* sym);

typedef struct {
  double tol;  /* stop when ||g||_2 < tol (the paper uses 1e-10, Sec. V-A) */
  int max_it;  /* Newton updates allowed (default 20) */
} opf_pf_opts;

typedef struct {
  int iterations;   /* Newton updates performed */
  double res2;      /* ||g||_2 at the returned x */
  double resinf;    /* ||g||_inf at the returned x */
} opf_pf_info;

/*
 * opf_powerflow: Newton-Raphson x <- x - G_x^{-1} g (eq.
 * projection:newtonraphson) at controls u[n_u] and loads pd, qd [n_bus]
 * (NULL = the nominal loads of the description), starting from
 * x_inout[n_x] and overwriting it.  Each iteration evaluates g and the
 * Jacobian values into the fixed pattern, refactorises, and solves; the
 * Jacobian at the returned x stays in the context and is factorised by the
 * first call that needs it (gradient, Hessian, step), so a power flow whose
 * factors are never used costs no refactorisation at the solution; a
 * singular Jacobian there is reported by that call (OPF_ESINGULAR).
 * opts NULL = {1e-10, 20}.  info (host) may be NULL.
 * Errors: OPF_ENOCONV, OPF_ESINGULAR (the context then has no valid state).
 */
opf_status opf_powerflow(opf_ctx* ctx, const double* u, const double* pd, const double* qd,
                         double* x_inout, const opf_pf_opts* opts, opf_pf_info* info);

/* Augmented-Lagrangian inputs: sigma_c, y, s [m] device arrays; omega [m]
 * optional second-order weights (NULL = rho sigma_c^2, i.e. the exact Hessian
 * of F; the Schur complement of Prop. 3 uses rho sigma^2 Sigma_s / (rho sigma^2
 * + Sigma_s)). */
typedef struct {
  double sigma_f;
  double rho;
  const double* sigma_c;
  const double* y;
  const double* s;
  const double* omega;
} opf_al_params;

/*
 * opf_reduced_gradient (Prop. 1 with the AL functional of eq.
 * gradient_auglag, scaled as in Sec. IV-A): at the state of the last
 * converged opf_powerflow, solve G_x^T lambda = -(d_x F)^T with the stored
 * factors (U^T then L^T) and form grad_u = d_u F + lambda^T G_u.  Outputs
 * (device, each may be NULL): F[1], grad_u[n_u], grad_s[m] = -phi' with
 * phi'_i = y_i sigma_i + rho sigma_i^2 (c_i - s_i), c[m], lambda[n_x],
 * grad_pd[n_bus], grad_qd[n_bus] (total derivatives of F w.r.t. the loads).
 * Errors: OPF_ESTATE without a converged power flow.
 */
opf_status opf_reduced_gradient(opf_ctx* ctx, const opf_al_params* p, double* F,
                                double* grad_u, double* grad_s, double* c, double* lambda,
                                double* grad_pd, double* grad_qd);

typedef struct {
  int block_k;   /* Hessian columns per CTA tile: 1, 2, 4, 8, 16 or 32
                    (0 = the context's autotuned choice, else 8) */
  int grid;      /* CTAs (0 = one per tile, capped at the resident CTAs per SM x SMs) */
  int plain;     /* 1: the k = 1 baseline: one direction per launch sequence, each column by
                    device-wide launches around two streamed single-RHS solves (block_k,
                    grid and threads are ignored; info->launches counts the kernels) */
  int col_begin; /* first Hessian column to compute (0) */
  int col_count; /* number of columns (0 = through n_u); the others of H are left untouched */
  int threads;   /* threads per tile CTA: 128, 256 or 512 (0 = 256) */
  int reuse_first_order; /* 1: the context's first-order quantities (c, phi', omega, lambda)
                            were just evaluated with these same parameters by
                            opf_reduced_gradient: skip re-evaluating them */
  int asymmetry; /* 1: report ||H - H^T||_F / ||H||_F of a full Hessian in info (one more
                    kernel after the timed region) */
  int phase_profile; /* 1: the tiles record the global timer at their phase boundaries and
                        info->phase_ms apportions the HVP time to the phases (diagnostics) */
} opf_hess_opts;

typedef struct {
  int block_k, grid, tiles, launches;
  float ms_total;  /* device time of the call (CUDA events on the context stream) */
  float ms_hvp;    /* device time of the HVP phase alone */
  double asymmetry; /* ||H - H^T||_F / ||H||_F when requested for a full Hessian (which is then
                       assembled column by column, not by symmetry), else -1 */
  float phase_ms[5]; /* with phase_profile: ms_hvp times each phase's share of the tiles'
                        summed durations -- (1) pruned L solve of Z, (2) U sweep of Z,
                        (3)-(4) second-order terms, (5)-(6) U^T and L^T sweeps of Psi,
                        (7) assembly of H; else 0 */
} opf_hess_info;

/*
 * opf_reduced_hessian: the dense reduced Hessian H[n_u * n_u] (column-major)
 * of F (or of the omega-weighted functional) at the state of the last
 * converged power flow, from n_u adjoint-adjoint HVPs (Prop. 2): for each
 * block of directions W, G_x Z = -G_u W (L then U sweeps), the second-order
 * terms of the injections, line flows and costs along every branch, then
 * G_x^T Psi = -(l_xu W + l_xx Z) (U^T then L^T sweeps) and
 * H[:, block] = l_uu W + l_ux Z + G_u^T Psi.  The factors of G_x are the ones
 * left by opf_powerflow (factorised once, Sec. III-C).  A full Hessian
 * (every column, tiled, no asymmetry report) is built by its symmetry unless
 * opf_set_hessian_symmetry turned that off: each tile keeps the rows of the
 * controls from its first column position on and one more kernel fills the
 * other entries from their transposes (info->launches counts it); otherwise H
 * is assembled column by column and not symmetrised.  opts/info may be NULL.
 * Errors: OPF_ESTATE, OPF_EINVAL.
 */
opf_status opf_reduced_hessian(opf_ctx* ctx, const opf_al_params* p, const opf_hess_opts* opts,
                               double* H, opf_hess_info* info);

/*
 * opf_reduced_jacobian: the reduced constraint Jacobian J = dc/du on the
 * manifold g = 0 (Sec. III-B, "Reduced sensitivities"), at the state of the
 * last converged power flow.  Column j is d_u c e_j + d_x c z_j with
 * z_j = -G_x^{-1} G_u e_j: the first adjoint of the HVP tiles (Prop. 2), so J
 * is a by-product of the Hessian's tiles.  The paper forms the reduced
 * Jacobians of h and r from m transposed solves; the tiles need the n_u
 * forward solves the Hessian already makes (n_u < m on every network here).
 *   J (device, required): m x n_u column-major, column j at J + j m; rows in
 *     the order of c (|S_f|^2 and |S_t|^2 per branch, v of each PQ bus, p_ref,
 *     q_ref, q of each PV unit).
 *   H (device, may be NULL): non-NULL computes the Hessian columns in the same
 *     launch, exactly as opf_reduced_hessian (p required).  NULL stops the
 *     tiles after the first adjoint (the L and U sweeps only); p may then be
 *     NULL (the branch tables are evaluated with zero multipliers; J does not
 *     depend on them).
 *   opts: as opf_reduced_hessian (block_k, grid, columns, threads,
 *     reuse_first_order, phase_profile); plain must be 0, and asymmetry is
 *     ignored without H.  Only the requested columns of J are written.
 * The call replaces the context's first-order quantities unless
 * reuse_first_order.  Errors: OPF_EINVAL, OPF_ESTATE, OPF_ESINGULAR.
 */
opf_status opf_reduced_jacobian(opf_ctx* ctx, const opf_al_params* p, const opf_hess_opts* opts, double* J,
                                double* H, opf_hess_info* info);

/*
 * opf_gradient_scaling: the scaling of the AL problem by the size of its
 * gradients (Sec. IV-A, "Scaling", where the paper cites the gradient-based
 * rule of interior-point codes without stating it), at the state of the last
 * converged power flow:
 *   scale(n)   = 1 if n <= g_max, else max(s_min, g_max / n)
 *   sigma_c[i] = p_i scale(p_i ||dc_i/du||_inf)  (p = prior, or 1: the rule on
 *                the constraint as the caller writes it, p_i c_i)
 *   sigma_f    = scale(||df/du||_inf), f the generation cost
 * Both derivatives are reduced ones (on g = 0): J from opf_reduced_jacobian,
 * the cost gradient from Prop. 1.  The usual values are g_max = 100 and
 * s_min = 1e-8.
 *   prior (device [m], may be NULL): the caller's own constraint scales.
 *   J (device, m x n_u column-major, 8 m n_u bytes): receives the Jacobian
 *     (the caller's workspace).
 *   sigma_c (device [m]): the constraint scales.  sigma_f (host, may be NULL).
 * The call replaces the context's first-order quantities (evaluated with zero
 * multipliers).  Errors: OPF_EINVAL (g_max <= 0 or not finite, s_min outside
 * (0, 1]), OPF_ESTATE, OPF_ESINGULAR.
 */
opf_status opf_gradient_scaling(opf_ctx* ctx, double g_max, double s_min, const double* prior, double* J,
                                double* sigma_c, double* sigma_f);

/*
 * opf_hessian_autotune: time opf_reduced_hessian on the context's current state
 * for each (block_k, threads) in {(4,128), (4,256), (8,128), (8,256), (8,512),
 * (16,256), (16,512), (32,256)} (one untimed and one timed call each, CUDA events on the
 * context stream), keep the fastest as the context's choice for block_k = 0,
 * and return it in best (host) with its time in best_ms (host, may be NULL).
 * H (device, n_u x n_u) is scratch for the trial calls.  Errors as
 * opf_reduced_hessian.
 */
opf_status opf_hessian_autotune(opf_ctx* ctx, const opf_al_params* p, double* H, opf_hess_opts* best,
                                float* best_ms);

/*
 * opf_set_sweep_merge: the level-merge schedule of the single-right-hand-side
 * solves (the Newton updates of the power flow, Sec. III-A, and the adjoint
 * solves of Prop. 1 and Prop. 3).  Their level loop is a chain of dependent
 * steps; a narrow level (a few blocks of 100-250 entries on the large grids)
 * costs a long dependent sum.  With lookahead = D > 0 each block of a level
 * chunk with at most `narrow` blocks keeps only the entries whose column the
 * chunk just before it writes; each other entry is summed in one of the D
 * chunks before it that already has its column (spread evenly over them),
 * beside those chunks' own work, and subtracted from the block's right-hand
 * side there.  D = 0: no merging.  The streams are rebuilt in place on the
 * host (tens of ms on the 9,200-bus grid; the context's stream is
 * synchronised first); results change only through the order of the sums.
 * A context whose solves use the level-record form (solution too large for
 * shared memory) ignores the call.  The schedule at load is (4, 4), the
 * fastest of the autotuner's candidates on the 9,200-bus grid.
 * Errors: OPF_EINVAL (D < 0, narrow < 1 with D > 0, a merged chunk too large
 * for the buffers), OPF_ECUDA.
 */
opf_status opf_set_sweep_merge(opf_ctx* ctx, int lookahead, int narrow);

/*
 * opf_sweep_autotune: for each level-merge schedule (lookahead, narrow) in
 * {(0, 0), (1, 4), (2, 4), (4, 4), (6, 4), (8, 4), (4, 2), (4, 8)}, time one
 * forward and one transposed single-right-hand-side solve at the current
 * factors (CUDA events on the context stream, best of three after a warm-up),
 * keep the fastest schedule (opf_set_sweep_merge) and return it (host
 * pointers, each may be NULL) with its time per forward + transposed pair;
 * ms_all (host [8], may be NULL) receives every candidate's time in the order
 * above.  Requires a converged power flow.  Errors: OPF_ESTATE,
 * OPF_ESINGULAR, OPF_ECUDA.
 */
opf_status opf_sweep_autotune(opf_ctx* ctx, int* lookahead, int* narrow, float* ms_pair, float* ms_all);

/*
 * opf_reduced_hessian_batched: the dense reduced Hessians of n contexts
 * (snapshots: the same or different networks, each at its own converged power
 * flow) in one persistent launch.  Per context the first-order quantities and
 * branch tables are evaluated as in opf_reduced_hessian; then one kernel walks
 * a queue of (context, column tile) pairs, tiles of the largest networks first
 * (longest processing time first), each CTA pulling the next pair when it
 * finishes one (the batched multi-right-hand-side HVPs of Sec. V-A across
 * snapshots).  params[k] and H[k] (n_u(k) x n_u(k) column-major) belong to
 * ctxs[k].  Everything runs on ctxs[0]'s stream; all contexts must live on
 * the same device.  opts: block_k and grid (0 = as many CTAs as fit), and
 * reuse_first_order (every context's first-order quantities were just
 * evaluated with its params); plain, columns and threads are ignored.  The workspace is held by ctxs[0] (grown on
 * demand).  Errors: OPF_EINVAL, OPF_ESTATE (a context without a converged
 * power flow).
 */
opf_status opf_reduced_hessian_batched(opf_ctx* const* ctxs, int n, const opf_al_params* params,
                                       double* const* H, const opf_hess_opts* opts,
                                       opf_hess_info* info);

/*
 * opf_reduced_hessian_noalloc: the same reduced Hessian as opf_reduced_hessian
 * (same tile kernel; every column computed in full, so the output equals
 * opf_reduced_hessian's symmetric form to rounding), for callers that must not allocate device
 * memory during the call: a real-time tracking loop that cannot stall on the
 * allocator (cudaMalloc may synchronise the device and its latency is
 * unbounded), or a process whose device-memory budget is fixed at start-up.
 * The paper has no counterpart: this is an interface choice of this library.
 *   - Options: block_k (0 = 8; the autotuned choice is not used), grid and the
 *     column range; plain, threads and reuse_first_order must be 0
 *     (OPF_EINVAL otherwise).  The first-order quantities are always evaluated.
 *   - Workspace: a fixed array of OPF_NOALLOC_SCRATCH_BYTES (32 MiB) in device
 *     memory, which every GPU that loads the library holds until the process
 *     exits.  No call allocates or frees anything.
 *   - Limit: one tile needs (2 n_x + n_ctrl + 1) block_k doubles, n_ctrl =
 *     n_pv + 1, rounded up to 32; a network/block_k whose tile does not fit is
 *     rejected with OPF_EINVAL and a message (checked before the state).  The
 *     grid is capped at the tiles that fit at once (32 MiB / tile bytes), and
 *     its CTAs loop over the remaining tiles, so it can be slower than
 *     opf_reduced_hessian.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any
 *     stream capture.
 *   - All calls share the one array and it keeps the last call's contents; the
 *     kernel clears what it needs per tile.  Calls that overlap on the GPU (two
 *     streams, two contexts, two threads) race on it: serialise them.
 * Errors: OPF_EINVAL (arguments, size limit), OPF_ESTATE, OPF_ESINGULAR, OPF_ECUDA.
 */
#define OPF_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
opf_status opf_reduced_hessian_noalloc(opf_ctx* ctx, const opf_al_params* p,
                                       const opf_hess_opts* opts, double* H, opf_hess_info* info);

/*
 * Reduced-Newton step of the augmented-Lagrangian subproblem (Sec. IV-B,
 * eq. ipm_kkt_reduced with the AL Hessian of eq. hessian_auglag, solved by the
 * Schur complement of Prop. 3), one primal-dual barrier step on w = (u, s):
 *   Sigma = Z_lo/(w - w_lo) + Z_hi/(w_hi - w);  grad psi = grad L_rho - mu/(w - w_lo) + mu/(w_hi - w)
 *   S_uu = H(omega) + Sigma_u [+ delta I],  omega_i = rho sigma_i^2 Sigma_s,i / (rho sigma_i^2 + Sigma_s,i)
 *          (H(omega) = opf_reduced_hessian with these weights, symmetrised)
 *   S_uu d_u = -grad_u psi - J^T [rho D^2 (rho D^2 + Sigma_s)^{-1} grad_s psi]   (J = dc/du on g = 0;
 *          the sign follows from eliminating d_s; the printed Prop. 3 has "+")
 *   d_s = (rho D^2 + Sigma_s)^{-1} (-grad_s psi + rho D^2 J d_u),  D = diag(sigma_c)
 *   dz_lo = mu/(w - w_lo) - z_lo - Sigma_lo d_w,  dz_hi = mu/(w_hi - w) - z_hi + Sigma_hi d_w
 * S_uu is factorised by a device FP64 Cholesky; delta (inertia correction) takes
 * 0, then 1e-8 * 10^k, k = 0 .. max_inertia - 1, until the factorisation succeeds
 * (with opts->delta_start > 0: delta_start, then 10x per try, as a loop that
 * carries the previous step's delta over).  Success is monotone in delta (S_uu
 * + delta I positive definite implies it for larger delta): from a carried-over
 * delta the candidates are tried in turn; from a fresh start, after delta = 0
 * fails, the rest are bisected -- the same delta as trying each in turn, with
 * fewer factorisations (6 instead of 18 for delta = 1e8).
 * Step lengths: fraction to the boundary with tau = max(0.99, 1 - mu) for the
 * primal and the dual variables; the power flow is re-solved at u + alpha_p d_u
 * (warm start from x) and alpha_p halved until it converges, so the new iterate
 * stays feasible.  Then u, s, x, and the duals are updated in place.
 * Requires a converged opf_powerflow at st->u.  The first call allocates the
 * step workspace of the context (two n_u x n_u matrices and vectors).
 * Errors: OPF_ESTATE, OPF_EINVAL, OPF_ENOTPD (no delta made S_uu positive
 * definite), OPF_ENOCONV (no trial point converged; the state is unchanged).
 */
typedef struct {
  double *u, *s;            /* [n_u], [m] primal, updated in place */
  double *zl_u, *zu_u;      /* [n_u] bound duals of u, updated in place (> 0) */
  double *zl_s, *zu_s;      /* [m] bound duals of s, updated in place (> 0) */
  const double *u_lo, *u_hi, *s_lo, *s_hi;  /* bounds, strictly around u and s */
  double* x;                /* [n_x] power-flow state at u; replaced by the state at the new u */
  double mu;                /* barrier parameter */
} opf_al_state;

typedef struct {
  int block_k;        /* Hessian tile width (0 = the context's autotuned choice, else 8) */
  int max_halvings;   /* trial power flows allowed after the first (0 = 10) */
  int max_inertia;    /* inertia-correction tries after the first (0 = 24) */
  double delta_start; /* first delta tried (0 = start at 0) */
  int line_search;    /* 1: also halve the step until the barrier function psi_mu = F - mu sum
                         log(w - w_lo) - mu sum log(w_hi - w) satisfies the Armijo rule
                         psi(w + a d) <= psi(w) + 1e-4 a grad psi^T d (the inertia-corrected
                         system makes d a descent direction); after max_halvings the last trial
                         with a converged power flow is taken.  0: accept the first one. */
} opf_step_opts;

typedef struct {
  double alpha_p, alpha_d, delta, du_inf, ds_inf;
  int halvings, inertia_tries, pf_iterations;
  float ms_hessian, ms_total;
  /* device time of the phases (ms): first-order quantities and Sigma; Schur
   * right-hand side; Cholesky with its inertia corrections; the two triangular
   * solves, J d_u and the fraction to the boundary; trial power flows and update */
  float ms_first_order, ms_rhs, ms_cholesky, ms_solve, ms_trial;
  int cholesky_fp64;  /* factorisations run with FP64 trailing updates (opf_set_cholesky_mode) */
  int factorisations; /* factorisations of the inertia search (inertia_tries is the index of the
                         chosen delta in the sequence, as trying each in turn would count it) */
} opf_step_info;

/* p supplies sigma_f, rho, sigma_c and y (its s and omega are ignored: s comes
 * from st).  du_out [n_u] and ds_out [m] (device, optional) receive the step. */
opf_status opf_al_step(opf_ctx* ctx, const opf_al_params* p, opf_al_state* st,
                       const opf_step_opts* opts, opf_step_info* info, double* du_out,
                       double* ds_out);

/*
 * opf_al_solve: the static OPF by the augmented-Lagrangian method (Sec. IV-B
 * "Static OPF algorithm", the scaled AL of Sec. IV-A).  Outer iteration k
 * solves the AL subproblem for fixed rho and y by barrier steps (opf_al_step),
 * warm-started from the previous primal-dual point, then updates y.  The paper
 * leaves the IPM's internals and the AL schedule unstated; the readings:
 *   E_mu = max(|grad_u L - zl_u + zu_u|_inf, |grad_s L - zl_s + zu_s|_inf,
 *              |(w - w_lo) zl - mu|_inf, |(w_hi - w) zu - mu|_inf)   (w = (u, s)),
 *   E_0 = the same at mu = 0 (the subproblem's own KKT error);
 *   inner loop: evaluate the gradient at the current point; stop when
 *     E_0 <= omega_k = max(eta_dual, 10^-(k+1)) or after max_inner steps; when
 *     E_mu <= 10 mu, mu <- max(eta_dual / 10, min(0.2 mu, mu^1.5)); then one
 *     opf_al_step with the Armijo line search on psi_mu (the subproblems are
 *     nonconvex away from a solution and full steps can diverge), its inertia
 *     correction starting at delta/10 of the previous step's delta when that was
 *     at least 1e-7, else at 0;
 *   outer update: eta_p = |sigma_c (c - s)|_inf; stop when eta_p <= eta_primal
 *     and E_0 <= eta_dual; else y <- y + rho sigma_c (c - s), and rho <-
 *     min(10 rho, rho_max) when eta_p fell by less than a factor 4.
 * p: sigma_f, rho (the initial penalty), sigma_c (its y, s and omega are
 * ignored); y [m] (device) the multipliers, updated in place; st the primal-
 * dual state and bounds as for opf_al_step (u, s, duals, x and mu updated in
 * place).  Requires a converged opf_powerflow at st->u.  history (host, may be
 * NULL): 8 doubles per outer iteration {steps, mu, rho, eta_p, E_0, F, delta,
 * 0}.  With opts->scaling_gmax > 0 the loop first scales the problem by its
 * gradients at the starting point (Sec. IV-A "Scaling", opf_gradient_scaling
 * with p->sigma_c as the prior and g_max = scaling_gmax): the constraint
 * scales become p->sigma_c times the rule's factors and sigma_f the rule's
 * scale of the cost (p->sigma_f is then unused); y, eta_p and E_0 refer to
 * the scaled problem.  The Jacobian this needs (8 m n_u bytes) is allocated
 * for the scaling and freed before the iterations.  Errors: those of
 * opf_al_step (the state is then the last accepted iterate), OPF_EINVAL,
 * OPF_ESTATE, OPF_ENOMEM.
 */
typedef struct {
  int max_outer;      /* outer iterations (0 = 20) */
  int max_inner;      /* reduced-Newton steps per subproblem (0 = 30) */
  double eta_primal;  /* stopping tolerance on |sigma_c (c - s)|_inf (0 = 1e-5) */
  double eta_dual;    /* stopping tolerance on E_0 (0 = 1e-4) */
  double rho_max;     /* penalty cap (0 = 1e6) */
  int block_k;        /* Hessian tile width of the steps (0 = autotuned, else 8) */
  double scaling_gmax;   /* > 0: gradient-based scaling at the start (above); 0: p's scales */
  double* sigma_c_used;  /* device [m], may be NULL: receives the constraint scales the loop used */
} opf_al_opts;

typedef struct {
  int outer, steps, converged;
  double primal_inf, dual_inf, F, rho, mu;
  float ms_total;  /* device time of the whole loop (the scaling included) */
  double sigma_f;  /* the objective scale the loop used */
} opf_al_info;

opf_status opf_al_solve(opf_ctx* ctx, const opf_al_params* p, double* y, opf_al_state* st,
                        const opf_al_opts* opts, opf_al_info* info, double* history);

/*
 * opf_tracking_update: one real-time OPF update (Sec. IV-C "Real-time optimal
 * power flow"), after opf_powerflow at the new loads and the current controls:
 *   1. g_t = grad L_rho,t(w_t; y) and the constant Hessian H_t of eq.
 *      hessian_auglag (scaled, Sec. IV-A) at w_t = (u_t, s_t);
 *   2. the bounded QP of eq. qp_rto, min g_t^T d + 1/2 d^T (H_t + delta I_u) d
 *      over w_lo <= w_t + d <= w_hi, solved by a primal-dual interior-point
 *      method whose Newton systems go through the Schur complement of Prop. 3
 *      (S = H(omega) + Sigma_u + delta I, H(omega) from opf_reduced_hessian at the
 *      fixed point w_t with the iteration's omega; dense Cholesky);
 *   3. w_{t+1} = the QP solution (the step from w_t halved until the power flow
 *      at u_{t+1} converges), then y <- y + rho D_c (c_t(u_{t+1}) - s_{t+1}).
 * Readings (the paper names the IPM, not its rules): KKT error of the QP as for
 * opf_al_solve with grad q(d) = g_t + (H_t + delta I_u) d in place of grad L;
 * stop when E_0 <= tol or after max_it iterations; mu <- max(tol / 10,
 * min(0.2 mu, mu^1.5)) when E_mu <= 10 mu; fraction to the boundary tau =
 * max(0.99, 1 - mu); delta starts at the smallest of 0 (or opts->delta_start),
 * 1e-8, 1e-7, ... that makes H_uu + delta I positive definite (H_uu = H(0), one
 * more Hessian and Cholesky before the iterations), so that the QP is convex,
 * and grows further only if an iteration's S is not positive definite (each
 * search as in opf_al_step: in turn from a delta > 0, bisecting after a failed
 * delta = 0, which success being monotone in delta makes equal to trying each
 * in turn); with
 * opts->inertia_only the convexity search is skipped (H_uu is indefinite even
 * at an OPF optimum, along the directions that move active constraints, while
 * S, which holds the barrier terms of those bounds, is not).  grad q is carried from iteration to iteration through the Newton
 * system: H d = -grad psi - Sigma d.
 * p: sigma_f, rho, sigma_c (y, s, omega ignored); y [m] updated in place; st:
 * u, s (w_t in, w_{t+1} out), bound duals (the QP's, warm start in, final out),
 * bounds, x (the state at u_t in, at u_{t+1} out), mu (the QP's first barrier
 * in, its last out).  Errors: OPF_ESTATE, OPF_EINVAL, OPF_ENOTPD, OPF_ENOCONV,
 * OPF_ETIMEOUT.
 */
typedef struct {
  int max_it;         /* QP iterations (0 = 50) */
  double tol;         /* stop when the QP's KKT error E_0 <= tol (0 = 1e-6) */
  int block_k;        /* Hessian tile width (0 = autotuned, else 8) */
  int max_halvings;   /* (0 = 10) */
  int max_inertia;    /* inertia-correction increases per factorisation (0 = 24) */
  double delta_start; /* the QP's first delta (0 = start at 0) */
  int inertia_only;   /* 1: no convexity search before the iterations: delta starts at delta_start
                         (or 0) and grows only where an iteration's S is not positive definite (the
                         usual inertia correction of an interior-point method; the barrier terms
                         Sigma of the active bounds supply the curvature H_uu lacks at an optimum) */
} opf_qp_opts;

typedef struct {
  int qp_iterations, halvings, pf_iterations, inertia_increases;
  double delta, delta_convex, kkt, mu, alpha_p;  /* delta at the end, at the start (convexity) */
  double kkt_first, alpha_p_min;  /* the QP's KKT error at d = 0; its smallest primal step length */
  float ms_total;     /* the whole update */
  float ms_qp;        /* gradient at w_t and the QP iterations */
  float ms_hessian;   /* summed device time of the QP's Hessians H(omega) */
  float ms_cholesky;  /* summed device time of its factorisations */
  int cholesky_fp64;  /* factorisations run with FP64 trailing updates (opf_set_cholesky_mode) */
} opf_qp_info;

opf_status opf_tracking_update(opf_ctx* ctx, const opf_al_params* p, double* y, opf_al_state* st,
                               const opf_qp_opts* opts, opf_qp_info* info);

/*
 * opf_set_cholesky_mode: how the dense Cholesky of the reduced-Newton step and
 * of the tracking QP (the Schur complement of Prop. 3) applies its trailing
 * updates.  The updates of each 128-column group are emulated in FP64 on the
 * tensor cores (exact digit products, FP64 sums), whose error per element is
 * below ~5 K u max_k|P_rk| max_k|P_ck| -- relative to the rows' largest panel
 * entries -- where an FP64 update errs by ~K u sum_k |P_rk P_ck|; on a Schur
 * complement whose rows span many decades (penalty weights rho sigma^2 of
 * 1e9 beside O(1) curvature) the emulation could make a pivot of a positive
 * definite matrix non-positive, and the inertia correction would then raise
 * delta for nothing.
 *   mode 1 (default): emulated only;
 *   mode 0: emulated; a failed pivot is re-checked with FP64 updates at the
 *     same delta before delta grows (the step and QP infos count them);
 *   mode 2: FP64 only (slower: four rank-32 updates of the trailing triangle
 *     per group).
 * On the workloads here modes 1 and 2 took the same inertia corrections, so
 * the default keeps the emulation; mode 0 costs an FP64 factorisation for
 * every genuine failure.  Errors: OPF_EINVAL.
 */
opf_status opf_set_cholesky_mode(opf_ctx* ctx, int mode);

/*
 * opf_set_update_engine: which tensor-core kernel runs the emulated trailing
 * updates of the dense Cholesky (modes 0 and 1 of opf_set_cholesky_mode):
 *   engine 0 (default): tcgen05.mma with the eight level sums of a 128 x 64
 *     tile held in tensor memory, one persistent CTA per SM, for the updates
 *     of at least 80 such tiles (trailing blocks above ~1,000 rows); the
 *     smaller updates, whose few 128-row tiles cannot hide their latency,
 *     run on warp-level mma.sync;
 *   engine 1: warp-level mma.sync on 64 x 64 tiles for every update;
 *   engine 2: tcgen05 for every update.
 * The tcgen05 kernel's waits for the tensor cores and its bulk copies are
 * bounded (opf_set_wait_limit); a wait that gives up makes the step or QP call
 * return OPF_ETIMEOUT.  All engines give bit-identical factors.  Errors:
 * OPF_EINVAL.
 */
opf_status opf_set_update_engine(opf_ctx* ctx, int engine);

/*
 * opf_set_wait_limit: iteration limit of every bounded device-side wait of
 * this context (the flag polls of the dense block's cluster LU and of the
 * dense triangular solves of opf_al_step, the mbarrier polls of the tcgen05
 * emulated Cholesky update); 0 restores each kernel's default (2^22, 2^24
 * and 2^24 polls).  A wait that reaches the limit stops waiting, records
 * the timeout and lets its kernel finish; the call then returns OPF_ETIMEOUT
 * (a refactorisation also drops the context's state, as OPF_ESINGULAR does)
 * and the context stays usable.  Errors: OPF_EINVAL (spins < 0), OPF_ECUDA.
 */
opf_status opf_set_wait_limit(opf_ctx* ctx, int spins);

/*
 * opf_set_hessian_symmetry: whether a full reduced Hessian (opf_reduced_hessian
 * over all columns, tiled, without the asymmetry report; also inside
 * opf_al_step and opf_tracking_update) is built by its symmetry (on = 1, the
 * default) or column by column in full (on = 0).  With symmetry, the tile of
 * columns [p, p + k) in the tiling's column order (the elimination-tree order
 * of the controls) keeps only the rows of the controls at positions >= p: its
 * second adjoint Psi is needed on the elimination-tree ancestors of those
 * controls' right-hand-side rows only, so its L^T sweep skips the other rows
 * (on the 9.2k-bus grid 43% of that sweep's entries), and a mirror kernel
 * fills the remaining entries from their transposes.  The result equals the
 * full computation up to rounding (each entry is one of the two computed
 * values of the symmetric pair).  Errors: OPF_EINVAL.
 */
opf_status opf_set_hessian_symmetry(opf_ctx* ctx, int on);

/*
 * Measurement and verification entry points (no context; ordered on `stream`,
 * a cudaStream_t, NULL = legacy default stream; each call synchronises it).
 *
 * opf_fp64_peak: the device's FP64 FMA rate, the denominator of the FP64
 * roofline of the solves and second-order terms (Sec. V-A runs them in FP64):
 * every resident thread runs eight independent chains of dependent FMAs; the
 * fastest of five timed launches (CUDA events) after one warm-up.  tflops
 * (host) receives 2 x FMAs / time in TFLOP/s, ms_out (host, may be NULL) that
 * launch's time.  Errors: OPF_EINVAL, OPF_ENOMEM, OPF_ECUDA.
 *
 * opf_pivot_reciprocal: r[i] = 1 / u[i] (device arrays of n doubles) computed
 * as the LU refactorisation computes its pivots' reciprocals (hardware
 * approximate reciprocal, flushing subnormal inputs to zero, then two
 * Newton-Raphson steps), so that the tests can compare it with IEEE division:
 * equal except for u just below a power of two (every mantissa bit set: one
 * unit in the last place off); NaN
 * for zero and subnormal u.
 *
 * opf_dense_syrk_emulated: the trailing update of one column group of the
 * Schur-complement Cholesky (Prop. 3; dense FP64 Cholesky on the device):
 * A[r0:n, r0:n] (lower triangle) -= P P^T with P = A[r0:n, c0:c0+K], A column-
 * major n x n on the device, K in {32, 64, 96, 128}, c0 + K <= r0 < n,
 * emulated in FP64 on the bf16 tensor cores (rows of P in eight signed 7-bit
 * digits against a per-row power of two; digit products accumulated exactly;
 * levels i + j >= 8 and the digit tails dropped).  Element (r, c) of the
 * update then errs by less than 5 K 2^-53 max_k |P_rk| max_k |P_ck| before the
 * final FP64 roundings.  engine as in opf_set_update_engine (0: tcgen05 MMAs
 * with the level sums in tensor memory for updates of at least 80 tiles of
 * 128 x 64, mma.sync below; 1: warp-level mma.sync; 2: tcgen05).  The engines
 * sum the same exact integers and round the same way, so their results are
 * bit-identical.  Allocates and frees its workspace.  Errors: OPF_EINVAL,
 * OPF_ENOMEM, OPF_ECUDA, OPF_ETIMEOUT (a bounded wait of the tcgen05 kernel
 * gave up; the result is void).
 */
opf_status opf_fp64_peak(void* stream, double* tflops, float* ms_out);
opf_status opf_pivot_reciprocal(void* stream, const double* u, double* r, int n);
opf_status opf_dense_syrk_emulated(void* stream, double* A, int n, int c0, int K, int r0, int engine);

/*
 * opf_al_step_batched: one tracking update for each of n snapshots (contexts of
 * the same or different networks on one device): optionally the power flow at
 * the snapshot's new loads pd[k], qd[k] (device, NULL entries or NULL arrays =
 * keep the context's state), then the reduced-Newton step of opf_al_step with
 * params[k] and states[k] -- with every snapshot's Schur Hessian H(omega_k) in
 * one persistent launch over a shared tile queue (opf_reduced_hessian_batched,
 * largest networks first; Sec. V-A batches the multi-right-hand-side solves).
 * The per-snapshot parts (power flows, first-order quantities, Cholesky,
 * solves, trial power flows) run on each context's own stream, driven by host
 * threads that take the snapshots largest first, so the GPU overlaps them.
 * infos[k] (host, may be NULL) and status[k] (host, may be NULL) report each
 * snapshot; binfo (host, may be NULL) the phase times.  A snapshot that fails
 * keeps its state and does not stop the others; the call returns the first
 * failure's status (OPF_OK when all succeed).  Errors of the batch itself:
 * OPF_EINVAL (null or repeated context, mixed devices), those of
 * opf_reduced_hessian_batched.
 */
typedef struct {
  float ms_powerflow_first_order;  /* host wall time of the power flows and pre-Hessian parts */
  float ms_hessians;               /* the batched Hessian launch (with its set-up) */
  float ms_steps;                  /* Cholesky, solves, trial power flows, updates */
  float ms_total;
  int hessian_tiles, host_threads, failed;
} opf_batch_info;

opf_status opf_al_step_batched(opf_ctx* const* ctxs, int n, const opf_al_params* params,
                               opf_al_state* states, const double* const* pd, const double* const* qd,
                               const opf_step_opts* opts, opf_step_info* infos, opf_status* status,
                               opf_batch_info* binfo);

/*
 * opf_objective_batched: for n load scenarios of one network, the power flow
 * (from the common warm start x0 [n_x]) at u[k], pd[k], qd[k] and the reduced
 * objective F[k] of the scaled AL with slacks s[k] -- and, for every non-NULL
 * gradient array, its adjoint gradient (Prop. 1): grad_u [n][n_u], grad_pd and
 * grad_qd [n][n_bus] (total derivatives through g and the slack generation),
 * grad_s [n][m] = -phi'.  Row-major device arrays, scenario k at offset k times
 * the row length; pd/qd NULL = nominal loads; x_out [n][n_x] (may be NULL)
 * receives the states; with x0 == x_out each scenario starts from its own row
 * of x_out instead (for example the states of a previous call at the same
 * inputs, which converge at once: one factorisation, no Newton iteration, as
 * an autograd backward pass needs).  p: sigma_f, rho, sigma_c, y shared by the scenarios
 * (its s and omega are ignored).  The scenarios are spread over a pool of nctx
 * contexts of that network, each on its own stream and host thread (give each
 * its own stream with opf_set_stream for the GPU to overlap them); the outputs
 * are complete when the call returns.  status[k] (host, may be NULL) reports
 * each scenario; the call returns the first failure.  Errors: OPF_EINVAL
 * (contexts of different networks or devices, a repeated context), those of
 * opf_powerflow and opf_reduced_gradient.
 */
opf_status opf_objective_batched(opf_ctx* const* ctxs, int nctx, int n, const opf_al_params* p,
                                 const double* u, const double* pd, const double* qd, const double* s,
                                 const double* x0, double* x_out, double* F, double* grad_u,
                                 double* grad_pd, double* grad_qd, double* grad_s, opf_status* status);

/* Number of kernels this context has launched since it was created (host output). */
opf_status opf_launch_count(const opf_ctx* ctx, long long* launches);

/* Human-readable status and the last error message of this thread. */
const char* opf_status_str(int status);
const char* opf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OPF_H */
