/*
 * CPU oracle for the feasible reduced-space OPF hot path (Pacaud et al., arXiv 2110.02590).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64 C code that computes the
 * quantities of the method from their definitions.  Only the test suite, the
 * smoke check and the CPU baseline leg of the benchmark may load it; the
 * library never does.  It shares no code with the CUDA path.
 *
 * Conventions (all per unit):
 *   buses 0..nb-1, ref bus = `ref`, one generator per bus at most; PV buses are
 *   generator buses other than ref, PQ buses the rest, both in ascending id.
 *   u = (v_ref, v_pv, p_pv)            n_u = 1 + 2 n_pv          (eq. statecontrol, Sec. II-B)
 *   x = (theta_pv, theta_pq, v_pq)     n_x = n_pv + 2 n_pq
 *   g = (P_pv - p_pv + pd_pv, P_pq + pd_pq, Q_pq + qd_pq)       (power balance, Sec. II-A)
 *   c = (|S_f|^2 per branch, |S_t|^2 per branch, v_pq, p_ref, q_ref, q_pv)
 *       m = 2 n_l + n_pq + n_pv + 2                              (Sec. II-B, Sec. IV-A)
 *   F = sigma_f f + sum_i [ y_i sigma_i (c_i - s_i) + rho/2 sigma_i^2 (c_i - s_i)^2 ]
 *       (scaled augmented Lagrangian, Sec. IV-A "Scaling")
 *   second-order weights omega_i default to rho sigma_i^2; a caller may pass others.
 *
 * Every function returns 0 on success and a negative code on failure.
 */
#ifndef OPF_ORACLE_H
#define OPF_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_net orc_net;

orc_net* orc_net_new(int nb, int nl, int ng, int ref,
                     const double* pd, const double* qd, const double* vmin, const double* vmax,
                     const int* f, const int* t, const double* r, const double* x,
                     const double* b, const double* tap, const double* rate,
                     const int* gbus, const double* c2, const double* c1, const double* c0,
                     const double* pmin, const double* pmax, const double* qmin, const double* qmax);
void orc_net_free(orc_net* net);
int orc_dims(const orc_net* net, int* nx, int* nu, int* m, int* npv, int* npq);

/* Symbolic analysis: exact minimum degree on the bus graph, fill pattern, level sets. */
int orc_symbolic_sizes(orc_net* net, int* nnz_full, int* n_state_bus);
int orc_symbolic_export(orc_net* net, int* bus_order, int* perm, int* rowptr, int* colidx,
                        int* lev_f, int* lev_b);

/* Newton-Raphson power flow (eq. projection:newtonraphson); x_inout is the start point. */
int orc_powerflow(orc_net* net, const double* u, const double* pd, const double* qd,
                  double* x_inout, double tol, int max_it, int* iters, double* res2, double* resinf);

/* g(x,u) and c(x,u); P,Q are the bus injections (nb each). */
int orc_eval(orc_net* net, const double* x, const double* u, const double* pd, const double* qd,
             double* g, double* c, double* P, double* Q, double* f_cost);

/* Reduced gradient by the adjoint method (Prop. 1) of the scaled AL functional. */
int orc_reduced_gradient(orc_net* net, const double* x, const double* u, const double* pd,
                         const double* qd, double sigma_f, double rho, const double* sigma_c,
                         const double* y, const double* s, double* F, double* grad_u,
                         double* grad_s, double* c, double* lambda, double* grad_pd,
                         double* grad_qd);

/* Columns `cols` of the reduced Hessian by adjoint-adjoint HVPs (Prop. 2).
 * H is n_u x ncols, column-major.  omega may be NULL (then rho sigma^2). */
int orc_reduced_hessian(orc_net* net, const double* x, const double* u, const double* pd,
                        const double* qd, double sigma_f, double rho, const double* sigma_c,
                        const double* y, const double* s, const double* omega, const int* cols,
                        int ncols, double* H);

/* Hessian-vector product for one direction w (Prop. 2). */
int orc_hvp(orc_net* net, const double* x, const double* u, const double* pd, const double* qd,
            double sigma_f, double rho, const double* sigma_c, const double* y, const double* s,
            const double* omega, const double* w, double* Hw);

/* Reduced Jacobian products: Jv = (d c / d u) v and Jtw = (d c / d u)^T w. */
int orc_reduced_jac_prod(orc_net* net, const double* x, const double* u, const double* pd,
                         const double* qd, const double* v, double* Jv, const double* w,
                         double* Jtw);

/* Dense brute force on small nets (hyper-dual numbers on the complex-voltage form):
 * H (n_u x n_u), J (m x n_u), grad_u, all column-major. */
int orc_bruteforce(orc_net* net, const double* x, const double* u, const double* pd,
                   const double* qd, double sigma_f, double rho, const double* sigma_c,
                   const double* y, const double* s, const double* omega, double* H, double* J,
                   double* grad_u);

#ifdef __cplusplus
}
#endif
#endif
