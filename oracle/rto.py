"""Real-time OPF tracking update (TEST INFRASTRUCTURE ONLY).

Sec. IV-C "Real-time optimal power flow": at new loads, with the power flow
re-solved at the current controls,
  1. g_t = grad_w L_rho,t(w_t; y_t) and the Hessian H_t of eq. hessian_auglag
     (scaled as in Sec. IV-A): [[H_uu + J^T R J, -J^T R], [-R J, R]],
     R = rho D_c^2, H_uu the reduced Hessian with zero Gauss-Newton weights,
     J = dc/du on the manifold (explicit, one product per control);
  2. the bounded QP of eq. qp_rto, min g^T d + 1/2 d^T (H_t + delta I_u) d over
     w_lo <= w_t + d <= w_hi, by a primal-dual interior-point method whose
     Newton system is reduced by Prop. 3 with the Schur complement written as
     eq. schur_matrix: S = H_uu + Sigma_u + J^T (R - R (R + Sigma_s)^-1 R) J
     (+ delta I), formed explicitly from H_uu and J;
  3. w_{t+1} = the QP solution (the step halved until the power flow at u_{t+1}
     converges); y_{t+1} = y_t + rho D_c (c_t(u_{t+1}) - s_{t+1}).
grad q(d) = g + (H_t + delta I_u) d is evaluated from its definition every
iteration.  The IPM's rules are the readings the library's
opf_tracking_update takes (stated there and in al_loop.kkt_errors): KKT error,
barrier update mu <- max(tol/10, min(0.2 mu, mu^1.5)) when E_mu <= 10 mu,
fraction to the boundary tau = max(0.99, 1 - mu), and a regularisation delta
that only grows within one QP, starting at the smallest of {delta_start or 0,
1e-8, 1e-7, ...} that makes H_uu + delta I positive definite, so that the QP is
convex (away from an optimum the reduced Hessian of the AL is indefinite and
the bounded QP unbounded along negative curvature).  Option inertia_only: no
convexity search; delta starts at delta_start and grows only where an
iteration's Schur complement S is not positive definite, as in an
interior-point method's inertia correction (H_uu lacks curvature along the
directions that move active constraints even at an optimum; S holds the
barrier terms of those bounds).
"""
import numpy as np

from oracle.al_loop import kkt_errors


def _max_step(w, d, lo, hi, tau):
    a = 1.0
    neg, pos = d < 0, d > 0
    if neg.any():
        a = min(a, float(np.min(-tau * (w[neg] - lo[neg]) / d[neg])))
    if pos.any():
        a = min(a, float(np.min(tau * (hi[pos] - w[pos]) / d[pos])))
    return a


def _max_step_dual(z, dz, tau):
    neg = dz < 0
    return 1.0 if not neg.any() else min(1.0, float(np.min(-tau * z[neg] / dz[neg])))


def explicit_jacobian(on, x, u, pd=None, qd=None):
    """J = dc/du on g = 0, column by column (m x n_u)."""
    J = np.zeros((on.m, on.nu))
    for j in range(on.nu):
        e = np.zeros(on.nu)
        e[j] = 1.0
        J[:, j], _ = on.jac_prod(x, u, v=e, pd=pd, qd=qd)
    return J


def tracking_update(on, x, u, s, y, st, al, pd=None, qd=None, tol=1e-6, max_it=50, max_halvings=10,
                    delta_start=0.0, inertia_only=False):
    """One update from w_t = (u, s) with the state x at u and the new loads.  st: bounds, bound duals
    and mu (the QP's first barrier).  Returns the new point, duals, y, and the QP's record."""
    alt = dict(al, y=y, s=s)
    g = on.reduced_gradient(x, u, alt, pd=pd, qd=qd)
    H0 = on.reduced_hessian(x, u, alt, omega=np.zeros(on.m), pd=pd, qd=qd)
    H0 = 0.5 * (H0 + H0.T)
    J = explicit_jacobian(on, x, u, pd, qd)
    R = al["rho"] * al["sigma_c"] ** 2
    nu = on.nu
    u0, s0 = u.copy(), s.copy()
    w_u, w_s = u.copy(), s.copy()
    z = {k: st[k].copy() for k in ("zl_u", "zu_u", "zl_s", "zu_s")}
    bnd = {k: st[k] for k in ("u_lo", "u_hi", "s_lo", "s_hi")}
    mu = st["mu"]
    # convexity: the smallest delta in {delta_start or 0, 1e-8, 1e-7, ...} with H_uu + delta I
    # positive definite (the QP's Hessian is then positive semidefinite); with inertia_only delta
    # grows only where an iteration's Schur complement S is not positive definite
    delta = delta_start
    while not inertia_only:
        try:
            np.linalg.cholesky(H0 + delta * np.eye(nu))
            break
        except np.linalg.LinAlgError:
            delta = 10.0 * delta if delta > 0 else 1e-8
    delta_convex = delta

    def grad_q(delta):
        du, ds = w_u - u0, w_s - s0
        Jdu = J @ du
        gu = g["grad_u"] + H0 @ du + J.T @ (R * Jdu) - J.T @ (R * ds) + delta * du
        gs = g["grad_s"] - R * Jdu + R * ds
        return gu, gs

    it = 0
    rec = []
    while True:
        gu, gs = grad_q(delta)
        e_mu, e_0, _ = kkt_errors(dict(grad_u=gu, grad_s=gs), w_u, w_s, dict(bnd, **z), mu)
        rec.append((mu, delta, e_0))
        if e_0 <= tol or it == max_it:
            break
        if e_mu <= 10.0 * mu:
            mu = max(tol / 10.0, min(0.2 * mu, mu ** 1.5))
        dlu, dhu = w_u - bnd["u_lo"], bnd["u_hi"] - w_u
        dls, dhs = w_s - bnd["s_lo"], bnd["s_hi"] - w_s
        sig_u = z["zl_u"] / dlu + z["zu_u"] / dhu
        sig_s = z["zl_s"] / dls + z["zu_s"] / dhs
        omega = R * sig_s / (R + sig_s)
        S = H0 + J.T @ (omega[:, None] * J) + np.diag(sig_u)
        while True:
            try:
                L = np.linalg.cholesky(S + delta * np.eye(nu))
                break
            except np.linalg.LinAlgError:
                delta = 10.0 * delta if delta > 0 else 1e-8
        gu, gs = grad_q(delta)
        gpsi_u = gu - mu / dlu + mu / dhu
        gpsi_s = gs - mu / dls + mu / dhs
        v = R / (R + sig_s) * gpsi_s
        r = -gpsi_u - J.T @ v
        du = np.linalg.solve(L.T, np.linalg.solve(L, r))
        ds = (-gpsi_s + R * (J @ du)) / (R + sig_s)
        tau = max(0.99, 1.0 - mu)
        dz = {"zl_u": mu / dlu - z["zl_u"] - z["zl_u"] / dlu * du,
              "zu_u": mu / dhu - z["zu_u"] + z["zu_u"] / dhu * du,
              "zl_s": mu / dls - z["zl_s"] - z["zl_s"] / dls * ds,
              "zu_s": mu / dhs - z["zu_s"] + z["zu_s"] / dhs * ds}
        ap = min(_max_step(w_u, du, bnd["u_lo"], bnd["u_hi"], tau), _max_step(w_s, ds, bnd["s_lo"], bnd["s_hi"], tau))
        ad = min(_max_step_dual(z[k], dz[k], tau) for k in dz)
        w_u = w_u + ap * du
        w_s = w_s + ap * ds
        z = {k: z[k] + ad * dz[k] for k in z}
        it += 1
    halvings = 0
    while True:
        xn, info = on.powerflow(w_u, pd=pd, qd=qd, x0=x)
        if info["rc"] == 0:
            break
        if halvings >= max_halvings:
            raise RuntimeError("no control toward the QP solution with a converged power flow")
        w_u = u0 + 0.5 * (w_u - u0)
        w_s = s0 + 0.5 * (w_s - s0)
        halvings += 1
    c_new = on.eval(xn, w_u, pd=pd, qd=qd)["c"]
    y_new = y + al["rho"] * al["sigma_c"] * (c_new - w_s)
    return dict(u=w_u, s=w_s, x=xn, y=y_new, duals=z, mu=mu, delta=delta, delta_convex=delta_convex,
                iterations=it, kkt=rec[-1][2], halvings=halvings, record=rec)
