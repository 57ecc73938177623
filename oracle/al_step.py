"""Reduced-Newton step of the augmented-Lagrangian subproblem (TEST INFRASTRUCTURE ONLY).

One primal-dual barrier Newton step on w = (u, s) for
    psi_mu(w) = L_rho(u, s; y) - mu sum log(w - w_lo) - mu sum log(w_hi - w)
(Sec. IV-B, eq. ipm_subproblem and eq. ipm_firstorderconditions), with the
scaled AL of Sec. IV-A:  L_rho = sigma_f f + y^T D (c - s) + rho/2 |D (c - s)|^2,
D = diag(sigma_c).  The Newton system is eq. ipm_kkt_reduced,
    [grad^2 L_rho + Sigma] d_w = -grad psi_mu,   Sigma = Z_lo/(w - w_lo) + Z_hi/(w_hi - w),
with the Hessian of eq. hessian_auglag (scaled):
    [[H_uu + J^T rho D^2 J, -J^T rho D^2], [-rho D^2 J, rho D^2]],
J = dc/du on the manifold.  `schur_step` eliminates d_s as in Prop. 3:
    S_uu = H_uu + Sigma_u + J^T (rho D^2 - rho D^2 (rho D^2 + Sigma_s)^{-1} rho D^2) J
         = H(omega) + Sigma_u,  omega_i = rho sigma_i^2 Sigma_s,i / (rho sigma_i^2 + Sigma_s,i),
    S_uu d_u = -grad_u psi - J^T [rho D^2 (rho D^2 + Sigma_s)^{-1}] grad_s psi,
    d_s = (rho D^2 + Sigma_s)^{-1} (-grad_s psi + rho D^2 J d_u),
and H(omega) is the reduced Hessian with Gauss-Newton weights omega (the oracle's
Prop. 2 HVPs).  Reading: the sign of the second term of the d_u right-hand side
follows from eliminating the second block row of eq. ipm_kkt_reduced; the
printed statement of Prop. 3 has the opposite sign.  `direct_step` solves the
full (n_u + m) system densely (small nets) and pins `schur_step`.

Dual step (eq. ipm_kkt, second block row): dz_lo = mu/(w - w_lo) - z_lo - Sigma_lo d_w,
dz_hi = mu/(w_hi - w) - z_hi + Sigma_hi d_w.  Fraction to the boundary with
tau = max(0.99, 1 - mu); the trial control is accepted when the power flow
converges, else alpha is halved (feasibility of every iterate, Sec. I).
Inertia correction: delta in {0, 1e-8, 1e-7, ..., 1e16} added to the u-block
(i.e. to S_uu) until the Cholesky factorisation succeeds; with delta_start > 0
the tries are delta_start, 10 delta_start, ... (carrying a previous step's delta).  The reduced Hessian
of the AL is indefinite away from a solution, so the correction is needed.
"""
import numpy as np


def _bound_terms(w, lo, hi, zlo, zhi, mu):
    dlo, dhi = w - lo, hi - w
    sig = zlo / dlo + zhi / dhi
    bar = -mu / dlo + mu / dhi      # gradient of the barrier
    return sig, bar, dlo, dhi


def newton_pieces(on, x, u, s, st, al, pd=None, qd=None):
    """Gradient, Sigma, grad psi and omega at (u, s).  st: dict of duals/bounds/mu."""
    al_s = dict(al, s=s)
    g = on.reduced_gradient(x, u, al_s, pd=pd, qd=qd)
    sig_u, bar_u, _, _ = _bound_terms(u, st["u_lo"], st["u_hi"], st["zl_u"], st["zu_u"], st["mu"])
    sig_s, bar_s, _, _ = _bound_terms(s, st["s_lo"], st["s_hi"], st["zl_s"], st["zu_s"], st["mu"])
    rd2 = al["rho"] * al["sigma_c"] ** 2
    return dict(g=g, sig_u=sig_u, sig_s=sig_s, gpsi_u=g["grad_u"] + bar_u, gpsi_s=g["grad_s"] + bar_s,
                rd2=rd2, omega=rd2 * sig_s / (rd2 + sig_s))


def cholesky_with_inertia(S, max_tries=24, delta_start=0.0):
    delta = delta_start
    for k in range(max_tries + 1):
        try:
            L = np.linalg.cholesky(S + delta * np.eye(S.shape[0]))
            return L, delta
        except np.linalg.LinAlgError:
            delta = delta_start * 10.0 ** (k + 1) if delta_start > 0 else 1e-8 * 10.0 ** k
    raise np.linalg.LinAlgError("not positive definite after inertia corrections")


def schur_step(on, x, u, s, st, al, pd=None, qd=None, delta_start=0.0):
    """(d_u, d_s) by Prop. 3 with the oracle's reduced Hessian and reduced Jacobian products."""
    P = newton_pieces(on, x, u, s, st, al, pd, qd)
    H = on.reduced_hessian(x, u, dict(al, s=s), omega=P["omega"], pd=pd, qd=qd)
    S = 0.5 * (H + H.T) + np.diag(P["sig_u"])
    v = P["rd2"] / (P["rd2"] + P["sig_s"]) * P["gpsi_s"]
    _, Jtv = on.jac_prod(x, u, w=v, pd=pd, qd=qd)
    r = -P["gpsi_u"] - Jtv
    L, delta = cholesky_with_inertia(S, delta_start=delta_start)
    du = np.linalg.solve(L.T, np.linalg.solve(L, r))
    Jdu, _ = on.jac_prod(x, u, v=du, pd=pd, qd=qd)
    ds = (-P["gpsi_s"] + P["rd2"] * Jdu) / (P["rd2"] + P["sig_s"])
    return dict(du=du, ds=ds, S=S, r=r, delta=delta, pieces=P)


def direct_step(on, x, u, s, st, al, pd=None, qd=None, delta=0.0):
    """(d_u, d_s) from the full (n_u + m) system of eq. ipm_kkt_reduced, dense (small nets only),
    with the inertia correction delta on the u-block."""
    P = newton_pieces(on, x, u, s, st, al, pd, qd)
    H0 = on.reduced_hessian(x, u, dict(al, s=s), omega=np.zeros(on.m), pd=pd, qd=qd)
    J = on.bruteforce(x, u, dict(al, s=s), pd=pd, qd=qd)["J"]
    nu, m = on.nu, on.m
    R = np.diag(P["rd2"])
    K = np.zeros((nu + m, nu + m))
    K[:nu, :nu] = 0.5 * (H0 + H0.T) + J.T @ R @ J + np.diag(P["sig_u"]) + delta * np.eye(nu)
    K[:nu, nu:] = -J.T @ R
    K[nu:, :nu] = -R @ J
    K[nu:, nu:] = R + np.diag(P["sig_s"])
    d = np.linalg.solve(K, -np.concatenate([P["gpsi_u"], P["gpsi_s"]]))
    return dict(du=d[:nu], ds=d[nu:])


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


def barrier(u, s, st, mu):
    """-mu sum log(w - w_lo) - mu sum log(w_hi - w) over w = (u, s) (eq. ipm_subproblem)."""
    t = 0.0
    for w, nm in ((u, "u"), (s, "s")):
        t += np.log(w - st[nm + "_lo"]).sum() + np.log(st[nm + "_hi"] - w).sum()
    return -mu * t


def al_step(on, x, u, s, st, al, pd=None, qd=None, max_halvings=10, delta_start=0.0, line_search=False):
    """One reduced-Newton step: Schur solve, dual step, fraction to the boundary,
    power flow at the trial control with halving.  Returns the new iterate and the step data.

    line_search: also halve the step until the barrier function psi_mu = F + barrier
    decreases by the Armijo rule psi(w + a d) <= psi(w) + 1e-4 a grad psi^T d (the step
    solves a positive definite system, so it is a descent direction); after max_halvings
    the last trial with a converged power flow is taken."""
    out = schur_step(on, x, u, s, st, al, pd, qd, delta_start=delta_start)
    du, ds = out["du"], out["ds"]
    mu = st["mu"]
    tau = max(0.99, 1.0 - mu)
    dz = {}
    for nm, w, dw in (("u", u, du), ("s", s, ds)):
        lo, hi = st[nm + "_lo"], st[nm + "_hi"]
        zl, zu = st["zl_" + nm], st["zu_" + nm]
        dz["zl_" + nm] = mu / (w - lo) - zl - zl / (w - lo) * dw
        dz["zu_" + nm] = mu / (hi - w) - zu + zu / (hi - w) * dw
    ap = min(_max_step(u, du, st["u_lo"], st["u_hi"], tau), _max_step(s, ds, st["s_lo"], st["s_hi"], tau))
    ad = min(_max_step_dual(st[k], dz[k], tau) for k in dz)
    x_new = None
    halvings = 0
    P = out["pieces"]
    psi0 = P["g"]["F"] + barrier(u, s, st, mu)
    slope = float(P["gpsi_u"] @ du + P["gpsi_s"] @ ds)
    while True:
        xt, info = on.powerflow(u + ap * du, pd=pd, qd=qd, x0=x)
        if info["rc"] == 0:
            x_new = xt
            if not line_search or halvings >= max_halvings:
                break
            st_ = s + ap * ds
            F_t = on.reduced_gradient(xt, u + ap * du, dict(al, s=st_), pd=pd, qd=qd)["F"]
            if F_t + barrier(u + ap * du, st_, st, mu) <= psi0 + 1e-4 * ap * slope:
                break
        elif halvings >= max_halvings:
            raise RuntimeError("no feasible trial point after halvings")
        ap *= 0.5
        halvings += 1
    new = {k: st[k] + ad * dz[k] for k in dz}
    return dict(out, dz=dz, alpha_p=ap, alpha_d=ad, halvings=halvings, u=u + ap * du, s=s + ap * ds,
                x=x_new, duals=new)


def interior_state(net_al, u, s_lo, s_hi, u_lo, u_hi, mu=0.1):
    """A primal-dual start with z = mu / distance to each bound (on the central path)."""
    s = net_al["s"]
    return dict(u_lo=u_lo, u_hi=u_hi, s_lo=s_lo, s_hi=s_hi, mu=mu,
                zl_u=mu / (u - u_lo), zu_u=mu / (u_hi - u), zl_s=mu / (s - s_lo), zu_s=mu / (s_hi - s))
