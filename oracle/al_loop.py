"""Static OPF augmented-Lagrangian outer loop (TEST INFRASTRUCTURE ONLY).

Sec. IV-B "Static OPF algorithm": each outer iteration solves the AL
subproblem (eq. auglag_subproblem, scaled as in Sec. IV-A "Scaling") for a
fixed penalty rho and multiplier y with the interior-point method of
Sec. IV-B (one reduced-Newton step per iteration, `al_step.al_step`),
warm-started from the previous primal-dual point, then updates the
multiplier y <- y + rho D_c (c - s) and the penalty.

The paper leaves the IPM's internals and the AL schedule to MadNLP and the
textbook; the readings (the same ones the library's opf_al_solve takes):
  * KKT error of the barrier subproblem at w = (u, s) with bound duals z:
        E_mu = max(|grad_u L - zl_u + zu_u|_inf, |grad_s L - zl_s + zu_s|_inf,
                   |(w - w_lo) zl - mu|_inf, |(w_hi - w) zu - mu|_inf),
    E_0 the same with mu = 0 (the error of the AL subproblem itself);
  * inner loop: evaluate the gradient; stop when E_0 <= omega_k =
    max(eta_dual, 10^-(k+1)) or after max_inner steps; when E_mu <= 10 mu the
    barrier drops to max(eta_dual / 10, min(0.2 mu, mu^1.5)) (Wachter &
    Biegler's rule); then one reduced-Newton step;
  * inertia correction of a step starts at delta/10 of the previous step's
    delta when that was at least 1e-7, else at 0; each step backtracks on the
    barrier function (Armijo rule, al_step's line_search): the subproblems are
    nonconvex away from a solution, and full Newton steps there can increase
    psi_mu and diverge;
  * after the subproblem: primal infeasibility eta_p = |D_c (c - s)|_inf; stop
    when eta_p <= eta_primal and E_0 <= eta_dual; else y <- y + rho D_c (c - s),
    and rho <- min(10 rho, rho_max) when eta_p fell by less than a factor 4;
  * optional gradient-based scaling before the first iteration (Sec. IV-A
    "Scaling", `scaling.gradient_scaling` at the starting point with the
    caller's sigma_c as the prior; sigma_f from the cost gradient alone).
"""
import numpy as np

from oracle import al_step as A
from oracle import scaling as S


def kkt_errors(g, u, s, st, mu):
    """(E_mu, E_0, dual part) of the barrier subproblem from the reduced gradient dict g."""
    du = g["grad_u"] - st["zl_u"] + st["zu_u"]
    ds = g["grad_s"] - st["zl_s"] + st["zu_s"]
    dual = max(np.abs(du).max(initial=0.0), np.abs(ds).max(initial=0.0))
    comp = []
    for mm in (mu, 0.0):
        c = 0.0
        for w, nm in ((u, "u"), (s, "s")):
            c = max(c, np.abs((w - st[nm + "_lo"]) * st["zl_" + nm] - mm).max(initial=0.0),
                    np.abs((st[nm + "_hi"] - w) * st["zu_" + nm] - mm).max(initial=0.0))
        comp.append(c)
    return max(dual, comp[0]), max(dual, comp[1]), dual


def al_solve(on, x, u, s, y, st, al, rho, max_outer=20, max_inner=30, eta_primal=1e-5, eta_dual=1e-4,
             rho_max=1e6, scaling_gmax=0.0):
    """Run the outer loop from (x, u, s, y, duals in st, st['mu'], rho).  Returns the final point, the
    scales used and one history row per outer iteration: (inner steps, mu, rho, eta_p, E_0, F)."""
    if scaling_gmax > 0.0:
        J = S.explicit_jacobian(on, x, u)
        sig, sf = S.gradient_scaling(J, S.cost_gradient(on, x, u), g_max=scaling_gmax, prior=al["sigma_c"])
        al = dict(al, sigma_c=sig, sigma_f=sf)
    st = dict(st)
    u, s, y, x = u.copy(), s.copy(), y.copy(), x.copy()
    mu = st["mu"]
    prev_eta = np.inf
    delta = 0.0
    hist = []
    converged = False
    steps_total = 0
    for k in range(max_outer):
        omega_k = max(eta_dual, 10.0 ** -(k + 1))
        steps = 0
        for j in range(max_inner + 1):
            alk = dict(al, y=y, rho=rho)
            g = on.reduced_gradient(x, u, dict(alk, s=s))
            e_mu, e_0, _ = kkt_errors(g, u, s, st, mu)
            if e_0 <= omega_k or j == max_inner:
                break
            if e_mu <= 10.0 * mu:
                mu = max(eta_dual / 10.0, min(0.2 * mu, mu ** 1.5))
            st["mu"] = mu
            out = A.al_step(on, x, u, s, st, alk, delta_start=(delta / 10.0 if delta >= 1e-7 else 0.0),
                            line_search=True)
            delta = out["delta"]
            u, s, x = out["u"], out["s"], out["x"]
            st.update(out["duals"])
            steps += 1
        steps_total += steps
        eta_p = float(np.abs(al["sigma_c"] * (g["c"] - s)).max())
        hist.append((steps, mu, rho, eta_p, e_0, g["F"]))
        if eta_p <= eta_primal and e_0 <= eta_dual:
            converged = True
            break
        y = y + rho * al["sigma_c"] * (g["c"] - s)
        if eta_p > 0.25 * prev_eta:
            rho = min(10.0 * rho, rho_max)
        prev_eta = eta_p
    st["mu"] = mu
    return dict(x=x, u=u, s=s, y=y, rho=rho, mu=mu, duals={k: st[k] for k in ("zl_u", "zu_u", "zl_s", "zu_s")},
                history=hist, converged=converged, steps=steps_total, delta=delta,
                sigma_c=np.asarray(al["sigma_c"], dtype=np.float64).copy(), sigma_f=float(al["sigma_f"]))
