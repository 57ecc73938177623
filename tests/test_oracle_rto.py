"""Pins of the oracle's real-time tracking update (Sec. IV-C, eq. qp_rto), no GPU.

The interior-point QP solve is checked against an independent solver of the
same bounded QP: L-BFGS-B (box constraints handled natively) on
q(d) = g^T d + 1/2 d^T (H_t + delta I_u) d with H_t assembled here from the
explicit blocks of eq. hessian_auglag.  With delta_start above -lambda_min of
the reduced block the QP is strictly convex, so both must reach the same
minimiser (the IPM stops at a barrier of ~tol/10, which moves the active
bounds' components by ~1e-7).
"""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import rto
from paper_2110_02590_b300 import synth
from tests.test_oracle_al_loop import static_setup


def tracking_instance(name, step=1, mu=1e-2):
    net, on, x, u, s, al, st = static_setup(name, mu=mu)
    pds, qds = synth.ar1_loads(net, step + 1, seed=100)
    pd, qd = pds[step], qds[step]
    x1, info = on.powerflow(u, pd=pd, qd=qd, x0=x)
    assert info["rc"] == 0
    return net, on, x1, u, s, al, st, pd, qd


@pytest.mark.parametrize("inertia_only", [False, True])
def test_qp_solution_matches_lbfgsb_on_the_convex_qp(inertia_only):
    """With and without the convexity search (inertia_only: delta grows only where an
    iteration's S is not positive definite; here the QP is convex from delta_start on)."""
    net, on, x, u, s, al, st, pd, qd = tracking_instance("tiny30")
    y = np.zeros(on.m)
    alt = dict(al, y=y, s=s)
    g = on.reduced_gradient(x, u, alt, pd=pd, qd=qd)
    H0 = on.reduced_hessian(x, u, alt, omega=np.zeros(on.m), pd=pd, qd=qd)
    H0 = 0.5 * (H0 + H0.T)
    delta = max(0.0, -np.linalg.eigvalsh(H0).min()) + 1e-3
    out = rto.tracking_update(on, x, u, s, y, st, al, pd=pd, qd=qd, tol=1e-8, delta_start=delta,
                              inertia_only=inertia_only)
    assert out["kkt"] <= 1e-8 and out["delta"] == delta and out["halvings"] == 0
    J = rto.explicit_jacobian(on, x, u, pd, qd)
    R = al["rho"] * al["sigma_c"] ** 2
    nu = on.nu

    def q(d):
        du, ds = d[:nu], d[nu:]
        Jdu = J @ du
        gu = g["grad_u"] + H0 @ du + J.T @ (R * (Jdu - ds)) + delta * du
        gs = g["grad_s"] + R * (ds - Jdu)
        val = g["grad_u"] @ du + g["grad_s"] @ ds + 0.5 * (du @ H0 @ du + delta * du @ du + (R * (Jdu - ds)) @ (Jdu - ds))
        return val, np.concatenate([gu, gs])

    lo = np.concatenate([st["u_lo"] - u, st["s_lo"] - s])
    hi = np.concatenate([st["u_hi"] - u, st["s_hi"] - s])
    res = minimize(q, np.zeros(nu + on.m), jac=True, method="L-BFGS-B", bounds=list(zip(lo, hi)),
                   options=dict(maxiter=20000, ftol=1e-15, gtol=1e-11, maxcor=50))
    d_ipm = np.concatenate([out["u"] - u, out["s"] - s])
    assert np.abs(d_ipm - res.x).max() <= 1e-5 * max(1.0, np.abs(res.x).max())
    assert q(d_ipm)[0] - res.fun <= 1e-8 * max(1.0, abs(res.fun))


def test_tracking_update_feasible_and_interior():
    net, on, x, u, s, al, st, pd, qd = tracking_instance("tiny30")
    out = rto.tracking_update(on, x, u, s, np.zeros(on.m), st, al, pd=pd, qd=qd)
    assert 0 < out["iterations"] <= 50 and out["kkt"] <= 1e-6
    assert np.all(out["u"] > st["u_lo"]) and np.all(out["u"] < st["u_hi"])
    assert np.all(out["s"] > st["s_lo"]) and np.all(out["s"] < st["s_hi"])
    for k, z in out["duals"].items():
        assert np.all(z > 0), k
    assert np.linalg.norm(on.eval(out["x"], out["u"], pd=pd, qd=qd)["g"]) < 1e-10
    c_new = on.eval(out["x"], out["u"], pd=pd, qd=qd)["c"]
    assert np.allclose(out["y"], al["rho"] * al["sigma_c"] * (c_new - out["s"]), rtol=0, atol=1e-12)
