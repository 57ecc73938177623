"""Pins of the oracle's static-OPF augmented-Lagrangian loop (Sec. IV-B), no GPU.

The loop's end point must be a local solution of the OPF itself, which an
independent method finds too: scipy's SLSQP on the reduced problem
    min sigma_f f(u)  s.t.  c_lo <= c(u) <= c_hi,  u_lo <= u <= u_hi,
with f and c evaluated through the oracle's power flow and constraint
functions (their definitions, pinned elsewhere).  A wrong sign or weight in
the multiplier update, the penalty rule or the step would leave the loop
infeasible or at another cost.  The 30-bus grid's line limits are widened
1.5x for this instance: at 1.2x the base-case DC flows the AC flows of the
base case exceed them and the loop stalls at a primal infeasibility of 0.8.
"""
import numpy as np
import pytest

import oracle
from oracle import al_loop as L
from oracle import al_step as A
from paper_2110_02590_b300 import synth


def static_setup(name, rate_factor=1.5, mu=0.1, seed=5):
    """Static OPF instance: nominal loads, line limits rate_factor x the generator's, y = 0,
    rho = 10; controls 2% inside their bounds, slacks at c clipped 1% inside theirs, duals on
    the central path at mu."""
    net = synth.workload(name)
    on = oracle.OracleNet(net)
    u_lo, u_hi = synth.control_bounds(net)
    u = np.clip(synth.flat_control(net), u_lo + 0.02 * (u_hi - u_lo), u_hi - 0.02 * (u_hi - u_lo))
    x, info = on.powerflow(u)
    assert info["rc"] == 0
    al = synth.al_inputs(net, seed=seed)
    nl = net.n_branch
    al["s_hi"][:2 * nl] *= rate_factor ** 2
    al["sigma_c"][:2 * nl] /= rate_factor ** 2
    al["y"] = np.zeros(on.m)
    al["rho"] = 10.0
    lo, hi = al["s_lo"], al["s_hi"]
    s = np.clip(on.eval(x, u)["c"], lo + 0.01 * (hi - lo), hi - 0.01 * (hi - lo))
    al["s"] = s
    st = A.interior_state(al, u, lo, hi, u_lo, u_hi, mu=mu)
    return net, on, x, u, s, al, st


@pytest.fixture(scope="module")
def tiny_run():
    net, on, x, u, s, al, st = static_setup("tiny30")
    out = L.al_solve(on, x, u, s, al["y"], st, al, rho=10.0, max_outer=40, max_inner=10)
    return net, on, x, u, al, st, out


def test_al_loop_converges_to_the_slsqp_optimum(tiny_run):
    from scipy.optimize import minimize
    net, on, x, u0, al, st, out = tiny_run
    assert out["converged"]
    lo, hi = al["s_lo"], al["s_hi"]

    def ev(uu):
        xx, info = on.powerflow(uu, x0=x)
        assert info["rc"] == 0
        return on.eval(xx, uu)

    res = minimize(lambda uu: al["sigma_f"] * ev(uu)["cost"], u0, method="SLSQP",
                   bounds=list(zip(st["u_lo"], st["u_hi"])),
                   constraints=[{"type": "ineq",
                                 "fun": lambda uu: np.concatenate([(ev(uu)["c"] - lo) * al["sigma_c"],
                                                                   (hi - ev(uu)["c"]) * al["sigma_c"]])}],
                   options=dict(maxiter=500, ftol=1e-12))
    c_sq = ev(res.x)["c"]
    assert np.all((c_sq - lo) * al["sigma_c"] > -1e-6) and np.all((hi - c_sq) * al["sigma_c"] > -1e-6)
    f_al = al["sigma_f"] * ev(out["u"])["cost"]
    # the barrier (mu = 1e-5 at the end) and eta_p <= 1e-5 keep the AL point within ~1e-4 of the optimum
    assert abs(f_al - res.fun) <= 2e-4 * abs(res.fun), (f_al, res.fun)
    assert np.abs(out["u"] - res.x).max() < 2e-2


def test_al_loop_invariants(tiny_run):
    net, on, x, u0, al, st, out = tiny_run
    assert np.all(out["u"] > st["u_lo"]) and np.all(out["u"] < st["u_hi"])
    assert np.all(out["s"] > st["s_lo"]) and np.all(out["s"] < st["s_hi"])
    for k, z in out["duals"].items():
        assert np.all(z > 0), k
    assert np.linalg.norm(on.eval(out["x"], out["u"])["g"]) < 1e-10
    hist = np.array(out["history"])
    mus, rhos = hist[:, 1], hist[:, 2]
    assert np.all(np.diff(mus) <= 0) and mus[-1] >= 1e-5
    assert np.all(np.diff(rhos) >= 0) and rhos.max() <= 1e6
    # the last row is the stopping test
    assert hist[-1, 3] <= 1e-5 and hist[-1, 4] <= 1e-4
    # the multipliers are those of the final subproblem's constraints: y + rho D (c - s) at the end
    # reproduces the gradient of the Lagrangian (E_0 small) -- checked through the stopping test


def test_kkt_errors_definition():
    """E_mu and E_0 on hand-made numbers (the formula, with both bound sides)."""
    g = dict(grad_u=np.array([1.0, -2.0]), grad_s=np.array([0.5]))
    st = dict(zl_u=np.array([1.0, 0.5]), zu_u=np.array([0.25, 2.0]), zl_s=np.array([0.1]), zu_s=np.array([0.3]),
              u_lo=np.array([0.0, 0.0]), u_hi=np.array([1.0, 1.0]), s_lo=np.array([-1.0]), s_hi=np.array([1.0]))
    u, s = np.array([0.5, 0.25]), np.array([0.0])
    e_mu, e_0, dual = L.kkt_errors(g, u, s, st, mu=0.1)
    # dual: |1 - 1 + 0.25| = 0.25, |-2 - 0.5 + 2| = 0.5, |0.5 - 0.1 + 0.3| = 0.7
    assert dual == pytest.approx(0.7)
    # complementarity at 0: (0.5)(1) = 0.5, (0.5)(0.25), (0.25)(0.5), (0.75)(2) = 1.5, (1)(0.1), (1)(0.3)
    assert e_0 == pytest.approx(1.5)
    assert e_mu == pytest.approx(1.4)
