"""Pins of the oracle's static-OPF augmented-Lagrangian loop (Sec. IV-B), no GPU.

The loop's end point must be a local solution of the OPF itself, which an
independent method finds too: scipy's SLSQP on the reduced problem
    min sigma_f f(u)  s.t.  c_lo <= c(u) <= c_hi,  u_lo <= u <= u_hi,
with f and c evaluated through the oracle's power flow and constraint
functions (their definitions, pinned elsewhere).  A wrong sign or weight in
the multiplier update, the penalty rule or the step would leave the loop
infeasible or at another cost.

The static OPF instances are built so that their AC base case is feasible
(`synth.static_instance`): line limits max(rate, 1.2 |S| of the base-case
flow) with an inactive lower bound, reactive limits widened to 1.2 |q| of the
base case, PQ voltage bounds widened to 2% around the base-case voltages.
The generator's own limits come from DC flows and per-unit bounds that the AC
base case violates (line flows up to 33x on the 9,200-bus grid, reactive
output up to 2x, voltages down to 0.81), and with them the loop stalled at a
primal infeasibility of 0.05 to 100.
"""
import numpy as np
import pytest

import oracle
from oracle import al_loop as L
from oracle import al_step as A
from paper_2110_02590_b300 import synth


def static_setup(name, mu=0.1, seed=5):
    """Static OPF instance: nominal loads, bounds from the AC base case (synth.static_instance),
    y = 0, rho = 10; controls 2% inside their bounds, slacks at c clipped 1% inside theirs,
    duals on the central path at mu."""
    net = synth.workload(name)
    on = oracle.OracleNet(net)
    u_lo, u_hi = synth.control_bounds(net)
    u0 = synth.flat_control(net)
    x0, info = on.powerflow(u0)
    assert info["rc"] == 0
    al = synth.static_instance(net, synth.al_inputs(net, seed=seed), on.eval(x0, u0)["c"])
    u = np.clip(u0, u_lo + 0.02 * (u_hi - u_lo), u_hi - 0.02 * (u_hi - u_lo))
    x, info = on.powerflow(u, x0=x0)
    assert info["rc"] == 0
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
    out = L.al_solve(on, x, u, s, al["y"], st, al, rho=10.0, max_outer=40, max_inner=30)
    return net, on, x, u, al, st, out


def test_al_loop_converges_to_the_slsqp_optimum(tiny_run):
    """SLSQP with exact derivatives: the objective's gradient from the oracle's adjoint with the
    AL terms switched off (y = 0, rho = 0), the constraints' Jacobian from the hyper-dual brute
    force (independent of the adjoint code)."""
    from scipy.optimize import minimize
    net, on, x, u0, al, st, out = tiny_run
    assert out["converged"]
    lo, hi, sc = al["s_lo"], al["s_hi"], al["sigma_c"]

    def ev(uu):
        xx, info = on.powerflow(uu, x0=x)
        assert info["rc"] == 0
        return xx, on.eval(xx, uu)

    def grad(uu):
        xx, e = ev(uu)
        return on.reduced_gradient(xx, uu, dict(al, y=np.zeros(on.m), rho=0.0, s=e["c"]))["grad_u"]

    def cons(uu):
        c = ev(uu)[1]["c"]
        return np.concatenate([(c - lo) * sc, (hi - c) * sc])

    def cons_jac(uu):
        xx, e = ev(uu)
        J = on.bruteforce(xx, uu, dict(al, s=e["c"]))["J"] * sc[:, None]
        return np.vstack([J, -J])

    res = minimize(lambda uu: al["sigma_f"] * ev(uu)[1]["cost"], u0, jac=grad, method="SLSQP",
                   bounds=list(zip(st["u_lo"], st["u_hi"])),
                   constraints=[{"type": "ineq", "fun": cons, "jac": cons_jac}],
                   options=dict(maxiter=1000, ftol=1e-12))  # 1e-14 ends on its line-search precision limit
    assert res.success, res.message
    assert cons(res.x).min() > -1e-9
    f_al = al["sigma_f"] * ev(out["u"])[1]["cost"]
    # the barrier (mu = 1e-5 at the end) and eta_p <= 1e-5 keep the AL point within ~1e-4 of the optimum
    assert abs(f_al - res.fun) <= 2e-4 * abs(res.fun), (f_al, res.fun)
    assert np.abs(out["u"] - res.x).max() < 3e-2


def test_scaled_loop_reaches_the_same_optimum(tiny_run):
    """The gradient-based scaling (Sec. IV-A) changes the path of the loop, not the OPF it solves: the
    scaled loop stops at the same controls and generation cost (the SLSQP pin above fixes that
    point), with the rule's scales: the caller's sigma_c times factors in (0, 1], sigma_f from the
    cost gradient."""
    net, on, x, u0, al, st, out = tiny_run
    s0 = np.clip(on.eval(x, u0)["c"], al["s_lo"] + 0.01 * (al["s_hi"] - al["s_lo"]),
                 al["s_hi"] - 0.01 * (al["s_hi"] - al["s_lo"]))
    sc = L.al_solve(on, x, u0, s0, np.zeros(on.m), st, al, rho=10.0, max_outer=40, max_inner=30,
                    scaling_gmax=100.0)
    assert sc["converged"]
    assert np.all(sc["sigma_c"] <= al["sigma_c"]) and np.all(sc["sigma_c"] > 0)
    assert 0 < sc["sigma_f"] <= 1
    cost = lambda uu: on.eval(on.powerflow(uu, x0=x)[0], uu)["cost"]  # noqa: E731
    assert abs(cost(sc["u"]) - cost(out["u"])) <= 2e-4 * abs(cost(out["u"]))
    assert np.abs(sc["u"] - out["u"]).max() < 3e-2


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
