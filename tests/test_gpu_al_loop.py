"""GPU parity of the static-OPF augmented-Lagrangian loop (opf_al_solve) with the oracle's loop.

Both sides run the same readings (KKT errors, barrier and penalty rules, the
multiplier update y <- y + rho D_c (c - s)) from the same start; each outer
iteration's decisions (steps taken, mu, rho) must coincide and its measured
quantities (eta_p, E_0, F) agree; the end points agree within the step
tolerance (each step agrees to ~1e-9 and the loop is self-correcting).
"""
import numpy as np
import pytest

from oracle import al_loop as L
from tests.test_oracle_al_loop import static_setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2110_02590_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def run_both(name, max_outer, max_inner=30, scaling_gmax=0.0):
    net, on, x, u, s, al, st = static_setup(name)
    ref = L.al_solve(on, x, u, s, al["y"], st, al, rho=10.0, max_outer=max_outer, max_inner=max_inner,
                     scaling_gmax=scaling_gmax)
    ctx = P.OPFContext(net)
    xg, _ = ctx.powerflow(dev(u))
    state = {k: dev(v) for k, v in st.items() if k != "mu"}
    state.update(u=dev(u), s=dev(s), x=xg, mu=st["mu"])
    y = dev(al["y"])
    info, hist = ctx.al_solve(dict(sigma_f=al["sigma_f"], rho=10.0, sigma_c=dev(al["sigma_c"])), state, y,
                              max_outer=max_outer, max_inner=max_inner, scaling_gmax=scaling_gmax)
    return ref, info, hist, state, y


@pytest.mark.parametrize("name,max_outer,gmax", [("tiny30", 1, 0.0), ("tiny30", 3, 0.0), ("medium1400", 2, 0.0),
                                                 ("tiny30", 3, 100.0), ("medium1400", 2, 100.0)])
def test_al_loop_parity(name, max_outer, gmax):
    """Iterate by iterate over the first outer iterations (a few dozen line-searched steps): the
    decisions (steps per subproblem, mu, rho, stop) coincide exactly.  E_0 is the infinity norm of
    grad L - z_lo + z_hi, a difference of bound-dual terms of up to ~1e4 near the bounds, so
    rounding-level differences of the iterates show in it at ~1e-4; eta_p, F and the iterates agree
    far more closely.  (Over longer runs an Armijo test or a subproblem stop that falls within
    rounding of its threshold can go the other way; the converged run is compared at its end.)"""
    ref, info, hist, state, y = run_both(name, max_outer, scaling_gmax=gmax)
    # the scales (the caller's, or the gradient rule's at the start) agree first; the rule's
    # scales are g_max over the largest |entry| of a row of the reduced Jacobian J (or of the
    # cost gradient), and J's entries differ from the oracle's by summation order (the tile
    # width is autotuned by timing), up to ~2e-12 relative here against 1e-9 in J's own parity
    assert rel(info["sigma_c"].cpu().numpy(), ref["sigma_c"]) < 1e-10
    assert abs(info["sigma_f"] - ref["sigma_f"]) <= 1e-10 * ref["sigma_f"]
    rh = np.array(ref["history"])
    assert info["outer"] == len(rh)
    assert info["converged"] == int(ref["converged"])
    assert info["steps"] == ref["steps"]
    assert np.array_equal(hist[:, 0], rh[:, 0])                     # steps per outer iteration
    assert np.allclose(hist[:, 1], rh[:, 1], rtol=1e-12, atol=0)   # mu
    assert np.array_equal(hist[:, 2], rh[:, 2])                     # rho
    assert np.all(np.abs(hist[:, 3] - rh[:, 3]) <= 1e-5 * np.maximum(1.0, np.abs(rh[:, 3])))  # eta_p
    assert np.all(np.abs(hist[:, 4] - rh[:, 4]) <= 1e-3 * np.maximum(1.0, np.abs(rh[:, 4])))  # E_0
    assert np.all(np.abs(hist[:, 5] - rh[:, 5]) <= 1e-7 * np.abs(rh[:, 5]))  # F
    assert rel(state["u"].cpu().numpy(), ref["u"]) < 1e-5
    assert rel(state["s"].cpu().numpy(), ref["s"]) < 1e-5
    # y moves by rho D_c (c - s) per outer iteration: rho up to 1e3 scales the rounding-level
    # differences of c - s into y
    assert rel(y.cpu().numpy(), ref["y"]) < 1e-3
    assert info["rho"] == ref["rho"] and abs(state["mu"] - ref["mu"]) <= 1e-12 * ref["mu"]
    assert np.abs(state["x"].cpu().numpy() - ref["x"]).max() < 1e-5


@pytest.mark.parametrize("gmax", [0.0, 100.0])
def test_al_loop_reaches_the_oracle_optimum(gmax):
    """To convergence (rho climbs to 1e6, where the subproblems are ill conditioned and
    rounding-level differences change how many outer iterations each side takes): both
    sides stop at the tolerances, at the same point and cost."""
    ref, info, hist, state, y = run_both("tiny30", 40, scaling_gmax=gmax)
    assert ref["converged"] and info["converged"]
    assert info["primal_inf"] <= 1e-5 and info["dual_inf"] <= 1e-4
    assert abs(len(ref["history"]) - info["outer"]) <= 3
    assert rel(state["u"].cpu().numpy(), ref["u"]) < 1e-4
    assert abs(info["F"] - ref["history"][-1][5]) <= 1e-5 * abs(ref["history"][-1][5])


@pytest.mark.parametrize("name", ["medium1400", "large9200"])
def test_scaled_static_opf_converges(name):
    """The static OPF of the 1,400- and 9,200-bus instances with the gradient-based scaling runs to
    the tolerances (eta_p <= 1e-5, E_0 <= 1e-4) at a feasible, interior point of the manifold."""
    net, on, x, u, s, al, st = static_setup(name)
    ctx = P.OPFContext(net)
    xg, _ = ctx.powerflow(dev(u))
    state = {k: dev(v) for k, v in st.items() if k != "mu"}
    state.update(u=dev(u), s=dev(s), x=xg, mu=st["mu"])
    y = dev(al["y"])
    info, hist = ctx.al_solve(dict(sigma_f=al["sigma_f"], rho=10.0, sigma_c=dev(al["sigma_c"])), state, y,
                              max_outer=20, max_inner=60, scaling_gmax=100.0)
    assert info["converged"], (info, hist)
    assert info["primal_inf"] <= 1e-5 and info["dual_inf"] <= 1e-4
    uu, ss = state["u"].cpu().numpy(), state["s"].cpu().numpy()
    assert np.all(uu > st["u_lo"]) and np.all(uu < st["u_hi"])
    assert np.all(ss > st["s_lo"]) and np.all(ss < st["s_hi"])
    # the state is the power flow at the final controls
    x2, pinfo = ctx.powerflow(state["u"], x0=state["x"])
    assert pinfo["iterations"] == 0 and np.abs(x2.cpu().numpy() - state["x"].cpu().numpy()).max() == 0.0
