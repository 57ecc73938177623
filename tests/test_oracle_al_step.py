"""Pins of the oracle's reduced-Newton step (Prop. 3) against the direct dense
solve of eq. ipm_kkt_reduced (no GPU)."""
import numpy as np
import pytest

import oracle
from oracle import al_step as A
from paper_2110_02590_b300 import synth


def setup(net, mu=0.1, seed=5):
    """Interior primal-dual point: controls 2% inside their bounds, slacks at the constraint
    values clipped 1% inside theirs, duals on the central path."""
    on = oracle.OracleNet(net)
    u_lo, u_hi = synth.control_bounds(net)
    u = np.clip(synth.flat_control(net), u_lo + 0.02 * (u_hi - u_lo), u_hi - 0.02 * (u_hi - u_lo))
    x, info = on.powerflow(u)
    assert info["rc"] == 0
    al = synth.al_inputs(net, seed=seed)
    lo, hi = al["s_lo"], al["s_hi"]
    al["s"] = np.clip(on.eval(x, u)["c"], lo + 0.01 * (hi - lo), hi - 0.01 * (hi - lo))
    st = A.interior_state(al, u, lo, hi, u_lo, u_hi, mu=mu)
    return on, x, u, al, st


@pytest.mark.parametrize("which", ["tiny30", "mesh12"])
def test_schur_step_equals_direct_solve(which):
    net = synth.workload("tiny30") if which == "tiny30" else synth.make_network(12, 4, 18, seed=5,
                                                                                transformer_frac=0.3)
    on, x, u, al, st = setup(net)
    sch = A.schur_step(on, x, u, al["s"], st, al)
    dirs = A.direct_step(on, x, u, al["s"], st, al, delta=sch["delta"])
    assert np.abs(sch["du"] - dirs["du"]).max() <= 1e-9 * np.abs(dirs["du"]).max()
    assert np.abs(sch["ds"] - dirs["ds"]).max() <= 1e-9 * np.abs(dirs["ds"]).max()


def test_printed_sign_of_prop3_does_not_solve_the_system():
    """With the opposite sign on the J^T term of the d_u right-hand side the step is not
    the solution of eq. ipm_kkt_reduced (records the reading of Prop. 3)."""
    on, x, u, al, st = setup(synth.workload("tiny30"))
    P = A.newton_pieces(on, x, u, al["s"], st, al)
    sch = A.schur_step(on, x, u, al["s"], st, al)
    v = P["rd2"] / (P["rd2"] + P["sig_s"]) * P["gpsi_s"]
    _, Jtv = on.jac_prod(x, u, w=v)
    du_printed = np.linalg.solve(sch["S"] + sch["delta"] * np.eye(on.nu), -P["gpsi_u"] + Jtv)
    dirs = A.direct_step(on, x, u, al["s"], st, al, delta=sch["delta"])
    assert np.abs(du_printed - dirs["du"]).max() > 1e-3 * np.abs(dirs["du"]).max()


def test_al_step_keeps_feasibility_and_interior():
    on, x, u, al, st = setup(synth.workload("medium1400"))
    out = A.al_step(on, x, u, al["s"], st, al)
    assert 0.0 < out["alpha_p"] <= 1.0 and 0.0 < out["alpha_d"] <= 1.0
    assert np.all(out["u"] > st["u_lo"]) and np.all(out["u"] < st["u_hi"])
    assert np.all(out["s"] > st["s_lo"]) and np.all(out["s"] < st["s_hi"])
    for k, z in out["duals"].items():
        assert np.all(z > 0), k
    assert np.linalg.norm(on.eval(out["x"], out["u"])["g"]) < 1e-10
