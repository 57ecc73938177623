"""GPU parity of the real-time tracking update (opf_tracking_update, Sec. IV-C) with the oracle.

The library forms each QP iteration's Schur complement from HVPs at the
fixed linearisation point with the iteration's weights and carries grad q
through the Newton system; the oracle forms S from the explicit reduced
Hessian and Jacobian (eq. schur_matrix) and evaluates grad q from its
definition.  Both take the same decisions (iterations, delta, halvings) and
reach the same point: the QP solution agrees to the step tolerance (1e-6
relative, as for one reduced-Newton step) and the new state, multipliers and
bound duals with it.
"""
import numpy as np
import pytest

from oracle import rto
from tests.test_oracle_rto import tracking_instance

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


@pytest.mark.parametrize("name,seed_y,inertia_only", [("tiny30", None, False), ("tiny30", 3, False),
                                                     ("medium1400", None, False), ("tiny30", 3, True),
                                                     ("medium1400", None, True)])
def test_tracking_update_parity(name, seed_y, inertia_only):
    net, on, x, u, s, al, st, pd, qd = tracking_instance(name)
    y = np.zeros(on.m) if seed_y is None else np.random.default_rng(seed_y).uniform(-0.05, 0.05, on.m)
    ref = rto.tracking_update(on, x, u, s, y, st, al, pd=pd, qd=qd, inertia_only=inertia_only)
    ctx = P.OPFContext(net)
    x0, _ = ctx.powerflow(dev(u))  # the state before the load change, as a warm start
    xg, _ = ctx.powerflow(dev(u), pd=dev(pd), qd=dev(qd), x0=x0)
    state = {k: dev(v) for k, v in st.items() if k != "mu"}
    state.update(u=dev(u), s=dev(s), x=xg, mu=st["mu"])
    yg = dev(y)
    info = ctx.tracking_update(dict(sigma_f=al["sigma_f"], rho=al["rho"], sigma_c=dev(al["sigma_c"])), state, yg,
                               inertia_only=inertia_only)
    assert info["qp_iterations"] == ref["iterations"]
    assert info["delta"] == ref["delta"] and info["halvings"] == ref["halvings"]
    assert info["delta_convex"] == ref["delta_convex"]
    assert info["kkt"] <= 1e-6 and abs(state["mu"] - ref["mu"]) <= 1e-12 * ref["mu"]
    assert rel(state["u"].cpu().numpy() - u, ref["u"] - u) < 1e-6
    assert rel(state["s"].cpu().numpy() - s, ref["s"] - s) < 1e-6
    assert rel(state["u"].cpu().numpy(), ref["u"]) < 1e-9
    assert np.abs(state["x"].cpu().numpy() - ref["x"]).max() < 1e-8
    assert rel(yg.cpu().numpy() - y, ref["y"] - y) < 1e-6
    for k, v in ref["duals"].items():
        assert rel(state[k].cpu().numpy(), v) < 1e-5, k
    # the context holds the power flow at the new controls
    g = ctx.reduced_gradient(dict(sigma_f=al["sigma_f"], rho=al["rho"], sigma_c=dev(al["sigma_c"]), y=yg,
                                  s=state["s"]))
    assert torch.isfinite(g["grad_u"]).all()
