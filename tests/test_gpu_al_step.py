"""GPU parity of the reduced-Newton step (Prop. 3) against the oracle's step.

Tolerance: the step solves S_uu d_u = r with S_uu from the Hessian (parity
~1e-12 relative between the two sides) and cond(S_uu + delta I) below ~1e4 at
these points, so d_u agrees to ~1e-8; the test uses 1e-6 relative (infinity
norm).  The inertia correction, step lengths and halvings must coincide.  The
9.2k-bus case (n_u = 2899, 23 column groups of the Cholesky, so 22 rank-128
trailing updates emulated on the tensor cores) checks the factorisation at
full size, including which inertia corrections fail.
"""
import numpy as np
import pytest

from oracle import al_step as A
from paper_2110_02590_b300 import synth
from tests.test_oracle_al_step import setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2110_02590_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
STEP_TOL = 1e-6


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name,mu,delta_start", [("tiny30", 0.1, 0.0), ("medium1400", 0.1, 0.0),
                                                  ("medium1400", 1e-3, 0.0), ("medium1400", 0.1, 3e4),
                                                  ("large9200", 0.1, 0.0)])
def test_al_step_parity(name, mu, delta_start):
    net = synth.workload(name)
    on, x, u, al, st = setup(net, mu=mu)
    ref = A.al_step(on, x, u, al["s"], st, al, delta_start=delta_start)
    ctx = P.OPFContext(net)
    xg, info = ctx.powerflow(dev(u))
    state = {k: dev(v) for k, v in st.items() if k != "mu"}
    state.update(u=dev(u), s=dev(al["s"]), x=xg, mu=mu)
    al_dev = {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}
    du, ds, inf = ctx.al_step(al_dev, state, delta_start=delta_start)
    assert inf["delta"] == ref["delta"]
    assert rel(du.cpu().numpy(), ref["du"]) < STEP_TOL
    assert rel(ds.cpu().numpy(), ref["ds"]) < STEP_TOL
    assert abs(inf["alpha_p"] - ref["alpha_p"]) <= STEP_TOL * ref["alpha_p"]
    assert abs(inf["alpha_d"] - ref["alpha_d"]) <= STEP_TOL * ref["alpha_d"]
    assert inf["halvings"] == ref["halvings"]
    assert rel(state["u"].cpu().numpy(), ref["u"]) < 1e-9
    assert rel(state["s"].cpu().numpy(), ref["s"]) < 1e-9
    for k, v in ref["duals"].items():
        assert rel(state[k].cpu().numpy(), v) < 1e-6, k
    assert np.abs(state["x"].cpu().numpy() - ref["x"]).max() < 1e-8
    # the new iterate is feasible and the context holds its power flow
    g = ctx.reduced_gradient(dict(al_dev, s=state["s"]))
    assert torch.isfinite(g["grad_u"]).all()


def search_factorisations(t, max_raises=24, carried=False):
    """Factorisations of the library's inertia search when the first succeeding candidate is t:
    in turn from a carried-over delta; from a fresh start delta = 0, then a bisection over
    1 .. max_raises, and the chosen candidate again when the bisection's last probe failed."""
    if carried or t == 0:
        return t + 1
    n, lo, hi, last = 1, 0, max_raises + 1, 0
    while hi - lo > 1:
        mid = lo + (hi - lo) // 2
        n, last = n + 1, mid
        if mid >= t:
            hi = mid
        else:
            lo = mid
    return n + (last != hi)


@pytest.mark.parametrize("mode", [0, 2])
def test_al_step_cholesky_modes(mode):
    """The 9.2k-bus step with FP64 trailing updates (mode 2) and with the FP64 re-check of failed
    pivots (mode 0): the same inertia corrections and step as the oracle's LAPACK-style FP64 step
    (the test above runs the default, emulated updates)."""
    net = synth.workload("large9200")
    on, x, u, al, st = setup(net, mu=0.1)
    ref = A.al_step(on, x, u, al["s"], st, al)
    ctx = P.OPFContext(net)
    ctx.set_cholesky_mode(mode)
    xg, _ = ctx.powerflow(dev(u))
    state = {k: dev(v) for k, v in st.items() if k != "mu"}
    state.update(u=dev(u), s=dev(al["s"]), x=xg, mu=0.1)
    al_dev = {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}
    du, ds, inf = ctx.al_step(al_dev, state)
    assert inf["delta"] == ref["delta"]
    assert rel(du.cpu().numpy(), ref["du"]) < STEP_TOL
    assert rel(ds.cpu().numpy(), ref["ds"]) < STEP_TOL
    # mode 2 factorises in FP64 every time; mode 0 once per failed emulated try (the search
    # factorises at the chosen delta and at some failing ones: at least one of those when delta > 0)
    if mode == 2:
        assert inf["cholesky_fp64"] == inf["factorisations"]
    else:
        assert (inf["inertia_tries"] > 0) <= inf["cholesky_fp64"] <= inf["factorisations"]
    # a fresh start: delta = 0, then a bisection over the other 24 candidates
    assert inf["factorisations"] == search_factorisations(inf["inertia_tries"])
    with pytest.raises(P.OPFError):
        ctx.set_cholesky_mode(3)


def test_al_step_carried_delta():
    """The inertia search from a carried-over delta tries the candidates in turn and reaches the
    same delta as a fresh start: from delta / 100 on the 9.2k grid, two raises, three
    factorisations (the fresh start's bisection took search_factorisations(t) for its t)."""
    net = synth.workload("large9200")
    on, x, u, al, st = setup(net, mu=0.1)
    al_dev = {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}
    out = []
    for start in (0.0, None):
        ctx = P.OPFContext(net)
        xg, _ = ctx.powerflow(dev(u))
        state = {k: dev(v) for k, v in st.items() if k != "mu"}
        state.update(u=dev(u), s=dev(al["s"]), x=xg, mu=0.1)
        d0 = start if start is not None else out[0][0] / 100.0
        du, ds, inf = ctx.al_step(al_dev, state, delta_start=d0)
        out.append((inf["delta"], inf["inertia_tries"], inf["factorisations"], du.cpu().numpy()))
    (d_f, t_f, n_f, du_f), (d_c, t_c, n_c, du_c) = out
    assert d_f > 0.0 and n_f == search_factorisations(t_f) < t_f + 1
    assert abs(d_c - d_f) <= 1e-12 * d_f and t_c == 2 and n_c == 3
    assert rel(du_c, du_f) < 1e-9


@pytest.mark.parametrize("name", ["medium1400", "large9200"])
def test_al_step_update_engines_identical(name):
    """The step with every emulated Cholesky update on tcgen05 and on warp-level mma.sync (the
    default takes tcgen05 for the large updates only).  The two engines produce bit-identical updates (test_gpu_numerics); the rest of a
    step is not bit-reproducible from run to run (scalar reductions use atomics), so the steps
    agree to 1e-12 with the same inertia corrections."""
    net = synth.workload(name)
    on, x, u, al, st = setup(net, mu=0.1)
    al_dev = {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}
    out = []
    for engine in (2, 1):
        ctx = P.OPFContext(net)
        ctx.set_update_engine(engine)
        xg, _ = ctx.powerflow(dev(u))
        state = {k: dev(v) for k, v in st.items() if k != "mu"}
        state.update(u=dev(u), s=dev(al["s"]), x=xg, mu=0.1)
        du, ds, inf = ctx.al_step(al_dev, state)
        out.append((du.cpu().numpy(), ds.cpu().numpy(), inf["delta"], inf["inertia_tries"],
                    state["u"].cpu().numpy()))
    (du0, ds0, d0, t0, u0), (du1, ds1, d1, t1, u1) = out
    assert d0 == d1 and t0 == t1
    assert rel(du0, du1) < 1e-12 and rel(ds0, ds1) < 1e-12 and rel(u0, u1) < 1e-12
    with pytest.raises(P.OPFError):
        P.OPFContext(synth.workload("tiny30")).set_update_engine(3)


def test_al_step_requires_state():
    net = synth.workload("tiny30")
    ctx = P.OPFContext(net)
    on, x, u, al, st = setup(net)
    state = {k: dev(v) for k, v in st.items() if k != "mu"}
    state.update(u=dev(u), s=dev(al["s"]), x=dev(x), mu=0.1)
    with pytest.raises(P.OPFError) as ei:
        ctx.al_step({k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}, state)
    assert ei.value.status == 7
