"""Failure paths of the C ABI on the GPU, made on the host or by bounded waits.

No test faults, traps or hangs the GPU: a non-finite load, a state whose
Jacobian has exactly zero pivots and an indefinite Schur complement with too
few inertia corrections are ordinary inputs that the library must reject
with a status; the timeouts come from a spin limit of one poll
(opf_set_wait_limit), so a bounded wait gives up, records it and lets its
kernel finish.  After each failure the same context must still give the
normal result.
"""
import numpy as np
import pytest

from paper_2110_02590_b300 import synth
from tests.test_oracle_al_step import setup

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2110_02590_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
ENOCONV, ESINGULAR, ENOTPD, ESTATE, ETIMEOUT = 4, 5, 6, 7, 8


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def al_dev(al):
    return {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}


def test_nan_load_is_enoconv_and_context_recovers():
    net = synth.workload("medium1400")
    ctx = P.OPFContext(net)
    u = dev(synth.flat_control(net))
    pd = dev(net.pd)
    pd[7] = float("nan")
    _, info = ctx.powerflow(u, pd=pd, check=False)
    assert info["status"] == ENOCONV
    with pytest.raises(P.OPFError) as ei:  # no state after a failed power flow
        ctx.reduced_gradient(al_dev(synth.al_inputs(net, seed=7)))
    assert ei.value.status == ESTATE
    x, info = ctx.powerflow(u)
    assert info["status"] == 0 and info["res2"] < 1e-10


def test_zero_pivot_is_esingular_and_context_recovers():
    """At |V| = 0 on every PQ bus the injections do not depend on the PQ angles: the
    Jacobian's theta columns of those buses are zero and the refactorisation meets zero
    pivots (the library checks each pivot for zero or non-finite values)."""
    net = synth.workload("medium1400")
    ctx = P.OPFContext(net)
    u = dev(synth.flat_control(net))
    x0 = dev(synth.flat_state(net))
    x0[ctx.npv + ctx.npq:] = 0.0
    _, info = ctx.powerflow(u, x0=x0, check=False)
    assert info["status"] == ESINGULAR
    x, info = ctx.powerflow(u)
    assert info["status"] == 0 and info["res2"] < 1e-10


def step_state(net, mu=0.1):
    on, x, u, al, st = setup(net, mu=mu)
    state = {k: dev(v) for k, v in st.items() if k != "mu"}
    state.update(u=dev(u), s=dev(al["s"]), mu=mu)
    return u, al, state


def test_indefinite_schur_with_one_correction_is_enotpd():
    net = synth.workload("medium1400")
    u, al, state = step_state(net)
    ctx = P.OPFContext(net)
    # the step at this point needs an inertia correction above 1e-8
    probe = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in state.items()}
    probe["x"], _ = ctx.powerflow(dev(u))
    _, _, inf = ctx.al_step(al_dev(al), probe)
    assert inf["delta"] > 1e-8
    state["x"], _ = ctx.powerflow(dev(u))
    before = {k: v.clone() for k, v in state.items() if torch.is_tensor(v)}
    with pytest.raises(P.OPFError) as ei:
        ctx.al_step(al_dev(al), state, max_inertia=1)
    assert ei.value.status == ENOTPD
    for k, v in before.items():  # the state is left as it was
        assert torch.equal(state[k], v), k
    _, _, inf2 = ctx.al_step(al_dev(al), state)
    assert inf2["delta"] == inf["delta"]
    assert torch.allclose(state["u"], probe["u"], rtol=0, atol=1e-12)


def test_dense_solve_wait_limit_is_etimeout_and_context_recovers():
    """With a limit of one poll, the blocks of the dense triangular solve that wait for
    their predecessors give up: the step returns OPF_ETIMEOUT without touching the state;
    with the default limit the same context takes the normal step."""
    net = synth.workload("medium1400")
    u, al, state = step_state(net)
    ctx = P.OPFContext(net)
    probe = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in state.items()}
    probe["x"], _ = ctx.powerflow(dev(u))
    ctx.al_step(al_dev(al), probe)
    state["x"], _ = ctx.powerflow(dev(u))
    ctx.reduced_gradient(dict(al_dev(al), s=state["s"]))  # factors ready: the wait limit hits the solves
    before = {k: v.clone() for k, v in state.items() if torch.is_tensor(v)}
    ctx.set_wait_limit(1)
    try:
        with pytest.raises(P.OPFError) as ei:
            ctx.al_step(al_dev(al), state)
        assert ei.value.status == ETIMEOUT
    finally:
        ctx.set_wait_limit(0)
    for k, v in before.items():
        assert torch.equal(state[k], v), k
    ctx.al_step(al_dev(al), state)
    assert torch.allclose(state["u"], probe["u"], rtol=0, atol=1e-12)
    assert torch.allclose(state["s"], probe["s"], rtol=0, atol=1e-12)


def test_tcgen05_update_wait_limit_is_etimeout_and_context_recovers():
    """The tcgen05 emulated Cholesky update waits on mbarriers for its bulk copies and MMAs;
    with a one-poll limit those waits give up, the kernel drains what it issued, frees its
    tensor memory and the step returns OPF_ETIMEOUT with the state untouched.  The same
    context then takes the normal step (the factorisation graph re-captured with the default
    limit) and the later tcgen05 launches allocate their tensor memory again."""
    net = synth.workload("medium1400")
    u, al, state = step_state(net)
    ctx = P.OPFContext(net)
    ctx.set_update_engine(2)  # every emulated update on tcgen05 (the default keeps small ones on mma.sync)
    probe = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in state.items()}
    probe["x"], _ = ctx.powerflow(dev(u))
    ctx.al_step(al_dev(al), probe)
    state["x"], _ = ctx.powerflow(dev(u))
    ctx.reduced_gradient(dict(al_dev(al), s=state["s"]))  # factors ready: the limit hits the step's waits
    before = {k: v.clone() for k, v in state.items() if torch.is_tensor(v)}
    ctx.set_wait_limit(1)
    try:
        with pytest.raises(P.OPFError) as ei:
            ctx.al_step(al_dev(al), state)
        assert ei.value.status == ETIMEOUT and "tensor cores" in str(ei.value)
    finally:
        ctx.set_wait_limit(0)
    for k, v in before.items():
        assert torch.equal(state[k], v), k
    ctx.al_step(al_dev(al), state)
    assert torch.allclose(state["u"], probe["u"], rtol=0, atol=1e-12)
    assert torch.allclose(state["s"], probe["s"], rtol=0, atol=1e-12)


def test_cluster_lu_wait_limit_is_etimeout_and_context_recovers():
    """The dense trailing block of the LU runs on a thread-block cluster whose CTAs poll
    per-step flags in shared memory; with a one-poll limit they give up (every CTA still
    reaches the cluster's final barrier) and the power flow returns OPF_ETIMEOUT."""
    net = synth.workload("medium1400")
    ctx = P.OPFContext(net)
    u = dev(synth.flat_control(net))
    ctx.set_wait_limit(1)
    try:
        _, info = ctx.powerflow(u, check=False)
    finally:
        ctx.set_wait_limit(0)
    assert info["status"] == ETIMEOUT
    x, info = ctx.powerflow(u)
    assert info["status"] == 0 and info["res2"] < 1e-10


def test_hessian_asymmetry_report():
    net = synth.workload("medium1400")
    ctx = P.OPFContext(net)
    ctx.powerflow(dev(synth.flat_control(net)))
    H, info = ctx.reduced_hessian(al_dev(synth.al_inputs(net, seed=7)), asymmetry=True)
    h = H.cpu().numpy()
    ref = np.linalg.norm(h - h.T) / np.linalg.norm(h)
    assert 0.0 <= info["asymmetry"] < 1e-10
    assert abs(info["asymmetry"] - ref) <= 1e-6 * max(ref, 1e-300) + 1e-18
    _, info = ctx.reduced_hessian(al_dev(synth.al_inputs(net, seed=7)))
    assert info["asymmetry"] == -1.0
