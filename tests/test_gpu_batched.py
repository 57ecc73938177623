"""GPU: the batched persistent Hessian launch over snapshots of uneven networks
equals the per-context Hessians (same kernels, same arithmetic per column) and
the oracle."""
import numpy as np
import pytest

import oracle
from paper_2110_02590_b300 import synth

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


def snapshot(name, k):
    net = synth.workload(name)
    pds, qds = synth.ar1_loads(net, k + 1, seed=300)
    ctx = P.OPFContext(net)
    u = synth.flat_control(net)
    ctx.powerflow(dev(u), pd=dev(pds[k]), qd=dev(qds[k]))
    al = synth.al_inputs(net, seed=10 + k)
    if k == 1:
        al["omega"] = np.abs(np.cos(np.arange(ctx.m))) * 3.0
    return dict(net=net, ctx=ctx, u=u, pd=pds[k], qd=qds[k], al=al,
                al_dev={kk: (dev(v) if isinstance(v, np.ndarray) else v) for kk, v in al.items()})


@pytest.mark.parametrize("block_k", [4, 8])
def test_batched_equals_per_context(block_k):
    snaps = [snapshot("batchA500", k) for k in range(3)] + [snapshot("batchB2000", k) for k in range(2)] + \
            [snapshot("tiny30", 0), snapshot("medium1400", 1)]
    Hb, info = P.reduced_hessian_batched([s["ctx"] for s in snaps], [s["al_dev"] for s in snaps], block_k=block_k)
    # one launch for all tiles, then each Hessian's mirror (symmetric form)
    assert info["launches"] == 1 + len(snaps) and info["tiles"] == sum(-(-s["ctx"].nu // block_k) for s in snaps)
    for s, H in zip(snaps, Hb):
        Href, _ = s["ctx"].reduced_hessian(s["al_dev"], block_k=block_k)
        assert float((H - Href).abs().max()) <= 1e-12 * float(Href.abs().max())
    # one snapshot against the oracle
    s = snaps[3]
    on = oracle.OracleNet(s["net"])
    xo, _ = on.powerflow(s["u"], pd=s["pd"], qd=s["qd"])
    Ho = on.reduced_hessian(xo, s["u"], s["al"], omega=s["al"].get("omega"), pd=s["pd"], qd=s["qd"])
    assert np.linalg.norm(Hb[3].cpu().numpy() - Ho) <= 1e-8 * np.linalg.norm(Ho)


def test_batched_rejects_missing_state():
    a = snapshot("tiny30", 0)
    fresh = P.OPFContext(synth.workload("tiny30"))
    with pytest.raises(P.OPFError) as ei:
        P.reduced_hessian_batched([a["ctx"], fresh], [a["al_dev"], a["al_dev"]])
    assert ei.value.status == 7


def test_batched_tracking_steps_match_the_oracle():
    """opf_al_step_batched on snapshots of uneven networks (two 30-bus, one 500-bus, one
    1,400-bus), each at its own AR(1) load snapshot: the power flow at the new loads, then
    the reduced-Newton step with all Schur Hessians in one launch.  Every snapshot's new
    (u, s, x) and step data agree with the oracle's step at those loads, at the tolerances
    of the single-step parity test."""
    from oracle import al_step as A
    from tests.test_oracle_al_step import setup
    snaps = []
    for name, seed in (("tiny30", 11), ("batchA500", 12), ("tiny30", 13), ("medium1400", 14)):
        net = synth.workload(name)
        on, x, u, al, st = setup(net, mu=0.1)
        pds, qds = synth.ar1_loads(net, 2, seed=seed)
        xo, io = on.powerflow(u, pd=pds[1], qd=qds[1], x0=x)
        assert io["rc"] == 0
        ref = A.al_step(on, xo, u, al["s"], st, al, pd=pds[1], qd=qds[1])
        ctx = P.OPFContext(net)
        xg, _ = ctx.powerflow(dev(u))
        state = {k: dev(v) for k, v in st.items() if k != "mu"}
        state.update(u=dev(u), s=dev(al["s"]), x=xg, mu=0.1)
        snaps.append((ctx, {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}, state,
                      (dev(pds[1]), dev(qds[1])), ref))
    infos, stat, binfo = P.al_step_batched([s[0] for s in snaps], [s[1] for s in snaps], [s[2] for s in snaps],
                                           loads=[s[3] for s in snaps])
    assert stat == [0] * len(snaps) and binfo["failed"] == 0
    assert binfo["hessian_tiles"] > 0 and binfo["ms_total"] > 0
    for (ctx, al, state, _, ref), inf in zip(snaps, infos):
        assert inf["delta"] == ref["delta"] and inf["halvings"] == ref["halvings"]
        assert abs(inf["alpha_p"] - ref["alpha_p"]) <= 1e-6 * ref["alpha_p"]
        assert rel(state["u"].cpu().numpy(), ref["u"]) < 1e-9
        assert rel(state["s"].cpu().numpy(), ref["s"]) < 1e-9
        assert np.abs(state["x"].cpu().numpy() - ref["x"]).max() < 1e-8
        for k, v in ref["duals"].items():
            assert rel(state[k].cpu().numpy(), v) < 1e-6, k


def test_batched_steps_report_a_failed_snapshot_and_finish_the_others():
    """A snapshot whose loads are not finite fails its power flow (OPF_ENOCONV); the others
    take their steps and the call returns the failure's status."""
    from tests.test_oracle_al_step import setup
    snaps = []
    for name in ("tiny30", "batchA500"):
        net = synth.workload(name)
        on, x, u, al, st = setup(net, mu=0.1)
        ctx = P.OPFContext(net)
        xg, _ = ctx.powerflow(dev(u))
        state = {k: dev(v) for k, v in st.items() if k != "mu"}
        state.update(u=dev(u), s=dev(al["s"]), x=xg, mu=0.1)
        pd = dev(net.pd)
        if name == "tiny30":
            pd[3] = float("nan")
        snaps.append((ctx, {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()}, state,
                      (pd, dev(net.qd)), u))
    infos, stat, binfo = P.al_step_batched([s[0] for s in snaps], [s[1] for s in snaps], [s[2] for s in snaps],
                                           loads=[s[3] for s in snaps])
    assert stat == [4, 0] and binfo["failed"] == 1
    assert np.array_equal(snaps[0][2]["u"].cpu().numpy(), snaps[0][4])      # kept its state
    assert not np.array_equal(snaps[1][2]["u"].cpu().numpy(), snaps[1][4])  # took its step
