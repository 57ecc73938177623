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
    assert info["launches"] == 1 and info["tiles"] == sum(-(-s["ctx"].nu // block_k) for s in snaps)
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
