"""Level-merge schedules of the single-right-hand-side solves (opf_set_sweep_merge, opf_sweep_autotune).

A schedule only moves each narrow block's early entries into an earlier chunk,
so every schedule must give the oracle's power flow (same Newton iterations,
state within 1e-9) and reduced gradient (1e-9 relative), and the schedules
agree with one another to rounding.
"""
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
SCHEDULES = [(0, 0), (1, 4), (2, 2), (4, 4), (6, 4), (8, 4), (4, 8), (12, 16)]


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _dev(al):
    return {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v) for k, v in al.items()}


@pytest.mark.parametrize("name", ["medium1400", "batchB2000", "large9200"])
def test_every_schedule_keeps_parity(name):
    net = synth.workload(name)
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    al = synth.al_inputs(net, seed=7)
    x_o, info_o = on.powerflow(u)
    assert info_o["rc"] == 0
    g_o = on.reduced_gradient(x_o, u, al)
    ctx = P.OPFContext(net)
    ud = torch.as_tensor(u, device=DEV)
    ref = None
    for D, W in SCHEDULES:
        ctx.set_sweep_merge(D, W)
        x, info = ctx.powerflow(ud)
        assert info["iterations"] == info_o["iterations"], (D, W)
        xn = x.cpu().numpy()
        assert np.abs(xn - x_o).max() < 1e-9, (D, W)
        g = ctx.reduced_gradient(_dev(al))
        for k in ("grad_u", "grad_s", "lam", "grad_pd", "grad_qd"):
            assert rel_inf(g[k].cpu().numpy(), g_o[k]) < 1e-9, (D, W, k)
        gu = g["grad_u"].cpu().numpy()
        if ref is None:
            ref = (xn, gu)
        else:  # the schedules differ only in the order of the sums
            assert np.abs(xn - ref[0]).max() <= 1e-12, (D, W)
            assert rel_inf(gu, ref[1]) <= 1e-11, (D, W)


def test_schedule_change_with_current_factors_and_autotune():
    """A schedule set while the factors are current re-gathers the factor values into the new
    layout at once; the autotuner leaves one of its candidates in place and the results unchanged."""
    net = synth.workload("large9200")
    ctx = P.OPFContext(net)
    al = _dev(synth.al_inputs(net, seed=3))
    ctx.powerflow(torch.as_tensor(synth.flat_control(net), device=DEV))
    g0 = ctx.reduced_gradient(al)["grad_u"].cpu().numpy()  # factorises the converged state
    ctx.set_sweep_merge(2, 4)
    g1 = ctx.reduced_gradient(al)["grad_u"].cpu().numpy()
    assert rel_inf(g1, g0) <= 1e-11
    d, w, ms = ctx.sweep_autotune()
    assert (d, w) in P.OPFContext.SWEEP_MERGE_CANDIDATES and ms > 0
    g2 = ctx.reduced_gradient(al)["grad_u"].cpu().numpy()
    assert rel_inf(g2, g0) <= 1e-11


def test_schedule_arguments():
    net = synth.workload("tiny30")
    ctx = P.OPFContext(net)
    for D, W in ((-1, 4), (1, 0)):
        with pytest.raises(P.OPFError) as ei:
            ctx.set_sweep_merge(D, W)
        assert ei.value.status == 1  # OPF_EINVAL
    with pytest.raises(P.OPFError) as ei:
        ctx.sweep_autotune()
    assert ei.value.status == 7  # OPF_ESTATE: no power flow yet
