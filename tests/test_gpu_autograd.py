"""GPU: the autograd objective against central finite differences (step 1e-6,
power flow re-solved) and against the oracle's adjoint gradient."""
import numpy as np
import pytest

import oracle
from paper_2110_02590_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2110_02590_b300 as P  # noqa: E402
from paper_2110_02590_b300.autograd import ReducedObjective  # noqa: E402

DEV = torch.device("cuda", 0)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def make(name, nscen, seed=200, pool=4):
    net = synth.workload(name)
    ctx = P.OPFContext(net)
    al = synth.al_inputs(net, seed=7)
    obj = ReducedObjective(ctx, {k: (dev(v) if isinstance(v, np.ndarray) else v) for k, v in al.items()},
                           pool=pool)
    x0, _ = ctx.powerflow(dev(synth.flat_control(net)))
    obj.set_warm_start(x0)
    pds, qds = synth.ar1_loads(net, nscen, seed=seed)
    u = dev(np.tile(synth.flat_control(net), (nscen, 1)))
    s = dev(np.tile(al["s"], (nscen, 1)))
    return net, ctx, al, obj, u, dev(pds), dev(qds), s


def test_autograd_matches_oracle_gradient():
    """Six scenarios over a pool of four contexts (two workers take two scenarios each)."""
    net, ctx, al, obj, u, pd, qd, s = make("batchB2000", 6)
    for t in (u, pd, qd, s):
        t.requires_grad_(True)
    F = obj(u, pd, qd, s)
    F.sum().backward()
    on = oracle.OracleNet(net)
    for b in range(6):
        xo, io = on.powerflow(u[b].detach().cpu().numpy(), pd=pd[b].detach().cpu().numpy(),
                              qd=qd[b].detach().cpu().numpy())
        assert io["rc"] == 0
        go = on.reduced_gradient(xo, u[b].detach().cpu().numpy(), dict(al, s=s[b].detach().cpu().numpy()),
                                 pd=pd[b].detach().cpu().numpy(), qd=qd[b].detach().cpu().numpy())
        assert abs(F[b].item() - go["F"]) <= 1e-9 * abs(go["F"])
        for mine, ref in ((u.grad[b], go["grad_u"]), (pd.grad[b], go["grad_pd"]), (qd.grad[b], go["grad_qd"]),
                          (s.grad[b], go["grad_s"])):
            ref = np.asarray(ref)
            assert np.abs(mine.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_autograd_central_fd():
    net, ctx, al, obj, u, pd, qd, s = make("batchA500", 1)
    u1, pd1, qd1, s1 = u[0].clone(), pd[0].clone(), qd[0].clone(), s[0].clone()
    for t in (u1, pd1, qd1):
        t.requires_grad_(True)
    F = obj(u1, pd1, qd1, s1)
    F.backward()
    h = 1e-6
    rng = np.random.default_rng(0)
    checks = [("u", u1, j) for j in rng.choice(ctx.nu, 6, replace=False)]
    loaded = np.nonzero(net.pd)[0]
    checks += [("pd", pd1, j) for j in rng.choice(loaded, 4, replace=False)]
    checks += [("qd", qd1, j) for j in rng.choice(loaded, 3, replace=False)] + [("pd", pd1, net.ref_bus)]
    scale = max(u1.grad.abs().max().item(), pd1.grad.abs().max().item())
    with torch.no_grad():
        for name, t, j in checks:
            vals = []
            for sgn in (1.0, -1.0):
                args = {"u": u1.detach().clone(), "pd": pd1.detach().clone(), "qd": qd1.detach().clone()}
                args[name][j] += sgn * h
                vals.append(obj(args["u"], args["pd"], args["qd"], s1).item())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - t.grad[j].item()) <= 2e-6 * scale, (name, j, fd, t.grad[j].item())


def test_autograd_big_grid_single_scenario():
    """The 20,000-bus grid: one scenario, gradient against the oracle."""
    net, ctx, al, obj, u, pd, qd, s = make("big20000", 1, pool=1)
    u1 = u[0].clone().requires_grad_(True)
    F = obj(u1, pd[0], qd[0], s[0])
    F.backward()
    on = oracle.OracleNet(net)
    xo, io = on.powerflow(u[0].cpu().numpy(), pd=pd[0].cpu().numpy(), qd=qd[0].cpu().numpy())
    go = on.reduced_gradient(xo, u[0].cpu().numpy(), dict(al, s=s[0].cpu().numpy()), pd=pd[0].cpu().numpy(),
                             qd=qd[0].cpu().numpy())
    assert np.abs(u1.grad.cpu().numpy() - go["grad_u"]).max() <= 1e-9 * np.abs(go["grad_u"]).max()
