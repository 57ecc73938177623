"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (FP64 on both sides): power-flow state 1e-9 absolute, reduced
gradient 1e-9 relative (infinity norm of the difference over that of the
oracle), reduced Hessian 1e-8 relative Frobenius norm.  Each side solves its
own power flow from the same start; no value crosses from the GPU to the
oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2110_02590_b300 import synth
from tests.netutil import custom_network, with_costs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts skip the module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2110_02590_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
GRAD_TOL = 1e-9
HESS_TOL = 1e-8


def rel_inf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Case:
    """One network solved on both sides at the base-case controls."""

    def __init__(self, net, al_seed=7, omega=None):
        self.net = net
        self.on = oracle.OracleNet(net)
        self.ctx = P.OPFContext(net)
        self.u = synth.flat_control(net)
        self.al = synth.al_inputs(net, seed=al_seed)
        if omega is not None:
            self.al["omega"] = omega
        self.x_orc, self.pf_orc = self.on.powerflow(self.u)
        assert self.pf_orc["rc"] == 0
        self.solve_gpu()
        self.al_dev = {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
                       for k, v in self.al.items()}

    def solve_gpu(self):
        x, info = self.ctx.powerflow(torch.as_tensor(self.u, device=DEV))
        self.x_gpu, self.pf_gpu = x.cpu().numpy(), info


_CASES = {}


def case(name, **kw):
    key = (name, tuple(sorted(kw)))
    if key not in _CASES:
        _CASES[key] = Case(synth.workload(name), **kw)
    return _CASES[key]


# ---------------------------------------------------------------- symbolic

@pytest.mark.parametrize("name", ["tiny30", "medium1400"])
def test_context_symbolic_equals_oracle(name):
    c = case(name)
    a = c.ctx.symbolic()
    b = c.on.symbolic()
    for k in ("bus_order", "perm", "rowptr", "colidx", "lev_f", "lev_b"):
        assert np.array_equal(a[k], b[k]), k


# ---------------------------------------------------------------- power flow

@pytest.mark.parametrize("name", ["tiny30", "medium1400", "batchA500", "batchB2000", "large9200"])
def test_powerflow_parity(name):
    c = case(name)
    assert c.pf_gpu["status"] == 0
    assert c.pf_gpu["res2"] < 1e-10
    assert c.pf_gpu["iterations"] == c.pf_orc["iterations"]
    assert np.abs(c.x_gpu - c.x_orc).max() < 1e-9


def test_powerflow_warm_start_and_loads():
    c = case("medium1400")
    pds, qds = synth.ar1_loads(c.net, 2, seed=101)
    x0 = torch.as_tensor(c.x_gpu, device=DEV)
    x, info = c.ctx.powerflow(torch.as_tensor(c.u, device=DEV), pd=torch.as_tensor(pds[1], device=DEV),
                              qd=torch.as_tensor(qds[1], device=DEV), x0=x0)
    xo, io = c.on.powerflow(c.u, pd=pds[1], qd=qds[1], x0=c.x_orc)
    assert info["status"] == 0 and io["rc"] == 0
    assert np.abs(x.cpu().numpy() - xo).max() < 1e-9
    c.solve_gpu()  # restore the base-case state for the other tests


# ---------------------------------------------------------------- gradient

@pytest.mark.parametrize("name", ["tiny30", "medium1400", "batchA500", "large9200"])
def test_reduced_gradient_parity(name):
    c = case(name)
    g = c.ctx.reduced_gradient(c.al_dev)
    o = c.on.reduced_gradient(c.x_orc, c.u, c.al)
    assert rel_inf(g["grad_u"].cpu().numpy(), o["grad_u"]) < GRAD_TOL
    assert rel_inf(g["grad_s"].cpu().numpy(), o["grad_s"]) < GRAD_TOL
    assert rel_inf(g["c"].cpu().numpy(), o["c"]) < GRAD_TOL
    assert rel_inf(g["lam"].cpu().numpy(), o["lam"]) < GRAD_TOL
    assert rel_inf(g["grad_pd"].cpu().numpy(), o["grad_pd"]) < GRAD_TOL
    assert rel_inf(g["grad_qd"].cpu().numpy(), o["grad_qd"]) < GRAD_TOL
    assert abs(g["F"].item() - o["F"]) <= GRAD_TOL * abs(o["F"])


# ---------------------------------------------------------------- Hessian

@pytest.mark.parametrize("block_k", [1, 2, 4, 8, 16, 32])
def test_hessian_parity_tiny_all_tiles(block_k):
    c = case("tiny30")
    H, info = c.ctx.reduced_hessian(c.al_dev, block_k=block_k)
    Ho = c.on.reduced_hessian(c.x_orc, c.u, c.al)
    assert rel_fro(H.cpu().numpy(), Ho) < HESS_TOL
    assert info["tiles"] == -(-c.on.nu // block_k)


def test_hessian_plain_equals_batched():
    """The plain form (one direction per launch sequence: device-wide kernels around two
    streamed single-RHS solves, 9 kernels per column) against the oracle and the tiles."""
    c = case("tiny30")
    Hp, ip = c.ctx.reduced_hessian(c.al_dev, block_k=1, plain=True)
    Hb, _ = c.ctx.reduced_hessian(c.al_dev, block_k=8)
    Ho = c.on.reduced_hessian(c.x_orc, c.u, c.al)
    assert ip["launches"] == 9 * c.on.nu and ip["block_k"] == 1 and ip["tiles"] == c.on.nu
    assert rel_fro(Hp.cpu().numpy(), Ho) < HESS_TOL
    assert rel_fro(Hp.cpu().numpy(), Hb.cpu().numpy()) < 1e-12


@pytest.mark.parametrize("name,col0,ncol", [("medium1400", 0, 40), ("large9200", 1500, 24)])
def test_hessian_plain_columns_match_tiles(name, col0, ncol):
    """Plain-form columns on the larger grids (the streamed solves, the dense trailing
    triangles and the PV/slack cases of the gathers) equal the tiled Hessian's; the other
    columns of the output are left untouched."""
    c = case(name)
    Hb, _ = c.ctx.reduced_hessian(c.al_dev, block_k=8)
    Hb = Hb.cpu().numpy()
    out = torch.full((c.ctx.nu, c.ctx.nu), 7.0, dtype=torch.float64, device=DEV)
    Hp, ip = c.ctx.reduced_hessian(c.al_dev, plain=True, col_begin=col0, col_count=ncol, out=out)
    Hp = Hp.cpu().numpy()
    cols = slice(col0, col0 + ncol)
    assert rel_fro(Hp[:, cols], Hb[:, cols]) < 1e-11
    assert np.all(np.delete(Hp, np.arange(col0, col0 + ncol), axis=1) == 7.0)


@pytest.mark.parametrize("name,block_k,grid", [("medium1400", 8, 0), ("medium1400", 16, 37),
                                               ("medium1400", 32, 0), ("batchA500", 4, 0),
                                               ("batchB2000", 8, 0)])
def test_hessian_parity_full(name, block_k, grid):
    c = case(name)
    H, info = c.ctx.reduced_hessian(c.al_dev, block_k=block_k, grid=grid)
    Ho = c.on.reduced_hessian(c.x_orc, c.u, c.al)
    Hn = H.cpu().numpy()
    assert rel_fro(Hn, Ho) < HESS_TOL
    assert np.linalg.norm(Hn - Hn.T) <= 1e-10 * np.linalg.norm(Hn)


def test_hessian_large_sampled_columns():
    """Full 9.2k-bus Hessian in the benchmark configuration; oracle columns sampled
    across tiles, including the ragged last tile."""
    c = case("large9200")
    H, info = c.ctx.reduced_hessian(c.al_dev, block_k=8)
    nu = c.on.nu
    cols = sorted({0, 1, 7, 8, 9, 100, 1449, 1450, 1451, 2000, nu - 3, nu - 2, nu - 1})
    Ho = c.on.reduced_hessian(c.x_orc, c.u, c.al, cols=cols)
    Hn = H.cpu().numpy()[:, cols]
    assert rel_fro(Hn, Ho) < HESS_TOL
    full = H.cpu().numpy()
    assert np.isfinite(full).all()
    assert np.linalg.norm(full - full.T) <= 1e-10 * np.linalg.norm(full)


@pytest.mark.parametrize("name,block_k", [("tiny30", 4), ("medium1400", 8), ("batchB2000", 16), ("large9200", 8)])
def test_hessian_by_symmetry_equals_full(name, block_k):
    """The full Hessian by its symmetry (the default: a tile keeps the rows of the controls
    from its first column position on, its L^T sweep pruned to their Psi rows, and a mirror
    kernel completes H) against every column computed in full: each entry is one of the two
    computed values of its symmetric pair, so the two agree to rounding; and both match the
    oracle."""
    c = case(name)
    Hs, info_s = c.ctx.reduced_hessian(c.al_dev, block_k=block_k)
    Hs = Hs.cpu().numpy().copy()
    c.ctx.set_hessian_symmetry(False)
    try:
        Hf, info_f = c.ctx.reduced_hessian(c.al_dev, block_k=block_k)
    finally:
        c.ctx.set_hessian_symmetry(True)
    Hf = Hf.cpu().numpy()
    assert info_s["launches"] == info_f["launches"] + 1
    # pairs inside a tile's own columns are both computed (equal to rounding); the rest mirrored
    assert np.linalg.norm(Hs - Hs.T) <= 1e-13 * np.linalg.norm(Hs)
    assert np.isfinite(Hs).all()
    scale = np.abs(Hf).max()
    assert np.minimum(np.abs(Hs - Hf), np.abs(Hs - Hf.T)).max() <= 1e-12 * scale
    assert rel_fro(Hs, Hf) < 1e-12
    if name != "large9200":
        Ho = c.on.reduced_hessian(c.x_orc, c.u, c.al)
        assert rel_fro(Hs, Ho) < HESS_TOL


def test_hessian_custom_omega():
    """Second-order weights of the Schur complement (Prop. 3) go through the same kernels."""
    net = synth.workload("medium1400")
    om = np.abs(np.sin(np.arange(synth.constraint_count(net)))) * 5.0
    c = case("medium1400", omega=om)
    H, _ = c.ctx.reduced_hessian(c.al_dev, block_k=8)
    Ho = c.on.reduced_hessian(c.x_orc, c.u, c.al, omega=om)
    assert rel_fro(H.cpu().numpy(), Ho) < HESS_TOL


def test_special_case_diagonal_hessian():
    base = synth.workload("tiny30")
    c2 = base.gen_c2.copy()
    c1 = base.gen_c1.copy()
    c2[0] = c1[0] = 0.0
    net = with_costs(base, c2, c1)
    cs = Case(net)
    cs.al_dev["y"] = torch.zeros(cs.on.m, dtype=torch.float64, device=DEV)
    cs.al_dev["rho"] = 0.0
    g = cs.ctx.reduced_gradient(cs.al_dev)
    assert float(g["lam"].abs().max()) == 0.0
    H, _ = cs.ctx.reduced_hessian(cs.al_dev, block_k=4)
    npv = cs.on.npv
    Hn = H.cpu().numpy()
    off = Hn.copy()
    off[1 + npv:, 1 + npv:] -= np.diag(np.diag(Hn)[1 + npv:])
    assert np.abs(off).max() <= 1e-14 * np.abs(Hn).max()


@pytest.mark.parametrize("kind", ["two_bus", "parallel"])
def test_degenerate_networks(kind):
    if kind == "two_bus":
        net = custom_network(2, [(0, 1, 0.02, 0.08, 0.0, 1.0)], gen_bus=[0], pd=[0, 0.8], qd=[0, 0.3])
    else:
        net = custom_network(4, [(0, 1, 0.01, 0.05, 0.01, 1.0), (1, 2, 0.01, 0.04, 0.0, 1.0),
                                 (1, 2, 0.02, 0.06, 0.0, 1.0), (2, 3, 0.01, 0.05, 0.02, 0.98)],
                             gen_bus=[0, 3], pd=[0, 0.5, 0.4, 0.1], qd=[0, 0.1, 0.1, 0.0])
    cs = Case(net)
    assert np.abs(cs.x_gpu - cs.x_orc).max() < 1e-10
    g = cs.ctx.reduced_gradient(cs.al_dev)
    o = cs.on.reduced_gradient(cs.x_orc, cs.u, cs.al)
    assert rel_inf(g["grad_u"].cpu().numpy(), o["grad_u"]) < GRAD_TOL
    H, _ = cs.ctx.reduced_hessian(cs.al_dev, block_k=2)
    assert rel_fro(H.cpu().numpy(), cs.on.bruteforce(cs.x_orc, cs.u, cs.al)["H"]) < HESS_TOL


# ---------------------------------------------------------------- errors

def test_state_and_argument_errors():
    ctx = P.OPFContext(synth.workload("tiny30"))
    al = {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
          for k, v in synth.al_inputs(synth.workload("tiny30"), seed=1).items()}
    with pytest.raises(P.OPFError) as ei:
        ctx.reduced_gradient(al)
    assert ei.value.status == 7  # OPF_ESTATE
    ctx.powerflow(torch.as_tensor(synth.flat_control(synth.workload("tiny30")), device=DEV))
    with pytest.raises(P.OPFError) as ei:
        ctx.reduced_hessian(al, block_k=3)
    assert ei.value.status == 1  # OPF_EINVAL


def test_nonconvergent_powerflow_reports_status():
    """Loads x20 have no power-flow solution: Newton-Raphson must stop with a status, not fault."""
    net = synth.workload("tiny30")
    ctx = P.OPFContext(net)
    u = torch.as_tensor(synth.flat_control(net), device=DEV)
    x, info = ctx.powerflow(u, pd=torch.as_tensor(net.pd * 20, device=DEV),
                            qd=torch.as_tensor(net.qd * 20, device=DEV), check=False)
    assert info["status"] in (4, 5)  # OPF_ENOCONV or OPF_ESINGULAR
    with pytest.raises(P.OPFError):
        ctx.reduced_gradient({k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
                              for k, v in synth.al_inputs(net, seed=1).items()})
    # the context recovers with a feasible solve
    x, info = ctx.powerflow(u)
    assert info["status"] == 0


def test_hessian_large_launch_forms_agree():
    """The 9.2k-bus Hessian by every launch form: the split tiling (default: waves
    of 8-wide tiles plus one 4-wide tile per SM), the balanced form (explicit grid),
    512-thread tiles, 4-wide tiles and column ranges in natural order; each tile
    computes its columns independently, so all agree to rounding."""
    c = case("large9200")
    nu = c.on.nu
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    H0, i0 = c.ctx.reduced_hessian(c.al_dev, block_k=8)
    waves = nu // (8 * sm)
    rem = nu - waves * sm * 8
    if waves >= 1 and 0 < rem and -(-rem // 4) <= sm:
        assert i0["tiles"] == waves * sm + -(-rem // 4) and i0["launches"] == 2  # tiles, then the mirror
    H0 = H0.cpu().numpy()
    ref = np.linalg.norm(H0)
    for kw in (dict(block_k=8, grid=sm), dict(block_k=8, threads=512), dict(block_k=4)):
        H, _ = c.ctx.reduced_hessian(c.al_dev, **kw)
        assert np.linalg.norm(H.cpu().numpy() - H0) <= 1e-12 * ref, kw
    pieces = np.zeros_like(H0)
    for a, b in ((0, 1000), (1000, 1001), (1001, nu)):
        Hp, _ = c.ctx.reduced_hessian(c.al_dev, block_k=8, col_begin=a, col_count=b - a)
        pieces[:, a:b] = Hp.cpu().numpy()[:, a:b]
    assert np.linalg.norm(pieces - H0) <= 1e-12 * ref
