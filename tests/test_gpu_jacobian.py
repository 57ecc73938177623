"""GPU parity of the reduced constraint Jacobian J = dc/du (the HVP tiles' by-product, Sec. III-B)
and of the gradient-based scaling built on it (Sec. IV-A, "Scaling").

Tolerances (FP64 on both sides): J 1e-9 relative per column (infinity norm of
the difference over that of the oracle's column), scales 1e-9 relative.  The
oracle's J is one Jacobian-vector product per control (`oracle.scaling`).
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from oracle import scaling
from paper_2110_02590_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts skip the module
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2110_02590_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
JAC_TOL = 1e-9


def col_rel(a, b):
    """Largest per-column relative difference (infinity norms)."""
    den = np.maximum(np.abs(b).max(axis=0), 1e-300)
    return float((np.abs(a - b).max(axis=0) / den).max())


class Case:
    def __init__(self, name):
        self.net = synth.workload(name)
        self.on = oracle.OracleNet(self.net)
        self.ctx = P.OPFContext(self.net)
        self.u = synth.flat_control(self.net)
        self.al = synth.al_inputs(self.net, seed=7)
        self.al_dev = {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
                       for k, v in self.al.items()}
        self.x_orc, info = self.on.powerflow(self.u)
        assert info["rc"] == 0
        self.ctx.powerflow(torch.as_tensor(self.u, device=DEV))


_CASES = {}


def case(name):
    if name not in _CASES:
        _CASES[name] = Case(name)
    return _CASES[name]


@pytest.mark.parametrize("block_k", [1, 2, 4, 8, 16, 32])
def test_jacobian_parity_tiny_all_widths(block_k):
    c = case("tiny30")
    J, H, info = c.ctx.reduced_jacobian(block_k=block_k)
    assert H is None and info["tiles"] == -(-c.on.nu // block_k)
    Jo = scaling.explicit_jacobian(c.on, c.x_orc, c.u)
    assert col_rel(J.cpu().numpy(), Jo) < JAC_TOL


@pytest.mark.parametrize("name,block_k", [("medium1400", 8), ("batchB2000", 16), ("batchA500", 4)])
def test_jacobian_parity_full(name, block_k):
    """Every column of J against the oracle; with the Hessian in the same launch, H is the one
    opf_reduced_hessian gives (bit for bit: the same tiles, J only adds writes), and J does not
    depend on the AL parameters."""
    c = case(name)
    J, H, _ = c.ctx.reduced_jacobian(c.al_dev, hessian=True, block_k=block_k)
    Jn = J.cpu().numpy()
    Jo = scaling.explicit_jacobian(c.on, c.x_orc, c.u)
    assert col_rel(Jn, Jo) < JAC_TOL
    H0, _ = c.ctx.reduced_hessian(c.al_dev, block_k=block_k)
    assert torch.equal(H, H0)
    J2, _, _ = c.ctx.reduced_jacobian(None, block_k=block_k)
    assert torch.equal(J2, J)


def test_jacobian_large_sampled_columns():
    """9.2k-bus grid in the benchmark's launch form (split tiling, with the Hessian): oracle
    columns sampled across tiles, including the ragged end; J alone equals J beside H."""
    c = case("large9200")
    nu = c.on.nu
    J, H, info = c.ctx.reduced_jacobian(c.al_dev, hessian=True, block_k=8)
    assert info["launches"] == 2  # the tiles (J beside H), then the Hessian's mirror
    cols = sorted({0, 1, 7, 8, 9, 100, 1449, 1450, 1451, 2000, nu - 3, nu - 2, nu - 1})
    Jo = scaling.explicit_jacobian(c.on, c.x_orc, c.u, cols=cols)
    Jn = J[:, cols].cpu().numpy()
    assert col_rel(Jn, Jo) < JAC_TOL
    assert bool(torch.isfinite(J).all())
    J2, _, _ = c.ctx.reduced_jacobian(block_k=8)
    assert torch.equal(J2, J)
    H0, _ = c.ctx.reduced_hessian(c.al_dev, block_k=8)
    assert torch.equal(H, H0)


def test_jacobian_column_range_leaves_the_rest():
    c = case("medium1400")
    Jfull, _, _ = c.ctx.reduced_jacobian(block_k=8)
    out = torch.full((c.on.nu, c.on.m), 7.0, dtype=torch.float64, device=DEV)
    J, _, _ = c.ctx.reduced_jacobian(block_k=8, col_begin=100, col_count=37, out=out)
    Jn, Jf = J.cpu().numpy(), Jfull.cpu().numpy()
    assert np.array_equal(Jn[:, 100:137], Jf[:, 100:137])
    assert np.all(np.delete(Jn, np.arange(100, 137), axis=1) == 7.0)


def test_jacobian_gauss_newton_identity():
    """H(omega) - H(0) = J^T diag(omega) J: the GPU Jacobian against two GPU Hessians."""
    c = case("medium1400")
    J, _, _ = c.ctx.reduced_jacobian(block_k=8)
    Jn = J.cpu().numpy()
    om = np.exp(np.linspace(-1.0, 1.0, c.on.m))
    a1 = dict(c.al_dev, omega=torch.as_tensor(om, device=DEV))
    a0 = dict(c.al_dev, omega=torch.zeros(c.on.m, dtype=torch.float64, device=DEV))
    H1, _ = c.ctx.reduced_hessian(a1, block_k=8)
    H0, _ = c.ctx.reduced_hessian(a0, block_k=8)
    ref = Jn.T @ (om[:, None] * Jn)
    diff = (H1 - H0).cpu().numpy()
    assert np.linalg.norm(diff - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("g_max", [1.0, 100.0])
def test_gradient_scaling_parity(g_max):
    c = case("medium1400")
    sig, sf, J = c.ctx.gradient_scaling(g_max=g_max)
    Jo = scaling.explicit_jacobian(c.on, c.x_orc, c.u)
    sig_o, sf_o = scaling.gradient_scaling(Jo, scaling.cost_gradient(c.on, c.x_orc, c.u), g_max=g_max)
    s = sig.cpu().numpy()
    assert np.abs(s - sig_o).max() <= 1e-9 * np.abs(sig_o).max()
    assert abs(sf - sf_o) <= 1e-9 * sf_o
    assert col_rel(J.cpu().numpy(), Jo) < JAC_TOL
    # rows that need no scaling keep exactly 1 on both sides, away from the threshold
    rows = np.abs(Jo).max(axis=1)
    clear = rows < g_max * (1 - 1e-6)
    assert np.all(s[clear] == 1.0)


def test_jacobian_and_scaling_errors():
    net = synth.workload("tiny30")
    ctx = P.OPFContext(net)
    with pytest.raises(P.OPFError) as ei:
        ctx.reduced_jacobian()
    assert ei.value.status == 7  # OPF_ESTATE
    with pytest.raises(P.OPFError) as ei:
        ctx.gradient_scaling()
    assert ei.value.status == 7
    ctx.powerflow(torch.as_tensor(synth.flat_control(net), device=DEV))
    L = P.lib()
    J = torch.empty((ctx.nu, ctx.m), dtype=torch.float64, device=DEV)
    info = P.HessInfo()
    assert L.opf_reduced_jacobian(ctx.h, None, C.byref(P.HessOpts(8, 0, 0, 0, 0, 0, 0, 0, 0)), None, None,
                                  C.byref(info)) == 1  # no J
    assert L.opf_reduced_jacobian(ctx.h, None, C.byref(P.HessOpts(1, 0, 1, 0, 0, 0, 0, 0, 0)),
                                  C.c_void_p(J.data_ptr()), None, C.byref(info)) == 1  # plain form
    H = torch.empty((ctx.nu, ctx.nu), dtype=torch.float64, device=DEV)
    assert L.opf_reduced_jacobian(ctx.h, None, None, C.c_void_p(J.data_ptr()), C.c_void_p(H.data_ptr()),
                                  C.byref(info)) == 1  # H without parameters
    for g_max, s_min in ((0.0, 1e-8), (float("inf"), 1e-8), (100.0, 0.0), (100.0, 2.0)):
        with pytest.raises(P.OPFError) as ei:
            ctx.gradient_scaling(g_max=g_max, s_min=s_min)
        assert ei.value.status == 1
    # the context still answers normally
    J2, _, _ = ctx.reduced_jacobian()
    assert bool(torch.isfinite(J2).all())
