"""The no-allocation Hessian entry point against the regular one (GPU).

opf_reduced_hessian_noalloc serves callers that cannot allocate device memory
during a call: a real-time loop that must not stall on cudaMalloc (it may
synchronise the device, with unbounded latency), or a process whose
device-memory budget is fixed at start-up.  It uses the library's fixed
32 MiB static workspace instead of a per-context allocation.
These tests call it twice in a row through the C ABI (the second call sees
the first call's leftovers in the shared workspace) and compare each result
with opf_reduced_hessian within the Hessian tolerance of the parity tests.
This file is collected last so a failure here does not hide the other tests.
"""
import numpy as np
import pytest

from paper_2110_02590_b300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2110_02590_b300 as P  # noqa: E402

DEV = torch.device("cuda", 0)
HESS_TOL = 1e-8


def rel_fro(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def full_tiles(nu, C):
    """Tiles of a full Hessian: ceil(nu / C), rounded up to whole waves over the
    SMs when that keeps the tiles at least half full."""
    t = -(-nu // C)
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    if t >= sm:
        tr = -(-t // sm) * sm
        if 2 * nu >= tr * C:
            t = tr
    return t


@pytest.mark.parametrize("name,block_k", [("medium1400", 8), ("large9200", 8), ("large9200", 32)])
def test_noalloc_matches_regular_twice(name, block_k):
    net = synth.workload(name)
    ctx = P.OPFContext(net)
    ctx.powerflow(torch.as_tensor(synth.flat_control(net), device=DEV))
    al = {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
          for k, v in synth.al_inputs(net, seed=7).items()}
    H_ref, _ = ctx.reduced_hessian(al, block_k=block_k)
    H_ref = H_ref.clone()
    out = torch.empty((ctx.nu, ctx.nu), dtype=torch.float64, device=DEV)
    for call in range(2):
        out.fill_(float("nan"))
        H, info = ctx.reduced_hessian_noalloc(al, block_k=block_k, out=out)
        assert info["tiles"] == full_tiles(ctx.nu, block_k)
        assert 1 <= info["grid"] <= info["tiles"]
        assert bool(torch.isfinite(H).all())
        assert rel_fro(H, H_ref) < HESS_TOL, (call, rel_fro(H, H_ref))


SCRATCH_BYTES = 32 * 1024 * 1024  # OPF_NOALLOC_SCRATCH_BYTES


def tile_doubles(ctx, C):
    """Workspace of one tile: (2 n_x + n_ctrl + 1) C doubles rounded up to 32, n_ctrl = n_pv + 1."""
    s = (2 * ctx.nx + ctx.npv + 1 + 1) * C
    return (s + 31) // 32 * 32


def test_noalloc_grid_clamp_large():
    """On the 9.2k-bus grid with 32-wide tiles only a few tiles fit in the array at once: the
    grid is capped there and its CTAs loop over the other tiles, with the same Hessian."""
    net = synth.workload("large9200")
    ctx = P.OPFContext(net)
    ctx.powerflow(torch.as_tensor(synth.flat_control(net), device=DEV))
    al = {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
          for k, v in synth.al_inputs(net, seed=7).items()}
    tiles = full_tiles(ctx.nu, 32)
    fit = SCRATCH_BYTES // (8 * tile_doubles(ctx, 32))
    assert 1 <= fit < tiles
    H_ref, _ = ctx.reduced_hessian(al, block_k=32)
    H_ref = H_ref.clone()
    out = torch.full((ctx.nu, ctx.nu), float("nan"), dtype=torch.float64, device=DEV)
    H, info = ctx.reduced_hessian_noalloc(al, block_k=32, out=out)
    assert info["grid"] == min(tiles, fit)
    assert rel_fro(H, H_ref) < HESS_TOL


def test_noalloc_size_limit():
    """A network whose single 32-wide tile needs more than the static array is rejected with
    OPF_EINVAL (before any state check); 16-wide tiles of the same network fit."""
    net = synth.make_network(n_bus=34000, n_gen=200, n_branch=48000, seed=11, transformer_frac=0.1,
                             load_scale=0.5)
    ctx = P.OPFContext(net)
    assert 8 * tile_doubles(ctx, 32) > SCRATCH_BYTES >= 8 * tile_doubles(ctx, 16)
    al = {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
          for k, v in synth.al_inputs(net, seed=1).items()}
    out = torch.empty((ctx.nu, ctx.nu), dtype=torch.float64, device=DEV)
    with pytest.raises(P.OPFError) as ei:
        ctx.reduced_hessian_noalloc(al, block_k=32, out=out)
    assert ei.value.status == 1 and "static workspace" in str(ei.value)
    with pytest.raises(P.OPFError) as ei:  # fits: the call gets as far as the state check
        ctx.reduced_hessian_noalloc(al, block_k=16, out=out)
    assert ei.value.status == 7


def test_noalloc_rejects_bad_output():
    net = synth.workload("tiny30")
    ctx = P.OPFContext(net)
    ctx.powerflow(torch.as_tensor(synth.flat_control(net), device=DEV))
    al = {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
          for k, v in synth.al_inputs(net, seed=1).items()}
    with pytest.raises(ValueError):
        ctx.reduced_hessian_noalloc(al, out=torch.empty((ctx.nu, ctx.nu - 1), dtype=torch.float64, device=DEV))
    with pytest.raises(ValueError):
        ctx.reduced_hessian_noalloc(al, out=torch.empty((ctx.nu, ctx.nu), dtype=torch.float32, device=DEV))


def test_noalloc_state_error():
    net = synth.workload("tiny30")
    ctx = P.OPFContext(net)
    al = {k: (torch.as_tensor(v, device=DEV) if isinstance(v, np.ndarray) else v)
          for k, v in synth.al_inputs(net, seed=1).items()}
    with pytest.raises(P.OPFError) as ei:
        ctx.reduced_hessian_noalloc(al)
    assert ei.value.status == 7
