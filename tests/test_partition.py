"""The multi-GPU partitions on CPU: LPT assignment of uneven snapshots, the column
ranges of a split Hessian, and the all-gather that reassembles it, over two and
three gloo ranks.  The columns come from the CPU oracle (each rank computes its
own range), so the reassembled matrix is compared with the oracle's one-rank
Hessian; no GPU is involved."""
import os
import socket
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2110_02590_b300 import partition  # noqa: E402


def test_lpt_assignment_by_hand():
    """Items by descending cost: 7 -> r0 (all empty, lowest rank); 5 -> r1; 4 -> r2; 4 -> r2
    (load 4 is the smallest); 3 -> r1 (5); 2 -> r0 (7); 2 -> r1 (r1 and r2 at 8, lowest rank)."""
    costs = [7, 5, 4, 4, 3, 2, 2]
    parts, loads = partition.lpt_assign(costs, 3)
    assert parts == [[0, 5], [1, 4, 6], [2, 3]]
    assert loads == [9.0, 10.0, 8.0]


def test_lpt_config3_batch_balances_within_the_largest_item():
    # the config-3 batch: 16 x 9.2k, 64 x 2k, 128 x 500 buses, cost ~ n_x nnz(LU) n_u
    costs = [16949 * 337123 * 2899] * 16 + [3699 * 43385 * 599] * 64 + [909 * 9143 * 179] * 128
    for nranks in (2, 3, 4, 8):
        parts, loads = partition.lpt_assign(costs, nranks)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        assert max(loads) - min(loads) <= max(costs)
        assert max(loads) <= sum(costs) / nranks + max(costs)


@pytest.mark.parametrize("nu,nranks,k", [(2899, 2, 8), (2899, 8, 8), (11, 3, 4), (519, 4, 32), (5, 4, 8)])
def test_column_ranges_cover_once_in_whole_tiles(nu, nranks, k):
    r = partition.column_ranges(nu, nranks, k)
    assert len(r) == nranks and r[0][0] == 0 and r[-1][1] == nu
    for (b0, e0), (b1, e1) in zip(r, r[1:]):
        assert e0 == b1
    tiles = [-(-(e - b) // k) for b, e in r]
    assert max(tiles) - min(tiles) <= 1 or sum(tiles) < nranks
    assert all(b % k == 0 for b, _ in r if b < nu)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2110_02590_b300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net = synth.workload("tiny30")
        on = oracle.OracleNet(net)
        u = synth.flat_control(net)
        x, _ = on.powerflow(u)  # every rank solves the power flow (replicas)
        al = synth.al_inputs(net, seed=7)

        def cols(b, n):
            return torch.as_tensor(on.reduced_hessian(x, u, al, cols=np.arange(b, b + n)).T.copy())

        H = partition.sharded_hessian(cols, on.nu, block_k=4)
        np.save(os.path.join(out_dir, f"H{rank}.npy"), H.numpy().T)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_hessian_equals_one_rank(tmp_path, world):
    import torch.multiprocessing as mp
    import oracle
    from paper_2110_02590_b300 import synth
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn",
                       join=True)
    net = synth.workload("tiny30")
    on = oracle.OracleNet(net)
    u = synth.flat_control(net)
    x, _ = on.powerflow(u)
    H1 = on.reduced_hessian(x, u, synth.al_inputs(net, seed=7))
    for r in range(world):
        Hr = np.load(os.path.join(tmp_path, f"H{r}.npy"))
        assert np.array_equal(Hr, H1), r
