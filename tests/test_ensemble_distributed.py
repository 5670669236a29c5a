"""Multi-rank host logic on CPU with the gloo backend (world size 2)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1906_01632_gb300 import ensemble as EN


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _local_moments(cs):
    """Per-rank moments as elder_moments returns them (weights 1/S_r)."""
    return cs.mean(0), ((cs - cs.mean(0)) ** 2).mean(0), (cs > 0.5).mean(0)


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(123)
    allc = rng.uniform(0, 1, (sum(sizes), 57))
    own = EN.shard_even(sum(sizes), world, rank) if sizes[0] == sizes[1] else \
        range(sum(sizes[:rank]), sum(sizes[:rank + 1]))
    cs = allc[list(own)]
    m, v, p = (torch.tensor(a) for a in _local_moments(cs))
    gm, gv, gp = EN.combine_moments(m, v, p, len(own))
    q.put((rank, gm.numpy(), gv.numpy(), gp.numpy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("sizes", [(20, 20), (7, 30)])
def test_combined_moments_equal_global_moments(sizes):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(123)
    allc = rng.uniform(0, 1, (sum(sizes), 57))
    ref = _local_moments(allc)
    for _, gm, gv, gp in res:
        np.testing.assert_allclose(gm, ref[0], rtol=1e-13)
        np.testing.assert_allclose(gv, ref[1], rtol=1e-12)
        np.testing.assert_allclose(gp, ref[2], rtol=1e-13)


def test_shard_even_covers_every_sample_once():
    for total in (0, 1, 7, 256, 257):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in EN.shard_even(total, world, r)]
            assert got == list(range(total))
            sizes = [len(EN.shard_even(total, world, r)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def test_lpt_assign_uneven_batch():
    """48 samples of 1,098,306 unknowns and 16 of 8,586,370 (two grid sizes
    in one ensemble) over 8 ranks: every sample once, and the makespan within
    4/3 of the lower bound max(largest job, total/ranks)."""
    costs = [1098306] * 48 + [8586370] * 16
    for world in (1, 2, 4, 8, 5):
        parts = EN.lpt_assign(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        bound = max(max(costs), sum(costs) / world)
        assert max(loads) <= 4.0 / 3.0 * bound + 1
    # tie-free exact case
    assert EN.lpt_assign([5, 4, 3, 3, 3], 2) == [[0, 3], [1, 2, 4]]


def test_combine_moments_without_process_group_is_identity():
    m = torch.rand(5)
    v = torch.rand(5)
    p = torch.rand(5)
    assert EN.combine_moments(m, v, p, 3) == (m, v, p)
