"""Multi-GPU split of one batch of independent 1D convolutions (no GPU
needed): the longest-processing-time partition of the C ABI
(dc_partition_lpt) is disjoint, covering, deterministic and balanced, and
a world_size-2 gloo run, each rank convolving its own share with the FP64
oracle on the CPU, reproduces the single-process result instance by
instance."""

import itertools
import os
import socket

import numpy as np
import pytest

from paper_1008_1366_gb300 import synthetic


@pytest.fixture(scope="module")
def api():
    from paper_1008_1366_gb300 import api, build
    build.build()
    return api


def cost(m):
    return m * max(1.0, np.log2(m))


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_disjoint_covering_balanced(api, world):
    sizes = [int(x) for x in synthetic.batched_sizes(4096, 1012)]
    owner, load = api.partition_lpt(sizes, world)
    assert len(owner) == len(sizes) and all(0 <= o < world for o in owner)
    # every instance in exactly one share
    shares = [api.shard(sizes, r, world) for r in range(world)]
    assert sorted(itertools.chain.from_iterable(shares)) == list(range(len(sizes)))
    for r in range(world):
        assert abs(load[r] - sum(cost(sizes[i]) for i in shares[r])) <= 1e-9 * max(load)
    # the list-scheduling bound: no rank above the mean by more than one instance
    assert max(load) <= sum(load) / world + max(cost(m) for m in sizes) + 1e-6
    # deterministic
    assert api.partition_lpt(sizes, world) == (owner, load)


def test_partition_within_lpt_bound_of_optimum(api):
    # brute force over every assignment of small batches: LPT's makespan is
    # at most (4/3 - 1/(3p)) times the optimum (Graham's bound)
    rng = np.random.default_rng(3)
    for trial in range(30):
        n = int(rng.integers(1, 9))
        p = int(rng.integers(2, 4))
        sizes = [int(x) for x in rng.choice(synthetic.SIZES_31, n)]
        _, load = api.partition_lpt(sizes, p)
        best = min(max(sum(cost(sizes[i]) for i in range(n) if a[i] == r) for r in range(p))
                   for a in itertools.product(range(p), repeat=n))
        assert max(load) <= (4 / 3 - 1 / (3 * p)) * best + 1e-6, (sizes, p)


def test_partition_edge_cases(api):
    assert api.partition_lpt([], 3) == ([], [0.0, 0.0, 0.0])
    owner, load = api.partition_lpt([64], 4)
    assert owner == [0] and load[0] > 0 and load[1:] == [0.0, 0.0, 0.0]
    with pytest.raises(api.DealiasError):
        api.partition_lpt([64, 0], 2)
    with pytest.raises(api.DealiasError):
        api.partition_lpt([64], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, sizes, seed, q):
    import torch.distributed as dist
    import oracle
    from paper_1008_1366_gb300 import api
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ids = api.shard(sizes, rank, world)
        f, g, off = synthetic.batched_inputs(sizes, seed)
        mine = {i: oracle.conv_complex(f[off[i]:off[i + 1]], g[off[i]:off[i + 1]]) for i in ids}
        gathered = [None] * world
        dist.all_gather_object(gathered, (rank, ids, mine))
        if rank == 0:
            q.put(gathered)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_reproduce_single_process():
    import torch.multiprocessing as mp
    import oracle
    sizes = [int(x) for x in synthetic.batched_sizes(40, 77, sizes=[64, 80, 96, 128, 160, 192, 256, 320, 384, 512])]
    seed = 78
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, sizes, seed, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    seen = {}
    for rank, ids, mine in gathered:
        assert sorted(mine) == ids
        for i in ids:
            assert i not in seen
            seen[i] = mine[i]
    assert sorted(seen) == list(range(len(sizes)))
    f, g, off = synthetic.batched_inputs(sizes, seed)
    for i in range(len(sizes)):
        assert np.array_equal(seen[i], oracle.conv_complex(f[off[i]:off[i + 1]], g[off[i]:off[i + 1]]))
    # both ranks held work
    assert all(len(ids) > 0 for _, ids, _ in gathered)
