"""The N > 1 bench path on CPU: two gloo ranks take disjoint batch counters, their draws
together are exactly the single-process draws over the same counters (checked with the
oracle's Philox), and the end-of-run reduction is max(time) / sum(accepted)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2112_15083_gb300 import replicas
    T, steps, seed, b_bits = 64, 3, 11, 22
    t0s = [replicas.batch_t0(rank, k, T) for k in range(steps)]
    js = np.concatenate([oracle.batch_draws(seed, T, b_bits, t0=t0) for t0 in t0s])
    ms, acc = 10.0 + 5.0 * rank, 100 + rank
    red = replicas.reduce_run(ms, acc)
    gathered = [None] * world
    dist.all_gather_object(gathered, (t0s, js.tolist()))
    if rank == 0:
        q.put((red, gathered))
    dist.destroy_process_group()


def test_two_gloo_ranks_disjoint_batches_and_reduction():
    import oracle
    from paper_2112_15083_gb300 import replicas
    oracle.lib()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    red, gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert red == (15.0, 201.0)
    T, steps, seed, b_bits = 64, 3, 11, 22
    ranges = []
    for t0s, js in gathered:
        ranges += [(t0, t0 + T) for t0 in t0s]
        ref = np.concatenate([oracle.batch_draws(seed, T, b_bits, t0=t0) for t0 in t0s])
        assert np.array_equal(np.asarray(js, dtype=ref.dtype), ref)
    ranges.sort()
    assert all(a1 >= b0 for (a0, b0), (a1, b1) in zip(ranges, ranges[1:]))  # disjoint
    assert replicas.batch_t0(1, 0, T) == replicas.RANK_STRIDE
