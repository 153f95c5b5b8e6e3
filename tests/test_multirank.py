"""The multi-GPU host path on CPU: two gloo ranks shard the batched domains
(every domain on exactly one rank, DOFs balanced, each share's state and R
equal to the batch's restricted to it) and reduce the timing (slowest rank) and
the work (sum)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2502_19342_gb300 import ranks, workloads as W
    prob, U = W.batched_domains(n_domains=24)
    share, Us, ids = W.shard_domains(prob, U, rank, world)
    # the share's R (oracle) equals the batch's R restricted to its domains
    R_all = oracle.eval_rhs(prob, U)
    slices = W.domain_slices(prob)
    R_share = oracle.eval_rhs(share, Us)
    ok = np.array_equal(R_share, np.concatenate([R_all[slices[d][1]] for d in ids]))
    ms, units = ranks.aggregate(10.0 + rank, 100.0 * (rank + 1), dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, (ids, int(Us.size), bool(ok)))
    if rank == 0:
        out.put((gathered, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_domains_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, ms, units = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids = sorted(i for g in gathered for i in g[0])
    assert ids == list(range(24))
    sizes = [g[1] for g in gathered]
    assert max(sizes) <= 1.6 * min(sizes)
    assert all(g[2] for g in gathered)
    assert ms == 11.0 and units == 300.0
