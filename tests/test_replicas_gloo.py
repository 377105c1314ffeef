"""The replica path on CPU ranks (gloo, world size 2): each rank evaluates its
slice of the Lambda batch (with the oracle standing in for the GPU library), the
slices gather back to the unsharded result bit for bit, and the timing max and
barrier behave as the benchmark uses them."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import oracle
    from paper_1904_02863_gb300 import replicas, synth
    r, local, w = replicas.init_from_env()
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    cat = synth.make_catalog(3, 40, 6, seed=31)
    inj = synth.make_injections(3000, 6, seed=32)
    K = 11
    lam = synth.make_lambdas(K, 11, seed=33)
    a, b = replicas.shard(K, r, w)
    mine = oracle.loglik(cat, inj, lam[a:b], nthreads=1)[0]
    full = replicas.gather_rows(mine, K, w)
    slowest = replicas.max_over_ranks(float(rank + 1), w)
    replicas.barrier(w)
    if rank == 0:
        np.savez(out_path, full=full, slowest=slowest)
    dist.destroy_process_group()


def test_replicas_on_two_cpu_ranks(tmp_path, oracle):
    import torch.multiprocessing as mp

    from paper_1904_02863_gb300 import synth
    out = str(tmp_path / "res.npz")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = np.load(out)
    cat = synth.make_catalog(3, 40, 6, seed=31)
    inj = synth.make_injections(3000, 6, seed=32)
    ref = oracle.loglik(cat, inj, synth.make_lambdas(11, 11, seed=33), nthreads=1)[0]
    np.testing.assert_array_equal(res["full"], ref)
    assert float(res["slowest"]) == 2.0


@pytest.mark.parametrize("K,world", [(1024, 1), (1024, 8), (11, 2), (3, 4), (0, 3)])
def test_shards_cover_the_batch_once(K, world):
    from paper_1904_02863_gb300 import replicas
    cuts = [replicas.shard(K, r, world) for r in range(world)]
    assert cuts[0][0] == 0 and cuts[-1][1] == K
    assert all(cuts[i][1] == cuts[i + 1][0] for i in range(world - 1))
    sizes = [b - a for a, b in cuts]
    assert max(sizes) - min(sizes) <= 1
