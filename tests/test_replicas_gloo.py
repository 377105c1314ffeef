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


def _partition_case():
    from paper_1904_02863_gb300 import synth
    cat = synth.make_catalog(7, np.array([30, 5, 60, 1, 44, 17, 90]), 6, seed=41)
    inj = synth.make_injections(4000, 6, seed=42)
    lam = synth.make_lambdas(9, 11, seed=43)
    lam[2, 6] = -1.0                    # invalid
    lam[3, 2], lam[3, 3] = 4.0, 5.2     # mass range below most samples: zero events
    return cat, inj, lam


def _partition_worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import oracle
    from paper_1904_02863_gb300 import replicas
    r, _, w = replicas.init_from_env()
    cat, inj, lam = _partition_case()
    e0, e1 = replicas.event_range(cat.offsets, r, w)
    ev, sw, sw2, fl = oracle.loglik_parts(replicas.sub_catalog(cat, e0, e1), replicas.sub_injections(inj, r, w),
                                          lam, nthreads=1)
    tot = replicas.all_reduce_sum(np.stack([ev, sw, sw2]), w)
    res = replicas.combine_parts(tot[0], tot[1], tot[2], cat.n_events, inj.n_draw, (fl & 1) != 0)
    if rank == 0:
        np.savez(out_path, lnL=res[0], lnxi=res[1], neff=res[2], flags=res[3])
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_event_partition_on_cpu_ranks(tmp_path, oracle, world):
    """Events split by CSR ranges and injections by shares over gloo ranks; one all-reduce of the
    parts reproduces the unsharded ln L, ln xi, N_eff and flags (1e-13 relative)."""
    import torch.multiprocessing as mp
    out = str(tmp_path / "part.npz")
    mp.spawn(_partition_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    res = np.load(out)
    cat, inj, lam = _partition_case()
    lnL, lnxi, neff, flags = oracle.loglik(cat, inj, lam, nthreads=1)
    np.testing.assert_array_equal(res["flags"], flags)
    assert flags[2] == 1 and flags[3] & 2
    fin = np.isfinite(lnL)
    np.testing.assert_array_equal(np.isfinite(res["lnL"]), fin)
    scale = np.abs(lnL[fin] + cat.n_events * lnxi[fin]) + cat.n_events * np.abs(lnxi[fin])
    assert (np.abs(res["lnL"][fin] - lnL[fin]) <= 1e-13 * scale).all()
    np.testing.assert_allclose(res["lnxi"], lnxi, rtol=1e-13, atol=0)
    np.testing.assert_allclose(res["neff"], neff, rtol=1e-12)


def test_combine_of_the_whole_set_is_the_oracle(oracle):
    """One part holding everything: combine_parts gives the oracle's ln L bit for bit."""
    from paper_1904_02863_gb300 import replicas
    cat, inj, lam = _partition_case()
    ev, sw, sw2, fl = oracle.loglik_parts(cat, inj, lam)
    got = replicas.combine_parts(ev, sw, sw2, cat.n_events, inj.n_draw, (fl & 1) != 0)
    ref = oracle.loglik(cat, inj, lam)
    for g, r in zip(got, ref):
        np.testing.assert_array_equal(g, r)


@pytest.mark.parametrize("sizes,world", [([1] * 5, 5), ([100, 1, 1, 1], 2), ([3, 3, 3, 3, 3, 3], 4), ([50], 1)])
def test_event_ranges_cover_every_event_once(sizes, world):
    from paper_1904_02863_gb300 import replicas
    off = np.concatenate([[0], np.cumsum(sizes)])
    cuts = [replicas.event_range(off, r, world) for r in range(world)]
    assert cuts[0][0] == 0 and cuts[-1][1] == len(sizes)
    assert all(a < b for a, b in cuts) and all(cuts[i][1] == cuts[i + 1][0] for i in range(world - 1))
    with pytest.raises(ValueError):
        replicas.event_range(off, 0, len(sizes) + 1)
