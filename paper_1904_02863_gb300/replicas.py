"""Data parallelism: one process per GPU.

Replicas (the default).  Every Lambda point is an independent problem (a
sampler's walkers are independent too), so each rank loads the same catalog
and injections and evaluates its own slice of the Lambda batch: nothing on the
data path needs a collective.  torch.distributed is used only for the timing
barrier, the max over ranks and, when a caller wants every result on every
rank, an all-gather of the K output rows.

Event partition (for a catalog too large for one GPU).  ln L is a sum over
events minus N ln xi, and xi a sum over injections (paper, Sec. "Population
acceleration"), so each rank loads a range of events balanced by sample count
and a share of the found injections, returns the additive parts
(sum_i ln(S_i/n_i), sum w, sum w^2) per Lambda, and one all-reduce of K x 3
doubles gives the whole; ln L, ln xi and N_eff then follow on the host exactly
as the library's finalise forms them.
"""
from __future__ import annotations

import os

import numpy as np


def init_from_env():
    """(rank, local_rank, world) from torchrun's environment; initialises the process group for world > 1."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, local, world


def shard(K, rank, world):
    """Contiguous, balanced slice [start, stop) of K Lambda rows for this rank."""
    base, extra = divmod(int(K), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _device():
    import torch
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x, world):
    """Largest value of a float across ranks (the slowest rank's time)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local, K, world):
    """All-gather the per-rank slices (shard order) of a length-K float64 array."""
    local = np.ascontiguousarray(local, dtype=np.float64)
    if world == 1:
        return local
    import torch
    import torch.distributed as dist
    sizes = [shard(K, r, world)[1] - shard(K, r, world)[0] for r in range(world)]
    width = max(sizes)
    buf = torch.zeros(width, dtype=torch.float64, device=_device())
    buf[:local.size] = torch.from_numpy(local).to(buf.device)
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    return np.concatenate([p[:n].cpu().numpy() for p, n in zip(parts, sizes)])


# ---------------------------------------------------------------- event partition
FLAG_INVALID_LAMBDA, FLAG_ZERO_EVENT, FLAG_LOW_NEFF, FLAG_ZERO_XI = 1, 2, 4, 32


def event_range(offsets, rank, world):
    """CSR event range [e0, e1) of this rank: cuts near equal sample counts, at least one event each."""
    off = np.asarray(offsets, dtype=np.int64)
    n = len(off) - 1
    if n < world:
        raise ValueError(f"{n} events cannot be split over {world} ranks")
    cuts = [0] + [int(np.searchsorted(off, off[-1] * r / world, side="left")) for r in range(1, world)] + [n]
    for r in range(1, world):
        cuts[r] = min(max(cuts[r], cuts[r - 1] + 1), n - (world - r))
    return cuts[rank], cuts[rank + 1]


def sub_catalog(catalog, e0, e1):
    """Events [e0, e1) of a catalog, offsets rebased to 0."""
    from . import synth
    off = np.asarray(catalog.offsets, dtype=np.int64)
    a, b = int(off[e0]), int(off[e1])
    return synth.Catalog(off[e0:e1 + 1] - a, catalog.theta[a:b], catalog.prior[a:b])


def sub_injections(injections, rank, world):
    """This rank's share of the found injections; n_draw stays the total number of draws."""
    from . import synth
    a, b = shard(injections.n_found, rank, world)
    if b <= a:
        raise ValueError(f"{injections.n_found} injections cannot be split over {world} ranks")
    return synth.Injections(injections.theta[a:b], injections.p_draw[a:b], injections.n_draw)


def all_reduce_sum(x, world):
    """Sum of a float64 array over ranks (every rank gets the result)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(x.copy()).to(_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def combine_parts(events, sum_w, sum_w2, n_events, n_draw, invalid):
    """ln L, ln xi, N_eff and flags from summed parts (the finalise formulas of the library).

    events = sum over all events of ln(S_i/n_i) (-inf when some S_i = 0), sum_w and
    sum_w2 over all found injections, n_events the total event count, n_draw the
    total number of draws, invalid the per-Lambda invalid flag."""
    events, sum_w, sum_w2 = (np.asarray(x, dtype=np.float64) for x in (events, sum_w, sum_w2))
    invalid = np.asarray(invalid, dtype=bool)
    nd = float(n_draw)
    xi = sum_w / nd
    var = sum_w2 / (nd * nd) - xi * xi / nd
    with np.errstate(divide="ignore", invalid="ignore"):
        neff = np.where(var > 0.0, xi * xi / np.where(var > 0.0, var, 1.0), np.inf)
        lnxi = np.where(xi > 0.0, np.log(np.where(xi > 0.0, xi, 1.0)), -np.inf)
        zero_event = np.isneginf(events)
        zero_xi = xi == 0.0
        lnL = np.where(zero_event | zero_xi, -np.inf, events - n_events * lnxi)
    neff = np.where(zero_xi, 0.0, neff)
    flags = (np.where(zero_event, FLAG_ZERO_EVENT, 0) | np.where(zero_xi, FLAG_ZERO_XI, 0) |
             np.where(neff < 4.0 * n_events, FLAG_LOW_NEFF, 0)).astype(np.uint32)
    lnL = np.where(invalid, -np.inf, lnL)
    lnxi = np.where(invalid, 0.0, lnxi)
    neff = np.where(invalid, 0.0, neff)
    flags = np.where(invalid, np.uint32(FLAG_INVALID_LAMBDA), flags).astype(np.uint32)
    return lnL, lnxi, neff, flags


class EventPartition:
    """A catalog split over ranks by events and injections; one all-reduce of K x 3 per batch."""

    def __init__(self, catalog, injections, rank, world, device=0, stream=None, storage=None):
        from . import binding as B
        self.B, self.world = B, world
        self.n_events, self.n_draw = catalog.n_events, injections.n_draw
        self.events = event_range(catalog.offsets, rank, world)
        cat = sub_catalog(catalog, *self.events)
        inj = sub_injections(injections, rank, world)
        st = storage if storage is not None else B.POP_STORE_F64 | B.POP_STORE_F32
        self.like = B.Likelihood(device, stream).load(cat, inj, storage=st)

    def __call__(self, lambdas, mode=None):
        B = self.B
        ev, sw, sw2, fl = B.pop_loglik_parts(self.like.ctx, lambdas, B.POP_MODE_F64 if mode is None else mode)
        tot = all_reduce_sum(np.stack([ev, sw, sw2]), self.world)
        return combine_parts(tot[0], tot[1], tot[2], self.n_events, self.n_draw,
                             (fl & FLAG_INVALID_LAMBDA) != 0)

    def close(self):
        self.like.close()
