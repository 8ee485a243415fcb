"""One SMC population sharded over ranks: the exchange step of parallel
systematic resampling (Section 3.3) between GPUs.

Rank r holds particles [first_r, first_r + n_r) of a population of n_total, in
slices that start on whole tiles of SMC_RESAMPLE_TILE (4096) particles.  One
resampling of the population is:

  1. each rank reduces its slice to its tiles' records (smc_shard_reduce);
  2. the records of all ranks are all-gathered in rank order (16 bytes a tile:
     the only exchange the normaliser needs);
  3. each rank combines all records (the same exact integers on every rank: S,
     the log-Z increment, the search scalars) and searches the offsets its own
     tiles own (smc_shard_ancestors): offsets [lo_r, hi_r), whose ancestors all
     lie in its slice;
  4. the states of those ancestors are gathered on the rank (smc_gather) and
     sent to the ranks whose slices hold the new indices; since systematic
     ancestors are non-decreasing, a rank's offsets mostly stay on it and only
     the ends of its range move to its neighbours.

The ancestors, S and the log-Z increment equal smc_resample's on the whole
population, bit for bit.  torch.distributed carries the records and the states
(NCCL with CUDA tensors; gloo through host copies).  Steps 1 and 3 run the
library's kernels; this module only exchanges.
"""
from __future__ import annotations

from . import smc

TILE = 4096


def slices(n_total: int, world: int) -> list[tuple[int, int]]:
    """(first, n) of every rank: whole tiles, as even as they go."""
    nt = -(-n_total // TILE)
    per, extra = divmod(nt, world)
    out, t = [], 0
    for r in range(world):
        k = per + (1 if r < extra else 0)
        first = t * TILE
        last = min(n_total, (t + k) * TILE)
        out.append((first, max(0, last - first)))
        t += k
    return out


def _on_comm_device(x, group, device):
    """x on the device the group's backend carries: `device` (a CUDA device) for
    NCCL, the host for gloo."""
    import torch.distributed as dist

    return x.to(device) if dist.get_backend(group) == "nccl" else x.cpu()


def gather_records(rec_local, group=None):
    """All-gather the ranks' tile records in rank order (a uint8 tensor of the
    whole population's records, on rec_local's device)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    x = _on_comm_device(rec_local, group, rec_local.device)
    n = torch.tensor([x.numel()], dtype=torch.int64, device=x.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    pad = torch.zeros(max(sizes), dtype=torch.uint8, device=x.device)
    pad[: x.numel()] = x
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = torch.cat([p[:s] for p, s in zip(parts, sizes)])
    return out.to(rec_local.device)


def exchange_states(produced, lo: int, hi: int, all_slices, group=None):
    """Send the states of the offsets this rank searched, [lo, hi) (produced:
    [F, hi - lo]), to the ranks whose slices hold those new indices, and
    receive the new particles of this rank's slice ([F, n_r]) from the ranks
    that searched them."""
    import torch
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    F = produced.shape[0]
    dev = produced.device
    mine = _on_comm_device(torch.tensor([lo, hi], dtype=torch.int64), group, dev)
    ranges = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(ranges, mine, group=group)
    ranges = [tuple(int(v) for v in r.cpu().tolist()) for r in ranges]
    first_r, n_r = all_slices[rank]
    out = torch.empty((F, n_r), dtype=produced.dtype, device=produced.device)
    sends, recvs, keep = [], [], []
    for q, (first_q, n_q) in enumerate(all_slices):  # what this rank sends to q
        a, b = max(lo, first_q), min(hi, first_q + n_q)
        if a >= b:
            continue
        piece = produced[:, a - lo:b - lo]
        if q == rank:
            out[:, a - first_r:b - first_r] = piece
        else:
            buf = _on_comm_device(piece.contiguous(), group, dev)
            keep.append(buf)
            sends.append(dist.isend(buf, dst=q, group=group))
    for p, (lo_p, hi_p) in enumerate(ranges):  # what rank p sends to this rank
        a, b = max(lo_p, first_r), min(hi_p, first_r + n_r)
        if p == rank or a >= b:
            continue
        buf = _on_comm_device(torch.empty((F, b - a), dtype=produced.dtype, device=dev),
                              group, dev)
        recvs.append((dist.irecv(buf, src=p, group=group), buf, a, b))
    for req, buf, a, b in recvs:
        req.wait()
        out[:, a - first_r:b - first_r] = buf.to(out.device)
    for req in sends:
        req.wait()
    return out


def resample(logw_local, state_local, first: int, n_total: int, u: float, group=None):
    """Resample a sharded population and move the states: logw_local [n_r] f64 and
    state_local [F, n_r] (4- or 8-byte elements) on this rank's GPU, first its
    slice's start (see slices()), u the checkpoint's uniform (the same on every
    rank).  Returns (the new states [F, n_r], out3 = {m, S, log-Z increment}, the
    population's near-boundary offsets, this rank's [lo, hi))."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    all_slices = slices(n_total, world)
    if any(n == 0 for _, n in all_slices):
        raise ValueError(f"{n_total} particles fill fewer than one tile of {TILE} per rank")
    if (first, logw_local.numel()) != all_slices[dist.get_rank(group)]:
        raise ValueError("logw_local is not this rank's slice (see slices())")
    state_local = state_local.contiguous()
    rec = smc.shard_reduce(logw_local)
    records_all = gather_records(rec, group)
    anc, rng, o3, nn = smc.shard_ancestors(logw_local, first, records_all, n_total, u)
    lo, hi = (int(v) for v in rng.cpu().tolist())
    F = state_local.shape[0]
    produced = torch.empty((F, max(0, hi - lo)), dtype=state_local.dtype,
                           device=state_local.device)
    if hi > lo:
        for f in range(F):  # produced[f][i] = state[f][anc[lo + i] - first]
            smc.gather_row(state_local[f], produced[f], anc[lo:hi], first)
    new_state = exchange_states(produced, lo, hi, all_slices, group)
    n_near = _on_comm_device(nn.clone(), group, nn.device)
    dist.all_reduce(n_near, group=group)
    return new_state, o3, int(n_near.item()), (lo, hi)
