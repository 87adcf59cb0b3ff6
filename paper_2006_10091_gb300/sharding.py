"""The paper's workers sharded over GPUs, one process per GPU (Sec. 4, Fig. 1;
Algorithms 1 and 2).

Workers are independent between refreshes: each rank steps the workers it
owns with the library's batched entry point and exchanges nothing.  The only
exchange is the key holder's aggregation (Algorithm 2): every rank sums its
workers' encrypted weights (he_sum, modular addition of residues), the ranks'
partial sums are all-gathered as raw uint64 residues (bitwise: a plain NCCL
sum would add the integers, not the residues modulo each prime) and summed
again with he_sum, and rank 0, the key holder, decrypts that sum read at K
times its scale -- the average of the K workers' weights -- re-encodes and
re-encrypts it at the top level, and broadcasts the residues; every worker
continues from them.

The partition gives each rank a set of workers with about the same number of
data ciphertexts (largest first, to the least loaded rank), which is what a
step costs.

Failure detection is on the host: before each aggregation every rank checks in
through a key-value store (refresh_check_in) and waits, bounded, for all the
others.  A rank that dropped out or stalled past the limit, or one that
arrives with a stale or duplicated refresh (another iteration, level or
scale), raises an error on every rank before any collective starts, so no rank
is left waiting in all_gather.
"""
from __future__ import annotations

import datetime

import torch

from . import (HE_ETIMEOUT, HE_ESCALE, Ciphertext, he_lr_gradient_step_workers, he_refresh, he_sum)


class RefreshError(RuntimeError):
    """A rank's refresh could not proceed; `code` is HE_ETIMEOUT (a rank did not
    check in within the limit) or HE_ESCALE (ranks disagree on the iteration,
    level or scale of the weights they bring)."""

    def __init__(self, code: int, msg: str):
        super().__init__(msg)
        self.code = code


def refresh_check_in(store, iteration: int, rank: int, world: int, level: int, scale: float,
                     timeout_s: float = 60.0, prefix: str = "he_refresh") -> None:
    """Publish this rank's (iteration, level, scale) under
    prefix/iteration/rank in `store` (a torch.distributed Store) and wait at
    most timeout_s for every rank's entry; then check that all agree.  Raises
    RefreshError(HE_ETIMEOUT) naming the ranks missing after the limit, or
    RefreshError(HE_ESCALE) when the entries differ."""
    mine = f"{iteration}:{level}:{float(scale).hex()}"
    keys = [f"{prefix}/{iteration}/{r}" for r in range(world)]
    store.set(keys[rank], mine)
    try:
        store.wait(keys, datetime.timedelta(seconds=timeout_s))
    except Exception as e:  # the store's own timeout error
        missing = [r for r in range(world) if not store.check([keys[r]])]
        raise RefreshError(HE_ETIMEOUT, f"refresh {iteration}: ranks {missing} did not check in within "
                                        f"{timeout_s} s ({type(e).__name__})") from None
    vals = [store.get(k).decode() for k in keys]
    if any(v != mine for v in vals):
        raise RefreshError(HE_ESCALE, f"refresh {iteration}: ranks bring different weights "
                                      f"(iteration:level:scale) {vals}")


def partition_shards(sizes, world: int) -> list[list[int]]:
    """Worker indices per rank: workers in decreasing order of size (data
    ciphertexts; ties by index) each go to the rank with the least total so
    far (ties to the lower rank).  Deterministic; every rank computes the
    same partition."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for k in sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i)):
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(k)
        load[r] += int(sizes[k])
    return [sorted(p) for p in parts]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def allreduce_ciphertext(ctx, ct: Ciphertext, out: Ciphertext, group=None, add=None) -> Ciphertext:
    """out = the sum over ranks of every rank's `ct` (same level and scale on
    all ranks), by element-wise modular addition of residues.  The residues
    [2][level][N] travel as int64 words through all_gather; the sum of the
    gathered copies is the library's he_sum (`add(ctx, list, out)` replaces
    it, e.g. an oracle on CPU ranks).  One process: out = ct."""
    add = add or he_sum
    dist = _dist()
    world = dist.get_world_size(group) if dist else 1
    local = ct.tensor[:, : ct.level].contiguous()
    if world == 1:
        return add(ctx, [Ciphertext(local, ct.level, ct.level, ct.scale)], out)
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local, group=group)
    stacked = torch.stack(parts)  # [world][2][level][N], one allocation: a uniform batch
    cts = [Ciphertext(stacked[r], ct.level, ct.level, ct.scale) for r in range(world)]
    return add(ctx, cts, out)


def broadcast_ciphertext(ct: Ciphertext, src: int = 0, group=None) -> Ciphertext:
    """Every rank's `ct` (capacity >= the level) receives rank src's residues,
    level and scale."""
    dist = _dist()
    if not dist or dist.get_world_size(group) == 1:
        return ct
    meta = torch.tensor([float(ct.level), ct.scale], dtype=torch.float64, device=ct.tensor.device)
    dist.broadcast(meta, src, group=group)
    level = int(meta[0].item())
    buf = ct.tensor[:, :level].contiguous()
    dist.broadcast(buf, src, group=group)
    ct.tensor[:, :level].copy_(buf)
    ct.level, ct.scale = level, float(meta[1].item())
    return ct


def key_holder_refresh(ctx, total: Ciphertext, n_workers: int, top_level: int, scale: float, cid: int,
                       out: Ciphertext, group=None) -> Ciphertext:
    """Algorithm 2 on rank 0: `total` (the sum of all workers' weights) read at
    n_workers times its scale decrypts to their average; it is re-encoded at
    `scale` and encrypted at `top_level` (random stream cid) into `out`, which
    every rank then receives."""
    dist = _dist()
    rank = dist.get_rank(group) if dist else 0
    if rank == 0:
        avg = Ciphertext(total.tensor, total.cap, total.level, total.scale * n_workers)
        he_refresh(ctx, avg, top_level, scale, cid, out)
    return broadcast_ciphertext(out, 0, group)


def train_sharded(ctx, shards: list, cfg, iterations: int, refresh_every: int, top_level: int, cid0: int,
                  n_workers: int, group=None, store=None, timeout_s: float = 60.0) -> Ciphertext:
    """Algorithms 1 and 2 over ranks: `shards` = this rank's workers as
    (Z list, W) with W at top_level (all workers start from the same
    weights); `n_workers` = the workers of all ranks.  Every worker runs
    `iterations` gradient steps (Eq. 7-8) on its own data; after every
    `refresh_every` steps and after the last, the weights of all workers are
    summed across ranks and the key holder replaces them by the re-encrypted
    average (random stream cid0 + iteration).  With a `store` (the ranks'
    torch.distributed Store) every rank checks in before each aggregation
    (refresh_check_in, bounded by timeout_s).  Returns the final average (at
    top_level), identical on every rank."""
    if top_level < 5 * refresh_every + 1:
        raise ValueError("the weights run out of limbs before the refresh")
    if not shards:
        raise ValueError("every rank needs at least one worker")
    scale = shards[0][1].scale
    cap = top_level
    cur = [ctx.new_ct(cap) for _ in shards]
    nxt = [ctx.new_ct(cap) for _ in shards]
    for (Z, W), c in zip(shards, cur):
        c.tensor[:, :top_level].copy_(W.tensor[:, :top_level])
        c.level, c.scale = top_level, W.scale
    local_sum, total, fresh = ctx.new_ct(cap), ctx.new_ct(cap), ctx.new_ct(cap)
    for it in range(1, iterations + 1):
        he_lr_gradient_step_workers(ctx, [(Z, c, o) for (Z, _), c, o in zip(shards, cur, nxt)], cfg)
        cur, nxt = nxt, cur
        if it % refresh_every == 0 or it == iterations:
            he_sum(ctx, cur, local_sum)
            if store is not None:
                dist = _dist()
                rank = dist.get_rank(group) if dist else 0
                world = dist.get_world_size(group) if dist else 1
                refresh_check_in(store, it, rank, world, local_sum.level, local_sum.scale, timeout_s)
            allreduce_ciphertext(ctx, local_sum, total, group)
            key_holder_refresh(ctx, total, n_workers, top_level, scale, cid0 + it, fresh, group)
            for c in cur:
                c.tensor[:, :top_level].copy_(fresh.tensor[:, :top_level])
                c.level, c.scale = fresh.level, fresh.scale
    return cur[0]
