"""Sharding across ranks (one GPU per rank).

Channels are imaged independently (Sec. 5: each GPU of the deployment takes its
own slice of the band), so a multi-GPU run splits the channels into contiguous,
balanced ranges with no data-path collective.  Collectives appear only off the
hot path: assembling the full image set on one rank, and the max-over-ranks
timing of a benchmark.

A block can instead be split over time: images with the autocorrelation term
removed are additive over samples, so every rank images its own range of samples
of all channels and one sum all-reduce of the [n_chan][4][N][N] accumulators per
block gives the block's image (up to the order of the FP32 additions).
"""
from __future__ import annotations


def channel_shard(n_chan: int, rank: int, world: int) -> tuple[int, int]:
    """[c_lo, c_hi) of rank's channels: contiguous, sizes differing by at most 1."""
    if world < 1 or not 0 <= rank < world or n_chan < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_chan, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_channels(n_chan: int, rank: int, world: int, mode: str) -> tuple[int, int]:
    """[c_lo, c_hi) of the band a rank images in a multi-GPU run.

    mode "replicate": every rank images the whole band of its own block (weak
    scaling: per-GPU work fixed as ranks are added); mode "channels": the ranks
    split one block's band into contiguous balanced ranges (strong scaling: the
    paper's per-GPU bandwidth split, Sec. 5.1)."""
    if mode == "replicate":
        if world < 1 or not 0 <= rank < world:
            raise ValueError("bad shard request")
        return 0, n_chan
    if mode == "channels":
        return channel_shard(n_chan, rank, world)
    raise ValueError(f"unknown shard mode {mode!r}")


def job_units(block_units: int, world: int, mode: str) -> int:
    """Antenna x channel x sample units the whole job images per step: one block
    per rank when replicating, one block split over the ranks otherwise."""
    return block_units * world if mode == "replicate" else block_units


def scaling(mode: str) -> str:
    """The bench line's "scaling" key for a shard mode."""
    return "weak" if mode == "replicate" else "strong"


def time_shard(n_time: int, rank: int, world: int) -> tuple[int, int]:
    """[t_lo, t_hi) of rank's samples of a block: contiguous, sizes differing by at most 1."""
    return channel_shard(n_time, rank, world)


def sum_images(local, group=None):
    """The sum over ranks of each rank's image accumulators (in place; every rank
    receives the block's image).  The one exchange of a time-split block."""
    import torch.distributed as dist
    dist.all_reduce(local, op=dist.ReduceOp.SUM, group=group)
    return local


def gather_channels(local, n_chan: int, group=None):
    """All ranks' [c_hi-c_lo][...] image blocks concatenated in channel order
    (every rank receives the full [n_chan][...] tensor).  Off the hot path."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [channel_shard(n_chan, r, world) for r in range(world)]
    width = max(hi - lo for lo, hi in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: hi - lo] for r, (lo, hi) in enumerate(sizes)], dim=0)


def max_over_ranks(x: float, device=None, group=None) -> float:
    """The largest value of x over all ranks (timing: the slowest rank decides)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
