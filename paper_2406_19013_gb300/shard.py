"""Channel bands across processes, one GPU per process.

The X-engine correlates every frequency channel on its own (Sec. 2.3), and
the paper's system splits the band over servers and over pipeline instances
inside each server (Sec. 2.2).  A multi-GPU job therefore gives every rank a
contiguous band of channels and needs no exchange while it integrates.  The
only collectives sit outside the data path:
- the maximum of the ranks' timings;
- an optional gather of the dumped bands to one rank.

Every function works on any torch.distributed backend: gloo on the CPU,
nccl with CUDA tensors.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def band(rank: int, world: int, n_chan: int) -> tuple[int, int]:
    """First channel and channel count of `rank`'s band.

    The band is contiguous and near-equal. The first n_chan % world ranks
    take one extra channel. A rank gets zero channels when world > n_chan.
    """
    if world <= 0 or not 0 <= rank < world or n_chan < 0:
        raise ValueError(f"bad band request: rank {rank} of {world}, {n_chan} channels")
    base, extra = divmod(n_chan, world)
    return rank * base + min(rank, extra), base + (1 if rank < extra else 0)


def _device() -> torch.device:
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(value: float) -> float:
    """Maximum of a float over all ranks (the job time is the slowest rank's)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float) -> float:
    """Sum of a float over all ranks (the job's work is every rank's work)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_bands(local: torch.Tensor, n_chan: int, dst: int = 0) -> torch.Tensor | None:
    """Stitch every rank's band of a per-channel array on rank `dst`.

    `local` is this rank's rows: shape [n_local, ...], where n_local and the
    band follow `band(rank, world, n_chan)`. Each band is padded to the
    largest band's size and sent with one gather.

    Returns [n_chan, ...] on `dst` and None elsewhere. Raises ValueError if
    `local` does not match this rank's band.
    """
    if not (dist.is_available() and dist.is_initialized()):
        if local.shape[0] != n_chan:
            raise ValueError("single process: the local band must hold every channel")
        return local
    rank, world = dist.get_rank(), dist.get_world_size()
    c0, n = band(rank, world, n_chan)
    if local.shape[0] != n:
        raise ValueError(f"rank {rank}: band holds {n} channels, tensor has {local.shape[0]}")
    width = -(-n_chan // world)
    dev = _device()
    padded = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=dev)
    padded[:n] = local.to(dev)
    bufs = None
    if rank == dst:
        bufs = [torch.empty_like(padded) for _ in range(world)]
    dist.gather(padded, gather_list=bufs, dst=dst)
    if rank != dst:
        return None
    out = torch.empty((n_chan,) + tuple(local.shape[1:]), dtype=local.dtype, device=dev)
    for r in range(world):
        r0, rn = band(r, world, n_chan)
        out[r0:r0 + rn] = bufs[r][:rn]
    return out
