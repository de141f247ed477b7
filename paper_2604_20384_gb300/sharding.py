"""Sharding the samples of one problem across processes (host logic).

The sampled cost is a mean over independent samples (Eq. costHS; the paper
notes that its evaluation is embarrassingly parallel), so every output is a
sample-weighted mean of per-shard outputs:
    C      = 1 - sum_r N_r (1 - C_r) / N
    grad   = sum_r N_r grad_r / N,   hvp = sum_r N_r hvp_r / N
(the Riemannian forms are linear in (grad, hvp) for fixed G and V, so they
combine the same way). One sum of a few kB per call is the only exchange.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n_samples: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) sample range of a rank; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_samples, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def pack(n_shard: int, loss: float, grad: np.ndarray, hvp: np.ndarray | None = None) -> np.ndarray:
    """Per-shard sums over samples as one FP64 vector (what an all-reduce sums)."""
    parts = [np.array([n_shard * (1.0 - loss), float(n_shard)])]
    parts.append(n_shard * np.ascontiguousarray(grad, dtype=np.complex128).view(np.float64).ravel())
    if hvp is not None:
        parts.append(n_shard * np.ascontiguousarray(hvp, dtype=np.complex128).view(np.float64).ravel())
    return np.concatenate(parts)


def unpack(buf: np.ndarray, K: int, with_hvp: bool = True):
    """Inverse of the summed :func:`pack`: (loss, grad, hvp) of all samples."""
    n = buf[1]
    loss = 1.0 - buf[0] / n
    g = (buf[2:2 + 32 * K] / n).copy().view(np.complex128).reshape(K, 4, 4)
    h = None
    if with_hvp:
        h = (buf[2 + 32 * K:2 + 64 * K] / n).copy().view(np.complex128).reshape(K, 4, 4)
    return loss, g, h


def allreduce(n_shard: int, loss: float, grad: np.ndarray, hvp: np.ndarray | None = None, group=None):
    """Combine per-rank results with one torch.distributed all-reduce (sum)."""
    import torch
    import torch.distributed as dist

    buf = torch.from_numpy(pack(n_shard, loss, grad, hvp))
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    K = np.asarray(grad).shape[0]
    return unpack(buf.numpy(), K, hvp is not None)
