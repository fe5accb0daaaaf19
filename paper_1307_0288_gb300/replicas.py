"""Replica parallelism over processes (one GPU per rank).

Random vectors and disorder realisations are independent units, so the path shards
with no collective on the data path: rank k gets its own vector seeds, runs the whole
moment computation on its GPU, and the per-rank moment arrays are summed once at the
end (the trace estimator is an average over vectors, Sec. 3.1.1).  This module holds
the host logic: the seed assignment and the one reduction.  It works with any
torch.distributed backend (NCCL on GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

import numpy as np


def rank_vector_seed(base_seed: int, rank: int, vectors_per_rank: int) -> int:
    """Seed of rank `rank`'s vector block: vectors r of rank k use streams of seed
    base + k * vectors_per_rank, so no two ranks draw the same random phases."""
    if rank < 0 or vectors_per_rank < 1:
        raise ValueError("bad rank or vector count")
    return base_seed + rank * vectors_per_rank


def average_moments(mu: np.ndarray, n_local: int, group=None) -> np.ndarray:
    """Average over all ranks' vectors of moment arrays shaped [R_local, ...].

    Sums the local vector sums and vector counts with one all_reduce and divides.
    Raises (never hangs) when a peer has failed: the collective fails or times out
    with the process group's timeout.
    """
    import torch
    import torch.distributed as dist

    local = np.asarray(mu)
    if local.shape[0] != n_local:
        raise ValueError("leading dimension must be the local vector count")
    s = torch.from_numpy(np.ascontiguousarray(local.sum(axis=0)))
    if s.is_complex():
        s = torch.view_as_real(s).contiguous()
    count = torch.tensor([float(n_local)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(s, group=group)
        dist.all_reduce(count, group=group)
    out = s.numpy()
    if np.iscomplexobj(local):
        out = out[..., 0] + 1j * out[..., 1]
    return out / count.item()
