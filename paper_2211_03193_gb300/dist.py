"""Chains over several GPUs: each rank runs its own chains (independent MCMC
chains, Sec. 2.4 "Inter-Block parallelism"), so the sampling path needs no
collective; the one exchange is the final merge of the best states, an
all-gather of each rank's lowest-energy chain followed by an argmin (ties go
to the lowest rank).  Works with any torch.distributed backend (gloo on CPU
tensors, NCCL on CUDA tensors)."""
from __future__ import annotations

import numpy as np


def local_best(best_E: np.ndarray, best_theta: np.ndarray):
    """The lowest-energy chain of this rank: (energy, torsions)."""
    best_theta = np.asarray(best_theta).reshape(best_E.shape[0], -1)
    i = int(np.argmin(best_E))
    return float(best_E[i]), best_theta[i]


def merge_best(best_E: np.ndarray, best_theta: np.ndarray, device: str = "cpu"):
    """Global best over all ranks: returns (energy, torsions, rank) on every rank."""
    import torch
    import torch.distributed as dist
    e, th = local_best(np.asarray(best_E, dtype=np.float64), best_theta)
    world = dist.get_world_size()
    e_t = torch.tensor([e], dtype=torch.float64, device=device)
    th_t = torch.tensor(np.asarray(th, dtype=np.float32), device=device)
    es = [torch.empty_like(e_t) for _ in range(world)]
    ths = [torch.empty_like(th_t) for _ in range(world)]
    dist.all_gather(es, e_t)
    dist.all_gather(ths, th_t)
    vals = torch.cat(es).cpu().numpy()
    r = int(np.argmin(vals))
    return float(vals[r]), ths[r].cpu().numpy(), r
