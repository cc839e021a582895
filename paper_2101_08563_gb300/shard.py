"""One mixture over several GPUs by contiguous frequency ranges.

FastFCA treats every frequency bin on its own (Sec. IV-G: the parameters of one frequency
never enter another's update), so a mixture splits over ranks along f with no exchange
during the iterations.  Each rank runs its own context on x[f0:f1] and the only collective
is one FP64 sum of the per-iteration log-likelihood (Eq. 31 summed over f) over the ranks.
The images of a rank's range are the rows f0:f1 of the whole result.

The per-rank work is any object with `iterate(n_iter) -> ll per iteration (float64)` and
`loglik() -> float` over that rank's frequencies: a `fastfca.Separator` on the GPU.
"""
from __future__ import annotations

import numpy as np


def frequency_ranges(F: int, world: int):
    """Contiguous [f0, f1) ranges, one per rank, sizes differing by at most one (the lower
    ranks take the extra frequencies).  Every frequency is in exactly one range."""
    if F < 1 or world < 1:
        raise ValueError("F and world must be positive")
    base, extra = divmod(F, world)
    out, f0 = [], 0
    for r in range(world):
        f1 = f0 + base + (1 if r < extra else 0)
        out.append((f0, f1))
        f0 = f1
    return out


def allreduce_sum_f64(values, world: int, device=None):
    """Sum of a float64 vector over the ranks (one all-reduce); the vector itself when
    world == 1."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    if world == 1:
        return v.copy()
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(v.copy())
    if device is not None:
        t = t.to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


class FrequencyShard:
    """This rank's share of one mixture: `local` runs the frequencies [f0, f1) of the rank;
    `iterate` and `loglik` return whole-mixture log-likelihoods (one FP64 all-reduce each)."""

    def __init__(self, local, F: int, rank: int, world: int, device=None):
        self.local = local
        self.F, self.rank, self.world, self.device = F, rank, world, device
        self.f0, self.f1 = frequency_ranges(F, world)[rank]

    def iterate(self, n_iter: int):
        ll_local = np.asarray(self.local.iterate(n_iter), dtype=np.float64)
        return allreduce_sum_f64(ll_local, self.world, self.device)

    def loglik(self) -> float:
        return float(allreduce_sum_f64([self.local.loglik()], self.world, self.device)[0])


def gpu_shard(x, N: int, rank: int, world: int, device, **separator_kwargs):
    """A FrequencyShard whose local work is a GPU Separator on this rank's rows of x
    (complex64 (F, T, M), host or CUDA); the Separator is `shard.local`."""
    from . import fastfca
    F = int(x.shape[0])
    f0, f1 = frequency_ranges(F, world)[rank]
    xs = x[f0:f1]
    if hasattr(xs, "data_ptr") and xs.data_ptr() % 16:   # the library loads frames as 16-byte vectors
        xs = xs.clone()
    sep = fastfca.Separator(xs, N, **separator_kwargs)
    return FrequencyShard(sep, F, rank, world, device)
