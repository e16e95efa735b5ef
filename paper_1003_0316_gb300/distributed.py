"""Multi-GPU sharding of the hot path (one process per GPU).

P, eps/W^c and the Sigma pair coefficients are independent per q, and the frequency
convolution is linear in the pair coefficients, so every rank runs the whole path on
its own block of q points and produces a partial Sigma^c(i w); the one exchange is a
sum over ranks of that [n_sigma][n_omega_out] complex array (a few KB). The fit of the
analytic continuation then runs on the summed curves.
"""
import torch


def shard(n, rank, world):
    """Contiguous block of the n units (q points) owned by rank: [lo, hi)."""
    return n * rank // world, n * (rank + 1) // world


def allreduce_sum_(t, group=None):
    """In-place sum over ranks of a real or complex tensor (complex as pairs of reals, which
    every backend reduces)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return t
    v = torch.view_as_real(t) if t.is_complex() else t
    dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    return t
