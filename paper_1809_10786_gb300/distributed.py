"""Multi-GPU layout of the transform (one process per GPU).

The points are independent, so ranks split them: each rank evaluates the forward
transform and the point gradient on its own shard with no communication (the
factorization is exact for every rho >= max r, so each rank may use its own rho).
The adjoint sums over all points, so the per-rank partial coefficient vectors are
added with one all-reduce of Nc complex numbers -- the only exchange of the path.
"""
import torch
import torch.distributed as dist


def shard(M_total, rank, world):
    """(start, count) of rank's contiguous share of M_total points (sizes differ by at most 1)."""
    base, extra = divmod(int(M_total), int(world))
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def allreduce_coefficients(coef, group=None):
    """Sum complex coefficient vectors over ranks in place (real view, one all-reduce)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(torch.view_as_real(coef), op=dist.ReduceOp.SUM, group=group)
    return coef


def max_over_ranks(value, device=None):
    """Maximum of a float over ranks (the bench's whole-job time)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sharded_adjoint(adjoint_fn, xyz, vals, rank, world, group=None):
    """Lambda^H vals over all points, given a per-shard adjoint callable (xyz_shard, vals_shard) -> coef."""
    start, count = shard(xyz.shape[0], rank, world)
    part = adjoint_fn(xyz[start:start + count], vals[start:start + count])
    return allreduce_coefficients(part, group)
