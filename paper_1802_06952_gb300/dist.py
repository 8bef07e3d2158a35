"""Copy sharding across ranks (one process per GPU).

The copies of the cut circuit are independent (Supplementary B: each partition is
computed independently), so a rank evolves the halves of its own copies and
contracts them into a partial amplitude block; one sum-reduce of the blocks gives
A(x_u, x_l) = sum_k U_k[x_u] L_k[x_l] (Supplementary A, Eq. 8).

Copies are dealt out as contiguous ranges of the copy index.  The copy tree's
first level holds the lowest copy bits, so a rank's range keeps the prefix
sharing of every level whose bits lie above the range boundary.  Ranges are
balanced to within one copy.
"""
import torch.distributed as dist


def copy_ranges(copies, world):
    """[begin, end) of each rank: contiguous, balanced to within one copy."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(copies, world)
    out, b = [], 0
    for r in range(world):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def rank_range(copies, world, rank):
    return copy_ranges(copies, world)[rank]


def reduce_amplitudes(block, group=None):
    """Sum the ranks' partial amplitude blocks in place (all ranks get the sum).
    The block is a torch tensor (complex or real view); complex tensors are
    reduced through their real view."""
    t = block
    if t.is_complex():
        t = torch_view_as_real(t)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return block


def torch_view_as_real(t):
    import torch
    return torch.view_as_real(t)


def max_over_ranks(value, device=None, group=None):
    """The largest of the ranks' values (step times are taken as the slowest rank's)."""
    import torch
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
