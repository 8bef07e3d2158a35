"""Copy sharding across ranks (one process per GPU).

The copies of the cut circuit are independent (Supplementary B: each partition is
computed independently), so a rank evolves the halves of its own copies and
contracts them into a partial amplitude block; one sum-reduce of the blocks gives
A(x_u, x_l) = sum_k U_k[x_u] L_k[x_l] (Supplementary A, Eq. 8).

Which copies go together matters for the prefix sharing of Section 2.3.2.  Copy
bit m belongs to the m-th cut CZ in (layer, qubit) order, so the copy tree's first
branch level fixes the LOWEST bits of k and its leaves the highest.  Two copies
share the evolution of every level whose bits they agree on.  copy_lists therefore
deals out copies by their bit-reversed index: a rank's copies agree on the low
(early-layer) bits, i.e. they form whole subtrees of the copy tree, and no tree
node below the split is evolved on two ranks.  (A contiguous range of k agrees on
the high bits instead, so every rank would evolve every node of the early levels;
copy_ranges is kept for callers that want plain ranges.)
"""
import numpy as np
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


def _bit_reverse(k, bits):
    r = np.zeros_like(k)
    for i in range(bits):
        r |= ((k >> np.uint64(i)) & np.uint64(1)) << np.uint64(bits - 1 - i)
    return r


def copy_lists(c, world):
    """The copies 0 .. 2^c - 1 dealt out as subtrees of the copy tree: sorted by
    bit-reversed index and cut into world contiguous runs, balanced to within one
    copy.  With world a power of two (<= 2^c), rank r gets exactly the copies whose
    low log2(world) bits spell r in reverse: one subtree per rank.  Each list is
    ascending by bit-reversed index, so copies that share a prefix are adjacent."""
    if world < 1:
        raise ValueError("world must be >= 1")
    k = np.arange(1 << c, dtype=np.uint64)
    order = k[np.argsort(_bit_reverse(k, c), kind="stable")]
    return [order[b:e] for b, e in copy_ranges(1 << c, world)]


def rank_list(c, world, rank):
    return copy_lists(c, world)[rank]


def tree_nodes(copies, level_bits):
    """Nodes of each copy-tree level that a set of copies evolves: a level that has
    fixed the low b copy bits runs once per distinct value of k mod 2^b among them
    (level_bits lists b for every level, as sim_plan_levels reports them)."""
    k = np.asarray(copies, dtype=np.uint64)
    return [int(np.unique(k & np.uint64((1 << b) - 1)).size) for b in level_bits]


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
