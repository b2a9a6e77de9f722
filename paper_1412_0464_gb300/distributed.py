"""Sources of one adjoint gradient split over the ranks of a process group.

Each rank holds the whole medium and its own factorised solver (one GPU per
rank), takes a contiguous share of the sources, computes the misfit and the
gradient of its share with ``Solver.grad`` (``hz_grad``), and the partial
misfits and gradients are summed over the ranks (one all-reduce each): the
misfit and its gradient are sums over sources, so the result equals the
one-rank gradient up to the order of the floating-point sums.  The right-hand
sides of one solve have no exchange between them, so sharding needs no other
communication.
"""

from __future__ import annotations


def shard(n: int, rank: int, world: int) -> range:
    """Contiguous share of n items for `rank`: sizes differ by at most one, the
    first n mod world ranks take one more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def sharded_grad(grad_fn, src, rec, d, shape, group=None, device=None):
    """(misfit, gradient) of all sources, each rank computing its share.

    grad_fn(src_part, rec, d_part) -> (phi, grad) is the per-rank gradient
    (normally ``Solver.grad`` without its stats); src are the source indices
    (flat), d the observed data [n_src, n_rec]; the gradient has ``shape``.
    A rank with no sources contributes zeros.  Without an initialised process
    group this is grad_fn on all sources."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        phi, g = grad_fn(src, rec, d)
        return float(phi), torch.as_tensor(g, dtype=torch.float64)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    part = shard(len(src), rank, world)
    if len(part) > 0:
        phi, g = grad_fn(src[part.start:part.stop], rec, d[part.start:part.stop])
        g = torch.as_tensor(g, dtype=torch.float64)
        if device is not None:
            g = g.to(device)
    else:
        phi = 0.0
        g = torch.zeros(shape, dtype=torch.float64, device=device)
    g = g.contiguous()
    phi_t = torch.tensor([float(phi)], dtype=torch.float64, device=g.device)
    dist.all_reduce(g, group=group)
    dist.all_reduce(phi_t, group=group)
    return float(phi_t.item()), g
