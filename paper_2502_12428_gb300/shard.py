"""Replica sharding of quartic batches across ranks (no collective on the data path).

Quartics are independent, so a batch splits into contiguous row ranges, one per rank; each rank runs the whole
hot path on its range and the int8 heights concatenate in rank order.  Under weak scaling every rank instead
takes its own n rows of the seeded generator, rows rank*n .. rank*n + n - 1.
"""


def shard_range(n_total, world, rank):
    """Contiguous [begin, end) of rank `rank` when n_total rows split over `world` ranks (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def weak_rows(n_per_rank, rank):
    """Generator rows of rank `rank` under weak scaling."""
    return rank * n_per_rank, (rank + 1) * n_per_rank
