"""Query sharding across ranks (one process per GPU).

Every query of a batch is independent and the textures are read-only, so a batch is
split into contiguous query ranges, one per rank, with the texture replicated on
every GPU; there is no exchange step.  A rank passes its range start as the lookup's
query_offset, so each query keeps the variates it would get in a single-process run
and the concatenated shard results equal the unsharded result.
"""


def shard(n, rank, world):
    """(start, count) of rank's contiguous share of n queries (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank %r of world %r" % (rank, world))
    base, extra = divmod(int(n), int(world))
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)
