"""Work partition across GPUs (one process per GPU).

OSPR sub-frames are independent given the draw index (Fig. 3: sub-frame s starts at draw
start + s*stride), so the N sub-frames of a frame split into contiguous ranges, one per
rank: rank r runs ospr_generate on its range with start_index advanced to its first
sub-frame, and the frame's replay is the sum of the ranks' partial sums divided by N (one
sum-reduction of H*W floats per frame). Frames of a batch are independent too and split
the same way with no exchange at all. GS is sequential per frame: frames only.
"""


def contiguous_range(n, rank, world):
    """[lo, hi) of n items for `rank` of `world`, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def subframe_shard(N, start_index, stride, rank, world):
    """(first sub-frame, count, start_index of that first sub-frame) for this rank."""
    lo, hi = contiguous_range(N, rank, world)
    return lo, hi - lo, start_index + lo * stride
