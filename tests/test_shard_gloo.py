"""Multi-process split of OSPR sub-frames across ranks (world size 2, gloo, CPU): each rank
computes its contiguous range of sub-frames with the draw index advanced to its first
sub-frame, the partial replay sums are all-reduced, and the result equals the
single-process replay; the bits of every sub-frame are the same as well."""

import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import lut as olut
from oracle import ospr as oospr
from paper_2004_04049_gb300 import shard
from synthetic import blob_target

H = W = 32
N, L, SEED = 5, 257, 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        T = blob_target(H, W, 1000)
        table = olut.lut_codes(SEED, L)
        P = H * W
        first, count, start = shard.subframe_shard(N, 0, P, rank, world)
        bits, I, _ = oospr.ospr(T, count, table, L, SEED, start=start, stride=P)
        part = torch.from_numpy(I * count)
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        np.save(os.path.join(out_dir, f"I_{rank}.npy"), part.numpy() / N)
        np.save(os.path.join(out_dir, f"bits_{rank}.npy"), bits)
        np.save(os.path.join(out_dir, f"first_{rank}.npy"), np.array([first, count]))
    finally:
        dist.destroy_process_group()


def test_contiguous_ranges():
    for n in (0, 1, 5, 24, 37):
        for world in (1, 2, 3, 8):
            spans = [shard.contiguous_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1


def test_two_rank_subframe_split(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    T = blob_target(H, W, 1000)
    table = olut.lut_codes(SEED, L)
    bits_ref, I_ref, _ = oospr.ospr(T, N, table, L, SEED)
    for r in range(world):
        I = np.load(tmp_path / f"I_{r}.npy")
        assert np.max(np.abs(I - I_ref)) <= 1e-12 * I_ref.max()
        first, count = np.load(tmp_path / f"first_{r}.npy")
        assert np.array_equal(np.load(tmp_path / f"bits_{r}.npy"), bits_ref[first:first + count])


def _failing_worker(rank, world, port, out_dir):
    """Rank 1 fails before the frame's sum-reduction (it raises, as a crashed rank would);
    rank 0 must learn of it from the collective, within the process group's timeout,
    instead of waiting forever."""
    import datetime

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        raise RuntimeError("rank 1 fails before the reduction")
    T = blob_target(H, W, 1000)
    table = olut.lut_codes(SEED, L)
    first, count, start = shard.subframe_shard(N, 0, H * W, rank, world)
    _, I, _ = oospr.ospr(T, count, table, L, SEED, start=start, stride=H * W)
    part = torch.from_numpy(I * count)
    try:
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        outcome = "completed"
    except RuntimeError as e:
        outcome = "detected: " + str(e).splitlines()[0][:200]
    with open(os.path.join(out_dir, "rank0.txt"), "w") as f:
        f.write(outcome)


def test_failed_rank_is_detected(tmp_path):
    world = 2
    ctx = mp.start_processes(_failing_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                             join=False, start_method="spawn")
    for p in ctx.processes:
        p.join(120)
    codes = {i: p.exitcode for i, p in enumerate(ctx.processes)}
    assert codes[1] not in (0, None)                 # the failing rank exits with an error
    assert codes[0] == 0                             # the survivor returns, it does not hang
    assert (tmp_path / "rank0.txt").read_text().startswith("detected")
