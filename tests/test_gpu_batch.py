"""ospr_generate_batch and its CUDA graph: a batch of mixed-shape frames, each with its
own table, gives exactly the per-frame results (the same kernels run per frame, only
spread over internal streams), as a direct call and as a replayed graph."""

import numpy as np
import pytest
import torch

from paper_2004_04049_gb300 import holo, pipeline
from synthetic import blob_target, noise_target

pytestmark = pytest.mark.gpu

FRAMES = [  # H, W, N, L, seed
    (128, 128, 5, 1031, 11),
    (256, 512, 8, 4099, 12),
    (64, 64, 1, 0, 13),
    (512, 256, 3, holo.L_UNREPEATED, 14),
    (1024, 1024, 6, 10007, 15),
    (256, 256, 32, 65537, 16),
]


def _alloc(cuda, spec, k):
    H, W, N, L, seed = spec
    T = blob_target(H, W, 1100 + k) if k % 2 == 0 else noise_target(H, W, 2100 + k)
    return {
        "T": torch.from_numpy(T).to(cuda),
        "codes": torch.zeros(max(L, 1), dtype=torch.uint8, device=cuda),
        "bits": torch.zeros((N, H * W // 32), dtype=torch.int32, device=cuda),
        "I": torch.zeros((H, W), dtype=torch.float32, device=cuda),
        "err": torch.zeros(3, dtype=torch.float64, device=cuda),
    }


def _descs(bufs):
    out = []
    for (H, W, N, L, seed), b in zip(FRAMES, bufs):
        out.append(holo.frame_desc(b["T"], H, W, N, b["codes"], L, 256, seed, L > 0, 0, 0,
                                   b["bits"], b["I"], b["err"]))
    return holo.frame_array(out)


def _per_frame(cuda, bufs):
    ref = []
    for (H, W, N, L, seed), b in zip(FRAMES, bufs):
        codes = pipeline.lut(seed, L, device=cuda) if L > 0 else None
        bits, I = pipeline.ospr(b["T"], N, codes, L, 256, seed)
        err = pipeline.error(I, b["T"])
        ref.append((bits.cpu().numpy(), I.cpu().numpy(), err.cpu().numpy()))
    return ref


def _check(bufs, ref):
    for k, (b, r) in enumerate(zip(bufs, ref)):
        assert np.array_equal(b["bits"].cpu().numpy(), r[0]), k
        assert np.array_equal(b["I"].cpu().numpy(), r[1]), k
        assert np.array_equal(b["err"].cpu().numpy(), r[2]), k


def test_batch_equals_per_frame(cuda):
    bufs = [_alloc(cuda, s, k) for k, s in enumerate(FRAMES)]
    arr = _descs(bufs)
    ws = torch.empty(holo.ospr_batch_workspace_size(arr), dtype=torch.uint8, device=cuda)
    holo.ospr_generate_batch(arr, holo.HOLO_FP32, ws)
    torch.cuda.synchronize()
    _check(bufs, _per_frame(cuda, bufs))


@pytest.mark.parametrize("prec", [holo.HOLO_FP16X2, holo.HOLO_BF16X2])
def test_batch_tensor_core_equals_per_frame(cuda, prec):
    """Frames of the tensor-core shapes in one batch call in a split precision equal the
    per-frame calls in that precision (same tcgen05 kernels, internal streams)."""
    specs = [(1024, 1024, 6, 10007, 21), (2048, 1024, 3, 4099, 22), (1024, 2048, 4, 0, 23)]
    bufs, descs = [], []
    for k, (H, W, N, L, seed) in enumerate(specs):
        b = _alloc(cuda, (H, W, N, L, seed), k)
        bufs.append(b)
        descs.append(holo.frame_desc(b["T"], H, W, N, b["codes"], L, 256, seed, L > 0, 0, 0,
                                     b["bits"], b["I"], b["err"]))
    arr = holo.frame_array(descs)
    holo.holo_tc_status(clear=True)
    ws = torch.empty(holo.ospr_batch_workspace_size(arr, prec), dtype=torch.uint8, device=cuda)
    holo.ospr_generate_batch(arr, prec, ws)
    torch.cuda.synchronize()
    for k, ((H, W, N, L, seed), b) in enumerate(zip(specs, bufs)):
        codes = pipeline.lut(seed, L, device=cuda) if L > 0 else None
        bits, I = pipeline.ospr(b["T"], N, codes, L, 256, seed, precision=prec)
        err = pipeline.error(I, b["T"])
        torch.cuda.synchronize()
        assert torch.equal(b["bits"], bits) and torch.equal(b["I"], I) and torch.equal(b["err"], err), k
    assert holo.holo_tc_status() == 0


def test_graph_replays_batch(cuda):
    bufs = [_alloc(cuda, s, k) for k, s in enumerate(FRAMES)]
    arr = _descs(bufs)
    ws = torch.empty(holo.ospr_batch_workspace_size(arr), dtype=torch.uint8, device=cuda)
    g = holo.ospr_batch_graph_create(arr, holo.HOLO_FP32, ws)
    try:
        for b in bufs:
            b["I"].zero_()
            b["bits"].zero_()
        holo.holo_graph_launch(g)
        torch.cuda.synchronize()
        _check(bufs, _per_frame(cuda, bufs))
        # new target contents in the same buffers: the replay follows them
        for k, b in enumerate(bufs):
            b["T"].copy_(torch.flip(b["T"], dims=[0]))
        holo.holo_graph_launch(g)
        torch.cuda.synchronize()
        _check(bufs, _per_frame(cuda, bufs))
    finally:
        holo.holo_graph_destroy(g)


def test_batch_reports_bad_frame(cuda):
    bufs = [_alloc(cuda, s, k) for k, s in enumerate(FRAMES[:2])]
    descs = [holo.frame_desc(bufs[0]["T"], 128, 128, 5, bufs[0]["codes"], 1031, 256, 1, True, 0, 0,
                             bufs[0]["bits"], bufs[0]["I"], None),
             holo.frame_desc(bufs[1]["T"], 100, 512, 8, None, 0, 256, 1, False, 0, 0,
                             bufs[1]["bits"], bufs[1]["I"], None)]
    arr = holo.frame_array(descs)
    with pytest.raises(holo.HoloError) as ei:
        holo.ospr_batch_workspace_size(arr)
    assert "frame 1" in str(ei.value)


def test_batch_with_host_buffers(cuda):
    # the same frames with their targets coming from and their results going back to
    # page-locked host memory, the copies issued by the library around each frame
    bufs = [_alloc(cuda, s, k) for k, s in enumerate(FRAMES)]
    arr = _descs(bufs)
    ws = torch.empty(holo.ospr_batch_workspace_size(arr), dtype=torch.uint8, device=cuda)
    holo.ospr_generate_batch(arr, holo.HOLO_FP32, ws)
    torch.cuda.synchronize()
    ref = [(b["bits"].cpu(), b["I"].cpu(), b["err"].cpu()) for b in bufs]
    hosts, h = [], []
    for b in bufs:
        t = b["T"].cpu().pin_memory()
        b["T"].zero_()                                  # the call must copy the target in
        o = {"T": t, "bits": torch.zeros(b["bits"].shape, dtype=torch.int32).pin_memory(),
             "I": torch.zeros(b["I"].shape, dtype=torch.float32).pin_memory(),
             "err": torch.zeros(3, dtype=torch.float64).pin_memory()}
        h.append(o)
        hosts.append(holo.frame_host(o["T"], o["bits"], o["I"], o["err"]))
    holo.ospr_generate_batch_host(arr, holo.frame_host_array(hosts), holo.HOLO_FP32, ws)
    torch.cuda.synchronize()
    for k, (o, r) in enumerate(zip(h, ref)):
        assert torch.equal(o["bits"], r[0]), k
        assert torch.equal(o["I"], r[1]), k
        assert torch.equal(o["err"], r[2]), k
    with pytest.raises(holo.HoloError) as ei:
        bad = holo.frame_host_array([holo.frame_host(None, None, h[0]["I"], None)] +
                                    [holo.frame_host() for _ in bufs[1:]])
        nodev = holo.frame_array([holo.frame_desc(bufs[0]["T"], *FRAMES[0][:3], bufs[0]["codes"], FRAMES[0][3], 256,
                                                  FRAMES[0][4], True, 0, 0, bufs[0]["bits"], None, None)] +
                                 list(_descs(bufs))[1:])
        holo.ospr_generate_batch_host(nodev, bad, holo.HOLO_FP32, ws)
    assert ei.value.status == holo.HOLO_EINVAL


def test_batch_with_host_buffers_more_frames_than_streams(cuda):
    """Twelve frames on the library's eight internal streams (four streams run two frames,
    the second one's target copied in after the first one's results went out). Two calls
    in a row, the second with other targets, each equal to the device-resident batch."""
    specs = FRAMES + [(H, W, N, L, seed + 100) for (H, W, N, L, seed) in FRAMES]
    bufs = [_alloc(cuda, sp, k) for k, sp in enumerate(specs)]
    arr = holo.frame_array([holo.frame_desc(b["T"], H, W, N, b["codes"], L, 256, seed, L > 0, 0, 0,
                                            b["bits"], b["I"], b["err"])
                            for (H, W, N, L, seed), b in zip(specs, bufs)])
    ws = torch.empty(holo.ospr_batch_workspace_size(arr), dtype=torch.uint8, device=cuda)
    for rnd in range(2):
        if rnd == 1:
            for b in bufs:
                b["T"].copy_(torch.flip(b["T"], dims=[1]))
        holo.ospr_generate_batch(arr, holo.HOLO_FP32, ws)
        torch.cuda.synchronize()
        ref = [(b["bits"].cpu(), b["I"].cpu(), b["err"].cpu()) for b in bufs]
        h, hosts = [], []
        for b in bufs:
            o = {"T": b["T"].cpu().pin_memory(), "bits": torch.zeros(b["bits"].shape, dtype=torch.int32).pin_memory(),
                 "I": torch.zeros(b["I"].shape, dtype=torch.float32).pin_memory(),
                 "err": torch.zeros(3, dtype=torch.float64).pin_memory()}
            b["T"].zero_()
            h.append(o)
            hosts.append(holo.frame_host(o["T"], o["bits"], o["I"], o["err"]))
        holo.ospr_generate_batch_host(arr, holo.frame_host_array(hosts), holo.HOLO_FP32, ws)
        torch.cuda.synchronize()
        for k, (o, r) in enumerate(zip(h, ref)):
            assert torch.equal(o["bits"], r[0]) and torch.equal(o["I"], r[1]) and torch.equal(o["err"], r[2]), \
                (rnd, k)
            assert torch.equal(bufs[k]["T"].cpu(), o["T"]), (rnd, k)   # the target was copied in


def test_batch_calls_from_two_threads(cuda):
    # two host threads issue batch calls at the same time, each on its own stream with its
    # own frames and workspace; the calls share the library's internal streams and events,
    # so they must not interleave their forks and joins: each thread's results equal the
    # per-frame results
    import threading

    sets = []
    for r in range(2):
        bufs = [_alloc(cuda, s, k + 10 * r) for k, s in enumerate(FRAMES)]
        arr = _descs(bufs)
        ws = torch.empty(holo.ospr_batch_workspace_size(arr), dtype=torch.uint8, device=cuda)
        sets.append((bufs, arr, ws, torch.cuda.Stream(cuda)))
    torch.cuda.synchronize()
    errors = []

    def work(bufs, arr, ws, st):
        try:
            torch.cuda.set_device(cuda)
            for _ in range(3):
                holo.ospr_generate_batch(arr, holo.HOLO_FP32, ws, stream=st)
            st.synchronize()
        except Exception as e:   # reported after the join
            errors.append(e)

    threads = [threading.Thread(target=work, args=s) for s in sets]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    for bufs, _, _, _ in sets:
        _check(bufs, _per_frame(cuda, bufs))


# ----------------------------------------------------------------- persistent ----
PFRAMES = [  # H, W, N, L, seed: the shapes of the mixed batch, odd and even N, several tables
    (512, 512, 5, 1031, 21),
    (1024, 2048, 8, 4099, 22),
    (2048, 512, 3, 65537, 23),
    (1024, 1024, 24, 10007, 24),
    (512, 1024, 1, 0, 25),
    (2048, 2048, 4, holo.L_UNREPEATED, 26),
    (512, 512, 33, 2 ** 18, 27),          # more pairs than one chunk: accumulation across chunks
]


def _pdescs(bufs, specs):
    return holo.frame_array([holo.frame_desc(b["T"], H, W, N, b["codes"], L, 256, seed, L > 0, 0, 0,
                                             b["bits"], b["I"], b["err"])
                             for (H, W, N, L, seed), b in zip(specs, bufs)])


def _pref(cuda, bufs, specs):
    """Per-frame calls under the persistent launch's tiles: variant 0, the shape's chunking."""
    ref = []
    for (H, W, N, L, seed), b in zip(specs, bufs):
        t = holo.ospr_tuning_get(H, W)
        holo.ospr_tuning_set(H, W, 0, 0, 0, t["chunk"], t["groups"])
        try:
            codes = pipeline.lut(seed, L, device=cuda) if L > 0 else None
            bits, I = pipeline.ospr(b["T"], N, codes, L, 256, seed)
            err = pipeline.error(I, b["T"])
            ref.append((bits.cpu().numpy(), I.cpu().numpy(), err.cpu().numpy()))
        finally:
            holo.ospr_tuning_set(H, W, t["col_ifft_variant"], t["col_fft_variant"], t["row_variant"], t["chunk"],
                                 t["groups"])
    return ref


def test_persistent_equals_per_frame(cuda):
    bufs = [_alloc(cuda, s, k) for k, s in enumerate(PFRAMES)]
    arr = _pdescs(bufs, PFRAMES)
    ws = torch.empty(holo.ospr_batch_persistent_workspace_size(arr), dtype=torch.uint8, device=cuda)
    holo.holo_tc_status(clear=True)
    holo.ospr_generate_batch_persistent(arr, ws)
    torch.cuda.synchronize()
    assert holo.holo_tc_status() == 0
    holo.holo_check()
    _check(bufs, _pref(cuda, bufs, PFRAMES))
    # a second launch on the same workspace (counters cleared by the call) and the graph
    for b in bufs:
        b["I"].zero_()
        b["bits"].zero_()
        b["err"].zero_()
    g = holo.ospr_batch_persistent_graph_create(arr, ws)
    try:
        for _ in range(2):
            holo.holo_graph_launch(g)
        torch.cuda.synchronize()
    finally:
        holo.holo_graph_destroy(g)
    assert holo.holo_tc_status() == 0
    _check(bufs, _pref(cuda, bufs, PFRAMES))


def test_persistent_bounded_wait_expires(cuda, monkeypatch):
    # a test hook makes the first dependency wait wait for a count nothing reaches: the wait
    # gives up after its limit, the fault flag is set, every CTA stops, and the context
    # stays usable
    bufs = [_alloc(cuda, s, k) for k, s in enumerate(PFRAMES[:2])]
    arr = _pdescs(bufs, PFRAMES[:2])
    ws = torch.empty(holo.ospr_batch_persistent_workspace_size(arr), dtype=torch.uint8, device=cuda)
    holo.holo_tc_status(clear=True)
    monkeypatch.setenv("HOLO_FAULT_INJECT", "persist_wait")
    holo.ospr_generate_batch_persistent(arr, ws, wait_limit_us=2000)
    torch.cuda.synchronize()
    monkeypatch.delenv("HOLO_FAULT_INJECT")
    assert holo.holo_tc_status() == 1
    with pytest.raises(holo.HoloError) as ei:
        holo.holo_check()
    assert ei.value.status == holo.HOLO_ETIMEOUT
    assert holo.holo_tc_status(clear=True) == 1
    assert holo.holo_tc_status() == 0
    holo.ospr_generate_batch_persistent(arr, ws)
    torch.cuda.synchronize()
    assert holo.holo_tc_status() == 0
    _check(bufs, _pref(cuda, bufs, PFRAMES[:2]))


def test_persistent_rejects_unsupported(cuda):
    bufs = [_alloc(cuda, s, k) for k, s in enumerate(FRAMES[:1])]   # 128x128
    arr = _descs(bufs)[:1]
    with pytest.raises(holo.HoloError) as ei:
        holo.ospr_batch_persistent_workspace_size(holo.frame_array(list(arr)))
    assert ei.value.status == holo.HOLO_EUNSUPPORTED


def test_persistent_frames_without_error_or_bits(cuda):
    # frames that ask for no error (done after their last finalize item) and no bits,
    # following a frame on the same workspace slot (one slot: every frame waits for the
    # previous one), against the per-frame kernels under the same tiles
    specs = [(1024, 512, 6, 4099, 31), (512, 512, 3, 1031, 32), (512, 1024, 4, 0, 33)]
    bufs = [_alloc(cuda, s, k + 40) for k, s in enumerate(specs)]
    arr = holo.frame_array([holo.frame_desc(b["T"], H, W, N, b["codes"], L, 256, seed, L > 0, 0, 0,
                                            b["bits"] if k != 1 else None, b["I"], b["err"] if k != 0 else None)
                            for k, ((H, W, N, L, seed), b) in enumerate(zip(specs, bufs))])
    import os
    os.environ["HOLO_BATCH_STREAMS"] = "1"
    try:
        ws = torch.empty(holo.ospr_batch_persistent_workspace_size(arr), dtype=torch.uint8, device=cuda)
        holo.holo_tc_status(clear=True)
        holo.ospr_generate_batch_persistent(arr, ws)
        torch.cuda.synchronize()
    finally:
        del os.environ["HOLO_BATCH_STREAMS"]
    assert holo.holo_tc_status() == 0
    ref = _pref(cuda, bufs, specs)
    for k, (b, r) in enumerate(zip(bufs, ref)):
        assert np.array_equal(b["I"].cpu().numpy(), r[1]), k
        if k != 1:
            assert np.array_equal(b["bits"].cpu().numpy(), r[0]), k
        if k != 0:
            assert np.array_equal(b["err"].cpu().numpy(), r[2]), k
