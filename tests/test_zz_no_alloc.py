"""ospr_generate_noalloc: OSPR for callers that cannot allocate device memory.

Some callers can't call cudaMalloc or pass a workspace: a display loop with a hard
per-frame deadline (allocation can synchronise the device), a plug-in whose host
application owns all device memory, or a host that partitions device memory once at
start-up. For them the library keeps one fixed 32 MiB scratch array in device memory.
This test calls that entry point through the C ABI, twice in a row with different
inputs, and checks each result against ospr_generate with a caller workspace: identical
bits, replay within the parity tolerance. It runs last (file name) so that a failure here
stops a -x run only after every other test has run, and it passes in a fresh process too.
"""

import numpy as np
import pytest
import torch

from paper_2004_04049_gb300 import holo, pipeline
from parity import REPLAY_REL
from synthetic import blob_target, noise_target

pytestmark = pytest.mark.gpu


def _both(cuda, T, N, L, seed):
    H, W = T.shape
    t = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(seed, L, device=cuda)
    b_ws, I_ws = pipeline.ospr(t, N, codes, L, 256, seed)
    b_na = torch.empty_like(b_ws)
    I_na = torch.empty_like(I_ws)
    holo.ospr_generate_noalloc(t, H, W, N, codes, L, 256, seed, 0, 0, holo.HOLO_FP32, b_na, I_na)
    holo.holo_check()
    return b_ws.cpu().numpy(), I_ws.cpu().numpy(), b_na.cpu().numpy(), I_na.cpu().numpy()


def test_noalloc_matches_workspace_path_twice(cuda):
    # 1024x1024, N = 24: the scratch holds 3 sub-frame pairs, so the call runs 4 chunks and
    # carries the accumulator across them; then a different shape and target reuses the
    # same scratch, which still holds the first call's data
    cases = [(blob_target(1024, 1024, 1000), 24, 10007, 7),
             (noise_target(256, 512, 2003), 5, 4099, 3)]
    for T, N, L, seed in cases:
        b_ws, I_ws, b_na, I_na = _both(cuda, T, N, L, seed)
        assert np.array_equal(b_na, b_ws)
        rel = np.abs(I_na.astype(np.float64) - I_ws).max() / np.abs(I_ws).max()
        assert rel <= REPLAY_REL, rel


def test_noalloc_rejects_shapes_beyond_scratch(cuda):
    H = W = 2048
    t = torch.zeros((H, W), dtype=torch.float32, device=cuda)
    bits = torch.empty((4, H * W // 32), dtype=torch.int32, device=cuda)
    with pytest.raises(holo.HoloError) as ei:
        holo.ospr_generate_noalloc(t, H, W, 4, None, 0, 256, 0, 0, 0, holo.HOLO_FP32, bits, None)
    assert ei.value.status == holo.HOLO_EWORKSPACE
    assert "scratch" in holo.last_error()
