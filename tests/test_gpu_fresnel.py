"""ospr_generate_fresnel on the GPU against the float64 oracle (Fresnel propagation, the
near-field regime of Section 2; the quadratic-phase model is stated in include/holo.h).

Element-by-element parity at sizes the oracle finishes in seconds: several FFT tiles,
non-square shapes, odd and even N, every table mode and a range of kappa, stage-wise
(the oracle replays the GPU's own bits). Tolerances: tests/parity.py.
"""

import numpy as np
import pytest
import torch

from oracle import lut as olut
from oracle import ospr as oospr
from paper_2004_04049_gb300 import holo, pipeline
from parity import check_bits, check_replay
from synthetic import blob_target, noise_target

pytestmark = pytest.mark.gpu

CASES = [
    # H, W, N, L, kappa, target
    (64, 64, 3, 1031, 0.01, "blob"),
    (128, 256, 4, 4099, 0.002, "noise"),
    (256, 128, 5, 10007, 7.5e-4, "blob"),
    (64, 128, 2, holo.L_UNREPEATED, 0.05, "blob"),
    (128, 128, 3, 0, 0.004, "blob"),          # flat phase: the lens-like hologram of the target
    (512, 512, 2, 65537, 2.4e-4, "noise"),    # pitch 8 um, 532 nm, z = 0.5 m
    (64, 4096, 2, 10007, 1e-4, "blob"),       # extreme aspect ratios
    (4096, 64, 2, 10007, 1e-4, "noise"),
    (1024, 1024, 2, 1048583, 2.4e-4, "blob"),   # the benchmark's frame size
]


def _gpu(cuda, T, N, L, kappa, seed=7, levels=256):
    t = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(seed, L, levels, device=cuda) if L > 0 else None
    bits, I = pipeline.ospr_fresnel(t, N, kappa, codes, L, levels, seed)
    torch.cuda.synchronize()
    return bits.cpu().numpy().view(np.uint32), I.cpu().numpy()


@pytest.mark.parametrize("H,W,N,L,kappa,kind", CASES)
def test_fresnel_parity(cuda, H, W, N, L, kappa, kind):
    T = blob_target(H, W, 1000) if kind == "blob" else noise_target(H, W, 2000)
    gb, gI = _gpu(cuda, T, N, L, kappa)
    table = olut.lut_codes(7, L) if L > 0 else None
    ob, oI, ex = oospr.ospr_fresnel(T, N, table, L, 7, kappa, keep_fields=True)
    check_bits(gb, ob, ex["re_h"], H * W)
    check_replay(gI, oospr.replay_from_bits_fresnel(gb, H, W, kappa))
    assert abs(gI.sum() / (H * W) - 1.0) < 1e-4          # unitarity: energy P per sub-frame


def test_kappa_zero_matches_the_far_field_path(cuda):
    H, W, N, L = 128, 128, 6, 4099
    T = blob_target(H, W, 1005)
    t = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(7, L, device=cuda)
    fb, fI = pipeline.ospr_fresnel(t, N, 0.0, codes, L, 256, 7)
    b, I = pipeline.ospr(t, N, codes, L, 256, 7)
    torch.cuda.synchronize()
    ob, _, ex = oospr.ospr(T, N, olut.lut_codes(7, L), L, 7, keep_fields=True)
    check_bits(fb.cpu().numpy().view(np.uint32), ob, ex["re_h"], H * W)
    check_replay(fI.cpu().numpy(), I.cpu().numpy().astype(np.float64))


def test_replay_is_not_centrosymmetric(cuda):
    H = W = 256
    T = noise_target(H, W, 2003)
    _, gI = _gpu(cuda, T, 4, 10007, 0.003)
    twin = np.roll(np.flip(gI), shift=(1, 1), axis=(0, 1))
    assert np.abs(gI - twin).max() / gI.max() > 1e-2


def test_workspace_and_arguments(cuda):
    H = W = 64
    t = torch.from_numpy(blob_target(H, W, 1000)).to(cuda)
    need = holo.ospr_fresnel_workspace_size(H, W, 3)
    assert need >= 3 * H * W * 8 + H * W * 4 + (H + W) * 8
    ws = torch.empty(need - 256, dtype=torch.uint8, device=cuda)
    bits = torch.empty((3, H * W // 32), dtype=torch.int32, device=cuda)
    with pytest.raises(holo.HoloError) as ei:
        holo.ospr_generate_fresnel(t, H, W, 3, None, 0, 256, 0, 0, 0, 0.01, bits, None, ws)
    assert ei.value.status == holo.HOLO_EWORKSPACE
    ws = torch.empty(need, dtype=torch.uint8, device=cuda)
    with pytest.raises(holo.HoloError) as ei:
        holo.ospr_generate_fresnel(t, H, W, 3, None, 0, 256, 0, 0, 0, float("nan"), bits, None, ws)
    assert ei.value.status == holo.HOLO_EINVAL
