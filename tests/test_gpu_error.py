"""replay_error on the GPU against the oracle (Section 5.2, Eq. 3 reading)."""

import json
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import error as oerr
from paper_2004_04049_gb300 import pipeline
from parity import check_nmse

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H,W", [(1024, 1024), (256, 256), (33, 17), (1, 5), (2048, 1024),
                                 (1000, 1001),      # odd pixel count: the scalar path over 245 blocks
                                 (4096, 4096)])     # 4096 blocks: the last block loops over the partials
def test_matches_oracle(cuda, H, W):
    rng = np.random.default_rng(H * 7 + W)
    T = rng.random((H, W)).astype(np.float32)
    I = (T ** 2 * (1 + 0.2 * rng.standard_normal((H, W)))).astype(np.float32) ** 2
    g = pipeline.error(torch.from_numpy(I).to(cuda), torch.from_numpy(T).to(cuda)).cpu().numpy()
    o = oerr.replay_error(I, T)
    assert abs(g[0] - o[0]) <= 1e-6 * abs(o[0])
    check_nmse(g[1], o[1])
    check_nmse(g[2], o[2])


def test_golden_2x2(cuda, golden_dir):
    gd = json.load(open(os.path.join(golden_dir, "replay_error_2x2.json")))
    I = torch.tensor(gd["I"], dtype=torch.float32, device=cuda)
    T = torch.tensor(gd["T"], dtype=torch.float32, device=cuda)
    g = pipeline.error(I, T).cpu().numpy()
    assert abs(g[0] - float(Fraction(*gd["alpha"]))) < 1e-7
    assert abs(g[1] - float(Fraction(*gd["mse"]))) < 1e-7
    assert abs(g[2] - float(Fraction(*gd["nmse"]))) < 1e-7


def test_mask_and_unaligned_views(cuda):
    rng = np.random.default_rng(3)
    H, W = 64, 96
    T = rng.random((H, W)).astype(np.float32)
    I = rng.random((H, W)).astype(np.float32)
    mask = (rng.random((H, W)) < 0.3).astype(np.uint8)
    g = pipeline.error(torch.from_numpy(I).to(cuda), torch.from_numpy(T).to(cuda),
                       torch.from_numpy(mask).to(cuda)).cpu().numpy()
    o = oerr.replay_error(I, T, mask)
    check_nmse(g[2], o[2])
    check_nmse(g[1], o[1])
    # a view starting one float in: the scalar (unaligned) path
    big_i = torch.from_numpy(np.concatenate([[0.0], I.reshape(-1)]).astype(np.float32)).to(cuda)
    big_t = torch.from_numpy(np.concatenate([[0.0], T.reshape(-1)]).astype(np.float32)).to(cuda)
    g2 = pipeline.error(big_i[1:].view(H, W), big_t[1:].view(H, W)).cpu().numpy()
    o2 = oerr.replay_error(I, T)
    check_nmse(g2[2], o2[2])


def test_exact_replay_zero_error_and_reproducible(cuda):
    rng = np.random.default_rng(4)
    T = rng.random((512, 512)).astype(np.float32)
    I = (2.0 * T.astype(np.float64) ** 2).astype(np.float32)
    t, i = torch.from_numpy(T).to(cuda), torch.from_numpy(I).to(cuda)
    a = pipeline.error(i, t).cpu().numpy()
    b = pipeline.error(i, t).cpu().numpy()
    assert np.array_equal(a, b)
    assert abs(a[0] - 0.5) < 1e-6
    assert a[2] < 1e-12


def test_blocks_with_different_scales(cuda):
    # the error is formed per block of 4096 pixels at the block's own scale and combined
    # through an exact identity; blocks whose best scales differ widely (here 1, 3 and 0.2
    # by region) and a near-exact fit inside each block exercise every term of it
    rng = np.random.default_rng(5)
    H, W = 512, 768
    T = (0.2 + rng.random((H, W))).astype(np.float32)
    scale = np.where(np.arange(H * W).reshape(H, W) // 4096 % 3 == 0, 1.0,
                     np.where(np.arange(H * W).reshape(H, W) // 4096 % 3 == 1, 3.0, 0.2))
    I = (scale * T.astype(np.float64) ** 2 * (1 + 1e-3 * rng.standard_normal((H, W)))).astype(np.float32)
    g = pipeline.error(torch.from_numpy(I).to(cuda), torch.from_numpy(T).to(cuda)).cpu().numpy()
    o = oerr.replay_error(I, T)
    assert abs(g[0] - o[0]) <= 1e-6 * abs(o[0])
    check_nmse(g[1], o[1])
    check_nmse(g[2], o[2])


def test_bright_half_and_dark_noise_half(cuda):
    # half the frame a bright blob replayed faithfully, the other half a near-zero target
    # under replay noise: the dark blocks' own scales a_b are far from the global alpha
    # (|alpha - a_b| of the order of alpha), so the correction terms 2(alpha - a_b) S2_b and
    # (alpha - a_b)^2 sum_b I^2 carry most of the squared error there
    from synthetic import blob_target
    rng = np.random.default_rng(6)
    H, W = 1024, 1024
    T = blob_target(H, W, 777).astype(np.float64)
    T[H // 2:, :] = 1e-3 * rng.random((H // 2, W))
    I = T ** 2 * (1 + 0.05 * rng.standard_normal((H, W)))
    I[H // 2:, :] = 1e-4 * rng.random((H // 2, W))
    T, I = T.astype(np.float32), np.abs(I).astype(np.float32)
    g = pipeline.error(torch.from_numpy(I).to(cuda), torch.from_numpy(T).to(cuda)).cpu().numpy()
    o = oerr.replay_error(I, T)
    assert abs(g[0] - o[0]) <= 1e-6 * abs(o[0])
    check_nmse(g[1], o[1])
    check_nmse(g[2], o[2])
