"""OSPR tile variants and chunking (the autotuner's search space) against the oracle, and
the autotuner itself. Every setting must give oracle parity; the tuner must install a
valid setting and record it in the cache file."""

import json
import os

import numpy as np
import pytest
import torch

from oracle import lut as olut
from oracle import ospr as oospr
from paper_2004_04049_gb300 import holo, pipeline
from parity import check_bits, check_replay
from synthetic import blob_target

pytestmark = pytest.mark.gpu

# (column IDFT variant, column DFT variant, row variant, chunk, groups)
SETTINGS = [(1, 1, 0, 16, 4), (0, 0, 1, 16, 4), (2, 1, 1, 2, 1), (1, 2, 1, 3, 2), (2, 2, 0, 5, 3), (0, 0, 0, 1, 1)]
_ORACLE = {}


def _oracle(T, H, W, N, L, seed):
    key = (H, W, N, L, seed)
    if key not in _ORACLE:
        table = olut.lut_codes(seed, L)
        ob, _, ex = oospr.ospr(T, N, table, L, seed, keep_fields=True)
        _ORACLE[key] = (ob, ex["re_h"])
    return _ORACLE[key]


# (1024, 1024, 5): with 16 pairs in flight the column IDFT of variant 0 runs 192 tiles on one
# CTA per SM, so a CTA takes a tile of a two-sub-frame slot and then one of the odd slot
@pytest.mark.parametrize("H,W,N", [(512, 512, 7), (1024, 1024, 4), (1024, 1024, 5), (2048, 512, 3), (512, 2048, 3)])
@pytest.mark.parametrize("setting", SETTINGS)
def test_setting_parity(cuda, H, W, N, setting):
    L, seed = 10007, 5
    T = blob_target(H, W, 1200)
    holo.ospr_tuning_set(H, W, *setting)
    try:
        t = torch.from_numpy(T).to(cuda)
        codes = pipeline.lut(seed, L, device=cuda)
        bits, I = pipeline.ospr(t, N, codes, L, 256, seed)
        torch.cuda.synchronize()
        gb = bits.cpu().numpy().view(np.uint32)
        gI = I.cpu().numpy()
    finally:
        holo.ospr_tuning_set(H, W)
    ob, re_h = _oracle(T, H, W, N, L, seed)
    check_bits(gb, ob, re_h, H * W)
    check_replay(gI, oospr.replay_from_bits(gb, H, W))


@pytest.mark.parametrize("H,W,N", [(1024, 1024, 4), (512, 1024, 3)])
@pytest.mark.parametrize("setting", [(1, 1, 0, 16, 4), (2, 2, 1, 3, 2)])
def test_fresnel_setting_parity(cuda, H, W, N, setting):
    # the Fresnel row pass under other tile variants, pairs in flight and groups
    L, seed, kappa = 10007, 5, 2.4e-4
    T = blob_target(H, W, 1200)
    holo.ospr_tuning_set(H, W, *setting)
    try:
        t = torch.from_numpy(T).to(cuda)
        codes = pipeline.lut(seed, L, device=cuda)
        fb, fI = pipeline.ospr_fresnel(t, N, kappa, codes, L, 256, seed)
        torch.cuda.synchronize()
    finally:
        holo.ospr_tuning_set(H, W)
    fgb = fb.cpu().numpy().view(np.uint32)
    fob, _, fex = oospr.ospr_fresnel(T, N, olut.lut_codes(seed, L), L, seed, kappa, keep_fields=True)
    check_bits(fgb, fob, fex["re_h"], H * W)
    check_replay(fI.cpu().numpy(), oospr.replay_from_bits_fresnel(fgb, H, W, kappa))


def test_autotune_installs_and_records(cuda, tmp_path):
    path = tmp_path / "tune.jsonl"
    os.environ["HOLO_TUNE_CACHE"] = str(path)
    try:
        ms = holo.ospr_autotune(512, 1024, 10, reps=2)
        t = holo.ospr_tuning_get(512, 1024)
    finally:
        os.environ.pop("HOLO_TUNE_CACHE", None)
    assert ms > 0.0
    assert t["col_ifft_variant"] in (0, 1, 2) and t["col_fft_variant"] in (0, 1, 2) and t["row_variant"] in (0, 1)
    assert 1 <= t["chunk"] <= 16 and 1 <= t["groups"] <= min(4, t["chunk"])
    rows = [json.loads(x) for x in path.read_text().splitlines()]
    rec = [r for r in rows if r["H"] == 512 and r["W"] == 1024]
    assert rec and rec[0]["chunk"] == t["chunk"] and rec[0]["col_ifft_variant"] == t["col_ifft_variant"]
    assert rec[0]["col_fft_variant"] == t["col_fft_variant"] and rec[0]["row_variant"] == t["row_variant"]
    # the tuned setting still computes the same bits as the default one, up to ties
    T = blob_target(512, 1024, 1201)
    tt = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(3, 4099, device=cuda)
    b1, _ = pipeline.ospr(tt, 10, codes, 4099, 256, 3)
    holo.ospr_tuning_set(512, 1024)
    b0, _ = pipeline.ospr(tt, 10, codes, 4099, 256, 3)
    torch.cuda.synchronize()
    diff = np.unpackbits(b1.cpu().numpy().view(np.uint8)) != np.unpackbits(b0.cpu().numpy().view(np.uint8))
    assert diff.mean() < 1e-4
