"""Tensor-core DFT-32 precisions (HOLO_FP16X2, HOLO_BF16X2: split hi/lo operands, float32
accumulation) against the float64 oracle, with the same tolerances as the float32 path;
the measured errors are printed for the record."""

import numpy as np
import pytest
import torch

from oracle import error as oerr
from oracle import lut as olut
from oracle import ospr as oospr
from paper_2004_04049_gb300 import holo, pipeline
from parity import check_bits, check_nmse, check_replay, unpack
from synthetic import blob_target, noise_target

pytestmark = pytest.mark.gpu

_ORACLE = {}


def _oracle(T, H, W, N, L, seed):
    key = (H, W, N, L, seed)
    if key not in _ORACLE:
        table = olut.lut_codes(seed, L)
        ob, oI, ex = oospr.ospr(T, N, table, L, seed, keep_fields=True)
        _ORACLE[key] = (ob, oI, ex["re_h"])
    return _ORACLE[key]


@pytest.mark.parametrize("prec", [holo.HOLO_FP16X2, holo.HOLO_BF16X2])
@pytest.mark.parametrize("H,W,N,kind", [(1024, 1024, 6, "blob"), (2048, 1024, 3, "noise"),
                                        (1024, 2048, 3, "blob")])
def test_tc_parity(cuda, prec, H, W, N, kind):
    L, seed = 10007, 9
    T = blob_target(H, W, 1300) if kind == "blob" else noise_target(H, W, 2300)
    t = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(seed, L, device=cuda)
    holo.holo_tc_status(clear=True)
    bits, I = pipeline.ospr(t, N, codes, L, 256, seed, precision=prec)
    b32, I32 = pipeline.ospr(t, N, codes, L, 256, seed)
    err = pipeline.error(I, t)
    torch.cuda.synchronize()
    gb = bits.cpu().numpy().view(np.uint32)
    gI = I.cpu().numpy()
    ob, oI, re_h = _oracle(T, H, W, N, L, seed)
    agree, undecidable = check_bits(gb, ob, re_h, H * W)
    rel = check_replay(gI, oospr.replay_from_bits(gb, H, W))
    o_stage = oerr.replay_error(gI, T)
    check_nmse(err.cpu().numpy()[2], o_stage[2])
    o_e2e = oerr.replay_error(oI, T)
    nmse_rel = abs(err.cpu().numpy()[2] - o_e2e[2]) / o_e2e[2]
    vs32 = np.mean(unpack(gb, H * W) == unpack(b32.cpu().numpy().view(np.uint32), H * W))
    print(f"prec={prec} {H}x{W} N={N}: bits agree {agree:.7f} (vs fp32 path {vs32:.7f}), "
          f"replay rel {rel:.2e}, nmse rel vs oracle {nmse_rel:.2e}")
    assert vs32 >= 0.9999
    assert holo.holo_tc_status() == 0


def test_tc_rejects_other_shapes(cuda):
    t = torch.zeros((512, 512), dtype=torch.float32, device=cuda)
    with pytest.raises(holo.HoloError) as ei:
        pipeline.ospr(t, 2, None, 0, 256, 0, precision=holo.HOLO_BF16X2)
    assert ei.value.status == holo.HOLO_EUNSUPPORTED
