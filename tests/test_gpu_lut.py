"""lut_build on the GPU against the oracle's table (Section 4; 8-bit codes, Section 5.2):
codes bit-exact, (cos, sin) within float32 rounding of the float64 values."""

import numpy as np
import pytest
import torch

from oracle import lut as olut
from paper_2004_04049_gb300 import holo, pipeline

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,L,levels", [(7, 4096, 256), (1234567, 10007, 256), (3, 1, 256),
                                           (5, 97, 2), (11, 1000, 16), (42, (1 << 20) + 7, 256)])
def test_codes_bit_exact(cuda, seed, L, levels):
    codes, cs = pipeline.lut(seed, L, levels, device=cuda, with_cs=True)
    torch.cuda.synchronize()
    g = codes.cpu().numpy().astype(np.int64)
    o = olut.lut_codes(seed, L, levels)
    assert np.array_equal(g, o)
    th = olut.phase_of_codes(o, levels)
    c = cs.cpu().numpy().reshape(-1, 2).astype(np.float64)
    assert np.max(np.abs(c[:, 0] - np.cos(th))) <= 6e-8
    assert np.max(np.abs(c[:, 1] - np.sin(th))) <= 6e-8


def test_rejects_bad_arguments(cuda):
    codes = torch.empty(16, dtype=torch.uint8, device=cuda)
    with pytest.raises(holo.HoloError):
        holo.lut_build(1, 16, 257, codes)
    with pytest.raises(holo.HoloError):
        holo.lut_build(1, -3, 256, codes)
