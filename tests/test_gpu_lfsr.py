"""m-sequence phase codes (Section 7's PRNG alternative) on the GPU: bit-exact against the
oracle's register, including far jumps, and an OSPR frame whose every sub-frame pixel draws
its own m-sequence code, against the oracle (tolerances: tests/parity.py)."""

import numpy as np
import pytest
import torch

from oracle import lfsr as olfsr
from oracle import ospr as oospr
from paper_2004_04049_gb300 import holo, pipeline
from parity import check_bits, check_replay
from synthetic import blob_target

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,start,count,levels", [(1, 0, 5000, 256), (0x2545F491, 10 ** 9 + 7, 3001, 256),
                                                     (12345, 777, 4099, 4), (7, 2 ** 40 + 3, 1000, 2),
                                                     (2 ** 31 - 1, 513, 1, 256), (99, 0, 70000, 16)])
def test_codes_bit_exact(cuda, seed, start, count, levels):
    d = torch.empty(count, dtype=torch.uint8, device=cuda)
    holo.lfsr_build(seed, start, count, levels, d)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy().astype(np.int64), olfsr.codes(seed, start, count, levels))


def test_codes_unaligned_output(cuda):
    # an output pointer off a 16-byte boundary takes the byte-store path
    d = torch.zeros(4100, dtype=torch.uint8, device=cuda)
    holo.lfsr_build(321, 10, 4097, 256, d[3:])
    torch.cuda.synchronize()
    got = d.cpu().numpy().astype(np.int64)
    assert np.array_equal(got[3:3 + 4097], olfsr.codes(321, 10, 4097))
    assert got[:3].sum() == 0


def test_ospr_with_m_sequence_codes(cuda):
    H = W = 128
    N = 4
    P = H * W
    T = blob_target(H, W, 1003)
    seed = 0x1D872B41
    d = torch.empty(N * P, dtype=torch.uint8, device=cuda)
    holo.lfsr_build(seed, 0, N * P, 256, d)
    t = torch.from_numpy(T).to(cuda)
    bits, I = pipeline.ospr(t, N, d, N * P, 256, 0)
    torch.cuda.synchronize()
    gb = bits.cpu().numpy().view(np.uint32)
    table = olfsr.codes(seed, 0, N * P)
    ob, _, ex = oospr.ospr(T, N, table, N * P, 0, keep_fields=True)
    check_bits(gb, ob, ex["re_h"], P)
    check_replay(I.cpu().numpy(), oospr.replay_from_bits(gb, H, W))
