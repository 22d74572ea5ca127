"""gs_iterate_batch: B targets of one shape in the same launches. Each target's codes,
replay, errors and final state equal gs_iterate's for that target with the table draw
continued by b*H*W (bit for bit: the same kernels run per target, grid.y selecting the
target), and the first iteration of every target meets the oracle's bounds (Section 2;
Fig. 3 continuation across frames). Tolerances: tests/parity.py."""

import numpy as np
import pytest
import torch

from oracle import fft as offt
from oracle import gs as ogs
from oracle import lut as olut
from paper_2004_04049_gb300 import holo, pipeline
from parity import NMSE_REL, check_codes
from synthetic import blob_target, noise_target

pytestmark = pytest.mark.gpu


def _batch(cuda, T, iters, levels=256, codes=None, L=0, seed=0, start=0, init=None, states_in=None,
           precision=holo.HOLO_FP32):
    B, H, W = T.shape
    ws = torch.empty(holo.gs_batch_workspace_size(B, H, W, iters, precision), dtype=torch.uint8, device=cuda)
    out = {"codes": torch.empty((B, H, W), dtype=torch.uint8, device=cuda),
           "replay": torch.empty((B, H, W), dtype=torch.float32, device=cuda),
           "err": torch.empty((B, iters), dtype=torch.float64, device=cuda),
           "state": torch.empty((B, H, W, 2), dtype=torch.float32, device=cuda)}
    holo.gs_iterate_batch(T, B, H, W, iters, levels, init, codes, L, 256, seed, start, precision,
                          out["codes"], out["replay"], out["err"], states_in, out["state"], ws)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("H,W,B,iters,levels", [(256, 512, 3, 5, 256), (64, 64, 7, 3, 2), (1024, 1024, 2, 2, 256)])
def test_batch_equals_per_target_calls(cuda, H, W, B, iters, levels):
    T = torch.stack([torch.from_numpy(blob_target(H, W, 3000 + b) if b % 2 == 0 else noise_target(H, W, 3100 + b))
                     for b in range(B)]).to(cuda)
    L, seed, start = 10007, 4, 123
    codes = pipeline.lut(seed, L, device=cuda)
    got = _batch(cuda, T, iters, levels, codes, L, seed, start)
    P = H * W
    for b in range(B):
        ref = pipeline.gs(T[b], iters, levels, codes, L, 256, seed, start=start + b * P, want_state=True)
        torch.cuda.synchronize()
        assert torch.equal(got["codes"][b], ref["codes"]), b
        assert torch.equal(got["replay"][b], ref["replay"]), b
        assert torch.equal(got["err"][b], ref["err"]), b
        assert torch.equal(got["state"][b], ref["state"]), b


@pytest.mark.parametrize("prec", [holo.HOLO_FP16X2, holo.HOLO_BF16X2])
def test_batch_tensor_core_equals_per_target_calls(cuda, prec):
    """The tensor-core passes take the target from grid.y like the float32 ones: a batch of
    a 1024x2048 and a flipped copy equals two gs_iterate calls in the same precision."""
    H, W, iters = 1024, 2048, 2
    t0 = torch.from_numpy(blob_target(H, W, 3300)).to(cuda)
    T = torch.stack([t0, torch.flip(t0, dims=[1])]).contiguous()
    L, seed = 10007, 6
    codes = pipeline.lut(seed, L, device=cuda)
    holo.holo_tc_status(clear=True)
    got = _batch(cuda, T, iters, 256, codes, L, seed, 0, precision=prec)
    for b in range(2):
        ref = pipeline.gs(T[b], iters, 256, codes, L, 256, seed, start=b * H * W, want_state=True, precision=prec)
        torch.cuda.synchronize()
        assert torch.equal(got["codes"][b], ref["codes"]), b
        assert torch.equal(got["err"][b], ref["err"]), b
        assert torch.equal(got["state"][b], ref["state"]), b
    assert holo.holo_tc_status() == 0


def test_batch_with_caller_phases_and_states(cuda):
    H, W, B = 128, 256, 3
    rng = np.random.default_rng(5)
    T = torch.from_numpy(np.stack([blob_target(H, W, 3200 + b) for b in range(B)])).to(cuda)
    ph = torch.from_numpy(rng.uniform(-np.pi, np.pi, (B, H, W)).astype(np.float32)).to(cuda)
    a = _batch(cuda, T, 2, init=ph)
    b = _batch(cuda, T, 2, states_in=a["state"])
    for k in range(B):
        ra = pipeline.gs(T[k], 2, 256, init_phase=ph[k], want_state=True)
        rb = pipeline.gs(T[k], 2, 256, state_in=ra["state"], want_state=True)
        torch.cuda.synchronize()
        assert torch.equal(a["codes"][k], ra["codes"]) and torch.equal(a["err"][k], ra["err"])
        assert torch.equal(b["codes"][k], rb["codes"]) and torch.equal(b["state"][k], rb["state"])


def test_batch_first_iteration_against_oracle(cuda):
    # every target starts from its own continued LUT draw; one iteration each against the
    # oracle's quantiser and error
    H, W, B = 64, 128, 4
    L, seed = 4099, 6
    T = np.stack([blob_target(H, W, 3300 + b) if b % 2 == 0 else noise_target(H, W, 3400 + b) for b in range(B)])
    codes = pipeline.lut(seed, L, device=cuda)
    got = _batch(cuda, torch.from_numpy(T).to(cuda), 1, 256, codes, L, seed, 0)
    table = olut.lut_codes(seed, L)
    P = H * W
    for b in range(B):
        E = ogs.initial_field(T[b], table, L, seed, start=b * P)
        Hf = offt.ifft2(E)
        check_codes(got["codes"][b].cpu().numpy(), ogs.quantise_phase(Hf, 256), Hf, 256)
        _, _, oeps, _ = ogs.gs(T[b], 1, table, L, seed, start=b * P)
        geps = float(got["err"][b, 0].item())
        assert abs(geps - oeps[0]) <= 10 * NMSE_REL * oeps[0], (b, geps, oeps[0])


def test_batch_rejects_bad_sizes(cuda):
    with pytest.raises(holo.HoloError) as ei:
        holo.gs_batch_workspace_size(0, 64, 64, 1)
    assert ei.value.status == holo.HOLO_EINVAL
    with pytest.raises(holo.HoloError) as ei:
        holo.gs_batch_workspace_size(1024, 4096, 4096, 1)   # B*H*W beyond 2^31
    assert ei.value.status == holo.HOLO_EINVAL
