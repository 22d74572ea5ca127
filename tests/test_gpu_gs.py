"""gs_iterate on the GPU against the float64 oracle (Section 2, Section 3, Section 8).

Single-iteration parity from one shared state (the oracle starts from the GPU's float32
state), the stage-wise replay, error and next state from the GPU's own codes, the
error-reduction property on the GPU trajectory, resume, and the global-phase
equivariance. Tolerances: tests/parity.py.
"""

import numpy as np
import pytest
import torch

from oracle import fft as offt
from oracle import gs as ogs
from oracle import lut as olut
from paper_2004_04049_gb300 import holo, pipeline
from parity import BIT_AGREE_TC, CODE_TIE_TC, NMSE_REL, REPLAY_REL, check_codes, check_replay
from synthetic import blob_target, noise_target

pytestmark = pytest.mark.gpu


def _init_state(T, L, seed):
    table = olut.lut_codes(seed, L)
    E = ogs.initial_field(T, table, L, seed)
    return E.astype(np.complex64)


@pytest.mark.parametrize("H,W,levels,kind", [(64, 64, 256, "blob"), (256, 256, 256, "noise"),
                                             (128, 512, 256, "blob"), (256, 128, 2, "blob"),
                                             (1024, 1024, 256, "blob"), (1024, 2048, 256, "noise"),
                                             (64, 4096, 256, "noise"),
                                             (4096, 64, 4, "blob")])
def test_single_iteration_parity(cuda, H, W, levels, kind):
    _single_iteration(cuda, H, W, levels, kind)


@pytest.mark.parametrize("H,W", [(512, 1024), (2048, 512)])
@pytest.mark.parametrize("tiles", [(0, 0), (1, 2), (2, 1), (1, 1)])
def test_tile_variants_parity(cuda, H, W, tiles):
    holo.gs_tuning_set(H, W, *tiles)
    try:
        assert holo.gs_tuning_get(H, W) == {"col_variant": tiles[0], "row_variant": tiles[1]}
        _single_iteration(cuda, H, W, 256, "noise")
    finally:
        holo.gs_tuning_set(H, W)


@pytest.mark.parametrize("H,W", [(1024, 1024), (1024, 2048), (2048, 1024)])
@pytest.mark.parametrize("prec", [holo.HOLO_FP16X2, holo.HOLO_BF16X2])
def test_single_iteration_parity_tensor_core(cuda, H, W, prec):
    # the DFT-32 stages on the tensor cores with split hi/lo operands: codes against the
    # widened tie band of parity.py, replay, error and next state against the float32 bounds
    _single_iteration(cuda, H, W, 256, "noise", precision=prec)


def test_tensor_core_trajectory_tracks_fp32(cuda):
    # 20 iterations from the LUT start: the error trajectory of each tensor-core precision
    # stays non-increasing and within the 5% drift bound that float32 keeps against the
    # oracle (a code that ties differently parts the trajectories)
    H = W = 1024
    T = torch.from_numpy(blob_target(H, W, 1015)).to(cuda)
    codes = pipeline.lut(5, 10007, device=cuda)
    ref = pipeline.gs(T, 20, 256, codes, 10007, 256, 5)["err"].cpu().numpy()
    for prec in (holo.HOLO_FP16X2, holo.HOLO_BF16X2):
        e = pipeline.gs(T, 20, 256, codes, 10007, 256, 5, precision=prec)["err"].cpu().numpy()
        assert np.all(np.diff(e) <= 1e-5 * e[0]), prec
        assert np.all(np.abs(e - ref) <= 0.05 * ref), (prec, np.abs(e - ref).max() / ref.max())
    with pytest.raises(holo.HoloError) as ei:
        pipeline.gs(torch.zeros((512, 512), device=cuda), 1, 256, precision=holo.HOLO_BF16X2)
    assert ei.value.status == holo.HOLO_EUNSUPPORTED


def _single_iteration(cuda, H, W, levels, kind, precision=holo.HOLO_FP32):
    T = blob_target(H, W, 1010) if kind == "blob" else noise_target(H, W, 2010)
    E32 = _init_state(T, 10007, 3)
    t = torch.from_numpy(T).to(cuda)
    st = torch.from_numpy(np.stack([E32.real, E32.imag], -1).astype(np.float32)).to(cuda)
    out = pipeline.gs(t, 1, levels, state_in=st, want_state=True, precision=precision)
    torch.cuda.synchronize()
    gq = out["codes"].cpu().numpy()
    gI = out["replay"].cpu().numpy()
    geps = out["err"].cpu().numpy()
    gE = out["state"].cpu().numpy()
    E = E32.astype(np.complex128)
    Hf = offt.ifft2(E)
    oq = ogs.quantise_phase(Hf, levels)
    if precision == holo.HOLO_FP32:
        check_codes(gq, oq, Hf, levels)
    else:
        check_codes(gq, oq, Hf, levels, tie=CODE_TIE_TC, agree_floor=BIT_AGREE_TC)
    # stage-wise: the oracle continues from the GPU's codes
    Ts = ogs.energy_scaled_target(T)
    R = offt.fft2(ogs.hologram_of_codes(gq.astype(np.int64), levels))
    check_replay(gI, np.abs(R) ** 2)
    eps = np.sum((np.abs(R) - Ts) ** 2)
    assert abs(geps[0] - eps) <= 10 * NMSE_REL * eps, (geps[0], eps)
    En = ogs.amplitude_constraint(R, Ts)
    gEc = gE[..., 0] + 1j * gE[..., 1]
    # E = T_s exp(i arg R): an error dR in the float32 replay field turns the phase by up to
    # |dR|/|R|, so the state error at a pixel is bounded by T_s |dR| / |R| (ill-conditioned
    # where R nearly vanishes) plus the rounding of E itself
    dR = REPLAY_REL * np.abs(R).max()
    bound = Ts * np.minimum(2.0, dR / np.maximum(np.abs(R), 1e-30)) + REPLAY_REL * np.abs(En).max()
    assert np.all(np.abs(gEc - En) <= bound), np.max(np.abs(gEc - En) / bound)


@pytest.mark.parametrize("levels", [256, 2])
def test_error_non_increasing_and_tracks_oracle(cuda, levels):
    H = W = 256
    T = blob_target(H, W, 1011)
    L, seed, iters = 10007, 5, 20
    t = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(seed, L, device=cuda)
    out = pipeline.gs(t, iters, levels, codes, L, 256, seed)
    geps = out["err"].cpu().numpy()
    d = np.diff(geps)
    assert np.all(d <= 1e-5 * geps[0]), d.max()
    _, _, oeps, _ = ogs.gs(T, iters, olut.lut_codes(seed, L), L, seed, levels=levels, lut_levels=256)
    drift = np.abs(geps - oeps) / oeps
    # reported, with a loose bound: the trajectories may part where codes tie
    assert drift[0] < 1e-4
    assert drift.max() < 0.05, drift


def test_resume_equals_continuous_run(cuda):
    H = W = 128
    T = noise_target(H, W, 2012)
    t = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(1, 4099, device=cuda)
    six = pipeline.gs(t, 6, 256, codes, 4099, 256, 1)
    three = pipeline.gs(t, 3, 256, codes, 4099, 256, 1, want_state=True)
    more = pipeline.gs(t, 3, 256, state_in=three["state"])
    torch.cuda.synchronize()
    assert torch.equal(more["codes"], six["codes"])
    assert np.allclose(np.concatenate([three["err"].cpu().numpy(), more["err"].cpu().numpy()]),
                       six["err"].cpu().numpy(), rtol=1e-6)


def test_global_phase_equivariance(cuda):
    # One iteration: a single code that ties differently perturbs the whole next field by
    # ~1e-4 and flips ~1% of the following iteration's codes, so code-level comparisons are
    # per iteration. The target is broadband so that no pixel of H sits at float32 noise.
    # Each run is checked against the oracle (differences only at quantiser ties), and the
    # two runs' codes differ by c0 wherever neither sits at a tie.
    H = W = 256
    T = np.random.default_rng(13).random((H, W)).astype(np.float32)
    t = torch.from_numpy(T).to(cuda)
    c0 = 77
    one = torch.tensor([c0], dtype=torch.uint8, device=cuda)
    a = pipeline.gs(t, 1, 256, one, 1, 256, 0)
    b = pipeline.gs(t, 1, 256, None, 0, 256, 0)
    qa = a["codes"].cpu().numpy().astype(np.int64)
    qb = b["codes"].cpu().numpy().astype(np.int64)
    Ts = ogs.energy_scaled_target(T)
    Hb = offt.ifft2(Ts.astype(np.complex128))
    Ha = offt.ifft2(Ts * np.exp(2j * np.pi * c0 / 256))
    check_codes(qb, ogs.quantise_phase(Hb, 256), Hb, 256)
    check_codes(qa, ogs.quantise_phase(Ha, 256), Ha, 256)
    assert np.mean((qb + c0) % 256 == qa) >= 0.999
    assert np.allclose(a["err"].cpu().numpy(), b["err"].cpu().numpy(), rtol=1e-5)


# start index k*P + j: frame k of a GS video continues the table draw (Fig. 3 continuation;
# Section 8 allows LUT reuse across frames when L is prime and longer than the image side)
@pytest.mark.parametrize("start", [0, 5 * 128 * 128 + 17])
def test_caller_phase_equals_lut_phase(cuda, start):
    H = W = 128
    T = blob_target(H, W, 1014)
    t = torch.from_numpy(T).to(cuda)
    L, seed = 521, 8
    codes = pipeline.lut(seed, L, device=cuda)
    theta = olut.phase_of_codes(olut.subframe_codes(olut.lut_codes(seed, L), L, seed, start, 0,
                                                    H * W, H * W)).reshape(H, W)
    a = pipeline.gs(t, 1, 256, codes, L, 256, seed, start=start)
    b = pipeline.gs(t, 1, 256, init_phase=torch.from_numpy(theta.astype(np.float32)).to(cuda))
    qa, qb = a["codes"].cpu().numpy(), b["codes"].cpu().numpy()
    assert np.mean(qa == qb) >= 0.9999


def test_bench_configuration_trajectory(cuda):
    # the GS leg of the benchmark as it runs there: 1024x1024 blob target (seed 1000),
    # 20 iterations, 256 levels, LUT start (L = 10007, seed 7); the error trajectory against
    # the oracle's, and the last iteration's codes and replay stage-wise from the GPU's
    # own state before it
    H = W = 1024
    T = blob_target(H, W, 1000)
    L, seed, iters = 10007, 7, 20
    t = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(seed, L, device=cuda)
    out = pipeline.gs(t, iters, 256, codes, L, 256, seed)
    geps = out["err"].cpu().numpy()
    assert np.all(np.diff(geps) <= 1e-5 * geps[0])
    table = olut.lut_codes(seed, L)
    _, _, oeps, _ = ogs.gs(T, iters, table, L, seed)
    drift = np.abs(geps - oeps) / oeps
    assert drift[0] < 1e-4 and drift.max() < 0.05, drift
    # stage-wise last iteration: 19 iterations on the GPU, then one more from that state
    st19 = pipeline.gs(t, iters - 1, 256, codes, L, 256, seed, want_state=True)["state"]
    last = pipeline.gs(t, 1, 256, state_in=st19)
    torch.cuda.synchronize()
    s = st19.cpu().numpy().astype(np.float64)
    Hf = offt.ifft2(s[..., 0] + 1j * s[..., 1])
    check_codes(last["codes"].cpu().numpy(), ogs.quantise_phase(Hf, 256), Hf, 256)
    assert torch.equal(last["codes"], out["codes"])
    R = offt.fft2(ogs.hologram_of_codes(last["codes"].cpu().numpy().astype(np.int64), 256))
    check_replay(last["replay"].cpu().numpy(), np.abs(R) ** 2)
