"""GPU parity of the warm start's last mile against the float64 oracle, through the C ABI:
the bilinear phase resample that maps the network's 256x256 (u, v) output onto the GS
grid (ws_phase_resample, the kernel ws_infer ends with), the Adam update of every
training step (ws_adam_update), the training label (gs_state_phase: the phase of a GS
state), and ws_infer's input area average and output phase checked end to end."""

import numpy as np
import pytest
import torch

from oracle import conv as oc
from oracle import gs as ogs
from paper_2004_04049_gb300 import holo, pipeline
from synthetic import blob_target

pytestmark = pytest.mark.gpu


def _wrapped(d):
    return np.abs(np.angle(np.exp(1j * d)))


def _check_phase(gpu_phase, uv64, Ho, Wo):
    """Element-wise: |GPU - oracle| (wrapped to (-pi, pi]) within 1e-5 rad plus the float32
    rounding of the interpolation (weights and sums, relative 2^-24 each, of values up to
    M = max |u|, |v|), which grows as M/|(u, v)| where the neighbours cancel."""
    ref = oc.phase_of_uv(uv64, Ho, Wo)
    u = oc.bilinear_resample(uv64[..., 0], Ho, Wo)
    v = oc.bilinear_resample(uv64[..., 1], Ho, Wo)
    M = np.abs(uv64[..., :2]).max()
    mag = np.hypot(u, v)
    tol = 1e-5 + 1e-6 * M / np.maximum(mag, 1e-30)
    err = _wrapped(gpu_phase.astype(np.float64) - ref)
    bad = err > tol
    assert not bad.any(), (int(bad.sum()), float(err.max()))
    return float(err[mag > 1e-3 * mag.max()].max())


@pytest.mark.parametrize("H,W,Ho,Wo,C", [(256, 256, 1024, 1024, 8), (256, 256, 256, 256, 8),
                                         (37, 53, 333, 517, 2), (64, 48, 40, 100, 4), (1, 3, 1, 5, 2)])
def test_phase_resample_parity(cuda, H, W, Ho, Wo, C):
    rng = np.random.default_rng(H * 7 + Wo)
    uv = rng.standard_normal((H, W, C)).astype(np.float32)
    d_uv = torch.from_numpy(uv).to(cuda)
    d_ph = torch.full((Ho, Wo), 99.0, dtype=torch.float32, device=cuda)
    holo.ws_phase_resample(d_uv, C, H, W, Ho, Wo, d_ph)
    ph = d_ph.cpu().numpy()
    assert np.all(np.abs(ph) <= np.float32(np.pi))
    worst = _check_phase(ph, uv.astype(np.float64), Ho, Wo)
    print(f"resample {H}x{W} -> {Ho}x{Wo}: max wrapped error {worst:.2e} rad away from cancellation")


def test_phase_resample_rejects_bad_arguments(cuda):
    d = torch.zeros((4, 4, 2), dtype=torch.float32, device=cuda)
    with pytest.raises(holo.HoloError):
        holo.ws_phase_resample(d, 1, 4, 4, 8, 8, d)
    with pytest.raises(holo.HoloError):
        holo.ws_phase_resample(d, 2, 4, 4, 0, 8, d)


@pytest.mark.parametrize("step,eps", [(1, 1e-8), (2, 0.0), (7, 1e-8), (1000, 1e-6)])
def test_adam_parity(cuda, step, eps):
    n = 100003   # several blocks and a ragged tail
    rng = np.random.default_rng(step)
    w = rng.standard_normal(n).astype(np.float32)
    g = (rng.standard_normal(n) * 10.0 ** rng.uniform(-4, 1, n)).astype(np.float32)
    if step == 1:
        m = np.zeros(n, np.float32)
        v = np.zeros(n, np.float32)
    else:
        m = (rng.standard_normal(n) * 0.1).astype(np.float32)
        v = (rng.uniform(0, 1, n) ** 2 * 0.01).astype(np.float32)
    # the C ABI takes float32 hyper-parameters: the oracle gets the same (rounded) values,
    # so 1 - beta2 is 1 - float32(0.999) on both sides
    f32 = lambda x: float(np.float32(x))
    lr, b1, b2, eps = f32(1e-3), f32(0.9), f32(0.999), f32(eps)
    dw, dg, dm, dv = (torch.from_numpy(x.copy()).to(cuda) for x in (w, g, m, v))
    holo.ws_adam_update(dw, dg, dm, dv, n, lr, b1, b2, eps, step)
    rw, rm, rv = oc.adam_step(w, g, m, v, step, lr, b1, b2, eps)
    gw, gm, gv = (x.cpu().numpy().astype(np.float64) for x in (dw, dm, dv))
    # float32 rounding of a two-term sum: a few units of 2^-24 of the terms' magnitudes
    u = 2.0 ** -24
    m_terms = np.abs(b1 * m) + np.abs((1 - b1) * g)
    v_terms = np.abs(b2 * v) + np.abs((1 - b2) * g.astype(np.float64) ** 2)
    assert np.all(np.abs(gm - rm) <= 4 * u * m_terms + 1e-30)
    assert np.all(np.abs(gv - rv) <= 4 * u * v_terms + 1e-30)
    # the weight update to 1e-5 relative (bias corrections use float32 powf); the stored
    # weight to float32 rounding
    step_gpu = w.astype(np.float64) - gw
    step_ref = w.astype(np.float64) - rw
    assert np.all(np.abs(step_gpu - step_ref) <= 1e-5 * np.abs(step_ref) + u * np.abs(w) + 1e-12)


def test_adam_hand_worked_two_steps_on_gpu(cuda, golden_dir):
    import json
    import os
    g = json.load(open(os.path.join(golden_dir, "warmstart_resample_adam.json")))["adam_two_steps"]
    dw = torch.tensor(g["w0"], dtype=torch.float32, device=cuda)
    dm = torch.zeros(3, dtype=torch.float32, device=cuda)
    dv = torch.zeros(3, dtype=torch.float32, device=cuda)
    for k, (gk, wk) in enumerate([(g["g1"], g["w1"]), (g["g2"], g["w2"])], start=1):
        dg = torch.tensor(gk, dtype=torch.float32, device=cuda)
        holo.ws_adam_update(dw, dg, dm, dv, 3, g["lr"], g["beta1"], g["beta2"], g["eps"], k)
        assert np.allclose(dw.cpu().numpy(), wk, atol=1e-6), (k, dw.cpu().numpy(), wk)


@pytest.mark.parametrize("H,W,iters", [(256, 256, 3), (64, 128, 2)])
def test_gs_state_phase_parity(cuda, H, W, iters):
    T = blob_target(H, W, 4242 + H)
    T[: H // 8, :] = 0.0   # zero amplitude: the state is exactly zero there, arg 0 := 0
    t = torch.from_numpy(T).to(cuda)
    codes = pipeline.lut(7, 10007, device=cuda)
    ws = torch.empty(holo.gs_workspace_size(H, W, iters), dtype=torch.uint8, device=cuda)
    state = torch.empty((H, W, 2), dtype=torch.float32, device=cuda)
    holo.gs_iterate(t, H, W, iters, 256, None, codes, 10007, 256, 7, 0, holo.HOLO_FP32, None, None, None, None,
                    state, ws)
    ph = torch.full((H, W), 99.0, dtype=torch.float32, device=cuda)
    holo.gs_state_phase(state, H, W, ph)
    s = state.cpu().numpy().astype(np.float64)
    ref = ogs.replay_phase(s[..., 0] + 1j * s[..., 1])
    got = ph.cpu().numpy().astype(np.float64)
    assert np.all(_wrapped(got - ref) <= 1e-6)
    zero = (s[..., 0] == 0) & (s[..., 1] == 0)
    assert zero[: H // 8].all() and np.all(got[zero] == 0.0)


def test_ws_infer_matches_oracle_last_mile(cuda):
    """ws_infer end to end: the network input is the 4x4 area average of the 1024^2 target
    (rounded to bf16), and the output phase is the oracle's bilinear phase of the network's
    own stored float32 head output."""
    net = holo.ws_net_create(21, 1)
    try:
        T = blob_target(1024, 1024, 31337)
        t = torch.from_numpy(T).to(cuda)
        ph = torch.empty((1024, 1024), dtype=torch.float32, device=cuda)
        holo.ws_infer(net, t, 1024, 1024, ph)
        torch.cuda.synchronize()
        x0 = holo.ws_get_activation(net, "x0", 1).reshape(256, 256, 8).astype(np.float64)
        avg = oc.area_average(T, 256)
        assert np.all(np.abs(x0[..., 0] - avg) <= 1.001 * 2.0 ** -8 * np.abs(avg) + 1e-30)
        assert not x0[..., 1:].any()
        out = holo.ws_get_activation(net, "out", 1).reshape(256, 256, 8).astype(np.float64)
        _check_phase(ph.cpu().numpy(), out, 1024, 1024)
    finally:
        holo.ws_net_destroy(net)
