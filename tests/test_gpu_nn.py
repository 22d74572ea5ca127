"""The warm-start network's kernels against the float64 oracle.

Convolution forward, input gradient and weight gradient are compared element by element
on bf16-representable inputs (so only the float32 accumulation order differs); the whole
network's loss and weight gradients are compared with a float64 network of the same
architecture that rounds its stored activations to bf16 as the GPU does."""

import numpy as np
import pytest
import torch

from oracle import conv as oc
from paper_2004_04049_gb300 import holo
from synthetic import blob_target, noise_target

pytestmark = pytest.mark.gpu


def bf16_round(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _dev_bf16(x, cuda):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(cuda).contiguous()


@pytest.mark.parametrize("B,H,W,Ci,Co", [(2, 16, 16, 16, 24), (1, 32, 8, 8, 64), (3, 8, 8, 128, 32)])
def test_conv_forward(cuda, B, H, W, Ci, Co):
    rng = np.random.default_rng(B * 100 + Ci)
    x = bf16_round(rng.standard_normal((B, H, W, Ci)))
    w = bf16_round(rng.standard_normal((Co, 3, 3, Ci)) * 0.2)
    b = rng.standard_normal(Co).astype(np.float32)
    res = bf16_round(rng.standard_normal((B, H, W, Co)))
    out = torch.zeros((B, H, W, Co), dtype=torch.float32, device=cuda)
    holo.nn_conv3x3(0, B, H, W, Ci, Co, _dev_bf16(x, cuda), _dev_bf16(w.reshape(Co, -1), cuda),
                    d_bias=torch.from_numpy(b).to(cuda), d_residual=_dev_bf16(res, cuda), relu=True,
                    d_out_f32=out)
    ref = np.maximum(oc.conv3x3(x, w, b) + res, 0.0)
    g = out.cpu().numpy()
    assert np.max(np.abs(g - ref)) <= 1e-5 * max(1.0, np.abs(ref).max())


# tcgen05 path: output widths 32/64/128, pixel counts that leave a partial 128-pixel tile,
# K = 9*Cin that leaves a partial 64-element slice, batches that cross images in one tile
@pytest.mark.parametrize("B,H,W,Ci,Co", [(1, 24, 24, 40, 128), (3, 10, 14, 32, 32), (2, 64, 64, 64, 64),
                                         (1, 8, 16, 128, 128), (3, 10, 14, 8, 32)])
@pytest.mark.parametrize("legacy", [False, True])
def test_conv_forward_tcgen05_and_legacy(cuda, B, H, W, Ci, Co, legacy):
    rng = np.random.default_rng(B * 1000 + H * 10 + Ci)
    x = bf16_round(rng.standard_normal((B, H, W, Ci)))
    w = bf16_round(rng.standard_normal((Co, 3, 3, Ci)) * 0.1)
    b = rng.standard_normal(Co).astype(np.float32)
    res = bf16_round(rng.standard_normal((B, H, W, Co)))
    out = torch.zeros((B, H, W, Co), dtype=torch.float32, device=cuda)
    outb = torch.zeros((B, H, W, Co), dtype=torch.bfloat16, device=cuda)
    mode = holo.HOLO_CONV_LEGACY if legacy else 0
    holo.holo_tc_status(clear=True)
    holo.nn_conv3x3(mode, B, H, W, Ci, Co, _dev_bf16(x, cuda), _dev_bf16(w.reshape(Co, -1), cuda),
                    d_bias=torch.from_numpy(b).to(cuda), d_residual=_dev_bf16(res, cuda), relu=True,
                    d_out=outb, d_out_f32=out)
    torch.cuda.synchronize()
    assert holo.holo_tc_status() == 0
    ref = np.maximum(oc.conv3x3(x, w, b) + res, 0.0)
    g = out.cpu().numpy()
    assert np.max(np.abs(g - ref)) <= 1e-5 * max(1.0, np.abs(ref).max())
    # the bf16 output is the float32 result rounded to nearest even
    assert torch.equal(outb.cpu(), out.cpu().to(torch.bfloat16))


@pytest.mark.parametrize("B,H,W,Ci,Co", [(2, 16, 16, 16, 24), (1, 32, 8, 64, 8), (2, 20, 12, 128, 32),
                                         (1, 16, 16, 32, 128)])
def test_conv_input_gradient(cuda, B, H, W, Ci, Co):
    rng = np.random.default_rng(7 + Ci)
    dy = bf16_round(rng.standard_normal((B, H, W, Co)))
    w = bf16_round(rng.standard_normal((Co, 3, 3, Ci)) * 0.2)
    wt = np.ascontiguousarray(np.transpose(w, (3, 1, 2, 0)).reshape(Ci, -1))   # [Ci][tap][Co]
    out = torch.zeros((B, H, W, Ci), dtype=torch.float32, device=cuda)
    holo.nn_conv3x3(1, B, H, W, Co, Ci, _dev_bf16(dy, cuda), _dev_bf16(wt, cuda), d_out_f32=out)
    ref = oc.conv3x3_dgrad(dy, w)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("B,H,W,Ci,Co", [(2, 16, 16, 16, 24), (4, 32, 32, 8, 32)])
def test_conv_weight_gradient(cuda, B, H, W, Ci, Co):
    rng = np.random.default_rng(11 + Co)
    x = bf16_round(rng.standard_normal((B, H, W, Ci)))
    dy = bf16_round(rng.standard_normal((B, H, W, Co)))
    dw = torch.zeros((Co, 9 * Ci), dtype=torch.float32, device=cuda)
    holo.nn_conv3x3(2, B, H, W, Ci, Co, _dev_bf16(x, cuda), d_dy=_dev_bf16(dy, cuda), d_dw=dw)
    ref = oc.conv3x3_wgrad(x, dy).reshape(Co, -1)
    assert np.max(np.abs(dw.cpu().numpy() - ref)) <= 1e-5 * np.abs(ref).max()


def _oracle_forward(params, T):
    """float64 forward of the same architecture; stored activations rounded to bf16."""
    r = bf16_round
    W = [r(w) for w, _ in params]
    Bb = [b.astype(np.float64) for _, b in params]
    x0 = np.zeros(T.shape + (8,))
    x0[..., 0] = T
    x0 = r(x0)

    def layer(i, x, res=None, relu=True):
        y = oc.conv3x3(x, W[i], Bb[i])
        if res is not None:
            y = y + res
        return r(np.maximum(y, 0.0)) if relu else y

    a1 = layer(0, x0)
    s1 = layer(1, a1)
    a2 = layer(2, r(oc.avgpool2(s1)))
    s2 = layer(3, a2)
    a3 = layer(4, r(oc.avgpool2(s2)))
    s3 = layer(5, a3)
    a4 = layer(6, r(oc.avgpool2(s3)))
    b4 = layer(7, a4)
    u5 = layer(8, oc.upsample2(b4), s3)
    u6 = layer(9, oc.upsample2(u5), s2)
    u7 = layer(10, oc.upsample2(u6), s1)
    return layer(11, u7, relu=False), W


def test_network_loss_and_gradients_match_oracle(cuda):
    """End to end: the loss of the whole network; stage-wise (the oracle fed the GPU's own
    stored tensors, since bf16 rounding differences that accumulate over ten layers flip
    ReLU masks at a few percent of pixels and the gradients are sums with cancellation):
    the loss gradient, the head's and the last decoder layer's weight gradients, and the
    gradient reaching the first skip."""
    net = holo.ws_net_create(5, 1)
    try:
        T = blob_target(256, 256, 1400).astype(np.float32)
        label = np.random.default_rng(1).uniform(-np.pi, np.pi, (256, 256)).astype(np.float32)
        loss = torch.zeros(1, dtype=torch.float32, device=cuda)
        holo.ws_forward_backward(net, torch.from_numpy(T).to(cuda), torch.from_numpy(label).to(cuda), 1, loss)
        torch.cuda.synchronize()
        params = [(holo.ws_get_tensor(net, i, 0), holo.ws_get_tensor(net, i, 1)) for i in range(12)]
        out, W = _oracle_forward(params, T[None].astype(np.float64))
        z = np.exp(1j * label[None].astype(np.float64))
        wts = T[None].astype(np.float64) ** 2
        oloss = oc.phase_loss(out[..., :2], z, wts, eps=1e-20)
        assert abs(float(loss.item()) - oloss) <= 2e-3 * max(oloss, 1e-3)
        # stage-wise backward from the GPU's own tensors
        g_out_gpu = holo.ws_get_activation(net, "out").astype(np.float64)
        gref = oc.phase_loss_grad(g_out_gpu[..., :2], z, wts, eps=1e-20)
        g_out = holo.ws_get_activation(net, "g_out").astype(np.float64)
        assert np.linalg.norm(g_out[..., :2] - gref) <= 1e-2 * np.linalg.norm(gref)
        assert np.all(g_out[..., 2:] == 0.0)
        u7 = holo.ws_get_activation(net, "u7").astype(np.float64)
        up6 = holo.ws_get_activation(net, "up6").astype(np.float64)
        checks = {11: oc.conv3x3_wgrad(u7, g_out)}
        g_u7 = bf16_round(oc.conv3x3_dgrad(g_out, W[11])) * (u7 > 0)
        g_u7_gpu = holo.ws_get_activation(net, "g_u7").astype(np.float64)
        assert np.linalg.norm(g_u7_gpu - g_u7) <= 1e-2 * np.linalg.norm(g_u7)
        checks[10] = oc.conv3x3_wgrad(up6, g_u7_gpu)
        for layer, ref in checks.items():
            g = holo.ws_get_tensor(net, layer, 2).astype(np.float64)
            rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
            assert rel < 1e-2, (layer, rel)
            db = holo.ws_get_tensor(net, layer, 3).astype(np.float64)
            gsrc = g_out if layer == 11 else g_u7_gpu
            dbref = oc.bias_grad(gsrc)
            assert np.linalg.norm(db - dbref) <= 1e-2 * np.linalg.norm(dbref) + 1e-30
        g_up6 = holo.ws_get_activation(net, "g_up6").astype(np.float64)
        ref = oc.conv3x3_dgrad(g_u7_gpu, W[10])
        assert np.linalg.norm(g_up6 - ref) <= 1e-2 * np.linalg.norm(ref)
    finally:
        holo.ws_net_destroy(net)


def test_training_reduces_loss(cuda, tmp_path):
    net = holo.ws_net_create(3, 4)
    try:
        rng = np.random.default_rng(2)
        T = np.stack([blob_target(256, 256, 1500 + i) if i % 2 == 0 else noise_target(256, 256, 2500 + i)
                      for i in range(4)]).astype(np.float32)
        # a learnable label: a smooth phase made from the target itself
        label = (2.0 * np.pi * T - np.pi).astype(np.float32)
        t = torch.from_numpy(T).to(cuda)
        lab = torch.from_numpy(label).to(cuda)
        loss = torch.zeros(1, dtype=torch.float32, device=cuda)
        losses = []
        for step in range(120):
            holo.ws_train_step(net, t, lab, 4, 1e-3, loss)
            losses.append(float(loss.item()))
        # the weight gradients are summed with float atomics, so the trajectory differs from
        # run to run, and under Adam the per-step loss oscillates on its way down (steps 20 to
        # 60 range from ~0.5 of the start down to ~0.02); from step 80 on every run seen sits
        # below 0.03 of the start: judge the median of the last ten of 120 steps, not one step
        assert np.median(losses[-10:]) < 0.5 * losses[0], (losses[0], losses[-10:])
        path = tmp_path / "ws.bin"
        holo.ws_save(net, path)
        net2 = holo.ws_net_create(99, 1)
        try:
            holo.ws_load(net2, path)
            for i in (0, 5, 11):
                assert np.array_equal(holo.ws_get_tensor(net, i, 0), holo.ws_get_tensor(net2, i, 0))
            ph1 = torch.empty((1024, 1024), dtype=torch.float32, device=cuda)
            ph2 = torch.empty((1024, 1024), dtype=torch.float32, device=cuda)
            big = torch.from_numpy(blob_target(1024, 1024, 1600)).to(cuda)
            holo.ws_infer(net, big, 1024, 1024, ph1)
            holo.ws_infer(net2, big, 1024, 1024, ph2)
            torch.cuda.synchronize()
            assert torch.equal(ph1, ph2)
            assert float(ph1.abs().max()) <= np.pi + 1e-6
        finally:
            holo.ws_net_destroy(net2)
    finally:
        holo.ws_net_destroy(net)
