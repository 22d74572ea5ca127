"""The learned GS warm start end to end at a small scale: labels from gs_iterate, training
by the library's own forward/backward kernels, and what the trained network gains (or
loses) against the paper's LUT-random start: GS iterations to the error the random start
reaches after 20 iterations, evaluated at 512x512 (the 256x256 prediction upsampled)."""

import numpy as np
import pytest
import torch

from paper_2004_04049_gb300 import holo, warmstart
from synthetic import blob_target, noise_target

pytestmark = pytest.mark.gpu


def test_small_pipeline(cuda):
    n = 192
    T = torch.stack([torch.from_numpy(blob_target(256, 256, 5000 + i) if i % 2 == 0
                                      else noise_target(256, 256, 6000 + i)) for i in range(n)]).to(cuda)
    labels = warmstart.make_dataset(T, iters=30)
    assert torch.isfinite(labels).all() and float(labels.abs().max()) <= np.pi + 1e-5
    net = holo.ws_net_create(11, 8)
    try:
        # GS phases from a random start barely move the loss in a few epochs (they are
        # nearly unlearnable), so the training machinery is checked on labels that are a
        # smooth function of the target (phase = pi * T): the loss must fall quickly
        easy = (np.pi * T).contiguous()
        losses = warmstart.train(net, T[:64], easy[:64], epochs=6, batch=8, lr=1e-3)
        first, last = np.mean(losses[:4]), np.mean(losses[-4:])
        print(f"training loss, phase = pi*T: {first:.4f} -> {last:.4f} over {len(losses)} steps")
        assert last < 0.7 * first
        warmstart.train(net, T, labels, epochs=1, batch=8, lr=1e-3)
        ev = [torch.from_numpy(blob_target(512, 512, 7000)).to(cuda),
              torch.from_numpy(noise_target(512, 512, 7001)).to(cuda)]
        rows = warmstart.evaluate(net, ev, iters=60, ref_iter=20)
        for r in rows:
            print("warm start", r)
            assert r["iters_lut"] == 20
            assert np.isfinite(r["err0_learned"]) and np.isfinite(r["nmse_learned"])
    finally:
        holo.ws_net_destroy(net)
