"""Learned GS warm start: dataset, training and evaluation over the C ABI.

The network and every step of its training run in libholo.so (ws_* calls); this module
only sequences calls and holds torch device buffers. The paper's random start (LUT phases,
Section 3) is the baseline: `evaluate` runs GS from both starts and counts the iterations
each needs to reach the error that the LUT-random start reaches after `ref_iter`
iterations (the GS error eps_k / P, eps_k = sum (|R| - T_s)^2, from gs_iterate).
"""

import time

import numpy as np
import torch

from . import holo, pipeline

RES = 256


def make_dataset(targets, iters=100, L=10007, seed=7, levels=256, stream=None):
    """Labels for (n, 256, 256) float32 CUDA targets: the replay-plane phase after `iters`
    GS iterations from the LUT-random start (table seed fixed, so labels are a
    deterministic function of the target). Returns a float32 (n, 256, 256) tensor."""
    n = targets.shape[0]
    dev = targets.device
    codes = pipeline.lut(seed, L, device=dev)
    ws = torch.empty(holo.gs_workspace_size(RES, RES, iters), dtype=torch.uint8, device=dev)
    state = torch.empty((RES, RES, 2), dtype=torch.float32, device=dev)
    err = torch.empty(iters, dtype=torch.float64, device=dev)
    labels = torch.empty((n, RES, RES), dtype=torch.float32, device=dev)
    for i in range(n):
        holo.gs_iterate(targets[i], RES, RES, iters, levels, None, codes, L, 256, seed, 0, holo.HOLO_FP32,
                        None, None, err, None, state, ws, stream=stream)
        holo.gs_state_phase(state, RES, RES, labels[i], stream=stream)
    return labels


def train(net, targets, labels, epochs=2, batch=16, lr=1e-3, seed=0, stream=None):
    """Adam training over the dataset; returns the per-step losses (host floats)."""
    n = targets.shape[0]
    dev = targets.device
    g = torch.Generator(device="cpu").manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    xb = torch.empty((batch, RES, RES), dtype=torch.float32, device=dev)
    yb = torch.empty((batch, RES, RES), dtype=torch.float32, device=dev)
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(dev)
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            torch.index_select(targets, 0, idx, out=xb)
            torch.index_select(labels, 0, idx, out=yb)
            holo.ws_train_step(net, xb, yb, batch, lr, loss, stream=stream)
            hist.append(loss)
            loss = torch.zeros(1, dtype=torch.float32, device=dev)
    return [float(x.item()) for x in hist]


def gs_errors(target, iters, init_phase=None, L=10007, seed=7, levels=256, stream=None):
    """GS error trajectory eps_k / P (float64 host array) and the final replay NMSE."""
    H, W = target.shape
    dev = target.device
    codes = pipeline.lut(seed, L, device=dev) if init_phase is None else None
    out = pipeline.gs(target, iters, levels, codes, L if init_phase is None else 0, 256, seed,
                      init_phase=init_phase, want_codes=False, stream=stream)
    nmse = pipeline.error(out["replay"], target, stream=stream)
    return out["err"].cpu().numpy() / (H * W), float(nmse[2].item())


def iterations_to(err, level):
    hit = np.nonzero(err <= level)[0]
    return int(hit[0]) + 1 if hit.size else None


def evaluate(net, targets, iters=60, ref_iter=20, stream=None):
    """For each (S, S) target: GS iterations and time to reach the error that the LUT-random
    start reaches after ref_iter iterations, from the LUT-random and the learned start."""
    rows = []
    for t in targets:
        S = t.shape[0]
        lut_err, lut_nmse = gs_errors(t, iters, stream=stream)
        level = lut_err[ref_iter - 1]
        phase = torch.empty((S, S), dtype=torch.float32, device=t.device)
        holo.ws_infer(net, t, S, S, phase, stream=stream)
        ws_err, ws_nmse = gs_errors(t, iters, init_phase=phase, stream=stream)
        it_lut = iterations_to(lut_err, level)
        it_ws = iterations_to(ws_err, level)
        # wall time of the two routes to the error level (CUDA events)
        s = torch.cuda.current_stream(t.device)

        def timed(fn):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fn()
            torch.cuda.synchronize()
            e0.record(s)
            fn()
            e1.record(s)
            e1.synchronize()
            return e0.elapsed_time(e1)

        codes = pipeline.lut(7, 10007, device=t.device)
        gws = torch.empty(holo.gs_workspace_size(S, S, iters), dtype=torch.uint8, device=t.device)
        t_lut = timed(lambda: pipeline.gs(t, it_lut, 256, codes, 10007, 256, 7, want_codes=False, ws=gws))
        t_ws = None
        if it_ws is not None:
            t_ws = timed(lambda: (holo.ws_infer(net, t, S, S, phase),
                                  pipeline.gs(t, it_ws, 256, init_phase=phase, want_codes=False, ws=gws)))
        rows.append({"size": S, "level": float(level), "iters_lut": it_lut,
                     "iters_learned": it_ws, "ms_lut": t_lut, "ms_learned": t_ws,
                     "err0_lut": float(lut_err[0]), "err0_learned": float(ws_err[0]),
                     "nmse_lut": lut_nmse, "nmse_learned": ws_nmse})
    return rows


def run(n_train=20000, gs_iters=100, epochs=2, batch=16, lr=1e-3, n_eval=8, eval_size=1024, seed=5,
        device="cuda", log=print, extra_sizes=()):
    """The whole pipeline: seeded targets (half blobs, half band-limited noise), labels from
    GS, training, evaluation at eval_size (the 256^2 prediction upsampled); `extra_sizes`
    repeats the evaluation with 4 targets at other sizes (a larger field makes each saved
    GS iteration worth more against the fixed inference cost)."""
    from synthetic import blob_target, noise_target

    dev = torch.device(device)
    t0 = time.time()
    targets = torch.empty((n_train, RES, RES), dtype=torch.float32, device=dev)
    for i in range(n_train):
        a = blob_target(RES, RES, 100000 + i) if i % 2 == 0 else noise_target(RES, RES, 200000 + i)
        targets[i] = torch.from_numpy(a)
    t1 = time.time()
    labels = make_dataset(targets, iters=gs_iters)
    torch.cuda.synchronize()
    t2 = time.time()
    net = holo.ws_net_create(seed, batch)
    try:
        losses = train(net, targets, labels, epochs=epochs, batch=batch, lr=lr)
        torch.cuda.synchronize()
        t3 = time.time()
        ev = [torch.from_numpy(blob_target(eval_size, eval_size, 900000 + i) if i % 2 == 0
                               else noise_target(eval_size, eval_size, 900000 + i)).to(dev) for i in range(n_eval)]
        rows = evaluate(net, ev)
        extra = {}
        for S in extra_sizes:
            evs = [torch.from_numpy(blob_target(S, S, 910000 + i) if i % 2 == 0
                                    else noise_target(S, S, 910000 + i)).to(dev) for i in range(4)]
            extra[str(S)] = evaluate(net, evs)
    finally:
        holo.ws_net_destroy(net)
    log(f"targets {t1 - t0:.1f}s, GS labels {t2 - t1:.1f}s, training {t3 - t2:.1f}s")
    return {"losses": losses, "eval": rows, "eval_other_sizes": extra,
            "seconds": {"targets": t1 - t0, "labels": t2 - t1, "train": t3 - t2}}
