"""The LUT-length study of Section 5.2 (Figs. 5 and 6) on the GPU, with synthetic targets.

For each hologram size, every (target, run, L) triple is one OSPR frame of N binary
sub-frames whose table is built from the run's seed; the reference is the same frame with
unrepeated (generator) phases. The error of a frame is replay_error's NMSE (Eq. 3 reading:
intensity domain, optimal scale), divided by the mean unrepeated NMSE of the same target,
so 1 means "as good as independent random phases". The study reports, per L, the mean and
standard deviation of that ratio over targets and runs (the paper's red line and grey
+-2 sigma band), and per-target means. All frames go through ospr_generate_batch in chunks;
this module only lays out buffers and descriptors.
"""

import math

import numpy as np
import torch

from . import holo


def is_prime(n):
    """Deterministic Miller-Rabin for n < 3.3e24."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def next_prime(n):
    n = max(2, int(n))
    while not is_prime(n):
        n += 1
    return n


def prime_grid(S, N, points=40):
    """Prime table lengths from 2 to about 4*N*S^2 on a log grid, plus the primes next to
    N, to the image side S and the paper's 10007."""
    top = 4 * N * S * S
    grid = {next_prime(round(math.exp(x))) for x in np.linspace(math.log(2), math.log(top), points)}
    grid |= {next_prime(N), next_prime(S - S // 32), next_prime(S), 10007}
    return sorted(grid)


def _sample_std(v):
    """Sample standard deviation (n - 1 in the denominator); None for fewer than two samples,
    where it is undefined."""
    return float(np.std(v, ddof=1)) if np.size(v) > 1 else None


def lut_length_study(sizes=(256, 128, 64), N=24, runs=100, n_targets=6, points=40, chunk_bytes=1 << 30,
                     device="cuda", log=None):
    from synthetic import blob_target, noise_target

    dev = torch.device(device)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for S in sizes:
        P = S * S
        holo.ospr_autotune(S, S, N, reps=2, stream=stream.cuda_stream)
        targets = [torch.from_numpy(blob_target(S, S, 1000 + t) if t % 2 == 0 else noise_target(S, S, 2000 + t))
                   .to(dev) for t in range(n_targets)]
        Ls = prime_grid(S, N, points)
        frames = [(t, r, L) for L in [holo.L_UNREPEATED] + Ls for t in range(n_targets) for r in range(runs)]
        err = torch.zeros((len(frames), 3), dtype=torch.float64, device=dev)
        # chunks bounded by their table and replay bytes
        i = 0
        while i < len(frames):
            j, nbytes = i, 0
            while j < len(frames) and (j == i or nbytes + max(frames[j][2], 0) + 4 * P <= chunk_bytes):
                nbytes += max(frames[j][2], 0) + 4 * P
                j += 1
            part = frames[i:j]
            tab_off, o = [], 0
            for (_, _, L) in part:
                tab_off.append(o)
                o += (L + 255) // 256 * 256 if L > 0 else 0
            tables = torch.empty(max(o, 256), dtype=torch.uint8, device=dev)
            replay = torch.empty((len(part), S, S), dtype=torch.float32, device=dev)
            descs = []
            for k, (t, r, L) in enumerate(part):
                codes = tables[tab_off[k]:] if L > 0 else None
                descs.append(holo.frame_desc(targets[t], S, S, N, codes, L, 256, 1 + r, L > 0, 0, 0,
                                             None, replay[k], err[i + k]))
            arr = holo.frame_array(descs)
            ws = torch.empty(holo.ospr_batch_workspace_size(arr), dtype=torch.uint8, device=dev)
            holo.ospr_generate_batch(arr, holo.HOLO_FP32, ws, stream=stream.cuda_stream)
            torch.cuda.synchronize(dev)
            i = j
        nmse = err[:, 2].cpu().numpy().reshape(len(Ls) + 1, n_targets, runs)
        ref = nmse[0].mean(axis=1)                       # per target, unrepeated
        ratio = nmse[1:] / ref[None, :, None]
        rows = []
        for li, L in enumerate(Ls):
            v = ratio[li].ravel()
            rows.append({"L": L, "mean": float(v.mean()), "std": _sample_std(v),
                         "per_target": [float(x) for x in ratio[li].mean(axis=1)]})
        out[f"{S}x{S}"] = {"N": N, "runs": runs, "targets": n_targets,
                           "unrepeated_nmse": [float(x) for x in ref],
                           "unrepeated_ratio_std": _sample_std((nmse[0] / ref[:, None]).ravel()),
                           "rows": rows}
        if log:
            r10007 = next(r for r in rows if r["L"] == 10007)
            spread = "" if r10007["std"] is None else f" +- {2 * r10007['std']:.4f}"
            log(f"{S}x{S}: {len(frames)} frames, L=10007 ratio {r10007['mean']:.4f}{spread}")
    return out
