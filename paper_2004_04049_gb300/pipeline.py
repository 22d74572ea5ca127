"""Device-buffer helpers over the C-ABI binding: allocate outputs and workspaces as torch
CUDA tensors and call the library. Plumbing only; every computation is a library kernel.
"""

import torch

from . import holo


def _ws(nbytes, device):
    # 256-byte alignment: the caching allocator returns >= 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def lut(seed, L, levels=256, device="cuda", with_cs=False, stream=None):
    codes = torch.empty(L, dtype=torch.uint8, device=device)
    cs = torch.empty(2 * L, dtype=torch.float32, device=device) if with_cs else None
    holo.lut_build(seed, L, levels, codes, cs, stream=stream)
    return (codes, cs) if with_cs else codes


def ospr(target, N, codes=None, L=0, levels=256, seed=0, start=0, stride=0, bits=True, replay=True,
         ws=None, out_bits=None, out_replay=None, precision=holo.HOLO_FP32, stream=None):
    """Returns (bits int32 [N, H*W/32] or None, replay float32 [H, W] or None)."""
    H, W = target.shape
    dev = target.device
    need = holo.ospr_workspace_size(H, W, N, precision)
    if ws is None or ws.numel() < need:
        ws = _ws(need, dev)
    b = out_bits if out_bits is not None else (
        torch.empty((N, H * W // 32), dtype=torch.int32, device=dev) if bits else None)
    r = out_replay if out_replay is not None else (
        torch.empty((H, W), dtype=torch.float32, device=dev) if replay else None)
    holo.ospr_generate(target, H, W, N, codes, L, levels, seed, start, stride, precision,
                       b, r, ws, ws.numel(), stream=stream)
    return b, r


def ospr_fresnel(target, N, kappa, codes=None, L=0, levels=256, seed=0, start=0, stride=0, bits=True,
                 replay=True, ws=None, stream=None):
    """OSPR with Fresnel propagation; returns (bits int32 [N, H*W/32] or None, replay or None)."""
    H, W = target.shape
    dev = target.device
    need = holo.ospr_fresnel_workspace_size(H, W, N)
    if ws is None or ws.numel() < need:
        ws = _ws(need, dev)
    b = torch.empty((N, H * W // 32), dtype=torch.int32, device=dev) if bits else None
    r = torch.empty((H, W), dtype=torch.float32, device=dev) if replay else None
    holo.ospr_generate_fresnel(target, H, W, N, codes, L, levels, seed, start, stride, kappa, b, r, ws,
                               ws.numel(), stream=stream)
    return b, r


def gs(target, iters, levels=256, codes=None, L=0, lut_levels=256, seed=0, start=0,
       init_phase=None, state_in=None, want_state=False, want_codes=True, want_replay=True,
       ws=None, precision=holo.HOLO_FP32, stream=None):
    """Returns a dict with 'codes' uint8 [H,W], 'replay' float32, 'err' float64 [iters], 'state'."""
    H, W = target.shape
    dev = target.device
    need = holo.gs_workspace_size(H, W, iters, precision)
    if ws is None or ws.numel() < need:
        ws = _ws(need, dev)
    out = {
        "codes": torch.empty((H, W), dtype=torch.uint8, device=dev) if want_codes else None,
        "replay": torch.empty((H, W), dtype=torch.float32, device=dev) if want_replay else None,
        "err": torch.empty(iters, dtype=torch.float64, device=dev),
        "state": torch.empty((H, W, 2), dtype=torch.float32, device=dev) if want_state else None,
    }
    holo.gs_iterate(target, H, W, iters, levels, init_phase, codes, L, lut_levels, seed, start,
                    precision, out["codes"], out["replay"], out["err"], state_in, out["state"],
                    ws, ws.numel(), stream=stream)
    return out


def gs_fresnel(target, iters, kappa, levels=256, codes=None, L=0, lut_levels=256, seed=0, start=0,
               init_phase=None, ws=None, stream=None):
    """GS under Fresnel propagation; returns a dict with 'codes', 'replay' and 'err'."""
    H, W = target.shape
    dev = target.device
    need = holo.gs_workspace_size(H, W, iters)
    if ws is None or ws.numel() < need:
        ws = _ws(need, dev)
    out = {"codes": torch.empty((H, W), dtype=torch.uint8, device=dev),
           "replay": torch.empty((H, W), dtype=torch.float32, device=dev),
           "err": torch.empty(iters, dtype=torch.float64, device=dev)}
    holo.gs_iterate_fresnel(target, H, W, iters, levels, init_phase, codes, L, lut_levels, seed, start, kappa,
                            out["codes"], out["replay"], out["err"], None, None, ws, ws.numel(), stream=stream)
    return out


def error(replay, target, mask=None, ws=None, out=None, stream=None):
    """Returns a float64 tensor [alpha, mse, nmse] on the device."""
    H, W = target.shape
    dev = target.device
    need = holo.replay_error_workspace_size(H, W)
    if ws is None or ws.numel() < need:
        ws = _ws(need, dev)
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=dev)
    holo.replay_error(replay, target, mask, H, W, out, ws, ws.numel(), stream=stream)
    return out
