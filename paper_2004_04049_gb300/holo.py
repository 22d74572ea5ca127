"""ctypes binding of ``libholo.so`` with the C ABI's names (see include/holo.h).

Argument marshalling only: every buffer argument is a torch CUDA tensor (its
``data_ptr()`` is passed) or None for NULL, and ``stream`` defaults to PyTorch's current
stream on the tensor's device. Every step of the computation runs in the library's
kernels; there is no fallback. A missing library or a non-OK status raises.
"""

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libholo.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "holo.h")

HOLO_OK = 0
HOLO_EINVAL = -1
HOLO_EUNSUPPORTED = -2
HOLO_ECUDA = -3
HOLO_ETIMEOUT = -4
HOLO_ENOMEM = -5
HOLO_EWORKSPACE = -6
HOLO_FP32, HOLO_FP16X2, HOLO_BF16X2 = 0, 1, 2
NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024
L_UNREPEATED = -1

_STATUS_NAMES = {0: "HOLO_OK", -1: "HOLO_EINVAL", -2: "HOLO_EUNSUPPORTED", -3: "HOLO_ECUDA",
                 -4: "HOLO_ETIMEOUT", -5: "HOLO_ENOMEM", -6: "HOLO_EWORKSPACE"}


class HoloError(RuntimeError):
    def __init__(self, status, func, message):
        super().__init__(f"{func} -> {_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None

_c = ctypes


class FrameDesc(ctypes.Structure):
    """holo_frame_desc of include/holo.h (same field order and C layout)."""
    _fields_ = [("d_target", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("N", ctypes.c_int),
                ("d_codes", ctypes.c_void_p), ("L", ctypes.c_int64), ("levels", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("build_lut", ctypes.c_int), ("start_index", ctypes.c_int64),
                ("subframe_stride", ctypes.c_int64), ("d_holo_bits", ctypes.c_void_p),
                ("d_replay", ctypes.c_void_p), ("d_err", ctypes.c_void_p)]


def frame_desc(d_target, H, W, N, d_codes=None, L=0, levels=256, seed=0, build_lut=False, start_index=0,
               subframe_stride=0, d_holo_bits=None, d_replay=None, d_err=None):
    return FrameDesc(_ptr(d_target), H, W, N, _ptr(d_codes), L, levels, seed, 1 if build_lut else 0,
                     start_index, subframe_stride, _ptr(d_holo_bits), _ptr(d_replay), _ptr(d_err))


def frame_array(descs):
    arr = (FrameDesc * len(descs))(*descs)
    return arr


class FrameHost(ctypes.Structure):
    """holo_frame_host of include/holo.h: optional host buffers of one batch frame."""
    _fields_ = [("h_target", ctypes.c_void_p), ("h_holo_bits", ctypes.c_void_p), ("h_replay", ctypes.c_void_p),
                ("h_err", ctypes.c_void_p)]


def frame_host(h_target=None, h_holo_bits=None, h_replay=None, h_err=None):
    """Host tensors (page-locked for asynchronous copies) or addresses, each optional."""
    return FrameHost(_ptr(h_target), _ptr(h_holo_bits), _ptr(h_replay), _ptr(h_err))


def frame_host_array(hosts):
    return (FrameHost * len(hosts))(*hosts)
_SIGS = {
    "holo_version": (_c.c_int, []),
    "holo_last_error": (_c.c_char_p, []),
    "holo_check": (_c.c_int, [_c.c_void_p]),
    "holo_launch_count": (_c.c_int, [_c.POINTER(_c.c_uint64)]),
    "holo_profile_enable": (_c.c_int, [_c.c_int]),
    "holo_profile_reset": (_c.c_int, []),
    "holo_profile_read": (_c.c_int, [_c.c_char_p, _c.POINTER(_c.c_uint64), _c.POINTER(_c.c_double)]),
    "lut_build": (_c.c_int, [_c.c_uint64, _c.c_int64, _c.c_int, _c.c_void_p, _c.c_void_p, _c.c_void_p]),
    "lfsr_build": (_c.c_int, [_c.c_uint32, _c.c_int64, _c.c_int64, _c.c_int, _c.c_void_p, _c.c_void_p]),
    "ospr_workspace_size": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "ospr_generate": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int,
                                 _c.c_void_p, _c.c_int64, _c.c_int, _c.c_uint64,
                                 _c.c_int64, _c.c_int64, _c.c_int,
                                 _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_size_t, _c.c_void_p]),
    "ospr_fresnel_workspace_size": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "ospr_generate_fresnel": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int,
                                         _c.c_void_p, _c.c_int64, _c.c_int, _c.c_uint64,
                                         _c.c_int64, _c.c_int64, _c.c_double,
                                         _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_size_t, _c.c_void_p]),
    "ospr_generate_noalloc": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int,
                                         _c.c_void_p, _c.c_int64, _c.c_int, _c.c_uint64,
                                         _c.c_int64, _c.c_int64, _c.c_int,
                                         _c.c_void_p, _c.c_void_p, _c.c_void_p]),
    "ospr_batch_workspace_size": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "ospr_generate_batch": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_size_t, _c.c_void_p]),
    "ospr_generate_batch_host": (_c.c_int, [_c.c_void_p, _c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_size_t,
                                            _c.c_void_p]),
    "ospr_batch_graph_create": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_size_t,
                                           _c.POINTER(_c.c_void_p)]),
    "ospr_batch_persistent_workspace_size": (_c.c_int, [_c.c_void_p, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "ospr_generate_batch_persistent": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_size_t,
                                                  _c.c_void_p]),
    "ospr_batch_persistent_graph_create": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_size_t,
                                                      _c.POINTER(_c.c_void_p)]),
    "holo_graph_launch": (_c.c_int, [_c.c_void_p, _c.c_void_p]),
    "holo_graph_destroy": (_c.c_int, [_c.c_void_p]),
    "ospr_autotune": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_void_p, _c.POINTER(_c.c_double)]),
    "ospr_tuning_get": (_c.c_int, [_c.c_int, _c.c_int] + [_c.POINTER(_c.c_int)] * 5),
    "ospr_tuning_set": (_c.c_int, [_c.c_int] * 7),
    "gs_workspace_size": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "gs_tuning_set": (_c.c_int, [_c.c_int] * 4),
    "gs_tuning_get": (_c.c_int, [_c.c_int, _c.c_int, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "gs_iterate": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_void_p,
                              _c.c_void_p, _c.c_int64, _c.c_int, _c.c_uint64, _c.c_int64, _c.c_int,
                              _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p,
                              _c.c_void_p, _c.c_size_t, _c.c_void_p]),
    "gs_iterate_fresnel": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_void_p,
                                      _c.c_void_p, _c.c_int64, _c.c_int, _c.c_uint64, _c.c_int64, _c.c_double,
                                      _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p,
                                      _c.c_void_p, _c.c_size_t, _c.c_void_p]),
    "gs_state_phase": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_void_p]),
    "gs_batch_workspace_size": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int,
                                           _c.POINTER(_c.c_size_t)]),
    "gs_iterate_batch": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_void_p,
                                    _c.c_void_p, _c.c_int64, _c.c_int, _c.c_uint64, _c.c_int64, _c.c_int,
                                    _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p,
                                    _c.c_void_p, _c.c_size_t, _c.c_void_p]),
    "ws_phase_resample": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_void_p,
                                     _c.c_void_p]),
    "ws_adam_update": (_c.c_int, [_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int64, _c.c_float,
                                  _c.c_float, _c.c_float, _c.c_float, _c.c_int, _c.c_void_p]),
    "ws_net_create": (_c.c_int, [_c.POINTER(_c.c_void_p), _c.c_uint64, _c.c_int]),
    "ws_net_destroy": (_c.c_int, [_c.c_void_p]),
    "ws_net_param_count": (_c.c_int, [_c.c_void_p, _c.POINTER(_c.c_int64)]),
    "ws_train_step": (_c.c_int, [_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_float, _c.c_void_p,
                                 _c.c_void_p]),
    "ws_forward_backward": (_c.c_int, [_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_void_p, _c.c_void_p]),
    "ws_infer": (_c.c_int, [_c.c_void_p, _c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_void_p]),
    "ws_get_tensor": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_int64]),
    "ws_set_tensor": (_c.c_int, [_c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p, _c.c_int64]),
    "ws_layer_shape": (_c.c_int, [_c.c_int, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "ws_get_activation": (_c.c_int, [_c.c_void_p, _c.c_char_p, _c.c_int, _c.c_void_p, _c.c_int64]),
    "ws_save": (_c.c_int, [_c.c_void_p, _c.c_char_p]),
    "ws_load": (_c.c_int, [_c.c_void_p, _c.c_char_p]),
    "nn_conv3x3": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_void_p, _c.c_void_p,
                              _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_void_p, _c.c_void_p,
                              _c.c_void_p, _c.c_void_p]),
    "holo_tc_status": (_c.c_int, [_c.POINTER(_c.c_int), _c.c_int]),
    "holo_wait_selftest": (_c.c_int, [_c.c_int, _c.c_void_p]),
    "replay_error_workspace_size": (_c.c_int, [_c.c_int, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "replay_error": (_c.c_int, [_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_int,
                                _c.c_void_p, _c.c_void_p, _c.c_size_t, _c.c_void_p]),
}


def load(path=None):
    """Load libholo.so (once) and return the ctypes handle. Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run paper_2004_04049_gb300.build_lib.build() "
                           "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions(header=HEADER):
    """Names of the functions include/holo.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream, *tensors):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    dev = None
    for t in tensors:
        if t is not None and not isinstance(t, int):
            dev = t.device
            break
    if dev is None:
        return 0            # raw pointers: the legacy default stream
    import torch
    return torch.cuda.current_stream(dev).cuda_stream


def _call(name, *args):
    lib = load()
    rc = getattr(lib, name)(*args)
    if rc != HOLO_OK:
        msg = lib.holo_last_error().decode(errors="replace")
        raise HoloError(rc, name, msg)
    return rc


def last_error():
    return load().holo_last_error().decode(errors="replace")


# ------------------------------------------------------------------ utilities ----
def holo_version():
    return load().holo_version()


def holo_check(stream=None):
    return _call("holo_check", _stream(stream))


def holo_launch_count():
    n = ctypes.c_uint64(0)
    _call("holo_launch_count", ctypes.byref(n))
    return n.value


def holo_profile_enable(on=True):
    return _call("holo_profile_enable", 1 if on else 0)


def holo_profile_reset():
    return _call("holo_profile_reset")


def holo_profile_read(name):
    n = ctypes.c_uint64(0)
    ms = ctypes.c_double(0.0)
    _call("holo_profile_read", name.encode(), ctypes.byref(n), ctypes.byref(ms))
    return n.value, ms.value


# ------------------------------------------------------------------- compute ----
def lut_build(seed, L, levels, d_codes, d_cs=None, stream=None):
    return _call("lut_build", seed, L, levels, _ptr(d_codes), _ptr(d_cs), _stream(stream, d_codes))


def lfsr_build(seed_state, start, count, levels, d_codes, stream=None):
    """m-sequence codes start .. start+count-1 into d_codes (a table for table mode)."""
    return _call("lfsr_build", seed_state, start, count, levels, _ptr(d_codes), _stream(stream, d_codes))


def ospr_workspace_size(H, W, N, precision=HOLO_FP32):
    b = ctypes.c_size_t(0)
    _call("ospr_workspace_size", H, W, N, precision, ctypes.byref(b))
    return b.value


def ospr_generate(d_target, H, W, N, d_codes, L, levels, seed, start_index, subframe_stride,
                  precision, d_holo_bits, d_replay, d_ws, ws_bytes=None, stream=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("ospr_generate", _ptr(d_target), H, W, N, _ptr(d_codes), L, levels, seed,
                 start_index, subframe_stride, precision, _ptr(d_holo_bits), _ptr(d_replay),
                 _ptr(d_ws), ws_bytes, _stream(stream, d_target))


def ospr_fresnel_workspace_size(H, W, N):
    b = ctypes.c_size_t(0)
    _call("ospr_fresnel_workspace_size", H, W, N, ctypes.byref(b))
    return b.value


def ospr_generate_fresnel(d_target, H, W, N, d_codes, L, levels, seed, start_index, subframe_stride,
                          kappa, d_holo_bits, d_replay, d_ws, ws_bytes=None, stream=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("ospr_generate_fresnel", _ptr(d_target), H, W, N, _ptr(d_codes), L, levels, seed,
                 start_index, subframe_stride, float(kappa), _ptr(d_holo_bits), _ptr(d_replay),
                 _ptr(d_ws), ws_bytes, _stream(stream, d_target))


def ospr_generate_noalloc(d_target, H, W, N, d_codes, L, levels, seed, start_index,
                          subframe_stride, precision, d_holo_bits, d_replay, stream=None):
    """ospr_generate on the library's fixed scratch array (no workspace argument)."""
    return _call("ospr_generate_noalloc", _ptr(d_target), H, W, N, _ptr(d_codes), L, levels, seed,
                 start_index, subframe_stride, precision, _ptr(d_holo_bits), _ptr(d_replay),
                 _stream(stream, d_target))


def ospr_batch_workspace_size(frames, precision=HOLO_FP32):
    """frames: a ctypes array made by frame_array()."""
    b = ctypes.c_size_t(0)
    _call("ospr_batch_workspace_size", ctypes.cast(frames, ctypes.c_void_p), len(frames), precision,
          ctypes.byref(b))
    return b.value


def ospr_generate_batch(frames, precision, d_ws, ws_bytes=None, stream=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("ospr_generate_batch", ctypes.cast(frames, ctypes.c_void_p), len(frames), precision,
                 _ptr(d_ws), ws_bytes, _stream(stream, d_ws))


def ospr_generate_batch_host(frames, hosts, precision, d_ws, ws_bytes=None, stream=None):
    if len(hosts) != len(frames):
        raise ValueError("one host entry per frame")
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("ospr_generate_batch_host", ctypes.cast(frames, ctypes.c_void_p), ctypes.cast(hosts, ctypes.c_void_p),
                 len(frames), precision, _ptr(d_ws), ws_bytes, _stream(stream, d_ws))


def ospr_batch_graph_create(frames, precision, d_ws, ws_bytes=None):
    """Returns an opaque graph handle (int)."""
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    g = ctypes.c_void_p(0)
    _call("ospr_batch_graph_create", ctypes.cast(frames, ctypes.c_void_p), len(frames), precision,
          _ptr(d_ws), ws_bytes, ctypes.byref(g))
    return g.value


def ospr_batch_persistent_workspace_size(frames):
    b = ctypes.c_size_t(0)
    _call("ospr_batch_persistent_workspace_size", ctypes.cast(frames, ctypes.c_void_p), len(frames), ctypes.byref(b))
    return b.value


def ospr_generate_batch_persistent(frames, d_ws, wait_limit_us=0, ws_bytes=None, stream=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("ospr_generate_batch_persistent", ctypes.cast(frames, ctypes.c_void_p), len(frames), wait_limit_us,
                 _ptr(d_ws), ws_bytes, _stream(stream, d_ws))


def ospr_batch_persistent_graph_create(frames, d_ws, wait_limit_us=0, ws_bytes=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    g = ctypes.c_void_p(0)
    _call("ospr_batch_persistent_graph_create", ctypes.cast(frames, ctypes.c_void_p), len(frames), wait_limit_us,
          _ptr(d_ws), ws_bytes, ctypes.byref(g))
    return g.value


def holo_graph_launch(graph, stream=None):
    s = stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else None)
    if s is None:
        import torch
        s = torch.cuda.current_stream().cuda_stream
    return _call("holo_graph_launch", graph, s)


def holo_graph_destroy(graph):
    return _call("holo_graph_destroy", graph)


def ospr_autotune(H, W, N, reps=3, stream=None):
    """Times candidate tunings for this shape and installs the fastest; returns ms per call."""
    ms = ctypes.c_double(0.0)
    s = stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else None)
    if s is None:
        import torch
        s = torch.cuda.current_stream().cuda_stream
    _call("ospr_autotune", H, W, N, reps, s, ctypes.byref(ms))
    return ms.value


def ospr_tuning_get(H, W):
    v = [ctypes.c_int(0) for _ in range(5)]
    _call("ospr_tuning_get", H, W, *[ctypes.byref(x) for x in v])
    return {"col_ifft_variant": v[0].value, "col_fft_variant": v[1].value, "row_variant": v[2].value,
            "chunk": v[3].value, "groups": v[4].value}


def ospr_tuning_set(H, W, col_ifft_variant=0, col_fft_variant=0, row_variant=0, chunk=16, groups=4):
    return _call("ospr_tuning_set", H, W, col_ifft_variant, col_fft_variant, row_variant, chunk, groups)


def gs_tuning_set(H, W, col_variant=-1, row_variant=-1):
    """Tile variants of the GS passes for this shape; -1 restores the defaults."""
    return _call("gs_tuning_set", H, W, col_variant, row_variant)


def gs_tuning_get(H, W):
    v = [ctypes.c_int(0) for _ in range(2)]
    _call("gs_tuning_get", H, W, *[ctypes.byref(x) for x in v])
    return {"col_variant": v[0].value, "row_variant": v[1].value}


def gs_workspace_size(H, W, iters, precision=HOLO_FP32):
    b = ctypes.c_size_t(0)
    _call("gs_workspace_size", H, W, iters, precision, ctypes.byref(b))
    return b.value


def gs_iterate(d_target, H, W, iters, levels, d_init_phase, d_codes, L, lut_levels, seed,
               start_index, precision, d_phase_codes, d_replay, d_err, d_state_in, d_state_out,
               d_ws, ws_bytes=None, stream=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("gs_iterate", _ptr(d_target), H, W, iters, levels, _ptr(d_init_phase),
                 _ptr(d_codes), L, lut_levels, seed, start_index, precision,
                 _ptr(d_phase_codes), _ptr(d_replay), _ptr(d_err), _ptr(d_state_in),
                 _ptr(d_state_out), _ptr(d_ws), ws_bytes, _stream(stream, d_target))


def gs_iterate_fresnel(d_target, H, W, iters, levels, d_init_phase, d_codes, L, lut_levels, seed,
                       start_index, kappa, d_phase_codes, d_replay, d_err, d_state_in, d_state_out,
                       d_ws, ws_bytes=None, stream=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("gs_iterate_fresnel", _ptr(d_target), H, W, iters, levels, _ptr(d_init_phase),
                 _ptr(d_codes), L, lut_levels, seed, start_index, float(kappa),
                 _ptr(d_phase_codes), _ptr(d_replay), _ptr(d_err), _ptr(d_state_in),
                 _ptr(d_state_out), _ptr(d_ws), ws_bytes, _stream(stream, d_target))


def gs_batch_workspace_size(B, H, W, iters, precision=HOLO_FP32):
    b = ctypes.c_size_t(0)
    _call("gs_batch_workspace_size", B, H, W, iters, precision, ctypes.byref(b))
    return b.value


def gs_iterate_batch(d_targets, B, H, W, iters, levels, d_init_phases, d_codes, L, lut_levels, seed,
                     start_index, precision, d_phase_codes, d_replay, d_err, d_states_in, d_states_out,
                     d_ws, ws_bytes=None, stream=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("gs_iterate_batch", _ptr(d_targets), B, H, W, iters, levels, _ptr(d_init_phases),
                 _ptr(d_codes), L, lut_levels, seed, start_index, precision,
                 _ptr(d_phase_codes), _ptr(d_replay), _ptr(d_err), _ptr(d_states_in),
                 _ptr(d_states_out), _ptr(d_ws), ws_bytes, _stream(stream, d_targets))


def gs_state_phase(d_state, H, W, d_phase, stream=None):
    return _call("gs_state_phase", _ptr(d_state), H, W, _ptr(d_phase), _stream(stream, d_state))


def replay_error_workspace_size(H, W):
    b = ctypes.c_size_t(0)
    _call("replay_error_workspace_size", H, W, ctypes.byref(b))
    return b.value


def replay_error(d_replay, d_target, d_mask, H, W, d_out, d_ws, ws_bytes=None, stream=None):
    if ws_bytes is None:
        ws_bytes = d_ws.numel() * d_ws.element_size()
    return _call("replay_error", _ptr(d_replay), _ptr(d_target), _ptr(d_mask), H, W, _ptr(d_out),
                 _ptr(d_ws), ws_bytes, _stream(stream, d_replay))


# -------------------------------------------------------- learned warm start ----
def ws_net_create(seed, max_batch):
    h = ctypes.c_void_p(0)
    _call("ws_net_create", ctypes.byref(h), seed, max_batch)
    return h.value


def ws_net_destroy(net):
    return _call("ws_net_destroy", net)


def ws_net_param_count(net):
    n = ctypes.c_int64(0)
    _call("ws_net_param_count", net, ctypes.byref(n))
    return n.value


def ws_train_step(net, d_targets, d_label_phase, batch, lr, d_loss=None, stream=None):
    return _call("ws_train_step", net, _ptr(d_targets), _ptr(d_label_phase), batch, lr, _ptr(d_loss),
                 _stream(stream, d_targets))


def ws_forward_backward(net, d_targets, d_label_phase, batch, d_loss=None, stream=None):
    return _call("ws_forward_backward", net, _ptr(d_targets), _ptr(d_label_phase), batch, _ptr(d_loss),
                 _stream(stream, d_targets))


def ws_infer(net, d_target, H, W, d_phase_out, stream=None):
    return _call("ws_infer", net, _ptr(d_target), H, W, _ptr(d_phase_out), _stream(stream, d_target))


def ws_phase_resample(d_uv, channels, H, W, Ho, Wo, d_phase, stream=None):
    return _call("ws_phase_resample", _ptr(d_uv), channels, H, W, Ho, Wo, _ptr(d_phase), _stream(stream, d_uv))


def ws_adam_update(d_w, d_g, d_m, d_v, n, lr, beta1, beta2, eps, step, stream=None):
    return _call("ws_adam_update", _ptr(d_w), _ptr(d_g), _ptr(d_m), _ptr(d_v), n, lr, beta1, beta2, eps, step,
                 _stream(stream, d_w))


def ws_layer_shape(layer):
    a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _call("ws_layer_shape", layer, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def ws_get_tensor(net, layer, which):
    """Host numpy copy: which 0 weights [Cout,3,3,Cin], 1 biases, 2 dW, 3 db."""
    import numpy as np
    cin, cout, _ = ws_layer_shape(layer)
    shape = (cout, 3, 3, cin) if which in (0, 2) else (cout,)
    out = np.zeros(shape, dtype=np.float32)
    _call("ws_get_tensor", net, layer, which, out.ctypes.data, out.size)
    return out


def ws_set_tensor(net, layer, which, array):
    import numpy as np
    a = np.ascontiguousarray(array, dtype=np.float32)
    return _call("ws_set_tensor", net, layer, which, a.ctypes.data, a.size)


_ACT_SHAPES = {"x0": (8, 1), "a1": (32, 1), "s1": (32, 1), "p1": (32, 2), "a2": (64, 2), "s2": (64, 2),
               "p2": (64, 4), "a3": (128, 4), "s3": (128, 4), "p3": (128, 8), "a4": (128, 8), "b4": (128, 8),
               "up4": (128, 4), "u5": (128, 4), "up5": (128, 2), "u6": (64, 2), "up6": (64, 1), "u7": (32, 1),
               "out": (8, 1), "g_out": (8, 1), "g_u7": (32, 1), "g_up6": (64, 1), "g_u6": (64, 2), "g_s1": (32, 1)}


def ws_get_activation(net, name, batch=1):
    """Host float32 copy [batch, H, W, C] of a stored tensor of the last pass."""
    import numpy as np
    c, div = _ACT_SHAPES[name]
    r = 256 // div
    out = np.zeros((batch, r, r, c), dtype=np.float32)
    _call("ws_get_activation", net, name.encode(), batch, out.ctypes.data, out.size)
    return out


def ws_save(net, path):
    return _call("ws_save", net, str(path).encode())


def ws_load(net, path):
    return _call("ws_load", net, str(path).encode())


def nn_conv3x3(mode, B, H, W, Cin, Cout, d_in, d_wmat=None, d_dy=None, d_bias=None, d_residual=None, relu=False,
               d_out=None, d_out_f32=None, d_dw=None, stream=None):
    return _call("nn_conv3x3", mode, B, H, W, Cin, Cout, _ptr(d_in), _ptr(d_wmat), _ptr(d_dy), _ptr(d_bias),
                 _ptr(d_residual), 1 if relu else 0, _ptr(d_out), _ptr(d_out_f32), _ptr(d_dw),
                 _stream(stream, d_in))


HOLO_CONV_LEGACY = 16


def holo_tc_status(clear=False):
    """1 if a tcgen05 kernel gave up on a bounded wait since the last clear."""
    v = ctypes.c_int(0)
    _call("holo_tc_status", ctypes.byref(v), 1 if clear else 0)
    return v.value


def holo_wait_selftest(limit=1000, stream=None):
    """Raw status of the bounded-wait self-test (HOLO_ETIMEOUT is the expected result)."""
    s = stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else None)
    if s is None:
        import torch
        s = torch.cuda.current_stream().cuda_stream
    return load().holo_wait_selftest(limit, s)
