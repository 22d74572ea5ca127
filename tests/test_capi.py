"""The C-ABI library builds for sm_103a, loads, and exports every function include/holo.h
declares. Only host-side paths run here (sizes, argument validation): no GPU is needed."""

import ctypes

import pytest

from paper_2004_04049_gb300 import build_lib, holo


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return holo.load()


def test_header_declares_the_boundary():
    names = holo.header_functions()
    for required in ("lut_build", "ospr_generate", "gs_iterate", "replay_error",
                     "ospr_workspace_size", "gs_workspace_size", "replay_error_workspace_size",
                     "holo_last_error", "holo_check"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = holo.header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding marshals every declared function
    assert set(names) <= set(holo._SIGS), set(names) - set(holo._SIGS)


def test_version_and_empty_error(lib):
    assert holo.holo_version() >= 10000
    assert isinstance(holo.last_error(), str)


def test_workspace_sizes_are_host_only(lib):
    a = holo.ospr_workspace_size(1024, 1024, 24)
    # 12 pairs of complex64 fields in flight plus 4 float32 accumulators
    assert a >= 12 * 1024 * 1024 * 8 + 4 * 1024 * 1024 * 4
    assert holo.ospr_workspace_size(256, 256, 1) >= 256 * 256 * 8
    assert holo.gs_workspace_size(1024, 1024, 20) >= 1024 * 1024 * 8
    assert holo.replay_error_workspace_size(2, 2) > 0


@pytest.mark.parametrize("H,W", [(100, 128), (32, 64), (8192, 64), (64, 0)])
def test_unsupported_shapes_rejected(lib, H, W):
    with pytest.raises(holo.HoloError) as ei:
        holo.ospr_workspace_size(H, W, 4)
    assert ei.value.status in (holo.HOLO_EUNSUPPORTED, holo.HOLO_EINVAL)
    assert "H=" in holo.last_error()


def test_argument_validation_before_any_cuda_call(lib):
    # rejected on the host: no device is touched
    with pytest.raises(holo.HoloError) as ei:
        holo.lut_build(1, 0, 256, None)
    assert ei.value.status == holo.HOLO_EINVAL
    with pytest.raises(holo.HoloError) as ei:
        holo.lut_build(1, 16, 3, 1 << 20)
    assert ei.value.status == holo.HOLO_EINVAL
    rc = lib.ospr_generate(None, 256, 256, 4, None, 0, 256, 0, 0, 0, 0, None, None, None, 0, None)
    assert rc == holo.HOLO_EINVAL
    rc = lib.ospr_generate(1 << 20, 256, 256, 4, None, 0, 256, 0, 0, 0, 7, None, 1 << 20, 1 << 20,
                           1 << 30, None)
    assert rc == holo.HOLO_EINVAL
    # tensor-core precisions exist for line lengths 1024 and 2048 only
    rc = lib.ospr_generate(1 << 20, 256, 256, 4, None, 0, 256, 0, 0, 0, holo.HOLO_BF16X2, None, 1 << 20,
                           1 << 20, 1 << 30, None)
    assert rc == holo.HOLO_EUNSUPPORTED
    assert holo.ospr_workspace_size(1024, 2048, 24, holo.HOLO_FP16X2) > 0
    rc = lib.ospr_generate(1 << 20, 256, 256, 4, None, 0, 256, 0, 0, 0, 0, None, 1 << 20, 1 << 20,
                           16, None)
    assert rc == holo.HOLO_EWORKSPACE
    rc = lib.gs_iterate(1 << 20, 256, 256, 0, 256, None, None, 0, 256, 0, 0, 0,
                        None, None, None, None, None, None, 0, None)
    assert rc == holo.HOLO_EINVAL
    rc = lib.replay_error(None, None, None, 4, 4, None, None, 0, None)
    assert rc == holo.HOLO_EINVAL
    # the fixed-scratch variant checks its shape against the scratch before looking it up
    for args, status in [((2048, 2048, 4, 0), holo.HOLO_EWORKSPACE), ((1024, 1024, 0, 0), holo.HOLO_EINVAL),
                         ((1024, 1024, 4, holo.HOLO_BF16X2), holo.HOLO_EUNSUPPORTED),
                         ((96, 512, 4, 0), holo.HOLO_EUNSUPPORTED)]:
        H, W, N, prec = args
        with pytest.raises(holo.HoloError) as ei:
            holo.ospr_generate_noalloc(1 << 20, H, W, N, None, 0, 256, 0, 0, 0, prec, 1 << 22, None)
        assert ei.value.status == status, args
    n = ctypes.c_uint64(0)
    assert lib.holo_launch_count(ctypes.byref(n)) == 0


def test_batch_workspace_is_host_only(lib):
    fr = [holo.frame_desc(1 << 20, 512, 512, 9, 1 << 21, 1031, 256, 1, True, 0, 0, 1 << 22, 1 << 23, 1 << 24),
          holo.frame_desc(1 << 20, 1024, 2048, 30, 1 << 21, 4096, 256, 2, True, 0, 0, 1 << 22, 1 << 23, None)]
    arr = holo.frame_array(fr)
    total = holo.ospr_batch_workspace_size(arr)
    assert total >= 2 * holo.ospr_workspace_size(1024, 2048, 30)
    bad = holo.frame_array([holo.frame_desc(1 << 20, 96, 512, 9, None, 0, 256, 0, False, 0, 0, 1 << 22, None, None)])
    with pytest.raises(holo.HoloError) as ei:
        holo.ospr_batch_workspace_size(bad)
    assert "frame 0" in str(ei.value)


def test_persistent_workspace_is_host_only(lib):
    # planning the persistent launch needs no GPU: slots sized for the largest frame, one
    # slot per frame up to eight, plus counters, frame table and queue
    def desc(H, W, N, replay=1 << 23):
        return holo.frame_desc(1 << 20, H, W, N, 1 << 21, 1031, 256, 1, True, 0, 0, 1 << 22, replay, None)
    one = holo.ospr_batch_persistent_workspace_size(holo.frame_array([desc(1024, 1024, 24)]))
    three = holo.ospr_batch_persistent_workspace_size(holo.frame_array([desc(1024, 1024, 24)] * 3))
    assert one >= holo.ospr_workspace_size(1024, 1024, 24) and three > 2 * one
    mixed = holo.ospr_batch_persistent_workspace_size(holo.frame_array([desc(512, 512, 8), desc(2048, 2048, 4)]))
    assert mixed >= 2 * holo.ospr_workspace_size(2048, 2048, 4)
    for bad, status in [(desc(256, 256, 8), holo.HOLO_EUNSUPPORTED), (desc(1024, 1024, 8, None), holo.HOLO_EINVAL),
                        (desc(1024, 1024, 0), holo.HOLO_EINVAL)]:
        with pytest.raises(holo.HoloError) as ei:
            holo.ospr_batch_persistent_workspace_size(holo.frame_array([desc(512, 512, 8), bad]))
        assert ei.value.status == status and "frame 1" in str(ei.value)


def test_tuning_set_get_host_only(lib):
    # 256-point columns have one tile variant: column variants fall back to 0; 512-point
    # rows keep variant 1
    holo.ospr_tuning_set(256, 512, 2, 1, 1, 5, 3)
    try:
        t = holo.ospr_tuning_get(256, 512)
        assert t == {"col_ifft_variant": 0, "col_fft_variant": 0, "row_variant": 1, "chunk": 5, "groups": 3}
        holo.ospr_tuning_set(1024, 1024, 2, 1, 0, 12, 2)
        t = holo.ospr_tuning_get(1024, 1024)
        assert (t["col_ifft_variant"], t["col_fft_variant"], t["chunk"], t["groups"]) == (2, 1, 12, 2)
        # the workspace follows the setting: 12 complex64 fields and 2 float32 accumulators
        assert holo.ospr_workspace_size(1024, 1024, 24) == 12 * 8 * 2**20 + 2 * 4 * 2**20
        for bad in [(3, 0, 0, 4, 1), (0, -1, 0, 4, 1), (0, 0, 2, 4, 1), (0, 0, 0, 17, 1), (0, 0, 0, 4, 5)]:
            with pytest.raises(holo.HoloError) as ei:
                holo.ospr_tuning_set(1024, 1024, *bad)
            assert ei.value.status == holo.HOLO_EINVAL
    finally:
        holo.ospr_tuning_set(256, 512)
        holo.ospr_tuning_set(1024, 1024)


def test_gs_tuning_host_only(lib):
    assert holo.gs_tuning_get(1024, 1024) == {"col_variant": 0, "row_variant": 1}
    assert holo.gs_tuning_get(2048, 2048) == {"col_variant": 1, "row_variant": 1}
    holo.gs_tuning_set(256, 1024, 2, 2)   # 256-point columns have one variant
    try:
        assert holo.gs_tuning_get(256, 1024) == {"col_variant": 0, "row_variant": 2}
        with pytest.raises(holo.HoloError) as ei:
            holo.gs_tuning_set(256, 1024, 3, 0)
        assert ei.value.status == holo.HOLO_EINVAL
    finally:
        holo.gs_tuning_set(256, 1024)
    assert holo.gs_tuning_get(256, 1024) == {"col_variant": 0, "row_variant": 1}


def test_lfsr_build_validation_host_only(lib):
    for args in [(0, 0, 16, 256), (1 << 31, 0, 16, 256), (1, -1, 16, 256), (1, 0, 0, 256), (1, 0, 16, 3)]:
        with pytest.raises(holo.HoloError) as ei:
            holo.lfsr_build(*args, 1 << 20)
        assert ei.value.status == holo.HOLO_EINVAL
    with pytest.raises(holo.HoloError):
        holo.lfsr_build(1, 0, 16, 256, None)


def test_host_fault_injection(lib, monkeypatch):
    monkeypatch.setenv("HOLO_FAULT_INJECT", "plan,timeout,alloc")
    assert lib.holo_check(None) == holo.HOLO_ETIMEOUT
    assert "injected" in holo.last_error()
    v = ctypes.c_double(0.0)
    assert lib.ospr_autotune(256, 256, 4, 1, None, ctypes.byref(v)) == holo.HOLO_ENOMEM
    arr = holo.frame_array([holo.frame_desc(1 << 20, 512, 512, 9, None, 0, 256, 0, False, 0, 0, 1 << 22, None, None)])
    with pytest.raises(holo.HoloError) as ei:
        holo.ospr_batch_workspace_size(arr)
    assert ei.value.status == holo.HOLO_EINVAL and "injected" in str(ei.value)
    monkeypatch.setenv("HOLO_FAULT_INJECT", "allocx")
    assert holo.ospr_batch_workspace_size(arr) > 0
