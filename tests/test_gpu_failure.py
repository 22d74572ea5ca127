"""Failure detection without a GPU fault: the bounded wait of the tcgen05 kernels, made to
run out on an mbarrier that nothing arrives at, returns HOLO_ETIMEOUT, sets the sticky
status that holo_check reports, and leaves the context usable."""

import pytest
import torch

from paper_2004_04049_gb300 import holo, pipeline
from synthetic import blob_target

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(cuda):
    s = torch.cuda.current_stream(cuda).cuda_stream
    holo.holo_tc_status(clear=True)
    holo.holo_check(s)
    assert holo.holo_wait_selftest(1000, s) == holo.HOLO_ETIMEOUT
    assert "gave up" in holo.last_error()
    assert holo.holo_tc_status() == 1
    with pytest.raises(holo.HoloError) as ei:
        holo.holo_check(s)
    assert ei.value.status == holo.HOLO_ETIMEOUT
    assert holo.holo_tc_status(clear=True) == 1
    assert holo.holo_tc_status() == 0
    holo.holo_check(s)
    # the context still computes: a small frame matches a second run of itself
    T = torch.from_numpy(blob_target(128, 128, 1000)).to(cuda)
    codes = pipeline.lut(5, 1031, device=cuda)
    b1, I1 = pipeline.ospr(T, 4, codes, 1031, 256, 5)
    b2, I2 = pipeline.ospr(T, 4, codes, 1031, 256, 5)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2) and torch.equal(I1, I2) and float(I1.sum()) > 0


def test_selftest_rejects_bad_limits(cuda):
    s = torch.cuda.current_stream(cuda).cuda_stream
    assert holo.holo_wait_selftest(0, s) == holo.HOLO_EINVAL
    assert holo.holo_wait_selftest(1 << 25, s) == holo.HOLO_EINVAL
