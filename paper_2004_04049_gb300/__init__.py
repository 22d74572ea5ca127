"""GB300-native LUT phase randomisation for OSPR and GS hologram generation.

The compute path is the C-ABI CUDA library ``libholo.so`` (include/holo.h); ``holo``
binds it with the same names. ``pipeline`` holds small device-buffer helpers used by the
tests and the benchmark.
"""

from . import holo  # noqa: F401
