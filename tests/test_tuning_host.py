"""Host-side tuning state, no GPU: a tuning cache named by HOLO_TUNE_CACHE is read on first
use (a line with chunk or groups out of range is skipped; a variant that the line length
lacks falls back to 0) and the workspace size follows the installed setting;
HOLO_OSPR_CHUNK and HOLO_OSPR_GROUPS set the chunking of shapes without a setting. Each
case runs in a child process, since both are read once per process."""

import json
import os
import subprocess
import sys
import textwrap

import pytest

from paper_2004_04049_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import json, sys
    sys.path.insert(0, {root!r})
    from paper_2004_04049_gb300 import holo
    holo.load()
    out = {{"t1024": holo.ospr_tuning_get(1024, 1024), "t256x512": holo.ospr_tuning_get(256, 512),
            "t512": holo.ospr_tuning_get(512, 512),
            "ws1024": holo.ospr_workspace_size(1024, 1024, 24), "ws512": holo.ospr_workspace_size(512, 512, 24)}}
    print(json.dumps(out))
""")


@pytest.fixture(scope="module")
def built():
    build_lib.build()


def _child(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def _line(H, W, ci, cf, rv, chunk, groups):
    return (f'{{"H": {H}, "W": {W}, "col_ifft_variant": {ci}, "col_fft_variant": {cf}, '
            f'"row_variant": {rv}, "chunk": {chunk}, "groups": {groups}}}\n')


def test_tuning_cache_and_chunking_defaults(built, tmp_path):
    cache = tmp_path / "tune.jsonl"
    cache.write_text(_line(1024, 1024, 1, 2, 1, 6, 3)       # installed as written
                     + _line(256, 512, 2, 1, 1, 5, 2)        # 256-point columns: variants fall back to 0
                     + _line(512, 512, 1, 1, 0, 99, 2))      # chunk out of range: skipped
    out = _child({"HOLO_TUNE_CACHE": str(cache), "HOLO_OSPR_CHUNK": "8", "HOLO_OSPR_GROUPS": "2"})
    assert out["t1024"] == {"col_ifft_variant": 1, "col_fft_variant": 2, "row_variant": 1, "chunk": 6, "groups": 3}
    assert out["t256x512"] == {"col_ifft_variant": 0, "col_fft_variant": 0, "row_variant": 1, "chunk": 5,
                               "groups": 2}
    # 512^2 has no setting: the environment's chunking, variant 0 tiles
    assert out["t512"] == {"col_ifft_variant": 0, "col_fft_variant": 0, "row_variant": 0, "chunk": 8, "groups": 2}
    P1, P5 = 1024 * 1024, 512 * 512
    assert out["ws1024"] == 6 * 8 * P1 + 3 * 4 * P1     # 6 complex64 fields, 3 float32 accumulators
    assert out["ws512"] == 8 * 8 * P5 + 2 * 4 * P5       # 12 pairs, 8 in flight


def test_no_cache_gives_the_built_in_defaults(built):
    env = {k: "" for k in ("HOLO_TUNE_CACHE", "HOLO_OSPR_CHUNK", "HOLO_OSPR_GROUPS")}
    out = _child(env)
    assert out["t1024"] == {"col_ifft_variant": 0, "col_fft_variant": 0, "row_variant": 0, "chunk": 16,
                            "groups": 4}
    assert out["ws1024"] == 12 * 8 * 1024 * 1024 + 4 * 4 * 1024 * 1024   # N = 24: 12 pairs, 4 groups
