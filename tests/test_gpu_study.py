"""The LUT-length study (Section 5.2, Figs. 5-6) driver on a small configuration: its frames
are ordinary batch frames, so one of them is checked against the oracle end to end; the
study's summary must show the paper's qualitative facts (tiny tables far worse, long prime
tables as good as independent phases)."""

import numpy as np
import pytest

from oracle import error as oerr
from oracle import lut as olut
from oracle import ospr as oospr
from paper_2004_04049_gb300 import study
from parity import NMSE_REL
from synthetic import blob_target

pytestmark = pytest.mark.gpu


def test_small_study_against_oracle(cuda):
    S, N, runs = 64, 8, 4
    res = study.lut_length_study(sizes=(S,), N=N, runs=runs, n_targets=2, points=8, device=cuda)
    rows = {r["L"]: r for r in res[f"{S}x{S}"]["rows"]}
    assert rows[2]["mean"] > 1.5                     # two table entries: far worse
    big = [r for L, r in rows.items() if L > 4 * N * S * S // 2]
    assert big and all(abs(r["mean"] - 1.0) < 0.1 for r in big)
    # frame (target 0, run 0, L = 10007) end to end against the oracle
    T = blob_target(S, S, 1000)
    L, seed = 10007, 1
    table = olut.lut_codes(seed, L)
    _, I, _ = oospr.ospr(T.astype(np.float64), N, table, L, seed)
    _, _, nmse = oerr.replay_error(I, T.astype(np.float64))
    res1 = study.lut_length_study(sizes=(S,), N=N, runs=1, n_targets=1, points=2, device=cuda)
    r1 = {r["L"]: r for r in res1[f"{S}x{S}"]["rows"]}[L]
    g1 = r1["per_target"][0] * res1[f"{S}x{S}"]["unrepeated_nmse"][0]
    assert abs(g1 - nmse) <= 10 * NMSE_REL * nmse, (g1, nmse)
