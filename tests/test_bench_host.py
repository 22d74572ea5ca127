"""Host-side pieces of bench.py (no GPU): the byte models behind the roofline numbers, the
ncu traffic records and the launch signatures they are matched against."""

import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_subframe_byte_model(bench):
    # Section 8(d) model: 16 B/px of transform round trips, P/8 bits, and the per-frame
    # target (4 B/px), accumulator (8 B/px) and table bytes shared by the N sub-frames
    P = 1024 * 1024
    assert bench.subframe_bytes(P, 24, 0) == 16 * P + P // 8 + 12 * P / 24
    assert bench.subframe_bytes(P, 24, 1 << 20) == 16 * P + P // 8 + (12 * P + (1 << 20)) / 24
    # a table longer than every draw of the frame counts only the draws
    assert bench.subframe_bytes(P, 24, 1 << 40) == 16 * P + P // 8 + (12 * P + 24 * P) / 24


def test_kernel_byte_models(bench):
    P = 1 << 20
    assert bench.kernel_bytes("ospr_row", P, 12, 2, 24) == 12 * (16 * P + 2 * P // 8)
    assert bench.kernel_bytes("ospr_col_ifft", P, 12, 2, 24) == 4 * P + 12 * 8 * P + (1 << 20)
    assert bench.kernel_bytes("ospr_col_fft", P, 12, 2, 24) == 12 * 8 * P + 2 * 4 * P
    assert bench.kernel_bytes("ospr_finalize", P, 12, 2, 24) == 2 * 4 * P + 4 * P
    assert bench.kernel_bytes("replay_error", P, 12, 2, 24) == 8 * P
    assert bench.kernel_bytes("no_such_kernel", P, 12, 2, 24) is None


def _ncu_csv(path, rows):
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
           "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]
    with open(path, "w") as fh:
        fh.write("==PROF== some preamble line\n")
        fh.write(",".join(f'"{h}"' for h in hdr) + "\n")
        for i, (kernel, grid, metric, value) in enumerate(rows):
            r = [str(i), "1", "python3", "127.0.0.1", kernel, "1", "7", "(512, 1, 1)", grid, "0", "10.3",
                 "Command line profiler metrics", metric, "byte", value]
            fh.write(",".join(f'"{x}"' for x in r) + "\n")


def test_traffic_record_round_trip(bench, tmp_path, monkeypatch):
    csv_path = tmp_path / "t.csv"
    kernel = "void holo::k_ospr_col_ifft<1024, 0>(holo::OsprArgs)"
    _ncu_csv(csv_path, [(kernel, "(64, 12, 1)", "dram__bytes_read.sum", "4,000,000"),
                        (kernel, "(64, 12, 1)", "dram__bytes_write.sum", "40,000,000"),
                        (kernel, "(64, 12, 1)", "smsp__inst_executed.sum", "37,000,000"),
                        # a later launch of the same family with another grid is ignored
                        (kernel, "(64, 4, 1)", "dram__bytes_read.sum", "1")])
    out = tmp_path / "traffic.json"
    bench.record_traffic(str(csv_path), "ncu ...", str(out))
    rec = json.loads(out.read_text())["ospr_col_ifft"]
    assert rec["kernel"] == "k_ospr_col_ifft<1024, 0>"     # namespace dropped
    assert rec["dram__bytes_read.sum"] == 4e6 and rec["dram__bytes_write.sum"] == 4e7
    assert rec["sources"] == bench.sources_digest("ospr_col_ifft")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(out))
    traffic, why = bench.measured_traffic("ospr_col_ifft", "k_ospr_col_ifft<1024, 0>", 12)
    assert traffic == 4.4e7
    assert bench.measured_instructions("ospr_col_ifft", "k_ospr_col_ifft<1024, 0>", 12) == 3.7e7
    assert rec["per_launch"] == 12
    # another tile variant or pairs per launch than the capture's: no traffic
    traffic, why = bench.measured_traffic("ospr_col_ifft", "k_ospr_col_ifft<1024, 1, 0>", 12)
    assert traffic is None and "capture is of" in why
    traffic, why = bench.measured_traffic("ospr_col_ifft", "k_ospr_col_ifft<1024, 0>", 8)
    assert traffic is None
    # a record whose kernel sources changed since the capture no longer applies
    data = json.loads(out.read_text())
    data["ospr_col_ifft"]["sources"] = "0" * 16
    out.write_text(json.dumps(data))
    traffic, why = bench.measured_traffic("ospr_col_ifft", "k_ospr_col_ifft<1024, 0>", 12)
    assert traffic is None and "changed" in why


def test_traffic_record_of_a_one_dimensional_grid(bench, tmp_path, monkeypatch):
    # the column IDFT launched as one CTA per resident slot: its pairs per launch are those
    # of the row pass in the same capture
    csv_path = tmp_path / "t.csv"
    ci = "void holo::k_ospr_col_ifft<1024, 0>(holo::OsprArgs)"
    row = "void holo::k_ospr_row<1024, 0, 1, 0>(holo::OsprArgs)"
    _ncu_csv(csv_path, [(ci, "(152, 1, 1)", "dram__bytes_read.sum", "4,000,000"),
                        (ci, "(152, 1, 1)", "dram__bytes_write.sum", "40,000,000"),
                        (row, "(256, 12, 1)", "dram__bytes_read.sum", "100,000,000"),
                        (row, "(256, 12, 1)", "dram__bytes_write.sum", "40,000,000")])
    out = tmp_path / "traffic.json"
    bench.record_traffic(str(csv_path), "ncu ...", str(out))
    data = json.loads(out.read_text())
    assert data["ospr_col_ifft"]["per_launch"] == 12 and data["ospr_row"]["per_launch"] == 12
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(out))
    traffic, _ = bench.measured_traffic("ospr_col_ifft", "k_ospr_col_ifft<1024, 0>", 12)
    assert traffic == 4.4e7
    assert bench.measured_traffic("ospr_col_ifft", "k_ospr_col_ifft<1024, 0>", 8)[0] is None


def test_launch_signatures(bench):
    t = {"col_ifft_variant": 1, "col_fft_variant": 2, "row_variant": 0}
    assert bench.launch_signature("ospr_col_ifft", t, 12, 2) == ("k_ospr_col_ifft<1024, 1>", 12)
    assert bench.launch_signature("ospr_col_fft", t, 12, 2) == ("k_ospr_col_fft<1024, 2>", 2)
    assert bench.launch_signature("ospr_row", t, 12, 2) == ("k_ospr_row<1024, 0, 1, 0>", 12)
    assert bench.launch_signature("replay_error", t, 12, 2) == (None, None)
