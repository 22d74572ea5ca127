"""Benchmark: OSPR 1024x1024 binary sub-frames/s (and GS iterations/s) on GB300.

Workload (one "step"): the L sweep of the 1024x1024 binary OSPR case, N = 24 sub-frames
per frame, one frame for each table length L in 2^8 .. 2^20 plus the unrepeated
generator (14 frames, 336 sub-frames), alternating seeded blob and band-limited-noise
targets. Each frame runs the whole hot path through the C ABI: lut_build ->
ospr_generate (LUT-apply, back-propagation IDFT, binarise, replay DFT, accumulate) ->
replay_error. The frames are independent, so the step is one ospr_generate_batch call
(the library runs them concurrently on its internal streams); the same step made of
per-frame calls on one stream is timed too ("sequential"). GS (1024x1024, 20
iterations, 256 levels, LUT-random start, L = 10007) is timed in the same run and
reported beside it.

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the launching
stream; L2 is flushed (a 512 MiB write) before every timed step, outside the events.
The dominant kernel's duration comes from the library's own CUDA-event profiling of
every launch in the sequential leg's timed steps, where kernels run one at a time.
`--impl reference` times the float64 CPU oracle on the host cores instead (a bounded
sample of the same workload).
"""

import argparse
import csv
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 1024
N_SF = 24
L_SWEEP = [1 << k for k in range(8, 21)] + [-1]          # 2^8 .. 2^20, unrepeated
LUT_SEED = 7
GS_ITERS = 20
GS_L = 10007
FLUSH_BYTES = 512 << 20


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def _query_once(self):
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                 timeout=10).stdout
            self._parse(out)
        except (OSError, subprocess.SubprocessError):
            pass

    def _parse(self, text):
        for line in text.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def start(self):
        self._query_once()
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.buf = []
            self.th = threading.Thread(target=lambda: self.buf.extend(self.proc.stdout), daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.th.join(timeout=2)
            self._parse("".join(self.buf))
        self._query_once()
        return self.summary()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except ValueError:
                continue
            for n, v in zip(names, r[3:]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ byte models ----
def kernel_bytes(family, P, pairs, groups, N):
    """Algorithmic HBM bytes of one launch (unique bytes the kernel must read and write)."""
    if family == "ospr_row":
        return pairs * (16 * P + 2 * P // 8)
    if family == "ospr_col_ifft":
        return 4 * P + pairs * 8 * P + min(2 * pairs * P, 1 << 20)
    if family == "ospr_col_fft":
        return pairs * 8 * P + groups * 4 * P
    if family == "ospr_finalize":
        return groups * 4 * P + 4 * P
    if family == "replay_error":
        return 8 * P
    if family == "lut_build":
        return 0
    return None


def subframe_bytes(P, N, L):
    """Section 8(d) model of one OSPR sub-frame: 16 B/px of transform round trips, the bits,
    and the per-frame target, accumulator and table bytes shared by the N sub-frames."""
    lut = min(L if L > 0 else 0, N * P)
    return 16 * P + P // 8 + (4 * P + 8 * P + lut) / N


# ------------------------------------------------------------ DRAM traffic ----
# `traffic` in the roofline object is dram__bytes_read.sum + dram__bytes_write.sum of one
# launch of the dominant kernel, from an ncu capture recorded in profiles/dram_traffic.json
# by `bench.py --record-traffic <ncu csv>`. Each record carries a digest of the sources the
# kernel is compiled from; once they change the record no longer applies and traffic is null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")
CSRC = os.path.join(ROOT, "paper_2004_04049_gb300", "csrc")
KERNEL_SOURCES = {
    "ospr_col_ifft": ["ospr_kernels.cuh", "fft_core.cuh", "phase_source.cuh", "ospr_col.cu"],
    "ospr_col_fft": ["ospr_kernels.cuh", "fft_core.cuh", "ospr_col.cu"],
    "ospr_row": ["ospr_kernels.cuh", "fft_core.cuh", "ospr_row.cu"],
    "ospr_finalize": ["ospr.cu"],
}
KERNEL_FAMILY = {"k_ospr_col_ifft": "ospr_col_ifft", "k_ospr_col_fft": "ospr_col_fft", "k_ospr_row": "ospr_row",
                 "k_ospr_finalize": "ospr_finalize"}


def sources_digest(family):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[family]:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def record_traffic(csv_path, command, out_path=TRAFFIC_FILE):
    """Per-launch DRAM bytes of the OSPR kernels from an ncu --csv metrics log."""
    with open(csv_path) as fh:
        rows = [r for r in csv.reader(fh)]
    hdr = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hdr]
    ki, mi, vi, gi = h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value"), h.index("Grid Size")
    out = {}
    for r in rows[hdr + 1:]:
        if len(r) <= vi:
            continue
        # "void holo::k_x<...>(holo::OsprArgs)" or "void k_x<...>(OsprArgs)", by ncu's mode
        name = re.sub(r"^(\w+::)+", "", r[ki].replace("void ", "").split("(")[0])
        fam = KERNEL_FAMILY.get(name.split("<")[0])
        if fam is None:
            continue
        rec = out.setdefault(fam, {"kernel": name, "grid": r[gi], "sources": sources_digest(fam),
                                   "command": command})
        if rec["kernel"] != name or rec["grid"] != r[gi]:
            continue   # first launch of the family only
        rec[r[mi]] = float(r[vi].replace(",", ""))
    # work per launch: the grid's y (pairs, or groups for the column DFT); a one-dimensional
    # grid (the column IDFT's one CTA per resident slot) runs the chunk the row pass of the
    # same capture runs
    for fam, rec in out.items():
        rec["per_launch"] = _grid_y(rec["grid"])
    if "ospr_col_ifft" in out and "ospr_row" in out and _grid_y(out["ospr_col_ifft"]["grid"]) == 1:
        out["ospr_col_ifft"]["per_launch"] = out["ospr_row"]["per_launch"]
    old = {}
    if os.path.exists(out_path):
        with open(out_path) as fh:
            old = json.load(fh)
    old.update(out)
    with open(out_path, "w") as fh:
        json.dump(old, fh, indent=1, sort_keys=True)
        fh.write("\n")
    print(json.dumps(out, indent=1))


def _grid_y(grid):
    gy = grid.strip("()").split(",")
    return int(gy[1]) if len(gy) >= 2 else None


def _record_per_launch(rec):
    return rec.get("per_launch", _grid_y(rec.get("grid", "")))


def measured_traffic(family, kernel, per_launch):
    """DRAM bytes of one launch of `per_launch` pairs (groups for the column DFT), or
    (None, why not)."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)[family]
    except (OSError, ValueError, KeyError):
        return None, "no ncu capture recorded"
    if rec.get("sources") != sources_digest(family):
        return None, "kernel sources changed since the capture"
    if rec.get("kernel") != kernel or _record_per_launch(rec) != per_launch:
        return None, f"capture is of {rec.get('kernel')} grid {rec.get('grid')}"
    return rec["dram__bytes_read.sum"] + rec["dram__bytes_write.sum"], \
        f"ncu capture of {kernel} grid {rec['grid']}: {rec['command']}"


def measured_instructions(family, kernel, per_launch):
    """Warp instructions of one launch from the ncu record (smsp__inst_executed.sum), or None."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)[family]
    except (OSError, ValueError, KeyError):
        return None
    if rec.get("sources") != sources_digest(family) or rec.get("kernel") != kernel \
            or _record_per_launch(rec) != per_launch:
        return None
    return rec.get("smsp__inst_executed.sum")


def launch_signature(family, tuning, chunk, groups):
    """Template instance and work per launch (pairs; groups for the column DFT) of one
    float32 launch of an OSPR pass at H x W."""
    ci, cf, rv = tuning["col_ifft_variant"], tuning["col_fft_variant"], tuning["row_variant"]
    return {"ospr_col_ifft": (f"k_ospr_col_ifft<{H}, {ci}>", chunk),
            "ospr_col_fft": (f"k_ospr_col_fft<{H}, {cf}>", groups),
            "ospr_row": (f"k_ospr_row<{W}, {rv}, 1, 0>", chunk)}.get(family, (None, None))


# ------------------------------------------------------------------ our arm ----
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2004_04049_gb300 import holo, pipeline
    from synthetic import blob_target, noise_target

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    holo.load()
    P = H * W
    stream = torch.cuda.current_stream(dev)

    targets = [torch.from_numpy(blob_target(H, W, 1000 + rank)).to(dev),
               torch.from_numpy(noise_target(H, W, 2000 + rank)).to(dev)]
    nfr = len(L_SWEEP)
    # every frame of the step has its own table, target copy and outputs, so the frames
    # are independent and one ospr_generate_batch call runs them all
    fr = []
    for i, L in enumerate(L_SWEEP):
        fr.append({"L": L, "T": targets[i % 2].clone(),
                   "codes": torch.empty(max(L, 1), dtype=torch.uint8, device=dev),
                   "bits": torch.empty((N_SF, P // 32), dtype=torch.int32, device=dev),
                   "I": torch.empty((H, W), dtype=torch.float32, device=dev),
                   "err": torch.empty(3, dtype=torch.float64, device=dev)})
    descs = [holo.frame_desc(f["T"], H, W, N_SF, f["codes"] if f["L"] > 0 else None, f["L"], 256, LUT_SEED,
                             f["L"] > 0, 0, 0, f["bits"], f["I"], f["err"]) for f in fr]
    arr = holo.frame_array(descs)
    ews = torch.empty(holo.replay_error_workspace_size(H, W), dtype=torch.uint8, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s = stream.cuda_stream

    def step_batch():
        holo.ospr_generate_batch(arr, holo.HOLO_FP32, bws, stream=s)

    def frame(f):
        if f["L"] > 0:
            holo.lut_build(LUT_SEED, f["L"], 256, f["codes"], None, stream=s)
        pipeline.ospr(f["T"], N_SF, f["codes"] if f["L"] > 0 else None, f["L"], 256, LUT_SEED, 0, 0,
                      ws=ws, out_bits=f["bits"], out_replay=f["I"], stream=s)
        pipeline.error(f["I"], f["T"], ws=ews, out=f["err"], stream=s)

    def step_sequential():
        for f in fr:
            frame(f)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    def timed_steps(fn, k, profile=False):
        """k steps, L2 flushed before each (outside the events); per-step ms."""
        if profile:
            holo.holo_profile_reset()
            holo.holo_profile_enable(True)
        times = []
        for _ in range(k):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            times.append((e0, e1))
        barrier()
        if profile:
            holo.holo_profile_enable(False)
        return [a.elapsed_time(b) for a, b in times]

    # FFT tile variants and chunking for this shape, picked by the library's autotuner
    tune_ms = holo.ospr_autotune(H, W, N_SF, reps=5, stream=s) if not args.no_tune else None
    tuning = holo.ospr_tuning_get(H, W)
    ws = torch.empty(holo.ospr_workspace_size(H, W, N_SF), dtype=torch.uint8, device=dev)
    bws = torch.empty(holo.ospr_batch_workspace_size(arr), dtype=torch.uint8, device=dev)

    # headline: the 14-frame step as one batch call (frames concurrent on internal streams)
    for _ in range(args.warmup):
        step_batch()
    barrier()
    launches0 = holo.holo_launch_count()
    sampler = ClockSampler(local)
    sampler.start()
    step_ms = timed_steps(step_batch, args.steps)
    clocks = sampler.stop()
    launches = holo.holo_launch_count() - launches0
    def max_over_ranks(ms):
        """The slowest rank's time (every rank runs the same work)."""
        if world == 1:
            return ms
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    total_ms = max_over_ranks(float(sum(step_ms)))
    subframes_per_step = nfr * N_SF
    value = world * subframes_per_step * args.steps / (total_ms / 1e3)
    nmse = np.array([float(f["err"][2].item()) for f in fr])

    # the same step one frame at a time on one stream: the kernels run alone, so their
    # per-launch CUDA-event durations are the kernels' own (roofline of the dominant one)
    for _ in range(args.warmup):
        step_sequential()
    barrier()
    seq_ms = timed_steps(step_sequential, args.steps, profile=True)
    seq_total = max_over_ranks(float(sum(seq_ms)))
    seq_value = world * subframes_per_step * args.steps / (seq_total / 1e3)
    fams = ["lut_build", "ospr_col_ifft", "ospr_row", "ospr_col_fft", "ospr_finalize", "replay_error"]
    prof = {f: holo.holo_profile_read(f) for f in fams}
    npairs = (N_SF + 1) // 2
    chunk = min(npairs, tuning["chunk"])
    groups = min(chunk, tuning["groups"])
    dom = max(fams, key=lambda f: prof[f][1])
    n_dom, ms_dom = prof[dom]
    peaks = _peaks()
    peak_bw = peaks["hbm_gbs"] if peaks else 6800.0
    bytes_dom = kernel_bytes(dom, P, chunk, groups, N_SF)
    achieved = bytes_dom / (ms_dom / n_dom / 1e3) / 1e9 if n_dom and bytes_dom else None
    kname, grid_y = launch_signature(dom, tuning, chunk, groups)
    traffic, traffic_src = measured_traffic(dom, kname, grid_y) if kname else (None, "no capture")
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak_bw, "unit": "GB/s",
                "frac": achieved / peak_bw if achieved else None, "traffic": traffic,
                "traffic_source": traffic_src,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                "timed_in": "sequential leg (one frame at a time, CUDA events around every launch)",
                "algorithmic_bytes_per_launch": bytes_dom,
                "avg_launch_us": ms_dom / n_dom * 1e3 if n_dom else None,
                "kernel_share": {f: round(prof[f][1] / max(1e-12, sum(v[1] for v in prof.values())), 4)
                                 for f in fams}}
    sf_bytes = np.mean([subframe_bytes(P, N_SF, L if L > 0 else N_SF * P) for L in L_SWEEP])
    path_gbs = value / world * sf_bytes / 1e9
    # the same kernel against instruction issue: 4 warp instructions per SM per clock
    insts = measured_instructions(dom, kname, grid_y) if kname else None
    issue = None
    if insts and n_dom:
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = 2070.0
        peak_issue = sm_count * 4 * mhz * 1e6
        got = insts / (ms_dom / n_dom / 1e3)
        issue = {"bound": "issue", "achieved": got / 1e12, "peak": peak_issue / 1e12, "unit": "T warp-inst/s",
                 "frac": got / peak_issue, "instructions_per_launch": insts,
                 "peak_source": f"{sm_count} SMs x 4 schedulers x {mhz:.0f} MHz (maximum SM clock)"}

    # GS leg: 1024^2, 20 iterations, LUT-random start
    gcodes = torch.empty(GS_L, dtype=torch.uint8, device=dev)
    holo.lut_build(LUT_SEED, GS_L, 256, gcodes, None, stream=s)
    gws = torch.empty(holo.gs_workspace_size(H, W, GS_ITERS), dtype=torch.uint8, device=dev)
    gq = torch.empty((H, W), dtype=torch.uint8, device=dev)
    gI = torch.empty((H, W), dtype=torch.float32, device=dev)
    gerr = torch.empty(GS_ITERS, dtype=torch.float64, device=dev)
    gout = torch.empty(3, dtype=torch.float64, device=dev)

    def gs_run():
        holo.gs_iterate(targets[0], H, W, GS_ITERS, 256, None, gcodes, GS_L, 256, LUT_SEED, 0, 0,
                        gq, gI, gerr, None, None, gws, gws.numel(), stream=stream.cuda_stream)

    for _ in range(3):
        gs_run()
    barrier()
    gs_runs = max(3, args.steps)
    gs_ms = 0.0
    for _ in range(gs_runs):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gs_run()
        e1.record(stream)
        e1.synchronize()
        gs_ms += e0.elapsed_time(e1)
    pipeline.error(gI, targets[0], out=gout, stream=stream.cuda_stream)
    gs_nmse = float(gout[2].item())
    gs_ips = GS_ITERS * gs_runs / (gs_ms / 1e3)

    # GS over a batch of targets in the same launches (gs_iterate_batch): 8 targets of
    # 1024^2 (the two seeded targets alternating), 20 iterations each
    GB = 8
    btargets = torch.stack([targets[b % 2] for b in range(GB)]).contiguous()
    gbws = torch.empty(holo.gs_batch_workspace_size(GB, H, W, GS_ITERS), dtype=torch.uint8, device=dev)
    bq = torch.empty((GB, H, W), dtype=torch.uint8, device=dev)
    bI = torch.empty((GB, H, W), dtype=torch.float32, device=dev)
    berr = torch.empty((GB, GS_ITERS), dtype=torch.float64, device=dev)

    def gs_batch_run():
        holo.gs_iterate_batch(btargets, GB, H, W, GS_ITERS, 256, None, gcodes, GS_L, 256, LUT_SEED, 0, 0,
                              bq, bI, berr, None, None, gbws, stream=stream.cuda_stream)

    for _ in range(3):
        gs_batch_run()
    barrier()
    gsb_ms = 0.0
    for _ in range(gs_runs):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gs_batch_run()
        e1.record(stream)
        e1.synchronize()
        gsb_ms += e0.elapsed_time(e1)
    gsb_ips = GB * GS_ITERS * gs_runs / (gsb_ms / 1e3)
    assert torch.equal(berr[0], gerr), "batch target 0 differs from the single-target run"

    # GS with the DFT-32 stages on the tensor cores (split hi/lo operands), same workload
    gs_prec = {}
    for pname, prec in (("fp16x2", holo.HOLO_FP16X2), ("bf16x2", holo.HOLO_BF16X2)):
        pws = torch.empty(holo.gs_workspace_size(H, W, GS_ITERS, prec), dtype=torch.uint8, device=dev)
        perr = torch.empty(GS_ITERS, dtype=torch.float64, device=dev)

        def gs_prec_run():
            holo.gs_iterate(targets[0], H, W, GS_ITERS, 256, None, gcodes, GS_L, 256, LUT_SEED, 0, prec,
                            gq, gI, perr, None, None, pws, pws.numel(), stream=stream.cuda_stream)

        gs_prec_run()
        barrier()
        pms = 0.0
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gs_prec_run()
            e1.record(stream)
            e1.synchronize()
            pms += e0.elapsed_time(e1)
        pe = perr.cpu().numpy()
        ge = gerr.cpu().numpy()
        gs_prec[pname] = {"value": GS_ITERS * 3 / (pms / 1e3), "unit": "iter/s",
                          "eps20_rel_to_fp32": float(abs(pe[-1] - ge[-1]) / ge[-1])}

    # end to end through the public API: every frame's target copied in from page-locked
    # host memory and every frame's result copied back (the hologram bits and the error;
    # in a second measurement the replay image too), all inside one
    # ospr_generate_batch_host call, which copies the targets in on a copy-in stream in
    # launch order and the results out on copy-out streams (the bits as soon as the last
    # row pass has written them), overlapping the kernels.
    h_targets = [t.cpu().pin_memory() for t in targets]
    h_out = [{"bits": torch.empty((N_SF, P // 32), dtype=torch.int32).pin_memory(),
              "I": torch.empty((H, W), dtype=torch.float32).pin_memory(),
              "err": torch.empty(3, dtype=torch.float64).pin_memory()} for _ in fr]
    e2e_steps = max(1, min(args.steps, 10))

    def host_table(replay):
        return holo.frame_host_array([holo.frame_host(h_targets[i % 2], h_out[i]["bits"],
                                                      h_out[i]["I"] if replay else None, h_out[i]["err"])
                                      for i in range(nfr)])

    hosts = {False: host_table(False), True: host_table(True)}
    with_replay = [False]

    def e2e_step():
        holo.ospr_generate_batch_host(arr, hosts[with_replay[0]], holo.HOLO_FP32, bws, stream=s)

    e2e_step()
    barrier()
    e2e_ms = max_over_ranks(float(sum(timed_steps(e2e_step, e2e_steps))))
    e2e_value = world * subframes_per_step * e2e_steps / (e2e_ms / 1e3)
    e2e_nmse = np.array([float(h["err"][2]) for h in h_out])
    assert np.allclose(e2e_nmse, nmse, rtol=0, atol=0), "end-to-end outputs differ from the device-resident run"
    with_replay[0] = True
    e2e_step()
    barrier()
    e2e_r_ms = max_over_ranks(float(sum(timed_steps(e2e_step, e2e_steps))))
    e2e_r_value = world * subframes_per_step * e2e_steps / (e2e_r_ms / 1e3)
    assert torch.equal(h_out[-1]["I"], fr[-1]["I"].cpu()), "replay copied back differs"

    batch = run_batch_leg(dev, stream) if not args.no_batch else None
    precision_leg = run_precision_leg(dev, stream) if not args.no_batch else None
    sources_leg = run_phase_source_leg(dev, stream) if not args.no_batch else None
    fresnel_leg = run_fresnel_leg(dev, stream) if not args.no_batch else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(seconds=args.cpu_seconds)

    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {
            "metric": "OSPR 1024x1024 binary sub-frames/s (L sweep 2^8..2^20 + unrepeated, N=24)",
            "value": value, "unit": "sub-frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "step_ms_p10_p50_p90": [float(np.percentile(step_ms, q)) for q in (10, 50, 90)],
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "tuning": dict(tuning, autotune_ms_per_frame=tune_ms),
            "config": {"workload": "ospr_1024x1024_N24_Lsweep", "H": H, "W": W, "N": N_SF,
                       "L": "2^8..2^20 + unrepeated", "frames_per_step": nfr,
                       "step": "one ospr_generate_batch call: per frame lut_build + ospr_generate + replay_error",
                       "targets": "seeded blob / band-limited noise", "l2": "flushed before each step",
                       "parallelism": f"replicas x{world}"},
            "sequential": {"value": seq_value, "unit": "sub-frames/s", "ms_per_step": seq_total / args.steps,
                           "how": "the same step one frame at a time on one stream (per-frame API calls)"},
            "roofline": roofline,
            "roofline_issue": issue,
            "path_bytes_model": {"bytes_per_subframe": sf_bytes, "achieved_GBps": path_gbs,
                                 "frac_of_hbm": path_gbs / peak_bw},
            "gs": {"metric": "GS 1024x1024 iterations/s (20 iterations, 256 levels, L=10007)",
                   "value": gs_ips, "unit": "iter/s", "nmse_after_20": gs_nmse,
                   "bytes_per_iter_model": 36 * P,
                   "achieved_GBps": gs_ips * 36 * P / 1e9,
                   "precision": gs_prec,
                   "batch": {"targets": GB, "value": gsb_ips, "unit": "iter/s",
                             "how": "gs_iterate_batch: every pass one launch for all targets",
                             "achieved_GBps": gsb_ips * 36 * P / 1e9,
                             "frac_of_hbm": gsb_ips * 36 * P / 1e9 / peak_bw}},
            "nmse_per_L": {str(L): float(v) for L, v in zip(L_SWEEP, nmse)},
            "e2e": {"value": e2e_value, "unit": "sub-frames/s",
                    "how": "one ospr_generate_batch_host call a step: host targets in, results out",
                    "h2d_bytes_per_step": len(L_SWEEP) * 4 * P,
                    "d2h_bytes_per_step": len(L_SWEEP) * (N_SF * P // 8 + 24),
                    "copied_back": "hologram bits and error of every frame",
                    "with_replay": {"value": e2e_r_value, "unit": "sub-frames/s",
                                    "d2h_bytes_per_step": len(L_SWEEP) * (N_SF * P // 8 + 4 * P + 24)}},
            "batch": batch,
            "precision": precision_leg,
            "phase_sources": sources_leg,
            "fresnel": fresnel_leg,
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------ mixed-shape batch leg ----
BATCH_SHAPES = [(512, 512), (1024, 1024), (2048, 2048), (1024, 2048)]


def batch_frames(n_frames=64, seed=42):
    """The mixed-shape batch: shape uniform over BATCH_SHAPES, N uniform in 8..32,
    L = 2^k with k uniform in 10..18, blob targets; table seed = base seed + frame."""
    rng = np.random.default_rng(seed)
    out = []
    for f in range(n_frames):
        H, W = BATCH_SHAPES[int(rng.integers(0, len(BATCH_SHAPES)))]
        N = int(rng.integers(8, 33))
        L = 1 << int(rng.integers(10, 19))
        out.append((H, W, N, L, seed + f))
    return out


def run_batch_leg(dev, stream, reps=3):
    import torch

    from paper_2004_04049_gb300 import holo, pipeline
    from synthetic import blob_target

    frames = batch_frames()
    tunings = {}
    for (H_, W_) in BATCH_SHAPES:
        holo.ospr_autotune(H_, W_, 24, reps=5, stream=stream.cuda_stream)
        tunings[f"{H_}x{W_}"] = holo.ospr_tuning_get(H_, W_)
    bufs = []
    descs = []
    for k, (H, W, N, L, seed) in enumerate(frames):
        b = {"T": torch.from_numpy(blob_target(H, W, 3000 + k)).to(dev),
             "codes": torch.empty(L, dtype=torch.uint8, device=dev),
             "bits": torch.empty((N, H * W // 32), dtype=torch.int32, device=dev),
             "I": torch.empty((H, W), dtype=torch.float32, device=dev),
             "err": torch.empty(3, dtype=torch.float64, device=dev)}
        bufs.append(b)
        descs.append(holo.frame_desc(b["T"], H, W, N, b["codes"], L, 256, seed, True, 0, 0,
                                     b["bits"], b["I"], b["err"]))
    arr = holo.frame_array(descs)
    ws = torch.empty(holo.ospr_batch_workspace_size(arr), dtype=torch.uint8, device=dev)
    sub = sum(f[2] for f in frames)
    s = stream.cuda_stream

    def per_frame():
        for (H, W, N, L, seed), b in zip(frames, bufs):
            holo.lut_build(seed, L, 256, b["codes"], None, stream=s)
            pipeline.ospr(b["T"], N, b["codes"], L, 256, seed, ws=ws, out_bits=b["bits"], out_replay=b["I"],
                          stream=s)
            pipeline.error(b["I"], b["T"], out=b["err"], stream=s)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        ms = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.median(ms))

    t_pf = timed(per_frame)
    t_batch = timed(lambda: holo.ospr_generate_batch(arr, holo.HOLO_FP32, ws, stream=s))
    g = holo.ospr_batch_graph_create(arr, holo.HOLO_FP32, ws)
    try:
        t_graph = timed(lambda: holo.holo_graph_launch(g, s))
    finally:
        holo.holo_graph_destroy(g)
    # the same batch as one persistent launch with its device work queue, eagerly and as a
    # graph (counter clear + launch)
    pws = torch.empty(holo.ospr_batch_persistent_workspace_size(arr), dtype=torch.uint8, device=dev)
    holo.holo_tc_status(clear=True)
    t_pers = timed(lambda: holo.ospr_generate_batch_persistent(arr, pws, stream=s))
    pg = holo.ospr_batch_persistent_graph_create(arr, pws)
    try:
        t_pgraph = timed(lambda: holo.holo_graph_launch(pg, s))
    finally:
        holo.holo_graph_destroy(pg)
    pers_fault = holo.holo_tc_status(clear=True)
    return {"workload": "64 frames, shapes {512^2, 1024^2, 2048^2, 1024x2048}, N in 8..32, L = 2^(10..18), "
                        "seed 42, blob targets; per frame lut_build + ospr_generate + replay_error",
            "subframes": sub, "unit": "sub-frames/s",
            "per_frame_launches": sub / (t_pf / 1e3), "batch_call": sub / (t_batch / 1e3),
            "graph_launch": sub / (t_graph / 1e3),
            "persistent": sub / (t_pers / 1e3), "persistent_graph": sub / (t_pgraph / 1e3),
            "persistent_wait_expired": bool(pers_fault),
            "ms": {"per_frame": t_pf, "batch": t_batch, "graph": t_graph, "persistent": t_pers,
                   "persistent_graph": t_pgraph},
            "tuning": tunings}


# ----------------------------------------------------------- phase sources leg ----
def run_phase_source_leg(dev, stream, reps=10):
    """One 1024x1024 N=24 frame (lut/lfsr build + ospr_generate + replay_error) with the
    phases from the paper's LUT (L = 10007), from an m-sequence (Section 7's alternative:
    a fresh code for every pixel of every sub-frame, built per frame) and from the
    counter-based SplitMix64 generator (no table)."""
    import torch

    from paper_2004_04049_gb300 import holo, pipeline
    from synthetic import blob_target

    s = stream.cuda_stream
    P = H * W
    T = torch.from_numpy(blob_target(H, W, 1000)).to(dev)
    ws = torch.empty(holo.ospr_workspace_size(H, W, N_SF), dtype=torch.uint8, device=dev)
    ews = torch.empty(holo.replay_error_workspace_size(H, W), dtype=torch.uint8, device=dev)
    bits = torch.empty((N_SF, P // 32), dtype=torch.int32, device=dev)
    I = torch.empty((H, W), dtype=torch.float32, device=dev)
    err = torch.empty(3, dtype=torch.float64, device=dev)
    lut = torch.empty(GS_L, dtype=torch.uint8, device=dev)
    mseq = torch.empty(N_SF * P, dtype=torch.uint8, device=dev)
    frame_no = [0]

    def run(kind):
        f = frame_no[0]
        frame_no[0] += 1
        if kind == "lut":
            holo.lut_build(LUT_SEED, GS_L, 256, lut, None, stream=s)
            pipeline.ospr(T, N_SF, lut, GS_L, 256, LUT_SEED, 0, 0, ws=ws, out_bits=bits, out_replay=I, stream=s)
        elif kind == "m_sequence":
            holo.lfsr_build(0x1D872B41, f * N_SF * P, N_SF * P, 256, mseq, stream=s)
            pipeline.ospr(T, N_SF, mseq, N_SF * P, 256, 0, 0, 0, ws=ws, out_bits=bits, out_replay=I, stream=s)
        else:
            pipeline.ospr(T, N_SF, None, holo.L_UNREPEATED, 256, LUT_SEED + f, 0, 0, ws=ws, out_bits=bits,
                          out_replay=I, stream=s)
        pipeline.error(I, T, ws=ews, out=err, stream=s)

    out = {}
    for kind in ("lut", "m_sequence", "splitmix64"):
        for _ in range(3):
            run(kind)
        torch.cuda.synchronize(dev)
        holo.holo_profile_reset()
        holo.holo_profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run(kind)
        e1.record(stream)
        e1.synchronize()
        holo.holo_profile_enable(False)
        ms = e0.elapsed_time(e1) / reps
        build = holo.holo_profile_read("lut_build" if kind == "lut" else "lfsr_build")
        gen = holo.holo_profile_read("ospr_col_ifft")
        out[kind] = {"ms_per_frame": ms, "subframes_per_s": N_SF / (ms / 1e3), "nmse": float(err[2].item()),
                     "table_build_us": build[1] / max(build[0], 1) * 1e3 if kind != "splitmix64" else 0.0,
                     "generation_pass_us": gen[1] / max(gen[0], 1) * 1e3}
    return out


# ------------------------------------------------------------------ Fresnel leg ----
def run_fresnel_leg(dev, stream, reps=10, kappa=2.4e-4):
    """One 1024x1024 N=24 frame (L = 10007) with Fresnel propagation (kappa = pitch^2 /
    (wavelength * z); 2.4e-4 is 8 um pixels, 532 nm light, z = 0.5 m) against the same frame
    in the far field: the Fresnel field is not Hermitian, so every sub-frame takes its own
    transforms."""
    import torch

    from paper_2004_04049_gb300 import holo, pipeline
    from synthetic import blob_target

    s = stream.cuda_stream
    P = H * W
    T = torch.from_numpy(blob_target(H, W, 1000)).to(dev)
    lut = torch.empty(GS_L, dtype=torch.uint8, device=dev)
    holo.lut_build(LUT_SEED, GS_L, 256, lut, None, stream=s)
    ws = torch.empty(holo.ospr_fresnel_workspace_size(H, W, N_SF), dtype=torch.uint8, device=dev)
    bits = torch.empty((N_SF, P // 32), dtype=torch.int32, device=dev)
    I = torch.empty((H, W), dtype=torch.float32, device=dev)

    def run():
        holo.ospr_generate_fresnel(T, H, W, N_SF, lut, GS_L, 256, LUT_SEED, 0, 0, kappa, bits, I, ws,
                                   stream=s)

    for _ in range(3):
        run()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # per-pass launch times (CUDA events around every launch, outside the timed loop)
    fams = ["fresnel_chirp", "ospr_col_ifft", "ospr_row", "ospr_col_fft", "ospr_finalize"]
    holo.holo_profile_reset()
    holo.holo_profile_enable(True)
    for _ in range(3):
        run()
    torch.cuda.synchronize(dev)
    holo.holo_profile_enable(False)
    passes = {}
    for f in fams:
        n, t = holo.holo_profile_read(f)
        passes[f] = {"launches_per_frame": n / 3, "us_per_launch": 1e3 * t / max(n, 1)}
    out = {"workload": f"1024x1024, N={N_SF}, L={GS_L}, kappa={kappa}", "ms_per_frame": ms,
           "subframes_per_s": N_SF / (ms / 1e3), "energy_per_pixel": float(I.sum().item()) / P,
           "passes": passes}
    # GS under Fresnel propagation: 20 iterations from the LUT start, as the far-field GS leg
    gws = torch.empty(holo.gs_workspace_size(H, W, GS_ITERS), dtype=torch.uint8, device=dev)
    q = torch.empty((H, W), dtype=torch.uint8, device=dev)
    err = torch.empty(GS_ITERS, dtype=torch.float64, device=dev)

    def run_gs():
        holo.gs_iterate_fresnel(T, H, W, GS_ITERS, 256, None, lut, GS_L, 256, LUT_SEED, 0, kappa, q, I, err, None,
                                None, gws, stream=s)

    for _ in range(3):
        run_gs()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        run_gs()
    e1.record(stream)
    e1.synchronize()
    gms = e0.elapsed_time(e1) / reps
    out["gs"] = {"iters": GS_ITERS, "ms_per_run": gms, "iter_per_s": GS_ITERS / (gms / 1e3),
                 "eps_per_pixel_after_iters": float(err[-1].item()) / P}
    return out


# --------------------------------------------------------- mixed precision leg ----
def run_precision_leg(dev, stream, reps=5):
    """OSPR at 1024^2 and 2048^2, N = 24, L = 10007, in float32 and with the DFT-32 stages
    on the tensor cores (fp16 / bf16 hi+lo operands, float32 accumulation). Errors are
    against the float32 path of the same run (the tests bound them against the oracle)."""
    import torch

    from paper_2004_04049_gb300 import holo, pipeline
    from synthetic import blob_target

    out = {}
    s = stream.cuda_stream
    for n in (1024, 2048):
        T = torch.from_numpy(blob_target(n, n, 1000)).to(dev)
        codes = pipeline.lut(LUT_SEED, GS_L, device=dev)
        res = {}
        ref = None
        for name, prec in (("fp32", holo.HOLO_FP32), ("fp16x2", holo.HOLO_FP16X2), ("bf16x2", holo.HOLO_BF16X2)):
            ws = torch.empty(holo.ospr_workspace_size(n, n, N_SF, prec), dtype=torch.uint8, device=dev)
            bits = torch.empty((N_SF, n * n // 32), dtype=torch.int32, device=dev)
            I = torch.empty((n, n), dtype=torch.float32, device=dev)

            def call():
                pipeline.ospr(T, N_SF, codes, GS_L, 256, LUT_SEED, ws=ws, out_bits=bits, out_replay=I,
                              precision=prec, stream=s)

            call()
            torch.cuda.synchronize(dev)
            ms = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            err = pipeline.error(I, T, stream=s).cpu().numpy()
            r = {"subframes_per_s": N_SF / (float(np.median(ms)) / 1e3), "nmse": float(err[2])}
            if ref is None:
                ref = (bits.clone(), I.clone(), float(err[2]))
            else:
                b0 = np.unpackbits(ref[0].cpu().numpy().view(np.uint8))
                b1 = np.unpackbits(bits.cpu().numpy().view(np.uint8))
                r["bits_agree_vs_fp32"] = float(np.mean(b0 == b1))
                r["replay_rel_vs_fp32"] = float((I - ref[1]).abs().max().item() / ref[1].abs().max().item())
                r["nmse_rel_vs_fp32"] = abs(float(err[2]) - ref[2]) / ref[2]
            res[name] = r
        out[f"{n}x{n}"] = res
    return out


# ------------------------------------------------------------- CPU oracle arm ----
def _oracle_partial(s0, n_sub, L=1 << 16):
    """Sub-frames s0 .. s0+n_sub-1 of the workload's 1024x1024 frame through the oracle:
    their bits and summed replay intensity."""
    from oracle import lut as olut
    from oracle import ospr as oospr
    from synthetic import blob_target

    T = blob_target(H, W, 1000)
    table = olut.lut_codes(LUT_SEED, L)
    P = H * W
    I = np.zeros((H, W))
    for s in range(s0, s0 + n_sub):
        c = olut.subframe_codes(table, L, LUT_SEED, 0, s, P, P)
        Hs = oospr.back_propagate(oospr.subframe_field(T, c))
        h = oospr.binarise(Hs.real)
        oospr.pack_bits(h)
        I += oospr.replay_intensity(h)
    return I


def _oracle_subframes(n_sub, L=1 << 16):
    """Runs n_sub sub-frames of the workload's 1024x1024 frame through the oracle."""
    from oracle import error as oerr
    from synthetic import blob_target

    I = _oracle_partial(0, n_sub, L)
    oerr.replay_error(I / n_sub, blob_target(H, W, 1000))


def _oracle_worker(job):
    return _oracle_partial(*job)


def cpu_baseline_sample(seconds=15.0):
    """The oracle as it stands on the host cores: sub-frames of the 1024x1024 workload, on
    one core and then on every core (one process per core, spawned)."""
    import multiprocessing as mp

    t0 = time.perf_counter()
    _oracle_subframes(1)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-3)))
    t0 = time.perf_counter()
    _oracle_subframes(n)
    dt = time.perf_counter() - t0
    single = {"value": n / dt, "cores": 1,
              "sample": f"{n} sub-frames of the 1024x1024 L=65536 frame (float64 numpy oracle, one process), "
                        f"{dt:.1f} s"}
    cores = os.cpu_count() or 1
    per = max(1, int(seconds / max(one, 1e-3)))
    jobs = [(k * per, per) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_worker, [(0, 1)] * cores)      # imports and table set-up in every worker
        t0 = time.perf_counter()
        parts = pool.map(_oracle_worker, jobs)
        dtp = time.perf_counter() - t0
    del parts
    nall = per * cores
    return {"value": nall / dtp, "unit": "sub-frames/s", "cores": cores, "kind": "oracle",
            "sample": f"{nall} sub-frames of the 1024x1024 L=65536 frame, {per} per process on {cores} spawned "
                      f"processes (float64 numpy oracle), {dtp:.1f} s",
            "single_core": single, "gs": _oracle_gs_rate()}


def _oracle_gs_rate(iters=3):
    """The oracle's GS at 1024x1024 (256 levels, LUT start L = 10007) on one core."""
    from oracle import gs as ogs
    from oracle import lut as olut
    from synthetic import blob_target

    T = blob_target(H, W, 1000)
    table = olut.lut_codes(LUT_SEED, GS_L)
    t0 = time.perf_counter()
    ogs.gs(T, iters, table, GS_L, LUT_SEED)
    dt = time.perf_counter() - t0
    return {"value": iters / dt, "unit": "iter/s", "cores": 1,
            "sample": f"{iters} GS iterations at 1024x1024 (float64 numpy oracle, one process), {dt:.1f} s"}


def run_reference(args):
    """The reference arm: the float64 oracle as it stands on every host core (one spawned
    process per core), each step a bounded sample of the workload: two sub-frames of the
    1024x1024 frame per process."""
    import multiprocessing as mp

    rank, world, _ = _env_rank()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    per = 2
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_worker, [(0, 1)] * cores)      # imports and table set-up in every worker
        for _ in range(args.warmup):
            pool.map(_oracle_worker, [(k, 1) for k in range(cores)])
        step_s = []
        for i in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_worker, [((i * cores + k) * per, per) for k in range(cores)])
            step_s.append(time.perf_counter() - t0)
    dt = float(sum(step_s))
    n = per * cores * args.steps
    value = n / dt
    sample = f"{per} sub-frames of the 1024x1024 L=65536 frame per process and step, {cores} spawned processes"
    line = {
        "impl": "reference",
        "metric": "OSPR 1024x1024 binary sub-frames/s (L sweep 2^8..2^20 + unrepeated, N=24)",
        "value": value, "unit": "sub-frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ospr_1024x1024_N24_Lsweep", "H": H, "W": W, "N": N_SF,
                   "sample_per_step": f"{per * cores} sub-frames"},
        "cpu_baseline": {"value": value, "unit": "sub-frames/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "sub-frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# (name, B, R, Cin, Cout): the warm-start network's layer shapes at the training batch
CONV_SHAPES = [("enc0_8to32_256sq", 16, 256, 8, 32), ("enc1_32to32_256sq", 16, 256, 32, 32),
               ("enc3_64to64_128sq", 16, 128, 64, 64), ("enc5_128to128_64sq", 16, 64, 128, 128),
               ("mid_128to128_32sq", 16, 32, 128, 128), ("dec9_128to64_128sq", 16, 128, 128, 64),
               ("dec10_64to32_256sq", 16, 256, 64, 32)]


def conv_throughput(reps=20):
    """Forward 3x3 convolution of every network layer shape: the tcgen05 kernel against the
    mma.sync kernel (TFLOP/s = 2*B*R^2*Cin*Cout*9 per call / CUDA-event time)."""
    import torch

    from paper_2004_04049_gb300 import holo

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, B, R, Ci, Co in CONV_SHAPES:
        x = torch.randn((B, R, R, Ci), device=dev).to(torch.bfloat16)
        w = (0.05 * torch.randn((Co, 9 * Ci), device=dev)).to(torch.bfloat16)
        bias = torch.zeros(Co, dtype=torch.float32, device=dev)
        y = torch.empty((B, R, R, Co), dtype=torch.bfloat16, device=dev)
        flops = 2.0 * B * R * R * Ci * Co * 9
        row = {}
        for kind, mode in (("tcgen05", 0), ("mma_sync", holo.HOLO_CONV_LEGACY)):
            def call():
                holo.nn_conv3x3(mode, B, R, R, Ci, Co, x, w, d_bias=bias, d_out=y, relu=True,
                                stream=stream.cuda_stream)

            for _ in range(3):
                call()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                call()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[kind] = {"us": ms * 1e3, "tflops": flops / (ms / 1e3) / 1e12}
        out[name] = row
    out["tc_fault"] = holo.holo_tc_status()
    return out


def gs_tile_sweep(sizes=(1024, 2048), iters=20, reps=10):
    """GS time per iteration for every (column, row) tile variant pair (gs_tuning_set)."""
    import torch

    from paper_2004_04049_gb300 import holo, pipeline
    from synthetic import blob_target

    dev = torch.device("cuda:0")
    s = torch.cuda.current_stream(dev).cuda_stream
    rows = []
    for n in sizes:
        T = torch.from_numpy(blob_target(n, n, 1000)).to(dev)
        codes = pipeline.lut(LUT_SEED, GS_L, device=dev)
        ws = torch.empty(holo.gs_workspace_size(n, n, iters), dtype=torch.uint8, device=dev)
        q = torch.empty((n, n), dtype=torch.uint8, device=dev)
        I = torch.empty((n, n), dtype=torch.float32, device=dev)
        err = torch.empty(iters, dtype=torch.float64, device=dev)
        for cv in range(3):
            for rv in range(3):
                holo.gs_tuning_set(n, n, cv, rv)

                def f():
                    holo.gs_iterate(T, n, n, iters, 256, None, codes, GS_L, 256, LUT_SEED, 0, 0, q, I, err, None,
                                    None, ws, ws.numel(), stream=s)

                for _ in range(3):
                    f()
                torch.cuda.synchronize(dev)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    f()
                e1.record()
                e1.synchronize()
                us = e0.elapsed_time(e1) / reps / iters * 1e3
                rows.append({"n": n, "col_variant": cv, "row_variant": rv, "us_per_iter": us,
                             "iter_per_s": 1e6 / us, "eps_last": float(err[-1].item()) / (n * n)})
        holo.gs_tuning_set(n, n)
    return rows


def run_learned(args):
    """Learned GS warm start at the configured scale (labels from 100-iteration GS on 20k
    seeded 256^2 targets, training by the library's kernels, evaluation at 1024^2), plus
    the tensor-core throughput of the network's convolution kernel."""
    import torch

    from paper_2004_04049_gb300 import build_lib, holo, warmstart

    build_lib.build()
    holo.load()
    conv = conv_throughput()
    res = warmstart.run(n_train=args.learned_n, gs_iters=100, epochs=args.learned_epochs, batch=16,
                        eval_size=1024, n_eval=8, log=lambda s: print(s, file=sys.stderr),
                        extra_sizes=(2048, 4096))
    peaks = _peaks()
    ev = res["eval"]
    line = {"metric": "learned GS warm start: GS iterations to the 20-iteration LUT-random error at 1024^2",
            "n_train": args.learned_n, "epochs": args.learned_epochs,
            "loss_first": float(np.mean(res["losses"][:20])), "loss_last": float(np.mean(res["losses"][-20:])),
            "iters_lut_mean": float(np.mean([r["iters_lut"] for r in ev])),
            "iters_learned_mean": float(np.mean([r["iters_learned"] or 60 for r in ev])),
            "ms_lut_mean": float(np.mean([r["ms_lut"] for r in ev])),
            "ms_learned_mean": float(np.mean([r["ms_learned"] or np.nan for r in ev])),
            "eval": ev, "seconds": res["seconds"], "conv_kernel": conv,
            "other_sizes": {S: {"iters_lut_mean": float(np.mean([r["iters_lut"] for r in rows])),
                                "iters_learned_mean": float(np.mean([r["iters_learned"] or 60 for r in rows])),
                                "ms_lut_mean": float(np.mean([r["ms_lut"] for r in rows])),
                                "ms_learned_mean": float(np.mean([r["ms_learned"] or np.nan for r in rows])),
                                "eval": rows}
                            for S, rows in res["eval_other_sizes"].items()},
            "bf16_peak_tflops": peaks["bf16_tflops"] if peaks else 1900.0}
    print(json.dumps(line), flush=True)


def run_case(name):
    """Small fixed workloads for profiler captures (no timing, no JSON line)."""
    import torch

    from paper_2004_04049_gb300 import pipeline
    from synthetic import blob_target

    dev = torch.device("cuda:0")
    if name == "frame":
        # one 1024x1024 OSPR frame (N=24, L=10007), its replay error and 2 GS iterations, twice
        T = torch.from_numpy(blob_target(H, W, 1000)).to(dev)
        codes = pipeline.lut(LUT_SEED, GS_L, device=dev)
        for _ in range(2):
            _, I = pipeline.ospr(T, N_SF, codes, GS_L)
            e = pipeline.error(I, T)
            pipeline.gs(T, 2, 256, codes, GS_L, 256, LUT_SEED)
        torch.cuda.synchronize()
        print("case frame ok, nmse", float(e[2]))
    elif name == "gs":
        # GS at 1024x1024: 20 iterations from the LUT-random start, default tiles, twice
        T = torch.from_numpy(blob_target(H, W, 1000)).to(dev)
        codes = pipeline.lut(LUT_SEED, GS_L, device=dev)
        for _ in range(2):
            out = pipeline.gs(T, GS_ITERS, 256, codes, GS_L, 256, LUT_SEED)
        torch.cuda.synchronize()
        print("case gs ok, eps_20 / P", float(out["err"][-1]) / (H * W))
    elif name == "fresnel":
        # one 1024x1024 OSPR frame under Fresnel propagation (N=24, L=10007, kappa=2.4e-4), twice
        T = torch.from_numpy(blob_target(H, W, 1000)).to(dev)
        codes = pipeline.lut(LUT_SEED, GS_L, device=dev)
        for _ in range(2):
            _, I = pipeline.ospr_fresnel(T, N_SF, 2.4e-4, codes, GS_L, 256, LUT_SEED)
        torch.cuda.synchronize()
        print("case fresnel ok, energy per pixel", float(I.sum()) / (H * W))
    elif name == "tc":
        # one 1024x1024 frame (N=24, L=10007) twice in float32, then twice in bf16x2
        from paper_2004_04049_gb300 import holo
        T = torch.from_numpy(blob_target(H, W, 1000)).to(dev)
        codes = pipeline.lut(LUT_SEED, GS_L, device=dev)
        for prec in (holo.HOLO_FP32, holo.HOLO_BF16X2):
            for _ in range(2):
                pipeline.ospr(T, N_SF, codes, GS_L, 256, LUT_SEED, precision=prec)
        torch.cuda.synchronize()
        print("case tc ok, tcgen05 fault flag", holo.holo_tc_status())
    elif name == "infer":
        # the learned warm start's inference at batch 1 on a 1024x1024 target, three times
        from paper_2004_04049_gb300 import holo
        net = holo.ws_net_create(11, 1)
        try:
            big = torch.from_numpy(blob_target(1024, 1024, 5)).to(dev)
            ph = torch.empty((1024, 1024), dtype=torch.float32, device=dev)
            for _ in range(3):
                holo.ws_infer(net, big, 1024, 1024, ph)
            torch.cuda.synchronize()
        finally:
            holo.ws_net_destroy(net)
        print("case infer ok, max |phase|", float(ph.abs().max()))
    elif name == "persistent":
        # four 1024x1024 frames (N=24, L=10007) as one persistent launch, twice
        from paper_2004_04049_gb300 import holo
        codes = pipeline.lut(LUT_SEED, GS_L, device=dev)
        bufs = []
        for k in range(4):
            bufs.append({"T": torch.from_numpy(blob_target(H, W, 1000 + k)).to(dev),
                         "bits": torch.empty((N_SF, H * W // 32), dtype=torch.int32, device=dev),
                         "I": torch.empty((H, W), dtype=torch.float32, device=dev),
                         "err": torch.empty(3, dtype=torch.float64, device=dev)})
        arr = holo.frame_array([holo.frame_desc(b["T"], H, W, N_SF, codes, GS_L, 256, LUT_SEED, False, 0, 0,
                                                b["bits"], b["I"], b["err"]) for b in bufs])
        pws = torch.empty(holo.ospr_batch_persistent_workspace_size(arr), dtype=torch.uint8, device=dev)
        for _ in range(2):
            holo.ospr_generate_batch_persistent(arr, pws)
        torch.cuda.synchronize()
        print("case persistent ok, wait expired", holo.holo_tc_status(clear=True))
    else:
        raise SystemExit(f"unknown case {name!r}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the mixed-shape batch leg")
    ap.add_argument("--no-tune", action="store_true", help="keep the default FFT tiles and chunking")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--case", default=None, help="run a small fixed workload for a profiler capture")
    ap.add_argument("--learned", action="store_true", help="run the learned GS warm-start experiment")
    ap.add_argument("--learned-n", type=int, default=20000)
    ap.add_argument("--learned-epochs", type=int, default=2)
    ap.add_argument("--conv", action="store_true", help="time the network's convolution kernels only")
    ap.add_argument("--study", action="store_true", help="run the LUT-length study of Figs. 5-6")
    ap.add_argument("--gs-tiles", action="store_true", help="time GS for every tile variant pair")
    ap.add_argument("--study-runs", type=int, default=100)
    ap.add_argument("--record-traffic", default=None, metavar="CSV",
                    help="store per-launch DRAM bytes from an ncu --csv log in profiles/dram_traffic.json")
    ap.add_argument("--traffic-command", default="", help="the ncu command that wrote the CSV")
    ap.add_argument("--traffic-out", default=TRAFFIC_FILE, help="where to store the records")
    args = ap.parse_args()
    if args.record_traffic:
        record_traffic(args.record_traffic, args.traffic_command, args.traffic_out)
        return
    if args.learned:
        run_learned(args)
        return
    if args.study:
        from paper_2004_04049_gb300 import build_lib, holo, study
        build_lib.build()
        holo.load()
        t0 = time.perf_counter()
        res = study.lut_length_study(sizes=(256, 128, 64), N=24, runs=args.study_runs, n_targets=6,
                                     log=lambda m: print(m, file=sys.stderr))
        print(json.dumps({"study": "LUT length vs NMSE ratio (Section 5.2, Figs. 5-6), synthetic targets",
                          "seconds": time.perf_counter() - t0, "results": res}), flush=True)
        return
    if args.gs_tiles:
        from paper_2004_04049_gb300 import build_lib, holo
        build_lib.build()
        holo.load()
        print(json.dumps({"gs_tiles": gs_tile_sweep()}), flush=True)
        return
    if args.conv:
        from paper_2004_04049_gb300 import build_lib, holo
        build_lib.build()
        holo.load()
        peaks = _peaks()
        print(json.dumps({"conv_kernel": conv_throughput(),
                          "bf16_peak_tflops": peaks["bf16_tflops"] if peaks else 1900.0}), flush=True)
        return
    if args.case:
        from paper_2004_04049_gb300 import build_lib
        build_lib.build()
        run_case(args.case)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
