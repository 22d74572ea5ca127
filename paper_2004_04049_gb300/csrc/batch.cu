// batch.cu - batched OSPR frames over internal streams, and their CUDA-graph capture.
//
// Frames of a batch are independent (each has its own target, table and outputs), so the
// scheduler spreads them over S internal streams: longest frame first onto the least
// loaded stream (LPT), each stream running its frames in order on its own slice of the
// workspace. The call forks from the caller's stream with an event and joins back with
// one event per internal stream, so it composes with other work on that stream and can
// be captured into a CUDA graph as S parallel branches. There are no device-side waits
// between blocks: every dependency is a stream order or an event.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "runtime.h"

namespace holo {

constexpr int kMaxBatchStreams = 32;

static int batch_stream_count() {
    static const int n = [] {
        const char* v = getenv("HOLO_BATCH_STREAMS");
        int x = v && *v ? atoi(v) : 8;
        return x < 1 ? 1 : (x > kMaxBatchStreams ? kMaxBatchStreams : x);
    }();
    return n;
}

// internal streams and fork/join events, created once per device; `run_mu` serialises
// the enqueue section of batch calls on the device (fork record to join wait), so that
// calls from several host threads, or an eager call during another thread's graph
// capture, never interleave their work on the shared streams and events
// ospr_generate_batch_host also uses one copy-in stream, one copy-out stream per internal
// stream and three events per frame (grown on demand, under run_mu)
struct DeviceStreams {
    cudaStream_t st[kMaxBatchStreams];
    cudaEvent_t fork;
    cudaEvent_t join[kMaxBatchStreams];
    cudaStream_t copy_in;
    cudaEvent_t copy_in_join;
    cudaStream_t copy_out[kMaxBatchStreams];
    cudaEvent_t copy_out_join[kMaxBatchStreams];
    std::vector<cudaEvent_t> frame_ev;
    bool ready = false;
    std::mutex run_mu;
};
static std::mutex g_streams_mu;
static DeviceStreams g_streams[64];

static int device_streams(DeviceStreams** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(HOLO_EUNSUPPORTED, "device index %d too large", dev);
    std::lock_guard<std::mutex> lk(g_streams_mu);
    DeviceStreams& ds = g_streams[dev];
    if (!ds.ready) {
        for (int i = 0; i < kMaxBatchStreams; ++i) {
            if ((e = cudaStreamCreateWithFlags(&ds.st[i], cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaStreamCreateWithFlags(&ds.copy_out[i], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_status(e, "batch: cudaStreamCreate");
            if ((e = cudaEventCreateWithFlags(&ds.join[i], cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&ds.copy_out_join[i], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_status(e, "batch: cudaEventCreate");
        }
        if ((e = cudaStreamCreateWithFlags(&ds.copy_in, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_status(e, "batch: cudaStreamCreate");
        if ((e = cudaEventCreateWithFlags(&ds.fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ds.copy_in_join, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_status(e, "batch: cudaEventCreate");
        ds.ready = true;
    }
    *out = &ds;
    return HOLO_OK;
}

struct BatchPlan {
    int streams;
    std::vector<int> order;          // frames in launch order
    std::vector<int> stream_of;      // per frame
    size_t slot_bytes;               // per-stream workspace slice
    size_t ospr_off, err_off;        // inside a slice
    size_t total;
};

static int plan_batch(const holo_frame_desc* f, int n, int precision, BatchPlan* pl) {
    if (!f || n < 1) return fail(HOLO_EINVAL, "batch: no frames");
    if (fault_injected("plan")) return fail(HOLO_EINVAL, "batch: injected planning failure (HOLO_FAULT_INJECT)");
    size_t max_ospr = 0, max_err = 0;
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        size_t b = 0;
        int rc = ospr_workspace_size(f[i].H, f[i].W, f[i].N, precision, &b);
        if (rc) return fail(rc, "batch frame %d: %s", i, holo_last_error());
        max_ospr = std::max(max_ospr, b);
        if (f[i].d_err) {
            size_t eb = 0;
            if ((rc = replay_error_workspace_size(f[i].H, f[i].W, &eb)))
                return fail(rc, "batch frame %d: %s", i, holo_last_error());
            max_err = std::max(max_err, eb);
            if (!f[i].d_replay) return fail(HOLO_EINVAL, "batch frame %d: d_err needs d_replay", i);
        }
        cost[i] = double(f[i].H) * double(f[i].W) * double((f[i].N + 1) / 2);
    }
    pl->streams = std::min(batch_stream_count(), n);
    pl->ospr_off = 0;
    pl->err_off = align_up(max_ospr, 256);
    pl->slot_bytes = pl->err_off + align_up(std::max<size_t>(max_err, 256), 256);
    pl->total = pl->slot_bytes * size_t(pl->streams);
    // longest processing time first onto the least-loaded stream
    pl->order.resize(n);
    for (int i = 0; i < n; ++i) pl->order[i] = i;
    std::stable_sort(pl->order.begin(), pl->order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(pl->streams, 0.0);
    pl->stream_of.assign(n, 0);
    for (int i : pl->order) {
        const int k = int(std::min_element(load.begin(), load.end()) - load.begin());
        pl->stream_of[i] = k;
        load[k] += cost[i];
    }
    return HOLO_OK;
}

// copies of one frame between host and device on that frame's internal stream
static int frame_copy(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st, int i,
                      const char* what) {
    if (!dst || !src || !bytes) return HOLO_OK;
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, st);
    if (e != cudaSuccess) return fail(cuda_status(e, what), "batch frame %d: %s", i, holo_last_error());
    return HOLO_OK;
}

static int run_batch(const holo_frame_desc* f, int n, int precision, void* d_ws, size_t ws_bytes,
                     cudaStream_t s, const BatchPlan& pl, const holo_frame_host* io = nullptr) {
    if (!d_ws || ws_bytes < pl.total)
        return fail(HOLO_EWORKSPACE, "batch: workspace %zu bytes, need %zu", ws_bytes, pl.total);
    if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0)
        return fail(HOLO_EWORKSPACE, "batch: workspace is not 256-byte aligned");
    DeviceStreams* ds = nullptr;
    int rc = device_streams(&ds);
    if (rc) return rc;
    std::lock_guard<std::mutex> run_lock(ds->run_mu);
    cudaError_t e;
    if (io) {   // three events per frame: its target is in, its bits are written, its work is done
        while (ds->frame_ev.size() < 3 * size_t(n)) {
            cudaEvent_t ev;
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_status(e, "batch: cudaEventCreate");
            ds->frame_ev.push_back(ev);
        }
    }
    if ((e = cudaEventRecord(ds->fork, s)) != cudaSuccess) return cuda_status(e, "batch: fork record");
    for (int k = 0; k < pl.streams; ++k) {
        if ((e = cudaStreamWaitEvent(ds->st[k], ds->fork, 0)) != cudaSuccess) return cuda_status(e, "batch: fork wait");
        if (io && (e = cudaStreamWaitEvent(ds->copy_out[k], ds->fork, 0)) != cudaSuccess)
            return cuda_status(e, "batch: fork wait");
    }
    if (io && (e = cudaStreamWaitEvent(ds->copy_in, ds->fork, 0)) != cudaSuccess)
        return cuda_status(e, "batch: fork wait");
    // With host buffers the targets go in on the copy-in stream in launch order, ahead of
    // the frames' work (each frame waits for its own target; frames own their targets), so
    // the first frames start one target copy apart; each frame's results go out on the
    // copy-out stream of its internal stream: the hologram bits as soon as the last row
    // pass has written them (while the frame's replay passes and error still run), the
    // replay and the error once the frame is done. The copies then neither wait for the
    // end of the frame nor hold up the next frame of the internal stream (frames own
    // their outputs).
    int first_rc = HOLO_OK;
    int frame_no = 0;
    for (int i : pl.order) {
        const holo_frame_desc& d = f[i];
        const int k = pl.stream_of[i];
        char* slot = static_cast<char*>(d_ws) + size_t(k) * pl.slot_bytes;
        holo_stream_t hs = reinterpret_cast<holo_stream_t>(ds->st[k]);
        const size_t P = size_t(d.H) * size_t(d.W);
        cudaEvent_t ev_in = io ? ds->frame_ev[3 * frame_no] : nullptr;
        cudaEvent_t ev_bits = io ? ds->frame_ev[3 * frame_no + 1] : nullptr;
        cudaEvent_t ev_done = io ? ds->frame_ev[3 * frame_no + 2] : nullptr;
        ++frame_no;
        if (io && io[i].h_target) {
            if ((rc = frame_copy(const_cast<float*>(d.d_target), io[i].h_target, P * sizeof(float),
                                 cudaMemcpyHostToDevice, ds->copy_in, i, "batch: target copy"))) {
                first_rc = rc;
                break;
            }
            if ((e = cudaEventRecord(ev_in, ds->copy_in)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(ds->st[k], ev_in, 0)) != cudaSuccess) {
                first_rc = cuda_status(e, "batch: target copy event");
                break;
            }
        }
        if (d.build_lut && d.L > 0)
            if ((rc = lut_build(d.seed, d.L, d.levels, d.d_codes, nullptr, hs))) {
                first_rc = fail(rc, "batch frame %d: %s", i, holo_last_error());
                break;
            }
        const bool bits_early = io && io[i].h_holo_bits && d.d_holo_bits;
        if ((rc = ospr_generate_ev(d.d_target, d.H, d.W, d.N, d.d_codes, d.L, d.levels, d.seed, d.start_index,
                                   d.subframe_stride, precision, d.d_holo_bits, d.d_replay, slot + pl.ospr_off,
                                   pl.err_off - pl.ospr_off, hs, bits_early ? ev_bits : nullptr))) {
            first_rc = fail(rc, "batch frame %d: %s", i, holo_last_error());
            break;
        }
        if (d.d_err && (rc = replay_error(d.d_replay, d.d_target, nullptr, d.H, d.W, d.d_err, slot + pl.err_off,
                                          pl.slot_bytes - pl.err_off, hs))) {
            first_rc = fail(rc, "batch frame %d: %s", i, holo_last_error());
            break;
        }
        if (io) {
            cudaStream_t co = ds->copy_out[k];
            const size_t words = size_t(d.N) * (P / 32);
            if (bits_early) {
                if ((e = cudaStreamWaitEvent(co, ev_bits, 0)) != cudaSuccess) {
                    first_rc = cuda_status(e, "batch: bits copy event");
                    break;
                }
                if ((rc = frame_copy(io[i].h_holo_bits, d.d_holo_bits, words * sizeof(uint32_t),
                                     cudaMemcpyDeviceToHost, co, i, "batch: bits copy"))) {
                    first_rc = rc;
                    break;
                }
            }
            if ((e = cudaEventRecord(ev_done, ds->st[k])) != cudaSuccess ||
                (e = cudaStreamWaitEvent(co, ev_done, 0)) != cudaSuccess) {
                first_rc = cuda_status(e, "batch: result copy event");
                break;
            }
            if ((rc = frame_copy(io[i].h_replay, d.d_replay, P * sizeof(float), cudaMemcpyDeviceToHost, co, i,
                                 "batch: replay copy")) ||
                (rc = frame_copy(io[i].h_err, d.d_err, 3 * sizeof(double), cudaMemcpyDeviceToHost, co, i,
                                 "batch: error copy"))) {
                first_rc = rc;
                break;
            }
        }
    }
    // join every branch back to the caller's stream, also after an error, so that no
    // internal stream is left forked from a capture
    for (int k = 0; k < pl.streams; ++k) {
        if ((e = cudaEventRecord(ds->join[k], ds->st[k])) != cudaSuccess) return cuda_status(e, "batch: join record");
        if ((e = cudaStreamWaitEvent(s, ds->join[k], 0)) != cudaSuccess) return cuda_status(e, "batch: join wait");
        if (io) {
            if ((e = cudaEventRecord(ds->copy_out_join[k], ds->copy_out[k])) != cudaSuccess)
                return cuda_status(e, "batch: join record");
            if ((e = cudaStreamWaitEvent(s, ds->copy_out_join[k], 0)) != cudaSuccess)
                return cuda_status(e, "batch: join wait");
        }
    }
    if (io) {
        if ((e = cudaEventRecord(ds->copy_in_join, ds->copy_in)) != cudaSuccess)
            return cuda_status(e, "batch: join record");
        if ((e = cudaStreamWaitEvent(s, ds->copy_in_join, 0)) != cudaSuccess) return cuda_status(e, "batch: join wait");
    }
    return first_rc;
}

}  // namespace holo

using namespace holo;

struct holo_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int device;
    int64_t kernels;   // kernels one launch replays (launch accounting)
};

namespace holo {
// a holo_graph for graphs built in other translation units (the persistent batch)
holo_graph* make_holo_graph(cudaGraph_t graph, cudaGraphExec_t exec, int device, int64_t kernels) {
    return new holo_graph{graph, exec, device, kernels};
}
}  // namespace holo

extern "C" int ospr_batch_workspace_size(const holo_frame_desc* h_frames, int n_frames, int precision,
                                         size_t* bytes) {
    clear_error();
    if (!bytes) return fail(HOLO_EINVAL, "ospr_batch_workspace_size: NULL output");
    BatchPlan pl;
    int rc = plan_batch(h_frames, n_frames, precision, &pl);
    if (rc) return rc;
    *bytes = pl.total;
    return HOLO_OK;
}

extern "C" int ospr_generate_batch(const holo_frame_desc* h_frames, int n_frames, int precision,
                                   void* d_ws, size_t ws_bytes, holo_stream_t s) {
    clear_error();
    BatchPlan pl;
    int rc = plan_batch(h_frames, n_frames, precision, &pl);
    if (rc) return rc;
    return run_batch(h_frames, n_frames, precision, d_ws, ws_bytes, reinterpret_cast<cudaStream_t>(s), pl);
}

extern "C" int ospr_generate_batch_host(const holo_frame_desc* h_frames, const holo_frame_host* h_io, int n_frames,
                                        int precision, void* d_ws, size_t ws_bytes, holo_stream_t s) {
    clear_error();
    if (!h_io) return fail(HOLO_EINVAL, "ospr_generate_batch_host: NULL host buffer table");
    BatchPlan pl;
    int rc = plan_batch(h_frames, n_frames, precision, &pl);
    if (rc) return rc;
    for (int i = 0; i < n_frames; ++i) {
        if (h_io[i].h_holo_bits && !h_frames[i].d_holo_bits)
            return fail(HOLO_EINVAL, "batch frame %d: h_holo_bits without d_holo_bits", i);
        if (h_io[i].h_replay && !h_frames[i].d_replay)
            return fail(HOLO_EINVAL, "batch frame %d: h_replay without d_replay", i);
        if (h_io[i].h_err && !h_frames[i].d_err) return fail(HOLO_EINVAL, "batch frame %d: h_err without d_err", i);
    }
    return run_batch(h_frames, n_frames, precision, d_ws, ws_bytes, reinterpret_cast<cudaStream_t>(s), pl, h_io);
}

extern "C" int ospr_batch_graph_create(const holo_frame_desc* h_frames, int n_frames, int precision,
                                       void* d_ws, size_t ws_bytes, holo_graph** out) {
    clear_error();
    if (!out) return fail(HOLO_EINVAL, "ospr_batch_graph_create: NULL output");
    *out = nullptr;
    BatchPlan pl;
    int rc = plan_batch(h_frames, n_frames, precision, &pl);
    if (rc) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_status(e, "graph: cudaStreamCreate");
    // one eager run finishes every lazy set-up (tables, shared-memory limits) outside capture
    rc = run_batch(h_frames, n_frames, precision, d_ws, ws_bytes, cs, pl);
    if (rc == HOLO_OK) rc = cuda_status(cudaStreamSynchronize(cs), "graph: warm-up run");
    if (rc) {
        cudaStreamDestroy(cs);
        return rc;
    }
    const int prof = profiling_swap(0);   // no event timing inside a capture
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        profiling_swap(prof);
        cudaStreamDestroy(cs);
        return cuda_status(e, "graph: begin capture");
    }
    uint64_t before = 0, after = 0;
    holo_launch_count(&before);
    rc = run_batch(h_frames, n_frames, precision, d_ws, ws_bytes, cs, pl);
    holo_launch_count(&after);
    add_launches(-int64_t(after - before));   // captured, not run
    e = cudaStreamEndCapture(cs, &graph);
    profiling_swap(prof);
    cudaStreamDestroy(cs);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_status(e, "graph: end capture");
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_status(e, "graph: instantiate");
    }
    holo_graph* g = new holo_graph{graph, exec, dev, int64_t(after - before)};
    *out = g;
    return HOLO_OK;
}

extern "C" int holo_graph_launch(holo_graph* g, holo_stream_t s) {
    clear_error();
    if (!g) return fail(HOLO_EINVAL, "holo_graph_launch: NULL graph");
    const int rc = cuda_status(cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(s)), "holo_graph_launch");
    if (!rc) add_launches(g->kernels);
    return rc;
}

extern "C" int holo_graph_destroy(holo_graph* g) {
    clear_error();
    if (!g) return HOLO_OK;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return HOLO_OK;
}
