// batch_persistent.cu - the mixed-shape OSPR batch as one persistent launch with a device
// work queue (an engineering extension for batches of frames; every frame computes what
// ospr_generate and replay_error compute, paper Sections 2, 3, 5.2, Eq. 1-3).
//
// One CTA of 512 threads per SM takes work items in queue order from a global counter.
// An item is one CTA's worth of one pass of one frame: a table build range, a column
// IDFT tile of a sub-frame pair, a tile of 4 x LPR rows of the row pass, a column DFT
// tile with its accumulator group, a finalize range or one replay-error block. The pass
// bodies are the device functions of the per-frame kernels (variant 0 tiles), so a frame
// gives the same bits as ospr_generate + replay_error with those tiles and the same
// chunking. Dependencies are per-frame completion counters in device memory:
//   column IDFT of pair p   after the table (if built here), after the previous frame of
//                           the same workspace slot, and (chunks after the first) after
//                           every column DFT tile has consumed the field slot it reuses
//   row tiles of pair p     after all column IDFT tiles of pair p
//   column DFT tiles        per pair, after all row tiles of that pair; after every column
//                           DFT tile of the previous chunk (accumulator order)
//   finalize                after every column DFT tile of the last chunk
//   error blocks            after every finalize item
// The host orders each slot's items so that every item an item waits for lies earlier in
// the queue (the passes of consecutive pairs interleaved), and interleaves the slots. An
// item is only taken by a running CTA, so every wait is for work that is running or done:
// the queue cannot deadlock. Every wait is still bounded (%globaltimer): when one expires
// the kernel records a fault (holo_tc_status), raises an abort flag that every other wait
// and every CTA's next take check, and all CTAs return; the results are then not to be
// trusted.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "error_block.cuh"
#include "ospr_kernels.cuh"

namespace holo {

constexpr int kPThreads = 512;
constexpr int kPLutPerItem = kPThreads * 64;      // table entries per build item
constexpr int kPFinPerItem = kPThreads * 8;       // finalize pixel pairs per item

enum PKind : uint16_t { kPLut = 0, kPColIfft = 1, kPRow = 2, kPColFft = 3, kPFin = 4, kPErr = 5 };

struct PItem {
    uint32_t frame;
    uint16_t kind;
    uint16_t pair;     // pair (column IDFT, row) or chunk (column DFT)
    uint32_t tile;     // tile / range / block index
};

struct PFrame {
    const OsprArgs* chunks;     // [nchunks] the pass arguments of each chunk (device table)
    int H, W;
    int chunk, npairs, nchunks;
    int lut_items, ci_tiles, row_tiles, row_rows, cf_tiles, fin_items, err_items;
    int ci_tiles_cf;            // column DFT tiles that read one pair (one per column tile)
    int prev;                   // previous frame on the same workspace slot, or -1
    uint8_t* codes;             // table to build (lut_items > 0)
    int64_t L;
    uint64_t seed;
    int code_bits;
    float* replay;
    double* err;
    float fin_scale;
    ff* err_part;
    // counters: [0] table items, [1] finalize items, [2] frame done, [3] error blocks,
    // then ci_done[npairs], row_done[npairs], cf_read[npairs], cf_fin[nchunks]
    unsigned* cnt;
};

__device__ int g_persist_fault;   // set when a dependency wait of the persistent kernel expired

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct PCtl {
    unsigned* next;        // queue cursor
    unsigned* abort_flag;  // nonzero: stop
    uint64_t limit_ns;     // bound of one wait
    int inject;            // test hook: every wait waits for a count nothing reaches
};

// Every thread of the CTA calls it: thread 0 polls (acquire) until *ctr >= target, the
// abort flag is raised or limit_ns passes; returns false (uniformly) on abort or expiry.
__device__ bool pwait(const PCtl& c, const unsigned* ctr, unsigned target) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (c.inject) target = 0xffffffffu;
        if (ld_acquire_u32(ctr) < target) {
            const uint64_t t0 = globaltimer_ns();
            unsigned ns = 32;
            while (ld_acquire_u32(ctr) < target) {
                if (*reinterpret_cast<volatile unsigned*>(c.abort_flag)) { ok = 0; break; }
                if (globaltimer_ns() - t0 > c.limit_ns) {
                    atomicExch(&g_persist_fault, 1);
                    atomicExch(c.abort_flag, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                ns = ns < 1024 ? 2 * ns : 1024;
            }
        }
        if (ok) asm volatile("fence.acq_rel.gpu;" ::: "memory");
        s_ok = ok;
    }
    __syncthreads();
    const bool r = s_ok != 0;
    __syncthreads();   // every thread has read s_ok before the next wait may rewrite it
    return r;
}

// after the CTA's work: *ctr += 1 with release semantics; returns the old value in thread 0
__device__ __forceinline__ unsigned psignal(unsigned* ctr) {
    __syncthreads();
    unsigned old = 0;
    if (threadIdx.x == 0) {
        __threadfence();
        old = atomicAdd(ctr, 1u);
    }
    return old;
}

__device__ __forceinline__ unsigned* ci_done(const PFrame& f) { return f.cnt + 4; }
__device__ __forceinline__ unsigned* row_done(const PFrame& f) { return f.cnt + 4 + f.npairs; }
__device__ __forceinline__ unsigned* cf_read(const PFrame& f) { return f.cnt + 4 + 2 * f.npairs; }
__device__ __forceinline__ unsigned* cf_fin(const PFrame& f) { return f.cnt + 4 + 3 * f.npairs; }

template <int NC>
__device__ __forceinline__ void p_col_ifft(const OsprArgs& a, int tile, int slot) {
    ospr_col_ifft_body<NC, 0>(a, tile, slot);
}
template <int NR>
__device__ __forceinline__ void p_row(const OsprArgs& a, int row0, int slot) {
    ospr_row_body<NR, 0, true, false>(a, row0, slot);
}

// the column DFT tile waits, before each of its pairs, for that pair's row tiles
template <int NC>
__device__ __forceinline__ bool p_col_fft(const PCtl& c, const PFrame& f, const OsprArgs& a, int tile, int g) {
    bool ok = true;
    auto before = [&](int j) {
        if (ok) ok = pwait(c, row_done(f) + a.first_pair + j, unsigned(f.row_tiles));
    };
    ospr_col_fft_body<NC, 0>(a, tile, g, before, NoHook{});
    return ok;
}

__global__ void __launch_bounds__(kPThreads, 1)
k_ospr_persistent(const PFrame* __restrict__ frames, const PItem* __restrict__ items, int n_items, PCtl c) {
    __shared__ unsigned s_item;
    for (;;) {
        __syncthreads();   // the previous item is done with shared memory and s_item
        if (threadIdx.x == 0) {
            unsigned i = unsigned(n_items);
            if (!*reinterpret_cast<volatile unsigned*>(c.abort_flag)) i = atomicAdd(c.next, 1u);
            s_item = i;
        }
        __syncthreads();
        const unsigned i = s_item;
        if (i >= unsigned(n_items)) return;
        const PItem it = items[i];
        const PFrame& f = frames[it.frame];
        const int H = f.H, W = f.W;
        bool ok = true;
        switch (it.kind) {
            case kPLut: {
                const int64_t base = int64_t(it.tile) * kPLutPerItem;
                for (int k = 0; k < kPLutPerItem / kPThreads; ++k) {
                    const int64_t e = base + int64_t(k) * kPThreads + threadIdx.x;
                    if (e < f.L) f.codes[e] = lut_entry(f.seed, uint64_t(e), f.code_bits);
                }
                psignal(f.cnt + 0);
                break;
            }
            case kPColIfft: {
                const int p = it.pair, k = p / f.chunk;
                if (f.lut_items) ok = pwait(c, f.cnt + 0, unsigned(f.lut_items));
                if (ok && k == 0 && f.prev >= 0) ok = pwait(c, frames[f.prev].cnt + 2, 1u);
                if (ok && k > 0) ok = pwait(c, cf_read(f) + (p - f.chunk), unsigned(f.ci_tiles_cf));
                if (!ok) break;
                const OsprArgs& a = f.chunks[k];
                const int slot = p - a.first_pair;
                if (H == 512) p_col_ifft<512>(a, it.tile, slot);
                else if (H == 1024) p_col_ifft<1024>(a, it.tile, slot);
                else p_col_ifft<2048>(a, it.tile, slot);
                psignal(ci_done(f) + p);
                break;
            }
            case kPRow: {
                const int p = it.pair, k = p / f.chunk;
                if (!pwait(c, ci_done(f) + p, unsigned(f.ci_tiles))) { ok = false; break; }
                const OsprArgs& a = f.chunks[k];
                const int slot = p - a.first_pair;
                const int row0 = int(it.tile) * f.row_rows;
                if (W == 512) p_row<512>(a, row0, slot);
                else if (W == 1024) p_row<1024>(a, row0, slot);
                else p_row<2048>(a, row0, slot);
                psignal(row_done(f) + p);
                break;
            }
            case kPColFft: {
                const int k = it.pair;
                if (k > 0 && !pwait(c, cf_fin(f) + (k - 1), unsigned(f.cf_tiles))) { ok = false; break; }
                const OsprArgs& a = f.chunks[k];
                const int tile = int(it.tile) / a.groups, g = int(it.tile) % a.groups;
                if (H == 512) ok = p_col_fft<512>(c, f, a, tile, g);
                else if (H == 1024) ok = p_col_fft<1024>(c, f, a, tile, g);
                else ok = p_col_fft<2048>(c, f, a, tile, g);
                if (!ok) break;
                // every pair of this tile's group has been read and transformed
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    for (int j = g; j < a.pairs; j += a.groups) atomicAdd(cf_read(f) + a.first_pair + j, 1u);
                }
                psignal(cf_fin(f) + k);
                break;
            }
            case kPFin: {
                if (!pwait(c, cf_fin(f) + (f.nchunks - 1), unsigned(f.cf_tiles))) { ok = false; break; }
                const size_t base = size_t(it.tile) * kPFinPerItem;
                for (int k = 0; k < kPFinPerItem / kPThreads; ++k)
                    ospr_finalize_pixel(f.chunks[0].sacc, f.chunks[0].groups, H, W, f.fin_scale, f.replay,
                                        base + size_t(k) * kPThreads + threadIdx.x);
                const unsigned old = psignal(f.cnt + 1);
                if (threadIdx.x == 0 && !f.err && old + 1 == unsigned(f.fin_items)) {
                    __threadfence();
                    atomicExch(f.cnt + 2, 1u);   // the frame is done
                }
                break;
            }
            case kPErr: {
                if (!pwait(c, f.cnt + 1, unsigned(f.fin_items))) { ok = false; break; }
                replay_error_block(f.replay, f.chunks[0].target, nullptr, int64_t(H) * W, f.err_part, f.cnt + 3, f.err,
                                   int(it.tile), f.err_items, f.cnt + 2);
                break;
            }
            default:
                break;
        }
        if (!ok) return;   // a wait expired or another CTA aborted: stop taking items
    }
}

// ------------------------------------------------------------------- host ----
static int persist_smem_bytes() {
    size_t m = 0;
    m = std::max(m, col_ifft_smem_bytes<512, 0>());
    m = std::max(m, col_ifft_smem_bytes<1024, 0>());
    m = std::max(m, col_ifft_smem_bytes<2048, 0>());
    m = std::max(m, col_fft_smem_bytes<512, 0>());
    m = std::max(m, col_fft_smem_bytes<1024, 0>());
    m = std::max(m, col_fft_smem_bytes<2048, 0>());
    m = std::max(m, 4 * row_smem_bytes<512, 0>());
    m = std::max(m, 4 * row_smem_bytes<1024, 0>());
    m = std::max(m, 4 * row_smem_bytes<2048, 0>());
    return int(m);
}

static bool persist_len(int n) { return n == 512 || n == 1024 || n == 2048; }
static int col_lpc(int H) { return H == 512 ? ColCfg<512, 0>::LPC : H == 1024 ? ColCfg<1024, 0>::LPC : ColCfg<2048, 0>::LPC; }
static int row_lpr(int W) { return W == 512 ? RowCfg<512, 0>::LPR : W == 1024 ? RowCfg<1024, 0>::LPR : RowCfg<2048, 0>::LPR; }

struct PPlan {
    int slots;
    std::vector<int> slot_of;
    size_t slot_bytes, z_off, s_off, e_off;     // one slot: fields, accumulators, error partials
    size_t cnt_off, cnt_bytes, frames_off, args_off, items_off, ctl_off, total;
    std::vector<PFrame> frames;
    std::vector<OsprArgs> args;   // every frame's chunks, in frame order
    std::vector<int> args_first;  // index of frame i's first chunk in `args`
    std::vector<PItem> items;
};

static int persist_plan(const holo_frame_desc* f, int n, PPlan* pl, bool build_items) {
    if (!f || n < 1 || n > 65535) return fail(HOLO_EINVAL, "persistent batch: %d frames", n);
    const char* env = getenv("HOLO_BATCH_STREAMS");
    int S = env && *env ? atoi(env) : 8;
    S = std::max(1, std::min(S, 32));
    pl->slots = std::min(S, n);
    size_t max_z = 0, max_s = 0, max_e = 0, cnt_words = 0, n_chunks = 0;
    std::vector<int> chunk(n), groups(n), npairs(n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        const holo_frame_desc& d = f[i];
        if (!persist_len(d.H) || !persist_len(d.W))
            return fail(HOLO_EUNSUPPORTED, "persistent batch frame %d: %dx%d (H and W in {512, 1024, 2048})", i, d.H, d.W);
        if (d.N < 1 || d.N > 4096) return fail(HOLO_EINVAL, "persistent batch frame %d: N=%d", i, d.N);
        if (!d.d_target || !d.d_replay)
            return fail(HOLO_EINVAL, "persistent batch frame %d: the target and the replay are required", i);
        int ci, cf, rv, ch, gr;
        int rc = ospr_tuning_get(d.H, d.W, &ci, &cf, &rv, &ch, &gr);
        if (rc) return rc;
        npairs[i] = (d.N + 1) / 2;
        chunk[i] = std::min(ch, npairs[i]);
        groups[i] = std::min(gr, chunk[i]);
        const size_t P = size_t(d.H) * d.W;
        max_z = std::max(max_z, align_up(size_t(chunk[i]) * P * sizeof(float2), 256));
        max_s = std::max(max_s, align_up(size_t(groups[i]) * P * sizeof(float), 256));
        max_e = std::max(max_e, align_up(sizeof(ff) * size_t(err_blocks(int64_t(P))) * kErrParts, 256));
        const int nchunks = (npairs[i] + chunk[i] - 1) / chunk[i];
        cnt_words += size_t(4 + 3 * npairs[i] + nchunks);
        n_chunks += size_t(nchunks);
        cost[i] = double(P) * double(npairs[i]);
    }
    pl->z_off = 0;
    pl->s_off = max_z;
    pl->e_off = max_z + max_s;
    pl->slot_bytes = max_z + max_s + max_e;
    pl->cnt_off = pl->slot_bytes * size_t(pl->slots);
    pl->cnt_bytes = align_up(cnt_words * sizeof(unsigned), 256);
    pl->ctl_off = pl->cnt_off + pl->cnt_bytes;                    // next, abort
    pl->frames_off = pl->ctl_off + 256;
    pl->args_off = pl->frames_off + align_up(sizeof(PFrame) * size_t(n), 256);
    pl->items_off = pl->args_off + align_up(sizeof(OsprArgs) * n_chunks, 256);
    // longest frame first onto the least-loaded slot
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(pl->slots, 0.0);
    pl->slot_of.assign(n, 0);
    std::vector<std::vector<int>> slot_frames(pl->slots);
    for (int i : order) {
        const int k = int(std::min_element(load.begin(), load.end()) - load.begin());
        pl->slot_of[i] = k;
        load[k] += cost[i];
        slot_frames[k].push_back(i);
    }
    // item count (for the workspace size) and, when asked, the items themselves
    size_t n_items = 0;
    std::vector<std::vector<PItem>> streams(pl->slots);
    pl->frames.assign(n, PFrame{});
    size_t cnt_pos = 0;
    for (int k = 0; k < pl->slots; ++k) {
        int prev = -1;
        for (int i : slot_frames[k]) {
            const holo_frame_desc& d = f[i];
            const int H = d.H, W = d.W, N = d.N;
            const int np = npairs[i], ch = chunk[i], gr = groups[i];
            const int nchunks = (np + ch - 1) / ch;
            PFrame& F = pl->frames[i];
            F.H = H;
            F.W = W;
            F.chunk = ch;
            F.npairs = np;
            F.nchunks = nchunks;
            F.lut_items = (d.build_lut && d.L > 0) ? int((d.L + kPLutPerItem - 1) / kPLutPerItem) : 0;
            F.ci_tiles = W / col_lpc(H);
            F.row_rows = 4 * row_lpr(W);
            F.row_tiles = H / F.row_rows;
            F.cf_tiles = (W / col_lpc(H)) * gr;
            F.ci_tiles_cf = W / col_lpc(H);
            const size_t P = size_t(H) * W;
            F.fin_items = int((P / 2 + W + kPFinPerItem - 1) / kPFinPerItem);
            F.err_items = d.d_err ? err_blocks(int64_t(P)) : 0;
            F.prev = prev;
            F.cnt = reinterpret_cast<unsigned*>(cnt_pos);   // offset, made a pointer at launch
            cnt_pos += size_t(4 + 3 * np + nchunks) * sizeof(unsigned);
            prev = i;
            (void)N;
            std::vector<PItem>& q = streams[k];
            auto push = [&](PKind kind, int pair, int tile) {
                ++n_items;
                if (build_items) q.push_back(PItem{uint32_t(i), uint16_t(kind), uint16_t(pair), uint32_t(tile)});
            };
            for (int t = 0; t < F.lut_items; ++t) push(kPLut, 0, t);
            for (int c = 0; c < nchunks; ++c) {
                const int p0 = c * ch, p1 = std::min(np, p0 + ch);
                // column IDFT of pair p, then the rows of pair p - 1: the row tiles of a pair
                // follow its column tiles by one pair's worth of items
                for (int p = p0; p <= p1; ++p) {
                    if (p < p1)
                        for (int t = 0; t < F.ci_tiles; ++t) push(kPColIfft, p, t);
                    if (p > p0)
                        for (int t = 0; t < F.row_tiles; ++t) push(kPRow, p - 1, t);
                }
                for (int t = 0; t < F.cf_tiles; ++t) push(kPColFft, c, t);
            }
            for (int t = 0; t < F.fin_items; ++t) push(kPFin, 0, t);
            for (int t = 0; t < F.err_items; ++t) push(kPErr, 0, t);
        }
    }
    if (build_items) {
        // round-robin merge of the slots' item streams
        pl->items.clear();
        pl->items.reserve(n_items);
        std::vector<size_t> pos(pl->slots, 0);
        for (bool more = true; more;) {
            more = false;
            for (int k = 0; k < pl->slots; ++k)
                if (pos[k] < streams[k].size()) {
                    pl->items.push_back(streams[k][pos[k]++]);
                    more = true;
                }
        }
    }
    pl->total = pl->items_off + align_up(sizeof(PItem) * n_items, 256);
    return HOLO_OK;
}

// fills the device-side frame table and every chunk's pass arguments: pointers into the
// workspace, the table draw, the chunk's pairs and accumulate flag
static int persist_frames(const holo_frame_desc* f, int n, PPlan& pl, char* ws, const Tables& tab) {
    pl.args.clear();
    pl.args_first.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        const holo_frame_desc& d = f[i];
        PFrame& F = pl.frames[i];
        const int64_t P = int64_t(d.H) * d.W;
        PhaseSource ps;
        int rc = make_phase_source("ospr_generate_batch_persistent", d.d_codes, d.L, d.levels, d.seed,
                                   d.start_index, d.subframe_stride == 0 ? P : d.subframe_stride, &ps);
        if (rc) return fail(rc, "persistent batch frame %d: %s", i, holo_last_error());
        char* slot = ws + size_t(pl.slot_of[i]) * pl.slot_bytes;
        int ci, cf, rv, ch, gr;
        if ((rc = ospr_tuning_get(d.H, d.W, &ci, &cf, &rv, &ch, &gr))) return rc;
        OsprArgs a{};
        a.target = d.d_target;
        a.H = d.H;
        a.W = d.W;
        a.N = d.N;
        a.ps = ps;
        a.zbuf = reinterpret_cast<float2*>(slot + pl.z_off);
        a.sacc = reinterpret_cast<float*>(slot + pl.s_off);
        a.groups = std::min(gr, F.chunk);
        a.bits = d.d_holo_bits;
        a.tw = tab.twiddles;
        a.cs256 = tab.cs256;
        a.tc05b = nullptr;
        a.fresnel = 0;
        a.chirp_y = a.chirp_x = nullptr;
        pl.args_first[i] = int(pl.args.size());
        for (int k = 0; k < F.nchunks; ++k) {
            a.first_pair = k * F.chunk;
            a.pairs = std::min(F.chunk, F.npairs - a.first_pair);
            a.accumulate = k > 0;
            pl.args.push_back(a);
        }
        F.chunks = reinterpret_cast<const OsprArgs*>(ws + pl.args_off) + pl.args_first[i];
        F.codes = d.build_lut && d.L > 0 ? const_cast<uint8_t*>(d.d_codes) : nullptr;
        F.L = d.L;
        F.seed = d.seed;
        F.code_bits = log2i(d.levels);
        F.replay = d.d_replay;
        F.err = d.d_err;
        F.fin_scale = float(1.0 / (2.0 * double(d.N) * double(P)));
        F.err_part = reinterpret_cast<ff*>(slot + pl.e_off);
        F.cnt = reinterpret_cast<unsigned*>(ws + pl.cnt_off + reinterpret_cast<size_t>(F.cnt));
    }
    return HOLO_OK;
}

static int persist_check_ws(void* d_ws, size_t ws_bytes, size_t need) {
    if (!d_ws || ws_bytes < need)
        return fail(HOLO_EWORKSPACE, "persistent batch: workspace %zu bytes, need %zu", ws_bytes, need);
    if (reinterpret_cast<uintptr_t>(d_ws) % 256 != 0)
        return fail(HOLO_EWORKSPACE, "persistent batch: workspace is not 256-byte aligned");
    return HOLO_OK;
}

// clears the counters and the queue state, then launches the kernel (capturable)
static int persist_launch(const PPlan& pl, char* ws, int wait_limit_us, cudaStream_t st) {
    static uint64_t mask = 0;
    const int smem = persist_smem_bytes();
    int rc = ensure_smem((const void*)k_ospr_persistent, size_t(smem), &mask);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(ws + pl.cnt_off, 0, pl.cnt_bytes + 256, st);
    if (e != cudaSuccess) return cuda_status(e, "persistent batch: counter clear");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_status(e, "persistent batch: SM count");
    PCtl c;
    c.next = reinterpret_cast<unsigned*>(ws + pl.ctl_off);
    c.abort_flag = c.next + 1;
    c.limit_ns = uint64_t(wait_limit_us > 0 ? wait_limit_us : 1000000) * 1000u;
    c.inject = fault_injected("persist_wait") ? 1 : 0;
    const int n_items = int(pl.items.size());
    const int grid = std::max(1, std::min(sms, n_items));
    Launch ln("ospr_persistent", st);
    k_ospr_persistent<<<grid, kPThreads, smem, st>>>(reinterpret_cast<const PFrame*>(ws + pl.frames_off),
                                                     reinterpret_cast<const PItem*>(ws + pl.items_off), n_items, c);
    return ln.done("ospr_persistent launch");
}

// writes the frame table and the queue into the workspace: a synchronous copy from pageable
// host memory, ordered on the stream before the launch
static int persist_upload(const PPlan& pl, char* ws, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(ws + pl.frames_off, pl.frames.data(), sizeof(PFrame) * pl.frames.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + pl.args_off, pl.args.data(), sizeof(OsprArgs) * pl.args.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + pl.items_off, pl.items.data(), sizeof(PItem) * pl.items.size(),
                            cudaMemcpyHostToDevice, st);
    return cuda_status(e, "persistent batch: queue upload");
}

int ospr_persistent_fault(int* out, bool clear) {
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_persist_fault, sizeof(int));
    if (e != cudaSuccess) return cuda_status(e, "ospr_persistent_fault");
    if (clear && v) {
        const int z = 0;
        if ((e = cudaMemcpyToSymbol(g_persist_fault, &z, sizeof(int))) != cudaSuccess)
            return cuda_status(e, "ospr_persistent_fault");
    }
    *out = v;
    return HOLO_OK;
}

}  // namespace holo

using namespace holo;

extern "C" int ospr_batch_persistent_workspace_size(const holo_frame_desc* h_frames, int n_frames, size_t* bytes) {
    clear_error();
    if (!bytes) return fail(HOLO_EINVAL, "ospr_batch_persistent_workspace_size: NULL output");
    PPlan pl;
    int rc = persist_plan(h_frames, n_frames, &pl, false);
    if (rc) return rc;
    *bytes = pl.total;
    return HOLO_OK;
}

extern "C" int ospr_generate_batch_persistent(const holo_frame_desc* h_frames, int n_frames, int wait_limit_us,
                                              void* d_ws, size_t ws_bytes, holo_stream_t s) {
    clear_error();
    if (wait_limit_us < 0) return fail(HOLO_EINVAL, "ospr_generate_batch_persistent: wait limit %d", wait_limit_us);
    PPlan pl;
    int rc = persist_plan(h_frames, n_frames, &pl, true);
    if (rc) return rc;
    if ((rc = persist_check_ws(d_ws, ws_bytes, pl.total))) return rc;
    Tables tab;
    if ((rc = device_tables(&tab))) return rc;
    char* ws = static_cast<char*>(d_ws);
    if ((rc = persist_frames(h_frames, n_frames, pl, ws, tab))) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
    if ((rc = persist_upload(pl, ws, st))) return rc;
    return persist_launch(pl, ws, wait_limit_us, st);
}

extern "C" int ospr_batch_persistent_graph_create(const holo_frame_desc* h_frames, int n_frames, int wait_limit_us,
                                                  void* d_ws, size_t ws_bytes, holo_graph** out) {
    clear_error();
    if (!out) return fail(HOLO_EINVAL, "ospr_batch_persistent_graph_create: NULL output");
    *out = nullptr;
    if (wait_limit_us < 0) return fail(HOLO_EINVAL, "ospr_batch_persistent_graph_create: wait limit %d", wait_limit_us);
    PPlan pl;
    int rc = persist_plan(h_frames, n_frames, &pl, true);
    if (rc) return rc;
    if ((rc = persist_check_ws(d_ws, ws_bytes, pl.total))) return rc;
    Tables tab;
    if ((rc = device_tables(&tab))) return rc;
    char* ws = static_cast<char*>(d_ws);
    if ((rc = persist_frames(h_frames, n_frames, pl, ws, tab))) return rc;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_status(e, "graph: cudaStreamCreate");
    // the frame table and the queue stay in the workspace: uploaded once, outside the capture
    rc = persist_upload(pl, ws, cs);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(cs), "graph: queue upload");
    static uint64_t mask = 0;
    if (!rc) rc = ensure_smem((const void*)k_ospr_persistent, size_t(persist_smem_bytes()), &mask);
    if (rc) {
        cudaStreamDestroy(cs);
        return rc;
    }
    const int prof = profiling_swap(0);
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        profiling_swap(prof);
        cudaStreamDestroy(cs);
        return cuda_status(e, "graph: begin capture");
    }
    uint64_t before = 0, after = 0;
    holo_launch_count(&before);
    rc = persist_launch(pl, ws, wait_limit_us, cs);
    holo_launch_count(&after);
    add_launches(-int64_t(after - before));
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
    *out = make_holo_graph(graph, exec, dev, int64_t(after - before));
    return HOLO_OK;
}
