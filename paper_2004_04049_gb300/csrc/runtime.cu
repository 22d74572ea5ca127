// runtime.cu - status, launch accounting, event profiling and device tables.
#include "runtime.h"

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fft_core.cuh"
#include "tc05_dft.cuh"

namespace holo {

// ------------------------------------------------------------------ status ----
static thread_local std::string t_last_error;

static void vrecord(const char* fmt, va_list ap) {
    char buf[1024];
    vsnprintf(buf, sizeof(buf), fmt, ap);
    t_last_error = buf;
}

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vrecord(fmt, ap);
    va_end(ap);
    return code;
}

void warn(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    char buf[1024];
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (!t_last_error.empty()) t_last_error += "; ";
    t_last_error += buf;
}

void clear_error() { t_last_error.clear(); }

int cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HOLO_OK;
    return fail(HOLO_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ------------------------------------------------------- launches/profiling ----
static std::atomic<uint64_t> g_launches{0};
static std::atomic<int> g_profiling{0};

struct PendingPair {
    cudaEvent_t start, stop;
};
struct FamilyStats {
    uint64_t launches = 0;
    double total_ms = 0.0;
    std::vector<PendingPair> pending;
};
static std::mutex g_prof_mu;
static std::map<std::string, FamilyStats> g_prof;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t take_event() {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

Launch::Launch(const char* family, cudaStream_t stream) : family_(family), stream_(stream) {
    if (g_profiling.load(std::memory_order_relaxed)) {
        start_ = take_event();
        if (start_ && cudaEventRecord(start_, stream_) != cudaSuccess) start_ = nullptr;
    }
}

int Launch::done(const char* what, cudaError_t launch) {
    cudaError_t e = cudaGetLastError();
    if (launch != cudaSuccess) e = launch;
    if (e != cudaSuccess) return cuda_status(e, what);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (start_) {
        cudaEvent_t stop = take_event();
        if (stop && cudaEventRecord(stop, stream_) == cudaSuccess) {
            std::lock_guard<std::mutex> lk(g_prof_mu);
            g_prof[family_].pending.push_back({start_, stop});
        }
    }
    return HOLO_OK;
}

int profiling_swap(int on) { return g_profiling.exchange(on ? 1 : 0); }

void add_launches(int64_t n) { g_launches.fetch_add(uint64_t(n), std::memory_order_relaxed); }

bool fault_injected(const char* kind) {
    const char* v = getenv("HOLO_FAULT_INJECT");
    if (!v || !*v) return false;
    const size_t n = strlen(kind);
    for (const char* p = v; *p;) {
        const char* e = strchr(p, ',');
        const size_t len = e ? size_t(e - p) : strlen(p);
        if (len == n && strncmp(p, kind, n) == 0) return true;
        if (!e) break;
        p = e + 1;
    }
    return false;
}

static int collect_locked() {
    for (auto& kv : g_prof) {
        FamilyStats& fs = kv.second;
        for (auto& pp : fs.pending) {
            cudaError_t e = cudaEventSynchronize(pp.stop);
            if (e != cudaSuccess) return cuda_status(e, "profile: cudaEventSynchronize");
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, pp.start, pp.stop);
            if (e != cudaSuccess) return cuda_status(e, "profile: cudaEventElapsedTime");
            fs.launches += 1;
            fs.total_ms += ms;
            g_event_pool.push_back(pp.start);
            g_event_pool.push_back(pp.stop);
        }
        fs.pending.clear();
    }
    return HOLO_OK;
}

// ---------------------------------------------------------- device tables ----
static __device__ float2 g_twiddles[kTwiddleTotal];
static __device__ float2 g_cs256[256];
// tcgen05 DFT-32 B operands: [precision fp16, bf16][direction -1, +1][hi, lo][8192 bytes].
// Row j (output) holds the coefficients of input i (K): outputs 0..31 are Re X_k, 32..63
// Im X_k; inputs 0..31 are Re x_n, 32..63 Im x_n; X_k = sum_n x_n exp(i DIR 2 pi n k / 32).
static __device__ uint4 g_tc05_b[2 * 2 * 2 * 8192 / 16];

static void host_tc05_b(uint8_t* out, bool bf16) {
    const double two_pi = 6.283185307179586476925286766559;
    auto conv = [&](float x) -> uint16_t {
        if (bf16) {
            const __nv_bfloat16 b = __float2bfloat16_rn(x);
            return *reinterpret_cast<const uint16_t*>(&b);
        }
        const __half h = __float2half_rn(x);
        return *reinterpret_cast<const uint16_t*>(&h);
    };
    auto back = [&](uint16_t u) -> float {
        if (bf16) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(&u));
        return __half2float(*reinterpret_cast<const __half*>(&u));
    };
    for (int d = 0; d < 2; ++d) {
        const double dir = d == 0 ? -1.0 : 1.0;
        uint8_t* hi = out + size_t(d) * 2 * 8192;
        uint8_t* lo = hi + 8192;
        for (int j = 0; j < 64; ++j)
            for (int i = 0; i < 64; ++i) {
                const int k = j & 31, n = i & 31;
                const double ang = two_pi * double(n) * double(k) / 32.0;
                double c;
                if (j < 32 && i < 32) c = std::cos(ang);
                else if (j < 32) c = -dir * std::sin(ang);
                else if (i < 32) c = dir * std::sin(ang);
                else c = std::cos(ang);
                const float x = float(c);
                const uint16_t h = conv(x);
                const uint16_t l = conv(x - back(h));
                const uint32_t off = sw128_offset(j, i);
                memcpy(hi + off, &h, 2);
                memcpy(lo + off, &l, 2);
            }
    }
}

static std::mutex g_tab_mu;
static const int kMaxDevices = 64;
static Tables g_tables[kMaxDevices];
static bool g_tables_ready[kMaxDevices];

static void host_twiddles(std::vector<float2>& out) {
    out.assign(kTwiddleTotal, make_float2(0.f, 0.f));
    const double two_pi = 6.283185307179586476925286766559;
    for (int lg = kMinLog2; lg <= kMaxLog2; ++lg)
        for (int lr = 1; lr <= 5; ++lr) {
            const int N = 1 << lg, R = 1 << lr;
            for (int s = 1; s < stage_count(N, R); ++s) {
                const int Ns = stage_ns(N, R, s), Rs = stage_radix(N, R, s);
                const int off = stage_offset(N, R, s);
                for (int m = 0; m < Rs; ++m)
                    for (int k = 0; k < Ns; ++k) {
                        const double ang = two_pi * double(k) * double(m) / double(Ns * Rs);
                        out[off + m * Ns + k] = make_float2(float(std::cos(ang)), float(std::sin(ang)));
                    }
            }
        }
}

int device_tables(Tables* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(HOLO_EUNSUPPORTED, "device index %d too large", dev);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (!g_tables_ready[dev]) {
        std::vector<float2> tw;
        host_twiddles(tw);
        std::vector<float2> cs(256);
        const double two_pi = 6.283185307179586476925286766559;
        for (int c = 0; c < 256; ++c)
            cs[c] = make_float2(float(std::cos(two_pi * c / 256.0)), float(std::sin(two_pi * c / 256.0)));
        e = cudaMemcpyToSymbol(g_twiddles, tw.data(), sizeof(float2) * tw.size());
        if (e != cudaSuccess) return cuda_status(e, "upload twiddles");
        e = cudaMemcpyToSymbol(g_cs256, cs.data(), sizeof(float2) * 256);
        if (e != cudaSuccess) return cuda_status(e, "upload cos/sin table");
        std::vector<uint8_t> b05(sizeof(g_tc05_b));
        host_tc05_b(b05.data(), false);
        host_tc05_b(b05.data() + b05.size() / 2, true);
        e = cudaMemcpyToSymbol(g_tc05_b, b05.data(), b05.size());
        if (e != cudaSuccess) return cuda_status(e, "upload tcgen05 DFT matrices");
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_twiddles);
        if (e != cudaSuccess) return cuda_status(e, "twiddle address");
        g_tables[dev].twiddles = static_cast<const float2*>(p);
        e = cudaGetSymbolAddress(&p, g_cs256);
        if (e != cudaSuccess) return cuda_status(e, "cos/sin table address");
        g_tables[dev].cs256 = static_cast<const float2*>(p);
        e = cudaGetSymbolAddress(&p, g_tc05_b);
        if (e != cudaSuccess) return cuda_status(e, "tcgen05 DFT matrix address");
        g_tables[dev].tc05b[0] = nullptr;
        g_tables[dev].tc05b[1] = static_cast<const uint8_t*>(p);
        g_tables[dev].tc05b[2] = static_cast<const uint8_t*>(p) + 4 * 8192;
        g_tables_ready[dev] = true;
    }
    *out = g_tables[dev];
    return HOLO_OK;
}

int ensure_smem(const void* fn, size_t bytes, uint64_t* device_mask) {
    if (bytes <= 48 * 1024) return HOLO_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    const uint64_t bit = 1ull << (dev & 63);
    if (__atomic_load_n(device_mask, __ATOMIC_ACQUIRE) & bit) return HOLO_OK;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(shared memory)");
    __atomic_fetch_or(device_mask, bit, __ATOMIC_ACQ_REL);
    return HOLO_OK;
}

int resident_ctas(const void* fn, int threads, size_t bytes, int* cache, int* ctas) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    int n = __atomic_load_n(cache + (dev & 63), __ATOMIC_ACQUIRE);
    if (n <= 0) {
        int per_sm = 0, sms = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, bytes)) != cudaSuccess)
            return cuda_status(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_status(e, "cudaDeviceGetAttribute(SM count)");
        if (per_sm < 1) return fail(HOLO_ECUDA, "a kernel of %d threads and %zu bytes fits no SM", threads, bytes);
        n = per_sm * sms;
        __atomic_store_n(cache + (dev & 63), n, __ATOMIC_RELEASE);
    }
    *ctas = n;
    return HOLO_OK;
}

}  // namespace holo

// ================================================================== C ABI ====
using namespace holo;

extern "C" int holo_version(void) { return 10000; }

extern "C" const char* holo_last_error(void) { return t_last_error.c_str(); }

extern "C" int holo_check(holo_stream_t s) {
    clear_error();
    if (fault_injected("timeout")) return fail(HOLO_ETIMEOUT, "holo_check: injected timeout (HOLO_FAULT_INJECT)");
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(s));
    if (e != cudaSuccess) return cuda_status(e, "holo_check: stream");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "holo_check");
    int fault = 0;
    int rc = holo_tc_status(&fault, 0);
    if (rc) return rc;
    if (fault) return fail(HOLO_ETIMEOUT, "holo_check: a tcgen05 kernel gave up on a bounded wait");
    return HOLO_OK;
}

extern "C" int holo_launch_count(uint64_t* out_count) {
    if (!out_count) return fail(HOLO_EINVAL, "holo_launch_count: NULL output");
    *out_count = g_launches.load();
    return HOLO_OK;
}

extern "C" int holo_profile_enable(int on) {
    g_profiling.store(on ? 1 : 0);
    return HOLO_OK;
}

extern "C" int holo_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int rc = collect_locked();
    for (auto& kv : g_prof) {
        kv.second.launches = 0;
        kv.second.total_ms = 0.0;
    }
    return rc;
}

extern "C" int holo_profile_read(const char* name, uint64_t* launches, double* total_ms) {
    if (!name || !launches || !total_ms) return fail(HOLO_EINVAL, "holo_profile_read: NULL argument");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int rc = collect_locked();
    if (rc != HOLO_OK) return rc;
    auto it = g_prof.find(name);
    *launches = it == g_prof.end() ? 0 : it->second.launches;
    *total_ms = it == g_prof.end() ? 0.0 : it->second.total_ms;
    return HOLO_OK;
}
