// Launch accounting and CUDA-event kernel profiling for every libvie launch.
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr int kProfCap = 1 << 20;

struct Rec {
    int kind, precision;
    int64_t bpu, fixed;
    bool device_units;
    cudaEvent_t e0, e1;
};

struct Profiler {
    std::mutex mu;
    bool enabled = false;
    bool overflow = false;
    int device = -1;
    int* d_units = nullptr;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    int pending = -1;   // index of the record whose end event is still to be placed
};

Profiler& prof() {
    static Profiler p;
    return p;
}

std::atomic<long long> g_launches{0};

const char* kKindNames[PK_COUNT] = {"x_fwd", "y_fwd", "z_green", "y_inv", "x_inv",
                                    "bicg_update", "bicg_dot", "spectrum", "field", "inner_block"};

cudaEvent_t take_event(Profiler& p) {
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

int* prof_begin(cudaStream_t s, int kind, int precision, int64_t bytes_per_unit, int64_t bytes_fixed,
                bool device_units) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    Profiler& p = prof();
    if (!p.enabled) return nullptr;
    std::lock_guard<std::mutex> lock(p.mu);
    if ((int)p.recs.size() >= kProfCap) {
        p.overflow = true;
        return nullptr;
    }
    Rec r;
    r.kind = kind;
    r.precision = precision;
    r.bpu = bytes_per_unit;
    r.fixed = bytes_fixed;
    r.device_units = device_units;
    r.e0 = take_event(p);
    r.e1 = take_event(p);
    cudaEventRecord(r.e0, s);
    p.pending = (int)p.recs.size();
    p.recs.push_back(r);
    return device_units ? p.d_units + p.pending : nullptr;
}

void prof_end(cudaStream_t s) {
    Profiler& p = prof();
    if (!p.enabled) return;
    std::lock_guard<std::mutex> lock(p.mu);
    if (p.pending >= 0) {
        cudaEventRecord(p.recs[p.pending].e1, s);
        p.pending = -1;
    }
}

}  // namespace vie

using namespace vie;

extern "C" int vie_profile_enable(int enable) {
    Profiler& p = prof();
    VIE_CK(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lock(p.mu);
    for (auto& r : p.recs) {
        p.pool.push_back(r.e0);
        p.pool.push_back(r.e1);
    }
    p.recs.clear();
    p.overflow = false;
    p.pending = -1;
    if (enable) {
        int dev = 0;
        VIE_CK(cudaGetDevice(&dev));
        if (p.d_units == nullptr || p.device != dev) {
            VIE_CK(cudaMalloc(&p.d_units, kProfCap * sizeof(int)));
            p.device = dev;
        }
        VIE_CK(cudaMemset(p.d_units, 0, kProfCap * sizeof(int)));
    }
    p.enabled = enable != 0;
    return VIE_OK;
}

extern "C" int vie_profile_read(vie_kernel_stat* out, int cap, int* n_out, int64_t* total_launches) {
    Profiler& p = prof();
    if (total_launches) *total_launches = (int64_t)g_launches.load();
    if (n_out) *n_out = 0;
    std::lock_guard<std::mutex> lock(p.mu);
    if (p.recs.empty()) return VIE_OK;
    VIE_CK(cudaDeviceSynchronize());
    std::vector<int> units(p.recs.size());
    VIE_CK(cudaMemcpy(units.data(), p.d_units, units.size() * sizeof(int), cudaMemcpyDeviceToHost));
    struct Agg { int64_t launches = 0; double ms = 0, bytes = 0; };
    Agg agg[PK_COUNT][3];
    for (size_t i = 0; i < p.recs.size(); ++i) {
        const Rec& r = p.recs[i];
        float ms = 0.f;
        VIE_CK(cudaEventElapsedTime(&ms, r.e0, r.e1));
        int64_t u = r.device_units ? units[i] : 1;
        Agg& a = agg[r.kind][r.precision];
        a.launches++;
        a.ms += ms;
        a.bytes += (double)u * (double)r.bpu + (u > 0 ? (double)r.fixed : 0.0);
    }
    int n = 0;
    for (int k = 0; k < PK_COUNT; ++k)
        for (int pr = 1; pr <= 2; ++pr) {
            if (agg[k][pr].launches == 0) continue;
            if (out && n < cap) {
                memset(&out[n], 0, sizeof(out[n]));
                strncpy(out[n].name, kKindNames[k], sizeof(out[n].name) - 1);
                out[n].precision = pr;
                out[n].launches = agg[k][pr].launches;
                out[n].total_ms = agg[k][pr].ms;
                out[n].bytes = agg[k][pr].bytes;
            }
            ++n;
        }
    if (n_out) *n_out = std::min(n, cap);
    if (p.overflow) return fail(VIE_ENOMEM, "profile capacity exceeded; later launches were not recorded");
    return VIE_OK;
}
