// C ABI of libvie: handle management and the host-side drivers of the
// block-preconditioned BiCGSTAB-FFT solver (Section II.B, Eq. 10).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>

#include "vie_internal.cuh"

namespace vie {

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
std::string last_error_message() { return g_last_error; }

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    std::string m = std::string(what) + " failed: " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) + ")";
    if (e == cudaErrorMemoryAllocation) return fail(VIE_ENOMEM, m);
    return fail(VIE_ECUDA, m);
}

// ---------------------------------------------------------------- twiddles (per device)
static std::mutex g_tw_mutex;
static std::map<int, Twiddles> g_tw;

int get_twiddles(Twiddles* out) {
    int dev = 0;
    VIE_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_tw_mutex);
    auto it = g_tw.find(dev);
    if (it != g_tw.end()) {
        *out = it->second;
        return VIE_OK;
    }
    // W^m = exp(-2 pi i m / Lmax), evaluated in long double and rounded once.
    std::vector<double2> h128(kLmax);
    std::vector<float2> h64(kLmax);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int m = 0; m < kLmax; ++m) {
        long double th = 2.0L * pi * (long double)m / (long double)kLmax;
        long double c = cosl(th), s = -sinl(th);
        h128[m] = make_double2((double)c, (double)s);
        h64[m] = make_float2((float)c, (float)s);
    }
    Twiddles t;
    VIE_CK(cudaMalloc(&t.d128, kLmax * sizeof(double2)));
    VIE_CK(cudaMalloc(&t.d64, kLmax * sizeof(float2)));
    VIE_CK(cudaMemcpy(t.d128, h128.data(), kLmax * sizeof(double2), cudaMemcpyHostToDevice));
    VIE_CK(cudaMemcpy(t.d64, h64.data(), kLmax * sizeof(float2), cudaMemcpyHostToDevice));
    // copies from pageable memory may return before their DMA lands, and later kernels may run on a
    // non-blocking stream that does not wait for the legacy stream: wait for the tables here
    VIE_CK(cudaDeviceSynchronize());
    g_tw[dev] = t;
    *out = t;
    return VIE_OK;
}

// ---------------------------------------------------------------- allocation
// Every device allocation a grid, spectrum or batch holds goes through dmalloc,
// which counts the bytes held by the whole process against an optional budget.
static std::mutex g_alloc_mu;
static std::map<void*, size_t> g_alloc_size;
static int64_t g_alloc_held = 0;
static int64_t g_alloc_budget = 0;        // 0: no budget
static int g_alloc_fault_after = -1;      // test hook: allocations left before an injected failure

int dmalloc(void** p, size_t bytes, const char* what) {
    *p = nullptr;
    if (bytes == 0) return VIE_OK;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    if (g_alloc_budget > 0 && g_alloc_held + (int64_t)bytes > g_alloc_budget)
        return fail(VIE_EBUSY, std::string(what) + ": admission refused: " + std::to_string(bytes) +
                                   " more bytes would exceed the device budget of " + std::to_string(g_alloc_budget) +
                                   " (held " + std::to_string(g_alloc_held) + ")");
    cudaError_t e;
    if (g_alloc_fault_after == 0) {
        g_alloc_fault_after = -1;
        e = cudaErrorMemoryAllocation;          // injected: no device call is made
    } else {
        if (g_alloc_fault_after > 0) --g_alloc_fault_after;
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(VIE_ENOMEM, std::string(what) + ": cudaMalloc of " + std::to_string(bytes) +
                                    " bytes failed: " + cudaGetErrorString(e));
    }
    g_alloc_size[*p] = bytes;
    g_alloc_held += (int64_t)bytes;
    return VIE_OK;
}

void dfree(void* p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        auto it = g_alloc_size.find(p);
        if (it != g_alloc_size.end()) {
            g_alloc_held -= (int64_t)it->second;
            g_alloc_size.erase(it);
        }
    }
    cudaFree(p);
}

template <class T>
static int dalloc(vie_grid* g, T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) return VIE_OK;
    size_t bytes = (size_t)count * sizeof(T);
    VIE_TRY(dmalloc((void**)p, bytes, "vie_grid_create"));
    g->allocations.push_back((void*)*p);
    g->device_bytes += (int64_t)bytes;
    return VIE_OK;
}

static int next_pow2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
static int ilog2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
// Smallest power of two >= 2b - 1: embeds offsets -(b-1) .. b-1 circularly.
static int padded_len(int b) { return next_pow2(2 * b - 1); }

static void set_shape(BoxSet& bs, int bx, int by, int bz) {
    bs.bx = bx; bs.by = by; bs.bz = bz;
    bs.Mx = padded_len(bx); bs.My = padded_len(by); bs.Mz = padded_len(bz);
    bs.lx = ilog2i(bs.Mx); bs.ly = ilog2i(bs.My); bs.lz = ilog2i(bs.Mz);
}

template <class C>
static int alloc_krylov(vie_grid* g, KrylovVecs<C>& k, int64_t n, bool with_bx, bool with_yz) {
    if (with_bx) {
        VIE_TRY(dalloc(g, &k.b, n));
        VIE_TRY(dalloc(g, &k.x, n));
    }
    VIE_TRY(dalloc(g, &k.r, n));
    VIE_TRY(dalloc(g, &k.rhat, n));
    VIE_TRY(dalloc(g, &k.p, n));
    VIE_TRY(dalloc(g, &k.v, n));
    VIE_TRY(dalloc(g, &k.s, n));
    VIE_TRY(dalloc(g, &k.t, n));
    if (with_yz) {
        VIE_TRY(dalloc(g, &k.y, n));
        VIE_TRY(dalloc(g, &k.z, n));
    } else {
        k.y = k.p;   // no preconditioner: y = p, z = s
        k.z = k.s;
    }
    return VIE_OK;
}

static int alloc_reduce(vie_grid* g, ReduceScratch& red, int nseg) {
    red.nseg = nseg;
    VIE_TRY(dalloc(g, &red.part, (int64_t)nseg * kMaxCtaPerSeg * 2));
    VIE_TRY(dalloc(g, &red.count, nseg));
    VIE_TRY(dalloc(g, &red.n_active, 1));
    VIE_CK(cudaMemset(red.count, 0, nseg * sizeof(unsigned)));
    VIE_CK(cudaMemset(red.n_active, 0, sizeof(int)));
    return VIE_OK;
}

static int alloc_fft_work(vie_grid* g, BoxSet& bs) {
    int64_t w1 = (int64_t)bs.nb * 3 * bs.bz * bs.by * bs.Mx;
    int64_t w2 = (int64_t)bs.nb * 3 * bs.bz * bs.My * bs.Mx;
    double2* p1 = nullptr;
    double2* p2 = nullptr;
    VIE_TRY(dalloc(g, &p1, w1));
    VIE_TRY(dalloc(g, &p2, w2));
    bs.w1 = p1;
    bs.w2 = p2;
    return VIE_OK;
}

static int upload_chi(vie_grid* g, BoxSet& bs, const std::vector<double2>& chi) {
    int64_t n = (int64_t)chi.size();
    VIE_TRY(dalloc(g, &bs.chi128, n));
    VIE_TRY(dalloc(g, &bs.chi64, n));
    std::vector<float2> c64(n);
    for (int64_t i = 0; i < n; ++i) c64[i] = make_float2((float)chi[i].x, (float)chi[i].y);
    VIE_CK(cudaMemcpy(bs.chi128, chi.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    VIE_CK(cudaMemcpy(bs.chi64, c64.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    return VIE_OK;
}

static void release_grid(vie_grid* g) {
    for (void* p : g->allocations) dfree(p);
    g->allocations.clear();
    if (g->h_ring) cudaFreeHost(g->h_ring);
    for (int i = 0; i < 2; ++i) {
        if (g->ev[i]) cudaEventDestroy(g->ev[i]);
        if (g->tev[i]) cudaEventDestroy(g->tev[i]);
    }
    if (g->fork_ev) cudaEventDestroy(g->fork_ev);
    if (g->join_ev) cudaEventDestroy(g->join_ev);
    if (g->s2) cudaStreamDestroy(g->s2);
    delete g;
}

// True for memory the device owns (cudaMalloc, torch CUDA tensors); host,
// pinned and managed memory are read in place.
static bool is_device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}

// Bounded host wait for an event (no device-side spin exists in this library;
// the bound protects callers from a device that stopped answering).
static int wait_event(cudaEvent_t ev, double timeout_ms) {
    if (timeout_ms <= 0) timeout_ms = 60000.0;
    auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return VIE_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery", __FILE__, __LINE__);
        if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
        double el = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_ms) return fail(VIE_ETIMEOUT, "device did not finish within the wait bound");
    }
}

}  // namespace vie

using namespace vie;

extern "C" int vie_version(void) { return 100; }

extern "C" int vie_set_device_budget(int64_t bytes) {
    if (bytes < 0) return fail(VIE_EINVAL, "vie_set_device_budget: bytes must be >= 0");
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc_budget = bytes;
    return VIE_OK;
}

extern "C" int vie_device_usage(int64_t* held, int64_t* budget) {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    if (held) *held = g_alloc_held;
    if (budget) *budget = g_alloc_budget;
    return VIE_OK;
}

extern "C" int vie_fault_inject_alloc(int32_t after) {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc_fault_after = after < 0 ? -1 : after;
    return VIE_OK;
}

extern "C" int vie_last_error(char* buf, size_t len) {
    if (buf && len) {
        size_t n = std::min(len - 1, g_last_error.size());
        memcpy(buf, g_last_error.data(), n);
        buf[n] = 0;
    }
    return (int)g_last_error.size();
}

extern "C" int vie_grid_create(const vie_grid_desc* d, vie_grid** out) {
    if (!d || !out) return fail(VIE_EINVAL, "vie_grid_create: null argument");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx > kLmax / 2 || d->ny > kLmax / 2 || d->nz > kLmax / 2)
        return fail(VIE_EINVAL, "vie_grid_create: each of nx, ny, nz must be in [1, 512]");
    if (!(d->h > 0.0) || !std::isfinite(d->h)) return fail(VIE_EINVAL, "vie_grid_create: h must be positive");
    if (!d->eps_r) return fail(VIE_EINVAL, "vie_grid_create: eps_r is null");
    if (d->flags > VIE_GRID_INNER_PERSISTENT) return fail(VIE_EINVAL, "vie_grid_create: unknown flags");
    if (d->block_expand < 0 || d->block_expand > 64)
        return fail(VIE_EINVAL, "vie_grid_create: block_expand must be in [0, 64]");

    vie_grid* g = new vie_grid();
    auto bail = [&](int rc) { release_grid(g); return rc; };
    if (cudaGetDevice(&g->device) != cudaSuccess) return bail(fail(VIE_ECUDA, "no CUDA device"));
    g->nx = d->nx; g->ny = d->ny; g->nz = d->nz; g->h = d->h;
    const int64_t N = (int64_t)d->nx * d->ny * d->nz;
    g->N = N;

    // eps_r and block_id may be host or device memory: device tables are read back once
    std::vector<double> eps_host;
    std::vector<int32_t> bid_host;
    const double* eps = d->eps_r;
    const int32_t* user_bid = d->block_id;
    if (is_device_pointer(eps)) {
        eps_host.resize(2 * N);
        if (cudaMemcpy(eps_host.data(), eps, 2 * N * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(fail(VIE_ECUDA, "vie_grid_create: reading the device eps_r failed"));
        eps = eps_host.data();
    }
    if (user_bid && is_device_pointer(user_bid)) {
        bid_host.resize(N);
        if (cudaMemcpy(bid_host.data(), user_bid, N * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(fail(VIE_ECUDA, "vie_grid_create: reading the device block_id failed"));
        user_bid = bid_host.data();
    }

    // contrast chi = eps_r - 1 (Eq. 2: J = j w eps0 chi E)
    std::vector<double2> chi(N);
    for (int64_t i = 0; i < N; ++i) {
        double re = eps[2 * i], im = eps[2 * i + 1];
        if (!std::isfinite(re) || !std::isfinite(im)) return bail(fail(VIE_EINVAL, "vie_grid_create: non-finite eps_r"));
        chi[i] = make_double2(re - 1.0, im);
    }
    g->full.nb = 1;
    set_shape(g->full, d->nx, d->ny, d->nz);
    g->full.oct = true;                   // the full-grid spectrum is stored octant-compressed
    int rc = upload_chi(g, g->full, chi);
    if (rc) return bail(rc);
    if ((rc = alloc_fft_work(g, g->full))) return bail(rc);

    // blocks of Eq. 10: compact ids in increasing order of the user's ids
    std::vector<int32_t> bid(N, -1);
    std::map<int32_t, int> ids;
    if (user_bid) {
        for (int64_t i = 0; i < N; ++i)
            if (user_bid[i] >= 0) ids.emplace(user_bid[i], 0);
        int k = 0;
        for (auto& kv : ids) kv.second = k++;
        for (int64_t i = 0; i < N; ++i)
            if (user_bid[i] >= 0) bid[i] = ids[user_bid[i]];
    }
    const int K = (int)ids.size();
    g->nblocks = K;
    std::vector<int> lo(3 * K, INT32_MAX), hi(3 * K, -1);
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                int b = bid[((int64_t)z * g->ny + y) * g->nx + x];
                if (b < 0) continue;
                int c[3] = {x, y, z};
                for (int a = 0; a < 3; ++a) {
                    lo[3 * b + a] = std::min(lo[3 * b + a], c[a]);
                    hi[3 * b + a] = std::max(hi[3 * b + a], c[a]);
                }
            }
    // the set each block is solved on: S_k itself, or with block_expand = E > 0 also every voxel with
    // chi != 0 within Chebyshev distance E of S_k (restricted additive Schwarz: only S_k is kept).
    // smask[b] covers the bounding box (slo, sext) of that set: 1 = S_k, 2 = halo, 0 = outside.
    const int E = d->block_expand;
    const int gn[3] = {g->nx, g->ny, g->nz};
    std::vector<std::vector<uint8_t>> smask(K);
    std::vector<int> slo(3 * K), sext(3 * K);
    for (int b = 0; b < K; ++b) {
        int elo[3], eext[3];
        for (int a = 0; a < 3; ++a) {
            elo[a] = std::max(0, lo[3 * b + a] - E);
            eext[a] = std::min(gn[a] - 1, hi[3 * b + a] + E) - elo[a] + 1;
        }
        const int64_t ev = (int64_t)eext[0] * eext[1] * eext[2];
        std::vector<uint8_t> own(ev, 0), dil;
        auto at = [&](int x, int y, int z) { return ((int64_t)z * eext[1] + y) * eext[0] + x; };
        for (int z = 0; z < eext[2]; ++z)
            for (int y = 0; y < eext[1]; ++y)
                for (int x = 0; x < eext[0]; ++x)
                    own[at(x, y, z)] = bid[((int64_t)(z + elo[2]) * g->ny + y + elo[1]) * g->nx + x + elo[0]] == b;
        dil = own;
        for (int a = 0; a < 3 && E > 0; ++a) {          // separable dilation by a (2E+1)^3 cube
            std::vector<uint8_t> nx_ = dil;
            for (int z = 0; z < eext[2]; ++z)
                for (int y = 0; y < eext[1]; ++y)
                    for (int x = 0; x < eext[0]; ++x) {
                        int c[3] = {x, y, z};
                        uint8_t m = 0;
                        for (int dd = -E; dd <= E && !m; ++dd) {
                            int q[3] = {c[0], c[1], c[2]};
                            q[a] += dd;
                            if (q[a] >= 0 && q[a] < eext[a]) m = dil[at(q[0], q[1], q[2])];
                        }
                        nx_[at(x, y, z)] = m;
                    }
            dil.swap(nx_);
        }
        int blo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, bhi[3] = {-1, -1, -1};
        std::vector<uint8_t> m(ev, 0);
        for (int z = 0; z < eext[2]; ++z)
            for (int y = 0; y < eext[1]; ++y)
                for (int x = 0; x < eext[0]; ++x) {
                    const int64_t gv = ((int64_t)(z + elo[2]) * g->ny + y + elo[1]) * g->nx + x + elo[0];
                    const bool nonair = chi[gv].x != 0.0 || chi[gv].y != 0.0;
                    const uint8_t v = own[at(x, y, z)] ? 1 : ((dil[at(x, y, z)] && nonair) ? 2 : 0);
                    m[at(x, y, z)] = v;
                    if (v) {
                        int c[3] = {x, y, z};
                        for (int a = 0; a < 3; ++a) {
                            blo[a] = std::min(blo[a], c[a]);
                            bhi[a] = std::max(bhi[a], c[a]);
                        }
                    }
                }
        for (int a = 0; a < 3; ++a) {
            slo[3 * b + a] = elo[a] + blo[a];
            sext[3 * b + a] = bhi[a] - blo[a] + 1;
        }
        std::vector<uint8_t>& sm = smask[b];
        sm.assign((int64_t)sext[3 * b] * sext[3 * b + 1] * sext[3 * b + 2], 0);
        for (int z = 0; z < sext[3 * b + 2]; ++z)
            for (int y = 0; y < sext[3 * b + 1]; ++y)
                for (int x = 0; x < sext[3 * b]; ++x)
                    sm[((int64_t)z * sext[3 * b + 1] + y) * sext[3 * b] + x] = m[at(x + blo[0], y + blo[1], z + blo[2])];
    }
    // group blocks by padded FFT shape of the bounding boxes of their sets
    std::map<std::tuple<int, int, int>, std::vector<int>> bykey;
    for (int b = 0; b < K; ++b)
        bykey[std::make_tuple(padded_len(sext[3 * b + 2]), padded_len(sext[3 * b + 1]), padded_len(sext[3 * b]))]
            .push_back(b);
    std::vector<int32_t> h_group(K), h_index(K), h_origin(3 * K);
    g->groups.resize(bykey.size());
    int gi = 0;
    for (auto& kv : bykey) {
        Group& gr = g->groups[gi];
        const std::vector<int>& mem = kv.second;
        int mx = 1, my = 1, mz = 1;
        for (int b : mem) {
            mx = std::max(mx, sext[3 * b]);
            my = std::max(my, sext[3 * b + 1]);
            mz = std::max(mz, sext[3 * b + 2]);
        }
        gr.bs.nb = (int)mem.size();
        set_shape(gr.bs, mx, my, mz);
        gr.bs.block_ids = mem;
        const int64_t box = gr.bs.box_elems();
        std::vector<double2> gchi(gr.bs.nb * box, make_double2(0, 0));
        std::vector<uint8_t> gmask(gr.bs.nb * box, 0);
        std::vector<int32_t> gorig(3 * gr.bs.nb);
        for (int j = 0; j < gr.bs.nb; ++j) {
            int b = mem[j];
            h_group[b] = gi;
            h_index[b] = j;
            for (int a = 0; a < 3; ++a) gorig[3 * j + a] = h_origin[3 * b + a] = slo[3 * b + a];
            const int ex = sext[3 * b], ey = sext[3 * b + 1], ez = sext[3 * b + 2];
            for (int lz = 0; lz < ez; ++lz)
                for (int ly = 0; ly < ey; ++ly)
                    for (int lx = 0; lx < ex; ++lx) {
                        const uint8_t v = smask[b][((int64_t)lz * ey + ly) * ex + lx];
                        if (!v) continue;
                        int x = slo[3 * b] + lx, y = slo[3 * b + 1] + ly, z = slo[3 * b + 2] + lz;
                        int64_t gv = ((int64_t)z * g->ny + y) * g->nx + x;
                        int64_t l = (int64_t)j * box + ((int64_t)lz * my + ly) * mx + lx;
                        gmask[l] = v;
                        gchi[l] = chi[gv];
                    }
        }
        if ((rc = upload_chi(g, gr.bs, gchi))) return bail(rc);
        if ((rc = dalloc(g, &gr.bs.mask, gr.bs.nb * box))) return bail(rc);
        if ((rc = dalloc(g, &gr.bs.origin, 3 * gr.bs.nb))) return bail(rc);
        if (cudaMemcpy(gr.bs.mask, gmask.data(), gmask.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(gr.bs.origin, gorig.data(), gorig.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(VIE_ECUDA, "upload of block tables failed"));
        if ((rc = alloc_fft_work(g, gr.bs))) return bail(rc);
        const int64_t nv = gr.bs.nb * gr.bs.vec_elems();
        if ((rc = alloc_krylov(g, gr.k128, nv, true, false))) return bail(rc);
        if ((rc = alloc_krylov(g, gr.k64, nv, true, false))) return bail(rc);
        if ((rc = dalloc(g, &gr.st, gr.bs.nb))) return bail(rc);
        if ((rc = alloc_reduce(g, gr.red, gr.bs.nb))) return bail(rc);
        ++gi;
    }
    // persistent block solver: eligible groups and their work lists, largest boxes first
    for (int prec = 0; prec < 2; ++prec) {
        const size_t es = prec == 0 ? 16 : 8;
        std::vector<std::pair<int64_t, int2>> items;
        int job = 0;
        // AUTO: every group whose plane fits joins one persistent launch when the
        // fitting groups hold at least kInnerMinBlocks blocks in total (fewer, larger
        // blocks iterate faster in the batched launches, which use the whole GPU per step)
        int fit_blocks = 0;
        for (auto& gr : g->groups)
            if (inner_persistent_ok(gr.bs, es, true)) fit_blocks += gr.bs.nb;
        const bool force = d->flags == VIE_GRID_INNER_PERSISTENT || fit_blocks >= kInnerMinBlocks;
        for (auto& gr : g->groups) {
            // merged launches across grids take the blocks the persistent solver would take here, and
            // complex64 blocks of the on-chip slab MVM (a few such blocks of one grid iterate faster in
            // the batched launches, which spread each block over the whole GPU, but many of them, from
            // several grids, fill the GPU in one launch; larger boxes stay batched)
            gr.fit[prec] = d->flags != VIE_GRID_INNER_BATCHED && inner_persistent_ok(gr.bs, es, true) &&
                           (force || (prec == 1 && slab_path_ok(gr.bs, es) && !slab_disabled()));
            gr.last_iters[prec].assign(gr.bs.nb, 0.f);
            bool ok = d->flags != VIE_GRID_INNER_BATCHED && inner_persistent_ok(gr.bs, es, force);
            (prec == 0 ? gr.persistent128 : gr.persistent64) = ok;
            if (!ok) continue;
            for (int b = 0; b < gr.bs.nb; ++b) items.push_back({gr.bs.spec_elems(), make_int2(job, b)});
            g->job_group[prec].push_back((int)(&gr - g->groups.data()));
            ++job;
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const std::pair<int64_t, int2>& a, const std::pair<int64_t, int2>& b) { return a.first > b.first; });
        std::vector<int2> w;
        for (auto& it : items) w.push_back(it.second);
        g->work_host[prec] = w;
        int2** dst = prec == 0 ? &g->work128 : &g->work64;
        (prec == 0 ? g->nwork128 : g->nwork64) = (int)w.size();
        if (!w.empty()) {
            if ((rc = dalloc(g, dst, (int64_t)w.size()))) return bail(rc);
            if (cudaMemcpy(*dst, w.data(), w.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(VIE_ECUDA, "upload of the block work list failed"));
        }
    }
    if (!g->groups.empty()) {
        char* descs = nullptr;
        if ((rc = dalloc(g, &descs, (int64_t)(g->groups.size() * inner_group_desc_bytes())))) return bail(rc);
        g->inner_groups = descs;
        if ((rc = dalloc(g, &g->inner_next, 2))) return bail(rc);
    }
    if ((rc = dalloc(g, &g->block_id, N))) return bail(rc);
    if (cudaMemcpy(g->block_id, bid.data(), N * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(VIE_ECUDA, "upload of block ids failed"));

    // outer Krylov workspace (b and x are the caller's vectors in a solve)
    const int64_t n3 = 3 * N;
    if ((rc = alloc_krylov(g, g->o128, n3, false, true))) return bail(rc);
    if ((rc = alloc_krylov(g, g->o64, n3, true, true))) return bail(rc);
    if ((rc = dalloc(g, &g->tmp128, n3))) return bail(rc);
    if ((rc = dalloc(g, &g->ost, 1))) return bail(rc);
    if ((rc = alloc_reduce(g, g->ored, 1))) return bail(rc);
    if ((rc = dalloc(g, &g->dscal, 8))) return bail(rc);
    size_t ring = 2 * (g->groups.size() + 1) * sizeof(int) + sizeof(SegState) + 8 * sizeof(double);
    if (cudaHostAlloc((void**)&g->h_ring, ring, cudaHostAllocDefault) != cudaSuccess)
        return bail(fail(VIE_ENOMEM, "pinned host allocation failed"));
    for (int i = 0; i < 2; ++i)
        if (cudaEventCreateWithFlags(&g->ev[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&g->tev[i]) != cudaSuccess)
            return bail(fail(VIE_ECUDA, "cudaEventCreate failed"));
    if (cudaStreamCreateWithFlags(&g->s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->join_ev, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(VIE_ECUDA, "stream or event creation failed"));
    *out = g;
    return VIE_OK;
}

extern "C" int vie_grid_destroy(vie_grid* g) {
    if (!g) return fail(VIE_EINVAL, "vie_grid_destroy: null grid");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    release_grid(g);
    cudaSetDevice(prev);
    return VIE_OK;
}

extern "C" int vie_grid_get_info(const vie_grid* g, vie_grid_info* info) {
    if (!g || !info) return fail(VIE_EINVAL, "vie_grid_get_info: null argument");
    info->nblocks = g->nblocks;
    info->ngroups = (int32_t)g->groups.size();
    info->Mx = g->full.Mx;
    info->My = g->full.My;
    info->Mz = g->full.Mz;
    info->device_bytes = g->device_bytes;
    info->inner_cluster[0] = g->tune_best[0];
    info->inner_cluster[1] = g->tune_best[1];
    return VIE_OK;
}

// ---------------------------------------------------------------- spectra
namespace vie {
static std::vector<int> shape_signature(const vie_grid* g);
}

static int green_spectrum(vie_grid* g, double k0, int mask, const NearRule& near, cudaStream_t stream,
                          vie_spectrum** out);

extern "C" int vie_green_spectrum(vie_grid* g, double k0, int mask, vie_stream_t stream, vie_spectrum** out) {
    return green_spectrum(g, k0, mask, NearRule(), (cudaStream_t)stream, out);
}

extern "C" int vie_green_spectrum_near(vie_grid* g, double k0, int mask, int32_t near_radius, int32_t near_order,
                                       vie_stream_t stream, vie_spectrum** out) {
    NearRule near;
    VIE_TRY(near_rule(near_radius, near_order, &near));
    return green_spectrum(g, k0, mask, near, (cudaStream_t)stream, out);
}

static int green_spectrum(vie_grid* g, double k0, int mask, const NearRule& near, cudaStream_t stream,
                          vie_spectrum** out) {
    if (!g || !out) return fail(VIE_EINVAL, "vie_green_spectrum: null argument");
    *out = nullptr;
    if (!(k0 > 0.0) || !std::isfinite(k0)) return fail(VIE_EINVAL, "vie_green_spectrum: k0 must be positive");
    if (mask == 0 || (mask & ~(VIE_C128 | VIE_C64))) return fail(VIE_EINVAL, "vie_green_spectrum: bad precision mask");
    cudaStream_t s = (cudaStream_t)stream;
    vie_spectrum* sp = new vie_spectrum();
    sp->grid = g;
    sp->h = g->h;
    sp->shape_sig = shape_signature(g);
    sp->k0 = k0;
    sp->precision_mask = mask;
    auto bail = [&](int rc) {
        cudaStreamSynchronize(s);         // kernels already queued may still use the spectra
        for (auto p : sp->g128) dfree(p);
        for (auto p : sp->g64) dfree(p);
        for (auto p : sp->go64) dfree(p);
        delete sp;
        return rc;
    };
    std::vector<const BoxSet*> sets;
    sets.push_back(&g->full);
    for (auto& gr : g->groups) sets.push_back(&gr.bs);
    {
        // full grid: octant-compressed spectra, built from an FP64 temporary
        const int64_t n = 6 * g->full.oct_elems();
        double2* G = nullptr;
        float2* G64 = nullptr;
        int arc = VIE_OK;
        if (mask & VIE_C128) arc = dmalloc((void**)&G, n * sizeof(double2), "vie_green_spectrum");
        if (!arc && (mask & VIE_C64)) arc = dmalloc((void**)&G64, n * sizeof(float2), "vie_green_spectrum");
        if (arc) {
            dfree(G);
            return bail(arc);
        }
        sp->g128.push_back(G);
        sp->g64.push_back(G64);
        sp->go64.push_back(nullptr);
        int rc = spectrum_build(g->full, k0, g->h, G, G64, nullptr, s, &near);
        if (rc) return bail(rc);
    }
    sets.erase(sets.begin());
    for (const BoxSet* bs : sets) {
        const int64_t n = 6 * bs->spec_elems();
        double2* G = nullptr;
        int arc = dmalloc((void**)&G, n * sizeof(double2), "vie_green_spectrum");
        if (arc) return bail(arc);
        sp->g128.push_back(G);
        int rc = green_sample(*bs, k0, g->h, G, s, &near);
        if (!rc) rc = spectrum_fft<double2>(*bs, G, s);
        if (rc) return bail(rc);
        float2* G64 = nullptr;
        if (mask & VIE_C64) {
            if ((arc = dmalloc((void**)&G64, n * sizeof(float2), "vie_green_spectrum"))) return bail(arc);
            if ((rc = convert_c128_to_c64(G, G64, n, s))) {
                sp->g64.push_back(G64);
                return bail(rc);
            }
        }
        sp->g64.push_back(G64);
        // the slab MVM of the block solver reads an octant of the spectrum in natural order
        float2* Go = nullptr;
        if ((mask & VIE_C64) && slab_path_ok(*bs, sizeof(float2))) {
            if ((arc = dmalloc((void**)&Go, 6 * bs->oct_elems() * sizeof(float2), "vie_green_spectrum")))
                return bail(arc);
            sp->go64.push_back(Go);
            if ((rc = slab_spectrum(*bs, G, Go, s))) return bail(rc);
        } else {
            sp->go64.push_back(nullptr);
        }
    }
    if (!(mask & VIE_C128)) {
        // the FP64 spectrum was only the source of the complex64 copy
        if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(VIE_ECUDA, "spectrum generation failed"));
        for (auto& p : sp->g128) {
            dfree(p);
            p = nullptr;
        }
    }
    *out = sp;
    return VIE_OK;
}

extern "C" int vie_spectrum_release(vie_spectrum* sp) {
    if (!sp) return fail(VIE_EINVAL, "vie_spectrum_release: null spectrum");
    cudaDeviceSynchronize();
    for (auto p : sp->g128) dfree(p);
    for (auto p : sp->g64) dfree(p);
    for (auto p : sp->go64) dfree(p);
    delete sp;
    return VIE_OK;
}

namespace vie {

template <class C> static const C* spec_of(const vie_spectrum* sp, int idx);
template <> const double2* spec_of<double2>(const vie_spectrum* sp, int idx) { return sp->g128[idx]; }
template <> const float2* spec_of<float2>(const vie_spectrum* sp, int idx) { return sp->g64[idx]; }
template <class C> static KrylovVecs<C>& group_vecs(Group& gr);
template <> KrylovVecs<double2>& group_vecs<double2>(Group& gr) { return gr.k128; }
template <> KrylovVecs<float2>& group_vecs<float2>(Group& gr) { return gr.k64; }
template <class C> static const C* chi_of(const BoxSet& bs);
template <> const double2* chi_of<double2>(const BoxSet& bs) { return bs.chi128; }
template <> const float2* chi_of<float2>(const BoxSet& bs) { return bs.chi64; }
template <class C> static int prec_of();
template <> int prec_of<double2>() { return VIE_C128; }
template <> int prec_of<float2>() { return VIE_C64; }

// A spectrum depends only on h, the padded shapes and the box extents of the
// grid and of its block groups, so it serves every grid that matches them.
static std::vector<int> shape_signature(const vie_grid* g) {
    std::vector<int> v;
    auto add = [&](const BoxSet& x) {
        int a[6] = {x.bx, x.by, x.bz, x.Mx, x.My, x.Mz};
        v.insert(v.end(), a, a + 6);
    };
    add(g->full);
    for (const auto& gr : g->groups) add(gr.bs);
    return v;
}

static bool spectrum_compatible(const vie_spectrum* sp, const vie_grid* g) {
    // compared by value: the address of a destroyed grid may be reused by a new one
    return sp->h == g->h && sp->shape_sig == shape_signature(g);
}

static int check_spectrum(const vie_grid* g, const vie_spectrum* sp, int precision) {
    if (!sp || !spectrum_compatible(sp, g))
        return fail(VIE_EINVAL, "spectrum was made for a grid of another shape, block layout or voxel size");
    if (precision != VIE_C128 && precision != VIE_C64) return fail(VIE_EINVAL, "precision must be VIE_C128 or VIE_C64");
    if (!(sp->precision_mask & precision)) return fail(VIE_EINVAL, "spectrum was not generated in this precision");
    return VIE_OK;
}

static bool overlaps(const void* a, const void* b, int64_t bytes) {
    const char* pa = (const char*)a;
    const char* pb = (const char*)b;
    return pa < pb + bytes && pb < pa + bytes;
}

template <class C>
static int mvm_full(vie_grid* g, const vie_spectrum* sp, const C* x, C* y, cudaStream_t s) {
    return mvm_boxes<C>(g->full, spec_of<C>(sp, 0), x, y, nullptr, s);
}

// ---------------------------------------------------------------- merged block-solver launches
// (vie_internal.cuh describes the session.) Members build their jobs and work items and arrive;
// the last member to arrive queues the launches on the session's stream.
static int merge_capacity(MergeCtx* mc, int64_t ngroups, int64_t nwork) {
    if (ngroups > mc->groups_cap) {
        char* p = nullptr;
        const int64_t cap = std::max<int64_t>(ngroups, 2 * mc->groups_cap);
        VIE_TRY(dmalloc((void**)&p, cap * inner_group_desc_bytes(), "merged block-solver launch"));
        if (mc->d_groups) mc->retired.push_back(mc->d_groups);
        mc->d_groups = p;
        mc->groups_cap = cap;
    }
    if (nwork > mc->work_cap) {
        int2* p = nullptr;
        const int64_t cap = std::max<int64_t>(nwork, 2 * mc->work_cap);
        VIE_TRY(dmalloc((void**)&p, cap * sizeof(int2), "merged block-solver launch"));
        if (mc->d_work) mc->retired.push_back(mc->d_work);
        mc->d_work = p;
        mc->work_cap = cap;
    }
    if (!mc->d_next) VIE_TRY(dmalloc((void**)&mc->d_next, 2 * sizeof(int), "merged block-solver launch"));
    return VIE_OK;
}

template <class C> static std::vector<InnerJob<C>>& req_jobs(MergeReq* r);
template <> std::vector<InnerJob<double2>>& req_jobs<double2>(MergeReq* r) { return r->j128; }
template <> std::vector<InnerJob<float2>>& req_jobs<float2>(MergeReq* r) { return r->j64; }

// One launch over the jobs of every request (same precision, tolerance and limit), the work
// items of all of them longest first.
template <class C>
static int merged_launch(MergeCtx* mc, const std::vector<MergeReq*>& reqs) {
    std::vector<InnerJob<C>> jobs;
    std::vector<std::pair<double, int2>> items;
    for (MergeReq* r : reqs) {
        const int off = (int)jobs.size();
        const std::vector<InnerJob<C>>& rj = req_jobs<C>(r);
        jobs.insert(jobs.end(), rj.begin(), rj.end());
        for (const auto& it : r->items) items.push_back({it.first, make_int2(it.second.x + off, it.second.y)});
    }
    if (jobs.empty() || items.empty()) return VIE_OK;
    VIE_TRY(merge_capacity(mc, (int64_t)jobs.size(), (int64_t)items.size()));
    std::stable_sort(items.begin(), items.end(), [](const std::pair<double, int2>& a, const std::pair<double, int2>& b) {
        return a.first > b.first;
    });
    std::vector<int2> w(items.size());
    for (size_t k = 0; k < items.size(); ++k) w[k] = items[k].second;
    VIE_CK(cudaMemcpyAsync(mc->d_work, w.data(), w.size() * sizeof(int2), cudaMemcpyHostToDevice, mc->ms));
    return inner_persistent<C>(jobs, mc->d_work, (int)w.size(), mc->d_groups, mc->d_next, reqs[0]->tol,
                               reqs[0]->maxit, mc->ms, 2, nullptr);
}

// Called with mc->m held: one launch per (precision, tolerance, limit) over every pending request.
static void merge_flush(MergeCtx* mc) {
    std::vector<MergeReq*> reqs;
    reqs.swap(mc->pending);
    std::stable_sort(reqs.begin(), reqs.end(), [](const MergeReq* a, const MergeReq* b) {
        return std::tie(a->prec, a->tol, a->maxit) < std::tie(b->prec, b->tol, b->maxit);
    });
    for (size_t i = 0; i < reqs.size();) {
        size_t j = i;
        while (j < reqs.size() && reqs[j]->prec == reqs[i]->prec && reqs[j]->tol == reqs[i]->tol &&
               reqs[j]->maxit == reqs[i]->maxit)
            ++j;
        std::vector<MergeReq*> part(reqs.begin() + i, reqs.begin() + j);
        int rc = VIE_OK;
        for (MergeReq* r : part) {
            cudaError_t e = cudaStreamWaitEvent(mc->ms, r->ready, 0);
            if (e != cudaSuccess && !rc) rc = cuda_fail(e, "cudaStreamWaitEvent(merge)", __FILE__, __LINE__);
        }
        if (!rc) rc = part[0]->prec == 0 ? merged_launch<double2>(mc, part) : merged_launch<float2>(mc, part);
        cudaEvent_t ev = nullptr;
        if (!rc) {
            cudaError_t e = cudaSuccess;
            if (!mc->free_events.empty()) {
                ev = mc->free_events.back();
                mc->free_events.pop_back();
            } else {
                e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            }
            if (e == cudaSuccess) e = cudaEventRecord(ev, mc->ms);
            if (e != cudaSuccess) rc = cuda_fail(e, "merge event", __FILE__, __LINE__);
        }
        if (rc) {
            if (mc->err.empty()) mc->err = g_last_error;
            if (ev) mc->free_events.push_back(ev);
            for (MergeReq* r : part) r->gen = -2;
        } else {
            const int64_t gen = mc->next_gen++;
            mc->launches_open[gen] = MergeLaunch{ev, (int)part.size()};
            for (MergeReq* r : part) r->gen = gen;
            mc->launches++;
            mc->members += (int64_t)part.size();
            mc->max_members = std::max(mc->max_members, (int)part.size());
        }
        i = j;
    }
    mc->cv.notify_all();
}

void merge_join(MergeMember* mm) {
    MergeCtx* mc = mm->ctx;
    std::lock_guard<std::mutex> lock(mc->m);
    mc->live++;
    mm->live = true;
}

void merge_arrive(MergeMember* mm, MergeReq* r) {
    MergeCtx* mc = mm->ctx;
    std::lock_guard<std::mutex> lock(mc->m);
    mc->pending.push_back(r);
    if ((int)mc->pending.size() >= mc->live) merge_flush(mc);
}

// Waits (on the host) until the launch holding r is queued; the member's stream then waits for it.
int merge_wait(MergeMember* mm, MergeReq* r, cudaStream_t s) {
    MergeCtx* mc = mm->ctx;
    std::unique_lock<std::mutex> lock(mc->m);
    mc->cv.wait(lock, [&] { return r->gen != -1; });
    if (r->gen == -2) return fail(VIE_ECUDA, "merged block-solver launch failed: " + mc->err);
    auto it = mc->launches_open.find(r->gen);
    cudaError_t e = cudaStreamWaitEvent(s, it->second.done, 0);
    if (--it->second.waiting == 0) {       // the event may be recorded again by a later launch
        mc->free_events.push_back(it->second.done);
        mc->launches_open.erase(it);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent(merged launch)", __FILE__, __LINE__);
    return VIE_OK;
}

void merge_leave(MergeMember* mm) {
    if (!mm || !mm->live) return;
    MergeCtx* mc = mm->ctx;
    std::lock_guard<std::mutex> lock(mc->m);
    mm->live = false;
    mc->live--;
    if (!mc->pending.empty() && (int)mc->pending.size() >= mc->live) merge_flush(mc);
}

// The grid's jobs and work items for a merged launch: every group that fits, each block costed by
// its iterations in its last application x its padded box.
template <class C>
static void grid_merge_jobs(vie_grid* g, const vie_spectrum* sp, MergeReq* r) {
    const int pi = prec_of<C>() == VIE_C128 ? 0 : 1;
    std::vector<InnerJob<C>>& jobs = req_jobs<C>(r);
    jobs.clear();
    r->items.clear();
    for (size_t i = 0; i < g->groups.size(); ++i) {
        Group& gr = g->groups[i];
        if (!gr.fit[pi]) continue;
        InnerJob<C> j;
        j.bs = &gr.bs;
        j.v = group_vecs<C>(gr);
        j.chi = chi_of<C>(gr.bs);
        j.G = spec_of<C>(sp, 1 + (int)i);
        j.st = gr.st;
        if (pi == 1 && !slab_disabled()) j.Go = reinterpret_cast<const C*>(sp->go64[1 + i]);
        const int job = (int)jobs.size();
        jobs.push_back(j);
        for (int b = 0; b < gr.bs.nb; ++b)
            r->items.push_back({(gr.last_iters[pi][b] + 1.0) * (double)gr.bs.spec_elems(), make_int2(job, b)});
    }
}

// y = K2^{-1} b: all blocks of all groups iterate together; a block stops
// when its own residual meets tol (or at maxit) and is skipped thereafter.
template <class C>
static int precond_apply(vie_grid* g, const vie_spectrum* sp, const C* b, C* y, double tol, int maxit,
                         cudaStream_t s, vie_precond_stats* stats, double timeout_ms,
                         MergeMember* mm = nullptr) {
    const int64_t n3 = 3 * g->N;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (g->nblocks == 0) return vec_copy<C>(b, y, n3, s);
    const int ng = (int)g->groups.size();
    const bool c128 = prec_of<C>() == VIE_C128;
    std::vector<InnerJob<C>> jobs;
    std::vector<int> batched;
    const bool merged = mm != nullptr && mm->live;
    bool any_fit = false;
    for (int i = 0; i < ng; ++i) {
        Group& gr = g->groups[i];
        KrylovVecs<C>& v = group_vecs<C>(gr);
        VIE_TRY(precond_gather<C>(g, gr, b, v.b, s));
        if (merged) {
            // blocks that fit the persistent solver go to the merged launch, the rest run here
            if (gr.fit[c128 ? 0 : 1]) any_fit = true;
            else batched.push_back(i);
        } else if (c128 ? gr.persistent128 : gr.persistent64) {
            InnerJob<C> j;
            j.bs = &gr.bs;
            j.v = v;
            j.chi = chi_of<C>(gr.bs);
            j.G = spec_of<C>(sp, 1 + i);
            j.st = gr.st;
            if (!c128 && !slab_disabled()) j.Go = reinterpret_cast<const C*>(sp->go64[1 + i]);
            jobs.push_back(j);
        } else {
            batched.push_back(i);
        }
    }
    // after arriving, the request is waited for on every path out of this function
    if (merged && !any_fit) merge_leave(mm);   // nothing of this grid fits: do not hold the others
    MergeReq req;
    struct Guard {
        MergeMember* mm;
        MergeReq* r;
        cudaStream_t s;
        bool armed = false;
        ~Guard() {
            if (armed) merge_wait(mm, r, s);
        }
    } guard{mm, &req, s};
    if (merged && any_fit) {
        VIE_CK(cudaEventRecord(g->fork_ev, s));
        grid_merge_jobs<C>(g, sp, &req);
        req.prec = c128 ? 0 : 1;
        req.tol = tol;
        req.maxit = maxit;
        req.ready = g->fork_ev;
        merge_arrive(mm, &req);
        guard.armed = true;
    }
    bool slab = false;
    for (const InnerJob<C>& j : jobs) slab = slab || j.Go != nullptr;
    // launch shape and MVM variant, tuned on the first applies, then the best. Register-FFT MVM: 2 and
    // 4 CTAs per block, then the split launch (the slowest blocks of the previous apply on 4 CTAs, the
    // rest on 2). Blocks the slab MVM takes (whole MVM on chip, the cluster splits the kz planes): 2, 1
    // and 4 CTAs with 4 planes per round where they fit, 2 CTAs with 2 planes per round (a split cannot
    // shorten the slowest block's solve, which bounds the apply once every block fits on the device at
    // once), and the register-FFT MVM with 2 CTAs instead of the slab MVM.
    // candidates (CTAs per block, kz planes per round of the slab MVM's plane stage with 0 = as many as
    // fit, slab MVM or register MVM)
    struct Cand {
        int cluster, npl;
        bool slab;
    };
    static const Cand kCand[3] = {{2, 0, false}, {4, 0, false}, {-1, 0, false}};
    static const Cand kCandSlab[5] = {{2, 4, true}, {1, 4, true}, {4, 4, true}, {2, 2, true}, {2, 0, false}};
    const int ncand = slab ? 5 : 3;
    const int pi = c128 ? 0 : 1;
    // the first apply only warms up (first launches of the kernel pay one-time costs that would bias
    // the candidate tried first); the candidates follow, one per apply
    const int tried = g->tune_count[pi] - 1;
    const bool tuning = !jobs.empty() && tried < ncand && !inner_cluster_forced();
    const Cand cand = tuning ? (slab ? kCandSlab : kCand)[std::max(tried, 0)]
                             : Cand{g->tune_best[pi] ? g->tune_best[pi] : 2, g->tune_npl[pi], !g->tune_noslab[pi]};
    const int choice = cand.cluster;
    if (slab && !cand.slab)
        for (InnerJob<C>& j : jobs) j.Go = nullptr;   // the register-FFT MVM for these blocks
    // with batched groups as well, the persistent launch runs on the grid's second stream beside
    // the batched steps (no split launch then)
    const bool beside = !jobs.empty() && !batched.empty();
    InnerSplit split;
    split.nheavy = choice == -1 && !beside ? g->nheavy[pi] : 0;
    split.cluster = slab ? 2 : 4;
    split.s2 = g->s2;
    split.fork = g->fork_ev;
    split.join = g->join_ev;
    cudaStream_t sp_stream = s;
    if (beside) {
        VIE_CK(cudaEventRecord(g->fork_ev, s));
        VIE_CK(cudaStreamWaitEvent(g->s2, g->fork_ev, 0));
        sp_stream = g->s2;
    }
    if (tuning) VIE_CK(cudaEventRecord(g->tev[0], sp_stream));
    VIE_TRY(inner_persistent<C>(jobs, c128 ? g->work128 : g->work64, c128 ? g->nwork128 : g->nwork64,
                                g->inner_groups, g->inner_next, tol, maxit, sp_stream,
                                choice == -1 ? (slab ? 1 : 2) : choice, &split, cand.npl));
    if (tuning) VIE_CK(cudaEventRecord(g->tev[1], sp_stream));
    std::vector<Bicg<C>> bk(ng);
    for (int i : batched) {
        Group& gr = g->groups[i];
        KrylovVecs<C>& v = group_vecs<C>(gr);
        bk[i].nseg = gr.bs.nb;
        bk[i].seglen = gr.bs.vec_elems();
        bk[i].v = v;
        bk[i].st = gr.st;
        bk[i].red = &gr.red;
        VIE_TRY(bicg_init<C>(bk[i], tol, maxit, s));
    }
    int* ring = (int*)g->h_ring;
    for (int it = 0; it < maxit && !batched.empty(); ++it) {
        const int slot = it & 1;
        for (int i : batched) {
            Group& gr = g->groups[i];
            Bicg<C>& k = bk[i];
            const C* G = spec_of<C>(sp, 1 + i);
            VIE_TRY(bicg_rho<C>(k, s));
            VIE_TRY(bicg_update_p<C>(k, s));
            VIE_TRY(mvm_boxes<C>(gr.bs, G, k.v.p, k.v.v, gr.st, s));
            VIE_TRY(bicg_sigma<C>(k, s));
            VIE_TRY(bicg_update_s<C>(k, s));
            VIE_TRY(bicg_x_half<C>(k, s));
            VIE_TRY(mvm_boxes<C>(gr.bs, G, k.v.s, k.v.t, gr.st, s));
            VIE_TRY(bicg_omega<C>(k, s));
            VIE_TRY(bicg_update_xr<C>(k, s));
            VIE_CK(cudaMemcpyAsync(ring + slot * (ng + 1) + i, gr.red.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
        }
        VIE_CK(cudaEventRecord(g->ev[slot], s));
        if (it > 0) {
            // one iteration stays in flight while the previous one's counts are read
            const int prev = slot ^ 1;
            VIE_TRY(wait_event(g->ev[prev], timeout_ms));
            int active = 0;
            for (int i : batched) active += ring[prev * (ng + 1) + i];
            if (active == 0) break;
        }
    }
    if (beside) {
        VIE_CK(cudaEventRecord(g->join_ev, g->s2));
        VIE_CK(cudaStreamWaitEvent(s, g->join_ev, 0));
    }
    if (guard.armed) {
        guard.armed = false;
        VIE_TRY(merge_wait(mm, &req, s));
    }
    VIE_TRY(precond_copy_unblocked<C>(g, b, y, s));
    for (int i = 0; i < ng; ++i) VIE_TRY(precond_scatter_group<C>(g, g->groups[i], group_vecs<C>(g->groups[i]).x, y, s));
    std::vector<int2>& wh = g->work_host[c128 ? 0 : 1];
    const bool reorder = !jobs.empty() && wh.size() > 1;
    if (stats || reorder || merged) {
        std::vector<std::vector<SegState>> hs(ng);
        for (int i = 0; i < ng; ++i) {
            Group& gr = g->groups[i];
            hs[i].resize(gr.bs.nb);
            VIE_CK(cudaMemcpyAsync(hs[i].data(), gr.st, gr.bs.nb * sizeof(SegState), cudaMemcpyDeviceToHost, s));
        }
        VIE_CK(cudaEventRecord(g->ev[0], s));
        VIE_TRY(wait_event(g->ev[0], timeout_ms));
        for (int i = 0; i < ng; ++i)
            for (int k = 0; k < g->groups[i].bs.nb; ++k) g->groups[i].last_iters[c128 ? 0 : 1][k] = (float)hs[i][k].iters;
        if (stats) {
            double sum = 0.0;
            stats->nblocks = g->nblocks;
            for (int i = 0; i < ng; ++i)
                for (auto& st : hs[i]) {
                    sum += st.iters;
                    stats->max_iters = std::max(stats->max_iters, (int32_t)std::ceil(st.iters));
                    if (st.status == SEG_MAXIT) stats->not_converged++;
                    if (st.status == SEG_BREAKDOWN) stats->breakdowns++;
                }
            stats->mean_iters = sum / std::max(1, g->nblocks);
        }
        if (reorder) {
            // longest-processing-time-first order for the next apply: the blocks' iteration counts
            // of this apply (they change little from one apply to the next) x their padded box size
            const std::vector<int>& jg = g->job_group[c128 ? 0 : 1];
            std::vector<std::pair<double, int2>> items;
            items.reserve(wh.size());
            for (const int2& w : wh) {
                const Group& gr = g->groups[jg[w.x]];
                items.push_back({(hs[jg[w.x]][w.y].iters + 1.0) * (double)gr.bs.spec_elems(), w});
            }
            std::stable_sort(items.begin(), items.end(), [](const std::pair<double, int2>& a,
                                                            const std::pair<double, int2>& b) { return a.first > b.first; });
            for (size_t k = 0; k < items.size(); ++k) wh[k] = items[k].second;
            // heavy part of a split launch: blocks that took at least 0.6 of the largest iteration
            // count, at most an eighth of the blocks (measured on the metasurface: 0.5 / 4, 0.75 / 16
            // and 0.9 / 32 were slower)
            double itmax = 0.0;
            for (const int2& w : wh) itmax = std::max(itmax, hs[jg[w.x]][w.y].iters);
            int nh = 0;
            for (const int2& w : wh) nh += hs[jg[w.x]][w.y].iters >= 0.6 * itmax ? 1 : 0;
            g->nheavy[c128 ? 0 : 1] = std::min<int>(nh, (int)wh.size() / 8);
            VIE_CK(cudaMemcpyAsync(c128 ? g->work128 : g->work64, wh.data(), wh.size() * sizeof(int2),
                                   cudaMemcpyHostToDevice, s));
        }
    }
    if (tuning) {
        VIE_TRY(wait_event(g->tev[1], timeout_ms));
        float ms = 0.f;
        VIE_CK(cudaEventElapsedTime(&ms, g->tev[0], g->tev[1]));
        // the applies differ in their blocks' iteration counts: score the launch time per unit of
        // block work (iterations x padded box of every persistent block), since with every block
        // queued the launch drains the whole queue at the rate its clusters sustain
        double work = 0.0;
        std::vector<SegState> hs;
        for (auto& gr : g->groups) {
            if (!(c128 ? gr.persistent128 : gr.persistent64)) continue;
            hs.resize(gr.bs.nb);
            VIE_CK(cudaMemcpy(hs.data(), gr.st, gr.bs.nb * sizeof(SegState), cudaMemcpyDeviceToHost));
            for (auto& st : hs) work += (st.iters + 1.0) * (double)gr.bs.spec_elems();
        }
        if (tried >= 0) g->tune_score[pi][tried] = ms / std::max(work, 1.0);
        if (++g->tune_count[pi] == ncand + 1) {
            int best = 0;
            for (int k = 1; k < ncand; ++k)
                if (g->tune_score[pi][k] < g->tune_score[pi][best]) best = k;
            g->tune_best[pi] = (slab ? kCandSlab : kCand)[best].cluster;
            g->tune_npl[pi] = (slab ? kCandSlab : kCand)[best].npl;
            g->tune_noslab[pi] = slab && !kCandSlab[best].slab;
        }
    }
    return VIE_OK;
}

static int read_outer_state(vie_grid* g, SegState* hs, cudaStream_t s, double timeout_ms) {
    SegState* h = (SegState*)(g->h_ring + 2 * (g->groups.size() + 1) * sizeof(int));
    VIE_CK(cudaMemcpyAsync(h, g->ost, sizeof(SegState), cudaMemcpyDeviceToHost, s));
    VIE_CK(cudaEventRecord(g->ev[0], s));
    VIE_TRY(wait_event(g->ev[0], timeout_ms));
    *hs = *h;
    return VIE_OK;
}

static int read_scalar(vie_grid* g, const double* d, double* out, cudaStream_t s, double timeout_ms) {
    double* h = (double*)(g->h_ring + 2 * (g->groups.size() + 1) * sizeof(int) + sizeof(SegState));
    VIE_CK(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CK(cudaEventRecord(g->ev[0], s));
    VIE_TRY(wait_event(g->ev[0], timeout_ms));
    *out = *h;
    return VIE_OK;
}

struct SolveAccum {
    int64_t inner_iters = 0;
    int precond_applies = 0;
    int mv128 = 0, mv64 = 0;
};

// Right-preconditioned BiCGSTAB on the full grid in precision C (Section II.B):
// y = K2^{-1} p and z = K2^{-1} s each iteration, x updated with the y, z computed.
template <class C>
static int bicgstab_full(vie_grid* g, const vie_spectrum* sp, KrylovVecs<C> v, const vie_solve_opts* o,
                         double tol, int maxit, cudaStream_t s, SolveAccum& acc, SegState* final_state,
                         MergeMember* mm) {
    const bool pre = o->use_precond && g->nblocks > 0;
    if (!pre) {
        v.y = v.p;
        v.z = v.s;
    }
    Bicg<C> k;
    k.nseg = 1;
    k.seglen = 3 * g->N;
    k.v = v;
    k.st = g->ost;
    k.red = &g->ored;
    VIE_TRY(bicg_init<C>(k, tol, maxit, s));
    SegState hs;
    VIE_TRY(read_outer_state(g, &hs, s, o->wait_timeout_ms));
    vie_precond_stats ps;
    auto precond = [&](const C* in, C* outv) -> int {
        VIE_TRY(precond_apply<C>(g, sp, in, outv, o->inner_tol, o->inner_maxit, s, &ps, o->wait_timeout_ms, mm));
        acc.precond_applies++;
        acc.inner_iters += (int64_t)std::llround(ps.mean_iters * ps.nblocks);
        return VIE_OK;
    };
    for (int it = 0; it < maxit && hs.status == SEG_ACTIVE; ++it) {
        VIE_TRY(bicg_rho<C>(k, s));
        VIE_TRY(bicg_update_p<C>(k, s));
        if (pre) VIE_TRY(precond(k.v.p, k.v.y));
        VIE_TRY(mvm_full<C>(g, sp, k.v.y, k.v.v, s));
        (prec_of<C>() == VIE_C128 ? acc.mv128 : acc.mv64)++;
        VIE_TRY(bicg_sigma<C>(k, s));
        VIE_TRY(bicg_update_s<C>(k, s));
        VIE_TRY(bicg_x_half<C>(k, s));
        VIE_TRY(read_outer_state(g, &hs, s, o->wait_timeout_ms));
        if (hs.status != SEG_ACTIVE) break;
        if (pre) VIE_TRY(precond(k.v.s, k.v.z));
        VIE_TRY(mvm_full<C>(g, sp, k.v.z, k.v.t, s));
        (prec_of<C>() == VIE_C128 ? acc.mv128 : acc.mv64)++;
        VIE_TRY(bicg_omega<C>(k, s));
        VIE_TRY(bicg_update_xr<C>(k, s));
        VIE_TRY(read_outer_state(g, &hs, s, o->wait_timeout_ms));
    }
    VIE_TRY(read_outer_state(g, &hs, s, o->wait_timeout_ms));
    *final_state = hs;
    return VIE_OK;
}

static int status_code(int seg_status) {
    switch (seg_status) {
        case SEG_CONVERGED: return VIE_OK;
        case SEG_MAXIT: return VIE_ENOTCONV;
        case SEG_ACTIVE: return VIE_ENOTCONV;
        default: return VIE_EBREAKDOWN;
    }
}

// ||E_inc - A E|| / ||E_inc|| in FP64 (complex128 MVM); r128 receives the residual.
static int true_residual(vie_grid* g, const vie_spectrum* sp, const double2* b, const double2* x, double2* r,
                         double bnorm2, double* rel, cudaStream_t s, double timeout_ms, SolveAccum& acc) {
    VIE_TRY(mvm_full<double2>(g, sp, x, g->tmp128, s));
    acc.mv128++;
    VIE_TRY(vec_residual128(b, g->tmp128, r, 3 * g->N, s));
    VIE_TRY(vec_norm2_128(r, 3 * g->N, &g->ored, g->dscal + 1, s));
    double rn2 = 0;
    VIE_TRY(read_scalar(g, g->dscal + 1, &rn2, s, timeout_ms));
    *rel = bnorm2 > 0 ? std::sqrt(rn2 / bnorm2) : 0.0;
    return VIE_OK;
}

}  // namespace vie

extern "C" int vie_plane_wave(const vie_grid* g, double k0, const double* khat, const double* pol, int precision,
                              void* out, vie_stream_t stream) {
    if (!g || !khat || !pol || !out) return fail(VIE_EINVAL, "vie_plane_wave: null argument");
    if (precision != VIE_C128 && precision != VIE_C64) return fail(VIE_EINVAL, "vie_plane_wave: bad precision");
    return plane_wave_launch(g, k0, khat, pol, precision, out, (cudaStream_t)stream);
}

extern "C" int vie_matvec(vie_grid* g, const vie_spectrum* sp, int precision, const void* x, void* y,
                          vie_stream_t stream) {
    if (!g || !x || !y) return fail(VIE_EINVAL, "vie_matvec: null argument");
    VIE_TRY(check_spectrum(g, sp, precision));
    const int64_t bytes = 3 * g->N * (precision == VIE_C128 ? 16 : 8);
    if (overlaps(x, y, bytes)) return fail(VIE_EINVAL, "vie_matvec: x and y overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == VIE_C128) return mvm_full<double2>(g, sp, (const double2*)x, (double2*)y, s);
    return mvm_full<float2>(g, sp, (const float2*)x, (float2*)y, s);
}

extern "C" int vie_block_precond_apply(vie_grid* g, const vie_spectrum* sp, int precision, const void* b, void* y,
                                       double inner_tol, int inner_maxit, vie_stream_t stream,
                                       vie_precond_stats* stats) {
    if (!g || !b || !y) return fail(VIE_EINVAL, "vie_block_precond_apply: null argument");
    VIE_TRY(check_spectrum(g, sp, precision));
    if (!(inner_tol > 0.0) || inner_maxit < 1) return fail(VIE_EINVAL, "vie_block_precond_apply: bad tolerance or maxit");
    const int64_t bytes = 3 * g->N * (precision == VIE_C128 ? 16 : 8);
    if (overlaps(b, y, bytes)) return fail(VIE_EINVAL, "vie_block_precond_apply: b and y overlap");
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if (precision == VIE_C128)
        rc = precond_apply<double2>(g, sp, (const double2*)b, (double2*)y, inner_tol, inner_maxit, s, stats, 0);
    else
        rc = precond_apply<float2>(g, sp, (const float2*)b, (float2*)y, inner_tol, inner_maxit, s, stats, 0);
    if (rc) return rc;
    VIE_CK(cudaEventRecord(g->ev[0], s));
    return wait_event(g->ev[0], 0);
}

namespace vie {
static int solve_impl(vie_grid* g, const vie_spectrum* sp, const void* einc, void* e, const vie_solve_opts* o,
                      cudaStream_t stream, vie_solve_stats* stats, MergeMember* mm);
}

extern "C" int vie_solve(vie_grid* g, const vie_spectrum* sp, const void* einc, void* e, const vie_solve_opts* o,
                         vie_stream_t stream, vie_solve_stats* stats) {
    return solve_impl(g, sp, einc, e, o, (cudaStream_t)stream, stats, nullptr);
}

namespace vie {
static int solve_impl(vie_grid* g, const vie_spectrum* sp, const void* einc, void* e, const vie_solve_opts* o,
                      cudaStream_t stream, vie_solve_stats* stats, MergeMember* mm) {
    if (!g || !einc || !e || !o) return fail(VIE_EINVAL, "vie_solve: null argument");
    VIE_TRY(check_spectrum(g, sp, VIE_C128));
    if (o->mode == VIE_MODE_MIXED) VIE_TRY(check_spectrum(g, sp, VIE_C64));
    else if (o->mode != VIE_MODE_PLAIN_C128) return fail(VIE_EINVAL, "vie_solve: bad mode");
    if (!(o->outer_tol > 0.0) || o->outer_maxit < 1) return fail(VIE_EINVAL, "vie_solve: bad outer tolerance or maxit");
    if (o->use_precond && (!(o->inner_tol > 0.0) || o->inner_maxit < 1))
        return fail(VIE_EINVAL, "vie_solve: bad inner tolerance or maxit");
    const int64_t n3 = 3 * g->N;
    if (overlaps(einc, e, n3 * 16)) return fail(VIE_EINVAL, "vie_solve: einc and e overlap");
    const double2* x0 = (const double2*)o->x0_dev;
    if (x0 && x0 != (const double2*)e && (overlaps(x0, e, n3 * 16) || overlaps(x0, einc, n3 * 16)))
        return fail(VIE_EINVAL, "vie_solve: x0 overlaps einc, or overlaps e without being e");
    const auto t_start = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const double tmo = o->wait_timeout_ms;
    SolveAccum acc;
    vie_solve_stats st;
    memset(&st, 0, sizeof(st));
    const double2* b = (const double2*)einc;
    double2* x = (double2*)e;

    VIE_TRY(vec_norm2_128(b, n3, &g->ored, g->dscal, s));
    double bn2 = 0;
    VIE_TRY(read_scalar(g, g->dscal, &bn2, s, tmo));
    if (!std::isfinite(bn2)) return fail(VIE_EINVAL, "vie_solve: einc has non-finite entries");
    if (!(bn2 > 0.0)) x0 = nullptr;        // E_inc = 0: the solution is 0 whatever the guess
    int rc = VIE_OK;
    bool stalled = false;                  // MIXED stopped on a correction that did not help
    if (o->mode == VIE_MODE_PLAIN_C128) {
        KrylovVecs<double2> v = g->o128;
        v.b = const_cast<double2*>(b);
        v.x = x;
        double tol = o->outer_tol;
        if (x0) {
            // BiCGSTAB from E_0 is BiCGSTAB from 0 on A d = r_0 = E_inc - A E_0, E = E_0 + d,
            // with the stopping test still relative to ||E_inc||
            double rel0 = 0;
            VIE_TRY(true_residual(g, sp, b, x0, g->tmp128, bn2, &rel0, s, tmo, acc));
            v.b = g->tmp128;
            if (x0 == (const double2*)x) {
                if (!g->x0buf) VIE_TRY(dalloc(g, &g->x0buf, n3));
                v.x = g->x0buf;
            }
            tol = rel0 > 0 ? o->outer_tol / rel0 : o->outer_tol;
        }
        SegState fs;
        VIE_TRY(bicgstab_full<double2>(g, sp, v, o, tol, o->outer_maxit, s, acc, &fs, mm));
        st.outer_iters = fs.iters;
        rc = status_code(fs.status);
        if (x0) VIE_TRY(vec_sum128(x0, v.x, x, n3, s));
        VIE_TRY(true_residual(g, sp, b, x, g->o128.r, bn2, &st.true_rel_res, s, tmo, acc));
    } else {
        // iterative refinement: FP64 residual, complex64 preconditioned correction. A correction is
        // kept only if it lowers the FP64 residual. Otherwise it is undone and, once, the correction
        // is solved again without the preconditioner: when inner block solves stall (blocks of a
        // metal with Re(eps_r) < 0 at a loose inner tolerance), the inexact preconditioner changes
        // from one application to the next and the preconditioned iteration can diverge.
        const int maxref = o->max_refinements > 0 ? o->max_refinements : 8;
        double rel = bn2 > 0 ? 1.0 : 0.0;
        if (x0) {
            if (x0 != (const double2*)x) VIE_TRY(vec_copy<double2>(x0, x, n3, s));
            VIE_TRY(true_residual(g, sp, b, x, g->o128.r, bn2, &rel, s, tmo, acc));
        } else {
            VIE_CK(cudaMemsetAsync(x, 0, n3 * sizeof(double2), s));
            VIE_TRY(vec_copy<double2>(b, g->o128.r, n3, s));
            VIE_CK(cudaMemcpyAsync(g->dscal + 1, g->dscal, sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        double prev = rel;
        vie_solve_opts oc = *o;            // options of the correction solves
        rc = VIE_ENOTCONV;
        for (int ref = 0; ref <= maxref; ++ref) {
            if (ref > 0) {
                VIE_TRY(true_residual(g, sp, b, x, g->o128.r, bn2, &rel, s, tmo, acc));
                st.refinements++;
                if (!(rel < prev)) {       // also catches a non-finite residual: restore E and r
                    VIE_TRY(vec_copy<double2>(g->o128.p, x, n3, s));
                    VIE_TRY(vec_copy<double2>(g->o128.s, g->o128.r, n3, s));
                    VIE_CK(cudaMemcpyAsync(g->dscal + 1, g->dscal + 2, sizeof(double), cudaMemcpyDeviceToDevice, s));
                    st.rejected++;
                    rel = prev;
                    if (!oc.use_precond || g->nblocks == 0) {
                        stalled = true;
                        break;
                    }
                    oc.use_precond = 0;
                    merge_leave(mm);
                }
            }
            if (rel <= o->outer_tol) {
                rc = VIE_OK;
                break;
            }
            if (ref == maxref) break;
            prev = rel;
            // E, r and ||r||^2 before this correction, kept for undoing it (p and s of the
            // complex128 Krylov set are free in this mode)
            VIE_TRY(vec_copy<double2>(x, g->o128.p, n3, s));
            VIE_TRY(vec_copy<double2>(g->o128.r, g->o128.s, n3, s));
            VIE_CK(cudaMemcpyAsync(g->dscal + 2, g->dscal + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
            VIE_TRY(vec_scale_to_c64(g->o128.r, g->dscal + 1, g->o64.b, n3, s));
            const double eta = std::max(0.5 * o->outer_tol / rel, 1e-4);
            SegState fs;
            VIE_TRY(bicgstab_full<float2>(g, sp, g->o64, &oc, std::min(eta, 0.5), o->outer_maxit, s, acc, &fs, mm));
            st.outer_iters += fs.iters;
            if (fs.status == SEG_BREAKDOWN && fs.iters == 0) {
                rc = VIE_EBREAKDOWN;
                break;
            }
            VIE_TRY(vec_add_scaled_c64(x, g->o64.x, g->dscal + 1, n3, s));
        }
        st.true_rel_res = rel;
    }
    st.inner_iters = acc.inner_iters;
    st.precond_applies = acc.precond_applies;
    st.matvecs_c128 = acc.mv128;
    st.matvecs_c64 = acc.mv64;
    st.status = rc;
    st.elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = st;
    if (rc != VIE_OK) {
        if (rc == VIE_ENOTCONV)
            set_error(stalled ? "vie_solve: a correction did not lower the FP64 residual (undone); stopped"
                                  : "vie_solve: iteration limit reached before the tolerance");
        if (rc == VIE_EBREAKDOWN) set_error("vie_solve: BiCGSTAB breakdown");
    }
    return rc;
}

}  // namespace vie

// A solve from host buffers: E_inc copied in and E copied out on `stream` around the solve, through
// two device vectors the grid keeps (allocated on first use).
extern "C" int vie_solve_host(vie_grid* g, const vie_spectrum* sp, const void* einc_host, void* e_host,
                              const vie_solve_opts* o, vie_stream_t stream, vie_solve_stats* stats) {
    if (!g || !einc_host || !e_host || !o) return fail(VIE_EINVAL, "vie_solve_host: null argument");
    const int64_t bytes = 3 * g->N * (int64_t)sizeof(double2);
    if (overlaps(einc_host, e_host, bytes)) return fail(VIE_EINVAL, "vie_solve_host: einc and e overlap");
    cudaStream_t s = (cudaStream_t)stream;
    for (auto& p : g->host_io)
        if (!p) VIE_TRY(dalloc(g, &p, 3 * g->N));
    VIE_CK(cudaMemcpyAsync(g->host_io[0], einc_host, bytes, cudaMemcpyHostToDevice, s));
    const int rc = solve_impl(g, sp, g->host_io[0], g->host_io[1], o, s, stats, nullptr);
    if (rc != VIE_OK && rc != VIE_ENOTCONV) return rc;
    const std::string msg = rc == VIE_OK ? std::string() : g_last_error;
    VIE_CK(cudaMemcpyAsync(e_host, g->host_io[1], bytes, cudaMemcpyDeviceToHost, s));
    VIE_CK(cudaEventRecord(g->ev[0], s));
    VIE_TRY(wait_event(g->ev[0], o->wait_timeout_ms));
    if (rc != VIE_OK) set_error(msg);
    return rc;
}

// ---------------------------------------------------------------- merge sessions
extern "C" int vie_merge_session_create(vie_merge_session** out) {
    if (!out) return fail(VIE_EINVAL, "vie_merge_session_create: null argument");
    *out = nullptr;
    auto* mc = new vie_merge_session();
    VIE_CK(cudaGetDevice(&mc->device));
    cudaError_t e = cudaStreamCreateWithFlags(&mc->ms, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete mc;
        return cuda_fail(e, "vie_merge_session_create: stream", __FILE__, __LINE__);
    }
    *out = mc;
    return VIE_OK;
}

extern "C" int vie_merge_session_destroy(vie_merge_session* mc) {
    if (!mc) return fail(VIE_EINVAL, "vie_merge_session_destroy: null session");
    {
        std::lock_guard<std::mutex> lock(mc->m);
        if (mc->inside > 0) return fail(VIE_EBUSY, "vie_merge_session_destroy: solves are still running in the session");
    }
    cudaStreamSynchronize(mc->ms);
    cudaStreamDestroy(mc->ms);
    for (auto& kv : mc->launches_open) cudaEventDestroy(kv.second.done);
    for (auto ev : mc->free_events) cudaEventDestroy(ev);
    for (void* p : mc->retired) dfree(p);
    dfree(mc->d_groups);
    dfree(mc->d_work);
    dfree(mc->d_next);
    delete mc;
    return VIE_OK;
}

extern "C" int vie_merge_session_stats(vie_merge_session* mc, vie_merge_stats* out) {
    if (!mc || !out) return fail(VIE_EINVAL, "vie_merge_session_stats: null argument");
    std::lock_guard<std::mutex> lock(mc->m);
    out->launches = mc->launches;
    out->max_solves = mc->max_members;
    out->mean_solves = mc->launches ? (double)mc->members / mc->launches : 0.0;
    return VIE_OK;
}

namespace vie {
// A solve inside a session: it takes part in the merged launches from its first preconditioner
// application on when its grid has blocks that fit the persistent solver (joined = already counted).
static int solve_member(vie_merge_session* mc, vie_grid* g, const vie_spectrum* sp, const void* einc, void* e,
                        const vie_solve_opts* o, cudaStream_t s, vie_solve_stats* stats, bool joined) {
    MergeMember mm;
    mm.ctx = mc;
    mm.live = joined;
    if (!joined && o && o->use_precond && g) {
        const int pi = o->mode == VIE_MODE_MIXED ? 1 : 0;
        bool fit = false;
        for (const Group& gr : g->groups) fit = fit || gr.fit[pi];
        if (fit) merge_join(&mm);
    }
    const int rc = solve_impl(g, sp, einc, e, o, s, stats, &mm);
    merge_leave(&mm);
    return rc;
}

static bool member_fits(const vie_grid* g, const vie_solve_opts* o) {
    if (!g || !o || !o->use_precond) return false;
    const int pi = o->mode == VIE_MODE_MIXED ? 1 : 0;
    for (const Group& gr : g->groups)
        if (gr.fit[pi]) return true;
    return false;
}
}  // namespace vie

extern "C" int vie_solve_merged(vie_merge_session* mc, vie_grid* g, const vie_spectrum* sp, const void* einc, void* e,
                                const vie_solve_opts* o, vie_stream_t stream, vie_solve_stats* stats) {
    if (!mc) return fail(VIE_EINVAL, "vie_solve_merged: null session");
    {
        std::lock_guard<std::mutex> lock(mc->m);
        mc->inside++;
    }
    const int rc = solve_member(mc, g, sp, einc, e, o, (cudaStream_t)stream, stats, false);
    std::lock_guard<std::mutex> lock(mc->m);
    mc->inside--;
    return rc;
}

// Several solves at once in a session of their own: one host thread and one stream per solve,
// all of them members from the start (so the first applications already merge).
extern "C" int vie_solve_many(int32_t n, vie_grid* const* grids, const vie_spectrum* const* spectra,
                              const void* const* einc_dev, void* const* e_dev, const vie_solve_opts* opts,
                              vie_stream_t stream, vie_solve_stats* stats, vie_merge_stats* merge) {
    if (n < 1 || !grids || !spectra || !einc_dev || !e_dev || !opts)
        return fail(VIE_EINVAL, "vie_solve_many: null argument or n < 1");
    if (merge) memset(merge, 0, sizeof(*merge));
    for (int i = 0; i < n; ++i) {
        if (!grids[i]) return fail(VIE_EINVAL, "vie_solve_many: null grid");
        for (int j = 0; j < i; ++j)
            if (grids[j] == grids[i]) return fail(VIE_EINVAL, "vie_solve_many: a grid appears twice");
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 1) return solve_impl(grids[0], spectra[0], einc_dev[0], e_dev[0], &opts[0], s, stats, nullptr);
    vie_merge_session* mc = nullptr;
    VIE_TRY(vie_merge_session_create(&mc));
    std::vector<cudaStream_t> st(n, nullptr);
    cudaEvent_t start = nullptr;
    cudaError_t ce = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventRecord(start, s);
    for (int i = 0; i < n && ce == cudaSuccess; ++i) {
        ce = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st[i], start, 0);
    }
    auto cleanup = [&]() {
        for (auto x : st)
            if (x) cudaStreamDestroy(x);
        if (start) cudaEventDestroy(start);
        vie_merge_session_destroy(mc);
    };
    if (ce != cudaSuccess) {
        const int rc = cuda_fail(ce, "vie_solve_many: stream set-up", __FILE__, __LINE__);
        cleanup();
        return rc;
    }
    std::vector<char> joined(n, 0);
    for (int i = 0; i < n; ++i)
        if (member_fits(grids[i], &opts[i])) {
            joined[i] = 1;
            mc->live++;
        }
    std::vector<int> rcs(n, VIE_OK);
    std::vector<std::string> errs(n);
    std::vector<vie_solve_stats> local(n);
    auto run = [&](int i) {
        memset(&local[i], 0, sizeof(vie_solve_stats));
        cudaError_t e = cudaSetDevice(grids[i]->device);
        int r = e == cudaSuccess
                    ? solve_member(mc, grids[i], spectra[i], einc_dev[i], e_dev[i], &opts[i], st[i], &local[i], joined[i])
                    : cuda_fail(e, "cudaSetDevice", __FILE__, __LINE__);
        if (r != VIE_OK) errs[i] = g_last_error;
        local[i].status = r;
        rcs[i] = r;
    };
    {
        std::vector<std::thread> th;
        th.reserve(n);
        for (int i = 0; i < n; ++i) th.emplace_back(run, i);
        for (auto& t : th) t.join();
    }
    if (stats)
        for (int i = 0; i < n; ++i) stats[i] = local[i];
    if (merge) vie_merge_session_stats(mc, merge);
    // the caller's stream continues after every solve's work
    for (int i = 0; i < n; ++i) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(ev, st[i]);
            cudaStreamWaitEvent(s, ev, 0);
            cudaEventDestroy(ev);
        }
    }
    cleanup();
    for (int i = 0; i < n; ++i)
        if (rcs[i] != VIE_OK) {
            set_error("vie_solve_many: solve " + std::to_string(i) + ": " + errs[i]);
            return rcs[i];
        }
    return VIE_OK;
}
