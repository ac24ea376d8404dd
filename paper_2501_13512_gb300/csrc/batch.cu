// Batched independent solves: many instances of one grid shape (each with its
// own permittivity, wavenumber and incident field) solved together. Each
// instance is the unpreconditioned system A E = E_inc of Eq. 4; the mixed
// solve is the same iterative refinement as vie_solve: FP64 residuals for all
// instances from one batched complex128 MVM, then one persistent complex64
// launch in which every instance's BiCGSTAB correction runs on its own CTA
// cluster (the block solver of inner.cu with the whole grid as the block).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "vie_internal.cuh"

struct vie_batch {
    int device = 0;
    int nx = 0, ny = 0, nz = 0, count = 0;
    double h = 0.0;
    int64_t n3 = 0;                       // 3 N per instance
    vie::BoxSet bs;                       // nb = count, box = grid, mask = all ones
    vie::KrylovVecs<float2> k64;          // correction solve vectors [count][3][nz][ny][nx]
    vie::SegState* st = nullptr;          // [count]
    vie::ReduceScratch red;
    double2* r128 = nullptr;              // FP64 residuals
    double2* tmp128 = nullptr;            // A x
    double2* xprev = nullptr;             // E before the last correction
    double* d_bn2 = nullptr;              // [count] ||E_inc||^2
    double* d_rn2 = nullptr;              // [count] ||r||^2
    double* d_tols = nullptr;             // [count] correction tolerances (0: instance done)
    double2** d_gb128 = nullptr;          // [count] spectrum per instance
    float2** d_gb64 = nullptr;
    int2* work = nullptr;                 // persistent work list (0, b)
    void* inner_groups = nullptr;
    int* inner_next = nullptr;
    bool persistent = false;
    double* h_scal = nullptr;             // pinned [2 count]
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_ready = nullptr;       // gathers queued before a merged launch
    std::map<double, std::pair<double2*, float2*>> spectra;   // cached per wavenumber
    std::vector<void*> allocations;
    int64_t device_bytes = 0;
};

namespace vie {
namespace {

template <class T>
int balloc(vie_batch* b, T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) return VIE_OK;
    VIE_TRY(dmalloc((void**)p, (size_t)count * sizeof(T), "vie_batch_create"));
    b->allocations.push_back((void*)*p);
    b->device_bytes += count * (int64_t)sizeof(T);
    return VIE_OK;
}

void release(vie_batch* b) {
    for (auto& kv : b->spectra) {
        dfree(kv.second.first);
        dfree(kv.second.second);
    }
    for (void* p : b->allocations) dfree(p);
    if (b->h_scal) cudaFreeHost(b->h_scal);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->ev_ready) cudaEventDestroy(b->ev_ready);
    delete b;
}

int p2(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
int lg2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// ||v_b||^2 per instance, one CTA per instance (fixed summation order).
__global__ void __launch_bounds__(512) k_seg_norm2(const double2* v, int64_t seglen, double* out) {
    const double2* p = v + (int64_t)blockIdx.x * seglen;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < seglen; i += blockDim.x) acc += p[i].x * p[i].x + p[i].y * p[i].y;
    __shared__ double sh[512];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// b64 = r / ||r|| for instances still being refined (tol > 0), else 0.
__global__ void k_seg_scale(const double2* r, const double* rn2, const double* tols, float2* b64, int64_t seglen,
                            int count) {
    const int64_t n = seglen * count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / seglen);
        const double inv = tols[b] > 0.0 ? 1.0 / sqrt(rn2[b]) : 0.0;
        b64[i] = make_float2((float)(r[i].x * inv), (float)(r[i].y * inv));
    }
}

// x += ||r|| d for instances being refined.
__global__ void k_seg_add(double2* x, const float2* d, const double* rn2, const double* tols, int64_t seglen,
                          int count) {
    const int64_t n = seglen * count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / seglen);
        if (!(tols[b] > 0.0)) continue;
        const double sc = sqrt(rn2[b]);
        x[i] = make_double2(x[i].x + sc * (double)d[i].x, x[i].y + sc * (double)d[i].y);
    }
}

// x = xprev for instances whose last correction is undone (sel > 0).
__global__ void k_seg_restore(double2* x, const double2* xprev, const double* sel, int64_t seglen, int count) {
    const int64_t n = seglen * count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (sel[i / seglen] > 0.0) x[i] = xprev[i];
}

__global__ void k_fill_u8(uint8_t* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 1;
}

unsigned grid1(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

int wait_ev(cudaEvent_t ev, double timeout_ms) {
    if (timeout_ms <= 0) timeout_ms = 60000.0;
    cudaError_t e;
    auto t0 = std::chrono::steady_clock::now();
    while ((e = cudaEventQuery(ev)) == cudaErrorNotReady) {
        if (std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > timeout_ms)
            return fail(VIE_ETIMEOUT, "vie_batch: device did not finish within the wait bound");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventQuery", __FILE__, __LINE__);
    return VIE_OK;
}

}  // namespace
}  // namespace vie

using namespace vie;

extern "C" int vie_batch_create(const vie_batch_desc* d, vie_batch** out) {
    if (!d || !out || !d->eps_r) return fail(VIE_EINVAL, "vie_batch_create: null argument");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->nx > kLmax / 2 || d->ny > kLmax / 2 || d->nz > kLmax / 2)
        return fail(VIE_EINVAL, "vie_batch_create: each of nx, ny, nz must be in [1, 512]");
    if (d->count < 1 || d->count > 21845) return fail(VIE_EINVAL, "vie_batch_create: count must be in [1, 21845]");
    if (!(d->h > 0.0) || !std::isfinite(d->h)) return fail(VIE_EINVAL, "vie_batch_create: h must be positive");
    if (d->flags != 0) return fail(VIE_EINVAL, "vie_batch_create: flags must be 0");
    vie_batch* b = new vie_batch();
    auto bail = [&](int rc) { release(b); return rc; };
    if (cudaGetDevice(&b->device) != cudaSuccess) return bail(fail(VIE_ECUDA, "no CUDA device"));
    b->nx = d->nx; b->ny = d->ny; b->nz = d->nz; b->h = d->h; b->count = d->count;
    const int64_t N = (int64_t)d->nx * d->ny * d->nz;
    b->n3 = 3 * N;
    BoxSet& bs = b->bs;
    bs.nb = d->count;
    bs.oct = true;      // complex128 spectra (and complex64 ones outside the persistent solver) are octant-compressed
    bs.bx = d->nx; bs.by = d->ny; bs.bz = d->nz;
    bs.Mx = p2(2 * d->nx - 1); bs.My = p2(2 * d->ny - 1); bs.Mz = p2(2 * d->nz - 1);
    bs.lx = lg2i(bs.Mx); bs.ly = lg2i(bs.My); bs.lz = lg2i(bs.Mz);
    const int64_t tot = N * d->count;
    std::vector<double2> chi(tot);
    std::vector<float2> chi64(tot);
    for (int64_t i = 0; i < tot; ++i) {
        double re = d->eps_r[2 * i] - 1.0, im = d->eps_r[2 * i + 1];
        if (!std::isfinite(re) || !std::isfinite(im)) return bail(fail(VIE_EINVAL, "vie_batch_create: non-finite eps_r"));
        chi[i] = make_double2(re, im);
        chi64[i] = make_float2((float)re, (float)im);
    }
    int rc;
    const int64_t w1 = (int64_t)bs.nb * 3 * bs.bz * bs.by * bs.Mx, w2 = (int64_t)bs.nb * 3 * bs.bz * bs.My * bs.Mx;
    double2 *pw1 = nullptr, *pw2 = nullptr;
    if ((rc = balloc(b, &bs.chi128, tot)) || (rc = balloc(b, &bs.chi64, tot)) || (rc = balloc(b, &bs.mask, tot)) ||
        (rc = balloc(b, &pw1, w1)) || (rc = balloc(b, &pw2, w2)))
        return bail(rc);
    bs.w1 = pw1;
    bs.w2 = pw2;
    const int64_t nv = b->n3 * d->count;
    KrylovVecs<float2>& k = b->k64;
    if ((rc = balloc(b, &k.b, nv)) || (rc = balloc(b, &k.x, nv)) || (rc = balloc(b, &k.r, nv)) ||
        (rc = balloc(b, &k.rhat, nv)) || (rc = balloc(b, &k.p, nv)) || (rc = balloc(b, &k.v, nv)) ||
        (rc = balloc(b, &k.s, nv)) || (rc = balloc(b, &k.t, nv)) || (rc = balloc(b, &b->r128, nv)) ||
        (rc = balloc(b, &b->tmp128, nv)) || (rc = balloc(b, &b->xprev, nv)) || (rc = balloc(b, &b->st, d->count)) ||
        (rc = balloc(b, &b->d_bn2, d->count)) || (rc = balloc(b, &b->d_rn2, d->count)) ||
        (rc = balloc(b, &b->d_tols, d->count)) || (rc = balloc(b, &b->d_gb128, d->count)) ||
        (rc = balloc(b, &b->d_gb64, d->count)))
        return bail(rc);
    k.y = k.p;
    k.z = k.s;
    b->red.nseg = d->count;
    if ((rc = balloc(b, &b->red.part, (int64_t)d->count * kMaxCtaPerSeg * 2)) ||
        (rc = balloc(b, &b->red.count, d->count)) || (rc = balloc(b, &b->red.n_active, 1)))
        return bail(rc);
    if (cudaMemset(b->red.count, 0, d->count * sizeof(unsigned)) != cudaSuccess ||
        cudaMemcpy(bs.chi128, chi.data(), tot * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(bs.chi64, chi64.data(), tot * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(VIE_ECUDA, "vie_batch_create: upload failed"));
    k_fill_u8<<<grid1(tot), 256>>>(bs.mask, tot);
    if (cudaGetLastError() != cudaSuccess) return bail(fail(VIE_ECUDA, "vie_batch_create: mask fill failed"));
    b->persistent = inner_persistent_ok(bs, sizeof(float2), true);
    if (b->persistent) {
        std::vector<int2> w(d->count);
        for (int i = 0; i < d->count; ++i) w[i] = make_int2(0, i);
        char* descs = nullptr;
        if ((rc = balloc(b, &b->work, d->count)) || (rc = balloc(b, &descs, (int64_t)inner_group_desc_bytes())) ||
            (rc = balloc(b, &b->inner_next, 1)))
            return bail(rc);
        b->inner_groups = descs;
        if (cudaMemcpy(b->work, w.data(), w.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(VIE_ECUDA, "vie_batch_create: upload failed"));
    }
    if (cudaHostAlloc((void**)&b->h_scal, 2 * d->count * sizeof(double), cudaHostAllocDefault) != cudaSuccess)
        return bail(fail(VIE_ENOMEM, "vie_batch_create: pinned allocation failed"));
    if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_ready, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(VIE_ECUDA, "vie_batch_create: event creation failed"));
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(fail(VIE_ECUDA, "vie_batch_create: set-up failed"));
    *out = b;
    return VIE_OK;
}

extern "C" int vie_batch_destroy(vie_batch* b) {
    if (!b) return fail(VIE_EINVAL, "vie_batch_destroy: null batch");
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    release(b);
    cudaSetDevice(prev);
    return VIE_OK;
}

namespace vie {
static int batch_solve_impl(vie_batch* b, const double* k0s, const void* einc_dev, void* e_dev,
                            const vie_solve_opts* o, cudaStream_t s, vie_solve_stats* stats, MergeMember* mm);
}

extern "C" int vie_batch_solve(vie_batch* b, const double* k0s, const void* einc_dev, void* e_dev,
                               const vie_solve_opts* o, vie_stream_t stream, vie_solve_stats* stats) {
    return batch_solve_impl(b, k0s, einc_dev, e_dev, o, (cudaStream_t)stream, stats, nullptr);
}

namespace vie {
// The batched mixed solve; mm (may be null): membership in a merge session, whose merged launches
// then take this batch's persistent correction launches.
static int batch_solve_impl(vie_batch* b, const double* k0s, const void* einc_dev, void* e_dev,
                            const vie_solve_opts* o, cudaStream_t s, vie_solve_stats* stats, MergeMember* mm) {
    if (!b || !k0s || !einc_dev || !e_dev || !o) return fail(VIE_EINVAL, "vie_batch_solve: null argument");
    if (o->mode != VIE_MODE_MIXED) return fail(VIE_EINVAL, "vie_batch_solve: only VIE_MODE_MIXED is supported");
    if (o->x0_dev) return fail(VIE_EINVAL, "vie_batch_solve: x0_dev must be NULL");
    const auto t_start = std::chrono::steady_clock::now();
    if (!(o->outer_tol > 0.0) || o->outer_maxit < 1) return fail(VIE_EINVAL, "vie_batch_solve: bad tolerance or maxit");
    const int nb = b->count;
    const int64_t nv = b->n3 * nb;
    const char* ea = (const char*)einc_dev;
    const char* xa = (const char*)e_dev;
    if (ea < xa + nv * 16 && xa < ea + nv * 16) return fail(VIE_EINVAL, "vie_batch_solve: einc and e overlap");
    for (int i = 0; i < nb; ++i)
        if (!(k0s[i] > 0.0) || !std::isfinite(k0s[i])) return fail(VIE_EINVAL, "vie_batch_solve: k0 must be positive");
    const double tmo = o->wait_timeout_ms;
    BoxSet& bs = b->bs;
    // spectra per distinct wavenumber (cached), one pointer per instance
    std::vector<double2*> gb128(nb);
    std::vector<float2*> gb64(nb);
    // complex128: octant layout (batched MVMs); complex64: full layout when the persistent
    // block solver reads it, else octant layout
    const int64_t so = 6 * bs.oct_elems();
    const int64_t s64 = b->persistent ? 6 * bs.spec_elems() : so;
    for (int i = 0; i < nb; ++i) {
        auto it = b->spectra.find(k0s[i]);
        if (it == b->spectra.end()) {
            double2* G = nullptr;
            float2* G64 = nullptr;
            int arc = dmalloc((void**)&G, so * sizeof(double2), "vie_batch_solve");
            if (!arc) arc = dmalloc((void**)&G64, s64 * sizeof(float2), "vie_batch_solve");
            if (arc) {
                dfree(G);
                return arc;
            }
            BoxSet one = bs;
            one.nb = 1;
            int rc = spectrum_build(one, k0s[i], b->h, G, b->persistent ? nullptr : G64,
                                    b->persistent ? G64 : nullptr, s);
            if (rc) {
                cudaStreamSynchronize(s);
                dfree(G);
                dfree(G64);
                return rc;
            }
            it = b->spectra.emplace(k0s[i], std::make_pair(G, G64)).first;
        }
        gb128[i] = it->second.first;
        gb64[i] = it->second.second;
    }
    VIE_CK(cudaMemcpyAsync(b->d_gb128, gb128.data(), nb * sizeof(double2*), cudaMemcpyHostToDevice, s));
    VIE_CK(cudaMemcpyAsync(b->d_gb64, gb64.data(), nb * sizeof(float2*), cudaMemcpyHostToDevice, s));
    const double2* einc = (const double2*)einc_dev;
    double2* x = (double2*)e_dev;
    std::vector<double> bn2(nb), rn2(nb), rel(nb, 1.0), iters(nb, 0.0);
    std::vector<int> status(nb, VIE_ENOTCONV), refs(nb, 0);
    k_seg_norm2<<<nb, 512, 0, s>>>(einc, b->n3, b->d_bn2);
    VIE_CK(cudaGetLastError());
    VIE_CK(cudaMemcpyAsync(b->h_scal, b->d_bn2, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    VIE_CK(cudaEventRecord(b->ev, s));
    VIE_TRY(wait_ev(b->ev, tmo));
    for (int i = 0; i < nb; ++i) {
        bn2[i] = b->h_scal[i];
        if (!std::isfinite(bn2[i]))
            return fail(VIE_EINVAL, "vie_batch_solve: einc of instance " + std::to_string(i) + " has non-finite entries");
    }
    VIE_CK(cudaMemsetAsync(x, 0, nv * sizeof(double2), s));
    VIE_TRY(vec_copy<double2>(einc, b->r128, nv, s));
    VIE_CK(cudaMemcpyAsync(b->d_rn2, b->d_bn2, nb * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rn2 = bn2;
    const int maxref = o->max_refinements > 0 ? o->max_refinements : 8;
    std::vector<double> tols(nb, 0.0), undo(nb, 0.0), prev(nb, 1.0);
    std::vector<char> stopped(nb, 0);
    int mv128 = 0;
    for (int ref = 0; ref <= maxref; ++ref) {
        if (ref > 0) {
            VIE_TRY(mvm_boxes<double2>(bs, nullptr, x, b->tmp128, nullptr, s, nullptr, b->d_gb128));
            ++mv128;
            VIE_TRY(vec_residual128(einc, b->tmp128, b->r128, nv, s));
            k_seg_norm2<<<nb, 512, 0, s>>>(b->r128, b->n3, b->d_rn2);
            VIE_CK(cudaGetLastError());
            VIE_CK(cudaMemcpyAsync(b->h_scal, b->d_rn2, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
            VIE_CK(cudaEventRecord(b->ev, s));
            VIE_TRY(wait_ev(b->ev, tmo));
            for (int i = 0; i < nb; ++i) rn2[i] = b->h_scal[i];
        }
        // an instance whose correction did not lower its FP64 residual gets it undone and stops
        int nundo = 0;
        for (int i = 0; i < nb; ++i) {
            rel[i] = bn2[i] > 0 ? std::sqrt(rn2[i] / bn2[i]) : 0.0;
            undo[i] = 0.0;
            if (ref > 0 && tols[i] > 0.0 && !(rel[i] < prev[i])) {
                undo[i] = 1.0;
                ++nundo;
                stopped[i] = 1;
                rel[i] = prev[i];
            }
        }
        if (nundo) {
            VIE_CK(cudaMemcpyAsync(b->d_tols, undo.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
            k_seg_restore<<<grid1(nv), 256, 0, s>>>(x, b->xprev, b->d_tols, b->n3, nb);
            VIE_CK(cudaGetLastError());
        }
        int active = 0;
        for (int i = 0; i < nb; ++i) {
            if (stopped[i]) {
                tols[i] = 0.0;
            } else if (rel[i] <= o->outer_tol) {
                if (status[i] != VIE_OK) refs[i] = ref;
                status[i] = VIE_OK;
                tols[i] = 0.0;
            } else {
                tols[i] = std::min(0.5, std::max(0.5 * o->outer_tol / rel[i], 1e-4));
                ++active;
            }
            prev[i] = rel[i];
        }
        if (active == 0 || ref == maxref) break;
        VIE_TRY(vec_copy<double2>(x, b->xprev, nv, s));
        VIE_CK(cudaMemcpyAsync(b->d_tols, tols.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
        k_seg_scale<<<grid1(nv), 256, 0, s>>>(b->r128, b->d_rn2, b->d_tols, b->k64.b, b->n3, nb);
        VIE_CK(cudaGetLastError());
        if (b->persistent) {
            std::vector<InnerJob<float2>> jobs(1);
            jobs[0].bs = &bs;
            jobs[0].v = b->k64;
            jobs[0].chi = bs.chi64;
            jobs[0].G = gb64[0];
            jobs[0].st = b->st;
            jobs[0].Gb = b->d_gb64;
            jobs[0].tols = b->d_tols;
            if (mm != nullptr && mm->live) {
                // the corrections of every batch of the session that reached this step, in one launch
                MergeReq req;
                req.prec = 1;
                req.tol = 0.5;
                req.maxit = o->outer_maxit;
                req.j64 = jobs;
                for (int i = 0; i < nb; ++i)
                    if (tols[i] > 0.0) req.items.push_back({(double)bs.spec_elems(), make_int2(0, i)});
                VIE_CK(cudaEventRecord(b->ev_ready, s));
                req.ready = b->ev_ready;
                merge_arrive(mm, &req);
                VIE_TRY(merge_wait(mm, &req, s));
            } else {
                VIE_TRY(inner_persistent<float2>(jobs, b->work, nb, b->inner_groups, b->inner_next, 0.5,
                                                 o->outer_maxit, s));
            }
        } else {
            Bicg<float2> k;
            k.nseg = nb;
            k.seglen = b->n3;
            k.v = b->k64;
            k.st = b->st;
            k.red = &b->red;
            VIE_TRY(bicg_init_tols<float2>(k, b->d_tols, o->outer_maxit, s));
            for (int it = 0; it < o->outer_maxit; ++it) {
                VIE_TRY(bicg_rho<float2>(k, s));
                VIE_TRY(bicg_update_p<float2>(k, s));
                VIE_TRY(mvm_boxes<float2>(bs, nullptr, k.v.p, k.v.v, b->st, s, nullptr, b->d_gb64));
                VIE_TRY(bicg_sigma<float2>(k, s));
                VIE_TRY(bicg_update_s<float2>(k, s));
                VIE_TRY(bicg_x_half<float2>(k, s));
                VIE_TRY(mvm_boxes<float2>(bs, nullptr, k.v.s, k.v.t, b->st, s, nullptr, b->d_gb64));
                VIE_TRY(bicg_omega<float2>(k, s));
                VIE_TRY(bicg_update_xr<float2>(k, s));
                if ((it & 7) == 7) {
                    VIE_CK(cudaMemcpyAsync(b->h_scal, b->red.n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
                    VIE_CK(cudaEventRecord(b->ev, s));
                    VIE_TRY(wait_ev(b->ev, tmo));
                    if (*(int*)b->h_scal == 0) break;
                }
            }
        }
        k_seg_add<<<grid1(nv), 256, 0, s>>>(x, b->k64.x, b->d_rn2, b->d_tols, b->n3, nb);
        VIE_CK(cudaGetLastError());
        // iteration counts of this correction
        std::vector<SegState> hs(nb);
        VIE_CK(cudaMemcpyAsync(hs.data(), b->st, nb * sizeof(SegState), cudaMemcpyDeviceToHost, s));
        VIE_CK(cudaEventRecord(b->ev, s));
        VIE_TRY(wait_ev(b->ev, tmo));
        for (int i = 0; i < nb; ++i)
            if (tols[i] > 0.0) iters[i] += hs[i].iters;
    }
    if (stats) {
        for (int i = 0; i < nb; ++i) {
            memset(&stats[i], 0, sizeof(stats[i]));
            stats[i].outer_iters = iters[i];
            stats[i].true_rel_res = rel[i];
            stats[i].status = status[i];
            stats[i].refinements = refs[i];
            stats[i].rejected = stopped[i];
            stats[i].elapsed_ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
            stats[i].matvecs_c128 = mv128;
        }
    }
    for (int i = 0; i < nb; ++i)
        if (status[i] != VIE_OK) {
            set_error("vie_batch_solve: some instances did not reach the tolerance");
            return VIE_ENOTCONV;
        }
    return VIE_OK;
}
}  // namespace vie

// Several batches (any grid shapes) at once in a session of their own: one host thread and stream
// per batch, the persistent correction launches of all batches at the same refinement step merged.
extern "C" int vie_batch_solve_many(int32_t n, vie_batch* const* batches, const double* const* k0s,
                                    const void* const* einc_dev, void* const* e_dev, const vie_solve_opts* opts,
                                    vie_stream_t stream, vie_solve_stats* const* stats, vie_merge_stats* merge) {
    if (n < 1 || !batches || !k0s || !einc_dev || !e_dev || !opts)
        return fail(VIE_EINVAL, "vie_batch_solve_many: null argument or n < 1");
    if (merge) memset(merge, 0, sizeof(*merge));
    for (int i = 0; i < n; ++i) {
        if (!batches[i]) return fail(VIE_EINVAL, "vie_batch_solve_many: null batch");
        for (int j = 0; j < i; ++j)
            if (batches[j] == batches[i]) return fail(VIE_EINVAL, "vie_batch_solve_many: a batch appears twice");
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 1) return batch_solve_impl(batches[0], k0s[0], einc_dev[0], e_dev[0], &opts[0], s,
                                        stats ? stats[0] : nullptr, nullptr);
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
        const int rc = cuda_fail(ce, "vie_batch_solve_many: stream set-up", __FILE__, __LINE__);
        cleanup();
        return rc;
    }
    std::vector<MergeMember> mm(n);
    for (int i = 0; i < n; ++i) {
        mm[i].ctx = mc;
        if (batches[i]->persistent) merge_join(&mm[i]);
    }
    std::vector<int> rcs(n, VIE_OK);
    std::vector<std::string> errs(n);
    auto run = [&](int i) {
        cudaError_t e = cudaSetDevice(batches[i]->device);
        int r = e == cudaSuccess ? batch_solve_impl(batches[i], k0s[i], einc_dev[i], e_dev[i], &opts[i], st[i],
                                                    stats ? stats[i] : nullptr, &mm[i])
                                 : cuda_fail(e, "cudaSetDevice", __FILE__, __LINE__);
        merge_leave(&mm[i]);
        if (r != VIE_OK) errs[i] = last_error_message();
        rcs[i] = r;
    };
    {
        std::vector<std::thread> th;
        th.reserve(n);
        for (int i = 0; i < n; ++i) th.emplace_back(run, i);
        for (auto& t : th) t.join();
    }
    if (merge) vie_merge_session_stats(mc, merge);
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
            set_error("vie_batch_solve_many: batch " + std::to_string(i) + ": " + errs[i]);
            return rcs[i];
        }
    return VIE_OK;
}

extern "C" int vie_batch_get_info(const vie_batch* b, int64_t* device_bytes, int32_t* persistent) {
    if (!b) return fail(VIE_EINVAL, "vie_batch_get_info: null batch");
    if (device_bytes) {
        int64_t sp = 0;
        for (auto& kv : b->spectra) sp += 6 * b->bs.spec_elems() * (16 + 8);
        *device_bytes = b->device_bytes + sp;
    }
    if (persistent) *persistent = b->persistent ? 1 : 0;
    return VIE_OK;
}
