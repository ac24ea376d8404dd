// The paper's rooftop-basis / pulse-testing discretisation of the VIE
// (Section II.A, Eqs. 5-9), on the GPU.
//
// Unknown w = J / (j w eps0) (units of E), component a on the face between
// cell c and cell c + e_a; a face carries a rooftop when both of its cells are
// inside the grid and non-air (the normal current vanishes on the object's
// surface, the case the paper's Section I says its MoM is built for). Tested
// with pulses on the dual cells (Eq. 6), Eq. 4 becomes
//
//   (A w)_(a,c) = [M_chi w]_(a,c) + sum_(b,c') K_ab(c - c') w_(b,c') = E_inc,a(face centre),
//   M_chi:  (3/8)(1/chi_c + 1/chi_(c+e_a)) w_(a,c) + (1/8)/chi_c w_(a,c-e_a) + (1/8)/chi_(c+e_a) w_(a,c+e_a),
//   K_ab(D) = -k^2 delta_ab gh(D) - [gh(D + e_a) - gh(D + e_a - e_b) - gh(D) + gh(D - e_b)] / h^2,
//
// the contrast and vector-potential terms of L^c (Eq. 8) and the scalar
// potential of L^q (Eq. 9, acting on w_j) with the sign of Eq. 4. gh(D) is the
// integral of g = e^{-jkR}/(4 pi R) over a cell at offset D: h^3 g(|D| h) for
// D != 0, the integral over the equivalent sphere of the cell at D = 0.
// K_ab is Toeplitz in the face indices, so the product runs through the same
// zero-padded pencil FFT passes as the collocation operator, with nine
// spectra (K_ab(D) = K_ba(-D), so the 3x3 multiply is not symmetric in a, b)
// in the z pass, the masked input and the Gram term fused into two
// elementwise kernels around it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>
#include <vector>

#include "vie_internal.cuh"

struct vie_rooftop {
    vie_grid* grid = nullptr;
    double k0 = 0.0;
    int precision_mask = 0;
    vie::BoxSet bs;                        // the grid's full box: shape and FFT scratch, ones as "chi"
    std::vector<void*> allocations;
    double2* G128 = nullptr;               // [9][Mz][My][Mx], -K_ab / (Mx My Mz), bit-reversed positions
    float2* G64 = nullptr;
    double2* inv128 = nullptr;             // [N] 1 / chi (0 in air)
    float2* inv64 = nullptr;
    uint8_t* act = nullptr;                // [3][N] face carries a rooftop
    double2 *in128 = nullptr, *gram128 = nullptr;   // [3N] masked input, Gram term
    float2 *in64 = nullptr, *gram64 = nullptr;
    // complex128 BiCGSTAB workspace
    vie::KrylovVecs<double2> k;
    vie::SegState* st = nullptr;
    vie::ReduceScratch red;
    vie::SegState* h_st = nullptr;         // pinned
    cudaEvent_t ev = nullptr;
};

namespace vie {
namespace {

template <class T>
int ralloc(vie_rooftop* r, T** p, int64_t count) {
    *p = nullptr;
    if (count <= 0) return VIE_OK;
    VIE_TRY(dmalloc((void**)p, (size_t)count * sizeof(T), "vie_rooftop_create"));
    r->allocations.push_back((void*)*p);
    return VIE_OK;
}

void release(vie_rooftop* r) {
    for (void* p : r->allocations) dfree(p);
    if (r->h_st) cudaFreeHost(r->h_st);
    if (r->ev) cudaEventDestroy(r->ev);
    delete r;
}

unsigned grid1(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); }

__device__ __forceinline__ bool wrap_off(int m, int M, int b, int& d) {
    if (m < b) { d = m; return true; }
    if (m > M - b) { d = m - M; return true; }
    return false;
}

// Integral of g over the cell at integer offset (dx, dy, dz).
__device__ __forceinline__ double2 cell_g(int dx, int dy, int dz, double h, double k0, double2 self) {
    if (dx == 0 && dy == 0 && dz == 0) return self;
    const double R = h * sqrt((double)dx * dx + (double)dy * dy + (double)dz * dz);
    double sn, cs;
    sincos(k0 * R, &sn, &cs);
    const double m = h * h * h * 0.25 / (3.14159265358979323846 * R);
    return make_double2(cs * m, -sn * m);
}

// -K_ab(D) / (Mx My Mz) on the padded grid (wrapped offsets; unused slots 0), natural order [9][Mz][My][Mx].
__global__ void k_rooftop_sample(double2* G, int Mx, int My, int Mz, int nx, int ny, int nz, double h, double k0,
                                 double2 self, double scale) {
    const int64_t vol = (int64_t)Mx * My * Mz;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < vol; idx += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(idx % Mx), iy = (int)((idx / Mx) % My), iz = (int)(idx / ((int64_t)Mx * My));
        int d[3];
        const bool used = wrap_off(ix, Mx, nx, d[0]) & wrap_off(iy, My, ny, d[1]) & wrap_off(iz, Mz, nz, d[2]);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double2 K = make_double2(0.0, 0.0);
                if (used) {
                    int pa[3] = {d[0], d[1], d[2]}, pab[3] = {d[0], d[1], d[2]}, mb[3] = {d[0], d[1], d[2]};
                    pa[a] += 1;
                    pab[a] += 1;
                    pab[b] -= 1;
                    mb[b] -= 1;
                    const double2 t = cell_g(pa[0], pa[1], pa[2], h, k0, self) - cell_g(pab[0], pab[1], pab[2], h, k0, self) -
                                      cell_g(d[0], d[1], d[2], h, k0, self) + cell_g(mb[0], mb[1], mb[2], h, k0, self);
                    const double ih2 = 1.0 / (h * h);
                    K = make_double2(-t.x * ih2, -t.y * ih2);
                    if (a == b) {
                        const double2 g0 = cell_g(d[0], d[1], d[2], h, k0, self);
                        K = make_double2(K.x - k0 * k0 * g0.x, K.y - k0 * k0 * g0.y);
                    }
                }
                G[(3 * a + b) * vol + idx] = make_double2(-K.x * scale, -K.y * scale);
            }
    }
}

// Face activity and the inverse contrast per cell.
__global__ void k_rooftop_tables(const double2* chi, uint8_t* act, double2* inv128, float2* inv64, int nx, int ny, int nz) {
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((int64_t)nx * ny));
        const double2 c = chi[idx];
        const bool solid = c.x != 0.0 || c.y != 0.0;
        const double d = c.x * c.x + c.y * c.y;
        const double2 inv = solid ? make_double2(c.x / d, -c.y / d) : make_double2(0.0, 0.0);
        inv128[idx] = inv;
        inv64[idx] = make_float2((float)inv.x, (float)inv.y);
        auto solid_at = [&](int64_t j) { return chi[j].x != 0.0 || chi[j].y != 0.0; };
        act[idx] = solid && x + 1 < nx && solid_at(idx + 1);
        act[N + idx] = solid && y + 1 < ny && solid_at(idx + nx);
        act[2 * N + idx] = solid && z + 1 < nz && solid_at(idx + (int64_t)nx * ny);
    }
}

// Masked input and the Gram (contrast) term of every face.
template <class C>
__global__ void k_rooftop_pre(const C* w, const uint8_t* act, const C* inv, C* win, C* gram, int nx, int ny, int nz) {
    const int64_t N = (int64_t)nx * ny * nz;
    const int64_t stride[3] = {1, nx, (int64_t)nx * ny};
    for (int64_t i3 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i3 < 3 * N; i3 += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i3 / N);
        const int64_t idx = i3 - a * N;
        const int coord[3] = {(int)(idx % nx), (int)((idx / nx) % ny), (int)(idx / ((int64_t)nx * ny))};
        const int n_a = a == 0 ? nx : (a == 1 ? ny : nz);
        const C* wa = w + a * N;
        const uint8_t* aa = act + a * N;
        const C v = aa[idx] ? wa[idx] : czero<C>();
        win[i3] = v;
        C g = czero<C>();
        if (aa[idx]) {
            const int64_t sa = stride[a];
            const C lo = inv[idx], hi = inv[idx + sa];           // face between c and c + e_a: both in the grid
            const C prev = coord[a] > 0 && aa[idx - sa] ? wa[idx - sa] : czero<C>();
            const C next = coord[a] + 1 < n_a && aa[idx + sa] ? wa[idx + sa] : czero<C>();
            const C lh = lo + hi;
            g = cmul(cmk<C>(0.375 * lh.x, 0.375 * lh.y), v) + cmul(cmk<C>(0.125 * lo.x, 0.125 * lo.y), prev) +
                cmul(cmk<C>(0.125 * hi.x, 0.125 * hi.y), next);
        }
        gram[i3] = g;
    }
}

template <class C>
__global__ void k_rooftop_mask(C* y, const uint8_t* act, int64_t n3) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
        if (!act[i]) y[i] = czero<C>();
}

// E_inc = pol exp(-j k0 khat . r) at the face centres of each component, 0 on inactive faces.
template <class C>
__global__ void k_rooftop_incident(C* out, const uint8_t* act, int nx, int ny, int nz, double h, double k0, double3 kh,
                                   double2 p0, double2 p1, double2 p2) {
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t i3 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i3 < 3 * N; i3 += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i3 / N);
        const int64_t idx = i3 - a * N;
        const int ix = (int)(idx % nx), iy = (int)((idx / nx) % ny), iz = (int)(idx / ((int64_t)nx * ny));
        double x = (ix + 0.5) * h - 0.5 * nx * h, y = (iy + 0.5) * h - 0.5 * ny * h, z = (iz + 0.5) * h - 0.5 * nz * h;
        if (a == 0) x += 0.5 * h;
        else if (a == 1) y += 0.5 * h;
        else z += 0.5 * h;
        double sn, cs;
        sincos(k0 * (kh.x * x + kh.y * y + kh.z * z), &sn, &cs);
        const double2 p = a == 0 ? p0 : (a == 1 ? p1 : p2);
        const double2 v = cmul(p, make_double2(cs, -sn));
        out[i3] = act[i3] ? from_c128<C>(v) : czero<C>();
    }
}

template <class C> const C* spec(const vie_rooftop* r);
template <> const double2* spec<double2>(const vie_rooftop* r) { return r->G128; }
template <> const float2* spec<float2>(const vie_rooftop* r) { return r->G64; }

template <class C>
int rooftop_mvm(vie_rooftop* r, const C* w, C* y, cudaStream_t s) {
    const vie_grid* g = r->grid;
    const int64_t N = g->N;
    C* win;
    C* gram;
    const C* inv;
    if constexpr (sizeof(C) == 16) {
        win = r->in128; gram = r->gram128; inv = r->inv128;
    } else {
        win = r->in64; gram = r->gram64; inv = r->inv64;
    }
    prof_begin(s, PK_FIELD, sizeof(C) == 16 ? VIE_C128 : VIE_C64, 0, 3 * N * (int64_t)(4 * sizeof(C) + 1), false);
    k_rooftop_pre<C><<<grid1(3 * N), 256, 0, s>>>(w, r->act, inv, win, gram, g->nx, g->ny, g->nz);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    // y = gram - u with u = (-K) w: the pencil passes with nine spectra, the update vector = the Gram term
    VIE_TRY(mvm_boxes<C>(r->bs, spec<C>(r), win, y, nullptr, s, nullptr, nullptr, gram, true));
    k_rooftop_mask<C><<<grid1(3 * N), 256, 0, s>>>(y, r->act, 3 * N);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

int wait_ev(cudaEvent_t ev, double timeout_ms) {
    if (timeout_ms <= 0) timeout_ms = 60000.0;
    auto t0 = std::chrono::steady_clock::now();
    int spins = 0;
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return VIE_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery", __FILE__, __LINE__);
        if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
        if (std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() > timeout_ms)
            return fail(VIE_ETIMEOUT, "vie_rooftop_solve: device did not finish within the wait bound");
    }
}

int read_state(vie_rooftop* r, SegState* out, cudaStream_t s, double tmo) {
    VIE_CK(cudaMemcpyAsync(r->h_st, r->st, sizeof(SegState), cudaMemcpyDeviceToHost, s));
    VIE_CK(cudaEventRecord(r->ev, s));
    VIE_TRY(wait_ev(r->ev, tmo));
    *out = *r->h_st;
    return VIE_OK;
}

}  // namespace
}  // namespace vie

using namespace vie;

extern "C" int vie_rooftop_create(vie_grid* g, double k0, int mask, vie_stream_t stream, vie_rooftop** out) {
    if (!g || !out) return fail(VIE_EINVAL, "vie_rooftop_create: null argument");
    *out = nullptr;
    if (!(k0 > 0.0) || !std::isfinite(k0)) return fail(VIE_EINVAL, "vie_rooftop_create: k0 must be positive");
    if (mask == 0 || (mask & ~(VIE_C128 | VIE_C64))) return fail(VIE_EINVAL, "vie_rooftop_create: bad precision mask");
    cudaStream_t s = (cudaStream_t)stream;
    vie_rooftop* r = new vie_rooftop();
    r->grid = g;
    r->k0 = k0;
    r->precision_mask = mask;
    auto bail = [&](int rc) {
        cudaStreamSynchronize(s);
        release(r);
        return rc;
    };
    const int64_t N = g->N, n3 = 3 * N;
    r->bs = g->full;
    r->bs.oct = false;
    r->bs.mask = nullptr;
    const int64_t vol = r->bs.spec_elems();
    int rc;
    if ((rc = ralloc(r, &r->G128, 9 * vol)) || (rc = ralloc(r, &r->inv128, N)) || (rc = ralloc(r, &r->inv64, N)) ||
        (rc = ralloc(r, &r->act, n3)) || (rc = ralloc(r, &r->bs.chi128, N)) || (rc = ralloc(r, &r->bs.chi64, N)))
        return bail(rc);
    if ((mask & VIE_C64) && ((rc = ralloc(r, &r->G64, 9 * vol)) || (rc = ralloc(r, &r->in64, n3)) ||
                             (rc = ralloc(r, &r->gram64, n3))))
        return bail(rc);
    if ((rc = ralloc(r, &r->in128, n3)) || (rc = ralloc(r, &r->gram128, n3))) return bail(rc);
    // BiCGSTAB workspace (complex128): r, rhat, p, v, s, t; y = p and z = s (no preconditioner)
    KrylovVecs<double2>& k = r->k;
    if ((rc = ralloc(r, &k.r, n3)) || (rc = ralloc(r, &k.rhat, n3)) || (rc = ralloc(r, &k.p, n3)) ||
        (rc = ralloc(r, &k.v, n3)) || (rc = ralloc(r, &k.s, n3)) || (rc = ralloc(r, &k.t, n3)) ||
        (rc = ralloc(r, &r->st, 1)) || (rc = ralloc(r, &r->red.part, (int64_t)kMaxCtaPerSeg * 2)) ||
        (rc = ralloc(r, &r->red.count, 1)) || (rc = ralloc(r, &r->red.n_active, 1)))
        return bail(rc);
    k.y = k.p;
    k.z = k.s;
    r->red.nseg = 1;
    if (cudaMemsetAsync(r->red.count, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(r->red.n_active, 0, sizeof(int), s) != cudaSuccess)
        return bail(fail(VIE_ECUDA, "vie_rooftop_create: workspace initialisation failed"));
    if (cudaHostAlloc((void**)&r->h_st, sizeof(SegState), cudaHostAllocDefault) != cudaSuccess)
        return bail(fail(VIE_ENOMEM, "vie_rooftop_create: pinned host allocation failed"));
    if (cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(VIE_ECUDA, "vie_rooftop_create: cudaEventCreate failed"));
    // "chi" of the forward pass: ones (the input is masked by the pre kernel instead)
    {
        std::vector<double2> ones(N, make_double2(1.0, 0.0));
        std::vector<float2> ones64(N, make_float2(1.f, 0.f));
        if (cudaMemcpyAsync(r->bs.chi128, ones.data(), N * sizeof(double2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(r->bs.chi64, ones64.data(), N * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return bail(fail(VIE_ECUDA, "vie_rooftop_create: upload failed"));
    }
    k_rooftop_tables<<<grid1(N), 256, 0, s>>>(g->full.chi128, r->act, r->inv128, r->inv64, g->nx, g->ny, g->nz);
    // cell integral of g over the equivalent sphere: [(1 + jka) e^{-jka} - 1] / k^2
    const double a = g->h * std::cbrt(3.0 / (4.0 * 3.14159265358979323846));
    const double ka = k0 * a, c = std::cos(ka), sn = std::sin(ka);
    const double2 self = make_double2((c + ka * sn - 1.0) / (k0 * k0), (ka * c - sn) / (k0 * k0));
    const BoxSet& bs = r->bs;
    k_rooftop_sample<<<grid1(vol), 256, 0, s>>>(r->G128, bs.Mx, bs.My, bs.Mz, g->nx, g->ny, g->nz, g->h, k0, self,
                                                 1.0 / (double)vol);
    if (cudaGetLastError() != cudaSuccess) return bail(fail(VIE_ECUDA, "vie_rooftop_create: launch failed"));
    if ((rc = spectrum_fft<double2>(bs, r->G128, s, nullptr, 9))) return bail(rc);
    if ((mask & VIE_C64) && (rc = convert_c128_to_c64(r->G128, r->G64, 9 * vol, s))) return bail(rc);
    *out = r;
    return VIE_OK;
}

extern "C" int vie_rooftop_release(vie_rooftop* r) {
    if (!r) return fail(VIE_EINVAL, "vie_rooftop_release: null operator");
    cudaDeviceSynchronize();
    release(r);
    return VIE_OK;
}

extern "C" int vie_rooftop_incident(const vie_rooftop* r, const double* khat, const double* pol, int precision,
                                    void* out, vie_stream_t stream) {
    if (!r || !khat || !pol || !out) return fail(VIE_EINVAL, "vie_rooftop_incident: null argument");
    if (precision != VIE_C128 && precision != VIE_C64) return fail(VIE_EINVAL, "vie_rooftop_incident: bad precision");
    const vie_grid* g = r->grid;
    cudaStream_t s = (cudaStream_t)stream;
    const double3 kh = make_double3(khat[0], khat[1], khat[2]);
    const double2 p0 = make_double2(pol[0], pol[1]), p1 = make_double2(pol[2], pol[3]), p2 = make_double2(pol[4], pol[5]);
    if (precision == VIE_C128)
        k_rooftop_incident<double2><<<grid1(3 * g->N), 256, 0, s>>>((double2*)out, r->act, g->nx, g->ny, g->nz, g->h,
                                                                    r->k0, kh, p0, p1, p2);
    else
        k_rooftop_incident<float2><<<grid1(3 * g->N), 256, 0, s>>>((float2*)out, r->act, g->nx, g->ny, g->nz, g->h,
                                                                   r->k0, kh, p0, p1, p2);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

extern "C" int vie_rooftop_matvec(vie_rooftop* r, int precision, const void* w, void* y, vie_stream_t stream) {
    if (!r || !w || !y) return fail(VIE_EINVAL, "vie_rooftop_matvec: null argument");
    const int64_t n3 = 3 * r->grid->N;
    const int64_t es = precision == VIE_C128 ? 16 : 8;
    const char* a = (const char*)w;
    const char* b = (const char*)y;
    if (a < b + n3 * es && b < a + n3 * es) return fail(VIE_EINVAL, "vie_rooftop_matvec: w and y overlap");
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == VIE_C128) return rooftop_mvm<double2>(r, (const double2*)w, (double2*)y, s);
    if (precision == VIE_C64) {
        if (!(r->precision_mask & VIE_C64)) return fail(VIE_EINVAL, "vie_rooftop_matvec: operator built without VIE_C64");
        return rooftop_mvm<float2>(r, (const float2*)w, (float2*)y, s);
    }
    return fail(VIE_EINVAL, "vie_rooftop_matvec: bad precision");
}

extern "C" int vie_rooftop_solve(vie_rooftop* r, const void* b_dev, void* w_dev, double tol, int32_t maxit,
                                 double wait_timeout_ms, vie_stream_t stream, vie_solve_stats* stats) {
    if (!r || !b_dev || !w_dev) return fail(VIE_EINVAL, "vie_rooftop_solve: null argument");
    if (!(tol > 0.0) || maxit < 1) return fail(VIE_EINVAL, "vie_rooftop_solve: bad tolerance or maxit");
    const int64_t n3 = 3 * r->grid->N;
    const char* a = (const char*)b_dev;
    const char* b = (const char*)w_dev;
    if (a < b + n3 * 16 && b < a + n3 * 16) return fail(VIE_EINVAL, "vie_rooftop_solve: b and w overlap");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    Bicg<double2> k;
    k.nseg = 1;
    k.seglen = n3;
    k.v = r->k;
    k.v.b = const_cast<double2*>((const double2*)b_dev);
    k.v.x = (double2*)w_dev;
    k.st = r->st;
    k.red = &r->red;
    int mv = 0;
    VIE_TRY(bicg_init<double2>(k, tol, maxit, s));
    SegState hs;
    VIE_TRY(read_state(r, &hs, s, wait_timeout_ms));
    for (int it = 0; it < maxit && hs.status == SEG_ACTIVE; ++it) {
        VIE_TRY(bicg_rho<double2>(k, s));
        VIE_TRY(bicg_update_p<double2>(k, s));
        VIE_TRY(rooftop_mvm<double2>(r, k.v.y, k.v.v, s));
        ++mv;
        VIE_TRY(bicg_sigma<double2>(k, s));
        VIE_TRY(bicg_update_s<double2>(k, s));
        VIE_TRY(bicg_x_half<double2>(k, s));
        VIE_TRY(read_state(r, &hs, s, wait_timeout_ms));
        if (hs.status != SEG_ACTIVE) break;
        VIE_TRY(rooftop_mvm<double2>(r, k.v.z, k.v.t, s));
        ++mv;
        VIE_TRY(bicg_omega<double2>(k, s));
        VIE_TRY(bicg_update_xr<double2>(k, s));
        VIE_TRY(read_state(r, &hs, s, wait_timeout_ms));
    }
    VIE_TRY(read_state(r, &hs, s, wait_timeout_ms));
    int rc = hs.status == SEG_CONVERGED ? VIE_OK : (hs.status == SEG_BREAKDOWN ? VIE_EBREAKDOWN : VIE_ENOTCONV);
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->outer_iters = hs.iters;
        stats->matvecs_c128 = mv;
        stats->true_rel_res = hs.bnorm2 > 0 ? std::sqrt(hs.res2 / hs.bnorm2) : 0.0;   // recursive residual
        stats->status = rc;
        stats->elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return rc;
}

extern "C" int vie_rooftop_far_field_rcs(const vie_rooftop* r, const void* w_dev, int32_t ndir, const double* dirs,
                                         double* rcs, vie_stream_t stream) {
    if (!r || !w_dev) return fail(VIE_EINVAL, "vie_rooftop_far_field_rcs: null argument");
    const vie_grid* g = r->grid;
    // faces sit half a cell above the cell centres along their own axis
    const double shift[3] = {0.5 * g->h, 0.5 * g->h, 0.5 * g->h};
    return far_field_rcs_impl(g->nx, g->ny, g->nz, g->h, r->k0, (const double2*)w_dev, r->bs.chi128, shift, ndir, dirs,
                              rcs, (cudaStream_t)stream);
}
