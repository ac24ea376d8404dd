// Far-zone scattered field and bistatic RCS of a solved total field (the
// far-zone limit of E_s = k0^2 int G chi E dv, Eq. 1 with J = j w eps0 chi E;
// the RCS comparisons of Section III, Figs. 1-2):
//   P(u)     = sum_j chi_j E_j h^3 exp(j k0 u . r_j)
//   sigma(u) = k0^4 / (4 pi) |(I - u u) P(u)|^2
// over voxel centres r_j = ((i + 1/2) h - n h / 2) per axis. The phase is
// separable, exp(j k0 (ux x + uy y + uz z)) = ex(x) ey(y) ez(z), so each CTA
// (one direction, one slab of z planes) tabulates the three 1D factors in
// shared memory and the voxel loop is two complex multiplies per voxel;
// partial sums are FP64 and are added on the host in a fixed order.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "vie_internal.cuh"

namespace vie {
namespace {

constexpr int kFfThreads = 256;
constexpr int kFfSlabs = 16;   // z slabs per direction (CTAs per direction)

__global__ void __launch_bounds__(kFfThreads) k_far_field(const double2* E, const double2* chi, const double3* dirs,
                                                           int nx, int ny, int nz, double h, double k0,
                                                           double2* partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* ex = reinterpret_cast<double2*>(smem_raw);    // [nx]
    double2* ey = ex + nx;                                  // [ny]
    double2* ez = ey + ny;                                  // [nz]
    double2* red = ez + nz;                                 // [3][kFfThreads / 32]
    const int d = blockIdx.x, slab = blockIdx.y;
    const double3 u = dirs[d];
    const double kh = k0 * h;
    for (int i = threadIdx.x; i < nx + ny + nz; i += blockDim.x) {
        double w, n, c;
        if (i < nx) { w = u.x; n = nx; c = i; }
        else if (i < nx + ny) { w = u.y; n = ny; c = i - nx; }
        else { w = u.z; n = nz; c = i - nx - ny; }
        double sn, cs;
        sincos(kh * w * (c + 0.5 - 0.5 * n), &sn, &cs);
        ex[i] = make_double2(cs, sn);
    }
    __syncthreads();
    const int z0 = (int)((int64_t)nz * slab / gridDim.y), z1 = (int)((int64_t)nz * (slab + 1) / gridDim.y);
    const int64_t N = (int64_t)nx * ny * nz;
    const int64_t plane = (int64_t)nx * ny;
    double2 acc[3] = {make_double2(0, 0), make_double2(0, 0), make_double2(0, 0)};
    for (int64_t l = (int64_t)z0 * plane + threadIdx.x; l < (int64_t)z1 * plane; l += blockDim.x) {
        const int z = (int)(l / plane);
        const int64_t r = l - z * plane;
        const int y = (int)(r / nx), x = (int)(r - (int64_t)y * nx);
        const double2 ph = cmul(cmul(ex[x], ey[y]), ez[z]);
        const double2 w = cmul(chi[l], ph);
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = acc[c] + cmul(w, E[c * N + l]);
    }
    // CTA sum in a fixed order: warp shuffles, then warp 0 over the warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double2 v = acc[c];
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
        if (lane == 0) red[c * nw + warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double2 v = make_double2(0, 0);
        for (int k = 0; k < nw; ++k) v = v + red[threadIdx.x * nw + k];
        partial[((int64_t)d * gridDim.y + slab) * 3 + threadIdx.x] = v;
    }
}

}  // namespace
}  // namespace vie

using namespace vie;

extern "C" int vie_far_field_rcs(const vie_grid* g, double k0, const void* e_dev, int32_t ndir, const double* dirs_host,
                                 double* rcs_host, vie_stream_t stream) {
    if (!g || !e_dev || !dirs_host || !rcs_host) return fail(VIE_EINVAL, "vie_far_field_rcs: null argument");
    return far_field_rcs_impl(g->nx, g->ny, g->nz, g->h, k0, (const double2*)e_dev, g->full.chi128, nullptr, ndir,
                              dirs_host, rcs_host, (cudaStream_t)stream);
}

namespace vie {

// P(u) = sum_j w_j E_j h^3 exp(j k0 u . (r_j + shift_c e_c)) per component c (w = chi for the
// collocation field; w = 1 and shift = h/2 for rooftop currents on faces), then the RCS.
int far_field_rcs_impl(int nx, int ny, int nz, double h, double k0, const double2* e_dev, const double2* wts,
                       const double* shift, int32_t ndir, const double* dirs_host, double* rcs_host, cudaStream_t s) {
    if (!e_dev || !dirs_host || !rcs_host) return fail(VIE_EINVAL, "vie_far_field_rcs: null argument");
    if (ndir < 1 || ndir > (1 << 20)) return fail(VIE_EINVAL, "vie_far_field_rcs: ndir must be in [1, 2^20]");
    if (!(k0 > 0.0) || !std::isfinite(k0)) return fail(VIE_EINVAL, "vie_far_field_rcs: k0 must be positive");
    std::vector<double3> dirs(ndir);
    for (int i = 0; i < ndir; ++i) {
        const double ux = dirs_host[3 * i], uy = dirs_host[3 * i + 1], uz = dirs_host[3 * i + 2];
        const double n2 = ux * ux + uy * uy + uz * uz;
        if (!(std::fabs(n2 - 1.0) <= 1e-9)) return fail(VIE_EINVAL, "vie_far_field_rcs: directions must be unit vectors");
        dirs[i] = make_double3(ux, uy, uz);
    }
    const int slabs = std::min(kFfSlabs, nz);
    double3* d_dirs = nullptr;
    double2* d_part = nullptr;
    const size_t part_n = (size_t)ndir * slabs * 3;
    VIE_CK(cudaMallocAsync((void**)&d_dirs, ndir * sizeof(double3), s));
    cudaError_t e = cudaMallocAsync((void**)&d_part, part_n * sizeof(double2), s);
    int rc = VIE_OK;
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMallocAsync", __FILE__, __LINE__);
    std::vector<double2> part(part_n);
    if (!rc) {
        e = cudaMemcpyAsync(d_dirs, dirs.data(), ndir * sizeof(double3), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync", __FILE__, __LINE__);
    }
    if (!rc) {
        const size_t smem = (size_t)(nx + ny + nz + 3 * (kFfThreads / 32)) * sizeof(double2);
        prof_begin(s, PK_FIELD, VIE_C128, 0, (int64_t)ndir * nx * ny * nz * 64, false);
        k_far_field<<<dim3(ndir, slabs), kFfThreads, smem, s>>>(e_dev, wts, d_dirs, nx, ny, nz, h, k0, d_part);
        prof_end(s);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "k_far_field launch", __FILE__, __LINE__);
    }
    if (!rc) {
        e = cudaMemcpyAsync(part.data(), d_part, part_n * sizeof(double2), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "far-field read-back", __FILE__, __LINE__);
    }
    if (d_part) cudaFreeAsync(d_part, s);
    if (d_dirs) cudaFreeAsync(d_dirs, s);
    if (rc) return rc;
    const double h3 = h * h * h;
    const double pref = k0 * k0 * k0 * k0 / (4.0 * 3.141592653589793238462643383279502884);
    for (int i = 0; i < ndir; ++i) {
        double2 P[3];
        for (int c = 0; c < 3; ++c) {
            P[c] = make_double2(0.0, 0.0);
            for (int sl = 0; sl < slabs; ++sl) P[c] = P[c] + part[((size_t)i * slabs + sl) * 3 + c];
            P[c] = make_double2(P[c].x * h3, P[c].y * h3);
        }
        const double3 u = dirs[i];
        if (shift) {
            const double uc[3] = {u.x, u.y, u.z};
            for (int c = 0; c < 3; ++c) {
                double sn, cs;
                sincos(k0 * uc[c] * shift[c], &sn, &cs);
                P[c] = cmul(P[c], make_double2(cs, sn));
            }
        }
        // (I - u u) P = P - u (u . P)
        const double2 up = make_double2(u.x * P[0].x + u.y * P[1].x + u.z * P[2].x,
                                        u.x * P[0].y + u.y * P[1].y + u.z * P[2].y);
        const double uu[3] = {u.x, u.y, u.z};
        double s2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double tx = P[c].x - uu[c] * up.x, ty = P[c].y - uu[c] * up.y;
            s2 += tx * tx + ty * ty;
        }
        rcs_host[i] = pref * s2;
    }
    return VIE_OK;
}

}  // namespace vie
