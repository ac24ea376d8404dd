// Field-level kernels: Green-tensor lattice samples (Eq. 1), incident plane
// wave, precision conversion, and the block restriction/prolongation of the
// block-diagonal preconditioner (Eq. 10).
#include <math.h>

#include <cmath>

#include "vie_internal.cuh"

namespace vie {

static unsigned grid_1d(int64_t n, int per_thread = 1) {
    int64_t g = (n + 256LL * per_thread - 1) / (256LL * per_thread);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

// Slot m of an axis of padded length M stores lattice offset m (m < b) or
// m - M (m > M - b); other slots are unused by any product of two in-box
// voxels (circulant embedding of the Toeplitz sum) and hold zero.
__device__ __forceinline__ bool wrap_offset(int m, int M, int b, int& d) {
    if (m < b) { d = m; return true; }
    if (m > M - b) { d = m - M; return true; }
    return false;
}

// The six components of k0^2 G(r) h^3 `scale` at a point r != 0 (Eq. 1:
// k^2 G = g [(k^2 - jk/R - 1/R^2) I + (-k^2 + 3jk/R + 3/R^2) rhat rhat]), added to K.
__device__ __forceinline__ void add_k2G(double rx, double ry, double rz, double k0, double hs, double wgt,
                                        double2 (&K)[6]) {
    const double inv4pi = 0.25 / 3.14159265358979323846;
    const double R2 = rx * rx + ry * ry + rz * rz;
    const double R = sqrt(R2);
    double sn, cs;
    sincos(k0 * R, &sn, &cs);
    // g h^3 scale = e^{-jkR} / (4 pi R) h^3 scale
    const double gm = inv4pi / R * hs * wgt;
    const double2 g = make_double2(cs * gm, -sn * gm);
    const double2 a = make_double2(k0 * k0 - 1.0 / R2, -k0 / R);
    const double2 b = make_double2(-k0 * k0 + 3.0 / R2, 3.0 * k0 / R);
    const double2 ga = cmul(g, a), gb = cmul(g, b);
    const double u[3] = {rx / R, ry / R, rz / R};
    const int P[6] = {0, 0, 0, 1, 1, 2}, Q[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const double uu = u[P[c]] * u[Q[c]];
        double2 v = make_double2(gb.x * uu, gb.y * uu);
        if (P[c] == Q[c]) v = v + ga;
        K[c] = K[c] + v;
    }
}

// K(D) = k0^2 G(D h) h^3 for D != 0 and s_self I at D = 0, times `scale`
// (1 / (Mx My Mz), the inverse-FFT normalisation folded into the spectrum);
// offsets with 0 < max|D| <= near.radius take the mean of k0^2 G over the cube
// of side h around D h instead (tensor Gauss-Legendre rule of order near.q).
// Output: natural order [6][Mz][My][Mx], components xx, xy, xz, yy, yz, zz.
__global__ void k_green_sample(double2* G, int Mx, int My, int Mz, int bx, int by, int bz,
                               double k0, double h, double scale, double2 self, NearRule near) {
    const int64_t vol = (int64_t)Mx * My * Mz;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < vol;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int ix = (int)(idx % Mx);
        int iy = (int)((idx / Mx) % My);
        int iz = (int)(idx / ((int64_t)Mx * My));
        int dx, dy, dz;
        double2 K[6];
        for (int c = 0; c < 6; ++c) K[c] = make_double2(0.0, 0.0);
        bool used = wrap_offset(ix, Mx, bx, dx) & wrap_offset(iy, My, by, dy) & wrap_offset(iz, Mz, bz, dz);
        if (used) {
            if (dx == 0 && dy == 0 && dz == 0) {
                double2 sd = make_double2(self.x * scale, self.y * scale);
                K[0] = sd;
                K[3] = sd;
                K[5] = sd;
            } else {
                const double hs = h * h * h * scale;
                const int dmax = max(abs(dx), max(abs(dy), abs(dz)));
                if (dmax <= near.radius) {
                    // mean over the cube: weights w_i w_j w_l / 8 of the rule on [-1, 1]^3
                    for (int l = 0; l < near.q; ++l)
                        for (int j = 0; j < near.q; ++j)
                            for (int i = 0; i < near.q; ++i)
                                add_k2G((dx + 0.5 * near.t[i]) * h, (dy + 0.5 * near.t[j]) * h,
                                        (dz + 0.5 * near.t[l]) * h, k0, hs,
                                        0.125 * near.w[i] * near.w[j] * near.w[l], K);
                } else {
                    add_k2G(dx * h, dy * h, dz * h, k0, hs, 1.0, K);
                }
            }
        }
        for (int c = 0; c < 6; ++c) G[c * vol + idx] = K[c];
    }
}

// Gauss-Legendre rule of order q on [-1, 1]: the nodes are the roots of the Legendre polynomial
// P_q, found by Newton's method from the Chebyshev-like first guesses cos(pi (i + 3/4) / (q + 1/2)),
// with P_q and P_q' from the three-term recurrence; weights 2 / ((1 - t^2) P_q'(t)^2).
int near_rule(int radius, int q, NearRule* out) {
    NearRule r;
    if (radius < 0 || radius > 8) return fail(VIE_EINVAL, "near-field radius must be in [0, 8]");
    r.radius = radius;
    if (radius == 0) {
        *out = r;
        return VIE_OK;
    }
    if (q < 1 || q > kNearMaxOrder) return fail(VIE_EINVAL, "near-field quadrature order must be in [1, 16]");
    r.q = q;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < q; ++i) {
        double t = std::cos(pi * (i + 0.75) / (q + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;                 // P_0, P_1
            for (int n = 2; n <= q; ++n) {
                const double p2 = ((2.0 * n - 1.0) * t * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            const double pq = q == 1 ? t : p1, pm = q == 1 ? 1.0 : p0;   // P_q, P_{q-1}
            dp = q * (t * pq - pm) / (t * t - 1.0);                      // P_q'
            const double dt = pq / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-16) break;
        }
        // recompute the derivative at the converged node
        double p0 = 1.0, p1 = t;
        for (int n = 2; n <= q; ++n) {
            const double p2 = ((2.0 * n - 1.0) * t * p1 - (n - 1.0) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        const double pq = q == 1 ? t : p1, pm = q == 1 ? 1.0 : p0;
        dp = q * (t * pq - pm) / (t * t - 1.0);
        r.t[i] = t;
        r.w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
    *out = r;
    return VIE_OK;
}

int green_sample(const BoxSet& bs, double k0, double h, double2* G, cudaStream_t s, const NearRule* near) {
    // equivalent-sphere self term: (2/3)[(1 + jka) e^{-jka} - 1] - 1/3
    const double a = h * cbrt(3.0 / (4.0 * 3.14159265358979323846));
    const double ka = k0 * a;
    const double c = cos(ka), sn = sin(ka);
    // (1 + j ka)(c - j sn) = c + ka sn + j (ka c - sn)
    double2 self = make_double2((2.0 / 3.0) * (c + ka * sn - 1.0) - 1.0 / 3.0, (2.0 / 3.0) * (ka * c - sn));
    const double scale = 1.0 / ((double)bs.Mx * bs.My * bs.Mz);
    prof_begin(s, PK_SPECTRUM, VIE_C128, 0, 6 * bs.spec_elems() * 16, false);
    const NearRule rule = near ? *near : NearRule();
    k_green_sample<<<grid_1d(bs.spec_elems()), 256, 0, s>>>(G, bs.Mx, bs.My, bs.Mz, bs.bx, bs.by, bs.bz,
                                                            k0, h, scale, self, rule);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

__global__ void k_c128_to_c64(const double2* a, float2* b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
int convert_c128_to_c64(const double2* a, float2* b, int64_t n, cudaStream_t s) {
    prof_begin(s, PK_SPECTRUM, VIE_C64, 0, n * 24, false);
    k_c128_to_c64<<<grid_1d(n), 256, 0, s>>>(a, b, n);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

// E_inc = pol exp(-j k0 khat . r), r the voxel centre relative to the grid centre.
template <class C>
__global__ void k_plane_wave(C* out, int nx, int ny, int nz, double h, double k0, double3 kh,
                             double2 p0, double2 p1, double2 p2) {
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int ix = (int)(idx % nx), iy = (int)((idx / nx) % ny), iz = (int)(idx / ((int64_t)nx * ny));
        double x = (ix + 0.5) * h - 0.5 * nx * h;
        double y = (iy + 0.5) * h - 0.5 * ny * h;
        double z = (iz + 0.5) * h - 0.5 * nz * h;
        double sn, cs;
        sincos(k0 * (kh.x * x + kh.y * y + kh.z * z), &sn, &cs);
        double2 ph = make_double2(cs, -sn);
        out[idx] = from_c128<C>(cmul(p0, ph));
        out[N + idx] = from_c128<C>(cmul(p1, ph));
        out[2 * N + idx] = from_c128<C>(cmul(p2, ph));
    }
}

int plane_wave_launch(const vie_grid* g, double k0, const double* khat, const double* pol,
                      int precision, void* out, cudaStream_t s) {
    double3 kh = make_double3(khat[0], khat[1], khat[2]);
    double2 p0 = make_double2(pol[0], pol[1]), p1 = make_double2(pol[2], pol[3]), p2 = make_double2(pol[4], pol[5]);
    prof_begin(s, PK_FIELD, precision, 0, 3 * g->N * (precision == VIE_C128 ? 16 : 8), false);
    if (precision == VIE_C128)
        k_plane_wave<double2><<<grid_1d(g->N), 256, 0, s>>>((double2*)out, g->nx, g->ny, g->nz, g->h, k0, kh, p0, p1, p2);
    else
        k_plane_wave<float2><<<grid_1d(g->N), 256, 0, s>>>((float2*)out, g->nx, g->ny, g->nz, g->h, k0, kh, p0, p1, p2);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

// ---------------------------------------------------------------- block restriction / prolongation
// b_k = b restricted to the voxels S_k of block k, laid out in the block's box
// [nb][3][bz][by][bx]; zero outside S_k.
template <class C>
__global__ void k_gather(const C* src, C* out, const uint8_t* mask, const int32_t* origin,
                         int nb, int bx, int by, int bz, int nx, int ny, int nz) {
    const int64_t box = (int64_t)bx * by * bz;
    const int64_t total = (int64_t)nb * 3 * box;
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = idx % box;
        int64_t bc = idx / box;
        int c = (int)(bc % 3), b = (int)(bc / 3);
        C v = czero<C>();
        if (mask[(int64_t)b * box + l]) {
            int lx = (int)(l % bx), ly = (int)((l / bx) % by), lz = (int)(l / ((int64_t)bx * by));
            int gx = origin[3 * b] + lx, gy = origin[3 * b + 1] + ly, gz = origin[3 * b + 2] + lz;
            v = src[c * N + ((int64_t)gz * ny + gy) * nx + gx];
        }
        out[idx] = v;
    }
}

// y = x_k on the voxels of block k (mask 1; the blocks are disjoint, so no write conflicts). Halo
// voxels of an expanded block (mask 2) belong to another block or to none and are not written.
template <class C>
__global__ void k_scatter(const C* xk, C* y, const uint8_t* mask, const int32_t* origin,
                          int nb, int bx, int by, int bz, int nx, int ny, int nz) {
    const int64_t box = (int64_t)bx * by * bz;
    const int64_t total = (int64_t)nb * 3 * box;
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = idx % box;
        int64_t bc = idx / box;
        int c = (int)(bc % 3), b = (int)(bc / 3);
        if (mask[(int64_t)b * box + l] != 1) continue;
        int lx = (int)(l % bx), ly = (int)((l / bx) % by), lz = (int)(l / ((int64_t)bx * by));
        int gx = origin[3 * b] + lx, gy = origin[3 * b + 1] + ly, gz = origin[3 * b + 2] + lz;
        y[c * N + ((int64_t)gz * ny + gy) * nx + gx] = xk[idx];
    }
}

// y = b on voxels that belong to no block (identity part of K2).
template <class C>
__global__ void k_copy_unblocked(const C* b, C* y, const int32_t* block_id, int64_t N) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (int64_t)gridDim.x * blockDim.x) {
        if (block_id[idx] < 0) {
            y[idx] = b[idx];
            y[N + idx] = b[N + idx];
            y[2 * N + idx] = b[2 * N + idx];
        }
    }
}

template <class C>
int precond_gather(const vie_grid* g, const Group& gr, const C* b, C* out, cudaStream_t s) {
    const BoxSet& bs = gr.bs;
    prof_begin(s, PK_FIELD, sizeof(C) == 16 ? VIE_C128 : VIE_C64, 0, 2 * bs.nb * bs.vec_elems() * (int64_t)sizeof(C), false);
    k_gather<C><<<grid_1d(bs.nb * bs.vec_elems()), 256, 0, s>>>(b, out, bs.mask, bs.origin, bs.nb, bs.bx, bs.by,
                                                                bs.bz, g->nx, g->ny, g->nz);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <class C>
int precond_scatter_group(const vie_grid* g, const Group& gr, const C* xk, C* y, cudaStream_t s) {
    const BoxSet& bs = gr.bs;
    prof_begin(s, PK_FIELD, sizeof(C) == 16 ? VIE_C128 : VIE_C64, 0, 2 * bs.nb * bs.vec_elems() * (int64_t)sizeof(C), false);
    k_scatter<C><<<grid_1d(bs.nb * bs.vec_elems()), 256, 0, s>>>(xk, y, bs.mask, bs.origin, bs.nb, bs.bx, bs.by,
                                                                 bs.bz, g->nx, g->ny, g->nz);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <class C>
int precond_copy_unblocked(const vie_grid* g, const C* b, C* y, cudaStream_t s) {
    prof_begin(s, PK_FIELD, sizeof(C) == 16 ? VIE_C128 : VIE_C64, 0, g->N * 4 + 6 * g->N * (int64_t)sizeof(C), false);
    k_copy_unblocked<C><<<grid_1d(g->N), 256, 0, s>>>(b, y, g->block_id, g->N);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template int precond_gather<double2>(const vie_grid*, const Group&, const double2*, double2*, cudaStream_t);
template int precond_gather<float2>(const vie_grid*, const Group&, const float2*, float2*, cudaStream_t);
template int precond_scatter_group<double2>(const vie_grid*, const Group&, const double2*, double2*, cudaStream_t);
template int precond_scatter_group<float2>(const vie_grid*, const Group&, const float2*, float2*, cudaStream_t);
template int precond_copy_unblocked<double2>(const vie_grid*, const double2*, double2*, cudaStream_t);
template int precond_copy_unblocked<float2>(const vie_grid*, const float2*, float2*, cudaStream_t);

}  // namespace vie
