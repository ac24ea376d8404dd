// Batched BiCGSTAB building blocks (Section II.B; van der Vorst's method, ref. [18]).
//
// A "segment" is one independent linear system: the outer system (one
// segment, the whole grid) or one diagonal block A_k of Eq. 10 (one segment
// per block, all blocks of a group stored back to back). Every kernel runs a
// 2D grid (CTAs within a segment) x (segments); each segment's scalars live in
// a SegState on the device, so the host never reads rho, alpha or omega.
//
// Reductions: each CTA writes its partial sums, and the last CTA of the
// segment to arrive (atomic ticket) adds all partials in a fixed order and
// applies the scalar update, so results are deterministic. Complex64 vectors
// are multiplied and summed in FP32 within a thread and in FP64 across
// threads; complex128 vectors use FP64 throughout. Scalars are FP64.
#include <math.h>

#include "vie_internal.cuh"

namespace vie {

constexpr int kRedThreads = 256;

enum VecOp { OP_INIT = 0, OP_P, OP_S, OP_XHALF, OP_XR, OP_RHO, OP_SIGMA, OP_OMEGA };

template <class C> struct VecArgs {
    KrylovVecs<C> v;
    SegState* st;
    double2* part;      // [nseg][maxcta][2]
    unsigned* count;    // [nseg]
    int* n_active;
    int64_t seglen;
    int maxcta;
    double tol;
    int maxit;
    int* units;         // profiling: active segments processed
    const double* tols; // optional per-segment relative tolerance (OP_INIT)
};

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ bool cfinite_nz(double2 a) {
    return isfinite(a.x) && isfinite(a.y) && (a.x != 0.0 || a.y != 0.0);
}

template <class C> struct Acc;
template <> struct Acc<double2> {
    typedef double2 T;
    static __device__ __forceinline__ double2 widen(double2 a) { return a; }
};
template <> struct Acc<float2> {
    typedef float2 T;
    static __device__ __forceinline__ double2 widen(float2 a) { return make_double2(a.x, a.y); }
};

// conj(a) * b accumulated into acc (same precision as the vectors)
template <class C> __device__ __forceinline__ void cdot_acc(C& acc, C a, C b) {
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// Deterministic block sum of two complex values; result valid in thread 0.
__device__ void block_sum2(double2& a, double2& b) {
    __shared__ double2 sh[2][kRedThreads / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = a; sh[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = l < nw ? sh[0][l] : make_double2(0, 0);
        b = l < nw ? sh[1][l] : make_double2(0, 0);
        a = warp_sum(a);
        b = warp_sum(b);
    }
    __syncthreads();
}

__device__ __forceinline__ void leave_active(int* n_active) { atomicSub(n_active, 1); }

// Scalar update of one segment, run by thread 0 of the last CTA.
template <int OP>
__device__ void finalize(SegState& s, double2 d1, double2 d2, int* n_active, double tol, int maxit) {
    // (tol already resolved per segment by the caller)
    if (OP == OP_INIT) {
        s.bnorm2 = d1.x;
        s.tol2 = tol * tol * d1.x;
        s.res2 = d1.x;
        s.rho = s.rho_prev = s.alpha = s.omega = make_double2(1.0, 0.0);
        s.iters = 0.0;
        s.maxit = maxit;
        if (!isfinite(d1.x)) {
            s.status = SEG_BREAKDOWN;
        } else if (d1.x == 0.0 || d1.x <= s.tol2) {   // x0 already meets the tolerance (tol >= 1)
            s.status = SEG_CONVERGED;
        } else {
            s.status = SEG_ACTIVE;
            atomicAdd(n_active, 1);
        }
    } else if (OP == OP_RHO) {
        s.rho = d1;
        if (!cfinite_nz(d1)) { s.status = SEG_BREAKDOWN; leave_active(n_active); }
    } else if (OP == OP_SIGMA) {
        if (!cfinite_nz(d1)) { s.status = SEG_BREAKDOWN; leave_active(n_active); }
        else s.alpha = cdiv(s.rho, d1);
    } else if (OP == OP_OMEGA) {
        if (!(d2.x > 0.0) || !isfinite(d2.x) || !isfinite(d1.x) || !isfinite(d1.y)) {
            s.status = SEG_BREAKDOWN;
            leave_active(n_active);
        } else {
            s.omega = make_double2(d1.x / d2.x, d1.y / d2.x);
        }
    } else if (OP == OP_S) {
        s.res2 = d1.x;
        if (!isfinite(d1.x)) { s.status = SEG_BREAKDOWN; leave_active(n_active); }
        else if (d1.x <= s.tol2) { s.status = SEG_HALF_PENDING; s.iters += 0.5; leave_active(n_active); }
    } else if (OP == OP_XHALF) {
        s.status = SEG_CONVERGED;
    } else if (OP == OP_XR) {
        s.res2 = d1.x;
        s.iters += 1.0;
        s.rho_prev = s.rho;
        if (!isfinite(d1.x)) { s.status = SEG_BREAKDOWN; leave_active(n_active); }
        else if (d1.x <= s.tol2) { s.status = SEG_CONVERGED; leave_active(n_active); }
        else if (s.iters >= (double)s.maxit) { s.status = SEG_MAXIT; leave_active(n_active); }
        else if (s.omega.x == 0.0 && s.omega.y == 0.0) { s.status = SEG_BREAKDOWN; leave_active(n_active); }
    }
}

// One fused pass over a segment: vector update and/or up to two inner products.
template <class C, int OP>
__global__ void __launch_bounds__(kRedThreads) k_bicg(VecArgs<C> a) {
    const int seg = blockIdx.y;
    SegState& S = a.st[seg];
    if (OP != OP_INIT) {
        const int need = (OP == OP_XHALF) ? SEG_HALF_PENDING : SEG_ACTIVE;
        if (S.status != need) return;       // same value for every CTA of the segment
    }
    if (a.units != nullptr && threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(a.units, 1);
    const int64_t off = (int64_t)seg * a.seglen;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    C acc1 = czero<C>(), acc2 = czero<C>();

    C alpha = cmk<C>(S.alpha.x, S.alpha.y), omega = cmk<C>(S.omega.x, S.omega.y), beta = czero<C>();
    if (OP == OP_P) {
        double2 bt = cmul(cdiv(S.rho, S.rho_prev), cdiv(S.alpha, S.omega));
        beta = cmk<C>(bt.x, bt.y);
    }
    KrylovVecs<C> v = a.v;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.seglen; i += stride) {
        const int64_t k = off + i;
        if (OP == OP_INIT) {
            C b = v.b[k];
            v.x[k] = czero<C>();
            v.r[k] = b;
            v.rhat[k] = b;
            v.p[k] = czero<C>();
            v.v[k] = czero<C>();
            cdot_acc(acc1, b, b);
        } else if (OP == OP_P) {
            v.p[k] = v.r[k] + cmul(beta, v.p[k] - cmul(omega, v.v[k]));
        } else if (OP == OP_S) {
            C s = v.r[k] - cmul(alpha, v.v[k]);
            v.s[k] = s;
            cdot_acc(acc1, s, s);
        } else if (OP == OP_XHALF) {
            v.x[k] = v.x[k] + cmul(alpha, v.y[k]);
        } else if (OP == OP_XR) {
            v.x[k] = v.x[k] + cmul(alpha, v.y[k]) + cmul(omega, v.z[k]);
            C r = v.s[k] - cmul(omega, v.t[k]);
            v.r[k] = r;
            cdot_acc(acc1, r, r);
        } else if (OP == OP_RHO) {
            cdot_acc(acc1, v.rhat[k], v.r[k]);
        } else if (OP == OP_SIGMA) {
            cdot_acc(acc1, v.rhat[k], v.v[k]);
        } else if (OP == OP_OMEGA) {
            C t = v.t[k];
            cdot_acc(acc1, t, v.s[k]);
            cdot_acc(acc2, t, t);
        }
    }
    double2 d1 = Acc<C>::widen(acc1), d2 = Acc<C>::widen(acc2);
    block_sum2(d1, d2);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double2* pp = a.part + ((int64_t)seg * a.maxcta + blockIdx.x) * 2;
        pp[0] = d1;
        pp[1] = d2;
        __threadfence();
        unsigned ticket = atomicAdd(&a.count[seg], 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // fixed-order sum of the partials of this segment
    double2 s1 = make_double2(0, 0), s2 = make_double2(0, 0);
    const volatile double2* pp = a.part + (int64_t)seg * a.maxcta * 2;
    for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x) {
        s1.x += pp[2 * c].x; s1.y += pp[2 * c].y;
        s2.x += pp[2 * c + 1].x; s2.y += pp[2 * c + 1].y;
    }
    block_sum2(s1, s2);
    if (threadIdx.x == 0) {
        a.count[seg] = 0;
        finalize<OP>(S, s1, s2, a.n_active, a.tols ? a.tols[seg] : a.tol, a.maxit);
    }
}

template <class C>
static int launch_bicg(Bicg<C>& k, int op, double tol, int maxit, cudaStream_t s, const double* tols = nullptr) {
    VecArgs<C> a;
    a.tols = tols;
    a.v = k.v;
    a.st = k.st;
    a.part = k.red->part;
    a.count = k.red->count;
    a.n_active = k.red->n_active;
    a.seglen = k.seglen;
    a.maxcta = kMaxCtaPerSeg;
    a.tol = tol;
    a.maxit = maxit;
    int64_t want = (k.seglen + (int64_t)kRedThreads * 8 - 1) / ((int64_t)kRedThreads * 8);
    int nct = (int)std::max<int64_t>(1, std::min<int64_t>(want, kMaxCtaPerSeg));
    dim3 grid(nct, k.nseg);
    // vectors touched per segment by each op (reads + writes)
    static const int nvec[] = {6, 4, 3, 3, 7, 2, 2, 2};
    const bool dot = op == OP_RHO || op == OP_SIGMA || op == OP_OMEGA;
    a.units = prof_begin(s, dot ? PK_BICG_DOT : PK_BICG_UPDATE, sizeof(C) == 16 ? VIE_C128 : VIE_C64,
                         (int64_t)nvec[op] * k.seglen * (int64_t)sizeof(C), 0, true);
    switch (op) {
        case OP_INIT: k_bicg<C, OP_INIT><<<grid, kRedThreads, 0, s>>>(a); break;
        case OP_P: k_bicg<C, OP_P><<<grid, kRedThreads, 0, s>>>(a); break;
        case OP_S: k_bicg<C, OP_S><<<grid, kRedThreads, 0, s>>>(a); break;
        case OP_XHALF: k_bicg<C, OP_XHALF><<<grid, kRedThreads, 0, s>>>(a); break;
        case OP_XR: k_bicg<C, OP_XR><<<grid, kRedThreads, 0, s>>>(a); break;
        case OP_RHO: k_bicg<C, OP_RHO><<<grid, kRedThreads, 0, s>>>(a); break;
        case OP_SIGMA: k_bicg<C, OP_SIGMA><<<grid, kRedThreads, 0, s>>>(a); break;
        case OP_OMEGA: k_bicg<C, OP_OMEGA><<<grid, kRedThreads, 0, s>>>(a); break;
        default: prof_end(s); return fail(VIE_EINVAL, "bad BiCGSTAB op");
    }
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <class C> int bicg_init(Bicg<C>& k, double tol, int maxit, cudaStream_t s) {
    VIE_CK(cudaMemsetAsync(k.red->n_active, 0, sizeof(int), s));
    return launch_bicg(k, OP_INIT, tol, maxit, s);
}
template <class C> int bicg_init_tols(Bicg<C>& k, const double* tols, int maxit, cudaStream_t s) {
    VIE_CK(cudaMemsetAsync(k.red->n_active, 0, sizeof(int), s));
    return launch_bicg(k, OP_INIT, 0.0, maxit, s, tols);
}
template <class C> int bicg_rho(Bicg<C>& k, cudaStream_t s) { return launch_bicg(k, OP_RHO, 0, 0, s); }
template <class C> int bicg_update_p(Bicg<C>& k, cudaStream_t s) { return launch_bicg(k, OP_P, 0, 0, s); }
template <class C> int bicg_sigma(Bicg<C>& k, cudaStream_t s) { return launch_bicg(k, OP_SIGMA, 0, 0, s); }
template <class C> int bicg_update_s(Bicg<C>& k, cudaStream_t s) { return launch_bicg(k, OP_S, 0, 0, s); }
template <class C> int bicg_x_half(Bicg<C>& k, cudaStream_t s) { return launch_bicg(k, OP_XHALF, 0, 0, s); }
template <class C> int bicg_omega(Bicg<C>& k, cudaStream_t s) { return launch_bicg(k, OP_OMEGA, 0, 0, s); }
template <class C> int bicg_update_xr(Bicg<C>& k, cudaStream_t s) { return launch_bicg(k, OP_XR, 0, 0, s); }

#define VIE_INST(C)                                                        \
    template int bicg_init<C>(Bicg<C>&, double, int, cudaStream_t);        \
    template int bicg_init_tols<C>(Bicg<C>&, const double*, int, cudaStream_t); \
    template int bicg_rho<C>(Bicg<C>&, cudaStream_t);                      \
    template int bicg_update_p<C>(Bicg<C>&, cudaStream_t);                 \
    template int bicg_sigma<C>(Bicg<C>&, cudaStream_t);                    \
    template int bicg_update_s<C>(Bicg<C>&, cudaStream_t);                 \
    template int bicg_x_half<C>(Bicg<C>&, cudaStream_t);                   \
    template int bicg_omega<C>(Bicg<C>&, cudaStream_t);                    \
    template int bicg_update_xr<C>(Bicg<C>&, cudaStream_t);
VIE_INST(double2)
VIE_INST(float2)
#undef VIE_INST

// ---------------------------------------------------------------- plain vector helpers
template <class C>
__global__ void k_copy(const C* a, C* b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = a[i];
}

static unsigned grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

template <class C> int vec_copy(const C* a, C* b, int64_t n, cudaStream_t s) {
    prof_begin(s, PK_FIELD, sizeof(C) == 16 ? VIE_C128 : VIE_C64, 0, 2 * n * (int64_t)sizeof(C), false);
    k_copy<C><<<grid_for(n), 256, 0, s>>>(a, b, n);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}
template int vec_copy<double2>(const double2*, double2*, int64_t, cudaStream_t);
template int vec_copy<float2>(const float2*, float2*, int64_t, cudaStream_t);

__global__ void k_residual128(const double2* b, const double2* ax, double2* r, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - ax[i];
}
int vec_residual128(const double2* b, const double2* ax, double2* r, int64_t n, cudaStream_t s) {
    prof_begin(s, PK_FIELD, VIE_C128, 0, 3 * n * 16, false);
    k_residual128<<<grid_for(n), 256, 0, s>>>(b, ax, r, n);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

// ||a||^2 in FP64 into d_out[0] (single segment, deterministic two-level sum).
__global__ void __launch_bounds__(kRedThreads) k_norm2(const double2* a, int64_t n, double2* part, unsigned* count, double* out) {
    double2 acc = make_double2(0, 0), zero = make_double2(0, 0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = a[i];
        acc.x += v.x * v.x + v.y * v.y;
    }
    block_sum2(acc, zero);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = acc;
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double2 s1 = make_double2(0, 0), s2 = make_double2(0, 0);
    const volatile double2* pp = part;
    for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x) s1.x += pp[2 * c].x;
    block_sum2(s1, s2);
    if (threadIdx.x == 0) {
        *count = 0;
        *out = s1.x;
    }
}
int vec_norm2_128(const double2* a, int64_t n, ReduceScratch* red, double* d_out, cudaStream_t s) {
    int64_t want = (n + (int64_t)kRedThreads * 8 - 1) / ((int64_t)kRedThreads * 8);
    int nct = (int)std::max<int64_t>(1, std::min<int64_t>(want, kMaxCtaPerSeg));
    prof_begin(s, PK_FIELD, VIE_C128, 0, n * 16, false);
    k_norm2<<<nct, kRedThreads, 0, s>>>(a, n, red->part, red->count, d_out);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

__global__ void k_sum128(const double2* a, const double2* b, double2* out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}
int vec_sum128(const double2* a, const double2* b, double2* out, int64_t n, cudaStream_t s) {
    prof_begin(s, PK_FIELD, VIE_C128, 0, 3 * n * 16, false);
    k_sum128<<<grid_for(n), 256, 0, s>>>(a, b, out, n);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

// b = a / ||a|| rounded to complex64 (the correction solve's right-hand side).
__global__ void k_scale_to_c64(const double2* a, const double* norm2, float2* b, int64_t n) {
    double inv = 1.0 / sqrt(*norm2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 v = a[i];
        b[i] = make_float2((float)(v.x * inv), (float)(v.y * inv));
    }
}
int vec_scale_to_c64(const double2* a, const double* d_norm2, float2* b, int64_t n, cudaStream_t s) {
    prof_begin(s, PK_FIELD, VIE_C128, 0, n * 24, false);
    k_scale_to_c64<<<grid_for(n), 256, 0, s>>>(a, d_norm2, b, n);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

// x += ||r|| d (FP64 accumulation of a complex64 correction).
__global__ void k_add_scaled_c64(double2* x, const float2* d, const double* norm2, int64_t n) {
    double sc = sqrt(*norm2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = d[i];
        double2 xv = x[i];
        x[i] = make_double2(xv.x + sc * (double)v.x, xv.y + sc * (double)v.y);
    }
}
int vec_add_scaled_c64(double2* x, const float2* d, const double* d_norm2, int64_t n, cudaStream_t s) {
    prof_begin(s, PK_FIELD, VIE_C128, 0, n * 40, false);
    k_add_scaled_c64<<<grid_for(n), 256, 0, s>>>(x, d, d_norm2, n);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

}  // namespace vie
