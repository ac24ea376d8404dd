// Persistent block solver for the block-diagonal preconditioner (Eq. 10;
// Section II.B: inner BiCGSTAB-FFT solves with a loose tolerance).
//
// The diagonal blocks are independent (no data exchange between blocks), so
// one CTA owns one block at a time and runs that block's whole BiCGSTAB
// without any grid-wide synchronisation; CTAs take blocks from an atomic work
// counter, largest boxes first. Each inner MVM A_k x = x - G(chi x) is done by
// the CTA in three phases over the block's padded box:
//   XY  for tiles of (component, z) planes: load the box plane with the
//       BiCGSTAB vector update fused in, multiply by chi, zero-pad, row FFTs
//       (x, pruned to the non-zero rows) and column FFTs (y) in shared
//       memory, store the plane spectrum to the block's scratch;
//   Z   for tiles of spectral columns: forward FFT along z, 3x3 symmetric
//       Green multiply, inverse FFT, keep z < bz;
//   XY' inverse column and row FFTs, keep the box, y = mask (x - u), with the
//       inner products of the iteration fused into the store.
// The block scratch ([3][bz][My][Mx]) stays L2-resident for the boxes this
// path accepts. Scalars are FP64; complex64 vectors accumulate products in
// FP32 within a thread and in FP64 across the CTA.
#include <cooperative_groups.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fft_core.cuh"
#include "fft_reg.cuh"
#include "vie_internal.cuh"

namespace cg = cooperative_groups;

namespace vie {

template <class C> struct InnerGroup {
    C *b, *x, *r, *rhat, *p, *v, *s, *t;   // [nb][3][bz][by][bx]
    C* w1;                                  // [nb][3][bz][by][Mx] (register path)
    C* w2;                                  // [nb][3][bz][My][Mx]
    const C* chi;                           // [nb][bz][by][bx]
    const uint8_t* mask;                    // [nb][bz][by][bx]
    const C* G;                             // [6][Mz][My][Mx], bit-reversed positions
    const C* const* Gb;                     // optional: one spectrum per box
    const double* tols;                     // optional: one relative tolerance per box
    SegState* st;                           // [nb]
    int nb, bx, by, bz, Mx, My, Mz, lx, ly, lz, lyb;   // lyb = log2 of nextpow2(by)
    int lpt;                                // log2 planes per XY tile
    int ltc;                                // log2 columns per Z tile
    int kb_mvm;                             // profiling: KB moved by one MVM and its fused updates
    int kb_upd;                             // profiling: KB moved by the x/r update pass
    int reg;                                // 1: register-FFT MVM (complex64, every padded axis <= 32)
    unsigned fd_bx[3], fd_plane[3];         // FastDiv constants (m, s, d) for bx and bz*by
    // slab MVM (complex64): the whole MVM on chip, kz planes of the box in shared memory
    int slab;                               // 1: the block uses the slab MVM
    int bxp;                                // row pitch of the slab (bx made odd: no bank conflicts)
    int npl;                                // kz planes per round of the plane stage (set per launch)
    unsigned fd_col[3];                     // FastDiv constants for by*bx
    const C* Go;                            // octant spectrum [Mz/2+1][6][My/2+1][Mx/2+1], natural order
};

constexpr int kInnerThreads = 256;


__device__ __forceinline__ double2 dcdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ bool dgood(double2 a) {
    return isfinite(a.x) && isfinite(a.y) && (a.x != 0.0 || a.y != 0.0);
}
template <class C> __device__ __forceinline__ void acc_dot(C& acc, C a, C b) {   // acc += conj(a) b
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
}

// A block is solved by a team: the R CTAs of one thread-block cluster. Every
// phase splits its rows / columns / planes over the ranks; phases that read
// what other ranks wrote are separated by cluster barriers (release/acquire at
// cluster scope), and sums go CTA -> distributed shared memory in rank order,
// so every CTA gets identical scalars.
__device__ __forceinline__ int team_rank() { return (int)cg::this_cluster().block_rank(); }
__device__ __forceinline__ int team_size() { return (int)cg::this_cluster().num_blocks(); }
__device__ __forceinline__ void team_sync() { cg::this_cluster().sync(); }

// Slot of the next cluster sum; reset to 0 by every CTA at kernel entry so all
// ranks of a cluster flip in step.
__shared__ int team_slot;

template <class T> __device__ __forceinline__ T shfl_dn(T v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }

// Team-wide sums of two complex partials a and b held by every thread (complex64
// or complex128). Each warp adds its lanes in the partials' precision; thread 0
// adds the warps' sums in FP64 in a fixed order (and, for R > 1, the ranks' sums
// in rank order through distributed shared memory), then calls fn(sum_a, sum_b):
// the iteration's FP64 scalar work runs in that one thread and reaches the others
// through the shared state fn writes, published by the closing barrier. Every rank
// computes identical sums. Two rank slots alternate between consecutive sums: a
// slot is rewritten two sums later, after every rank has passed the cluster
// barrier of the sum in between, so one cluster barrier per sum suffices.
constexpr int kTeamSumMax = 4;                 // complex values one team sum carries

template <int N, class C, class Fn>
__device__ __forceinline__ void team_sum_n(C (&v)[N], double2* red, Fn fn) {
    static_assert(N <= kTeamSumMax, "team_sum_n: too many values");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i) {
            v[i].x += shfl_dn(v[i].x, o);
            v[i].y += shfl_dn(v[i].y, o);
        }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) red[N * w + i] = make_double2(v[i].x, v[i].y);
    __syncthreads();
    cg::cluster_group cl = cg::this_cluster();
    const unsigned R = cl.num_blocks();
    __shared__ double2 xred[2][kTeamSumMax];
    double2 sum[N];
#pragma unroll
    for (int i = 0; i < N; ++i) sum[i] = make_double2(0, 0);
    if (threadIdx.x == 0) {
        for (int k = 0; k < nw; ++k)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                sum[i].x += red[N * k + i].x;
                sum[i].y += red[N * k + i].y;
            }
        if (R > 1) {
            team_slot ^= 1;
#pragma unroll
            for (int i = 0; i < N; ++i) xred[team_slot][i] = sum[i];
        }
    }
    if (R > 1) {
        cl.sync();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int i = 0; i < N; ++i) sum[i] = make_double2(0, 0);
            for (unsigned r = 0; r < R; ++r) {
                const double2* q = cl.map_shared_rank(&xred[team_slot][0], r);
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    sum[i].x += q[i].x;
                    sum[i].y += q[i].y;
                }
            }
        }
    }
    if (threadIdx.x == 0) fn(sum);
    __syncthreads();
}

template <class C, class Fn>
__device__ __forceinline__ void team_sum(C a, C b, double2* red, Fn fn) {
    C v[2] = {a, b};
    team_sum_n<2>(v, red, [&](const double2 (&s)[2]) { fn(s[0], s[1]); });
}

enum { IN_P = 0, IN_S = 1, IN_PX = 2 };   // IN_PX: p update with the previous step's x and r updates fused
enum { OUT_V = 0, OUT_T = 1, OUT_TX = 2 };   // OUT_TX: OUT_T with <rhat, s> and <rhat, t> as well

// Phase XY: plane tiles, fused vector update + chi, 2D forward FFT, store spectrum.
// IN_P: p = r + beta (p - omega v);  IN_S: s = r - alpha v (returns ||s||^2 in .x).
template <class C, int IN>
__device__ C phase_xy(const InnerGroup<C>& g, int64_t voff, C* W, const C* chi, C* sm, const C* tw, C c1, C c2) {
    const int planes = 3 * g.bz, P = g.Mx + 1, pe = g.My * P, tile = 1 << g.lpt;
    const int64_t box = (int64_t)g.bx * g.by * g.bz;
    C acc = czero<C>();
    const int rk = team_rank(), nrk = team_size();
    for (int pl0 = rk * tile; pl0 < planes; pl0 += nrk * tile) {
        const int n = tile * g.My * g.Mx;
        for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
            int xq = idx & (g.Mx - 1), t = idx >> g.lx;
            int yq = t & (g.My - 1), k = t >> g.ly;
            int pl = pl0 + k;
            C val = czero<C>();
            if (pl < planes && xq < g.bx && yq < g.by) {
                int comp = pl / g.bz, z = pl - comp * g.bz;
                int64_t lv = ((int64_t)z * g.by + yq) * g.bx + xq;
                int64_t e = voff + comp * box + lv;
                C in;
                if (IN == IN_P) {
                    in = g.r[e] + cmul(c1, g.p[e] - cmul(c2, g.v[e]));
                    g.p[e] = in;
                } else {
                    in = g.r[e] - cmul(c1, g.v[e]);
                    g.s[e] = in;
                    acc.x += in.x * in.x + in.y * in.y;
                }
                val = cmul(in, chi[lv]);
            }
            sm[k * pe + yq * P + xq] = val;
        }
        __syncthreads();
        smem_fft_g<C, true>(sm, g.lx, 1, g.lyb, P, g.lpt, pe, tw, kLogLmax - g.lx);     // rows (x)
        smem_fft_g<C, true>(sm, g.ly, P, g.lx, 1, g.lpt, pe, tw, kLogLmax - g.ly);      // columns (y)
        for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
            int xq = idx & (g.Mx - 1), t = idx >> g.lx;
            int yq = t & (g.My - 1), k = t >> g.ly;
            int pl = pl0 + k;
            if (pl < planes) W[((int64_t)pl * g.My + yq) * g.Mx + xq] = sm[k * pe + yq * P + xq];
        }
        __syncthreads();
    }
    return acc;   // this thread's partial; the caller folds it into a later sum
}

// Phase Z: forward FFT along z, Green multiply, inverse FFT (columns of the plane spectra).
template <class C>
__device__ void phase_z(const InnerGroup<C>& g, C* W, C* sm, const C* tw) {
    const int TC = 1 << g.ltc, pitch = 3 * TC;
    const int64_t plane = (int64_t)g.My * g.Mx;
    const int64_t cstride = (int64_t)g.bz * plane, gcomp = (int64_t)g.Mz * plane;
    const int L = g.Mz;
    const int rk = team_rank(), nrk = team_size();
    for (int64_t c0 = (int64_t)rk * TC; c0 < plane; c0 += (int64_t)nrk * TC) {
        for (int idx = threadIdx.x; idx < L * 3 * TC; idx += blockDim.x) {
            int c = idx & (TC - 1), t = idx >> g.ltc;
            int comp = t % 3, i = t / 3;
            C v = czero<C>();
            if (i < g.bz && c0 + c < plane) v = W[comp * cstride + i * plane + c0 + c];
            sm[idx] = v;
        }
        __syncthreads();
        smem_fft<C, true, 3>(sm, g.lz, pitch, g.ltc, tw, kLogLmax - g.lz);
        for (int idx = threadIdx.x; idx < L * TC; idx += blockDim.x) {
            int c = idx & (TC - 1), i = idx >> g.ltc;
            if (c0 + c >= plane) continue;
            const C* gp = g.G + i * plane + c0 + c;
            C gxx = gp[0], gxy = gp[gcomp], gxz = gp[2 * gcomp];
            C gyy = gp[3 * gcomp], gyz = gp[4 * gcomp], gzz = gp[5 * gcomp];
            C* q = sm + i * pitch + c;
            C X = q[0], Y = q[TC], Z = q[2 * TC];
            q[0] = cmul(gxx, X) + cmul(gxy, Y) + cmul(gxz, Z);
            q[TC] = cmul(gxy, X) + cmul(gyy, Y) + cmul(gyz, Z);
            q[2 * TC] = cmul(gxz, X) + cmul(gyz, Y) + cmul(gzz, Z);
        }
        __syncthreads();
        smem_fft<C, false, 3>(sm, g.lz, pitch, g.ltc, tw, kLogLmax - g.lz);
        for (int idx = threadIdx.x; idx < g.bz * 3 * TC; idx += blockDim.x) {
            int c = idx & (TC - 1), t = idx >> g.ltc;
            int comp = t % 3, i = t / 3;
            if (c0 + c < plane) W[comp * cstride + i * plane + c0 + c] = sm[idx];
        }
        __syncthreads();
    }
}

// Phase XY': inverse 2D FFT of the plane spectra, keep the box, out = mask (in - u).
// OUT_V: in = p, out = v, returns <rhat, v>.  OUT_T: in = s, out = t, returns (<t, s>, <t, t>).
template <class C, int OUT>
__device__ void phase_xy_inv(const InnerGroup<C>& g, int64_t voff, const C* W, const uint8_t* mask, C* sm,
                             const C* tw, C& a1, C& a2) {
    const int planes = 3 * g.bz, P = g.Mx + 1, pe = g.My * P, tile = 1 << g.lpt;
    const int64_t box = (int64_t)g.bx * g.by * g.bz;
    const int rk = team_rank(), nrk = team_size();
    for (int pl0 = rk * tile; pl0 < planes; pl0 += nrk * tile) {
        const int n = tile * g.My * g.Mx;
        for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
            int xq = idx & (g.Mx - 1), t = idx >> g.lx;
            int yq = t & (g.My - 1), k = t >> g.ly;
            int pl = pl0 + k;
            sm[k * pe + yq * P + xq] = pl < planes ? W[((int64_t)pl * g.My + yq) * g.Mx + xq] : czero<C>();
        }
        __syncthreads();
        smem_fft_g<C, false>(sm, g.ly, P, g.lx, 1, g.lpt, pe, tw, kLogLmax - g.ly);     // columns (y)
        smem_fft_g<C, false>(sm, g.lx, 1, g.lyb, P, g.lpt, pe, tw, kLogLmax - g.lx);    // rows (x), y < nextpow2(by)
        const int nb = tile * g.by * g.bx;
        for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
            int xq = idx % g.bx, t = idx / g.bx;
            int yq = t % g.by, k = t / g.by;
            int pl = pl0 + k;
            if (pl >= planes) continue;
            int comp = pl / g.bz, z = pl - comp * g.bz;
            int64_t lv = ((int64_t)z * g.by + yq) * g.bx + xq;
            int64_t e = voff + comp * box + lv;
            C u = sm[k * pe + yq * P + xq];
            C in = OUT == OUT_V ? g.p[e] : g.s[e];
            C o = mask[lv] ? in - u : czero<C>();
            if (OUT == OUT_V) {
                g.v[e] = o;
                acc_dot(a1, g.rhat[e], o);
            } else {
                g.t[e] = o;
                acc_dot(a1, o, in);
                a2.x += o.x * o.x + o.y * o.y;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- register-FFT box MVM (complex64)
// Division by a runtime divisor d (1 <= d < 2^31) of n < 2^31 with a multiply-high
// (Granlund and Montgomery, PLDI 1994): q = (umulhi(n, m) + n) >> s.
struct FastDiv {
    unsigned m, s, d;
};
__device__ __forceinline__ unsigned fdiv(unsigned n, FastDiv f) { return (__umulhi(n, f.m) + n) >> f.s; }
__device__ __forceinline__ FastDiv fd_of(const unsigned (&v)[3]) { return FastDiv{v[0], v[1], v[2]}; }

// 8-byte asynchronous copy global -> shared (sm_80+), and the wait for all of this thread's copies.
__device__ __forceinline__ void cp_async8(F* dst_smem, const F* src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// 16-byte asynchronous copy global -> shared, bypassing L1 (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

// Prefetch into L1: lets a loop with one pending element per thread overlap
// the L2 latency of later iterations without holding their values in registers.
__device__ __forceinline__ void pf(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
constexpr int kPf = 2;   // iterations ahead

constexpr int kU = 1;   // elements per thread whose loads are issued together in the row phases
constexpr int kUV = 1;  // elements per thread per batch in the block-vector passes
constexpr int kUG = 1;  // Green-multiply tasks per thread whose 6 spectrum loads are issued together

// X forward: rows (component, z, y) of the box. Coalesced loads (with the
// BiCGSTAB update fused) into IN, one pruned row FFT per thread into OUT,
// coalesced stores of OUT to W1. Shared memory: T (bx + 1) + T (LX + 1).
template <int LX, int IN>
__device__ __forceinline__ F x_fwd_reg(const InnerGroup<F>& g, int64_t voff, F* W1, const F* chi, F* sm,
                                       const F* tw, F c1, F c2) {
    const int NR = 3 * g.bz * g.by, bx = g.bx, plane = g.bz * g.by, T = blockDim.x, t = threadIdx.x;
    const FastDiv dbx = fd_of(g.fd_bx), dpl = fd_of(g.fd_plane);
    F* smi = sm;
    F* smo = sm + T * (bx + 1);
    F acc = czero<F>();
    const int rk = team_rank(), nrk = team_size();
    for (int r0 = rk * T; r0 < NR; r0 += nrk * T) {
        const int nr = min(T, NR - r0);
        const int64_t base = voff + (int64_t)r0 * bx;
        const int nk = nr * bx;
        for (int k0 = t; k0 < nk; k0 += kU * T) {
            {
                const int ka = k0 + kPf * kU * T;
                if (ka < nk) {
                    const int64_t e = base + ka;
                    pf(g.r + e);
                    pf(g.v + e);
                    if (IN == IN_P) pf(g.p + e);
                }
            }
            F ra[kU], pa[kU], va[kU], ca[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {          // all loads of the batch first
                const int k = k0 + u * T;
                if (k < nk) {
                    const int64_t e = base + k;
                    const int rr = (int)fdiv(k, dbx), x = k - rr * bx;
                    const int row = r0 + rr;
                    ra[u] = g.r[e];
                    va[u] = g.v[e];
                    if (IN == IN_P) pa[u] = g.p[e];
                    ca[u] = chi[(int64_t)(row - (int)fdiv(row, dpl) * plane) * bx + x];
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int k = k0 + u * T;
                if (k < nk) {
                    const int64_t e = base + k;
                    const int rr = (int)fdiv(k, dbx), x = k - rr * bx;
                    F in;
                    if (IN == IN_P) {
                        in = ra[u] + cmul(c1, pa[u] - cmul(c2, va[u]));
                        g.p[e] = in;
                    } else {
                        in = ra[u] - cmul(c1, va[u]);
                        g.s[e] = in;
                        acc.x += in.x * in.x + in.y * in.y;
                    }
                    smi[rr * (bx + 1) + x] = cmul(in, ca[u]);
                }
            }
        }
        __syncthreads();
        if (t < nr) {
            const F* row = smi + t * (bx + 1);
            F* out = smo + t * (LX + 1);
            fwd_half<LX>([&](int j) { return j < bx ? row[j] : czero<F>(); }, [&](int k, F v) { out[k] = v; }, tw);
        }
        __syncthreads();
        F* dst = W1 + (int64_t)r0 * LX;
        for (int k = t; k < nr * LX; k += T) dst[k] = smo[(k / LX) * (LX + 1) + (k & (LX - 1))];   // LX: power of two
        __syncthreads();
    }
    return acc;
}

// Y forward: one column (component, z, x) per thread, straight from W1 (coalesced along x).
template <int LY>
__device__ __forceinline__ void y_fwd_reg(const InnerGroup<F>& g, const F* W1, F* W2, const F* tw) {
    const int LX = g.Mx, cols = 3 * g.bz * LX, by = g.by;
    const int nrk = team_size();
    for (int col = team_rank() * blockDim.x + threadIdx.x; col < cols; col += nrk * blockDim.x) {
        int pz = col >> g.lx, x = col & (LX - 1);
        const F* src = W1 + (int64_t)pz * by * LX + x;
        F* dst = W2 + (int64_t)pz * LY * LX + x;
        fwd_half<LY>([&](int j) { return j < by ? src[j * LX] : czero<F>(); }, [&](int k, F v) { dst[k * LX] = v; },
                     tw);
    }
}

// Y inverse: one column per thread, keep y < by; the stash lives in W1's column.
template <int LY>
__device__ __forceinline__ void y_inv_reg(const InnerGroup<F>& g, const F* W2, F* W1, const F* tw) {
    const int LX = g.Mx, cols = 3 * g.bz * LX, by = g.by;
    const int nrk = team_size();
    for (int col = team_rank() * blockDim.x + threadIdx.x; col < cols; col += nrk * blockDim.x) {
        int pz = col >> g.lx, x = col & (LX - 1);
        const F* src = W2 + (int64_t)pz * LY * LX + x;
        F* dst = W1 + (int64_t)pz * by * LX + x;
        inv_half<LY>([&](int k) { return src[k * LX]; },
                     [&](int j, F v) { if (j < by) dst[j * LX] = v; },
                     [&](int j) { return j < by ? dst[j * LX] : czero<F>(); },
                     [&](int j, F v) { if (j < by) dst[j * LX] = v; }, tw);
    }
}

constexpr int kZCols = 128;   // spectral columns per Z round

// Z: forward along z, 3x3 Green multiply, inverse, keep z < bz. Per round the
// three transformed components of kZCols columns are staged in shared memory.
// Offsets are 32-bit (a padded plane has at most 2^20 points).
template <int LZ>
__device__ __forceinline__ void z_reg(const InnerGroup<F>& g, F* W2, F* sm, const F* tw) {
    constexpr int H = LZ / 2 > 0 ? LZ / 2 : 1;
    const int P = g.My * g.Mx, T = blockDim.x, t = threadIdx.x, bz = g.bz;
    const int cs = bz * P, gc = LZ * P;
    const int rk = team_rank(), nrk = team_size();
    for (int c0 = rk * kZCols; c0 < P; c0 += nrk * kZCols) {
        const int nc = min(kZCols, P - c0);     // a power of two (P and kZCols are)
        const int lnc = 31 - __clz(nc);
        for (int task = t; task < 3 * nc; task += T) {
            const int comp = task >> lnc, c = task & (nc - 1);
            const F* src = W2 + comp * cs + c0 + c;
            F* S = sm + comp * LZ * kZCols + c;
            if (LZ == 1) {
                S[0] = src[0];
                continue;
            }
            F a[H];
#pragma unroll
            for (int j = 0; j < H; ++j) a[j] = j < bz ? src[j * P] : czero<F>();
#pragma unroll
            for (int j = 0; j < H; ++j) a[j] = twc<true>(a[j], j * (kLmax / LZ));
            rfft<H, true>(a, tw);
#pragma unroll
            for (int j = 0; j < H; ++j) S[(H + j) * kZCols] = a[j];
#pragma unroll
            for (int j = 0; j < H; ++j) a[j] = j < bz ? src[j * P] : czero<F>();
            rfft<H, true>(a, tw);
#pragma unroll
            for (int j = 0; j < H; ++j) S[j * kZCols] = a[j];
        }
        __syncthreads();
        // K is even in the z offset for xx, xy, yy, zz and odd for xz, yz, so the spectrum at
        // frequency -f is +-(the one at f): one load of the six entries serves the z position p of
        // frequency f and the position pm of -f (mirror pairs; the smaller position does the work)
        const int cst = LZ * kZCols;
        constexpr int LGZ = ILog2<LZ>::v;
        // tasks = (frequency f in [0, LZ/2], column): exactly the working mirror pairs; two tasks per
        // step with all twelve spectrum loads issued before either multiply
        const int nwork = (LZ / 2 + 1) * nc;
        auto pair_of = [&](int task, int& i, int& im, int& c) {
            const int f = task >> lnc;
            c = task & (nc - 1);
            const int i1 = LGZ ? (int)(__brev((unsigned)f) >> (32 - LGZ)) : 0;
            const int i2 = LGZ ? (int)(__brev((unsigned)((LZ - f) & (LZ - 1))) >> (32 - LGZ)) : 0;
            i = min(i1, i2);
            im = max(i1, i2);
        };
        auto apply = [&](int i, int im, int c, F gxx, F gxy, F gxz, F gyy, F gyz, F gzz) {
            {
                F* q = sm + i * kZCols + c;
                F X = q[0], Y = q[cst], Z = q[2 * cst];
                q[0] = cmul(gxx, X) + cmul(gxy, Y) + cmul(gxz, Z);
                q[cst] = cmul(gxy, X) + cmul(gyy, Y) + cmul(gyz, Z);
                q[2 * cst] = cmul(gxz, X) + cmul(gyz, Y) + cmul(gzz, Z);
            }
            if (im != i) {
                F* q = sm + im * kZCols + c;
                F X = q[0], Y = q[cst], Z = q[2 * cst];
                q[0] = cmul(gxx, X) + cmul(gxy, Y) - cmul(gxz, Z);
                q[cst] = cmul(gxy, X) + cmul(gyy, Y) - cmul(gyz, Z);
                q[2 * cst] = cmul(gzz, Z) - cmul(gxz, X) - cmul(gyz, Y);
            }
        };
        for (int task = t; task < nwork; task += 2 * T) {
            int i0, im0, c0_, i1, im1, c1_;
            pair_of(task, i0, im0, c0_);
            const bool two = task + T < nwork;
            pair_of(two ? task + T : task, i1, im1, c1_);
            const F* gp0 = g.G + i0 * P + c0 + c0_;
            const F* gp1 = g.G + i1 * P + c0 + c1_;
            const F a0 = gp0[0], a1 = gp0[gc], a2 = gp0[2 * gc], a3 = gp0[3 * gc], a4 = gp0[4 * gc], a5 = gp0[5 * gc];
            const F b0 = gp1[0], b1 = gp1[gc], b2 = gp1[2 * gc], b3 = gp1[3 * gc], b4 = gp1[4 * gc], b5 = gp1[5 * gc];
            apply(i0, im0, c0_, a0, a1, a2, a3, a4, a5);
            if (two) apply(i1, im1, c1_, b0, b1, b2, b3, b4, b5);
        }
        __syncthreads();
        for (int task = t; task < 3 * nc; task += T) {
            const int comp = task >> lnc, c = task & (nc - 1);
            F* S = sm + comp * LZ * kZCols + c;
            F* dst = W2 + comp * cs + c0 + c;
            if (LZ == 1) {
                dst[0] = S[0];
                continue;
            }
            F a[H];
#pragma unroll
            for (int j = 0; j < H; ++j) a[j] = S[(H + j) * kZCols];
            rfft<H, false>(a, tw);
#pragma unroll
            for (int j = 0; j < H; ++j) S[(H + j) * kZCols] = twc<false>(a[j], j * (kLmax / LZ));
#pragma unroll
            for (int j = 0; j < H; ++j) a[j] = S[j * kZCols];
            rfft<H, false>(a, tw);
#pragma unroll
            for (int j = 0; j < H; ++j)
                if (j < bz) dst[j * P] = a[j] + S[(H + j) * kZCols];
        }
        __syncthreads();
    }
}

// X inverse: rows of W1, keep x < bx, out = mask (in - u) with the iteration's dots.
template <int LX, int OUT>
__device__ __forceinline__ void x_inv_reg(const InnerGroup<F>& g, int64_t voff, const F* W1, const uint8_t* mask,
                                          F* sm, const F* tw, F& a1, F& a2) {
    const int NR = 3 * g.bz * g.by, bx = g.bx, plane = g.bz * g.by, T = blockDim.x, t = threadIdx.x;
    const FastDiv dbx = fd_of(g.fd_bx), dpl = fd_of(g.fd_plane);
    F* smi = sm;
    F* smo = sm + T * (LX + 1);
    const int rk = team_rank(), nrk = team_size();
    for (int r0 = rk * T; r0 < NR; r0 += nrk * T) {
        const int nr = min(T, NR - r0);
        const F* src = W1 + (int64_t)r0 * LX;
        // asynchronous global -> shared copies (no registers held while in flight), one wait
        for (int k = t; k < nr * LX; k += T) cp_async8(smi + (k / LX) * (LX + 1) + (k & (LX - 1)), src + k);
        cp_async_wait_all();
        __syncthreads();
        if (t < nr) {
            const F* row = smi + t * (LX + 1);
            F* out = smo + t * (bx + 1);
            inv_half<LX>([&](int k) { return row[k]; },
                         [&](int j, F v) { if (j < bx) out[j] = v; },
                         [&](int j) { return j < bx ? out[j] : czero<F>(); },
                         [&](int j, F v) { if (j < bx) out[j] = v; }, tw);
        }
        __syncthreads();
        const int64_t base = voff + (int64_t)r0 * bx;
        const int nk = nr * bx;
        for (int k0 = t; k0 < nk; k0 += kU * T) {
            {
                const int ka = k0 + kPf * kU * T;
                if (ka < nk) {
                    const int64_t e = base + ka;
                    pf(OUT == OUT_V ? g.p + e : g.s + e);
                    if (OUT == OUT_V) pf(g.rhat + e);
                }
            }
            F ia[kU], ha[kU];
            uint8_t ma[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int k = k0 + u * T;
                if (k < nk) {
                    const int64_t e = base + k;
                    const int rr = (int)fdiv(k, dbx), x = k - rr * bx;
                    const int row = r0 + rr;
                    ia[u] = OUT == OUT_V ? g.p[e] : g.s[e];
                    if (OUT == OUT_V) ha[u] = g.rhat[e];
                    ma[u] = mask[(int64_t)(row - (int)fdiv(row, dpl) * plane) * bx + x];
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int k = k0 + u * T;
                if (k < nk) {
                    const int64_t e = base + k;
                    const int rr = (int)fdiv(k, dbx), x = k - rr * bx;
                    F o = ma[u] ? ia[u] - smo[rr * (bx + 1) + x] : czero<F>();
                    if (OUT == OUT_V) {
                        g.v[e] = o;
                        acc_dot(a1, ha[u], o);
                    } else {
                        g.t[e] = o;
                        acc_dot(a1, o, ia[u]);
                        a2.x += o.x * o.x + o.y * o.y;
                    }
                }
            }
        }
        __syncthreads();
    }
}

#define VIE_LEN_SWITCH(l, CALL)                                        \
    switch (l) {                                                       \
        case 3: { constexpr int LL = 8; CALL; } break;                 \
        case 4: { constexpr int LL = 16; CALL; } break;                \
        default: { constexpr int LL = 32; CALL; } break;               \
    }

// The two MVM implementations used by solve_block.
template <class C> struct SmemMvm {
    static constexpr int kUV = 1;       // elements per thread per batch in the block-vector passes
    static constexpr bool kMerged = false;
    template <int IN>
    static __device__ C fwd(const InnerGroup<C>& g, int64_t voff, C* W1, C* W2, const C* chi, C* sm, const C* tw,
                            C c1, C c2) {
        C r = phase_xy<C, IN>(g, voff, W2, chi, sm, tw, c1, c2);
        team_sync();
        return r;                                 // this thread's part of ||s||^2 (IN_S)
    }
    static __device__ void mid(const InnerGroup<C>& g, C* W2, C* sm, const C* tw) {
        phase_z<C>(g, W2, sm, tw);
        team_sync();
    }
    // this thread's partials of the iteration's inner products
    template <int OUT>
    static __device__ void inv(const InnerGroup<C>& g, int64_t voff, C* W1, C* W2, const uint8_t* mask, C* sm,
                               const C* tw, C& a1, C& a2) {
        phase_xy_inv<C, OUT>(g, voff, W2, mask, sm, tw, a1, a2);
    }
};

struct RegMvm {
    static constexpr int kUV = 1;
    static constexpr bool kMerged = false;
    template <int IN>
    static __device__ __forceinline__ F fwd(const InnerGroup<F>& g, int64_t voff, F* W1, F* W2, const F* chi, F* sm,
                                            const F* tw, F c1, F c2) {
        F acc = czero<F>();
        VIE_LEN_SWITCH(g.lx, (acc = x_fwd_reg<LL, IN>(g, voff, W1, chi, sm, tw, c1, c2)));
        team_sync();
        VIE_LEN_SWITCH(g.ly, (y_fwd_reg<LL>(g, W1, W2, tw)));
        team_sync();                            // W2 complete on every rank
        return acc;                             // this thread's part of ||s||^2 (IN_S), summed later
    }
    static __device__ __forceinline__ void mid(const InnerGroup<F>& g, F* W2, F* sm, const F* tw) {
        VIE_LEN_SWITCH(g.lz, (z_reg<LL>(g, W2, sm, tw)));
        team_sync();
    }
    template <int OUT>
    static __device__ __forceinline__ void inv(const InnerGroup<F>& g, int64_t voff, F* W1, F* W2, const uint8_t* mask,
                                               F* sm, const F* tw, F& a1, F& a2) {
        VIE_LEN_SWITCH(g.ly, (y_inv_reg<LL>(g, W2, W1, tw)));
        team_sync();
        VIE_LEN_SWITCH(g.lx, (x_inv_reg<LL, OUT>(g, voff, W1, mask, sm, tw, a1, a2)));
    }
};

// ---------------------------------------------------------------- slab MVM (complex64, on chip)
// The MVM of one block without any global scratch. z is transformed first: the
// box columns (component, y, x) go through a pruned z FFT in registers and land
// as kz planes [3][by][bx] in the shared memory of the cluster rank that owns
// kz (distributed shared memory stores). Each rank then takes its kz planes
// through the x and y FFTs, the 3x3 Green multiply and the inverse x and y FFTs
// in a shared-memory workspace, back into its slab. Last, the columns gather
// their kz values from the owners, take the inverse z FFT in registers and
// write v = mask (p - u) with the iteration's inner products. kz planes are
// dealt to ranks in mirror pairs (kz, Mz - kz), so one read of the octant
// spectrum (every component is even or odd along every axis) serves the eight
// frequencies (+-kx, +-ky, +-kz). Two cluster barriers per MVM (R > 1), plus the
// one inside the reduction that ends it.
#ifndef VIE_SLAB_THREADS
#define VIE_SLAB_THREADS 256
#endif
constexpr int kSlabThreads = VIE_SLAB_THREADS;
// The three stages of the slab MVM are separate functions (each allocates its own registers) unless
// VIE_SLAB_INLINE is defined as __forceinline__.
#ifndef VIE_SLAB_INLINE
#define VIE_SLAB_INLINE __noinline__
#endif
// CTAs per SM the slab kernel's register budget leaves room for (2 caps it at 128 registers)
#ifndef VIE_SLAB_MINB
#define VIE_SLAB_MINB 1
#endif
constexpr int kSlabMinBlocks = VIE_SLAB_MINB;
#ifndef VIE_SLAB_BATCH
#define VIE_SLAB_BATCH 1
#endif
constexpr int kSlabBatch = VIE_SLAB_BATCH;   // z planes per thread whose global loads are issued together

// Bit reversal of k over l <= 5 bits; with constant arguments (unrolled FFT positions) it folds away.
__host__ __device__ __forceinline__ constexpr int cbrev(int k, int l) {
    int r = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if (i < l) r |= ((k >> i) & 1) << (l - 1 - i);
    return r;
}

__device__ __forceinline__ F* rank_ptr(F* p, int r, int R) {
    return R == 1 ? p : cg::this_cluster().map_shared_rank(p, (unsigned)r);
}

// kz of slot s of rank r (P = Mz / R slots per rank): rank 0 holds the planes that are their own
// mirrors, kz = 0 and kz = Mz/2, in slots 0 and 1, then mirror pairs (u, Mz - u) in slots
// (2i, 2i + 1); ranks >= 1 hold mirror pairs only, in increasing u.
__device__ __forceinline__ int slab_kz(int r, int sl, int P, int Mz) {
    if (r == 0) {
        if (sl < 2) return sl == 0 ? 0 : Mz / 2;
        const int u = 1 + ((sl - 2) >> 1);
        return (sl & 1) ? Mz - u : u;
    }
    const int u = (P - 2) / 2 + 1 + (r - 1) * (P / 2) + (sl >> 1);
    return (sl & 1) ? Mz - u : u;
}
// Inverse of slab_kz: owner rank and slot of kz.
__device__ __forceinline__ void slab_owner(int kz, int P, int Mz, int& r, int& sl) {
    const int h = Mz / 2;
    if (kz == 0 || kz == h) {
        r = 0;
        sl = kz == 0 ? 0 : 1;
        return;
    }
    const int m = kz > h ? 1 : 0, u = m ? Mz - kz : kz, n0 = (P - 2) / 2;
    if (u <= n0) {
        r = 0;
        sl = 2 + 2 * (u - 1) + m;
        return;
    }
    const int q = u - n0 - 1, hp = P / 2, qr = q / hp;
    r = 1 + qr;
    sl = 2 * (q - qr * hp) + m;
}

// Per kz: generic address of its plane in the slab of the rank that owns it (local or distributed
// shared memory), so the unrolled column transforms index a table instead of mapping ranks.
__shared__ F* slab_tab[32];

__device__ __forceinline__ void slab_table(const InnerGroup<F>& g, F* sm) {
    const int R = team_size(), Mz = g.Mz, P = Mz / R, zpl = 3 * g.by * g.bxp;
    if ((int)threadIdx.x < Mz) {
        int r, sl;
        slab_owner(threadIdx.x, P, Mz, r, sl);
        slab_tab[threadIdx.x] = rank_ptr(sm + sl * zpl, r, R);
    }
    __syncthreads();
}

// Forward half of the slab MVM: update (IN_P: p = r + c1 (p - c2 v); IN_S: s = r - c1 v; IN_PX: the
// previous step's r = s - c2 t and x += c3 p + c2 s, then p = r + c1 (p - c2 v)), w = chi in, z FFT of
// every box column of this rank, kz values stored into their owners' slabs.
template <int LZ, int IN>
__device__ VIE_SLAB_INLINE F slab_fwd(const InnerGroup<F>& g, int64_t voff, const F* chi, F* sm, const F* tw, F c1,
                                      F c2, F c3) {
    constexpr int H = LZ / 2 > 0 ? LZ / 2 : 1, LG = ILog2<LZ>::v;
    const int bx = g.bx, by = g.by, bz = g.bz, plane = bx * by, ncol = 3 * plane;
    const int rk = team_rank(), R = team_size(), bxp = g.bxp;
    const FastDiv dbx = fd_of(g.fd_bx), dcol = fd_of(g.fd_col);
    const int64_t box = (int64_t)plane * bz;
    F acc = czero<F>();
    for (int col = rk * blockDim.x + threadIdx.x; col < ncol; col += R * blockDim.x) {
        const int comp = (int)fdiv(col, dcol), yx = col - comp * plane;
        const int y = (int)fdiv(yx, dbx), x = yx - y * bx;
        const int64_t e0 = voff + comp * box + yx;
        F a[H];
#pragma unroll
        for (int j0 = 0; j0 < H; j0 += kSlabBatch) {
            F ra[kSlabBatch], pa[kSlabBatch], va[kSlabBatch], ca[kSlabBatch], xa[kSlabBatch], ta[kSlabBatch];
#pragma unroll
            for (int u = 0; u < kSlabBatch; ++u) {       // every load of the batch first
                const int j = j0 + u;
                if (j < H && j < bz) {
                    const int64_t e = e0 + (int64_t)j * plane;
                    ra[u] = IN == IN_PX ? g.s[e] : g.r[e];
                    va[u] = g.v[e];
                    if (IN != IN_S) pa[u] = g.p[e];
                    if (IN == IN_PX) {
                        ta[u] = g.t[e];
                        xa[u] = g.x[e];
                    }
                    ca[u] = chi[j * plane + yx];
                }
            }
#pragma unroll
            for (int u = 0; u < kSlabBatch; ++u) {
                const int j = j0 + u;
                if (j >= H) continue;
                F w = czero<F>();
                if (j < bz) {
                    const int64_t e = e0 + (int64_t)j * plane;
                    F in;
                    if (IN == IN_PX) {
                        const F rr = ra[u] - cmul(c2, ta[u]);
                        g.r[e] = rr;
                        g.x[e] = xa[u] + cmul(c3, pa[u]) + cmul(c2, ra[u]);
                        in = rr + cmul(c1, pa[u] - cmul(c2, va[u]));
                        g.p[e] = in;
                    } else if (IN == IN_P) {
                        in = ra[u] + cmul(c1, pa[u] - cmul(c2, va[u]));
                        g.p[e] = in;
                    } else {
                        in = ra[u] - cmul(c1, va[u]);
                        g.s[e] = in;
                        acc.x += in.x * in.x + in.y * in.y;
                    }
                    w = cmul(in, ca[u]);
                }
                a[j] = w;
            }
        }
        const int off = comp * by * bxp + y * bxp + x;
        fwd_half<LZ>([&](int j) { return a[j]; }, [&](int k, F v) { slab_tab[cbrev(k, LG)][off] = v; }, tw);
    }
    return acc;
}

// Offset (in complex64 entries) of the staged spectrum rows after `used` entries: 16-byte aligned.
__host__ __device__ __forceinline__ int slab_gs_offset(int used) { return (used + 1) & ~1; }

// 3x3 symmetric Green multiply of the point q (components cs apart) with the octant entries and the
// sign flips of a point in the negative half of an axis (xy odd in x, y; xz in x, z; yz in y, z).
__device__ __forceinline__ void green_pt(F* q, int cs, const F (&gv)[6], int fx, int fy, int fz) {
    const F gxy = (fx ^ fy) ? make_float2(-gv[1].x, -gv[1].y) : gv[1];
    const F gxz = (fx ^ fz) ? make_float2(-gv[2].x, -gv[2].y) : gv[2];
    const F gyz = (fy ^ fz) ? make_float2(-gv[4].x, -gv[4].y) : gv[4];
    const F X = q[0], Y = q[cs], Z = q[2 * cs];
    q[0] = cmul(gv[0], X) + cmul(gxy, Y) + cmul(gxz, Z);
    q[cs] = cmul(gxy, X) + cmul(gv[3], Y) + cmul(gyz, Z);
    q[2 * cs] = cmul(gxz, X) + cmul(gyz, Y) + cmul(gv[5], Z);
}

// Plane stage: this rank's kz planes, npl at a time, through x and y FFTs, the Green multiply and
// the inverse y and x FFTs in the workspace after the slab.
template <int LX, int LY>
__device__ VIE_SLAB_INLINE void slab_planes(const InnerGroup<F>& g, F* sm, const F* tw) {
    constexpr int LGX = ILog2<LX>::v, LGY = ILog2<LY>::v, HX = LX / 2, HY = LY / 2;
    const int bx = g.bx, by = g.by, Mz = g.Mz;
    const int rk = team_rank(), R = team_size(), P = Mz / R, bxp = g.bxp, zpl = 3 * by * bxp;
    constexpr int wp = LX + 1, cs = LY * wp, wpl = 3 * cs;
    F* ws = sm + P * zpl;
    const int T = blockDim.x, t = threadIdx.x;
    constexpr int nkx = HX + 1, nky = HY + 1, ntk = nkx * nky;
    const F* Go = g.Go;
    // octant spectrum rows of the round's kz pairs, staged in shared memory while x and y transform
    F* gs = sm + slab_gs_offset(P * zpl + g.npl * wpl);
    for (int s0 = 0; s0 < P; s0 += g.npl) {
        const int np = min(g.npl, P - s0);
        const int nrow = np * 3 * by;
        {
            // row kz of the octant is 6 * ntk contiguous entries (a multiple of 16 bytes); the pair of
            // rank 0's self-mirror planes (kz = 0 and Mz/2) takes two rows, every other pair one
            constexpr int n16 = 6 * ntk / 2;          // 16-byte chunks per row
            const int npair = np >> 1;
            const bool two0 = rk == 0 && s0 == 0;
            const int nrows = npair + (two0 ? 1 : 0);
            for (int i = t; i < nrows * n16; i += T) {
                const int row = i / n16, c16 = i - row * n16;
                int kz;
                if (two0) kz = row == 0 ? 0 : (row == 1 ? Mz / 2 : slab_kz(rk, 2 * (row - 1), P, Mz));
                else kz = slab_kz(rk, s0 + 2 * row, P, Mz);
                const int kf = kz > Mz / 2 ? Mz - kz : kz;
                cp_async16(gs + (int64_t)row * 6 * ntk + 2 * c16, Go + (int64_t)kf * 6 * ntk + 2 * c16);
            }
        }
        // x forward: rows (plane, component, y < by) of the slab into the workspace (natural kx)
        for (int task = t; task < nrow; task += T) {
            const int pc = task / by, y = task - pc * by;           // pc = plane * 3 + component
            const F* src = sm + s0 * zpl + pc * by * bxp + y * bxp;
            F* dst = ws + pc * cs + y * wp;
            F in[HX];
#pragma unroll
            for (int j = 0; j < HX; ++j) in[j] = j < bx ? src[j] : czero<F>();
            fwd_half<LX>([&](int j) { return in[j]; }, [&](int k, F v) { dst[cbrev(k, LGX)] = v; }, tw);
        }
        __syncthreads();
        // y forward: columns (plane, component, kx), in place (natural ky)
        const int ncw = np * 3 * LX;
        for (int task = t; task < ncw; task += T) {
            const int kx = task & (LX - 1), pc = task >> LGX;
            F* colp = ws + pc * cs + kx;
            F in[HY];
#pragma unroll
            for (int j = 0; j < HY; ++j) in[j] = j < by ? colp[j * wp] : czero<F>();
            fwd_half<LY>([&](int j) { return in[j]; }, [&](int k, F v) { colp[cbrev(k, LGY) * wp] = v; }, tw);
        }
        cp_async_wait_all();                    // this thread's spectrum copies; the barrier publishes all
        __syncthreads();
        // Green multiply: one task per (pair of planes, ky, kx); the point's octant entry (kyf, kxf) and
        // the sign flips of its negative-half axes come from the staged rows
        const int ntask = (np >> 1) * LY * LX;
        for (int task = t; task < ntask; task += T) {
            const int kx = task & (LX - 1), r0 = task >> LGX;
            const int ky = r0 & (LY - 1), pp = r0 >> LGY;
            const int fx = kx > HX, fy = ky > HY;
            const int q = (fy ? LY - ky : ky) * nkx + (fx ? LX - kx : kx);
            const int sa = s0 + 2 * pp;
            const int kza = slab_kz(rk, sa, P, Mz), kzb = slab_kz(rk, sa + 1, P, Mz);
            const int fza = kza > Mz / 2, fzb = kzb > Mz / 2;
            const bool two0 = rk == 0 && s0 == 0;     // staged rows: see the prefetch above
            const int rowa = two0 ? (pp == 0 ? 0 : pp + 1) : pp;
            F ga[6], gb[6];
            const F* p0 = gs + rowa * 6 * ntk + q;
#pragma unroll
            for (int c = 0; c < 6; ++c) ga[c] = p0[c * ntk];
            if (two0 && pp == 0) {
                const F* p1 = gs + 6 * ntk + q;        // rank 0's kz = Mz/2 row
#pragma unroll
                for (int c = 0; c < 6; ++c) gb[c] = p1[c * ntk];
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) gb[c] = ga[c];
            }
            F* qa = ws + (2 * pp) * wpl + ky * wp + kx;
            green_pt(qa, cs, ga, fx, fy, fza);
            green_pt(qa + wpl, cs, gb, fx, fy, fzb);
        }
        __syncthreads();
        // y inverse: columns, keep y < by
        for (int task = t; task < ncw; task += T) {
            const int kx = task & (LX - 1), pc = task >> LGX;
            F* colp = ws + pc * cs + kx;
            F st[HY];
            inv_half<LY>([&](int k) { return colp[cbrev(k, LGY) * wp]; }, [&](int j, F v) { st[j] = v; },
                         [&](int j) { return st[j]; },
                         [&](int j, F v) {
                             if (j < by) colp[j * wp] = v;
                         },
                         tw);
        }
        __syncthreads();
        // x inverse: rows, keep x < bx, back into the slab
        for (int task = t; task < nrow; task += T) {
            const int pc = task / by, y = task - pc * by;
            const F* src = ws + pc * cs + y * wp;
            F* dst = sm + s0 * zpl + pc * by * bxp + y * bxp;
            F st[HX];
            inv_half<LX>([&](int k) { return src[cbrev(k, LGX)]; }, [&](int j, F v) { st[j] = v; },
                         [&](int j) { return st[j]; },
                         [&](int j, F v) {
                             if (j < bx) dst[j] = v;
                         },
                         tw);
        }
        __syncthreads();
    }
}

// Inverse half: every box column of this rank gathers its kz values from their owners, inverse z
// FFT, out = mask (in - u) with the iteration's inner products (OUT_V: <rhat, v>; OUT_T: <t, s>,
// <t, t>; OUT_TX: those and <rhat, s>, <rhat, t>) accumulated into acc[0..3].
template <int LZ, int OUT>
__device__ VIE_SLAB_INLINE void slab_inv(const InnerGroup<F>& g, int64_t voff, const uint8_t* mask, F* sm,
                                         const F* tw, F (&acc)[4]) {
    constexpr int H = LZ / 2 > 0 ? LZ / 2 : 1, LG = ILog2<LZ>::v;
    const int bx = g.bx, by = g.by, bz = g.bz, plane = bx * by, ncol = 3 * plane;
    const int rk = team_rank(), R = team_size(), bxp = g.bxp;
    const FastDiv dbx = fd_of(g.fd_bx), dcol = fd_of(g.fd_col);
    const int64_t box = (int64_t)plane * bz;
    for (int col = rk * blockDim.x + threadIdx.x; col < ncol; col += R * blockDim.x) {
        const int comp = (int)fdiv(col, dcol), yx = col - comp * plane;
        const int y = (int)fdiv(yx, dbx), x = yx - y * bx;
        const int off = comp * by * bxp + y * bxp + x;
        F u[H];                                 // the stash of the FFT's upper half, then its output
        inv_half<LZ>([&](int k) { return slab_tab[cbrev(k, LG)][off]; }, [&](int j, F v) { u[j] = v; },
                     [&](int j) { return u[j]; }, [&](int j, F v) { u[j] = v; }, tw);
        const int64_t e0 = voff + comp * box + yx;
#pragma unroll
        for (int j0 = 0; j0 < H; j0 += kSlabBatch) {
            F ia[kSlabBatch], ha[kSlabBatch];
            uint8_t ma[kSlabBatch];
#pragma unroll
            for (int q = 0; q < kSlabBatch; ++q) {       // every load of the batch first
                const int j = j0 + q;
                if (j < H && j < bz) {
                    const int64_t e = e0 + (int64_t)j * plane;
                    ia[q] = OUT == OUT_V ? g.p[e] : g.s[e];
                    if (OUT != OUT_T) ha[q] = g.rhat[e];
                    ma[q] = mask[j * plane + yx];
                }
            }
#pragma unroll
            for (int q = 0; q < kSlabBatch; ++q) {
                const int j = j0 + q;
                if (j >= H || j >= bz) continue;
                const int64_t e = e0 + (int64_t)j * plane;
                const F o = ma[q] ? ia[q] - u[j] : czero<F>();
                if (OUT == OUT_V) {
                    g.v[e] = o;
                    acc_dot(acc[0], ha[q], o);
                } else {
                    g.t[e] = o;
                    acc_dot(acc[0], o, ia[q]);
                    acc[1].x += o.x * o.x + o.y * o.y;
                    if (OUT == OUT_TX) {
                        acc_dot(acc[2], ha[q], ia[q]);
                        acc_dot(acc[3], ha[q], o);
                    }
                }
            }
        }
    }
}

struct SlabMvm {
    static constexpr int kUV = 4;
    static constexpr bool kMerged = true;       // the x/r update rides in the next p update (IN_PX, OUT_TX)
    template <int IN>
    static __device__ __forceinline__ F fwd(const InnerGroup<F>& g, int64_t voff, F*, F*, const F* chi, F* sm,
                                            const F* tw, F c1, F c2, F c3 = czero<F>()) {
        F acc = czero<F>();
        slab_table(g, sm);
        VIE_LEN_SWITCH(g.lz, (acc = slab_fwd<LL, IN>(g, voff, chi, sm, tw, c1, c2, c3)));
        team_sync();                            // every rank's kz planes complete
        return acc;                             // this thread's part of ||s||^2 (IN_S), summed later
    }
    static __device__ __forceinline__ void mid(const InnerGroup<F>& g, F*, F* sm, const F* tw) {
        switch (g.lx) {
            case 3: { constexpr int AX = 8; VIE_LEN_SWITCH(g.ly, (slab_planes<AX, LL>(g, sm, tw))); } break;
            case 4: { constexpr int AX = 16; VIE_LEN_SWITCH(g.ly, (slab_planes<AX, LL>(g, sm, tw))); } break;
            default: { constexpr int AX = 32; VIE_LEN_SWITCH(g.ly, (slab_planes<AX, LL>(g, sm, tw))); } break;
        }
        team_sync();                            // every rank's planes back in its slab
    }
    // the team sum that follows (its cluster barrier) also ends every read of the slabs
    template <int OUT>
    static __device__ __forceinline__ void inv(const InnerGroup<F>& g, int64_t voff, F*, F*, const uint8_t* mask, F* sm,
                                               const F* tw, F (&acc)[4]) {
        VIE_LEN_SWITCH(g.lz, (slab_inv<LL, OUT>(g, voff, mask, sm, tw, acc)));
    }
    template <int OUT>
    static __device__ __forceinline__ void inv(const InnerGroup<F>& g, int64_t voff, F* W1, F* W2, const uint8_t* mask,
                                               F* sm, const F* tw, F& a1, F& a2) {
        F acc[4] = {a1, a2, czero<F>(), czero<F>()};
        inv<OUT>(g, voff, W1, W2, mask, sm, tw, acc);
        a1 = acc[0];
        a2 = acc[1];
    }
};

// BiCGSTAB state of the block being solved, in shared memory: written by thread 0
// inside team_sum (the FP64 scalar work of an iteration runs in that one thread)
// and read by every thread after the sum's closing barrier.
template <class C> struct BiState {
    double2 rho, rho_prev, alpha, omega;
    double tol2, bn2, res2, iters;
    int status, half;
    int pend;                                   // merged form: the last full step's x update is pending
    C cbeta, comega, calpha;                    // coefficients of the vector updates
};

// beta = (rho / rho_prev)(alpha / omega) for the next p update, or a breakdown.
template <class C> __device__ __forceinline__ void next_beta(BiState<C>& S) {
    if (!dgood(S.rho)) {
        S.status = SEG_BREAKDOWN;
        return;
    }
    const double2 beta = cmul(dcdiv(S.rho, S.rho_prev), dcdiv(S.alpha, S.omega));
    S.cbeta = cmk<C>(beta.x, beta.y);
    S.comega = cmk<C>(S.omega.x, S.omega.y);
}

template <class C, class Mvm>
__device__ __forceinline__ void solve_block(const InnerGroup<C>& g, int b, double tol, int maxit, C* sm, const C* tw,
                            double2* red, int* units) {
    const int64_t box = (int64_t)g.bx * g.by * g.bz;
    const int64_t n = 3 * box;
    const int64_t voff = (int64_t)b * n;
    C* W = g.w2 + (int64_t)b * 3 * g.bz * g.My * g.Mx;
    C* W1 = g.w1 + (int64_t)b * 3 * g.bz * g.by * g.Mx;
    const C* chi = g.chi + (int64_t)b * box;
    const uint8_t* mask = g.mask + (int64_t)b * box;
    __shared__ BiState<C> S;

    // x = 0, r = rhat = b, p = v = 0
    const int rk = team_rank(), nrk = team_size();
    const int64_t first = (int64_t)rk * Mvm::kUV * blockDim.x, step = (int64_t)nrk * Mvm::kUV * blockDim.x;
    C acc = czero<C>();
    for (int64_t i0 = first + threadIdx.x; i0 < n; i0 += step) {
        C bv[Mvm::kUV];
#pragma unroll
        for (int u = 0; u < Mvm::kUV; ++u) {
            const int64_t i = i0 + u * blockDim.x;
            if (i < n) bv[u] = g.b[voff + i];
        }
#pragma unroll
        for (int u = 0; u < Mvm::kUV; ++u) {
            const int64_t i = i0 + u * blockDim.x;
            if (i < n) {
                const int64_t e = voff + i;
                g.x[e] = czero<C>();
                g.r[e] = bv[u];
                g.rhat[e] = bv[u];
                g.p[e] = czero<C>();
                g.v[e] = czero<C>();
                acc.x += bv[u].x * bv[u].x + bv[u].y * bv[u].y;
            }
        }
    }
    team_sum(acc, czero<C>(), red, [&](double2 sa, double2) {
        const double bn2 = sa.x;
        S.bn2 = bn2;
        S.tol2 = tol * tol * bn2;
        S.rho = make_double2(bn2, 0.0);
        S.rho_prev = S.alpha = S.omega = make_double2(1, 0);
        S.iters = 0.0;
        S.res2 = bn2;
        S.half = 0;
        S.pend = 0;
        S.status = SEG_ACTIVE;
        if (!(bn2 > 0.0) || !isfinite(bn2)) S.status = bn2 == 0.0 ? SEG_CONVERGED : SEG_BREAKDOWN;
        else next_beta(S);
    });
    if constexpr (Mvm::kMerged) {
        // One pass and one sum fewer per iteration: r = s - omega t and x += alpha p + omega s are
        // applied in the next p update (IN_PX), and <rhat, r> = <rhat, s> - omega <rhat, t> and
        // ||r||^2 = ||s||^2 - |<t, s>|^2 / ||t||^2 come from the sums of the t pass (OUT_TX).
        for (int it = 0; it < maxit && S.status == SEG_ACTIVE; ++it) {
            if (it == 0) Mvm::template fwd<IN_P>(g, voff, W1, W, chi, sm, tw, S.cbeta, S.comega);
            else Mvm::template fwd<IN_PX>(g, voff, W1, W, chi, sm, tw, S.cbeta, S.comega, S.calpha);
            Mvm::mid(g, W, sm, tw);
            if (units != nullptr && rk == 0 && threadIdx.x == 0) atomicAdd(units, g.kb_mvm);
            C p1 = czero<C>(), p2 = czero<C>();
            Mvm::template inv<OUT_V>(g, voff, W1, W, mask, sm, tw, p1, p2);
            team_sum(p1, p2, red, [&](double2 sigma, double2) {
                S.pend = 0;                     // the p update took the previous step's x update
                if (!dgood(sigma)) {
                    S.status = SEG_BREAKDOWN;
                    return;
                }
                S.alpha = dcdiv(S.rho, sigma);
                S.calpha = cmk<C>(S.alpha.x, S.alpha.y);
            });
            if (S.status != SEG_ACTIVE) break;
            const C snp = Mvm::template fwd<IN_S>(g, voff, W1, W, chi, sm, tw, S.calpha, czero<C>());
            Mvm::mid(g, W, sm, tw);
            if (units != nullptr && rk == 0 && threadIdx.x == 0) atomicAdd(units, g.kb_mvm);
            C q4[4] = {czero<C>(), czero<C>(), czero<C>(), czero<C>()};
            Mvm::template inv<OUT_TX>(g, voff, W1, W, mask, sm, tw, q4);
            q4[1].y = snp.x;                    // the deferred ||s||^2 rides in the unused slot
            team_sum_n<4>(q4, red, [&](const double2 (&q)[4]) {
                const double2 ts = q[0], rs = q[2], rt = q[3];
                const double tt = q[1].x, sn2 = q[1].y;
                if (sn2 <= S.tol2) {
                    S.half = 1;
                    S.res2 = sn2;
                    S.iters += 0.5;
                    S.status = SEG_CONVERGED;
                    return;
                }
                if (!(tt > 0.0) || !isfinite(tt)) {
                    S.status = SEG_BREAKDOWN;
                    return;
                }
                S.omega = make_double2(ts.x / tt, ts.y / tt);
                S.comega = cmk<C>(S.omega.x, S.omega.y);
                S.pend = 1;
                S.rho_prev = S.rho;
                S.rho = make_double2(rs.x - (S.omega.x * rt.x - S.omega.y * rt.y),
                                     rs.y - (S.omega.x * rt.y + S.omega.y * rt.x));
                S.res2 = fmax(sn2 - (ts.x * ts.x + ts.y * ts.y) / tt, 0.0);
                S.iters += 1.0;
                if (!isfinite(S.res2)) S.status = SEG_BREAKDOWN;
                else if (S.res2 <= S.tol2) S.status = SEG_CONVERGED;
                else if (S.omega.x == 0.0 && S.omega.y == 0.0) S.status = SEG_BREAKDOWN;
                else next_beta(S);
            });
            if (S.half) {
                const C ac = S.calpha;          // half-step convergence: x += alpha p
                for (int64_t i = (int64_t)rk * blockDim.x + threadIdx.x; i < n; i += (int64_t)nrk * blockDim.x) {
                    int64_t e = voff + i;
                    g.x[e] = g.x[e] + cmul(ac, g.p[e]);
                }
                break;
            }
        }
        if (S.pend) {
            // the last full step's x update (no p update followed it)
            const C ac = S.calpha, oc = S.comega;
            for (int64_t i = (int64_t)rk * blockDim.x + threadIdx.x; i < n; i += (int64_t)nrk * blockDim.x) {
                int64_t e = voff + i;
                g.x[e] = g.x[e] + cmul(ac, g.p[e]) + cmul(oc, g.s[e]);
            }
        }
    } else {
    for (int it = 0; it < maxit && S.status == SEG_ACTIVE; ++it) {
        // v = A p, p = r + beta (p - omega v)
        Mvm::template fwd<IN_P>(g, voff, W1, W, chi, sm, tw, S.cbeta, S.comega);
        Mvm::mid(g, W, sm, tw);
        if (units != nullptr && rk == 0 && threadIdx.x == 0) atomicAdd(units, g.kb_mvm);
        C p1 = czero<C>(), p2 = czero<C>();
        Mvm::template inv<OUT_V>(g, voff, W1, W, mask, sm, tw, p1, p2);
        team_sum(p1, p2, red, [&](double2 sigma, double2) {
            if (!dgood(sigma)) {
                S.status = SEG_BREAKDOWN;
                return;
            }
            S.alpha = dcdiv(S.rho, sigma);
            S.calpha = cmk<C>(S.alpha.x, S.alpha.y);
        });
        if (S.status != SEG_ACTIVE) break;
        // s = r - alpha v and t = A s; ||s||^2 is summed together with <t,s> and <t,t>, so the
        // half-step test (same value, same decision) costs no reduction of its own
        const C snp = Mvm::template fwd<IN_S>(g, voff, W1, W, chi, sm, tw, S.calpha, czero<C>());
        Mvm::mid(g, W, sm, tw);
        if (units != nullptr && rk == 0 && threadIdx.x == 0) atomicAdd(units, g.kb_mvm + g.kb_upd);
        p1 = czero<C>();
        p2 = czero<C>();
        Mvm::template inv<OUT_T>(g, voff, W1, W, mask, sm, tw, p1, p2);
        p2.y = snp.x;                           // the deferred ||s||^2 rides in the unused slot
        team_sum(p1, p2, red, [&](double2 ts, double2 tt) {
            const double sn2 = tt.y;
            if (sn2 <= S.tol2) {
                S.half = 1;
                S.res2 = sn2;
                S.iters += 0.5;
                S.status = SEG_CONVERGED;
                return;
            }
            if (!(tt.x > 0.0) || !isfinite(tt.x)) {
                S.status = SEG_BREAKDOWN;
                return;
            }
            S.omega = make_double2(ts.x / tt.x, ts.y / tt.x);
            S.comega = cmk<C>(S.omega.x, S.omega.y);
        });
        if (S.half) {
            // half-step convergence: x += alpha p (t is not needed)
            const C ac = S.calpha;
            for (int64_t i = (int64_t)rk * blockDim.x + threadIdx.x; i < n; i += (int64_t)nrk * blockDim.x) {
                int64_t e = voff + i;
                g.x[e] = g.x[e] + cmul(ac, g.p[e]);
            }
            break;
        }
        if (S.status != SEG_ACTIVE) break;
        // x += alpha p + omega s, r = s - omega t; rho = <rhat, r>, ||r||^2
        const C ac = S.calpha, oc = S.comega;
        C a1 = czero<C>(), a2 = czero<C>();
        for (int64_t i0 = first + threadIdx.x; i0 < n; i0 += step) {
            C sv[Mvm::kUV], xv[Mvm::kUV], pv[Mvm::kUV], tv[Mvm::kUV], hv[Mvm::kUV];
#pragma unroll
            for (int u = 0; u < Mvm::kUV; ++u) {
                const int64_t i = i0 + u * blockDim.x;
                if (i < n) {
                    const int64_t e = voff + i;
                    sv[u] = g.s[e];
                    xv[u] = g.x[e];
                    pv[u] = g.p[e];
                    tv[u] = g.t[e];
                    hv[u] = g.rhat[e];
                }
            }
#pragma unroll
            for (int u = 0; u < Mvm::kUV; ++u) {
                const int64_t i = i0 + u * blockDim.x;
                if (i < n) {
                    const int64_t e = voff + i;
                    g.x[e] = xv[u] + cmul(ac, pv[u]) + cmul(oc, sv[u]);
                    C rv = sv[u] - cmul(oc, tv[u]);
                    g.r[e] = rv;
                    acc_dot(a1, hv[u], rv);
                    a2.x += rv.x * rv.x + rv.y * rv.y;
                }
            }
        }
        team_sum(a1, a2, red, [&](double2 r1, double2 r2) {
            S.rho_prev = S.rho;
            S.rho = r1;
            S.res2 = r2.x;
            S.iters += 1.0;
            if (!isfinite(S.res2)) S.status = SEG_BREAKDOWN;
            else if (S.res2 <= S.tol2) S.status = SEG_CONVERGED;
            else if (S.omega.x == 0.0 && S.omega.y == 0.0) S.status = SEG_BREAKDOWN;
            else next_beta(S);
        });
    }
    }
    if (rk == 0 && threadIdx.x == 0) {
        SegState& St = g.st[b];
        St.bnorm2 = S.bn2;
        St.res2 = S.res2;
        St.iters = S.iters;
        St.status = S.status == SEG_ACTIVE ? SEG_MAXIT : S.status;
        St.maxit = maxit;
    }
    __syncthreads();
}

template <bool SLAB>
__device__ __forceinline__ void solve_dispatch(const InnerGroup<double2>& g, int b, double tol, int maxit,
                                               double2* sm, const double2* tw, double2* red, int* units) {
    solve_block<double2, SmemMvm<double2>>(g, b, tol, maxit, sm, tw, red, units);
}
template <bool SLAB>
__device__ __forceinline__ void solve_dispatch(const InnerGroup<float2>& g, int b, double tol, int maxit,
                                               float2* sm, const float2* tw, double2* red, int* units) {
    if constexpr (SLAB) {
        if (g.slab) solve_block<float2, SlabMvm>(g, b, tol, maxit, sm, tw, red, units);
        else solve_block<float2, SmemMvm<float2>>(g, b, tol, maxit, sm, tw, red, units);
    } else {
        if (g.reg) solve_block<float2, RegMvm>(g, b, tol, maxit, sm, tw, red, units);
        else solve_block<float2, SmemMvm<float2>>(g, b, tol, maxit, sm, tw, red, units);
    }
}

// SLAB: the kernel of launches whose complex64 groups use the slab MVM (kSlabThreads threads,
// kSlabMinBlocks CTAs per SM at least); otherwise 256 threads and two CTAs per SM. npl: kz planes per
// round of the slab plane stage.
template <class C, bool SLAB>
__global__ void __launch_bounds__(SLAB ? kSlabThreads : kInnerThreads, SLAB ? kSlabMinBlocks : 2)
    k_inner(const InnerGroup<C>* groups, const int2* work, int nwork, int* next, double tol, int maxit, const C* tw,
            int* units, int npl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    __shared__ double2 red[kTeamSumMax * ((SLAB ? kSlabThreads : kInnerThreads) / 32)];   // per-warp sums
    __shared__ int item;
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x == 0) team_slot = 0;
    __syncthreads();
    for (;;) {
        // rank 0 of the cluster takes the next block; every rank reads it from rank 0's shared memory
        if (cl.block_rank() == 0 && threadIdx.x == 0) item = atomicAdd(next, 1);
        cl.sync();
        const int it = *cl.map_shared_rank(&item, 0);
        cl.sync();
        if (it >= nwork) break;
        const int2 wk = work[it];
        // descriptor in shared memory: fields are reloaded after barriers instead of held in registers
        __shared__ InnerGroup<C> gsh;
        if (threadIdx.x == 0) {
            gsh = groups[wk.x];
            if (gsh.Gb) gsh.G = gsh.Gb[wk.y];
            gsh.npl = npl;
        }
        __syncthreads();
        solve_dispatch<SLAB>(gsh, wk.y, gsh.tols ? gsh.tols[wk.y] : tol, maxit, sm, tw, red, units);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- host side
static int lg2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

constexpr size_t kInnerSmemBudget = 96 * 1024;

// CTAs per block (thread-block cluster size) forced by the environment variable
// VIE_INNER_CLUSTER (1, 2, 4 or 8; read once), or 0 when unset.
int inner_cluster_forced() {
    static const int r = [] {
        const char* e = getenv("VIE_INNER_CLUSTER");
        int v = e ? atoi(e) : 0;
        return (v == 1 || v == 2 || v == 4 || v == 8) ? v : 0;
    }();
    return r;
}

// VIE_SLAB_NPL = 2 or 4: kz planes per round of the slab plane stage (default: 4 where it fits)
static int slab_npl_forced() {
    static const int r = [] {
        const char* e = getenv("VIE_SLAB_NPL");
        const int v = e ? atoi(e) : 0;
        return (v == 2 || v == 4) ? v : 0;
    }();
    return r;
}

bool slab_disabled() {
    static const bool r = [] {
        const char* e = getenv("VIE_INNER_SLAB");
        return e != nullptr && atoi(e) == 0;
    }();
    return r;
}

// Tiles for one group; false when a single plane does not fit the budget.
static bool inner_tiles(const BoxSet& bs, size_t es, int* lpt, int* ltc, size_t* smem) {
    const size_t pe = (size_t)bs.My * (bs.Mx + 1) * es;
    if (pe > kInnerSmemBudget) return false;
    int l = 0;
    while (((size_t)2 << l) * pe <= kInnerSmemBudget && (1 << (l + 1)) <= 3 * bs.bz * 2 && l < 6) ++l;
    while ((size_t)(1 << l) * pe > kInnerSmemBudget) --l;
    int t = 0;
    while ((size_t)bs.Mz * 3 * ((size_t)2 << t) * es <= kInnerSmemBudget && ((int64_t)2 << t) <= (int64_t)bs.Mx * bs.My &&
           t < 7)
        ++t;
    *lpt = l;
    *ltc = t;
    *smem = std::max((size_t)(1 << l) * pe, (size_t)bs.Mz * 3 * ((size_t)1 << t) * es);
    return true;
}

// Register-FFT MVM: complex64 and every padded axis in [8, 32] (pencils in registers).
static bool reg_path_ok(const BoxSet& bs, size_t es) {
    auto ok = [](int m) { return m >= 8 && m <= 32; };
    return es == sizeof(float2) && ok(bs.Mx) && ok(bs.My) && ok(bs.Mz);
}
static size_t reg_smem(const BoxSet& bs) {
    size_t rows = (size_t)kInnerThreads * (bs.bx + 1 + bs.Mx + 1);
    size_t zc = (size_t)3 * bs.Mz * kZCols;
    return std::max(rows, zc) * sizeof(float2);
}

// m and s of FastDiv for divisor d >= 1: s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1.
static void make_fastdiv(unsigned d, unsigned (&out)[3]) {
    unsigned sh = 0;
    while ((1ull << sh) < d) ++sh;
    unsigned long long m = (((1ull << 32) * ((1ull << sh) - d)) / d) + 1;
    out[0] = (unsigned)m;
    out[1] = sh;
    out[2] = d;
}


// Slab MVM: complex64 boxes with every padded axis in [8, 32].
bool slab_path_ok(const BoxSet& bs, size_t es) { return reg_path_ok(bs, es); }
constexpr size_t kSlabSmemLimit = 220 * 1024;
// Dynamic shared memory of the slab MVM with R ranks per block and npl planes per round.
static size_t slab_smem(const BoxSet& bs, int R, int npl) {
    const size_t bxp = (size_t)(bs.bx | 1);
    const size_t zb = (size_t)(bs.Mz / R) * 3 * bs.by * bxp;
    const size_t ws = (size_t)npl * 3 * bs.My * (bs.Mx + 1);
    const size_t gs = (size_t)(npl / 2 + 1) * 6 * (bs.Mx / 2 + 1) * (bs.My / 2 + 1);   // staged spectrum rows
    return ((size_t)slab_gs_offset((int)(zb + ws)) + gs) * sizeof(float2);
}
// Smallest cluster size (1, 2 or 4) whose slab fits, or 0.
static int slab_min_ranks(const BoxSet& bs) {
    for (int R = 1; R <= 4; R *= 2)
        if (bs.Mz / R >= 2 && slab_smem(bs, R, 2) <= kSlabSmemLimit) return R;
    return 0;
}

bool inner_persistent_ok(const BoxSet& bs, size_t es, bool force) {
    int a, b;
    size_t s;
    return (force || bs.nb >= kInnerMinBlocks) && inner_tiles(bs, es, &a, &b, &s) &&
           (!reg_path_ok(bs, es) || reg_smem(bs) <= 160 * 1024);
}

template <class C>
int inner_persistent(const std::vector<InnerJob<C>>& jobs, const int2* d_work, int nwork, void* d_groups,
                     int* d_next, double tol, int maxit, cudaStream_t s, int cluster, const InnerSplit* split,
                     int npl_pref) {
    if (jobs.empty() || nwork == 0) return VIE_OK;
    Twiddles tw;
    VIE_TRY(get_twiddles(&tw));
    std::vector<InnerGroup<C>> hg(jobs.size());
    size_t smem = 0;
    int64_t bytes_per_block = 0;
    bool any_slab = false;
    int rmin_slab = 1, rmax_slab = 8;
    std::vector<const BoxSet*> slab_sets;
    for (size_t i = 0; i < jobs.size(); ++i) {
        const InnerJob<C>& j = jobs[i];
        const BoxSet& bs = *j.bs;
        InnerGroup<C>& g = hg[i];
        g.b = j.v.b; g.x = j.v.x; g.r = j.v.r; g.rhat = j.v.rhat; g.p = j.v.p; g.v = j.v.v; g.s = j.v.s; g.t = j.v.t;
        g.w1 = reinterpret_cast<C*>(bs.w1);
        g.w2 = reinterpret_cast<C*>(bs.w2);
        g.chi = j.chi;
        g.mask = bs.mask;
        g.G = j.G;
        g.Gb = j.Gb;
        g.tols = j.tols;
        g.st = j.st;
        g.nb = bs.nb; g.bx = bs.bx; g.by = bs.by; g.bz = bs.bz;
        g.Mx = bs.Mx; g.My = bs.My; g.Mz = bs.Mz; g.lx = bs.lx; g.ly = bs.ly; g.lz = bs.lz;
        g.lyb = lg2(bs.by);
        size_t sm = 0;
        if (!inner_tiles(bs, sizeof(C), &g.lpt, &g.ltc, &sm)) return fail(VIE_EINVAL, "box too large for the persistent solver");
        g.reg = reg_path_ok(bs, sizeof(C)) ? 1 : 0;
        make_fastdiv((unsigned)bs.bx, g.fd_bx);
        make_fastdiv((unsigned)(bs.bz * bs.by), g.fd_plane);
        make_fastdiv((unsigned)(bs.by * bs.bx), g.fd_col);
        g.slab = (j.Go != nullptr && slab_path_ok(bs, sizeof(C)) && slab_min_ranks(bs) > 0) ? 1 : 0;
        g.bxp = bs.bx | 1;
        g.npl = 2;
        g.Go = j.Go;
        if (g.slab) {
            any_slab = true;
            rmin_slab = std::max(rmin_slab, slab_min_ranks(bs));
            rmax_slab = std::min(rmax_slab, bs.Mz / 2);
            slab_sets.push_back(&bs);
        }
        if (g.reg) sm = reg_smem(bs);
        // algorithmic bytes of one MVM with its fused vector work: plane spectra written, read and
        // rewritten along z, read back (4 x [3][bz][My][Mx]), the Green spectrum once, chi and mask,
        // and the 4 box vectors the fused update/inverse phases touch; the x/r pass moves 6 vectors.
        const int64_t es = sizeof(C), box = bs.box_elems();
        const int64_t w2b = 3LL * bs.bz * bs.My * bs.Mx * es;
        const int64_t w1b = 3LL * bs.bz * bs.by * bs.Mx * es;
        // slab (merged BiCGSTAB): an iteration's two MVMs and fused passes move 17 box vectors
        const int64_t mvm = g.slab ? 6LL * bs.oct_elems() * es + box * (es + 1) + 17 * 3 * box * es / 2
                            : g.reg ? 4 * w1b + 4 * w2b + 6LL * bs.spec_elems() * es + box * (es + 1) + 7 * 3 * box * es
                                    : 4 * w2b + 6LL * bs.spec_elems() * es + box * (es + 1) + 4 * 3 * box * es;
        g.kb_mvm = (int)((mvm + 1023) / 1024);
        g.kb_upd = (int)((6 * 3 * box * es + 1023) / 1024);
        smem = std::max(smem, sm);
        bytes_per_block = std::max<int64_t>(bytes_per_block, 3 * bs.box_elems() * (int64_t)sizeof(C));
    }
    VIE_TRY(reg_twiddles_ready(tw));   // constant-memory twiddles of the register path
    VIE_CK(cudaMemcpyAsync(d_groups, hg.data(), hg.size() * sizeof(InnerGroup<C>), cudaMemcpyHostToDevice, s));
    const bool two = split != nullptr && split->nheavy > 0 && split->nheavy < nwork && !inner_cluster_forced();
    VIE_CK(cudaMemsetAsync(d_next, 0, (two ? 2 : 1) * sizeof(int), s));
    auto kern = any_slab ? k_inner<C, true> : k_inner<C, false>;
    // dynamic shared memory and planes per round of a launch with R CTAs per block
    auto launch_smem = [&](int R, int* npl) -> size_t {
        size_t m = smem;
        *npl = slab_npl_forced() ? slab_npl_forced() : (npl_pref == 2 ? 2 : 4);
        for (const BoxSet* b : slab_sets)
            if (slab_smem(*b, R, *npl) > kSlabSmemLimit) *npl = 2;
        for (const BoxSet* b : slab_sets) m = std::max(m, slab_smem(*b, R, *npl));
        return m;
    };
    // one block per cluster of R CTAs; as many clusters as fit at once, pulling blocks from the queue
    auto launch = [&](const int2* work, int n, int* next, int R, cudaStream_t st, int* units) -> int {
        if (any_slab) R = std::min(std::max(R, rmin_slab), rmax_slab);   // every rank holds >= 2 kz planes
        int npl = 2;
        const size_t sm_bytes = launch_smem(R, &npl);
        // opt in to the exact dynamic size: the default 48 KB limit also counts the static shared memory
        VIE_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_bytes));
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = R;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(R);
        cfg.blockDim = dim3(any_slab ? kSlabThreads : kInnerThreads);
        cfg.dynamicSmemBytes = sm_bytes;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        VIE_CK(cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg));
        if (nclusters < 1) return fail(VIE_EINVAL, "block solver: no cluster of this size fits on the device");
        cfg.gridDim = dim3(std::max(1, std::min(n, nclusters)) * R);
        cudaError_t le = cudaLaunchKernelEx(&cfg, kern, reinterpret_cast<const InnerGroup<C>*>(d_groups), work, n,
                                            next, tol, maxit, tw_of<C>(tw), units, npl);
        if (le != cudaSuccess) return cuda_fail(le, "cudaLaunchKernelEx(k_inner)", __FILE__, __LINE__);
        return VIE_OK;
    };
    const int R = inner_cluster_forced() ? inner_cluster_forced() : (cluster > 0 ? cluster : 2);
    (void)bytes_per_block;
    // the kernels add the KB they move (per MVM) to one profiling counter; the profiled interval
    // covers both parts of a split launch
    int* units = prof_begin(s, PK_INNER, sizeof(C) == 16 ? VIE_C128 : VIE_C64, 1024, 0, true);
    int rc = VIE_OK;
    if (!two) {
        rc = launch(d_work, nwork, d_next, R, s, units);
    } else {
        // the heavy part first, so its clusters are resident before the light part fills the GPU
        cudaError_t e = cudaEventRecord(split->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(split->s2, split->fork, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "split launch fork", __FILE__, __LINE__);
        if (!rc) rc = launch(d_work, split->nheavy, d_next, split->cluster, s, units);
        if (!rc) rc = launch(d_work + split->nheavy, nwork - split->nheavy, d_next + 1, R, split->s2, units);
        e = cudaEventRecord(split->join, split->s2);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, split->join, 0);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "split launch join", __FILE__, __LINE__);
    }
    prof_end(s);
    if (rc) return rc;
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template int inner_persistent<double2>(const std::vector<InnerJob<double2>>&, const int2*, int, void*, int*, double,
                                       int, cudaStream_t, int, const InnerSplit*, int);
template int inner_persistent<float2>(const std::vector<InnerJob<float2>>&, const int2*, int, void*, int*, double, int,
                                      cudaStream_t, int, const InnerSplit*, int);

__global__ void k_slab_spectrum(const double2* __restrict__ G, float2* __restrict__ Go, int Mx, int My, int Mz, int lx,
                                int ly, int lz) {
    const int nkx = Mx / 2 + 1, nky = My / 2 + 1, nkz = Mz / 2 + 1;
    const int64_t n = (int64_t)nkz * 6 * nky * nkx;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % nkx);
        int64_t t = i / nkx;
        const int ky = (int)(t % nky);
        t /= nky;
        const int c = (int)(t % 6), kz = (int)(t / 6);
        const int64_t px = bit_reverse(kx, lx), py = bit_reverse(ky, ly), pz = bit_reverse(kz, lz);
        const double2 v = G[((c * (int64_t)Mz + pz) * My + py) * Mx + px];
        Go[i] = make_float2((float)v.x, (float)v.y);
    }
}

int slab_spectrum(const BoxSet& bs, const double2* G, float2* Go, cudaStream_t s) {
    const int64_t n = 6 * bs.oct_elems();
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_slab_spectrum<<<blocks, 256, 0, s>>>(G, Go, bs.Mx, bs.My, bs.Mz, bs.lx, bs.ly, bs.lz);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

size_t inner_group_desc_bytes() { return std::max(sizeof(InnerGroup<double2>), sizeof(InnerGroup<float2>)); }

}  // namespace vie
