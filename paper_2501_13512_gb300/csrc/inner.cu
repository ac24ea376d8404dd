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
#include "fft_core.cuh"
#include "vie_internal.cuh"

namespace vie {

template <class C> struct InnerGroup {
    C *b, *x, *r, *rhat, *p, *v, *s, *t;   // [nb][3][bz][by][bx]
    C* w2;                                  // [nb][3][bz][My][Mx]
    const C* chi;                           // [nb][bz][by][bx]
    const uint8_t* mask;                    // [nb][bz][by][bx]
    const C* G;                             // [6][Mz][My][Mx], bit-reversed positions
    SegState* st;                           // [nb]
    int nb, bx, by, bz, Mx, My, Mz, lx, ly, lz, lyb;   // lyb = log2 of nextpow2(by)
    int lpt;                                // log2 planes per XY tile
    int ltc;                                // log2 columns per Z tile
    int kb_mvm;                             // profiling: KB moved by one MVM and its fused updates
    int kb_upd;                             // profiling: KB moved by the x/r update pass
};

constexpr int kInnerThreads = 256;

template <class C> __device__ __forceinline__ double2 wide(C a);
template <> __device__ __forceinline__ double2 wide<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ double2 wide<float2>(float2 a) { return make_double2(a.x, a.y); }

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

// CTA-wide sum of two complex values (FP64), returned to every thread.
__device__ void cta_sum2(double2& a, double2& b, double2* red) {
    for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_down_sync(0xffffffffu, a.x, o);
        a.y += __shfl_down_sync(0xffffffffu, a.y, o);
        b.x += __shfl_down_sync(0xffffffffu, b.x, o);
        b.y += __shfl_down_sync(0xffffffffu, b.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
    __syncthreads();
    double2 sa = make_double2(0, 0), sb = make_double2(0, 0);
    for (int i = 0; i < nw; ++i) {   // fixed order: identical result in every thread
        sa.x += red[2 * i].x; sa.y += red[2 * i].y;
        sb.x += red[2 * i + 1].x; sb.y += red[2 * i + 1].y;
    }
    a = sa;
    b = sb;
}

enum { IN_P = 0, IN_S = 1 };
enum { OUT_V = 0, OUT_T = 1 };

// Phase XY: plane tiles, fused vector update + chi, 2D forward FFT, store spectrum.
// IN_P: p = r + beta (p - omega v);  IN_S: s = r - alpha v (returns ||s||^2 in .x).
template <class C, int IN>
__device__ double2 phase_xy(const InnerGroup<C>& g, int64_t voff, C* W, const C* chi, C* sm, const C* tw,
                            C c1, C c2, double2* red) {
    const int planes = 3 * g.bz, P = g.Mx + 1, pe = g.My * P, tile = 1 << g.lpt;
    const int64_t box = (int64_t)g.bx * g.by * g.bz;
    C acc = czero<C>();
    for (int pl0 = 0; pl0 < planes; pl0 += tile) {
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
    double2 a = wide<C>(acc), z = make_double2(0, 0);
    cta_sum2(a, z, red);
    return a;
}

// Phase Z: forward FFT along z, Green multiply, inverse FFT (columns of the plane spectra).
template <class C>
__device__ void phase_z(const InnerGroup<C>& g, C* W, C* sm, const C* tw) {
    const int TC = 1 << g.ltc, pitch = 3 * TC;
    const int64_t plane = (int64_t)g.My * g.Mx;
    const int64_t cstride = (int64_t)g.bz * plane, gcomp = (int64_t)g.Mz * plane;
    const int L = g.Mz;
    for (int64_t c0 = 0; c0 < plane; c0 += TC) {
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
                             const C* tw, double2* red, double2& d1, double2& d2) {
    const int planes = 3 * g.bz, P = g.Mx + 1, pe = g.My * P, tile = 1 << g.lpt;
    const int64_t box = (int64_t)g.bx * g.by * g.bz;
    C a1 = czero<C>(), a2 = czero<C>();
    for (int pl0 = 0; pl0 < planes; pl0 += tile) {
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
    d1 = wide<C>(a1);
    d2 = wide<C>(a2);
    cta_sum2(d1, d2, red);
}

template <class C>
__device__ void solve_block(const InnerGroup<C>& g, int b, double tol, int maxit, C* sm, const C* tw,
                            double2* red, int* units) {
    const int64_t box = (int64_t)g.bx * g.by * g.bz;
    const int64_t n = 3 * box;
    const int64_t voff = (int64_t)b * n;
    C* W = g.w2 + (int64_t)b * 3 * g.bz * g.My * g.Mx;
    const C* chi = g.chi + (int64_t)b * box;
    const uint8_t* mask = g.mask + (int64_t)b * box;

    // x = 0, r = rhat = b, p = v = 0
    C acc = czero<C>();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        int64_t e = voff + i;
        C bv = g.b[e];
        g.x[e] = czero<C>();
        g.r[e] = bv;
        g.rhat[e] = bv;
        g.p[e] = czero<C>();
        g.v[e] = czero<C>();
        acc.x += bv.x * bv.x + bv.y * bv.y;
    }
    double2 d1 = wide<C>(acc), d2 = make_double2(0, 0);
    cta_sum2(d1, d2, red);
    const double bn2 = d1.x;
    const double tol2 = tol * tol * bn2;
    double2 rho = make_double2(bn2, 0.0), rho_prev = make_double2(1, 0), alpha = make_double2(1, 0),
            omega = make_double2(1, 0);
    double iters = 0.0, res2 = bn2;
    int status = SEG_ACTIVE;
    if (!(bn2 > 0.0) || !isfinite(bn2)) status = bn2 == 0.0 ? SEG_CONVERGED : SEG_BREAKDOWN;
    for (int it = 0; it < maxit && status == SEG_ACTIVE; ++it) {
        if (!dgood(rho)) { status = SEG_BREAKDOWN; break; }
        double2 beta = cmul(dcdiv(rho, rho_prev), dcdiv(alpha, omega));
        // v = A p, p = r + beta (p - omega v)
        phase_xy<C, IN_P>(g, voff, W, chi, sm, tw, cmk<C>(beta.x, beta.y), cmk<C>(omega.x, omega.y), red);
        phase_z<C>(g, W, sm, tw);
        if (units != nullptr && threadIdx.x == 0) atomicAdd(units, g.kb_mvm);
        double2 sigma, unused;
        phase_xy_inv<C, OUT_V>(g, voff, W, mask, sm, tw, red, sigma, unused);
        if (!dgood(sigma)) { status = SEG_BREAKDOWN; break; }
        alpha = dcdiv(rho, sigma);
        // s = r - alpha v, and its transform for t = A s
        double2 sn = phase_xy<C, IN_S>(g, voff, W, chi, sm, tw, cmk<C>(alpha.x, alpha.y), czero<C>(), red);
        if (sn.x <= tol2) {
            // half-step convergence: x += alpha p
            C ac = cmk<C>(alpha.x, alpha.y);
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
                int64_t e = voff + i;
                g.x[e] = g.x[e] + cmul(ac, g.p[e]);
            }
            iters += 0.5;
            res2 = sn.x;
            status = SEG_CONVERGED;
            break;
        }
        phase_z<C>(g, W, sm, tw);
        if (units != nullptr && threadIdx.x == 0) atomicAdd(units, g.kb_mvm + g.kb_upd);
        double2 ts, tt;
        phase_xy_inv<C, OUT_T>(g, voff, W, mask, sm, tw, red, ts, tt);
        if (!(tt.x > 0.0) || !isfinite(tt.x)) { status = SEG_BREAKDOWN; break; }
        omega = make_double2(ts.x / tt.x, ts.y / tt.x);
        // x += alpha p + omega s, r = s - omega t; rho = <rhat, r>, ||r||^2
        C ac = cmk<C>(alpha.x, alpha.y), oc = cmk<C>(omega.x, omega.y);
        C a1 = czero<C>(), a2 = czero<C>();
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            int64_t e = voff + i;
            C sv = g.s[e];
            g.x[e] = g.x[e] + cmul(ac, g.p[e]) + cmul(oc, sv);
            C rv = sv - cmul(oc, g.t[e]);
            g.r[e] = rv;
            acc_dot(a1, g.rhat[e], rv);
            a2.x += rv.x * rv.x + rv.y * rv.y;
        }
        d1 = wide<C>(a1);
        d2 = wide<C>(a2);
        cta_sum2(d1, d2, red);
        rho_prev = rho;
        rho = d1;
        res2 = d2.x;
        iters += 1.0;
        if (!isfinite(res2)) { status = SEG_BREAKDOWN; break; }
        if (res2 <= tol2) { status = SEG_CONVERGED; break; }
        if (omega.x == 0.0 && omega.y == 0.0) { status = SEG_BREAKDOWN; break; }
    }
    if (status == SEG_ACTIVE) status = SEG_MAXIT;
    if (threadIdx.x == 0) {
        SegState& S = g.st[b];
        S.bnorm2 = bn2;
        S.res2 = res2;
        S.iters = iters;
        S.status = status;
        S.maxit = maxit;
    }
    __syncthreads();
}

template <class C>
__global__ void __launch_bounds__(kInnerThreads) k_inner(const InnerGroup<C>* groups, const int2* work, int nwork,
                                                          int* next, double tol, int maxit, const C* tw,
                                                          int* units) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    __shared__ double2 red[2 * (kInnerThreads / 32)];
    __shared__ int item;
    for (;;) {
        if (threadIdx.x == 0) item = atomicAdd(next, 1);
        __syncthreads();
        const int it = item;
        __syncthreads();
        if (it >= nwork) break;
        const int2 wk = work[it];
        solve_block<C>(groups[wk.x], wk.y, tol, maxit, sm, tw, red, units);
    }
}

// ---------------------------------------------------------------- host side
static int lg2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

constexpr size_t kInnerSmemBudget = 96 * 1024;

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

bool inner_persistent_ok(const BoxSet& bs, size_t es, bool force) {
    int a, b;
    size_t s;
    return (force || bs.nb >= kInnerMinBlocks) && inner_tiles(bs, es, &a, &b, &s);
}

template <class C>
int inner_persistent(const std::vector<InnerJob<C>>& jobs, const int2* d_work, int nwork, void* d_groups,
                     int* d_next, double tol, int maxit, cudaStream_t s) {
    if (jobs.empty() || nwork == 0) return VIE_OK;
    Twiddles tw;
    VIE_TRY(get_twiddles(&tw));
    std::vector<InnerGroup<C>> hg(jobs.size());
    size_t smem = 0;
    int64_t bytes_per_block = 0;
    for (size_t i = 0; i < jobs.size(); ++i) {
        const InnerJob<C>& j = jobs[i];
        const BoxSet& bs = *j.bs;
        InnerGroup<C>& g = hg[i];
        g.b = j.v.b; g.x = j.v.x; g.r = j.v.r; g.rhat = j.v.rhat; g.p = j.v.p; g.v = j.v.v; g.s = j.v.s; g.t = j.v.t;
        g.w2 = reinterpret_cast<C*>(bs.w2);
        g.chi = j.chi;
        g.mask = bs.mask;
        g.G = j.G;
        g.st = j.st;
        g.nb = bs.nb; g.bx = bs.bx; g.by = bs.by; g.bz = bs.bz;
        g.Mx = bs.Mx; g.My = bs.My; g.Mz = bs.Mz; g.lx = bs.lx; g.ly = bs.ly; g.lz = bs.lz;
        g.lyb = lg2(bs.by);
        size_t sm = 0;
        if (!inner_tiles(bs, sizeof(C), &g.lpt, &g.ltc, &sm)) return fail(VIE_EINVAL, "box too large for the persistent solver");
        // algorithmic bytes of one MVM with its fused vector work: plane spectra written, read and
        // rewritten along z, read back (4 x [3][bz][My][Mx]), the Green spectrum once, chi and mask,
        // and the 4 box vectors the fused update/inverse phases touch; the x/r pass moves 6 vectors.
        const int64_t es = sizeof(C), box = bs.box_elems();
        const int64_t w2b = 3LL * bs.bz * bs.My * bs.Mx * es;
        const int64_t mvm = 4 * w2b + 6LL * bs.spec_elems() * es + box * (es + 1) + 4 * 3 * box * es;
        g.kb_mvm = (int)((mvm + 1023) / 1024);
        g.kb_upd = (int)((6 * 3 * box * es + 1023) / 1024);
        smem = std::max(smem, sm);
        bytes_per_block = std::max<int64_t>(bytes_per_block, 3 * bs.box_elems() * (int64_t)sizeof(C));
    }
    VIE_CK(cudaMemcpyAsync(d_groups, hg.data(), hg.size() * sizeof(InnerGroup<C>), cudaMemcpyHostToDevice, s));
    VIE_CK(cudaMemsetAsync(d_next, 0, sizeof(int), s));
    // opt in to the exact dynamic size: the default 48 KB limit also counts the static shared memory
    VIE_CK(cudaFuncSetAttribute(k_inner<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, nsm = 0, per = 0;
    VIE_CK(cudaGetDevice(&dev));
    VIE_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    VIE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_inner<C>, kInnerThreads, smem));
    int grid = std::max(1, std::min(nwork, nsm * std::max(1, per)));
    // the kernel adds the KB it moves (per MVM) to its profiling counter
    (void)bytes_per_block;
    int* units = prof_begin(s, PK_INNER, sizeof(C) == 16 ? VIE_C128 : VIE_C64, 1024, 0, true);
    k_inner<C><<<grid, kInnerThreads, smem, s>>>(reinterpret_cast<const InnerGroup<C>*>(d_groups), d_work, nwork,
                                                 d_next, tol, maxit, tw_of<C>(tw), units);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template int inner_persistent<double2>(const std::vector<InnerJob<double2>>&, const int2*, int, void*, int*, double,
                                       int, cudaStream_t);
template int inner_persistent<float2>(const std::vector<InnerJob<float2>>&, const int2*, int, void*, int*, double, int,
                                      cudaStream_t);

size_t inner_group_desc_bytes() { return std::max(sizeof(InnerGroup<double2>), sizeof(InnerGroup<float2>)); }

}  // namespace vie
