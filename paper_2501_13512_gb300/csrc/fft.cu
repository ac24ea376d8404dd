// Pencil FFT passes and the FFT-accelerated MVM y = x - G(chi x) (Section I;
// Eq. 4 discretised on the voxel grid).
//
// Every 3D transform is split into three batched 1D passes. Forward passes are
// radix-4 (plus one radix-2) decimation-in-frequency: natural order in,
// bit-reversed order out. Inverse passes are decimation-in-time: bit-reversed
// in, natural out. Intermediate spectra therefore live in bit-reversed
// position order on every axis, and the Green spectrum is generated in the
// same order, so no pass ever reorders data.
//
// One MVM over a batch of boxes (BoxSet; the full grid is the batch of one):
//   pass X  rows of bx -> chi * x, zero-pad to Mx, forward   -> w1 [3][bz][by][Mx]
//   pass Y  columns of by -> zero-pad to My, forward         -> w2 [3][bz][My][Mx]
//   pass Z  columns of bz -> zero-pad to Mz, forward, 3x3 symmetric Green
//           multiply, inverse, keep z < bz                   -> w2 (in place)
//   pass Y' inverse, keep y < by                             -> w1
//   pass X' inverse, keep x < bx, y = x - u (masked)         -> y
// Each pass stages a tile of pencils in shared memory; global accesses are
// along the contiguous x axis in every pass.
#include <algorithm>
#include <type_traits>

#include "fft_core.cuh"
#include "fft_reg.cuh"
#include "vie_internal.cuh"

namespace vie {

constexpr int kThreads = 256;
constexpr int kSmemBudget = 32 * 1024;

__device__ __forceinline__ bool box_active(const SegState* st, int b) {
    return st == nullptr || st[b].status == SEG_ACTIVE;
}

// ---------------------------------------------------------------- pass X (rows)
enum RowMode { ROW_FWD_CHI = 0, ROW_INV_UPDATE = 1, ROW_FWD_PLAIN = 2 };

template <class C> struct RowArgs {
    const C* in;
    C* out;
    const C* chi;        // ROW_FWD_CHI: [nb][bz][by][bx]
    const C* xin;        // ROW_INV_UPDATE: x, same layout as out
    const uint8_t* mask; // ROW_INV_UPDATE: optional [nb][bz][by][bx]
    const SegState* st;  // optional per-box status
    const C* tw;
    int64_t nrows;
    int in_stride, out_stride, n_in, n_out, lL, ltr, twshift;
    int rows_per_box;    // 3 * bz * by
    int plane;           // bz * by
    int bx;
    int* units;          // profiling: boxes processed (null when off)
};

template <class C, int MODE>
__global__ void __launch_bounds__(kThreads) k_rows(RowArgs<C> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int TR = 1 << a.ltr;
    const int pitch = TR + 1;          // odd pitch: conflict-free transposed staging
    const int L = 1 << a.lL;
    const int64_t row0 = (int64_t)blockIdx.x * TR;
    if (a.units != nullptr && threadIdx.x == 0) {
        const int64_t rpb = a.rows_per_box;
        for (int64_t b = (row0 + rpb - 1) / rpb; b * rpb < row0 + TR && b * rpb < a.nrows; ++b)
            if (box_active(a.st, (int)b)) atomicAdd(a.units, 1);
    }

    for (int idx = threadIdx.x; idx < TR * a.n_in; idx += blockDim.x) {
        int r = idx / a.n_in, i = idx - r * a.n_in;
        int64_t row = row0 + r;
        C v = czero<C>();
        if (row < a.nrows) {
            int b = (int)(row / a.rows_per_box);
            if (box_active(a.st, b)) {
                v = a.in[row * a.in_stride + i];
                if (MODE == ROW_FWD_CHI) {
                    int64_t crow = (int64_t)b * a.plane + (row % a.plane);
                    v = cmul(v, a.chi[crow * a.bx + i]);
                }
            }
        }
        buf[i * pitch + r] = v;
    }
    for (int idx = threadIdx.x; idx < TR * (L - a.n_in); idx += blockDim.x) {
        int i = a.n_in + idx / TR, r = idx % TR;
        buf[i * pitch + r] = czero<C>();
    }
    __syncthreads();
    smem_fft<C, MODE != ROW_INV_UPDATE, 1>(buf, a.lL, pitch, a.ltr, a.tw, a.twshift);
    for (int idx = threadIdx.x; idx < TR * a.n_out; idx += blockDim.x) {
        int r = idx / a.n_out, i = idx - r * a.n_out;
        int64_t row = row0 + r;
        if (row >= a.nrows) continue;
        int b = (int)(row / a.rows_per_box);
        if (!box_active(a.st, b)) continue;
        C v = buf[i * pitch + r];
        if (MODE == ROW_INV_UPDATE) {
            int64_t o = row * a.out_stride + i;
            v = a.xin[o] - v;
            if (a.mask != nullptr) {
                int64_t mrow = (int64_t)b * a.plane + (row % a.plane);
                if (!a.mask[mrow * a.bx + i]) v = czero<C>();
            }
            a.out[o] = v;
        } else {
            a.out[row * a.out_stride + i] = v;
        }
    }
}

// ---------------------------------------------------------------- pass Y / spectrum passes (columns)
template <class C> struct ColArgs {
    const C* in;
    C* out;
    const SegState* st;
    const C* tw;
    int ncols, n_in, n_out, lL, ltc, twshift;
    int64_t in_axis, out_axis, in_s1, out_s1, in_s2, out_s2;
    int b2_per_box;      // blockIdx.z / b2_per_box = box index
    int* units;
};

template <class C, bool FWD>
__global__ void __launch_bounds__(kThreads) k_cols(ColArgs<C> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int TC = 1 << a.ltc;
    const int L = 1 << a.lL;
    const int col0 = blockIdx.x * TC;
    if (!box_active(a.st, blockIdx.z / a.b2_per_box)) return;   // uniform per CTA
    if (a.units != nullptr && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 &&
        blockIdx.z % a.b2_per_box == 0)
        atomicAdd(a.units, 1);
    const C* in = a.in + blockIdx.z * a.in_s2 + blockIdx.y * a.in_s1 + col0;
    C* out = a.out + blockIdx.z * a.out_s2 + blockIdx.y * a.out_s1 + col0;
    const int ncol = min(TC, a.ncols - col0);

    for (int idx = threadIdx.x; idx < L * TC; idx += blockDim.x) {
        int i = idx >> a.ltc, c = idx & (TC - 1);
        C v = czero<C>();
        if (i < a.n_in && c < ncol) v = in[i * a.in_axis + c];
        buf[idx] = v;
    }
    __syncthreads();
    smem_fft<C, FWD, 1>(buf, a.lL, TC, a.ltc, a.tw, a.twshift);
    for (int idx = threadIdx.x; idx < a.n_out * TC; idx += blockDim.x) {
        int i = idx >> a.ltc, c = idx & (TC - 1);
        if (c < ncol) out[i * a.out_axis + c] = buf[idx];
    }
}

// ---------------------------------------------------------------- pass Z fused with the Green multiply
template <class C> struct ZArgs {
    C* w;                 // w2 of the BoxSet
    const C* G;           // [6][Mz][My][Mx], or [6][Mz/2+1][My/2+1][Mx/2+1] when oct
    const C* const* Gb;   // optional: one spectrum per box (instances with their own wavenumber)
    const SegState* st;
    const C* tw;
    int ncols, nzb, lL, ltc, twshift;
    int oct, lx, ly;      // octant-compressed spectrum; log2 Mx, log2 My
    int nine;             // nine full spectra G_ab (3a + b), general 3x3 multiply
    int64_t axis, comp_stride, box_stride, gcomp;
    int* units;
};

template <class C>
__global__ void __launch_bounds__(kThreads) k_zgreen(ZArgs<C> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int TC = 1 << a.ltc;
    const int L = 1 << a.lL;
    const int pitch = 3 * TC;
    const int col0 = blockIdx.x * TC;
    const int b = blockIdx.y;
    if (!box_active(a.st, b)) return;
    if (a.units != nullptr && threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(a.units, 1);
    C* w = a.w + b * a.box_stride + col0;
    const int ncol = min(TC, a.ncols - col0);

    for (int idx = threadIdx.x; idx < L * 3 * TC; idx += blockDim.x) {
        int c = idx & (TC - 1), t = idx >> a.ltc;
        int comp = t % 3, i = t / 3;
        C v = czero<C>();
        if (i < a.nzb && c < ncol) v = w[comp * a.comp_stride + i * a.axis + c];
        buf[idx] = v;     // idx == i * pitch + comp * TC + c
    }
    __syncthreads();
    smem_fft<C, true, 3>(buf, a.lL, pitch, a.ltc, a.tw, a.twshift);
    for (int idx = threadIdx.x; idx < L * TC; idx += blockDim.x) {
        int c = idx & (TC - 1), i = idx >> a.ltc;
        if (c >= ncol) continue;
        const C* g = a.Gb ? a.Gb[b] : a.G;
        bool ux = false, uy = false, uz = false;
        if (a.oct) {
            const int col = col0 + c;
            const int qx = octant_slot(col & ((1 << a.lx) - 1), a.lx, ux);
            const int qy = octant_slot(col >> a.lx, a.ly, uy);
            const int qz = octant_slot(i, a.lL, uz);
            g += ((int64_t)qz * ((1 << a.ly) / 2 + 1) + qy) * ((1 << a.lx) / 2 + 1) + qx;
        } else {
            g += i * a.axis + col0 + c;
        }
        if (a.nine) {
            C* p = buf + i * pitch + c;
            const C X = p[0], Y = p[TC], Z = p[2 * TC];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                p[r * TC] = cmul(g[(3 * r) * a.gcomp], X) + cmul(g[(3 * r + 1) * a.gcomp], Y) +
                            cmul(g[(3 * r + 2) * a.gcomp], Z);
            continue;
        }
        C gxx = g[0], gxy = g[a.gcomp], gxz = g[2 * a.gcomp];
        C gyy = g[3 * a.gcomp], gyz = g[4 * a.gcomp], gzz = g[5 * a.gcomp];
        if (ux != uy) gxy = mk(-gxy.x, -gxy.y);
        if (ux != uz) gxz = mk(-gxz.x, -gxz.y);
        if (uy != uz) gyz = mk(-gyz.x, -gyz.y);
        C* p = buf + i * pitch + c;
        C X = p[0], Y = p[TC], Z = p[2 * TC];
        p[0] = cmul(gxx, X) + cmul(gxy, Y) + cmul(gxz, Z);
        p[TC] = cmul(gxy, X) + cmul(gyy, Y) + cmul(gyz, Z);
        p[2 * TC] = cmul(gxz, X) + cmul(gyz, Y) + cmul(gzz, Z);
    }
    __syncthreads();
    smem_fft<C, false, 3>(buf, a.lL, pitch, a.ltc, a.tw, a.twshift);
    for (int idx = threadIdx.x; idx < a.nzb * 3 * TC; idx += blockDim.x) {
        int c = idx & (TC - 1), t = idx >> a.ltc;
        int comp = t % 3, i = t / 3;
        if (c < ncol) w[comp * a.comp_stride + i * a.axis + c] = buf[idx];
    }
}

// Pass Z of complex64 MVMs with Mz <= 32, register-resident: each thread
// transforms one (component, column) pencil in registers (pruned: the box
// fills at most the lower half of the padded axis), the three transformed
// components of kZRegCols columns meet in shared memory for the 3x3 Green
// multiply, and each thread transforms its pencil back, keeping z < bz. The
// spectrum is even in z for xx, xy, yy, zz and odd for xz, yz, so one load of
// its six entries serves the z positions of frequencies f and -f.
constexpr int kZRegCols = 64;
constexpr int kZRegThreads = 3 * kZRegCols;

template <int LZ>
__global__ void __launch_bounds__(kZRegThreads) k_zgreen_reg(ZArgs<float2> a) {
    typedef float2 F;
    constexpr int H = LZ / 2 > 0 ? LZ / 2 : 1;
    constexpr int LGZ = ILog2<LZ>::v;
    constexpr int NC = kZRegCols;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F* sm = reinterpret_cast<F*>(smem_raw);          // [3][LZ][NC]
    const int b = blockIdx.y;
    if (!box_active(a.st, b)) return;
    if (a.units != nullptr && threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(a.units, 1);
    const int P = a.ncols, bz = a.nzb, c0 = blockIdx.x * NC, t = threadIdx.x;
    const int nc = min(NC, P - c0);
    F* W = a.w + (int64_t)b * a.box_stride + c0;
    const int64_t cs = a.comp_stride;
    {
        const int comp = t / NC, c = t - comp * NC;
        if (c < nc) {
            const F* src = W + comp * cs + c;
            F* S = sm + comp * LZ * NC + c;
            if (LZ == 1) {
                S[0] = src[0];
            } else {
                F v[H];
#pragma unroll
                for (int j = 0; j < H; ++j) v[j] = j < bz ? src[(int64_t)j * P] : czero<F>();
                F q[H];
#pragma unroll
                for (int j = 0; j < H; ++j) q[j] = twc<true>(v[j], j * (kLmax / LZ));
                rfft<H, true>(q, (const F*)nullptr);
#pragma unroll
                for (int j = 0; j < H; ++j) S[(H + j) * NC] = q[j];
                rfft<H, true>(v, (const F*)nullptr);
#pragma unroll
                for (int j = 0; j < H; ++j) S[j * NC] = v[j];
            }
        }
    }
    __syncthreads();
    const F* G = a.Gb ? a.Gb[b] : a.G;
    const int hx = (1 << a.lx) / 2 + 1, hy = (1 << a.ly) / 2 + 1;
    const int cst = LZ * NC;
    for (int task = t; task < LZ * NC; task += kZRegThreads) {
        const int i = task / NC, c = task - i * NC;
        if (c >= nc) continue;
        const int f = LGZ ? (int)(__brev((unsigned)i) >> (32 - LGZ)) : 0;
        const int fm = (LZ - f) & (LZ - 1);
        const int im = LGZ ? (int)(__brev((unsigned)fm) >> (32 - LGZ)) : 0;
        if (im < i) continue;
        const int col = c0 + c;
        bool ux, uy, uz;
        const int qx = octant_slot(col & ((1 << a.lx) - 1), a.lx, ux);
        const int qy = octant_slot(col >> a.lx, a.ly, uy);
        const int qz = octant_slot(i, LGZ, uz);
        const F* gp = G + ((int64_t)qz * hy + qy) * hx + qx;
        const F gxx = gp[0], gyy = gp[3 * a.gcomp], gzz = gp[5 * a.gcomp];
        F gxy = gp[a.gcomp], gxz = gp[2 * a.gcomp], gyz = gp[4 * a.gcomp];
        if (ux != uy) gxy = mk(-gxy.x, -gxy.y);
        if (ux != uz) gxz = mk(-gxz.x, -gxz.y);
        if (uy != uz) gyz = mk(-gyz.x, -gyz.y);
        {
            F* q = sm + i * NC + c;
            const F X = q[0], Y = q[cst], Z = q[2 * cst];
            q[0] = cmul(gxx, X) + cmul(gxy, Y) + cmul(gxz, Z);
            q[cst] = cmul(gxy, X) + cmul(gyy, Y) + cmul(gyz, Z);
            q[2 * cst] = cmul(gxz, X) + cmul(gyz, Y) + cmul(gzz, Z);
        }
        if (im != i) {   // frequency -f: xz and yz change sign
            F* q = sm + im * NC + c;
            const F X = q[0], Y = q[cst], Z = q[2 * cst];
            q[0] = cmul(gxx, X) + cmul(gxy, Y) - cmul(gxz, Z);
            q[cst] = cmul(gxy, X) + cmul(gyy, Y) - cmul(gyz, Z);
            q[2 * cst] = cmul(gzz, Z) - cmul(gxz, X) - cmul(gyz, Y);
        }
    }
    __syncthreads();
    {
        const int comp = t / NC, c = t - comp * NC;
        if (c < nc) {
            F* S = sm + comp * LZ * NC + c;
            F* dst = W + comp * cs + c;
            if (LZ == 1) {
                dst[0] = S[0];
            } else {
                F u[H], v[H];
#pragma unroll
                for (int j = 0; j < H; ++j) v[j] = S[(H + j) * NC];
                rfft<H, false>(v, (const F*)nullptr);
#pragma unroll
                for (int j = 0; j < H; ++j) u[j] = S[j * NC];
                rfft<H, false>(u, (const F*)nullptr);
#pragma unroll
                for (int j = 0; j < H; ++j)
                    if (j < bz) dst[(int64_t)j * P] = u[j] + twc<false>(v[j], j * (kLmax / LZ));
            }
        }
    }
}

// ---------------------------------------------------------------- four-step register passes (complex64)
// An L = 32 A point transform (A = 2 .. 32) of a line as two register passes
// with one shared-memory exchange, instead of log2 L shared-memory stages.
// Forward (decimation in frequency, natural -> bit-reversed, as smem_fft):
//   step A  thread j < 32 holds the positions j + 32 m (m < A) and applies the
//           radix-2 stages of spans L/2 .. 32; the pair (p, p + S) with p =
//           j + 32 mm (mm < S/32) takes the twiddle W_L^{p L/(2S)}, which is
//           W_Lmax^{16 j / s} W_Lmax^{512 mm / s} with s = S/32: one runtime
//           factor per stage and a compile-time one per pair;
//   step B  thread g < A holds the 32 positions 32 g + r and applies the
//           stages of spans 16 .. 1: a 32-point transform with compile-time
//           twiddles (rfft<32>).
// Inverse (decimation in time, bit-reversed -> natural): step B then step A,
// with conjugate twiddles in reverse span order. Inputs of the forward pass
// are zero beyond L/2 and outputs of the inverse pass beyond L/2 are dropped
// (pruning: a box of n voxels is padded to L >= 2n - 1).
constexpr int kB4 = 32;

template <int A>
__device__ __forceinline__ void step_a_fwd(float2 (&v)[A], int j, const float2* __restrict__ tw) {
#pragma unroll
    for (int sp = A / 2; sp >= 1; sp >>= 1) {
        const float2 wj = __ldg(&tw[(16 * j) / sp]);
#pragma unroll
        for (int m = 0; m < A; ++m) {
            if ((m & sp) != 0) continue;
            const int mm = m & (sp - 1);
            const float2 x0 = v[m], x1 = v[m + sp];
            v[m] = x0 + x1;
            v[m + sp] = twc<true>(cmul(x0 - x1, wj), (512 / sp) * mm);
        }
    }
}

// Inverse step A; only the outputs m < A/2 are formed by the last stage.
template <int A>
__device__ __forceinline__ void step_a_inv(float2 (&v)[A], int j, const float2* __restrict__ tw) {
#pragma unroll
    for (int sp = 1; sp <= A / 2; sp <<= 1) {
        const float2 wj = __ldg(&tw[(16 * j) / sp]);
#pragma unroll
        for (int m = 0; m < A; ++m) {
            if ((m & sp) != 0) continue;
            const int mm = m & (sp - 1);
            const float2 x0 = v[m];
            const float2 x1 = cmulc(twc<false>(v[m + sp], (512 / sp) * mm), wj);
            v[m] = x0 + x1;
            if (sp < A / 2) v[m + sp] = x0 - x1;
        }
    }
}

// shared-memory index of position p of a line: one pad per 32 positions
__device__ __forceinline__ int pad32(int p) { return p + (p >> 5); }

constexpr int kRows4 = 8;   // rows per CTA (256 threads: 8 rows x 32)

// Pass X forward: rows of bx -> chi * x, zero-padded to L = 32 A, forward transform.
template <int A>
__global__ void __launch_bounds__(256) k_rows4_fwd(RowArgs<float2> a) {
    constexpr int L = kB4 * A, LP = L + L / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);     // [kRows4][LP]
    const int64_t row0 = (int64_t)blockIdx.x * kRows4;
    if (a.units != nullptr && threadIdx.x == 0) {
        const int64_t rpb = a.rows_per_box;
        for (int64_t b = (row0 + rpb - 1) / rpb; b * rpb < row0 + kRows4 && b * rpb < a.nrows; ++b)
            if (box_active(a.st, (int)b)) atomicAdd(a.units, 1);
    }
    {
        const int r = threadIdx.x >> 5, j = threadIdx.x & 31;
        const int64_t row = row0 + r;
        float2 v[A];
        bool live = row < a.nrows;
        int b = 0;
        if (live) {
            b = (int)(row / a.rows_per_box);
            live = box_active(a.st, b);
        }
        const int64_t crow = live ? (int64_t)b * a.plane + (row % a.plane) : 0;
#pragma unroll
        for (int m = 0; m < A; ++m) {
            v[m] = czero<float2>();
            const int p = j + kB4 * m;
            if (m < A / 2 && live && p < a.n_in) v[m] = cmul(a.in[row * a.in_stride + p], a.chi[crow * a.bx + p]);
        }
        step_a_fwd<A>(v, j, a.tw);
#pragma unroll
        for (int m = 0; m < A; ++m) sm[r * LP + pad32(j + kB4 * m)] = v[m];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kRows4 * A; t += blockDim.x) {
        const int r = t / A, g = t - r * A;
        float2* q = sm + r * LP + g * (kB4 + 1);
        float2 u[kB4];
#pragma unroll
        for (int i = 0; i < kB4; ++i) u[i] = q[i];
        rfft<kB4, true>(u, (const float2*)nullptr);
#pragma unroll
        for (int i = 0; i < kB4; ++i) q[i] = u[i];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kRows4 * L; idx += blockDim.x) {
        const int r = idx / L, p = idx - r * L;
        const int64_t row = row0 + r;
        if (row >= a.nrows || !box_active(a.st, (int)(row / a.rows_per_box))) continue;
        a.out[row * a.out_stride + p] = sm[r * LP + pad32(p)];
    }
}

// Pass X inverse: rows of L = 32 A spectrum positions -> keep x < bx, y = mask (x - u).
template <int A>
__global__ void __launch_bounds__(256) k_rows4_inv(RowArgs<float2> a) {
    constexpr int L = kB4 * A, LP = L + L / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);     // [kRows4][LP]
    const int64_t row0 = (int64_t)blockIdx.x * kRows4;
    if (a.units != nullptr && threadIdx.x == 0) {
        const int64_t rpb = a.rows_per_box;
        for (int64_t b = (row0 + rpb - 1) / rpb; b * rpb < row0 + kRows4 && b * rpb < a.nrows; ++b)
            if (box_active(a.st, (int)b)) atomicAdd(a.units, 1);
    }
    for (int idx = threadIdx.x; idx < kRows4 * L; idx += blockDim.x) {
        const int r = idx / L, p = idx - r * L;
        const int64_t row = row0 + r;
        float2 v = czero<float2>();
        if (row < a.nrows && box_active(a.st, (int)(row / a.rows_per_box))) v = a.in[row * a.in_stride + p];
        sm[r * LP + pad32(p)] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kRows4 * A; t += blockDim.x) {
        const int r = t / A, g = t - r * A;
        float2* q = sm + r * LP + g * (kB4 + 1);
        float2 u[kB4];
#pragma unroll
        for (int i = 0; i < kB4; ++i) u[i] = q[i];
        rfft<kB4, false>(u, (const float2*)nullptr);
#pragma unroll
        for (int i = 0; i < kB4; ++i) q[i] = u[i];
    }
    __syncthreads();
    const int r = threadIdx.x >> 5, j = threadIdx.x & 31;
    const int64_t row = row0 + r;
    if (row >= a.nrows) return;
    const int b = (int)(row / a.rows_per_box);
    if (!box_active(a.st, b)) return;
    float2 v[A];
#pragma unroll
    for (int m = 0; m < A; ++m) v[m] = sm[r * LP + pad32(j + kB4 * m)];
    step_a_inv<A>(v, j, a.tw);
    const int64_t mrow = (int64_t)b * a.plane + (row % a.plane);
#pragma unroll
    for (int m = 0; m < A / 2; ++m) {
        const int p = j + kB4 * m;
        if (p >= a.n_out) continue;
        const int64_t o = row * a.out_stride + p;
        float2 y = a.xin[o] - v[m];
        if (a.mask != nullptr && !a.mask[mrow * a.bx + p]) y = czero<float2>();
        a.out[o] = y;
    }
}

constexpr int kCols4 = 16;   // columns per CTA (512 threads: 16 columns x 32)

// Pass Y (forward or inverse) over columns of L = 32 A, 16 adjacent columns per CTA.
template <int A, bool FWD>
__global__ void __launch_bounds__(512) k_cols4(ColArgs<float2> a) {
    constexpr int L = kB4 * A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* sm = reinterpret_cast<float2*>(smem_raw);     // [L][kCols4]
    const int col0 = blockIdx.x * kCols4;
    if (!box_active(a.st, blockIdx.z / a.b2_per_box)) return;
    if (a.units != nullptr && threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0 &&
        blockIdx.z % a.b2_per_box == 0)
        atomicAdd(a.units, 1);
    const float2* in = a.in + blockIdx.z * a.in_s2 + blockIdx.y * a.in_s1 + col0;
    float2* out = a.out + blockIdx.z * a.out_s2 + blockIdx.y * a.out_s1 + col0;
    const int ncol = min(kCols4, a.ncols - col0);
    const int c = threadIdx.x % kCols4, k = threadIdx.x / kCols4;    // k: j (step A) or g (step B)
    if (FWD) {
        if (c < ncol) {
            float2 v[A];
#pragma unroll
            for (int m = 0; m < A; ++m) {
                const int p = k + kB4 * m;
                v[m] = (m < A / 2 && p < a.n_in) ? in[p * a.in_axis + c] : czero<float2>();
            }
            step_a_fwd<A>(v, k, a.tw);
#pragma unroll
            for (int m = 0; m < A; ++m) sm[(k + kB4 * m) * kCols4 + c] = v[m];
        }
        __syncthreads();
        if (k < A && c < ncol) {
            float2 u[kB4];
#pragma unroll
            for (int i = 0; i < kB4; ++i) u[i] = sm[(kB4 * k + i) * kCols4 + c];
            rfft<kB4, true>(u, (const float2*)nullptr);
#pragma unroll
            for (int i = 0; i < kB4; ++i)
                if (kB4 * k + i < a.n_out) out[(kB4 * k + i) * a.out_axis + c] = u[i];
        }
    } else {
        if (k < A && c < ncol) {
            float2 u[kB4];
#pragma unroll
            for (int i = 0; i < kB4; ++i) u[i] = in[(kB4 * k + i) * a.in_axis + c];
            rfft<kB4, false>(u, (const float2*)nullptr);
#pragma unroll
            for (int i = 0; i < kB4; ++i) sm[(kB4 * k + i) * kCols4 + c] = u[i];
        }
        __syncthreads();
        if (c < ncol) {
            float2 v[A];
#pragma unroll
            for (int m = 0; m < A; ++m) v[m] = sm[(k + kB4 * m) * kCols4 + c];
            step_a_inv<A>(v, k, a.tw);
#pragma unroll
            for (int m = 0; m < A / 2; ++m) {
                const int p = k + kB4 * m;
                if (p < a.n_out) out[p * a.out_axis + c] = v[m];
            }
        }
    }
}

// ---------------------------------------------------------------- host side
static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// log2 of the pencils per CTA: as many as fit the shared-memory budget, at most 32.
static int pick_ltile(int lL, size_t esize, int ncomp, int pad) {
    int lt = 5;
    while (lt > 0 && (size_t)((1 << lL)) * (size_t)(ncomp * (1 << lt) + pad) * esize > (size_t)kSmemBudget) --lt;
    return lt;
}

template <class C> static const C* tw_ptr(const Twiddles& t);
template <> const double2* tw_ptr<double2>(const Twiddles& t) { return t.d128; }
template <> const float2* tw_ptr<float2>(const Twiddles& t) { return t.d64; }

template <class K>
static int prep_smem(K kernel, size_t bytes) {
    if (bytes > 46 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    }
    return VIE_OK;
}

struct Prof {
    int kind;
    int64_t bpu, fixed;
};
template <class C> static int prec_code() { return sizeof(C) == 16 ? VIE_C128 : VIE_C64; }

template <int A, bool FWD>
static int launch_rows4(RowArgs<float2> a, Prof pf, cudaStream_t s) {
    constexpr int L = kB4 * A;
    const size_t smem = (size_t)kRows4 * (L + L / 32) * sizeof(float2);
    auto kern = FWD ? k_rows4_fwd<A> : k_rows4_inv<A>;
    VIE_TRY(prep_smem(kern, smem));
    const int64_t grid = (a.nrows + kRows4 - 1) / kRows4;
    if (grid <= 0) return VIE_OK;
    a.units = prof_begin(s, pf.kind, VIE_C64, pf.bpu, pf.fixed, true);
    kern<<<(unsigned)grid, 256, smem, s>>>(a);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <bool FWD>
static int launch_rows4_any(RowArgs<float2> a, Prof pf, cudaStream_t s) {
    switch (a.lL) {
        case 6: return launch_rows4<2, FWD>(a, pf, s);
        case 7: return launch_rows4<4, FWD>(a, pf, s);
        case 8: return launch_rows4<8, FWD>(a, pf, s);
        case 9: return launch_rows4<16, FWD>(a, pf, s);
        default: return launch_rows4<32, FWD>(a, pf, s);
    }
}

template <class C, int MODE>
static int launch_rows(RowArgs<C> a, Prof pf, cudaStream_t s) {
    if constexpr (std::is_same<C, float2>::value) {
        // four-step register path: complex64 MVM rows of 64 .. 1024, pruned to half the length
        const int L = 1 << a.lL;
        if (a.lL >= 6 && a.lL <= kLogLmax) {
            if (MODE == ROW_FWD_CHI && 2 * a.n_in <= L && a.n_out == L) return launch_rows4_any<true>(a, pf, s);
            if (MODE == ROW_INV_UPDATE && 2 * a.n_out <= L && a.n_in == L) return launch_rows4_any<false>(a, pf, s);
        }
    }
    a.ltr = pick_ltile(a.lL, sizeof(C), 1, 1);
    const int TR = 1 << a.ltr;
    size_t smem = (size_t)(1 << a.lL) * (TR + 1) * sizeof(C);
    VIE_TRY(prep_smem(k_rows<C, MODE>, smem));
    int64_t grid = (a.nrows + TR - 1) / TR;
    if (grid <= 0) return VIE_OK;
    a.units = prof_begin(s, pf.kind, prec_code<C>(), pf.bpu, pf.fixed, true);
    k_rows<C, MODE><<<(unsigned)grid, kThreads, smem, s>>>(a);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <int A, bool FWD>
static int launch_cols4(ColArgs<float2> a, int nb1, int nb2, Prof pf, cudaStream_t s) {
    const size_t smem = (size_t)kB4 * A * kCols4 * sizeof(float2);
    VIE_TRY(prep_smem(k_cols4<A, FWD>, smem));
    dim3 grid((a.ncols + kCols4 - 1) / kCols4, nb1, nb2);
    a.units = prof_begin(s, pf.kind, VIE_C64, pf.bpu, pf.fixed, true);
    k_cols4<A, FWD><<<grid, kB4 * kCols4, smem, s>>>(a);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <class C, bool FWD>
static int launch_cols(ColArgs<C> a, int nb1, int nb2, Prof pf, cudaStream_t s) {
    if constexpr (std::is_same<C, float2>::value) {
        // four-step register path: complex64 columns of 64 .. 1024, pruned to half the length
        const int L = 1 << a.lL;
        if (a.lL >= 6 && a.lL <= kLogLmax && (FWD ? (2 * a.n_in <= L && a.n_out == L)
                                                   : (2 * a.n_out <= L && a.n_in == L))) {
            switch (a.lL) {
                case 6: return launch_cols4<2, FWD>(a, nb1, nb2, pf, s);
                case 7: return launch_cols4<4, FWD>(a, nb1, nb2, pf, s);
                case 8: return launch_cols4<8, FWD>(a, nb1, nb2, pf, s);
                case 9: return launch_cols4<16, FWD>(a, nb1, nb2, pf, s);
                default: return launch_cols4<32, FWD>(a, nb1, nb2, pf, s);
            }
        }
    }
    a.ltc = pick_ltile(a.lL, sizeof(C), 1, 0);
    if ((1 << a.ltc) > a.ncols) a.ltc = ilog2(a.ncols) - ((1 << ilog2(a.ncols)) > a.ncols ? 1 : 0);
    if (a.ltc < 0) a.ltc = 0;
    const int TC = 1 << a.ltc;
    size_t smem = (size_t)(1 << a.lL) * TC * sizeof(C);
    VIE_TRY(prep_smem(k_cols<C, FWD>, smem));
    dim3 grid((a.ncols + TC - 1) / TC, nb1, nb2);
    a.units = prof_begin(s, pf.kind, prec_code<C>(), pf.bpu, pf.fixed, true);
    k_cols<C, FWD><<<grid, kThreads, smem, s>>>(a);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <int LZ>
static int launch_zgreen_reg(ZArgs<float2> a, int nb, Prof pf, cudaStream_t s) {
    const size_t smem = (size_t)3 * LZ * kZRegCols * sizeof(float2);
    VIE_TRY(prep_smem(k_zgreen_reg<LZ>, smem));
    dim3 grid((a.ncols + kZRegCols - 1) / kZRegCols, nb);
    a.units = prof_begin(s, pf.kind, VIE_C64, pf.bpu, pf.fixed, true);
    k_zgreen_reg<LZ><<<grid, kZRegThreads, smem, s>>>(a);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <class C>
static int launch_zgreen(ZArgs<C> a, int nb, Prof pf, cudaStream_t s) {
    if constexpr (std::is_same<C, float2>::value) {
        if (a.oct && a.lL <= 5) {   // register path: complex64, octant spectrum, Mz <= 32
            switch (a.lL) {
                case 0: return launch_zgreen_reg<1>(a, nb, pf, s);
                case 1: return launch_zgreen_reg<2>(a, nb, pf, s);
                case 2: return launch_zgreen_reg<4>(a, nb, pf, s);
                case 3: return launch_zgreen_reg<8>(a, nb, pf, s);
                case 4: return launch_zgreen_reg<16>(a, nb, pf, s);
                default: return launch_zgreen_reg<32>(a, nb, pf, s);
            }
        }
    }
    a.ltc = pick_ltile(a.lL, sizeof(C), 3, 0);
    if ((1 << a.ltc) > a.ncols) a.ltc = ilog2(a.ncols) - ((1 << ilog2(a.ncols)) > a.ncols ? 1 : 0);
    if (a.ltc < 0) a.ltc = 0;
    const int TC = 1 << a.ltc;
    size_t smem = (size_t)(1 << a.lL) * 3 * TC * sizeof(C);
    VIE_TRY(prep_smem(k_zgreen<C>, smem));
    dim3 grid((a.ncols + TC - 1) / TC, nb);
    a.units = prof_begin(s, pf.kind, prec_code<C>(), pf.bpu, pf.fixed, true);
    k_zgreen<C><<<grid, kThreads, smem, s>>>(a);
    prof_end(s);
    VIE_CK(cudaGetLastError());
    return VIE_OK;
}

template <class C> static const C* chi_ptr(const BoxSet& bs);
template <> const double2* chi_ptr<double2>(const BoxSet& bs) { return bs.chi128; }
template <> const float2* chi_ptr<float2>(const BoxSet& bs) { return bs.chi64; }

template <class C>
int mvm_boxes(const BoxSet& bs, const C* G, const C* x, C* y, const SegState* st, cudaStream_t s,
              const Twiddles* twp, const C* const* Gb, const C* xupd, bool nine) {
    Twiddles tw;
    if (twp) tw = *twp;
    else VIE_TRY(get_twiddles(&tw));
    const C* T = tw_ptr<C>(tw);
    if (sizeof(C) == sizeof(float2)) VIE_TRY(reg_twiddles_ready(tw));   // constant table of the register passes
    C* w1 = reinterpret_cast<C*>(bs.w1);
    C* w2 = reinterpret_cast<C*>(bs.w2);
    const int64_t planeXY = (int64_t)bs.Mx * bs.My;
    // algorithmic bytes per box of each pass (inputs read + outputs written)
    const int64_t es = sizeof(C);
    const int64_t box = bs.box_elems();
    const int64_t b1 = 3LL * bs.bz * bs.by * bs.Mx * es;          // w1 per box
    const int64_t b2 = 3LL * bs.bz * planeXY * es;                // w2 per box
    const int64_t bv = 3LL * box * es;                            // x or y per box
    const Prof px{PK_X_FWD, bv + box * es + b1, 0};
    const Prof py{PK_Y_FWD, b1 + b2, 0};
    const Prof pz{PK_Z_GREEN, 2 * b2, (nine ? 9LL : 6LL) * (bs.oct ? bs.oct_elems() : bs.spec_elems()) * es};
    const Prof piy{PK_Y_INV, b2 + b1, 0};
    const Prof pix{PK_X_INV, b1 + 2 * bv + (bs.mask ? box : 0), 0};

    // pass X: chi * x, zero-padded forward FFT of every row
    RowArgs<C> rx{};
    rx.in = x; rx.out = w1; rx.chi = chi_ptr<C>(bs); rx.st = st; rx.tw = T;
    rx.nrows = (int64_t)bs.nb * 3 * bs.bz * bs.by;
    rx.in_stride = bs.bx; rx.out_stride = bs.Mx; rx.n_in = bs.bx; rx.n_out = bs.Mx;
    rx.lL = bs.lx; rx.twshift = kLogLmax - bs.lx;
    rx.rows_per_box = 3 * bs.bz * bs.by; rx.plane = bs.bz * bs.by; rx.bx = bs.bx;
    VIE_TRY((launch_rows<C, ROW_FWD_CHI>(rx, px, s)));

    // pass Y forward
    ColArgs<C> cy{};
    cy.in = w1; cy.out = w2; cy.st = st; cy.tw = T;
    cy.ncols = bs.Mx; cy.n_in = bs.by; cy.n_out = bs.My; cy.lL = bs.ly; cy.twshift = kLogLmax - bs.ly;
    cy.in_axis = bs.Mx; cy.out_axis = bs.Mx;
    cy.in_s1 = (int64_t)bs.by * bs.Mx; cy.out_s1 = planeXY;
    cy.in_s2 = (int64_t)bs.bz * bs.by * bs.Mx; cy.out_s2 = (int64_t)bs.bz * planeXY;
    cy.b2_per_box = 3;
    VIE_TRY((launch_cols<C, true>(cy, bs.bz, bs.nb * 3, py, s)));

    // pass Z: forward, Green multiply, inverse
    ZArgs<C> z{};
    z.w = w2; z.G = G; z.Gb = Gb; z.st = st; z.tw = T;
    z.ncols = (int)planeXY; z.nzb = bs.bz; z.lL = bs.lz; z.twshift = kLogLmax - bs.lz;
    z.axis = planeXY; z.comp_stride = (int64_t)bs.bz * planeXY; z.box_stride = 3 * z.comp_stride;
    z.gcomp = bs.oct ? bs.oct_elems() : (int64_t)bs.Mz * planeXY;
    z.oct = bs.oct ? 1 : 0; z.lx = bs.lx; z.ly = bs.ly;
    z.nine = nine ? 1 : 0;
    if (nine && bs.oct) return fail(VIE_EINVAL, "mvm_boxes: nine spectra need the full layout");
    VIE_TRY(launch_zgreen<C>(z, bs.nb, pz, s));

    // pass Y inverse: keep y < by
    ColArgs<C> iy = cy;
    iy.in = w2; iy.out = w1; iy.n_in = bs.My; iy.n_out = bs.by;
    iy.in_s1 = planeXY; iy.out_s1 = (int64_t)bs.by * bs.Mx;
    iy.in_s2 = (int64_t)bs.bz * planeXY; iy.out_s2 = (int64_t)bs.bz * bs.by * bs.Mx;
    VIE_TRY((launch_cols<C, false>(iy, bs.bz, bs.nb * 3, piy, s)));

    // pass X inverse: keep x < bx, y = x - u
    RowArgs<C> ix = rx;
    ix.in = w1; ix.out = y; ix.xin = xupd ? xupd : x; ix.mask = bs.mask; ix.chi = nullptr;
    ix.in_stride = bs.Mx; ix.out_stride = bs.bx; ix.n_in = bs.Mx; ix.n_out = bs.bx;
    VIE_TRY((launch_rows<C, ROW_INV_UPDATE>(ix, pix, s)));
    return VIE_OK;
}

template <class C>
int spectrum_fft(const BoxSet& bs, C* G, cudaStream_t s, const Twiddles* twp, int ncomp) {
    Twiddles tw;
    if (twp) tw = *twp;
    else VIE_TRY(get_twiddles(&tw));
    const C* T = tw_ptr<C>(tw);
    const int64_t planeXY = (int64_t)bs.Mx * bs.My;
    const int64_t vol = planeXY * bs.Mz;
    const int64_t es = sizeof(C);

    RowArgs<C> rx{};
    rx.in = G; rx.out = G; rx.tw = T;
    rx.nrows = ncomp * (int64_t)bs.Mz * bs.My;
    rx.in_stride = bs.Mx; rx.out_stride = bs.Mx; rx.n_in = bs.Mx; rx.n_out = bs.Mx;
    rx.lL = bs.lx; rx.twshift = kLogLmax - bs.lx;
    rx.rows_per_box = (int)std::min<int64_t>(rx.nrows, 1 << 30); rx.plane = 1; rx.bx = bs.Mx;
    VIE_TRY((launch_rows<C, ROW_FWD_PLAIN>(rx, Prof{PK_SPECTRUM, 12 * vol * es, 0}, s)));

    ColArgs<C> cy{};
    cy.in = G; cy.out = G; cy.tw = T; cy.b2_per_box = 1;
    cy.ncols = bs.Mx; cy.n_in = bs.My; cy.n_out = bs.My; cy.lL = bs.ly; cy.twshift = kLogLmax - bs.ly;
    cy.in_axis = cy.out_axis = bs.Mx;
    cy.in_s1 = cy.out_s1 = planeXY;
    cy.in_s2 = cy.out_s2 = vol;
    VIE_TRY((launch_cols<C, true>(cy, bs.Mz, ncomp, Prof{PK_SPECTRUM, 2 * vol * es, 0}, s)));

    ColArgs<C> cz{};
    cz.in = G; cz.out = G; cz.tw = T; cz.b2_per_box = 1;
    cz.ncols = (int)planeXY; cz.n_in = bs.Mz; cz.n_out = bs.Mz; cz.lL = bs.lz; cz.twshift = kLogLmax - bs.lz;
    cz.in_axis = cz.out_axis = planeXY;
    cz.in_s1 = cz.out_s1 = 0;
    cz.in_s2 = cz.out_s2 = vol;
    VIE_TRY((launch_cols<C, true>(cz, 1, ncomp, Prof{PK_SPECTRUM, 2 * vol * es, 0}, s)));
    return VIE_OK;
}

// Octant compression (layout in vie_internal.cuh): slot (c, qz, qy, qx) takes the
// entry at the positions of the folded frequencies, converted to C.
template <class C>
__global__ void k_octant_compress(const double2* full, C* oct, int lx, int ly, int lz) {
    const int hx = (1 << lx) / 2 + 1, hy = (1 << ly) / 2 + 1, hz = (1 << lz) / 2 + 1;
    const int64_t per = (int64_t)hx * hy * hz;
    const int64_t vol = (int64_t)1 << (lx + ly + lz);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 6 * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int comp = (int)(t / per);
        int64_t r = t - comp * per;
        const int qx = (int)(r % hx);
        r /= hx;
        const int qy = (int)(r % hy), qz = (int)(r / hy);
        const int px = (int)brev_bits((unsigned)octant_freq(qx, lx), lx);
        const int py = (int)brev_bits((unsigned)octant_freq(qy, ly), ly);
        const int pz = (int)brev_bits((unsigned)octant_freq(qz, lz), lz);
        const double2 v = full[comp * vol + (((int64_t)pz << ly) + py) * ((int64_t)1 << lx) + px];
        oct[t] = cmk<C>(v.x, v.y);
    }
}

int spectrum_build(const BoxSet& bs, double k0, double h, double2* oct128, float2* oct64, float2* full64,
                   cudaStream_t s, const NearRule* near) {
    const int64_t n = 6 * bs.spec_elems();
    double2* G = nullptr;
    VIE_CK(cudaMallocAsync((void**)&G, n * sizeof(double2), s));
    int rc = green_sample(bs, k0, h, G, s, near);
    if (!rc) rc = spectrum_fft<double2>(bs, G, s);
    const int64_t no = 6 * bs.oct_elems();
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((no + 255) / 256, 152 * 16));
    if (!rc && oct128) {
        prof_begin(s, PK_SPECTRUM, VIE_C128, 0, no * 32, false);
        k_octant_compress<double2><<<grid, 256, 0, s>>>(G, oct128, bs.lx, bs.ly, bs.lz);
        prof_end(s);
        if (cudaGetLastError() != cudaSuccess) rc = fail(VIE_ECUDA, "octant compression launch failed");
    }
    if (!rc && oct64) {
        prof_begin(s, PK_SPECTRUM, VIE_C64, 0, no * 24, false);
        k_octant_compress<float2><<<grid, 256, 0, s>>>(G, oct64, bs.lx, bs.ly, bs.lz);
        prof_end(s);
        if (cudaGetLastError() != cudaSuccess) rc = fail(VIE_ECUDA, "octant compression launch failed");
    }
    if (!rc && full64) rc = convert_c128_to_c64(G, full64, n, s);
    cudaError_t e = cudaFreeAsync(G, s);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync", __FILE__, __LINE__);
    return rc;
}

template int mvm_boxes<double2>(const BoxSet&, const double2*, const double2*, double2*, const SegState*, cudaStream_t,
                                const Twiddles*, const double2* const*, const double2*, bool);
template int mvm_boxes<float2>(const BoxSet&, const float2*, const float2*, float2*, const SegState*, cudaStream_t,
                               const Twiddles*, const float2* const*, const float2*, bool);
template int spectrum_fft<double2>(const BoxSet&, double2*, cudaStream_t, const Twiddles*, int);

}  // namespace vie
