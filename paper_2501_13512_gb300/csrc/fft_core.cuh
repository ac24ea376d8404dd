// Shared-memory FFT building blocks used by the pencil passes (fft.cu) and the
// persistent block solver (inner.cu).
#pragma once

#include "vie_internal.cuh"

namespace vie {

// ---------------------------------------------------------------- butterflies
// Forward radix-4 DIF butterfly on (x0, x1, x2, x3) = positions (a, a+s, a+2s, a+3s)
// of a group of 4s, with w_k = W_{4s}^{k j}; equals two radix-2 DIF stages.
template <class C>
__device__ __forceinline__ void bfly4_dif(C& x0, C& x1, C& x2, C& x3, C w1, C w2, C w3) {
    C a0 = x0 + x2, a1 = x1 + x3, d0 = x0 - x2, d1 = mul_mi(x1 - x3);
    x0 = a0 + a1;
    x1 = cmul(a0 - a1, w2);
    x2 = cmul(d0 + d1, w1);
    x3 = cmul(d0 - d1, w3);
}

// Inverse of bfly4_dif up to a factor 4 (conjugate twiddles, DIT order).
template <class C>
__device__ __forceinline__ void bfly4_dit(C& x0, C& x1, C& x2, C& x3, C w1, C w2, C w3) {
    C p = x0, q = cmulc(x1, w2), u = cmulc(x2, w1), v = cmulc(x3, w3);
    C pq = p + q, pmq = p - q, uv = u + v, iumv = mul_i(u - v);
    x0 = pq + uv;
    x2 = pq - uv;
    x1 = pmq + iumv;
    x3 = pmq - iumv;
}

// In-place FFT of NCOMP * (1 << ltc) columns of length L = 1 << lL held in
// shared memory: element (i, comp, c) at buf[i * pitch + comp * (1 << ltc) + c].
// FWD: natural -> bit-reversed (DIF). !FWD: bit-reversed -> natural (DIT),
// unnormalised (L times the inverse DFT). Ends with __syncthreads().
template <class C, bool FWD, int NCOMP>
__device__ void smem_fft(C* buf, int lL, int pitch, int ltc, const C* __restrict__ tw, int twshift) {
    const int tcm = (1 << ltc) - 1;
    const int nq = ((1 << lL) >> 2) * NCOMP << ltc;   // radix-4 butterflies per stage
    const int nr4 = lL >> 1;
    const bool odd = lL & 1;
    auto radix2 = [&]() {
        const int n2 = ((1 << lL) >> 1) * NCOMP << ltc;
        for (int idx = threadIdx.x; idx < n2; idx += blockDim.x) {
            int c = idx & tcm, t = idx >> ltc;
            int comp = t % NCOMP, q = t / NCOMP;
            C* p0 = buf + (2 * q) * pitch + (comp << ltc) + c;
            C x0 = p0[0], x1 = p0[pitch];
            p0[0] = x0 + x1;
            p0[pitch] = x0 - x1;
        }
        __syncthreads();
    };
    if (!FWD && odd) radix2();
    for (int st = 0; st < nr4; ++st) {
        const int ls = FWD ? (lL - 2 - 2 * st) : ((odd ? 1 : 0) + 2 * st);   // log2 of span s
        const int sm = (1 << ls) - 1;
        const int sp = pitch << ls;
        for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
            int c = idx & tcm, t = idx >> ltc;
            int comp = t % NCOMP, q = t / NCOMP;
            int j = q & sm, g = q >> ls;
            int a0 = (g << (ls + 2)) + j;
            int e = j << (lL - ls - 2);                  // j * L / (4 s)
            C w1 = tw[e << twshift], w2 = tw[(2 * e) << twshift], w3 = tw[(3 * e) << twshift];
            C* p0 = buf + a0 * pitch + (comp << ltc) + c;
            C x0 = p0[0], x1 = p0[sp], x2 = p0[2 * sp], x3 = p0[3 * sp];
            if (FWD) bfly4_dif(x0, x1, x2, x3, w1, w2, w3);
            else bfly4_dit(x0, x1, x2, x3, w1, w2, w3);
            p0[0] = x0;
            p0[sp] = x1;
            p0[2 * sp] = x2;
            p0[3 * sp] = x3;
        }
        __syncthreads();
    }
    if (FWD && odd) radix2();
}

// Generalised in-place shared-memory FFT of length L = 1 << lL over
// (1 << lc) lines in each of (1 << lp) planes: element i of line c of plane q
// sits at buf[i * es + c * cs + q * ps]. Same butterflies and orderings as
// smem_fft; used for the row and column transforms of 2D planes.
template <class C, bool FWD>
__device__ void smem_fft_g(C* buf, int lL, int es, int lc, int cs, int lp, int ps, const C* __restrict__ tw,
                           int twshift) {
    const int cm = (1 << lc) - 1, pm = (1 << lp) - 1;
    const int nq = ((1 << lL) >> 2) << (lc + lp);
    const int nr4 = lL >> 1;
    const bool odd = lL & 1;
    auto radix2 = [&]() {
        const int n2 = ((1 << lL) >> 1) << (lc + lp);
        for (int idx = threadIdx.x; idx < n2; idx += blockDim.x) {
            int c = idx & cm, t = idx >> lc;
            int q = t & pm, k = t >> lp;
            C* p0 = buf + (2 * k) * es + c * cs + q * ps;
            C x0 = p0[0], x1 = p0[es];
            p0[0] = x0 + x1;
            p0[es] = x0 - x1;
        }
        __syncthreads();
    };
    if (!FWD && odd) radix2();
    for (int st = 0; st < nr4; ++st) {
        const int ls = FWD ? (lL - 2 - 2 * st) : ((odd ? 1 : 0) + 2 * st);
        const int sm = (1 << ls) - 1;
        const int sp = es << ls;
        for (int idx = threadIdx.x; idx < nq; idx += blockDim.x) {
            int c = idx & cm, t = idx >> lc;
            int q = t & pm, k = t >> lp;
            int j = k & sm, gi = k >> ls;
            int a0 = (gi << (ls + 2)) + j;
            int e = j << (lL - ls - 2);
            C w1 = tw[e << twshift], w2 = tw[(2 * e) << twshift], w3 = tw[(3 * e) << twshift];
            C* p0 = buf + a0 * es + c * cs + q * ps;
            C x0 = p0[0], x1 = p0[sp], x2 = p0[2 * sp], x3 = p0[3 * sp];
            if (FWD) bfly4_dif(x0, x1, x2, x3, w1, w2, w3);
            else bfly4_dit(x0, x1, x2, x3, w1, w2, w3);
            p0[0] = x0;
            p0[sp] = x1;
            p0[2 * sp] = x2;
            p0[3 * sp] = x3;
        }
        __syncthreads();
    }
    if (FWD && odd) radix2();
}

}  // namespace vie
