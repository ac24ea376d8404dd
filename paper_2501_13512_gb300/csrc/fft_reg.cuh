// Register-resident FFTs shared by the full-grid z pass (fft.cu) and the
// persistent block solver (inner.cu). Each translation unit that includes
// this header has its own constant-memory twiddle table and calls
// reg_twiddles_ready() on the host before its first launch that uses them.
#pragma once

#include <algorithm>
#include <mutex>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

// Radix-2 FFT of one pencil held in registers, fully unrolled. FWD: natural
// order in, bit-reversed out (decimation in frequency); !FWD: bit-reversed in,
// natural out, unnormalised (decimation in time). Same ordering as the
// shared-memory passes, so spectra from either path are interchangeable.
template <bool FWD, class C>
__device__ __forceinline__ C twmul(C v, int m, const C* __restrict__ tw) {
    if (m == 0) return v;
    if (m == kLmax / 4) return FWD ? mul_mi(v) : mul_i(v);
    C w = __ldg(&tw[m]);
    return FWD ? cmul(v, w) : cmulc(v, w);
}

template <int L> struct ILog2 { static constexpr int v = 1 + ILog2<L / 2>::v; };
template <> struct ILog2<1> { static constexpr int v = 0; };

// Twiddle multiply used by the register FFTs (specialised below per precision).
template <class C> struct TwSel;

// One radix-2 stage of span S (a compile-time constant) on an L-point pencil.
template <int L, int S, bool FWD, class C>
__device__ __forceinline__ void rstage(C (&a)[L], const C* __restrict__ tw) {
#pragma unroll
    for (int g = 0; g < L; g += 2 * S) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int m = j * (kLmax / (2 * S));
            if (FWD) {
                C x0 = a[g + j], x1 = a[g + j + S];
                a[g + j] = x0 + x1;
                a[g + j + S] = TwSel<C>::template apply<true>(x0 - x1, m, tw);
            } else {
                C x0 = a[g + j], x1 = TwSel<C>::template apply<false>(a[g + j + S], m, tw);
                a[g + j] = x0 + x1;
                a[g + j + S] = x0 - x1;
            }
        }
    }
}

// Stages with spans S, S/2, ..., 1 (forward) or S, 2S, ..., L/2 (inverse).
template <int L, int S, bool FWD> struct RStages {
    template <class C> static __device__ __forceinline__ void run(C (&a)[L], const C* __restrict__ tw) {
        rstage<L, S, FWD>(a, tw);
        RStages<L, FWD ? S / 2 : S * 2, FWD>::run(a, tw);
    }
};
template <int L> struct RStages<L, 0, true> {
    template <class C> static __device__ __forceinline__ void run(C (&)[L], const C* __restrict__) {}
};
template <int L> struct RStages<L, L, false> {
    template <class C> static __device__ __forceinline__ void run(C (&)[L], const C* __restrict__) {}
};

template <int L, bool FWD, class C>
__device__ __forceinline__ void rfft(C (&a)[L], const C* __restrict__ tw) {
    if (L < 2) return;
    RStages<L, FWD ? L / 2 : 1, FWD>::run(a, tw);
}

typedef float2 F;

// Twiddles W_Lmax^m of the complex64 register path in constant memory: the
// register FFTs index them with compile-time offsets, so they become constant
// operands instead of loads. Copied once per device before the first launch.
static __constant__ F c_tw64[kLmax];

template <bool FWD>
__device__ __forceinline__ F twc(F v, int m) {
    if (m == 0) return v;
    if (m == kLmax / 4) return FWD ? mul_mi(v) : mul_i(v);
    F w = c_tw64[m];
    return FWD ? cmul(v, w) : cmulc(v, w);
}

template <> struct TwSel<double2> {
    template <bool FWD>
    static __device__ __forceinline__ double2 apply(double2 v, int m, const double2* __restrict__ tw) {
        return twmul<FWD>(v, m, tw);
    }
};
template <> struct TwSel<float2> {
    template <bool FWD>
    static __device__ __forceinline__ float2 apply(float2 v, int m, const float2* __restrict__) {
        return twc<FWD>(v, m);
    }
};

// Pruned transforms. A box of b voxels is padded to L >= 2b - 1, a power of
// two, so b <= L/2: forward inputs beyond L/2 are zero and inverse outputs
// beyond L/2 are discarded. The first DIF stage then splits the L-point
// transform into FFT_{L/2}(x) (positions [0, L/2)) and FFT_{L/2}(x_j W_L^j)
// (positions [L/2, L)); the last DIT stage of the inverse combines
// u = iFFT_{L/2}(lower half) and v = iFFT_{L/2}(upper half) as
// u_j + conj(W_L^j) v_j. Only L/2 values are live in registers at a time.

// Forward: get(j) gives input j < L/2 (zero where the box ends); put(k, v)
// receives output position k (bit-reversed order).
template <int L, class Get, class Put>
__device__ __forceinline__ void fwd_half(Get get, Put put, const F* __restrict__ tw) {
    if (L == 1) {
        put(0, get(0));
        return;
    }
    constexpr int H = L / 2 > 0 ? L / 2 : 1;
    F a[H];
#pragma unroll
    for (int j = 0; j < H; ++j) a[j] = twc<true>(get(j), j * (kLmax / L));
    rfft<H, true>(a, tw);
#pragma unroll
    for (int j = 0; j < H; ++j) put(H + j, a[j]);
#pragma unroll
    for (int j = 0; j < H; ++j) a[j] = get(j);
    rfft<H, true>(a, tw);
#pragma unroll
    for (int j = 0; j < H; ++j) put(j, a[j]);
}

// Inverse keeping outputs [0, L/2): get(k) gives input position k;
// stash(j, v) / unstash(j) hold conj(W_L^j) v_j between the two halves;
// put(j, v) receives output j (called for every j < L/2).
template <int L, class Get, class Stash, class Unstash, class Put>
__device__ __forceinline__ void inv_half(Get get, Stash stash, Unstash unstash, Put put, const F* __restrict__ tw) {
    if (L == 1) {
        put(0, get(0));
        return;
    }
    constexpr int H = L / 2 > 0 ? L / 2 : 1;
    F a[H];
#pragma unroll
    for (int j = 0; j < H; ++j) a[j] = get(H + j);
    rfft<H, false>(a, tw);
#pragma unroll
    for (int j = 0; j < H; ++j) stash(j, twc<false>(a[j], j * (kLmax / L)));
#pragma unroll
    for (int j = 0; j < H; ++j) a[j] = get(j);
    rfft<H, false>(a, tw);
#pragma unroll
    for (int j = 0; j < H; ++j) put(j, a[j] + unstash(j));
}

// Copies the complex64 twiddles into this translation unit's constant table, once per device.
static int reg_twiddles_ready(const Twiddles& tw) {
    static std::mutex mu;
    static std::vector<int> devs;
    int dev = 0;
    VIE_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(devs.begin(), devs.end(), dev) == devs.end()) {
        VIE_CK(cudaMemcpyToSymbol(c_tw64, tw.d64, kLmax * sizeof(float2), 0, cudaMemcpyDeviceToDevice));
        devs.push_back(dev);
    }
    return VIE_OK;
}

}  // namespace vie
