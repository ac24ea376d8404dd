// vie_matvec_noalloc: the FFT-accelerated MVM for small grids without any
// device allocation. For callers that must not allocate device memory at run
// time (a process whose device memory is owned by another framework's
// allocator, a real-time loop that cannot block on the driver's allocator, a
// deployment that forbids allocation after start-up), every intermediate of
// the MVM lives in one file-scope __device__ array instead of library-owned
// cudaMalloc workspace: the twiddle table, the six Green spectra and the two
// FFT scratch buffers.
#include <math.h>
#include <string.h>

#include <cmath>

#include <map>
#include <mutex>
#include <vector>

#include "vie_internal.cuh"

namespace vie {
namespace {

// Largest padded FFT volume Mx*My*Mz the static scratch holds (e.g. a 16^3 grid).
constexpr int64_t kNoAllocMaxVolume = 32 * 32 * 32;
constexpr size_t kTwBytes = kLmax * sizeof(double2);
// twiddles + 6 spectra + W2 (<= 3 * Mvol / 2 entries) + W1 (<= 3 * Mvol / 4 entries), complex128
constexpr size_t kNoAllocBytes = kTwBytes + (size_t)(6 * kNoAllocMaxVolume) * sizeof(double2) +
                                 (size_t)(3 * kNoAllocMaxVolume / 2) * sizeof(double2) +
                                 (size_t)(3 * kNoAllocMaxVolume / 4) * sizeof(double2);

// Held by every device that loads this library, for the life of the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
std::map<int, unsigned char*> g_addr;   // device address of the scratch, per device

// First call on a device (with that device current): resolve the array's
// device address and fill its twiddle table. No allocation is made.
int scratch_address(unsigned char** out) {
    int dev = 0;
    VIE_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_addr.find(dev);
    if (it != g_addr.end()) {
        *out = it->second;
        return VIE_OK;
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    double2 tw[kLmax];
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int m = 0; m < kLmax; ++m) {
        long double th = 2.0L * pi * (long double)m / (long double)kLmax;
        tw[m] = make_double2((double)cosl(th), (double)-sinl(th));
    }
    VIE_CK(cudaMemcpy(p, tw, kTwBytes, cudaMemcpyHostToDevice));
    // a copy from pageable memory may return before its DMA lands, and the caller's stream may be
    // a non-blocking one that does not wait for the legacy stream: wait for the table here
    VIE_CK(cudaDeviceSynchronize());
    g_addr[dev] = static_cast<unsigned char*>(p);
    *out = static_cast<unsigned char*>(p);
    return VIE_OK;
}

int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}
int lg(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace
}  // namespace vie

using namespace vie;

extern "C" int vie_matvec_noalloc(int32_t nx, int32_t ny, int32_t nz, double h, double k0, const double* chi_dev,
                                  const double* x_dev, double* y_dev, vie_stream_t stream) {
    if (!chi_dev || !x_dev || !y_dev) return fail(VIE_EINVAL, "vie_matvec_noalloc: null argument");
    if (nx < 1 || ny < 1 || nz < 1) return fail(VIE_EINVAL, "vie_matvec_noalloc: grid sizes must be >= 1");
    if (!(h > 0.0) || !(k0 > 0.0) || !std::isfinite(h) || !std::isfinite(k0))
        return fail(VIE_EINVAL, "vie_matvec_noalloc: h and k0 must be positive");
    BoxSet bs;
    bs.nb = 1;
    bs.bx = nx; bs.by = ny; bs.bz = nz;
    bs.Mx = pow2_at_least(2 * nx - 1);
    bs.My = pow2_at_least(2 * ny - 1);
    bs.Mz = pow2_at_least(2 * nz - 1);
    bs.lx = lg(bs.Mx); bs.ly = lg(bs.My); bs.lz = lg(bs.Mz);
    const int64_t vol = bs.spec_elems();
    if (vol > kNoAllocMaxVolume)
        return fail(VIE_EINVAL, "vie_matvec_noalloc: padded FFT volume " + std::to_string(vol) +
                                    " exceeds the static scratch limit of " + std::to_string(kNoAllocMaxVolume) +
                                    " points (e.g. a 16x16x16 grid); use vie_matvec");
    const int64_t need = (int64_t)kTwBytes +
                         (6 * vol + 3LL * bs.bz * bs.My * bs.Mx + 3LL * bs.bz * bs.by * bs.Mx) * (int64_t)sizeof(double2);
    if (need > (int64_t)kNoAllocBytes)
        return fail(VIE_EINVAL, "vie_matvec_noalloc: grid needs " + std::to_string(need) +
                                    " bytes of scratch, more than the static " + std::to_string(kNoAllocBytes) +
                                    "; use vie_matvec");
    const int64_t n3 = 3LL * nx * ny * nz;
    const char* xa = reinterpret_cast<const char*>(x_dev);
    const char* ya = reinterpret_cast<const char*>(y_dev);
    if (xa < ya + n3 * 16 && ya < xa + n3 * 16) return fail(VIE_EINVAL, "vie_matvec_noalloc: x and y overlap");
    const char* ca = reinterpret_cast<const char*>(chi_dev);
    const int64_t nchi = (int64_t)nx * ny * nz * 16;
    if (ca < ya + n3 * 16 && ya < ca + nchi) return fail(VIE_EINVAL, "vie_matvec_noalloc: chi and y overlap");

    unsigned char* base = nullptr;
    VIE_TRY(scratch_address(&base));
    Twiddles tw;
    tw.d128 = reinterpret_cast<double2*>(base);
    double2* G = reinterpret_cast<double2*>(base + kTwBytes);
    double2* w2 = G + 6 * vol;
    double2* w1 = w2 + 3LL * bs.bz * bs.My * bs.Mx;
    bs.w1 = w1;
    bs.w2 = w2;
    bs.chi128 = const_cast<double2*>(reinterpret_cast<const double2*>(chi_dev));
    cudaStream_t s = (cudaStream_t)stream;
    // every scratch entry a launch reads was written earlier in the same call: nothing needs clearing
    VIE_TRY(green_sample(bs, k0, h, G, s));
    VIE_TRY(spectrum_fft<double2>(bs, G, s, &tw));
    return mvm_boxes<double2>(bs, G, reinterpret_cast<const double2*>(x_dev), reinterpret_cast<double2*>(y_dev),
                              nullptr, s, &tw);
}
