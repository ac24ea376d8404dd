// Internal declarations of libvie: complex helpers, handle layouts, launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <condition_variable>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/vie.h"

namespace vie {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
std::string last_error_message();   // this thread's last error message
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define VIE_CK(call)                                                        \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return ::vie::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define VIE_TRY(call)                                                       \
    do {                                                                    \
        int rc_ = (call);                                                   \
        if (rc_ != VIE_OK) return rc_;                                      \
    } while (0)

// ---------------------------------------------------------------- complex
template <class C> struct real_of;
template <> struct real_of<double2> { typedef double type; };
template <> struct real_of<float2> { typedef float type; };

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
template <class C> __host__ __device__ __forceinline__ C cmk(double a, double b);
template <> __host__ __device__ __forceinline__ double2 cmk<double2>(double a, double b) { return make_double2(a, b); }
template <> __host__ __device__ __forceinline__ float2 cmk<float2>(double a, double b) { return make_float2((float)a, (float)b); }

#define VIE_CPLX_OPS(C)                                                                   \
    __host__ __device__ __forceinline__ C operator+(C a, C b) { return mk(a.x + b.x, a.y + b.y); } \
    __host__ __device__ __forceinline__ C operator-(C a, C b) { return mk(a.x - b.x, a.y - b.y); } \
    __host__ __device__ __forceinline__ C cmul(C a, C b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); } \
    __host__ __device__ __forceinline__ C cmulc(C a, C b) { /* a * conj(b) */ return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); } \
    __host__ __device__ __forceinline__ C mul_i(C a) { return mk(-a.y, a.x); }          \
    __host__ __device__ __forceinline__ C mul_mi(C a) { return mk(a.y, -a.x); }

VIE_CPLX_OPS(double2)
VIE_CPLX_OPS(float2)
#undef VIE_CPLX_OPS

template <class C> __host__ __device__ __forceinline__ C czero() { return cmk<C>(0.0, 0.0); }

__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__device__ __forceinline__ double2 to_c128(float2 a) { return make_double2(a.x, a.y); }
template <class C> __device__ __forceinline__ C from_c128(double2 a);
template <> __device__ __forceinline__ double2 from_c128<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_c128<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ---------------------------------------------------------------- FFT plan pieces
constexpr int kLmax = 1024;   // largest padded FFT length per axis
constexpr int kLogLmax = 10;

struct Twiddles {              // W_Lmax^m = exp(-2 pi i m / Lmax), m in [0, Lmax)
    double2* d128 = nullptr;
    float2* d64 = nullptr;
};
int get_twiddles(Twiddles* out);   // per device, created on first use

// Counted device allocations of the library's handles (grids, spectra, batches).
// dmalloc refuses with VIE_EBUSY, allocating nothing, when the bytes held would
// exceed the budget set by vie_set_device_budget (0 = none); a failing
// cudaMalloc gives VIE_ENOMEM. dfree returns the bytes of a pointer dmalloc gave.
int dmalloc(void** p, size_t bytes, const char* what);
void dfree(void* p);

// A batch of equal-shaped boxes sharing one padded FFT shape. The full-grid
// operator is the batch with nb = 1 and the box equal to the grid.
struct BoxSet {
    int nb = 0;
    int bx = 0, by = 0, bz = 0;        // box dimensions (voxels)
    int Mx = 0, My = 0, Mz = 0;        // padded FFT lengths (powers of two >= 2b - 1)
    int lx = 0, ly = 0, lz = 0;        // log2 of the padded lengths
    double2* chi128 = nullptr;         // [nb][bz][by][bx], chi masked to each block
    float2* chi64 = nullptr;
    uint8_t* mask = nullptr;           // [nb][bz][by][bx] block membership, or null (full grid)
    int32_t* origin = nullptr;         // [nb][3] grid coordinates of each box corner
    void* w1 = nullptr;                // [nb][3][bz][by][Mx] (sized for complex128)
    void* w2 = nullptr;                // [nb][3][bz][My][Mx]
    std::vector<int> block_ids;        // compact block index of each box
    bool oct = false;                  // the MVM reads octant-compressed spectra (octant_slot)

    int64_t box_elems() const { return (int64_t)bx * by * bz; }
    int64_t vec_elems() const { return 3 * box_elems(); }             // per box
    int64_t spec_elems() const { return (int64_t)Mx * My * Mz; }      // per component, full
    int64_t oct_elems() const {                                       // per component, octant
        return (int64_t)(Mx / 2 + 1) * (My / 2 + 1) * (Mz / 2 + 1);
    }
};

// Octant compression of a Green spectrum. Each component of the padded kernel
// is even or odd under m -> M - m along each axis (xx, yy, zz even; xy odd in
// x and y; xz odd in x and z; yz odd in y and z), so its DFT has the same
// parity and is fixed by the frequencies f in [0, M/2] of every axis. Along an
// axis of length M = 2^l, the spectrum entry at bit-reversed position p has
// frequency k = brev_l(p); it is stored at slot q of the folded frequency
// f = min(k, M - k), with q = brev_{l-1}(f) for f < M/2 and q = M/2 for
// f = M/2 (the two positions 2j, 2j+1 of a warp then read runs of contiguous
// slots), and `upper` (k > M/2) flips the sign of components odd along the axis.
__host__ __device__ __forceinline__ unsigned bit_reverse(unsigned v, int l) {
    unsigned r = 0;
    for (int i = 0; i < l; ++i) r |= ((v >> i) & 1u) << (l - 1 - i);
    return r;
}
#ifdef __CUDA_ARCH__
__device__ __forceinline__ unsigned brev_bits(unsigned v, int l) { return l ? __brev(v) >> (32 - l) : 0u; }
#else
inline unsigned brev_bits(unsigned v, int l) { return bit_reverse(v, l); }
#endif
__host__ __device__ __forceinline__ int octant_slot(int p, int l, bool& upper) {
    const int M = 1 << l, H = M >> 1;
    const int k = (int)brev_bits((unsigned)p, l);
    upper = k > H;
    const int f = upper ? M - k : k;
    if (f == H) return H;
    return l >= 2 ? (int)brev_bits((unsigned)f, l - 1) : 0;
}
// frequency f of slot q (inverse of octant_slot on [0, M/2])
__host__ __device__ __forceinline__ int octant_freq(int q, int l) {
    const int H = (1 << l) >> 1;
    if (q == H) return H;
    return l >= 2 ? (int)brev_bits((unsigned)q, l - 1) : 0;
}

// Per-segment BiCGSTAB state (FP64 scalars on the device).
enum SegStatus : int {
    SEG_ACTIVE = 0,
    SEG_CONVERGED = 1,
    SEG_HALF_PENDING = 2,  // converged at the half step, x += alpha y not applied yet
    SEG_MAXIT = 3,
    SEG_BREAKDOWN = 4,
    SEG_IDLE = 5           // not part of this solve
};

struct SegState {
    double2 rho, rho_prev, alpha, omega;
    double bnorm2, res2, tol2;
    double iters;          // half-steps counted as 0.5
    int status;
    int maxit;
};

// Batched Krylov workspace for one BoxSet (inner solves) or the full grid.
template <class C> struct KrylovVecs {
    C *b = nullptr, *x = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr,
      *v = nullptr, *s = nullptr, *t = nullptr, *y = nullptr, *z = nullptr;
};

struct ReduceScratch {
    double2* part = nullptr;     // [nseg][kMaxCtaPerSeg][2]
    unsigned* count = nullptr;   // [nseg]
    int* n_active = nullptr;     // [1]
    int nseg = 0;
};
constexpr int kMaxCtaPerSeg = 256;

struct Group {
    bool persistent128 = false;        // solved by the persistent block solver
    bool persistent64 = false;
    bool fit[2] = {false, false};      // may join a merged persistent launch (0: complex128, 1: complex64)
    std::vector<float> last_iters[2];  // inner iterations of each block in its last application
    BoxSet bs;
    KrylovVecs<double2> k128;
    KrylovVecs<float2> k64;
    SegState* st = nullptr;            // [nb]
    ReduceScratch red;
};

}  // namespace vie

struct vie_spectrum {
    vie_grid* grid = nullptr;             // the grid it was made for (identity only, never dereferenced)
    // what the spectrum depends on: h and (box extents, padded shape) of the
    // full grid and of every block group; any grid matching it may use it
    double h = 0.0;
    std::vector<int> shape_sig;
    double k0 = 0.0;
    int precision_mask = 0;
    // index 0: full grid; 1 + g: group g. Layout [6][Mz][My][Mx] (bit-reversed
    // frequency positions per axis), scaled by 1/(Mx My Mz).
    std::vector<double2*> g128;
    std::vector<float2*> g64;
    // index 1 + g: complex64 octant spectrum of group g in natural order for the slab MVM, or null
    std::vector<float2*> go64;
};

struct vie_grid {
    int device = 0;
    int nx = 0, ny = 0, nz = 0;
    double h = 0.0;
    int64_t N = 0;
    vie::BoxSet full;
    int32_t* block_id = nullptr;          // device [N], compact ids, -1 = none
    int nblocks = 0;
    std::vector<vie::Group> groups;
    int32_t* blk_group = nullptr;         // device [nblocks]
    int32_t* blk_index = nullptr;         // device [nblocks]
    int32_t* blk_origin = nullptr;        // device [nblocks][3]
    // outer Krylov vectors (full grid)
    vie::KrylovVecs<double2> o128;
    vie::KrylovVecs<float2> o64;
    double2* tmp128 = nullptr;            // full-grid scratch vector
    double2* x0buf = nullptr;             // plain solves warm-started in place (allocated on first use)
    double2* host_io[2] = {nullptr, nullptr};   // vie_solve_host: E_inc and E on the device (first use)
    float2* tmp64 = nullptr;
    vie::SegState* ost = nullptr;         // outer state [1]
    vie::ReduceScratch ored;
    double* dscal = nullptr;              // device scalars: [0] ||b||^2, [1] ||r||^2
    char* h_ring = nullptr;               // pinned host: active counts, state, scalar
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // persistent block solver: work lists (job, box), largest boxes first
    int2* work128 = nullptr;
    int2* work64 = nullptr;
    int nwork128 = 0, nwork64 = 0;
    // host copies of the work lists and the group of each job, per precision (0: c128, 1: c64);
    // after every apply the list is re-sorted by the blocks' measured cost (longest first)
    std::vector<int2> work_host[2];
    std::vector<int> job_group[2];
    void* inner_groups = nullptr;         // device copy of the per-group descriptors
    int* inner_next = nullptr;            // work counters [2] (second: the split launch's light part)
    cudaStream_t s2 = nullptr;            // stream of the light part of a split block-solver launch
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // cluster-size autotuning of the persistent solver, per precision (0: c128, 1: c64):
    // applies 0 and 1 try the candidates, later applies use the best
    int tune_count[2] = {0, 0};
    int tune_best[2] = {0, 0};
    int tune_npl[2] = {0, 0};             // slab MVM: kz planes per round of the best candidate (0: auto)
    bool tune_noslab[2] = {false, false}; // the best candidate ran the register-FFT MVM instead of the slab MVM
    double tune_score[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
    int nheavy[2] = {0, 0};               // blocks of the split launch's heavy part (from the last apply)
    cudaEvent_t tev[2] = {nullptr, nullptr};
    int64_t device_bytes = 0;
    std::vector<void*> allocations;
};

namespace vie {

// ---------------------------------------------------------------- launch profiling (profile.cu)
// Every kernel launch of the library goes through prof_begin / prof_end. When
// profiling is off only a launch counter is incremented. When on, CUDA events
// bracket the launch on its stream, and the kernel receives a device counter
// to which it adds the number of work units (boxes or segments) it actually
// processed, so the algorithmic bytes of launches that skip converged blocks
// are counted exactly: bytes = units * bytes_per_unit + (units ? fixed : 0).
enum ProfKind {
    PK_X_FWD = 0, PK_Y_FWD, PK_Z_GREEN, PK_Y_INV, PK_X_INV,
    PK_BICG_UPDATE, PK_BICG_DOT, PK_SPECTRUM, PK_FIELD, PK_INNER, PK_COUNT
};
int* prof_begin(cudaStream_t s, int kind, int precision, int64_t bytes_per_unit, int64_t bytes_fixed,
                bool device_units);
void prof_end(cudaStream_t s);

// ---------------------------------------------------------------- launchers (fft.cu)
// tw: twiddle tables to use; null = the per-device tables of get_twiddles()
// Gb: optional device array of one spectrum pointer per box (null: G for every box)
template <class C>
int mvm_boxes(const BoxSet& bs, const C* G, const C* x, C* y, const SegState* st,
              cudaStream_t s, const Twiddles* tw = nullptr, const C* const* Gb = nullptr,
              const C* xupd = nullptr, bool nine = false);
// xupd: the vector of the last pass's update y = xupd - u (default x); nine: G holds nine full
// spectra G_ab (a, b = x, y, z; index 3a + b) and the z pass multiplies by the general 3x3 matrix.
template <class C>
int spectrum_fft(const BoxSet& bs, C* G, cudaStream_t s, const Twiddles* tw = nullptr,
                 int ncomp = 6);   // in place, ncomp components
// Green spectrum of one box shape at wavenumber k0 (FP64 samples and FFT in a
// stream-ordered temporary), written to any of: oct128 / oct64 (octant
// layout [6][Mz/2+1][My/2+1][Mx/2+1]), full64 (full layout [6][Mz][My][Mx]).
// Cube-integrated near-neighbour entries (an accuracy variant; the paper does not say how
// near couplings are integrated): K(D) = mean over the cube of side h centred at D h of
// k0^2 G, times h^3, for 0 < max|D| <= radius, by tensor Gauss-Legendre quadrature of order q.
constexpr int kNearMaxOrder = 16;
struct NearRule {
    int radius = 0;                       // 0: point sampling everywhere
    int q = 0;
    double t[kNearMaxOrder], w[kNearMaxOrder];   // nodes and weights on [-1, 1]
};
int near_rule(int radius, int q, NearRule* out);   // VIE_EINVAL outside radius [0, 8], q [1, 16]
int spectrum_build(const BoxSet& bs, double k0, double h, double2* oct128, float2* oct64, float2* full64,
                   cudaStream_t s, const NearRule* near = nullptr);

// ---------------------------------------------------------------- green.cu
int green_sample(const BoxSet& bs, double k0, double h, double2* G, cudaStream_t s, const NearRule* near = nullptr);
int convert_c128_to_c64(const double2* a, float2* b, int64_t n, cudaStream_t s);
// Bistatic RCS of sum_j wts_j E_j h^3 exp(j k0 u . r_j) over voxel centres r_j, component c shifted by
// shift[c] along its own axis (shift may be null). Synchronises s.
int far_field_rcs_impl(int nx, int ny, int nz, double h, double k0, const double2* e_dev, const double2* wts,
                       const double* shift, int32_t ndir, const double* dirs_host, double* rcs_host, cudaStream_t s);
int plane_wave_launch(const vie_grid* g, double k0, const double* khat, const double* pol,
                      int precision, void* out, cudaStream_t s);

// ---------------------------------------------------------------- krylov.cu
template <class C>
struct Bicg {
    int nseg;
    int64_t seglen;
    KrylovVecs<C> v;
    SegState* st;
    ReduceScratch* red;
};
template <class C> int bicg_init(Bicg<C>& k, double tol, int maxit, cudaStream_t s);
template <class C> int bicg_init_tols(Bicg<C>& k, const double* tols, int maxit, cudaStream_t s);
template <class C> int bicg_rho(Bicg<C>& k, cudaStream_t s);
template <class C> int bicg_update_p(Bicg<C>& k, cudaStream_t s);
template <class C> int bicg_sigma(Bicg<C>& k, cudaStream_t s);
template <class C> int bicg_update_s(Bicg<C>& k, cudaStream_t s);
template <class C> int bicg_x_half(Bicg<C>& k, cudaStream_t s);
template <class C> int bicg_omega(Bicg<C>& k, cudaStream_t s);
template <class C> int bicg_update_xr(Bicg<C>& k, cudaStream_t s);
int reduce_count_active(const SegState* st, int nseg, int* n_active, cudaStream_t s);

// vector helpers (krylov.cu)
template <class C> int vec_copy(const C* a, C* b, int64_t n, cudaStream_t s);
int vec_residual128(const double2* b, const double2* ax, double2* r, int64_t n, cudaStream_t s);
int vec_norm2_128(const double2* a, int64_t n, ReduceScratch* red, double* d_out, cudaStream_t s);
int vec_sum128(const double2* a, const double2* b, double2* out, int64_t n, cudaStream_t s);   // out = a + b
int vec_scale_to_c64(const double2* a, const double* d_norm2, float2* b, int64_t n, cudaStream_t s);
int vec_add_scaled_c64(double2* x, const float2* d, const double* d_norm2, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------- inner.cu (persistent block solver)
constexpr int kInnerMinBlocks = 32;     // fewer blocks than this: batched multi-CTA path instead
template <class C> struct InnerJob {
    const BoxSet* bs;
    KrylovVecs<C> v;
    const C* chi;
    const C* G;
    SegState* st;
    const C* const* Gb = nullptr;   // optional device array: one spectrum per box
    const double* tols = nullptr;   // optional device array: one relative tolerance per box
    const C* Go = nullptr;          // optional octant spectrum in natural order (slab MVM, complex64)
};
bool inner_persistent_ok(const BoxSet& bs, size_t es, bool force);
bool slab_path_ok(const BoxSet& bs, size_t es);
// Octant spectrum of the slab MVM from a full FP64 spectrum [6][Mz][My][Mx] (bit-reversed positions):
// Go[kz][c][ky][kx] = G[c][brev(kz)][brev(ky)][brev(kx)] for k in [0, M/2] per axis, as complex64.
int slab_spectrum(const BoxSet& bs, const double2* G, float2* Go, cudaStream_t s);
size_t inner_group_desc_bytes();
// cluster: CTAs per block (1, 2, 4, 8; 0 = 2), unless VIE_INNER_CLUSTER forces one. npl: kz planes
// per round of the slab MVM's plane stage (2 or 4; 0: 4 where it fits), unless VIE_SLAB_NPL forces one.
// Split launch (split != null, 0 < split->nheavy < nwork): the first nheavy work items run
// with split->cluster CTAs per block on s while the rest run with `cluster` CTAs per block on
// split->s2, concurrently; d_next must hold two counters; s waits for both.
struct InnerSplit {
    int nheavy = 0;
    int cluster = 4;
    cudaStream_t s2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
template <class C>
int inner_persistent(const std::vector<InnerJob<C>>& jobs, const int2* d_work, int nwork, void* d_groups,
                     int* d_next, double tol, int maxit, cudaStream_t s, int cluster = 0,
                     const InnerSplit* split = nullptr, int npl = 0);
int inner_cluster_forced();

// ---------------------------------------------------------------- merge sessions (api.cu)
// Solves (or batched solves) that run at the same time, one host thread and one stream each,
// inside one session. A member's persistent block-solver launch is replaced by a request: the
// member queues its gathers, records `ready` on its stream and arrives; once every live member of
// the session has arrived, the last to arrive queues ONE persistent launch over the jobs of all
// requests (one per precision, tolerance and iteration limit) on the session's stream, and each
// member's stream waits for it (merge_wait) before using the results. Each block's work is the
// same as in a launch of its own.
struct MergeReq {
    int prec = 0;                                   // 0: complex128, 1: complex64
    double tol = 0.0;
    int maxit = 0;
    std::vector<InnerJob<double2>> j128;            // the member's jobs (prec 0)
    std::vector<InnerJob<float2>> j64;              // (prec 1)
    std::vector<std::pair<double, int2>> items;     // (cost, (job within the member's jobs, box))
    cudaEvent_t ready = nullptr;
    int64_t gen = -1;                               // launch that took it (-1: none yet, -2: failed)
};
struct MergeLaunch {
    cudaEvent_t done = nullptr;
    int waiting = 0;                                // members that have not yet waited for it
};
}  // namespace vie

struct vie_merge_session {
    std::mutex m;
    std::condition_variable cv;
    int device = 0;
    int live = 0;                  // members that may still arrive
    int inside = 0;                // vie_solve_merged calls running in the session
    std::vector<vie::MergeReq*> pending;
    cudaStream_t ms = nullptr;     // every merged launch, in order
    std::map<int64_t, vie::MergeLaunch> launches_open;
    std::vector<cudaEvent_t> free_events;
    int64_t next_gen = 0;
    char* d_groups = nullptr;      // group descriptors of a launch
    int2* d_work = nullptr;        // (job, box) work list of a launch
    int* d_next = nullptr;
    int64_t groups_cap = 0, work_cap = 0;
    std::vector<void*> retired;    // outgrown buffers (a queued launch may still read them)
    int launches = 0;
    int64_t members = 0;
    int max_members = 0;
    std::string err;
};

namespace vie {
using MergeCtx = vie_merge_session;
// One member's membership: it leaves (once) when it stops launching block solves.
struct MergeMember {
    MergeCtx* ctx = nullptr;
    bool live = false;
};
void merge_join(MergeMember* mm);
void merge_arrive(MergeMember* mm, MergeReq* r);
int merge_wait(MergeMember* mm, MergeReq* r, cudaStream_t s);
void merge_leave(MergeMember* mm);
// True when the environment variable VIE_INNER_SLAB is 0: complex64 blocks keep the register-FFT MVM
// instead of the slab MVM (read once).
bool slab_disabled();
template <class C> inline const C* tw_of(const Twiddles& t);
template <> inline const double2* tw_of<double2>(const Twiddles& t) { return t.d128; }
template <> inline const float2* tw_of<float2>(const Twiddles& t) { return t.d64; }

// ---------------------------------------------------------------- precond.cu
template <class C>
int precond_gather(const vie_grid* g, const Group& gr, const C* b, C* out, cudaStream_t s);
template <class C>
int precond_scatter_group(const vie_grid* g, const Group& gr, const C* xk, C* y, cudaStream_t s);
template <class C>
int precond_copy_unblocked(const vie_grid* g, const C* b, C* y, cudaStream_t s);

}  // namespace vie
