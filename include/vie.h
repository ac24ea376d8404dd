/*
 * vie.h -- C ABI of the GB300 VIE-FFT engine (libvie.so).
 *
 * The engine solves the volume integral equation of Section II.A (Eq. 4,
 * written in the total field E with chi = eps_r - 1):
 *
 *     (A E)_i = E_i - sum_j K(i - j) chi_j E_j = E_inc,i
 *
 * on a uniform Cartesian voxel grid, with K(D) = k0^2 G(D h) h^3 for D != 0
 * (G the dyadic Green's function of Eq. 1) and K(0) = s_self I (equivalent
 * sphere self term). Every product A x runs through the Toeplitz-to-circulant
 * FFT embedding (Section I), and the solver is BiCGSTAB right-preconditioned
 * with the block-diagonal matrix of Eq. 10, whose blocks are solved by inner
 * BiCGSTAB-FFT iterations to a loose tolerance (Section II.B).
 *
 * Conventions shared by every entry point
 *   - Status: every function returns VIE_OK (0) or one of the VIE_E* codes;
 *     vie_last_error() gives a text for the last failure on this thread.
 *   - Vectors: caller-owned DEVICE memory on the device that was current when
 *     the grid was created; complex interleaved (re, im); layout
 *     [3][nz][ny][nx] (component x, y, z; x fastest). VIE_C128 vectors are
 *     double pairs (16 B per entry), VIE_C64 vectors float pairs (8 B).
 *   - Streams: work is enqueued on the given cudaStream_t (NULL = legacy
 *     default stream). Functions that iterate (precond apply, solve) read
 *     convergence flags back to the host and therefore return only when the
 *     result is complete; vie_matvec, vie_plane_wave and vie_green_spectrum
 *     are asynchronous with respect to the host.
 *   - Handles (vie_grid, vie_spectrum) are opaque and owned by the library;
 *     the library allocates its own device workspace at grid creation.
 *   - Time convention exp(+j w t): a passive medium has Im(eps_r) <= 0.
 */
#ifndef VIE_H
#define VIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* vie_stream_t; /* identical to cudaStream_t */

enum vie_status {
    VIE_OK = 0,
    VIE_EINVAL = 1,      /* invalid argument (null pointer, bad size, aliasing)  */
    VIE_ENOMEM = 2,      /* device or host allocation failed                    */
    VIE_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed         */
    VIE_ENOTCONV = 4,    /* iteration limit reached; result and stats are valid */
    VIE_EBREAKDOWN = 5,  /* BiCGSTAB breakdown: rho, <rhat,v> or <t,t> is 0/NaN */
    VIE_ETIMEOUT = 6,    /* a bounded wait for the device gave up               */
    VIE_EBUSY = 7        /* admission refused: the allocation would exceed the
                            device budget of vie_set_device_budget              */
};

enum vie_precision {
    VIE_C128 = 1,        /* complex double: FP64 FFTs and arithmetic            */
    VIE_C64 = 2          /* complex float: FP32 FFTs, FP64 reductions/scalars   */
};

enum vie_solve_mode {
    VIE_MODE_PLAIN_C128 = 0, /* every MVM, inner solve and vector op in complex128 */
    VIE_MODE_MIXED = 1       /* FP64 true residuals + complex64 preconditioned
                                correction solves (iterative refinement)          */
};

typedef struct vie_grid vie_grid;
typedef struct vie_spectrum vie_spectrum;

/* Problem geometry (Section II.A: uniform hexahedral mesh; Eq. 10 blocks). */
typedef struct {
    int32_t nx, ny, nz;      /* voxels per axis, each in [1, 512]                    */
    double h;                /* voxel edge (same length unit as 2*pi/k0)             */
    const double* eps_r;     /* HOST or DEVICE, 2*nx*ny*nz doubles: relative
                                permittivity (re, im) per voxel, [nz][ny][nx];
                                copied (a device table is read back once)            */
    const int32_t* block_id; /* HOST or DEVICE, nx*ny*nz: subdomain of each voxel
                                for the block-diagonal preconditioner, -1 = no
                                block (identity); any non-negative ids; NULL = all
                                -1; copied                                           */
    uint32_t flags;          /* 0 or one VIE_GRID_INNER_* value                      */
    int32_t block_expand;    /* E in [0, 64]: each block is solved on its voxels plus
                                every voxel with chi != 0 within Chebyshev distance E,
                                and only its own voxels are kept (expanded blocks,
                                restricted additive Schwarz; 0 = the blocks of
                                Eq. 10 as given)                                     */
} vie_grid_desc;

/* How the inner block solves of the preconditioner run (vie_grid_desc.flags).
 * AUTO: a persistent kernel in which each CTA solves whole blocks on its own,
 * for every group whose padded (x, y) plane fits in shared memory, when those
 * groups hold at least 32 blocks together; batched multi-CTA launches per
 * BiCGSTAB step otherwise. The two
 * paths compute the same iterations; the flags force one of them. */
enum vie_grid_flags {
    VIE_GRID_INNER_AUTO = 0,
    VIE_GRID_INNER_BATCHED = 1,
    VIE_GRID_INNER_PERSISTENT = 2
};

typedef struct {
    int32_t nblocks;         /* non-empty blocks found in block_id                 */
    int32_t ngroups;         /* batches of blocks sharing one padded FFT shape     */
    int32_t Mx, My, Mz;      /* padded FFT shape of the full-grid operator         */
    int64_t device_bytes;    /* device memory held by the grid handle              */
    int32_t inner_cluster[2];/* CTAs per block chosen by the block solver's tuner for
                                complex128 [0] and complex64 [1]: 1, 2 or 4 for
                                every block, -1 for the split launch of the
                                register MVM (the slowest blocks on 4 CTAs and the
                                rest on 2); 0 = not yet tuned                      */
} vie_grid_info;

/* Creates the grid on the current CUDA device: uploads chi = eps_r - 1,
 * partitions the blocks (Eq. 10) into groups that share a padded FFT shape,
 * and allocates all workspace. Errors: VIE_EINVAL (sizes, flags, nulls,
 * non-finite eps_r), VIE_EBUSY (the workspace would exceed the device budget;
 * nothing is kept), VIE_ENOMEM, VIE_ECUDA. */
int vie_grid_create(const vie_grid_desc* desc, vie_grid** out);

/* Waits for the grid's device, then frees the grid and its workspace. Every
 * spectrum of the grid must have been released first. Errors: VIE_EINVAL. */
int vie_grid_destroy(vie_grid* grid);

/* Block count, group count, padded FFT shape and device bytes of a grid. */
int vie_grid_get_info(const vie_grid* grid, vie_grid_info* info);

/* Green-tensor spectra (Eq. 1, sampled at lattice offsets, self term at 0):
 * computes in FP64 on the device the 3D FFT of the six components of K for
 * the full grid and for every block group, at wavenumber k0 > 0.
 * precision_mask: VIE_C128, VIE_C64 or both (bitwise or); the complex64 copy
 * is rounded from the FP64 spectrum. Storage: the full-grid spectrum keeps
 * (Mx/2+1)(My/2+1)(Mz/2+1) entries per component (each component is even or
 * odd along every axis, so one octant of frequencies fixes it), block-group
 * spectra the full Mx My Mz. The spectrum is owned by the caller and
 * serves the grid it was made for and every other grid with the same h, padded
 * shapes and block-group box extents (e.g. the same structure created twice);
 * it must be released before the grid it was made for is destroyed.
 * Asynchronous on `stream`.
 * Errors: VIE_EINVAL, VIE_ENOMEM, VIE_ECUDA. */
int vie_green_spectrum(vie_grid* grid, double k0, int precision_mask,
                       vie_stream_t stream, vie_spectrum** out);

/* As vie_green_spectrum, with cube-integrated near-neighbour entries: for lattice
 * offsets D with 0 < max(|Dx|, |Dy|, |Dz|) <= near_radius, K(D) is the mean of
 * k0^2 G over the source voxel (the cube of side h centred at D h) times h^3,
 * by a tensor Gauss-Legendre rule of near_order points per axis, instead of
 * k0^2 G(D h) h^3 at the voxel centre. The paper does not say how it integrates
 * near couplings (Section II.A); this is an accuracy variant of the same
 * Toeplitz operator, used by every MVM and block solve with this spectrum.
 * near_radius 0 gives vie_green_spectrum. Errors: VIE_EINVAL (near_radius
 * outside [0, 8], near_order outside [1, 16] when near_radius > 0), as
 * vie_green_spectrum otherwise. */
int vie_green_spectrum_near(vie_grid* grid, double k0, int precision_mask, int32_t near_radius,
                            int32_t near_order, vie_stream_t stream, vie_spectrum** out);

/* Waits for the device, then frees the spectra. Errors: VIE_EINVAL. */
int vie_spectrum_release(vie_spectrum* spectrum);

/* Incident plane wave E_inc = pol * exp(-j k0 khat . r) at voxel centres
 * r = (i + 1/2) h - (grid centre). khat: 3 doubles (unit propagation
 * direction); pol: 6 doubles, complex polarisation (re, im) per component.
 * Writes one vector of `precision` to einc_dev. Asynchronous. */
int vie_plane_wave(const vie_grid* grid, double k0, const double* khat,
                   const double* pol, int precision, void* einc_dev,
                   vie_stream_t stream);

/* y = A x = x - G(chi x) (Eq. 4; FFT-accelerated MVM of Section I) with the
 * spectrum's k0, in `precision` (the spectrum must hold it). x and y must not
 * overlap (VIE_EINVAL). Asynchronous. */
int vie_matvec(vie_grid* grid, const vie_spectrum* spectrum, int precision,
               const void* x_dev, void* y_dev, vie_stream_t stream);

typedef struct {
    int32_t nblocks;         /* blocks solved                                       */
    int32_t max_iters;       /* largest inner BiCGSTAB iteration count              */
    double mean_iters;       /* mean inner iteration count (half-steps as 0.5)      */
    int32_t not_converged;   /* blocks that hit inner_maxit (not an error)          */
    int32_t breakdowns;      /* blocks whose inner BiCGSTAB broke down              */
} vie_precond_stats;

/* y = K2^{-1} b with K2 = diag(A_1, ..., A_N) (Eq. 10): for each block k the
 * system A_k x_k = b|S_k (rows/columns of A on the block's voxels, all three
 * components, Eq. 11) is solved by BiCGSTAB-FFT from x_k = 0 to
 * ||b_k - A_k x_k|| <= inner_tol ||b_k|| or inner_maxit iterations; y = b on
 * voxels of no block. The blocks of the groups the persistent solver takes
 * (vie_grid_flags) run in one persistent launch, each block solved to its own
 * tolerance by one thread-block cluster; the other groups iterate in lockstep
 * in batched launches, one per BiCGSTAB step. b and y are vectors of
 * `precision` and must not overlap. stats may be NULL. Synchronous with the
 * host at return. */
int vie_block_precond_apply(vie_grid* grid, const vie_spectrum* spectrum,
                            int precision, const void* b_dev, void* y_dev,
                            double inner_tol, int inner_maxit,
                            vie_stream_t stream, vie_precond_stats* stats);

typedef struct {
    double outer_tol;        /* stop when ||E_inc - A E|| <= outer_tol ||E_inc||   */
    double inner_tol;        /* block solves' relative tolerance (Section II.B)     */
    int32_t outer_maxit;     /* outer BiCGSTAB iterations (per refinement in MIXED) */
    int32_t inner_maxit;     /* cap on inner BiCGSTAB iterations per block apply;
                                a cap the blocks never reach (e.g. 1000) keeps K2
                                a converged block inverse (metal blocks need ~350) */
    int32_t use_precond;     /* 0: unpreconditioned BiCGSTAB                        */
    int32_t mode;            /* vie_solve_mode                                      */
    int32_t max_refinements; /* MIXED: FP64 residual corrections, 0 = default (8)   */
    double wait_timeout_ms;  /* bound on each host wait for the device, 0 = 60000   */
    const void* x0_dev;      /* initial guess E_0 (DEVICE complex128, the layout of
                                E), or NULL for E_0 = 0; may be e_dev itself (warm
                                start in place); must be NULL for vie_batch_solve  */
} vie_solve_opts;

typedef struct {
    double outer_iters;      /* outer BiCGSTAB iterations (half-steps as 0.5),
                                summed over refinements in MIXED                    */
    int64_t inner_iters;     /* inner BiCGSTAB iterations summed over all blocks    */
    int32_t precond_applies; /* K2^{-1} applications                                */
    int32_t matvecs_c128;    /* full-grid MVMs in complex128                        */
    int32_t matvecs_c64;     /* full-grid MVMs in complex64                         */
    int32_t refinements;     /* MIXED: FP64 residual evaluations after the first    */
    double true_rel_res;     /* ||E_inc - A E|| / ||E_inc||, FP64, at exit          */
    int32_t status;          /* same value as returned                              */
    int32_t rejected;        /* MIXED: corrections undone because they did not
                                lower the FP64 residual (vie_solve; batch: 0/1)    */
    double elapsed_ms;       /* host wall time of the call (batch: of the whole
                                batch, the same in every entry)                    */
} vie_solve_stats;

/* Solves A E = E_inc (Eq. 4) by right-preconditioned BiCGSTAB (Section II.B).
 * VIE_MODE_PLAIN_C128: one BiCGSTAB in complex128 throughout.
 * VIE_MODE_MIXED: FP64 residual r = E_inc - A E (complex128 MVM), then a
 *   complex64 preconditioned BiCGSTAB for A d = r with FP64 reductions and
 *   scalars, E += d, repeated until the FP64 residual meets outer_tol.
 *   A correction that does not lower the FP64 residual is undone; the next
 *   one is then solved without the preconditioner, and if that one fails too
 *   the solve stops with VIE_ENOTCONV and the best E so far.
 * einc_dev, e_dev: complex128 vectors (caller-owned, distinct). The spectrum
 * must hold VIE_C128, and VIE_C64 too for MIXED. Returns VIE_OK,
 * VIE_ENOTCONV (E and stats still valid), VIE_EBREAKDOWN, VIE_ETIMEOUT,
 * VIE_EINVAL, VIE_ECUDA. stats may be NULL. */
int vie_solve(vie_grid* grid, const vie_spectrum* spectrum, const void* einc_dev,
              void* e_dev, const vie_solve_opts* opts, vie_stream_t stream,
              vie_solve_stats* stats);

/* vie_solve from HOST buffers: einc_host (read) and e_host (written), complex128
 * [3][nz][ny][nx] in host memory (pinned memory lets the copies run at full
 * speed; pageable memory works too), distinct. E_inc is copied to a device
 * vector of the grid, solved there as by vie_solve (opts->x0_dev, if set, is a
 * DEVICE vector), and E copied back on `stream`; returns after E has landed in
 * e_host (also for VIE_ENOTCONV, whose E is valid). The grid keeps the two
 * device vectors (2 x 48 N bytes, allocated on the first call, counted in
 * device_bytes and the device budget). Errors as vie_solve. */
int vie_solve_host(vie_grid* grid, const vie_spectrum* spectrum, const void* einc_host,
                   void* e_host, const vie_solve_opts* opts, vie_stream_t stream,
                   vie_solve_stats* stats);

/* ---- Solves of many requests with merged block-solver launches. ----
 * Serving runs the solves of several requests at once, each on its own grid
 * (any shapes, modes and tolerances), host thread and stream. Inside a merge
 * session, every block-preconditioner application (Eq. 10) of a solve first
 * gathers its blocks and then waits (on the host) until every other solve of
 * the session that still applies a preconditioner has reached its next
 * application; their blocks then run in ONE persistent launch (one per
 * precision, inner tolerance and inner limit), the longest-running blocks
 * first. Merged are the blocks that the persistent block solver takes for
 * their grid alone (VIE_GRID_AUTO: grids with 32 or more fitting blocks) and
 * the complex64 blocks of its on-chip slab MVM (every padded axis in [8, 32]);
 * the other blocks run in their grid's batched launches meanwhile. A solve joins at its first application
 * and leaves when it stops applying the preconditioner, so requests that arrive
 * while others run share launches from then on (continuous batching). Each
 * solve runs exactly the iteration of vie_solve; its result equals the
 * vie_solve result up to rounding (the merged launches use clusters of 2 CTAs
 * per block, while vie_solve tunes the cluster size per grid). */
typedef struct vie_merge_session vie_merge_session;

typedef struct {
    int32_t launches;        /* merged persistent block-solver launches queued     */
    int32_t max_solves;      /* most solves whose blocks shared one launch         */
    double mean_solves;      /* solves per launch, averaged over the launches      */
} vie_merge_stats;

/* Creates a session on the current device (it owns a stream and the work
 * lists of the merged launches). Errors: VIE_EINVAL, VIE_ECUDA. */
int vie_merge_session_create(vie_merge_session** out);

/* Frees the session after its queued launches. VIE_EBUSY while a
 * vie_solve_merged call is running in it (nothing is freed then). */
int vie_merge_session_destroy(vie_merge_session* session);

/* The session's merged launches so far. */
int vie_merge_session_stats(vie_merge_session* session, vie_merge_stats* out);

/* vie_solve inside a session: same arguments, results and errors as vie_solve
 * (blocking; call it from one host thread per solve, with its own stream and
 * its own grid). A grid must not be in two running solves at once. */
int vie_solve_merged(vie_merge_session* session, vie_grid* grid, const vie_spectrum* spectrum,
                     const void* einc_dev, void* e_dev, const vie_solve_opts* opts,
                     vie_stream_t stream, vie_solve_stats* stats);

/* n solves at once in a session of their own (all members from the first
 * application on), one internal host thread and stream each; returns when all
 * have finished, their work ordered after the work queued on `stream` before
 * the call and before work queued on it after. grids[n]: distinct grids;
 * spectra[n], einc_dev[n], e_dev[n], opts[n]: as for vie_solve, per solve.
 * stats[n] (may be NULL): per solve, status = that solve's return code.
 * merge (may be NULL): the session's merged launches. n = 1 is vie_solve.
 * Returns VIE_OK when every solve returned VIE_OK, else the code of the first
 * solve (by index) that did not, with its message; VIE_EINVAL for n < 1, a
 * null array or a grid listed twice (nothing runs then). */
int vie_solve_many(int32_t n, vie_grid* const* grids, const vie_spectrum* const* spectra,
                   const void* const* einc_dev, void* const* e_dev, const vie_solve_opts* opts,
                   vie_stream_t stream, vie_solve_stats* stats, vie_merge_stats* merge);

/* ---- Batched independent solves (many instances of one grid shape). ---- */
typedef struct vie_batch vie_batch;

typedef struct {
    int32_t nx, ny, nz;      /* grid of every instance, each in [1, 512]               */
    double h;                /* voxel edge                                             */
    int32_t count;           /* instances, in [1, 21845]                               */
    const double* eps_r;     /* HOST, count * 2 * nx*ny*nz doubles: eps_r (re, im) of
                                instance i at [i][nz][ny][nx]; copied                  */
    uint32_t flags;          /* reserved, must be 0                                    */
} vie_batch_desc;

/* Creates `count` independent instances of the unpreconditioned system of Eq. 4
 * (each its own permittivity) sharing one grid shape, with all workspace.
 * Errors: VIE_EINVAL, VIE_ENOMEM, VIE_ECUDA. */
int vie_batch_create(const vie_batch_desc* desc, vie_batch** out);

/* Waits for the device, then frees the batch and its cached spectra. */
int vie_batch_destroy(vie_batch* batch);

/* Solves A_i E_i = E_inc,i for every instance i at wavenumber k0s[i] (HOST,
 * count doubles; spectra are computed in FP64 per distinct value and cached in
 * the batch). Mixed precision only (opts->mode = VIE_MODE_MIXED): FP64 true
 * residuals of all instances from one batched complex128 MVM, then one
 * complex64 correction solve for every instance still above outer_tol, all in
 * one persistent launch (one CTA cluster per instance) when the padded plane
 * fits in shared memory, else batched launches per BiCGSTAB step; E += d.
 * outer_maxit bounds each correction; inner_tol, inner_maxit and use_precond
 * are ignored (no blocks). An instance whose correction does not lower its
 * FP64 residual gets that correction undone and stops (VIE_ENOTCONV). einc_dev, e_dev: DEVICE complex128
 * [count][3][nz][ny][nx], distinct. stats: NULL or count entries
 * (outer_iters = correction iterations summed over refinements).
 * Returns VIE_OK when every instance meets outer_tol, VIE_ENOTCONV otherwise
 * (all outputs valid), VIE_EINVAL, VIE_ENOMEM, VIE_ECUDA, VIE_ETIMEOUT. */
int vie_batch_solve(vie_batch* batch, const double* k0s, const void* einc_dev,
                    void* e_dev, const vie_solve_opts* opts, vie_stream_t stream,
                    vie_solve_stats* stats);

/* n batches of different grid shapes at once, in a merge session of their own
 * (see vie_solve_merged): one internal host thread and stream per batch; at
 * every refinement step the persistent correction launches of all batches that
 * reached it run as ONE launch (one CTA cluster per instance, instances of all
 * sizes in one work queue, largest boxes first). Batches whose corrections use
 * batched launches (planes too large for shared memory) run beside it. Each
 * batch's result equals its vie_batch_solve result up to rounding.
 * batches[n]: distinct; k0s[n], einc_dev[n], e_dev[n], opts[n], stats[n] (stats
 * may be NULL, or stats[i] NULL): as for vie_batch_solve, per batch. merge (may
 * be NULL): the merged launches. Ordered after the work queued on `stream`
 * before the call and before work queued on it after. Returns VIE_OK when every
 * batch returned VIE_OK, else the code of the first batch (by index) that did
 * not, with its message; VIE_EINVAL for n < 1, a null array or a batch listed
 * twice (nothing runs then). */
int vie_batch_solve_many(int32_t n, vie_batch* const* batches, const double* const* k0s,
                         const void* const* einc_dev, void* const* e_dev, const vie_solve_opts* opts,
                         vie_stream_t stream, vie_solve_stats* const* stats, vie_merge_stats* merge);

/* ---- The paper's rooftop / pulse discretisation (Section II.A, Eqs. 5-9). ----
 * Unknown w = J / (j w eps0) (units of E; w = chi E in the continuum), expanded in rooftops (Eq. 5):
 * component a lives on the face between cell c and cell c + e_a, stored at index c of a vector
 * [3][nz][ny][nx]; a face carries a rooftop when both of its cells are inside the grid and non-air
 * (the normal current vanishes on the object's surface; other entries are 0). Tested with pulses on
 * the dual cells (Eq. 6) the equation reads
 *   (1/chi) Gram w - k0^2 int g w - grad int g div w = E_inc,
 * the contrast and vector-potential parts of L^c (Eq. 8) and the scalar potential of L^q (Eq. 9,
 * read as acting on w_j), with the sign of Eq. 4: the Gram of rooftops and pulses gives 3/8 per half
 * cell (times 1/chi of that cell) on the face and 1/8 to its two neighbours along a; cell charges are
 * the divergence of the rooftops; potentials use the integral of g over each cell (h^3 g at the cell
 * centre, the equivalent sphere at the source cell). The operator is Toeplitz in the face indices
 * and runs through the same FFT passes as vie_matvec, with nine spectra. */
typedef struct vie_rooftop vie_rooftop;

/* Builds the rooftop operator of the grid's permittivity at wavenumber k0 (spectra in FP64, also
 * rounded to complex64 with VIE_C64 in precision_mask), with its workspace. The operator uses the
 * grid's FFT scratch: calls on it and on the grid must be ordered on one stream. Release it before
 * the grid. Errors: VIE_EINVAL, VIE_EBUSY, VIE_ENOMEM, VIE_ECUDA. */
int vie_rooftop_create(vie_grid* grid, double k0, int precision_mask, vie_stream_t stream, vie_rooftop** out);

/* Waits for the device, then frees the operator. */
int vie_rooftop_release(vie_rooftop* op);

/* E_inc = pol exp(-j k0 khat . r) at the face centres of every component (0 on faces without a
 * rooftop), into a vector of `precision`. Asynchronous. */
int vie_rooftop_incident(const vie_rooftop* op, const double* khat, const double* pol, int precision,
                         void* out_dev, vie_stream_t stream);

/* y = A w, DEVICE vectors of `precision` ([3][nz][ny][nx]), not overlapping; entries of faces without
 * a rooftop are ignored in w and 0 in y. Asynchronous. Errors: VIE_EINVAL. */
int vie_rooftop_matvec(vie_rooftop* op, int precision, const void* w_dev, void* y_dev, vie_stream_t stream);

/* Solves A w = b (complex128, DEVICE, distinct) by unpreconditioned BiCGSTAB from w = 0 to
 * ||b - A w|| <= tol ||b|| (recursive residual, reported in stats->true_rel_res) or maxit
 * iterations; stats may be NULL (outer_iters, matvecs_c128, status, elapsed_ms are set). Returns
 * VIE_OK, VIE_ENOTCONV, VIE_EBREAKDOWN, VIE_ETIMEOUT (bounded host waits, 0 = 60000 ms), VIE_EINVAL. */
int vie_rooftop_solve(vie_rooftop* op, const void* b_dev, void* w_dev, double tol, int32_t maxit,
                      double wait_timeout_ms, vie_stream_t stream, vie_solve_stats* stats);

/* Bistatic RCS of a rooftop solution w (complex128, DEVICE): as vie_far_field_rcs with
 * P(u) = sum over faces of w h^3 exp(j k0 u . r_face). HOST directions and results; synchronises. */
int vie_rooftop_far_field_rcs(const vie_rooftop* op, const void* w_dev, int32_t ndir, const double* dirs_host,
                              double* rcs_host, vie_stream_t stream);

/* Bistatic radar cross section of a solved field (the far-zone limit of the
 * scattered field of Eq. 1 with J = j w eps0 chi E; Section III's RCS
 * comparisons, Figs. 1-2): for each direction u,
 *   P(u) = sum_j chi_j E_j h^3 exp(j k0 u . r_j),
 *   rcs[i] = k0^4 / (4 pi) |(I - u u) P(u)|^2,
 * with voxel centres r_j = ((i + 1/2) h - n h / 2) per axis (the grid's centre
 * at the origin) and chi = eps_r - 1 of the grid. e_dev: DEVICE complex128
 * [3][nz][ny][nx] (e.g. the output of vie_solve). dirs_host: HOST ndir x 3 unit
 * vectors (|u| = 1 within 1e-9, else VIE_EINVAL). rcs_host: HOST ndir doubles,
 * written before return (the call synchronises `stream`). FP64 throughout.
 * Returns VIE_OK, VIE_EINVAL, VIE_ENOMEM, VIE_ECUDA. No paper counterpart for
 * the interface; the quantity is the paper's validation metric. */
int vie_far_field_rcs(const vie_grid* grid, double k0, const void* e_dev,
                      int32_t ndir, const double* dirs_host, double* rcs_host,
                      vie_stream_t stream);

/* Device bytes held by the batch (with its cached spectra), and whether its
 * corrections run in the persistent kernel (1) or in batched launches (0). */
int vie_batch_get_info(const vie_batch* batch, int64_t* device_bytes, int32_t* persistent);

/* Kernel-level profile, aggregated per kernel kind and precision. */
typedef struct {
    char name[32];           /* x_fwd, y_fwd, z_green, y_inv, x_inv, bicg_update,
                                bicg_dot, spectrum, field, inner_block             */
    int32_t precision;       /* VIE_C128 or VIE_C64                                 */
    int64_t launches;        /* launches recorded                                   */
    double total_ms;         /* sum of CUDA-event durations, each measured on the
                                launching stream                                    */
    double bytes;            /* algorithmic bytes: inputs read + outputs written by
                                the work units (boxes, segments) each launch
                                actually processed                                  */
} vie_kernel_stat;

/* enable = 1 clears the profile and starts recording every launch of this
 * library in this process (CUDA events around each launch); 0 stops. The
 * recording itself adds two event records per launch. Errors: VIE_ECUDA. */
int vie_profile_enable(int enable);

/* Waits for the recorded work, then writes up to cap aggregated entries to
 * out (n_out receives the count) and the number of kernel launches the
 * library made since the process started to total_launches (counted whether
 * or not profiling is enabled). Any pointer may be NULL. Errors: VIE_ECUDA,
 * VIE_ENOMEM (more launches than the profile holds: 1,048,576). */
int vie_profile_read(vie_kernel_stat* out, int cap, int* n_out, int64_t* total_launches);

/* y = A x (as vie_matvec, complex128) for small grids WITHOUT ANY DEVICE
 * ALLOCATION. The paper has no counterpart: this entry point exists for
 * callers that must not allocate device memory at run time, such as code in a
 * process whose device memory is owned by another framework's allocator, a
 * real-time loop that cannot block on the driver's allocator, or a deployment
 * that forbids allocation after start-up. It needs no grid or spectrum
 * handle: it computes the Green spectrum (FP64) and the MVM with all
 * intermediates in one static device array of 4,341,760 bytes (about 4.1 MB)
 * that every device using the library holds until the process exits.
 *   nx, ny, nz: grid; the padded FFT volume nextpow2(2nx-1) * nextpow2(2ny-1)
 *       * nextpow2(2nz-1) must be at most 32768 (a 16x16x16 grid fits), else
 *       VIE_EINVAL with the limit in the message;
 *   h, k0: voxel edge and wavenumber (> 0);
 *   chi_dev: DEVICE, complex128 (re, im) chi = eps_r - 1, [nz][ny][nx];
 *   x_dev, y_dev: DEVICE, complex128 [3][nz][ny][nx]; y must overlap
 *       neither x nor chi (VIE_EINVAL).
 * The first call on a device, with that device current, resolves the array's
 * device address, writes its twiddle table (a synchronous host-to-device
 * copy) and waits for the device (cudaDeviceSynchronize), so that a caller's
 * non-blocking stream never reads the table early; make that first call
 * before any stream capture. Later calls only
 * enqueue kernels on `stream`. All calls share the one array and overwrite
 * it: calls that overlap on the GPU (different streams, or different host
 * threads without ordering) race and give wrong results. Nothing in the array
 * needs to start at zero. Errors: VIE_EINVAL, VIE_ECUDA. */
int vie_matvec_noalloc(int32_t nx, int32_t ny, int32_t nz, double h, double k0,
                       const double* chi_dev, const double* x_dev, double* y_dev,
                       vie_stream_t stream);

/* Device memory budget for admission by footprint (a serving process that
 * hosts several grids): every device allocation the library keeps for a grid,
 * a spectrum or a batch is counted, process-wide, and a call whose allocation
 * would take the count above `bytes` is refused with VIE_EBUSY and keeps
 * nothing. 0 (the default) removes the budget. Transient temporaries inside a
 * call (the FP64 spectrum source, far-field partial sums) are not counted.
 * Lowering the budget below the bytes held refuses later allocations only.
 * No paper counterpart. Errors: VIE_EINVAL (bytes < 0). */
int vie_set_device_budget(int64_t bytes);

/* Bytes the library's handles hold on the device now, and the budget (0 = none).
 * Either pointer may be NULL. */
int vie_device_usage(int64_t* held, int64_t* budget);

/* Test hook for the out-of-memory paths: the counted allocation after the next
 * `after` ones fails as if cudaMalloc had reported cudaErrorMemoryAllocation
 * (VIE_ENOMEM), without calling it; -1 cancels. One failure per call of this
 * function. No paper counterpart. */
int vie_fault_inject_alloc(int32_t after);

/* Copies the text of the last error on this thread into buf (NUL-terminated,
 * truncated to len). Returns the length of the full message. */
int vie_last_error(char* buf, size_t len);

/* Library version, e.g. 100 for 0.1.0. */
int vie_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VIE_H */
