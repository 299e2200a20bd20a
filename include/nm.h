/*
 * nm.h -- C ABI of libnestconv: gravitational potential on nested Cartesian
 * meshes by the convolution method (Vorobyov, McKevitt, Kulikov & Elbakyan
 * 2023, "Computing the gravitational potential on nested meshes using the
 * convolution method").
 *
 * What is computed
 * ----------------
 * A nested mesh has L levels m = 0 (coarsest) .. L-1 (finest), each of N^3
 * cubic cells, all centred on the origin.  Level m has cell size
 * dx_m = dx0 / 2^m (Sect. 2, Fig. 1: each level halves the physical size) and
 * level m+1 covers level-m cells [N/4, 3N/4) on every axis.
 *
 * For each level the cell masses M = rho dx_m^3 are convolved with the inverse
 * distance between cell centres, Phi_i = -G sum_j M_j calG(x_i - x_j)
 * (Eq. 10), the self-cell term being the exact integral of 1/r over the cell,
 * calG(0) = C / dx_m with C = 3 ln(2 + sqrt 3) - pi/2 (Eq. 13).  The sum is
 * evaluated with the convolution theorem on the domain doubled to (2N)^3 and
 * zero padded (Sect. 3, Eq. 11, Fig. 4), so it is the isolated sum exactly up
 * to rounding.
 *
 * Levels are combined as in Sect. 4 (Fig. 5, Eq. 14):
 *     Phi(Omega^n) = Phi^n + sum_{k<n} interp_{k->n}(Phi^k_hole)
 * where Phi^k_hole is level k's potential with the covered cells' mass
 * removed.  By default (NM_INTERP_DIAGONAL) the coarser holes reach level n
 * through the two-point rule of Eqs. 3-6 applied one level at a time:
 *     carry_n = D(carry_{n-1} + Phi^{n-1}_hole),  carry_1 = D(Phi^0_hole),
 *     Phi(Omega^n) = Phi^n + carry_n,
 * with D(f) at a fine centre = 3/4 f(nearest coarse centre) + 1/4 f(its
 * diagonal neighbour towards the fine centre).  NM_INTERP_TRILINEAR instead
 * interpolates each Phi^k_hole trilinearly from level-k centres straight to
 * level-n centres (see nm_options.interp).  With NM_METHOD_DIPOLE_PAIR the pairwise dipole
 * method of Sect. 7 and Appendix B (Eqs. 15, B.1-B.2) is used instead for
 * every level but the finest:
 *     Phi(Omega^n) = Phi^n_hole + reduce(Phi^{n+1}_dbl) + sum_{k<n} interp(Phi^k_hole)
 * with Phi^{n+1}_dbl the potential of level n+1's mass on a (2N)^3 grid of
 * level-(n+1) cells spanning level n, reduced to level n by the mean of the
 * 2^3 fine values in each coarse cell.
 *
 * Covered coarse cells take the mean of their 2^3 finer children (swept from
 * the finest level up), so the caller's values in those cells are ignored.
 *
 * Data layout
 * -----------
 * rho : L * N^3 densities, contiguous [level][z][y][x] (x fastest), level 0
 *       coarsest.  double for NM_FP64 plans, float for NM_FP32 plans.
 * phi : L * N^3 doubles, same layout; every cell of every level is written,
 *       covered cells included.  Device phi must be 16-byte aligned.
 * Pointers passed to nm_potential are DEVICE pointers (current device),
 * owned by the caller; nm_potential_host takes HOST pointers.
 *
 * Streams and errors
 * ------------------
 * `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 * stream.  Calls that take a stream are asynchronous with respect to the host
 * unless stated otherwise.  Argument errors are reported synchronously
 * (NM_EINVAL / NM_EUNSUPPORTED) and nothing is launched.  A CUDA error seen
 * at launch is returned as NM_ECUDA; errors of kernels still running surface
 * at the caller's next synchronisation.  nm_last_error() returns a message for
 * the calling thread's last failure.  Nothing here aborts the process.
 *
 * A plan owns its device workspace; calls that use the same plan must be
 * ordered (same stream, or synchronised) because they share that workspace.
 * Green spectra are cached per (device, N) and shared by all plans.
 */
#ifndef NESTCONV_NM_H
#define NESTCONV_NM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nm_plan_s* nm_plan_t;

typedef enum {
    NM_OK = 0,
    NM_EINVAL = 1,        /* bad argument (null pointer, bad size, bad option)   */
    NM_ENOMEM = 2,        /* device or host allocation failed                   */
    NM_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed        */
    NM_ETIMEOUT = 4,      /* a bounded device-side wait gave up                 */
    NM_EUNSUPPORTED = 5   /* valid request this build does not implement       */
} nm_status;

enum { NM_FP64 = 0, NM_FP32 = 1, NM_FP64X = 2 };
enum { NM_METHOD_ORIGINAL = 0, NM_METHOD_DIPOLE_PAIR = 1, NM_METHOD_DIPOLE_TRIPLE = 2, NM_METHOD_DIPOLE_TRIPLE_DIRECT = 3 };
enum { NM_INTERP_TRILINEAR = 0, NM_INTERP_DIAGONAL = 1 };
enum { NM_MAX_LEVELS = 16 };

typedef struct {
    int levels;      /* L, 1 .. NM_MAX_LEVELS                                   */
    int N;           /* cells per axis per level: a power of two, 4 .. 256      */
    double dx0;      /* coarsest cell size (> 0); level m has dx0 / 2^m         */
    double G;        /* gravitational constant (Eq. 9); nm_plan uses 1.0        */
    int precision;   /* NM_FP64: all arithmetic in double.  NM_FP64X: densities
                        and potentials in double, the transforms, spectrum
                        multiply and cross-level sums in double-float (two
                        floats, ~48 bits) on the FP32 pipe -- within 1e-12 of
                        the double result, several times faster on parts whose
                        FP64 rate is a small fraction of FP32 (original method,
                        N >= 8; NM_EUNSUPPORTED otherwise).  NM_FP32: FFT passes,
                        spectrum multiply, interpolation and the sum of the
                        coarser levels' terms in float; Green spectrum built in
                        double; the final per-cell addition of that sum to the
                        level's own potential in double.                        */
    int method;      /* NM_METHOD_ORIGINAL (Eq. 14), NM_METHOD_DIPOLE_PAIR
                        (Eqs. 15, B.1-B.2), NM_METHOD_DIPOLE_TRIPLE (Eqs. B.3-B.5:
                        below level L-2 the next level's ring on its doubled
                        grid and the level after on its quadrupled grid, 4N
                        cells, transforms of 8N points, so N <= 128) or
                        NM_METHOD_DIPOLE_TRIPLE_DIRECT (the same with the
                        quadrupled grid replaced by the direct sum of
                        Eq. B.6, O(N^6) per level)                              */
    int interp;      /* How the hole potentials reach the finer levels (the
                        stencil of Fig. 6):
                        NM_INTERP_TRILINEAR: tensor-product linear from each
                          level k straight to every finer level n;
                        NM_INTERP_DIAGONAL (default): the two-point rule of Eqs. 3-6
                          (3/4 of the nearest coarse value plus 1/4 of its
                          diagonal neighbour towards the fine centre), carried
                          one level at a time: carry_n = D(carry_{n-1} +
                          Phi^{n-1}_hole), carry_1 = D(Phi^0_hole).  Costs
                          L-2 extra small launches and (L-2)(N/2+2)^3 values
                          of workspace.                                          */
} nm_options;

/* Fill `opt` with the defaults used by nm_plan: G = 1, NM_FP64, original
 * method, NM_INTERP_DIAGONAL (the Eqs. 3-6 rule, the reading that reproduces
 * the paper's acceleration errors).  No device work. */
nm_status nm_default_options(int levels, int N, double dx0, nm_options* opt);

/* Create a plan for one nested mesh on the current CUDA device: validates the
 * geometry (Sect. 2), allocates the plan's device workspace and the kernel
 * schedule.  The Green spectrum is not built yet (see nm_green).
 * `out` receives an opaque handle owned by the caller; free with nm_destroy.
 * Errors: NM_EINVAL (bad sizes, null out), NM_EUNSUPPORTED (N outside the
 * built range), NM_ENOMEM, NM_ECUDA. */
nm_status nm_plan(int levels, int N, double dx0, nm_plan_t* out);
nm_status nm_plan_ex(const nm_options* opt, nm_plan_t* out);

/* Build (or take from the cache) the transform of the unit-cell kernel of
 * Eq. 10 with the Eq. 13 self term on the doubled domain of Fig. 4, in double
 * precision, on `stream`.  The spectrum is real and even, so only its octant
 * (N+1)^3 is kept.  Idempotent; nm_potential calls it when needed. */
nm_status nm_green(nm_plan_t plan, void* stream);

/* The potential of every cell of every level (see the header comment) from
 * densities `rho` (device, L*N^3, double or float by precision) into `phi`
 * (device, L*N^3 double).  Asynchronous on `stream`.  `rho` is read only.
 * A repeated call with the same (plan, rho, phi) replays a CUDA graph of the
 * solve captured on the first repeat (as nm_batch_potential does); inside a
 * caller's own stream capture the kernels are simply recorded. */
nm_status nm_potential(nm_plan_t plan, const void* rho, double* phi, void* stream);

/* Gravitational acceleration g = -grad Phi of a nested potential `phi`
 * (device, L*N^3 doubles, as written by nm_potential for this plan's mesh)
 * into `g` (device, L*3*N^3 doubles, [level][component x,y,z][z][y][x]),
 * asynchronously on `stream`.  Central six-point differences (Eq. 8) on every
 * level; at the boundary of a finer level the missing neighbour is the ghost
 * value interpolated from the coarser level by Eqs. 3-6 (method A of
 * Appendix A); an uncovered coarse cell next to the finer level takes the mean
 * of the 2^3 finer children for its covered neighbour (method B); the outer
 * boundary of the coarsest level uses second-order one-sided differences.
 * In double precision for both plan precisions.  phi and g must be 16-byte
 * aligned (NM_EINVAL otherwise). */
nm_status nm_acceleration(nm_plan_t plan, const double* phi, double* g, void* stream);

/* The coarse-side rule of the acceleration at a level interface (Appendix A):
 * NM_ACCEL_COARSE_MEAN (method B, what nm_acceleration uses) or
 * NM_ACCEL_COARSE_FLUX (method C): the covered neighbour of an uncovered cell
 * takes a virtual value V making the coarse gradient across their shared face
 * equal to the mean of the fine gradients across it ((V - Phi_C)/dx_n =
 * mean over the 2x2 touching fine cells of (Phi_f - Phi_B)/dx_{n+1}, Phi_B the
 * Eqs. 3-6 ghost values); the ghosts read V in turn, so the two steps are
 * repeated `iters` times (1..1000; each sweep halves the change, 32 gives
 * double precision), starting from the coarse level's own value, and the fine
 * cells' ghosts then use the final values too.  The face arrays live in the
 * plan's workspace (2 (L-1) 6 (N/2+2)^2 doubles), so calls on one plan must
 * not overlap on the GPU.  Otherwise as nm_acceleration. */
enum { NM_ACCEL_COARSE_MEAN = 0, NM_ACCEL_COARSE_FLUX = 1 };
nm_status nm_acceleration_ex(nm_plan_t plan, const double* phi, double* g, int coarse_side, int iters,
                             void* stream);

/* Same result from HOST buffers: copies rho to the device, solves, copies phi
 * back, all on `stream`, and waits for the stream before returning.  Host
 * buffers in pinned memory give asynchronous copies. */
/* n solves from HOST buffers, pipelined: the upload of solve i+1 and the
 * download of solve i-1 run on two copy streams of the plan while solve i runs
 * on `stream` (two device staging sets, allocated on first use and counted in
 * nm_workspace_bytes).  rho_host[i] and phi_host[i] as for nm_potential_host;
 * page-locked host memory lets the copies overlap.  Synchronous: returns when
 * every phi_host[i] is written.  Calls on one plan must not overlap. */
nm_status nm_potential_host_many(nm_plan_t plan, int n, const void* const* rho_host, double* const* phi_host,
                                 void* stream);

nm_status nm_potential_host(nm_plan_t plan, const void* rho_host, double* phi_host,
                            void* stream);

/* Device bytes held by the plan (workspace, excluding the shared spectrum),
 * and the bytes of the cached spectra it uses (each octant in double, float
 * and double-float; for FP32 plans with 2N >= 64 also the float rows over all
 * kx that both FP32 z-seams read); for admission control. */
nm_status nm_workspace_bytes(nm_plan_t plan, size_t* bytes);
nm_status nm_spectrum_bytes(nm_plan_t plan, size_t* bytes);

/* Device bytes nm_plan_ex(opt) would allocate for its workspace with the
 * default schedule (no device work, no allocation): lets a server admit a
 * request by footprint before creating its plan.  NM_EINVAL / NM_EUNSUPPORTED
 * as nm_plan_ex. */
nm_status nm_footprint_bytes(const nm_options* opt, size_t* bytes);

/* Solve `n` independent meshes in one batched schedule on `stream` (the
 * levels and meshes are independent sub-problems, Sect. 4).  The passes of all
 * meshes are issued round by round: in round r every mesh contributes its r-th
 * group of level convolutions, and all contributions with the same transform
 * size and schedule share one launch per pass.  The first call with a given
 * (plans, rho, phi) set runs eagerly; a repeated call with the same set
 * replays a CUDA graph captured from it (pointers are baked into the graph, so
 * change the set to change the buffers).  plans[i], rho[i], phi[i] as for
 * nm_potential; plans must be distinct and on the current device; FP32 and
 * FP64 plans may be mixed. */
nm_status nm_batch_potential(int n, const nm_plan_t* plans, const void* const* rho,
                             double* const* phi, void* stream);

/* Kernel schedule of a plan's level convolutions. */
typedef struct {
    int group;   /* level convolutions (pairs of real fields) per launch, >= 1;
                    larger groups fill the GPU, smaller ones keep a pass's
                    working set in L2 for the next pass                      */
    int radix;   /* values per thread = first-pass radix: 16 or 8             */
    int tile;    /* column tile of the strided passes: 0 = 128-byte rows,
                    1 = 256-byte rows; with fuse 2, the CTAs per kx plane:
                    0 = the default split for P, 1 = the alternative one
                    (P = 128: 4 instead of 2; P = 256: 2 instead of 4)        */
    int pipeline;/* z-seam pass: 0 = one tile per CTA, one column per thread
                    (the default; FP32 level grids with P = 2N >= 64 stage
                    the CTA's spectrum rows in shared memory by cp.async
                    while the column loads are in flight); 1 = persistent CTAs fed
                    by a two-stage TMA (cp.async.bulk.tensor) pipeline;
                    2 = two columns per thread on paired FP32 instructions
                    (FP32 plans, radix 16, P = 2N >= 64, fuse 0);
                    3 = the same as persistent CTAs, each fetching its next
                    tile's columns while it transforms the current one
                    (FP32 plans, radix 16, P = 2N = 256, tile 0, fuse 0)      */
    int fuse;    /* 1 = x and y passes fused per z-slab through a thread-block
                    cluster (distributed shared memory), 3 launches per level
                    group instead of 5; needs radix 16; 0 = five passes;
                    2 = three passes: x-forward writing kx-major planes, one
                    pass per kx plane doing the y, z, spectrum multiply,
                    inverse z and inverse y steps in shared memory (the ky
                    residues split over a thread-block cluster whose partial
                    sums meet in distributed shared memory), x-inverse
                    (FP32 plans of the original method, radix 16, pipeline
                    0, P = 2N in 64 .. 512)                                   */
} nm_schedule;

/* Read / set the schedule (set reallocates the work buffers when group
 * grows; synchronises the device).  NM_EINVAL for out-of-range fields. */
nm_status nm_get_schedule(nm_plan_t plan, nm_schedule* out);
nm_status nm_set_schedule(nm_plan_t plan, const nm_schedule* sched);

/* Autotuner: times every candidate schedule (group in {1, 2, all}, radix in
 * {16, 8}, tile in {0, 1}, pipeline in {0, 1, 2, 3}, fuse in {0, 1, 2, 3}, where valid) with CUDA events over `reps` solves of the
 * caller's rho into phi (phi is overwritten), on `stream`, keeps the fastest
 * on the plan and records it in a process-wide table keyed by (device name,
 * N, levels, precision, method) that later plans of the same key start from.
 * When the environment variable NM_AUTOTUNE_CACHE names a file, the table is
 * read from it at the first plan creation and appended to after each tuning
 * (one JSON object per line).  Synchronous. */
nm_status nm_autotune(nm_plan_t plan, const void* rho, double* phi, int reps, void* stream);

/* Copy the plan's unit-cell spectrum octant ((N+1)^3 doubles, [kz][ky][kx])
 * to host memory `host_out`.  Synchronous.  Test hook. */
nm_status nm_get_green_octant(nm_plan_t plan, double* host_out);

/* Read the plan's options back. */
nm_status nm_get_options(nm_plan_t plan, nm_options* out);

/* Free the plan and its workspace (synchronises the device first). */
nm_status nm_destroy(nm_plan_t plan);

/* Device status word: NM_ETIMEOUT once a bounded device-side wait of a
 * library kernel has run out since the last clear (that kernel stopped early
 * and the solve's results are invalid), NM_OK otherwise.  Synchronises the
 * current device; `clear` resets the word. */
nm_status nm_device_status(int clear);

/* Test hook for failure detection: while `on` is nonzero the TMA-fed z-seam
 * issues no loads, so its bounded waits run out (after about 0.1 s) and it
 * raises NM_ETIMEOUT instead of hanging.  Results computed meanwhile are
 * invalid.  Process-wide. */
nm_status nm_debug_fault_timeout(int on);

/* Test hook, host-side fault injection: with n > 0 the n-th workspace
 * allocation made by the next plan creations fails as if the device were out
 * of memory (nm_plan_ex then returns NM_ENOMEM after freeing what it had
 * allocated); 0 disarms.  NM_EINVAL for n < 0. */
nm_status nm_debug_fail_alloc(int n);

/* Test hook: transform `lines` contiguous lines of P complex values (P a
 * power of two, 8..1024) in place with the passes' line transform (fft.cuh):
 * forward X[k] = sum_j x[j] exp(-2 pi i jk/P), or with `inverse` the + sign and
 * no 1/P.  `data` is device memory, interleaved re/im, double for NM_FP64 and
 * float for NM_FP32; asynchronous on `stream`.  NM_EINVAL for bad arguments,
 * NM_EUNSUPPORTED for P out of range. */
nm_status nm_debug_fft(int P, int precision, int inverse, int lines, void* data, void* stream);

/* Number of kernels this library has launched in the process so far. */
uint64_t nm_kernel_launches(void);

/* Per-kernel timing for measurement.  While enabled, every kernel the library
 * launches is bracketed by two CUDA events recorded on its own stream.
 * nm_profile_enable(1) clears earlier records; nm_profile_read waits for the
 * recorded events and writes up to `max` aggregated entries (one per kernel
 * name: launches, units of work processed -- convolution pairs for the FFT
 * passes, levels for the others -- and summed event time in ms) and their
 * number to *count.  Host-side bookkeeping only; results are unchanged. */
typedef struct {
    char name[48];
    uint64_t launches;
    uint64_t units;
    double total_ms;
} nm_kernel_stat;
nm_status nm_profile_enable(int on);
nm_status nm_profile_read(nm_kernel_stat* out, int max, int* count);

/* Allocation-free solve.  No counterpart in the paper: this entry point exists
 * for callers that cannot call cudaMalloc while they run -- codes that size
 * their device pools at start-up and forbid later allocations, processes whose
 * device memory belongs to another framework's allocator, and loops that
 * cannot afford cudaMalloc's implicit device-wide synchronisation.
 * It computes the same potential as nm_potential with a plan made from `opt`
 * for the mesh described by `opt` (method must be NM_METHOD_ORIGINAL, else
 * NM_EUNSUPPORTED; precision NM_FP64 or NM_FP32; either interpolation), from
 * device `rho` to device `phi`, asynchronously on `stream`, and never
 * allocates: all scratch (spectrum, tables, work buffer, level potentials)
 * lives in one file-scope device array of NM_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library holds until exit.  Meshes whose scratch would not
 * fit are rejected with NM_EINVAL and a message giving the bytes needed.
 * What fits: N <= 16, every level count, both precisions; N = 32 in FP32,
 * every level count; N = 32 in FP64, up to 14 levels with NM_INTERP_DIAGONAL
 * and up to 15 with NM_INTERP_TRILINEAR; N >= 64 never.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents (each call writes every region before reading it); calls that
 * overlap on the GPU race on it, so serialise them. */
#define NM_NOALLOC_SCRATCH_BYTES (8u << 20)
nm_status nm_potential_noalloc(const nm_options* opt, const void* rho, double* phi, void* stream);

const char* nm_status_string(nm_status s);
const char* nm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NESTCONV_NM_H */
