/*
 * motjvie.h -- C ABI of libmotjvie: a single-GPU (sm_103a) marching-on-in-time
 * current-density volume integral equation (MOT-JVIE) solver for transient
 * dielectric scattering, whose present-time operator Z0 is applied matrix-free
 * through zero-padded 3-D FFTs (paper Sec. IV, Eq. 10-12).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Status: every call returns a mot_status; 0 is success, negative values are
 *   errors.  No call aborts or throws across the ABI.  mot_last_error() returns
 *   a thread-local message describing the last failure of the calling thread.
 * - Grid: n = {Nx, Ny, Nz} voxels of isotropic size h [m] (Sec. II: uniform
 *   Cartesian voxel grid; Table I lists only isotropic meshes).  Voxel arrays are
 *   [Nz][Ny][Nx] with x fastest.  Current vectors carry 3 Cartesian components
 *   per voxel, [3][Nz][Ny][Nx], and a batch of nrhs excitations is
 *   [nrhs][3][Nz][Ny][Nx].  Every voxel carries 3 unknowns, including voxels
 *   with eps_r = 1, where the current is identically zero (Sec. II).
 * - Time step: dt = alpha * dt_CFL with dt_CFL = h / (c0 sqrt 3) (Eq. 9), i.e.
 *   c0 dt / h = alpha / sqrt 3.
 * - Ownership: the caller owns every host array it passes; the library copies
 *   what it keeps.  Device memory of a problem or run is owned by the library
 *   (cudaMalloc on the context's device) and freed by the matching destroy.
 *   Device pointers passed in (mot_apply_Z0) stay owned by the caller and must
 *   hold at least the documented number of elements.  Borrowed device
 *   pointers handed out (mot_run_current_device) stay valid until the next
 *   mot_run_step or mot_run_destroy on that run.
 * - Streams: all device work of a context is ordered on the context's stream
 *   (the one given to mot_ctx_create; NULL = the legacy default stream).
 *   Calls that return host data synchronise that stream before returning.
 * - Threads: handles are not thread-safe; use one context per host thread.
 */
#ifndef MOTJVIE_H
#define MOTJVIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MOT_OK = 0,
    MOT_EINVAL = -1,       /* invalid argument (message says which)                    */
    MOT_ENOMEM = -2,       /* device or host allocation failed                         */
    MOT_ENOTCONV = -3,     /* TFQMR did not reach the tolerance within maxit          */
    MOT_EUNSUPPORTED = -4, /* valid request outside what this build supports          */
    MOT_ECUDA = -5,        /* a CUDA runtime call failed (message has the CUDA error)  */
    MOT_ETIMEOUT = -6,     /* a bounded device wait gave up                            */
    MOT_EBUSY = -7,
    MOT_ECANCELLED = -8
} mot_status;

/* arithmetic of a marching run (a5/a6 of the solver):
 * MOT_FP64   -- every product, FFT, history sum and Krylov vector in FP64;
 * MOT_MIXED  -- FFTs, spectral multiplies, the history sum and the inner TFQMR
 *               vectors in FP32; FP64 for Krylov inner products, the residual,
 *               the refinement correction and the marched solution J_n.
 * MOT_FP64DF -- the FP64 path's accuracy (tolerance 1e-11 by default) from the
 *               mixed path's structure: FP32 inner TFQMR solves refined against
 *               residuals whose Z0 product runs in double-float (FP32 pairs,
 *               about 48 bits), the history ring, its spectra and the history
 *               sum in double-float too; J_n and the residual in FP64.        */
typedef enum { MOT_FP64 = 0, MOT_MIXED = 1, MOT_FP64DF = 2 } mot_precision;

/* element type of device vectors handed to mot_apply_Z0, and the arithmetic
 * of its FFTs: MOT_F64 and MOT_F32 vectors computed in that precision;
 * MOT_F64DF -- FP64 vectors, the FFTs and the spectral multiply in
 * double-float (each value an unevaluated sum of two FP32 numbers, about 48
 * significant bits, on the FP32 pipe), the contrast terms in FP64.          */
typedef enum { MOT_F64 = 0, MOT_F32 = 1, MOT_F64DF = 2 } mot_dtype;

/* Modulated-Gaussian plane wave of Eq. 7-8:
 *   E^i(r,t) = E0 pol (1/(sigma sqrt(2 pi))) exp(-tau^2/(2 sigma^2)) cos(2 pi f0 tau),
 *   tau = t - t0 - khat.(r - r_ref)/c0,
 * with r_ref the grid corner that minimises khat.r, so the pulse enters the
 * grid at t = t0.  SI units: E0 [V/m], sigma and t0 [s], f0 [Hz].  khat and pol
 * must be unit vectors with khat.pol = 0 (|.|, dot checked to 1e-9).            */
typedef struct {
    double E0, sigma, t0, f0;
    double khat[3];
    double pol[3];
} mot_planewave;

/* Solver options; pass NULL for the defaults shown.                           */
typedef struct {
    double tol;       /* TFQMR relative residual target (paper: 1e-6, Sec. V-A).
                         Default 1e-11 for MOT_FP64 and MOT_FP64DF (outer), 1e-6
                         (outer) for MOT_MIXED                                      */
    int maxit;        /* TFQMR iteration cap per solve (default 500)             */
    double inner_tol; /* inner FP32 TFQMR tolerance of MOT_MIXED and MOT_FP64DF (default 1e-6),
                         relative to the refinement residual r; a sweep whose r
                         is already small against the outer right-hand side b
                         solves only to max(inner_tol, 0.3 tol ||b|| / ||r||)
                         (at most 1/2): the outer test is what it must pass     */
    int max_refine;   /* refinement sweeps cap of MOT_MIXED and MOT_FP64DF (default 6) */
    double delta;     /* diagonal shift of the delta-regularised MOT (Sec. II,
                         Z^delta_n = Z_n + delta_n I): here delta_0 = delta for the
                         present-time matrix (every Z0 product and the solve) and
                         delta_n = 0 for the history lags n >= 1.  The paper uses
                         0 (the default); any finite value is accepted           */
    int timing;       /* 1: time the history z-pass and the Z0 spectral z-pass
                         kernels of every step with CUDA events (fills
                         ms_zhist / ms_zgreen of mot_step_stats; adds event
                         overhead).  Default 0                                     */
    int guess;        /* initial guess of each step's solve (the paper does not
                         specify one): 0 = J_{n-1}; 1 = 2 J_{n-1} - J_{n-2}
                         (linear extrapolation); 2 = 3 J_{n-1} - 3 J_{n-2} +
                         J_{n-3} (quadratic, default; one more FP64 current
                         vector held by the run).  Products per step on the
                         256 x 256 x 80 pillar array: 21.0 / 19.8 / 19.0      */
    int graph;        /* 1 (default): after the first step each step is one CUDA
                         graph launch whose loops and tests run on the device; 0:
                         host-driven steps, each solve's TFQMR loop one graph
                         launch (the timing option times the products outside
                         it); 2: no CUDA graphs at all, every kernel launched
                         from the host and the TFQMR loop tested on the host
                         after each iteration (slowest; for per-kernel
                         profilers and the timing option over every product)  */
    int autotune;     /* 1 (default): the launch schedule of the Z0 product (columns
                         per z-pass block, rows per row-pass block, plane-pass
                         block sizes, generic-pass widths, programmatic dependent
                         launch) is picked by timing candidates on first use for
                         each (number of right-hand sides, precision); every
                         candidate's product is checked against the built-in
                         schedule's.  Results are cached per process.  0: the
                         built-in rules.  Not in the paper (a B300 tuning aid)     */
} mot_options;

typedef struct {
    int32_t n[3];    /* Nx, Ny, Nz                                              */
    int32_t M0[3];   /* padded FFT grid of the present-time product (>= N + r0)  */
    int32_t Mh[3];   /* padded FFT grid of the history sum (>= 2N - 1)           */
    int32_t r0;      /* reach of the lag-0 table: largest |d_i| with g_0(d) != 0 */
    int32_t ell;     /* history length ell = ceil(R_max/(c0 dt)) + 2 (Eq. 4)     */
    double rho;      /* c0 dt / h = alpha / sqrt 3                               */
    double dt;       /* time step [s]                                            */
} mot_problem_info;

typedef struct {
    int32_t iters;     /* TFQMR iterations (sum over refinement sweeps)          */
    int32_t sweeps;    /* refinement sweeps (1 for MOT_FP64)                     */
    double relres;     /* final ||b - Z0 J_n|| / ||b|| (max over the batch)       */
    float ms_history;  /* device time of the right-hand side (0 in graph mode)  */
    float ms_solve;    /* device time of the solve (graph mode: the whole step) */
    float ms_push;     /* device time of the ring update (0 in graph mode)      */
    int32_t mvps;      /* Z0 products applied in the step                        */
    float ms_zhist;    /* history z-pass kernel time (timing option, else 0)     */
    float ms_zgreen;   /* mean time of the step's timed Z0 spectral z passes
                          (timing option; graph = 0: those outside the TFQMR
                          loop graph, graph = 2: all of them)                    */
} mot_step_stats;

typedef struct mot_ctx mot_ctx;
typedef struct mot_problem mot_problem;
typedef struct mot_run mot_run;

/* Message of the calling thread's last failure ("" if none).                  */
const char *mot_last_error(void);

/* Context on CUDA device `device`, ordering all work on `cuda_stream` (a
 * cudaStream_t, borrowed; NULL is the CUDA legacy default stream, which is also
 * PyTorch's default stream).  Errors: MOT_EINVAL (bad device), MOT_ECUDA.      */
mot_status mot_ctx_create(int device, void *cuda_stream, mot_ctx **out);
void mot_ctx_destroy(mot_ctx *ctx);

/* Problem: grid n, spacing h [m] > 0, relative permittivity eps_r (host,
 * [Nz][Ny][Nx] doubles, each finite and >= 1; copied), time-step factor
 * alpha > 0 (dt = alpha dt_CFL, Eq. 9).  Computes the lag-0 Galerkin table,
 * its spectrum on the M0 grid and the device copies of eps_r.  The history
 * tables are computed on the first mot_run_create.  Sec. II, Eq. 4, Eq. 10-11.
 * Errors: MOT_EINVAL (sizes, h, alpha, eps_r), MOT_ENOMEM, MOT_ECUDA.           */
mot_status mot_problem_create(mot_ctx *ctx, const int32_t n[3], double h, const double *eps_r,
                              double alpha, const mot_options *opt, mot_problem **out);
mot_status mot_problem_info_get(const mot_problem *p, mot_problem_info *info);

/* The launch schedule the autotuner picked for the Z0 product of `nrhs`
 * right-hand sides in dtype (MOT_F64 / MOT_F32): 0 in a choice field means the
 * built-in rule.  Tuning happens in mot_run_create (the run's batch and
 * precision) and in the first mot_apply_Z0 of each (nrhs, dtype), when the
 * problem's autotune option is on.  Errors: MOT_EINVAL (nothing tuned for that
 * pair).                                                                       */
typedef struct {
    int32_t z_cols;      /* z-pass columns per block (4, 8, 16, 32)            */
    int32_t x_rows;      /* rows per block of the compiled row passes           */
    int32_t xy_fwd;      /* plane-pass threads per block, forward / inverse     */
    int32_t xy_inv;
    int32_t pdl;         /* programmatic dependent launch on (1) / off (0)      */
    int32_t gen_pairs;   /* generic row passes: row pairs per block             */
    int32_t gen_tile;    /* generic column passes: columns per block            */
    int32_t z_tma;       /* 1: the z pass stages its column tiles with TMA      */
    int32_t candidates;  /* candidates timed                                    */
    int32_t rejected;    /* candidates whose product differed (discarded)       */
    int32_t cached;      /* 1: taken from this process's cache, not re-timed    */
    float ms_default;    /* product time with the built-in rules [ms]           */
    float ms_tuned;      /* product time with the chosen schedule [ms]          */
    double max_rel_diff; /* largest relative L2 difference of a candidate's
                            product from the built-in schedule's                */
} mot_schedule;
mot_status mot_problem_schedule(const mot_problem *p, int nrhs, int dtype, mot_schedule *out);
void mot_problem_destroy(mot_problem *p);

/* y = Z0 x for nrhs current vectors (Eq. 12: Z0 x = D x - X (G x), with
 * (G x) from Eq. 11 through zero-padded FFTs on the M0 grid).  x_dev, y_dev:
 * device arrays of nrhs*3*Nz*Ny*Nx elements of `dtype` (MOT_F64 computes in
 * FP64, MOT_F32 in FP32, MOT_F64DF takes FP64 vectors and computes the FFTs in
 * double-float, relative error about 1e-14), x fastest; x and y must not overlap and must be
 * 16-byte aligned (the kernels move 16-byte packs).  Asynchronous on the
 * context stream.  Errors: MOT_EINVAL (null, nrhs < 1, dtype, alignment),
 * MOT_ENOMEM (workspace), MOT_ECUDA.                                          */
mot_status mot_apply_Z0(mot_problem *p, const void *x_dev, void *y_dev, int nrhs, int dtype);

/* Byte size of the scratch array behind mot_apply_Z0_static (64 MiB).        */
#define MOT_STATIC_SCRATCH_BYTES (64ull << 20)

/* y = Z0 x exactly as mot_apply_Z0 computes it, for callers that must not
 * allocate device memory when they call in: callers that run under a memory
 * pool or budget that forbids new allocations, and real-time loops where a
 * cudaMalloc stall (it synchronises the device) is not acceptable.  This call
 * allocates nothing: its scratch is one file-scope __device__ array of
 * MOT_STATIC_SCRATCH_BYTES bytes that every GPU which loads the library holds
 * until the process exits.  (No counterpart in the paper: an ABI addition.)
 * - The first call on a device resolves the array's device address with
 *   cudaGetSymbolAddress (with that device current) and keeps it for the
 *   process; make that first call before any stream capture.  cudaDeviceReset
 *   invalidates the kept address: do not call this entry point after one.
 * - All calls share the one array, which keeps the previous call's contents:
 *   every scratch element is written before it is read, so nothing needs to
 *   start at zero.  Calls whose kernels overlap on the GPU (other streams or
 *   threads) race on the array; order them on one stream.
 * - x_dev, y_dev, nrhs, dtype as mot_apply_Z0.  With c = the byte size of one
 *   complex element of the FFT (16 for MOT_F64 and MOT_F64DF, 8 for MOT_F32)
 *   and H0 = M0x/2 + 1, the scratch needed is
 *   round_up(nrhs * 3 * Nz * Ny * H0 * c, 256) + nrhs * 3 * Nz * M0y * H0 * c
 *   bytes; a request above MOT_STATIC_SCRATCH_BYTES fails with MOT_EINVAL
 *   (message gives both sizes) before any device work.
 * - No kernel-timing events are recorded by this call (mot_run_kernel_times
 *   is unaffected by it).
 * Errors: MOT_EINVAL, MOT_ECUDA.                                              */
mot_status mot_apply_Z0_static(mot_problem *p, const void *x_dev, void *y_dev, int nrhs, int dtype);

/* y = Z0 x by direct summation over the nonzero entries of the present-time
 * matrix (the paper's "direct" product, Sec. IV and V-A, here on the GPU):
 * (Z0 x)_p(m) = eps(m) T(0) x_p(m) - (eps(m) - 1) sum_d sum_q g0(d)_pq x_q(m - d)
 * over the offsets d of the lag-0 support (x = 0 outside the grid).  Same
 * arguments, layout and precision choice as mot_apply_Z0, same result up to
 * rounding; its cost grows with nnz(Z0) (the number of offsets grows as
 * alpha^3), the FFT product's does not, so it is the faster of the two at small
 * alpha only.  One kernel launch: shared-memory tiles of the input with a halo
 * of the table's reach, or neighbour reads through the caches where such a tile
 * does not fit.  Allocates the offset list on its first call (per precision).
 * Errors: MOT_EINVAL, MOT_ENOMEM, MOT_ECUDA.                                    */
mot_status mot_apply_Z0_direct(mot_problem *p, const void *x_dev, void *y_dev, int nrhs, int dtype);

/* The library's own Galerkin table of lag `lag` (0 <= lag <= ell):
 * g_out[6][2Rz+1][2Ry+1][2Rx+1] doubles, components (xx, yy, zz, xy, xz, yz),
 * offset d = (dx, dy, dz) at index (dz+Rz, dy+Ry, dx+Rx); R_out receives
 * (Rx, Ry, Rz) = min(reach of lag, N_i - 1).  If g_out is NULL only R_out is
 * written.  Synchronous.  Errors: MOT_EINVAL, MOT_ECUDA.                      */
mot_status mot_kernel_table(mot_problem *p, int lag, double *g_out, int32_t R_out[3]);

/* Replace the table of lag `lag` by a caller-supplied one (same layout as
 * mot_kernel_table, extents R; entries beyond N_i - 1 are ignored) and
 * recompute that lag's spectrum.  Used to feed an externally computed table
 * into the FFT path.  Lags >= 1 must be set before mot_run_create.
 * Errors: MOT_EINVAL, MOT_ENOMEM, MOT_ECUDA.                                   */
mot_status mot_set_kernel_table(mot_problem *p, int lag, const double *g, const int32_t R[3]);

/* Host-only table generator (no GPU needed): the lag-`lag` Galerkin table for
 * c0 dt / h = rho over |d_i| <= R_i, same layout as mot_kernel_table.
 * Errors: MOT_EINVAL.                                                          */
mot_status mot_table_host(double rho, int lag, const int32_t R[3], double *g_out);

/* A marching run of nrhs excitations sharing the problem's Z0 (host array of
 * nrhs plane waves, copied).  Allocates the device history ring (ell slots of
 * spectra on the Mh grid) and computes the history tables on first use.
 * Errors: MOT_EINVAL (nrhs < 1, bad plane wave), MOT_ENOMEM, MOT_ECUDA.        */
mot_status mot_run_create(mot_problem *p, int nrhs, const mot_planewave *exc, int precision,
                          mot_run **out);

/* Advance nsteps time steps (Eq. 3): b_n = E^i_n - sum_{k=1..ell} Z_k J_{n-k},
 * then Z0 J_n = b_n by TFQMR (x0 from options.guess).  J_out (host, nullable)
 * receives [nsteps][nrhs][3][Nz][Ny][Nx] doubles in A/m^2 (in graph mode each
 * J_n goes through a device staging buffer and reaches the host on its own
 * stream while the next step runs: page-locked J_out memory lets the copies
 * overlap the steps); stats (nullable) receives nsteps entries.  Synchronous
 * when J_out or stats is given; the first J_out use in graph mode allocates
 * two staging buffers of nrhs*3*n doubles.
 * Errors: MOT_EINVAL, MOT_ENOTCONV (state still advanced), MOT_ECUDA.         */
mot_status mot_run_step(mot_run *r, int nsteps, double *J_out, mot_step_stats *stats);

/* Checkpoint: write run r's state to the file at path -- the problem's
 * fingerprint (grid, h, alpha, a hash of eps_r), precision, plane waves, the
 * next step index, J_{n-1}, J_{n-2} (and J_{n-3} when the run's options.guess
 * is 2) and the whole history ring of spectra (ell slots; for large grids this
 * is most of the file) -- so that marching
 * can resume in another process.  Synchronises the context stream.  The
 * format is this library's own (little-endian, version 1).
 * Errors: MOT_EINVAL (null, file cannot be written), MOT_ECUDA.              */
mot_status mot_run_save(mot_run *r, const char *path);

/* Resume: create a run on problem p from a checkpoint written by
 * mot_run_save.  p must describe the same problem (grid, h, alpha and eps_r
 * are checked against the checkpoint; options may differ: a run whose guess
 * needs J_{n-3} but whose checkpoint has none takes J_{n-2} for it).  The first step
 * after loading runs host-driven, then graph mode resumes.  *out is owned by
 * the caller (mot_run_destroy).
 * Errors: MOT_EINVAL (null, unreadable/corrupt file, another problem),
 * MOT_ENOMEM, MOT_ECUDA.                                                      */
mot_status mot_run_load(mot_problem *p, const char *path, mot_run **out);

/* Device pointer to the latest J_n: nrhs*3*Nz*Ny*Nx doubles (borrowed).      */
mot_status mot_run_current_device(mot_run *r, const void **J_dev);

/* Number of CUDA kernels this library has launched in this process so far
 * (instrumentation for launch accounting; no counterpart in the paper).        */
mot_status mot_kernel_launches(uint64_t *count);

/* Measured FMA throughput of device `device` for dtype MOT_F64 or MOT_F32:
 * one microkernel of independent FMA chains (8 per thread, a whole multiple of
 * the SM count of 256-thread blocks), calibrated to about 100 ms per launch;
 * *flop_per_s = 2 * FMAs / time of the fastest of three launches (CUDA
 * events), *ms (nullable) that time.  The denominator of the FP64 product's
 * roofline (instrumentation; no counterpart in the paper).  Leaves no device
 * state behind; GPU clocks are read by the caller, never set.
 * Errors: MOT_EINVAL, MOT_ENOMEM, MOT_ECUDA.                                   */
mot_status mot_fma_peak(int device, int dtype, double *flop_per_s, double *ms);

/* Index of the next step to be computed.                                       */
mot_status mot_run_step_index(const mot_run *r, int64_t *n);

/* ---------------------------------------------------------------- serving
 * A server runs many scattering runs (different grids, permittivities, step
 * sizes) on one GPU with continuous batching: requests are admitted in arrival
 * order whenever a slot is free and their estimated device memory fits under
 * the budget and in free memory; each admitted run keeps its Green spectra and
 * history ring on the device and advances one MOT step per worker pass on its
 * own stream, so runs that arrive while others are on the GPU overlap with
 * them.  Each run's currents are the same as the run alone (the same kernels
 * and drivers).  No counterpart in the paper (a deployment pattern).          */
typedef struct mot_server mot_server;

typedef struct {
    int32_t n[3];              /* Nx, Ny, Nz                                        */
    double h;                  /* voxel size [m]                                   */
    const double *eps_r;       /* host [Nz][Ny][Nx], copied at submit               */
    double alpha;              /* dt = alpha dt_CFL                                */
    int32_t precision;         /* MOT_FP64, MOT_MIXED or MOT_FP64DF                */
    int32_t nrhs;              /* plane waves                                      */
    const mot_planewave *exc;  /* host [nrhs], copied at submit                    */
    int32_t nsteps;            /* steps to march                                  */
    const mot_options *opt;    /* nullable (defaults), copied at submit           */
    double *J_final;           /* host [nrhs][3][Nz][Ny][Nx] or NULL: receives J of
                                  the last step; must stay valid until the wait on
                                  this request's ticket returns                    */
} mot_request;

typedef struct {
    int32_t status;        /* MOT_OK, MOT_ENOTCONV (some step missed its tolerance),
                              MOT_ENOMEM (never fits the budget / free memory),
                              MOT_ECANCELLED (server destroyed), other errors     */
    int32_t steps;         /* steps completed                                     */
    double queue_ms;       /* submit -> admission (host clock)                   */
    double run_ms;         /* admission -> completion (host clock)               */
    float step_p50_ms;     /* per-step device time (CUDA events), median          */
    float step_p99_ms;     /* per-step device time, 99th percentile               */
    uint64_t device_bytes; /* device memory reserved for the run                  */
} mot_result;

/* Start a server on ctx's device with a device-memory budget in bytes (0:
 * 80% of the free memory now) and at most max_slots runs on the GPU at once.
 * Errors: MOT_EINVAL (null, max_slots outside [1, 256]), MOT_ECUDA.          */
mot_status mot_server_create(mot_ctx *ctx, size_t mem_budget, int max_slots, mot_server **out);

/* Queue a run; *ticket identifies it for mot_server_wait.  Host inputs are
 * copied before returning.  Errors: MOT_EINVAL (bad request), MOT_EBUSY
 * (4096 requests already waiting).                                          */
mot_status mot_server_submit(mot_server *s, const mot_request *req, uint64_t *ticket);

/* Wait up to timeout_s seconds for the run of ticket to finish and collect
 * its result (the ticket is then released).  Errors: MOT_EINVAL (null,
 * unknown or collected ticket), MOT_ETIMEOUT (not finished in time; the
 * ticket stays valid).                                                        */
mot_status mot_server_wait(mot_server *s, uint64_t ticket, double timeout_s, mot_result *res);

/* Stop the server: runs on the GPU finish their current step and are
 * abandoned, waiting requests are cancelled.  Call after every wait has
 * returned.                                                                    */
void mot_server_destroy(mot_server *s);

/* Kernel classes timed by the timing option (mot_options.timing = 1 with
 * graph = 0 or 2): CUDA events around every launch of these kernels during a
 * step (kernels inside CUDA graphs cannot be bracketed).  Instrumentation; no
 * counterpart in the paper.                                                    */
typedef enum {
    MOT_K_Z_GREEN = 0,      /* present-time z pass: FFT z, Lambda0 multiply, IFFT z (Eq. 11) */
    MOT_K_Z_HISTORY = 1,    /* history z pass: lag 1 onto the step's lags 2.. sum, IFFT z (Eq. 3) */
    MOT_K_FWD_HALF = 2,     /* forward xy pass of Z0 y2 with the first TFQMR half step     */
    MOT_K_FWD_Y1 = 3,       /* forward xy pass of Z0 y1 forming y1 = w + beta y2           */
    MOT_K_FWD_PLAIN = 4,    /* forward xy pass of a stored vector (other Z0 products)     */
    MOT_K_FWD_RING = 5,     /* forward xy pass of J_n into the history ring (Mh grid)      */
    MOT_K_INV_HALF = 6,     /* inverse xy pass of Z0 y2 with the second TFQMR half step    */
    MOT_K_INV_V = 7,        /* inverse xy pass of Z0 y1 with the v update                  */
    MOT_K_INV_Z0 = 8,       /* inverse xy pass with the plain Z0 epilogue (Eq. 12)         */
    MOT_K_INV_RESIDUAL = 9, /* inverse xy pass with the FP64 residual b - Z0 J            */
    MOT_K_INV_HISTORY = 10, /* inverse xy pass of the history sum forming b_n (Eq. 3)     */
    MOT_K_ROW_FWD = 11,     /* planes too large for shared memory: forward row pass (x)
                               and forward column pass (y) of a Z0 product                 */
    MOT_K_ROW_INV = 12,     /* the same: inverse column pass (y) and inverse row pass (x)
                               with the product's epilogue                                 */
    MOT_K_VEC = 13,         /* the TFQMR vector kernels of the path whose planes do not
                               fit in shared memory (half steps, y1, v updates)            */
    MOT_K_HIST_SIDE = 14,   /* time-blocked history: the block pass over the ring at a
                               block start and the near accumulation of lags 2.. of the
                               step (in graph mode they run beside the previous step)     */
    MOT_K_CLASSES = 15
} mot_kernel_class;

/* Timing-option results of the latest step of run r: the number of launches
 * of class cls and their mean device time in ms (0 and 0 when none was timed).
 * Synchronises the context stream.
 * Errors: MOT_EINVAL (null argument, cls out of range), MOT_ECUDA.           */
mot_status mot_run_kernel_times(mot_run *r, int cls, int32_t *launches, float *mean_ms);
void mot_run_destroy(mot_run *r);

#ifdef __cplusplus
}
#endif
#endif /* MOTJVIE_H */
