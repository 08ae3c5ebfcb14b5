/*
 * clb.h -- C ABI of libclb: the coupled D2Q9 (flow) + D2Q5 (temperature) central-moment lattice
 * Boltzmann method of Fei, Luo, Lin & Li, "Modeling incompressible thermal flows using a
 * central-moment-based lattice Boltzmann method" (arXiv:1710.10569), on one NVIDIA GB300 GPU.
 *
 * What one time step computes, per node x (the fused collide-and-stream step):
 *   pull    f_i(x) = f*_i(x - e_i), g_i(x) = g*_i(x - e_i)                       Eqs. (12), (22)
 *           (beyond a wall: halfway bounce-back for f; anti-bounce-back (Dirichlet T) or
 *            bounce-back (adiabatic) for g; periodic sides wrap)
 *   macro   rho = sum f, T = sum g, F = (Fv_x, Fv_y + rho0 g_beta (T - T0)),
 *           rho u = sum f e + F/2                                               Eqs. (3), (13), (23)
 *   D2Q9    Gamma~ = N(u) M f; Gamma~* = (I - S) Gamma~ + S Gamma~eq + (I - S/2) C;
 *           f* = M^-1 N(u)^-1 Gamma~*                                           Eqs. (6)-(11), Sec. 2.1
 *   D2Q5    Gamma~T = N_T(u) M_T g; Gamma~T* = (I - S_T) Gamma~T + S_T Gamma~T,eq;
 *           g* = M_T^-1 N_T(u)^-1 Gamma~T*                                      Eqs. (16)-(21), App. A
 *   store   f*, g* at x (two ping-pong buffers)
 * Relaxation rates: nu = (1/s_nu - 1/2)/3 (Sec. 2.1), alpha = (1/lambda1 - 1/2) cs2_T (Sec. 2.2).
 *
 * Conventions for every entry point:
 *  - Field arrays are double, row-major [ny][nx] (x fastest); node (x, y) sits at integer
 *    coordinates and walls lie halfway between nodes, so a wall-bounded extent of n nodes has
 *    length n. Population arrays exchanged with the caller are double [q][ny][nx].
 *  - "host" pointers are ordinary CPU memory (pinned memory makes copies faster); "device"
 *    pointers are CUDA global memory on the handle's device. The caller owns every buffer it
 *    passes; the library owns the populations and its scratch (unless memory is supplied to
 *    clb_create, in which case the caller keeps ownership and must keep it alive until destroy).
 *  - Work is enqueued on the handle's CUDA stream. Calls that return values to the host
 *    synchronise that stream; the others return after enqueueing.
 *  - Errors are status codes, never aborts. clb_last_error() returns a thread-local message for
 *    the last failing call on the calling thread. After CLB_ECUDA the handle should be destroyed.
 *  - Handles are not thread-safe: one thread at a time per handle.
 */
#ifndef CLB_H
#define CLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CLB_OK = 0,
    CLB_EINVAL = 1,   /* bad argument: size, rate outside (0, 2), unpaired periodic sides, NULL */
    CLB_ENOMEM = 2,   /* device memory or a memory budget is exhausted */
    CLB_ENAN = 3,     /* a NaN or Inf appeared in the fields (per instance for batches) */
    CLB_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    CLB_ECUDA = 5,    /* a CUDA runtime call failed; see clb_last_error() */
    CLB_EBUSY = 6     /* no free slot / the request is still running */
} clb_status;

/* Wall kind of one side. Every non-periodic wall is a stationary no-slip wall for the flow
 * (halfway bounce-back of f); the kind selects the temperature condition. */
typedef enum {
    CLB_PERIODIC = 0,        /* wraps to the opposite side, which must also be periodic */
    CLB_WALL_DIRICHLET_T = 1,/* g_i = -g*_opp + cs2_T * T_wall (anti-bounce-back, 2 w_i = cs2_T) */
    CLB_WALL_ADIABATIC = 2,  /* g_i = g*_opp (zero heat flux) */
    CLB_WALL_WET = 3         /* the paper's own conditions (Sec. 3): the wall lies ON the end row of
                              * nodes (y sides only, both, with periodic x; ny >= 3; H = ny - 1);
                              * velocity by non-equilibrium bounce-back with the half-force
                              * correction, temperature T_wall by non-equilibrium extrapolation
                              * from the adjacent fluid node. Nusselt averages use the trapezoid
                              * rule over [0, H]. */
} clb_wall;

/* Population storage. CLB_F64 stores f_i, g_i and computes in FP64. CLB_F32 and CLB_F16DEV store
 * the deviations from a rest state, f_i - w_i rho0 and g_i - w^T_i T_b(y) (w, w^T the rest
 * weights), in FP32 or IEEE half precision, and compute in FP32 on those deviations. T_b(y) is
 * T_ref, except between two Dirichlet (or two wet) y walls with periodic x, where it is the
 * conduction profile between the walls (linear in y), so that a layer near its conduction state
 * stores only its small departures from it. The choice changes rounding only. */
typedef enum { CLB_F64 = 0, CLB_F32 = 1, CLB_F16DEV = 2 } clb_storage;

/* Problem parameters (Sec. 2, Sec. 3 defaults from clb_params_default). */
typedef struct clb_params {
    double nu;        /* kinematic viscosity (lattice units), > 0 */
    double kappa;     /* thermal diffusivity alpha, > 0 */
    double g_beta;    /* |g| beta >= 0; gravity points to -y (Eq. 3) */
    double T0;        /* reference temperature of the Boussinesq force */
    double rho0;      /* reference density: force scale and FP16 deviation base */
    double s_b;       /* bulk-viscosity rate (Eq. 8 block), in (0, 2) */
    double s_3;       /* third-order rate (k~21, k~12), in (0, 2) */
    double s_4;       /* fourth-order rate (k~22), in (0, 2) */
    double lambda2;   /* D2Q5 second-order rate (k~20, k~02), in (0, 2) */
    double cs2_T;     /* D2Q5 sound speed squared, in (0, 1/2) */
    double Fv[2];     /* external body force density */
    int wall[4];      /* clb_wall for sides -x, +x, -y, +y */
    double T_wall[4]; /* wall temperatures for CLB_WALL_DIRICHLET_T sides */
    int storage;      /* clb_storage */
    double T_ref;     /* FP32/FP16 deviation base for g (normally T0; see clb_storage) */
    double u_ref;     /* residual floor scale for u (0: no floor) */
    double dT_ref;    /* residual floor scale for T (0: no floor) */
    double u_wall[4][2]; /* velocity of each wall (sides -x, +x, -y, +y; ignored on periodic sides):
                          * f_i = f*_opp + [f^eq_i - f^eq_opp](rho0, u_w) (moving-wall bounce-back,
                          * tangential motion and normal injection, Sec. 3.2) and
                          * g_i = -g*_opp + T_w (cs2_T + u_w,n^2) on Dirichlet walls */
} clb_params;

typedef struct clb_handle clb_handle;

/* Defaults of Sec. 3 (first paragraph): cs2_T = 1/4, high-order rates s_3 = s_4 = lambda2 = 1;
 * s_b = 1; rho0 = 1; all sides periodic; CLB_F64. */
clb_status clb_params_default(clb_params *p);

/* Device bytes one lattice of nx x ny needs (populations x 2, snapshot, staging, scratch). */
clb_status clb_footprint(int nx, int ny, const clb_params *p, size_t *bytes);

/* Create a lattice. stream: a cudaStream_t (NULL = legacy default stream). dev_mem / dev_bytes:
 * optional caller-owned device memory of at least clb_footprint() bytes, 256-byte aligned
 * (NULL: the library allocates and frees it). Validates parameters (EINVAL). Populations start
 * at rest (rho = 1, u = 0, T = T0) until clb_init_fields. */
clb_status clb_create(int nx, int ny, const clb_params *p, void *stream, void *dev_mem,
                      size_t dev_bytes, clb_handle **out);
void clb_destroy(clb_handle *h);

/* f(x, 0) = f^eq(rho, u), g(x, 0) = g^eq(T, u) with f^eq = M^-1 N(u)^-1 Gamma~eq (Eq. 9) and
 * g^eq = M_T^-1 N_T(u)^-1 Gamma~T,eq (Eq. 20). Host arrays; synchronous. Resets the step count
 * and takes the residual snapshot. Pinned host arrays (cudaMallocHost, cudaHostAlloc,
 * cudaHostRegister) are read by the initialisation kernel directly over the CPU-GPU link;
 * pageable arrays are copied to device staging first. */
clb_status clb_init_fields(clb_handle *h, const double *rho, const double *ux, const double *uy,
                           const double *T);
/* Same from device arrays; asynchronous on the handle's stream. */
clb_status clb_init_fields_device(clb_handle *h, const double *rho, const double *ux,
                                  const double *uy, const double *T);

/* Advance n >= 0 time steps (one fused collide-and-stream kernel per step, replayed from a CUDA
 * graph in chunks). Asynchronous. */
clb_status clb_step(clb_handle *h, long n);

/* rho, u (force-corrected, Eq. 13) and T (Eq. 23) at the current time, into host arrays (any may
 * be NULL). Synchronous. Pinned host arrays are written by the field kernel directly; pageable
 * ones through device staging. */
clb_status clb_fields(clb_handle *h, double *rho, double *ux, double *uy, double *T);
/* Same into device arrays (any may be NULL); asynchronous. */
clb_status clb_fields_device(clb_handle *h, double *rho, double *ux, double *uy, double *T);

/* Pre-collision populations at the current time (after streaming and boundaries), as double
 * host arrays f[9][ny][nx], g[5][ny][nx]; velocity order of Eq. (4). Synchronous. */
clb_status clb_populations(clb_handle *h, double *f, double *g);

/* Nusselt number of Eq. (29) along axis (0 = x, 1 = y): Nu = 1 + s <u_axis (T - T0)> H /
 * (kappa dT), averaged over all nodes, H = node count along axis, dT = |T_wall(lo) - T_wall(hi)|
 * (1 when equal), s = +1 when the low side is the hot one, else -1. Reduced in FP64 on the GPU in
 * a fixed order. Synchronous. CLB_ENAN when the fields are not finite. */
clb_status clb_nusselt(clb_handle *h, int axis, double *nu_out);

/* The Nusselt number of clb_nusselt computed without allocating any device memory, for callers
 * that cannot call cudaMalloc when they need it: for example a progress monitor in a server whose
 * device memory is already committed to resident lattices, or a latency-sensitive loop that must
 * not call cudaMalloc/cudaFree because they can synchronise the whole device. (The paper has no
 * counterpart; this is a service of the library.)
 * populations: device pointer to a population buffer in this library's layout for (nx, ny,
 * p->storage), e.g. the current buffer that clb_buffers returns; p: that lattice's parameters;
 * stream: the CUDA stream to run on; nu_out: host double, written on success. Synchronous: it
 * returns after the result has been copied back to the host and the stream has been synchronised.
 * Scratch is a fixed array of CLB_NOALLOC_MAX_ROWS rows of FP64 partial sums that the library keeps
 * in device memory on every device it is used on until the process exits; ny above that limit
 * returns CLB_EINVAL. The first call on a device looks up that array's address (with the device
 * current) and keeps it for later calls on that device. A cudaDeviceReset invalidates the kept address: do not call this entry point on a
 * device again after resetting it. All calls share the one array, so calls whose kernels overlap
 * on the GPU race: serialise them. Returns CLB_ENAN when the fields are not finite. The result
 * equals clb_nusselt on the same populations within rounding (bitwise for nx <= 2048; wider rows
 * are summed in one partial per row here and in several row segments by clb_nusselt). */
#define CLB_NOALLOC_MAX_ROWS 8192
clb_status clb_nusselt_noalloc(const void *populations, int nx, int ny, const clb_params *p, int axis,
                               void *stream, double *nu_out);

/* Steady-state residual against the snapshot taken by the previous call (or by init), then
 * retakes the snapshot: E_R = max over X in {u, T} of sqrt(sum|X - X_snap|^2 /
 * max(sum|X|^2, N (1e-3 X_ref)^2)), X_ref = u_ref, dT_ref. FP64 on the GPU. Synchronous. */
clb_status clb_residual(clb_handle *h, double *er_out);

/* Both diagnostics from one FP64 pass over the lattice: the Nusselt number along axis (as
 * clb_nusselt) and the residual E_R (as clb_residual, snapshot retaken). Either output may be
 * NULL. Synchronous. CLB_ENAN when the fields are not finite. */
clb_status clb_check(clb_handle *h, int axis, double *nu_out, double *er_out);

/* Step until E_R < tol, checked every `interval` steps, or until max_steps steps have been taken
 * by this call. Outputs may be NULL. CLB_ENAN if the fields blow up. */
clb_status clb_run(clb_handle *h, double tol, long max_steps, long interval, long *steps_out,
                   double *er_out);

/* Steps taken since init. */
clb_status clb_steps(clb_handle *h, long *steps_out);
/* Wait for all work of the handle. */
clb_status clb_sync(clb_handle *h);

/* Checkpoint: raw populations of the current time plus the step count. With buf == NULL,
 * *bytes receives the size. clb_load restores a checkpoint of the same size/storage. */
clb_status clb_save(clb_handle *h, void *buf, size_t *bytes);
clb_status clb_load(clb_handle *h, const void *buf, size_t bytes);

/* Launch shape of the step kernel: threads per block along x (32..256, multiple of 32), rows per
 * block (1..8, block_x * block_y <= 256) and nodes per thread along x (1, 2 or 4). 0 keeps the
 * current value. Defaults: 128 x 1 with 2 (FP32) or 4 (FP64, FP16) nodes per thread.
 * clb_autotune times candidate shapes on the live lattice (the populations are restored
 * afterwards; it allocates one buffer-sized scratch with cudaMallocAsync) and keeps the fastest;
 * results are cached per (storage, nx, ny) for later clb_create calls. The shape never changes
 * the results (the per-node arithmetic does not depend on it). */
clb_status clb_set_launch(clb_handle *h, int block_x, int block_y, int nodes_per_thread);
clb_status clb_get_launch(clb_handle *h, int *block_x, int *block_y, int *nodes_per_thread);
clb_status clb_autotune(clb_handle *h, int *block_x, int *block_y, int *nodes_per_thread);
/* Pipelined step kernel: stages = 0 uses the direct kernel; 2..4 stages of shared memory per warp
 * let each warp stage the pulled values of the next stages-1 rows with asynchronous copies while it
 * computes the current row; rows = rows each warp marches over (1..256; 0 keeps the value). Needs
 * 2 or 4 nodes per thread (clb_set_launch); the block is 128 threads. Results are bitwise those of
 * the direct kernel. clb_autotune also tries pipelined shapes and reports them here. */
clb_status clb_set_pipeline(clb_handle *h, int stages, int rows);
clb_status clb_get_pipeline(clb_handle *h, int *stages, int *rows);

/* The CUDA stream the handle enqueues on (to time its work with events on that stream). */
void *clb_stream(clb_handle *h);

/* How the FP16 storage form splits a time step (host only, no device work; for tools and tests).
 * The warps of the interior, whose 32 * npt nodes lie inside the row with no wall next to any of
 * them, run in one kernel; the others (rows next to a y wall or on a wet y wall, the columns next to
 * an x wall or on a wet x wall or holding the ragged end of the rows) run in a second kernel beside
 * it. Warp column c covers nodes c * 32 * npt .. c * 32 * npt + 32 * npt - 1 of a row. For a lattice
 * of nx x ny nodes with parameters p and npt nodes per thread (1, 2 or 4), geom receives 11 ints:
 * [0, 1] the interior rows [y0, y1); [2, 3] the interior warp columns [c0, c1); [4] warp columns per
 * row; [5] the number of edge rows and [6, 7] those rows (-1 if absent), every column of which goes
 * to the edge kernel; [8] the number of edge columns and [9, 10] those columns (-1 if absent), taken
 * in the rows [y0, y1). CLB_EINVAL for parameters that clb_create rejects or another npt. */
clb_status clb_step_partition(int nx, int ny, const clb_params *p, int npt, int *geom);

/* Device address of the current post-collision population buffer and of the other buffer, and
 * their layout (for profiling and checkpoint tools): chunked rows. Row y holds ceil(nx / chunk)
 * chunks of chunk consecutive nodes, the last one padded; a chunk holds its nodes' 14 populations
 * (f_0..f_8, g_0..g_4) one after another, chunk values each. Element (i, x, y) lies at
 *   y * row_elems + (x / chunk) * 14 * chunk + i * chunk + x % chunk
 * in elements of the storage type (chunk = 64, row_elems = 14 * 64 * ceil(nx / 64)). Any output
 * pointer may be NULL. */
clb_status clb_buffers(clb_handle *h, void **cur, void **other, size_t *row_elems, int *chunk);

const char *clb_last_error(void);
const char *clb_version(void);

/* ---------------------------------------------------------------------------------------------
 * Thermal-only mode: the D2Q5 central-moment equation alone (Eqs. 16-23) with a prescribed
 * velocity field, as in Sec. 3.1 where the velocity is given and only the temperature equation is
 * solved; usable for any convection-diffusion of a passive scalar (Sec. 4). Same walls (anti-bounce-
 * back / adiabatic / periodic), storage forms and parameters (nu, g_beta, Fv are unused). One step
 * moves 5 populations in and out plus the node's velocity (FP32: 48 bytes per node).
 */
typedef struct clb_thermal clb_thermal;

clb_status clb_thermal_create(int nx, int ny, const clb_params *p, void *stream, clb_thermal **out);
void clb_thermal_destroy(clb_thermal *h);
/* g = g^eq(T, u) (Eq. 20 back-transformed) and the velocity held fixed from here on. Host arrays
 * [ny][nx]; NULL means T = T0, u = 0. Synchronous; resets the step count. */
clb_status clb_thermal_init(clb_thermal *h, const double *T, const double *ux, const double *uy);
clb_status clb_thermal_step(clb_thermal *h, long n);
/* T (Eq. 23) at the current time into a host array. Synchronous. */
clb_status clb_thermal_fields(clb_thermal *h, double *T);
/* Pre-collision populations g[5][ny][nx] at the current time. Synchronous. */
clb_status clb_thermal_populations(clb_thermal *h, double *g);
clb_status clb_thermal_sync(clb_thermal *h);

/* ---------------------------------------------------------------------------------------------
 * Batches: many independent lattices of different sizes and parameters stepped together, one
 * launch per time step over the concatenated tiles of all active instances (captured in a CUDA
 * graph). Each instance computes exactly what a single lattice computes (bitwise the same).
 */
typedef struct clb_batch clb_batch;

/* n instances, sizes nx[k] x ny[k], parameters p[k] (all with the same storage). */
clb_status clb_batch_create(int n, const int *nx, const int *ny, const clb_params *p, void *stream,
                            clb_batch **out);
void clb_batch_destroy(clb_batch *b);
clb_status clb_batch_init_fields(clb_batch *b, int k, const double *rho, const double *ux,
                                 const double *uy, const double *T);
clb_status clb_batch_step(clb_batch *b, long n);
clb_status clb_batch_fields(clb_batch *b, int k, double *rho, double *ux, double *uy, double *T);
/* Nusselt number along axis[k] and residual (snapshot retaken) of every instance; FP64. */
clb_status clb_batch_diagnostics(clb_batch *b, const int *axis, double *nu, double *er);
/* Step all active instances; every `interval` steps retire those with E_R < tol or at max_steps
 * (their tiles leave the launch). steps[k], er[k], status[k] (clb_status) per instance. */
clb_status clb_batch_run(clb_batch *b, double tol, long max_steps, long interval, long *steps,
                         double *er, int *status);
/* State of every instance as of the last clb_batch_run or clb_batch_diagnostics: status[k]
 * (clb_status; CLB_ENAN for an instance whose fields blew up), the residual E_R and the Nusselt
 * number of its last check, and its steps since init. Host arrays of n entries, any may be NULL.
 * Reads host bookkeeping only (no device work). */
clb_status clb_batch_status(clb_batch *b, int *status, double *er, long *steps, double *nu);
/* Tile shape of the batched launch: threads along x (32..256), rows (block_x * rows <= 256) and
 * nodes per thread (1, 2, 4). Each block steps 1, 2, 4, ... such groups of rows one after another
 * (it fetches its lattice's descriptor once): as many as keep a block at 2048 nodes or fewer and
 * the launch at 8 or more rounds of the blocks the device holds at once. clb_batch_autotune times
 * candidates over the whole batch (the populations are restored afterwards) and keeps the
 * fastest. Results do not depend on it. */
clb_status clb_batch_set_tile(clb_batch *b, int tile_x, int tile_y, int nodes_per_thread);
clb_status clb_batch_autotune(clb_batch *b, int *tile_x, int *tile_y, int *nodes_per_thread);
/* Launch geometry of the next batched step over the active instances: tile shape, groups of rows
 * per block and blocks per launch. Any pointer may be NULL. */
clb_status clb_batch_get_launch(clb_batch *b, int *tile_x, int *tile_y, int *nodes_per_thread,
                                int *groups, long *blocks);

/* ---------------------------------------------------------------------------------------------
 * Serving: requests arrive over time; each is admitted when a slot and enough of the HBM budget
 * are free, stepped together with the other resident requests (one batched launch per step), and
 * retired when E_R < tol or its step cap is reached. Results stay until fetched.
 * clb_serve_open reserves all the device memory the server uses: the whole budget as one pool
 * (a request takes the smallest free block that holds its lattice and gives it back at
 * retirement or cancellation, so fragmentation can delay an admission) and the batched launch's
 * tables at fixed capacities. Submitting, admitting, stepping, retiring and cancelling then
 * allocate no device memory.
 */
typedef struct clb_server clb_server;

clb_status clb_serve_open(size_t hbm_budget_bytes, int max_slots, int storage, void *stream,
                          clb_server **out);
void clb_serve_close(clb_server *s);
/* Queue a request (host initial fields, copied). *req_id receives its id. */
clb_status clb_serve_submit(clb_server *s, int nx, int ny, const clb_params *p, const double *rho,
                            const double *ux, const double *uy, const double *T, int nu_axis,
                            long step_cap, double tol, long *req_id);
/* One scheduling round: admit queued requests that fit, advance every resident request by
 * `chunk` steps, check residuals and retire converged ones. *active / *queued receive counts. */
clb_status clb_serve_progress(clb_server *s, long chunk, int *active, int *queued);
/* Drop a request: queued ones leave the queue, running ones release their slot and memory at
 * once (no work of the server is in flight between calls). Its id becomes unknown. */
clb_status clb_serve_cancel(clb_server *s, long req_id);
/* Non-blocking state of a request: *done = 1 once retired. */
clb_status clb_serve_poll(clb_server *s, long req_id, int *done, double *nu, long *steps,
                          double *er);
/* Fields of a retired request (host arrays, any may be NULL); frees its result. */
clb_status clb_serve_fetch(clb_server *s, long req_id, double *rho, double *ux, double *uy,
                           double *T);

#ifdef __cplusplus
}
#endif

#endif /* CLB_H */
