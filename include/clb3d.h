/*
 * clb3d.h -- C ABI of the three-dimensional form of the coupled central-moment lattice Boltzmann
 * method (Fei, Luo, Lin & Li, arXiv:1710.10569): D3Q27 flow populations and D3Q7 temperature
 * populations, stepped by one fused collide-and-stream kernel on the GPU.
 *
 * The paper states the method in two dimensions (D2Q9 flow, Sec. 2.1, Eqs. 4-13; D2Q5 temperature,
 * Sec. 2.2, Eqs. 14-23) and says it extends to three dimensions directly (Sec. 4). This library
 * applies the same definitions on the 3-D lattices:
 *   - central moments k~_abc = sum_i (e_x-u_x)^a (e_y-u_y)^b (e_z-u_z)^c f_i, a, b, c in {0,1,2}
 *     (Eq. 5 on D3Q27);
 *   - equilibrium central moments rho m(a) m(b) m(c) with m(0) = 1, m(1) = 0, m(2) = 1/3 (Eq. 9);
 *   - forcing moments F_d prod_{d' != d} m(a_d') where exactly one index a_d is 1 (Eq. 11);
 *   - relaxation Gamma~* = Gamma~ - S (Gamma~ - Gamma~eq) + (I - S/2) C (Eq. 8): the trace of the
 *     three normal second moments with s_b, their deviators and the off-diagonal second moments
 *     with s_nu (nu = (1/s_nu - 1/2)/3), third- to sixth-order moments with s_3 .. s_6;
 *   - D3Q7 moments 1, e_d, e_d^2, equilibrium (T, 0, 0, 0, cs2_T T x3), rates
 *     (lambda0, lambda1 x3, lambda2 x3) with alpha = (1/lambda1 - 1/2) cs2_T (Eqs. 16-21);
 *   - Boussinesq force F = Fv + rho0 g_beta (T - T0) along +g_axis (Eq. 3), u = (sum f e + F/2)/rho
 *     (Eq. 13), T = sum g (Eq. 23);
 *   - walls halfway between nodes on any face: f bounces back, g anti-bounces back
 *     (g_i = -g*_opp + cs2_T T_w) on Dirichlet faces and bounces back on adiabatic faces; wall
 *     faces may move (tangential motion and normal injection), with the wall's equilibrium added
 *     as in the 2-D moving-wall rule.
 *
 * Status codes, clb_last_error() and the storage forms are those of clb.h.
 *
 * Layout. Fields passed in and out are FP64 host arrays of nz * ny * nx values, x fastest
 * (index (z * ny + y) * nx + x). Population arrays are [27][nz][ny][nx] and [7][nz][ny][nx]:
 * D3Q27 population i = a + 3 b + 9 c has velocity (v(a), v(b), v(c)) with v(0) = 0, v(1) = +1,
 * v(2) = -1; D3Q7 populations are ordered rest, +x, -x, +y, -y, +z, -z.
 *
 * Ownership. clb3d_create allocates the lattice's device memory (two population buffers of 34
 * planes, FP64 staging for the fields, the residual's FP64 snapshot and the reduction partials) and
 * owns it until
 * clb3d_destroy. All work is enqueued on the stream given at creation (NULL: the legacy default
 * stream); functions that return host data synchronise that stream.
 */
#ifndef CLB3D_H
#define CLB3D_H

#include <stddef.h>

#include "clb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct clb3d_lattice clb3d_lattice;

typedef struct {
    double nu;        /* kinematic viscosity, > 0 (gives s_nu; 0 < s_nu < 2) */
    double kappa;     /* thermal diffusivity, > 0 (gives lambda1; 0 < lambda1 < 2) */
    double g_beta;    /* |g| beta >= 0 */
    double T0;        /* reference temperature of the Boussinesq force */
    double rho0;      /* reference density (force, and the rest state of deviation storage) */
    double s_b, s_3, s_4, s_5, s_6; /* rates of the bulk, 3rd-, 4th-, 5th- and 6th-order moments, in (0, 2) */
    double lambda2;   /* rate of the second-order D3Q7 moments, in (0, 2) */
    double cs2_T;     /* D3Q7 sound speed squared, in (0, 1/3) */
    double Fv[3];     /* body force density */
    int g_axis;       /* buoyancy along +g_axis: 0, 1 or 2 */
    int wall[6];      /* clb_wall of faces -x, +x, -y, +y, -z, +z: periodic faces come in pairs;
                         CLB_WALL_WET is not supported in 3-D */
    double T_wall[6]; /* temperature of Dirichlet faces */
    int storage;      /* clb_storage: CLB_F64, CLB_F32 or CLB_F16DEV (FP32 or FP16 deviations from the rest
                         state; FP32 arithmetic for both) */
    double T_ref;     /* rest temperature of deviation storage */
    double u_wall[6][3]; /* velocity of each wall face, |component| <= 0.4 (ignored on periodic faces):
                            f_i = f*_opp + [f^eq_i - f^eq_opp](rho0, u_w) across the face and, on a
                            Dirichlet face, g_i = -g*_opp + T_w (cs2_T + u_wn^2); a link across an
                            edge or corner takes the velocity of the face of the highest axis */
    double u_ref;     /* velocity scale of the residual's floor (0: no floor) */
    double dT_ref;    /* temperature scale of the residual's floor (0: no floor) */
} clb3d_params;

/* Defaults: nu = kappa = 0.02, rho0 = 1, all rates 1, cs2_T = 1/4, g_axis = 2, periodic, FP64. */
clb_status clb3d_params_default(clb3d_params* p);

/* Device bytes clb3d_create will allocate for an nx x ny x nz lattice. */
clb_status clb3d_footprint(int nx, int ny, int nz, const clb3d_params* p, size_t* bytes);

/* Create a lattice (1 <= n <= 2^20 per axis, nx * ny * nz <= 2^30). Errors: CLB_EINVAL for bad sizes
 * or parameters, CLB_ENOMEM, CLB_ECUDA. The populations are undefined until clb3d_init_fields. */
clb_status clb3d_create(int nx, int ny, int nz, const clb3d_params* p, void* stream, clb3d_lattice** out);
void clb3d_destroy(clb3d_lattice* h);

/* f = f^eq(rho, u), g = g^eq(T, u) at every node from host fields (nz*ny*nx each); also takes the
 * residual's first snapshot. Synchronises. CLB_ENAN if a resulting field is not finite (the state
 * is set all the same). */
clb_status clb3d_init_fields(clb3d_lattice* h, const double* rho, const double* ux, const double* uy,
                             const double* uz, const double* T);

/* n >= 0 time steps (collision, then pull streaming with the face rules), enqueued on the stream;
 * returns after enqueueing. */
clb_status clb3d_step(clb3d_lattice* h, long n);

/* rho, u, T of the current (pre-collision) state into host arrays; synchronises. */
clb_status clb3d_fields(clb3d_lattice* h, double* rho, double* ux, double* uy, double* uz, double* T);

/* The current pre-collision populations, as FP64 populations (not deviations), into host arrays
 * f[27 * n], g[7 * n]; synchronises. */
clb_status clb3d_populations(clb3d_lattice* h, double* f, double* g);

/* Nusselt number along `axis` (Eq. 29 with H the node count of that axis): 1 + <u_axis (T - T0)>
 * H / (kappa dT), dT the difference of that axis's wall temperatures (1 if equal), heat from the
 * hot face counted positive. FP64 sums in a fixed order. CLB_ENAN if a field is not finite. */
clb_status clb3d_nusselt(clb3d_lattice* h, int axis, double* nu_out);

/* Steady-state residual since the previous call (or since clb3d_init_fields), the 2-D form's E_R
 * with u a 3-vector: max over X in {u, T} of sqrt(sum |X(t) - X(t')|^2 / max(sum |X(t)|^2,
 * N (1e-3 X_ref)^2)), X_ref = u_ref, dT_ref; FP64 sums in a fixed order over an FP64 snapshot of
 * u and T that the call then replaces. Synchronises; CLB_ENAN if a field is not finite. */
clb_status clb3d_residual(clb3d_lattice* h, double* er_out);

/* Step in chunks of `interval` until clb3d_residual < tol after a chunk or max_steps steps are
 * done; the steps taken and the last residual are returned. */
clb_status clb3d_run(clb3d_lattice* h, double tol, long max_steps, long interval, long* steps_out,
                     double* er_out);

/* Checkpoint: the current post-collision buffer as stored (populations or deviations) and the step
 * count, after a small header. With buf == NULL, *bytes receives the size; otherwise *bytes is the
 * buffer's capacity on entry and the bytes written on return. clb3d_load restores a checkpoint of a
 * lattice with the same extents and storage (CLB_EINVAL otherwise) and restarts the residual's
 * snapshot from the restored state. Both synchronise. */
clb_status clb3d_save(clb3d_lattice* h, void* buf, size_t* bytes);
clb_status clb3d_load(clb3d_lattice* h, const void* buf, size_t bytes);

/* Launch shape of the step kernel: block_x threads along x (a multiple of 32, <= 256) times block_y
 * rows (block_x * block_y <= 256). 0 keeps a value. */
clb_status clb3d_set_launch(clb3d_lattice* h, int block_x, int block_y);

clb_status clb3d_sync(clb3d_lattice* h);

/* The stream the lattice works on, and the device address of the buffer holding the current
 * post-collision state with its plane stride in elements (for device-side consumers). */
void* clb3d_stream(clb3d_lattice* h);
clb_status clb3d_buffers(clb3d_lattice* h, void** current, long long* plane_elems, int* row_pitch);

/* Batches: n independent lattices of different extents and parameters (all with the same storage)
 * stepped together by one launch per time step over their concatenated tiles (replayed from CUDA
 * graphs), each lattice computing exactly what it computes alone (bitwise the same). The paper
 * has no counterpart; this is the 3-D form of the clb_batch_* interface of clb.h.
 * Every lattice is an ordinary clb3d_lattice owned by the batch: clb3d_batch_lattice gives its
 * handle for clb3d_fields, clb3d_populations, clb3d_nusselt, clb3d_residual and clb3d_save; its
 * state changes only through clb3d_batch_init_fields and clb3d_batch_step (stepping, initialising
 * or loading it through its own handle breaks the batch's bookkeeping of which buffer is current).
 * Device memory: each lattice's own (clb3d_footprint), two small tables, and the graphs. */
typedef struct clb3d_batch clb3d_batch;
/* n >= 1 lattices nx[k] x ny[k] x nz[k] with parameters p[k]; CLB_EINVAL if any lattice is invalid
 * or the storages differ. The populations are undefined until clb3d_batch_init_fields. */
clb_status clb3d_batch_create(int n, const int* nx, const int* ny, const int* nz, const clb3d_params* p,
                              void* stream, clb3d_batch** out);
void clb3d_batch_destroy(clb3d_batch* b);
/* The handle of lattice k (0 <= k < n), owned by the batch. */
clb_status clb3d_batch_lattice(clb3d_batch* b, int k, clb3d_lattice** out);
/* clb3d_init_fields for lattice k (steps since init restart at 0); synchronises. */
clb_status clb3d_batch_init_fields(clb3d_batch* b, int k, const double* rho, const double* ux,
                                   const double* uy, const double* uz, const double* T);
/* n >= 0 time steps of every lattice, enqueued on the stream. */
clb_status clb3d_batch_step(clb3d_batch* b, long n);
/* Thread block of the batched step: block_x threads along x (a multiple of 32, <= 256) times block_y
 * rows (block_x * block_y <= 256). Each block steps 1, 2, 4, ... groups of block_y rows one after
 * another: as many as keep a block at 2048 nodes or fewer and the launch at 8 or more rounds of the
 * blocks the device holds at once. Results do not depend on it. */
clb_status clb3d_batch_set_tile(clb3d_batch* b, int block_x, int block_y);
/* The thread block, groups of rows per block and blocks per launch of the batched step. */
clb_status clb3d_batch_get_launch(clb3d_batch* b, int* block_x, int* block_y, int* groups,
                                  long long* blocks);

/* Thermal-only mode: the D3Q7 equation alone with a prescribed velocity field (the 3-D form of
 * the paper's Sec. 3.1 set-up, where only the temperature equation is solved for a given flow).
 * The same pull, face rules, collision and equilibrium as the coupled step's D3Q7 part; the flow
 * parameters of clb3d_params are not used (they are still validated). Device memory: two buffers
 * of 7 planes, the velocity (3 values per node in the arithmetic precision) and FP64 staging. */
typedef struct clb3d_thermal clb3d_thermal;
clb_status clb3d_thermal_create(int nx, int ny, int nz, const clb3d_params* p, void* stream,
                                clb3d_thermal** out);
void clb3d_thermal_destroy(clb3d_thermal* h);
/* g = g^eq(T, u) and the prescribed velocity u from host fields (nz*ny*nx each); synchronises. */
clb_status clb3d_thermal_init(clb3d_thermal* h, const double* T, const double* ux, const double* uy,
                              const double* uz);
clb_status clb3d_thermal_step(clb3d_thermal* h, long n);
/* T of the current state into a host array; synchronises. */
clb_status clb3d_thermal_fields(clb3d_thermal* h, double* T);
/* The current pre-collision D3Q7 populations (FP64, not deviations), [7][nz][ny][nx]; synchronises. */
clb_status clb3d_thermal_populations(clb3d_thermal* h, double* g);
clb_status clb3d_thermal_sync(clb3d_thermal* h);

#ifdef __cplusplus
}
#endif

#endif
