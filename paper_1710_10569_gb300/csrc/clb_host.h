// clb_host.h -- host-side helpers shared by the libclb translation units: thread-local error
// reporting, parameter validation, and the derivation of the per-lattice device constants
// (relaxation rates from nu and kappa, Sec. 2.1 and Sec. 2.2).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/clb.h"
#include "clb_core.cuh"

namespace clb {

clb_status set_error(clb_status st, const char* fmt, ...);

// An NVTX range over the rest of an entry point (shown by nsys/ncu timelines when a tool is
// attached; a no-op otherwise).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// An entry point's host allocation (a container, a handle) that fails: CLB_ENOMEM instead of an
// exception crossing the C boundary.
inline clb_status host_alloc_failed() { return set_error(CLB_ENOMEM, "host allocation failed"); }
void clear_error();

#define CLB_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return ::clb::set_error(e_ == cudaErrorMemoryAllocation ? CLB_ENOMEM : CLB_ECUDA,   \
                                    "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                                    __LINE__);                                                  \
    } while (0)

#define CLB_TRY(expr)                           \
    do {                                        \
        clb_status s_ = (expr);                 \
        if (s_ != CLB_OK) return s_;            \
    } while (0)

constexpr long long kMaxNodes = 1LL << 30;  // index arithmetic and memory bound
constexpr int kMaxEdge = 1 << 20;

inline size_t elem_size(int storage)
{
    return storage == ST_F64 ? 8 : storage == ST_F32 ? 4 : 2;
}

// Elements per chunked row of a coupled lattice (see chunk_off): ceil(nx / kRowChunk) chunks of
// NPOP * kRowChunk elements.
inline long long chunked_row_elems(int nx)
{
    return (long long)((nx + kRowChunk - 1) / kRowChunk) * NPOP * kRowChunk;
}

// Thermal-only mode (plane-major layout): row pitch in elements, rows on 128-byte boundaries.
inline int row_pitch(int nx, int storage)
{
    const int per = int(128 / elem_size(storage));
    return (nx + per - 1) / per * per;
}

// Thermal-only mode: elements between population planes, planes on 256-byte boundaries.
inline long long plane_elems(int nx, int ny, int storage)
{
    const long long per = 256 / (long long)elem_size(storage);
    const long long e = (long long)row_pitch(nx, storage) * ny;
    return (e + per - 1) / per * per;
}

// Bytes of one population buffer of a coupled lattice (chunked rows; a row is a multiple of
// NPOP * 64 elements, so rows start on 1,792-byte (FP16) or larger boundaries).
inline size_t buffer_bytes(int nx, int ny, int storage)
{
    return (size_t)ny * (size_t)chunked_row_elems(nx) * elem_size(storage);
}

inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Device bytes reserved per population buffer: the buffer plus a 1 KB guard. Every access of the
// kernels lies inside the chunks of the lattice's rows (the vector path covers whole warps inside a
// row, and the 4-byte copy of an edge pair of half-precision values stays inside its chunk); the
// guard is a margin against a change of that.
inline size_t buffer_slot_bytes(int nx, int ny, int storage)
{
    return align256(buffer_bytes(nx, ny, storage)) + 1024;
}

clb_status validate(int nx, int ny, const clb_params* p);

// One step of the staged-rows kernel (k_step_pipe, clb_pipe_*.cu) from buffer a into buffer b:
// V nodes per thread, S stages, R rows per warp; Pd or Pf by the storage form.
cudaError_t enqueue_pipe_any(int storage, const LatParams<double>& Pd, const LatParams<float>& Pf, int device,
                             int nx, int ny, const void* a, void* b, cudaStream_t s, int V, int S, int R);

// s_nu from nu = (1/s_nu - 1/2) c_s^2 with c_s^2 = 1/3 (Sec. 2.1).
inline double rate_nu(double nu) { return 1.0 / (3.0 * nu + 0.5); }
// lambda1 from alpha = (1/lambda1 - 1/2) c_T,s^2 (Sec. 2.2).
inline double rate_kappa(double kappa, double cs2T) { return 1.0 / (kappa / cs2T + 0.5); }

// Device constants of one lattice in arithmetic precision A.
template <typename A>
LatParams<A> make_lat_params(int nx, int ny, const clb_params& p)
{
    LatParams<A> P;
    std::memset(&P, 0, sizeof(P));
    P.nx = nx;
    P.ny = ny;
    P.crow = chunked_row_elems(nx);
    P.pitch = row_pitch(nx, p.storage);
    P.plane = plane_elems(nx, ny, p.storage);
    P.per_x = p.wall[0] == CLB_PERIODIC;
    P.per_y = p.wall[2] == CLB_PERIODIC;
    // Deviation storage is taken against a rest state (w rho0, w^T T_b(y)); FP64 stores populations.
    // Between two Dirichlet (or wet) y walls with periodic x the temperature base is the conduction
    // profile between the walls (walls halfway between nodes: T_b(y) = T_lo + (T_hi - T_lo)
    // (y + 1/2) / ny; wet walls on the end rows: T_lo + (T_hi - T_lo) y / (ny - 1)); otherwise T_ref.
    const bool dev = p.storage != ST_F64;
    const bool ywalls = (p.wall[2] == CLB_WALL_DIRICHLET_T || p.wall[2] == CLB_WALL_WET) &&
                        p.wall[3] == p.wall[2] && p.wall[0] == CLB_PERIODIC;
    double Tb0 = p.T_ref, Tdy = 0.0;
    if (ywalls) {
        const bool wet = p.wall[2] == CLB_WALL_WET;
        Tdy = (p.T_wall[3] - p.T_wall[2]) / (wet ? ny - 1 : ny);
        Tb0 = p.T_wall[2] + (wet ? 0.0 : 0.5 * Tdy);
    }
    if (!dev) Tb0 = Tdy = 0.0;
    P.rho_b = dev ? A(p.rho0) : A(0);
    P.T_b = A(Tb0);
    P.T_dy = A(Tdy);
    P.T_dyw = A(0.5 * p.cs2_T * Tdy);
    // base of the row each side's wall nodes (or wall-adjacent nodes) lie on; x sides only occur
    // with a flat base
    const double side_base[4] = {Tb0, Tb0, Tb0, Tb0 + Tdy * (ny - 1)};
    // Wall terms from the equilibria of the wall state (rho0, u_w) and (T_w, u_w): the moving-wall
    // bounce-back f_i = f*_opp + [f^eq_i - f^eq_opp] and the anti-bounce-back g_i = -g*_opp +
    // [g^eq_i + g^eq_opp] = -g*_opp + T_w (cs2_T + u_w,axis^2) for the pair i/opp along the wall's
    // normal (Eqs. 9 and 20 back-transformed: f^eq_i = rho p(e_x; u_x) p(e_y; u_y) with the 1-D
    // equilibrium p(0; u) = 2/3 - u^2, p(+-1; u) = (1/3 + u^2 +- u)/2).
    auto p1 = [](int e, double u) { return e == 0 ? 2.0 / 3.0 - u * u : 0.5 * (1.0 / 3.0 + u * u + e * u); };
    const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    P.moving = 0;
    for (int s = 0; s < 4; ++s) {
        P.kind[s] = p.wall[s];
        const double ux = p.u_wall[s][0], uy = p.u_wall[s][1];
        const double un = s < 2 ? ux : uy;
        P.Tw_c2[s] = A(p.T_wall[s] * (p.cs2_T + un * un) - p.cs2_T * side_base[s]);
        P.dTw[s] = A(p.T_wall[s] - side_base[s]);
        for (int i = 0; i < 9; ++i)
            P.fbb[s][i] = A(p.rho0 * (p1(ex[i], ux) * p1(ey[i], uy) - p1(-ex[i], ux) * p1(-ey[i], uy)));
        if (p.wall[s] != CLB_PERIODIC && p.wall[s] != CLB_WALL_WET && (ux != 0.0 || uy != 0.0)) P.moving = 1;
        P.Twall[s] = A(p.T_wall[s]);
        P.uwall[s][0] = A(ux);
        P.uwall[s][1] = A(uy);
    }
    P.wet_x = p.wall[0] == CLB_WALL_WET;
    P.wet_y = p.wall[2] == CLB_WALL_WET;
    const double s_nu = rate_nu(p.nu);
    P.s_nu = A(s_nu);
    P.sp = A(0.5 * (p.s_b + s_nu));
    P.sm = A(0.5 * (p.s_b - s_nu));
    P.s_3 = A(p.s_3);
    P.s_4 = A(p.s_4);
    P.lambda1 = A(rate_kappa(p.kappa, p.cs2_T));
    P.lambda2 = A(p.lambda2);
    P.cs2T = A(p.cs2_T);
    P.Fvx = A(p.Fv[0]);
    P.Fvy = A(p.Fv[1]);
    P.gb = A(p.rho0 * p.g_beta);
    P.T0 = A(p.T0);
    return P;
}

// Nusselt geometry of Eq. (29) for one axis: H, dT and the sign making heat flow from the hot
// side positive.
struct NuGeom {
    double H, dT, sign, cells;
};
inline NuGeom nu_geom(int nx, int ny, const clb_params& p, int axis)
{
    const int lo = axis == 0 ? 0 : 2, hi = lo + 1;
    NuGeom g;
    // wet walls lie on the end rows (columns) of nodes: one interval fewer along a wet direction,
    // and the trapezoid weights of the average sum to it
    const int Lx = p.wall[0] == CLB_WALL_WET ? nx - 1 : nx;
    const int Ly = p.wall[2] == CLB_WALL_WET ? ny - 1 : ny;
    g.H = axis == 0 ? Lx : Ly;
    g.cells = double(Lx) * Ly;
    const double d = std::fabs(p.T_wall[lo] - p.T_wall[hi]);
    g.dT = d > 0 ? d : 1.0;
    g.sign = p.T_wall[lo] >= p.T_wall[hi] ? 1.0 : -1.0;
    return g;
}

// Reduction partial sums of one row (or block), in this order.
enum { RS_UT = 0, RS_DU, RS_U, RS_DT, RS_T, RS_BAD, RS_N };

// Final scalars from the summed partials (host or device).
__host__ __device__ inline void finish_diagnostics(const double* s, double nodes, double cells,
                                                   double H, double dT, double sign, double kappa,
                                                   double u_ref, double dT_ref, double* nu,
                                                   double* er)
{
    *nu = 1.0 + sign * (s[RS_UT] / cells) * H / (kappa * dT);
    const double fu = nodes * (1e-3 * u_ref) * (1e-3 * u_ref);
    const double fT = nodes * (1e-3 * dT_ref) * (1e-3 * dT_ref);
    const double du = s[RS_U] > fu ? s[RS_U] : fu;
    const double dt = s[RS_T] > fT ? s[RS_T] : fT;
    const double ru = s[RS_DU] == 0.0 ? 0.0 : (du > 0 ? sqrt(s[RS_DU] / du) : INFINITY);
    const double rt = s[RS_DT] == 0.0 ? 0.0 : (dt > 0 ? sqrt(s[RS_DT] / dt) : INFINITY);
    *er = ru > rt ? ru : rt;
}

}  // namespace clb
