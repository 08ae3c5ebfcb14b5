// clb3d.cu -- the three-dimensional form of the coupled central-moment LBM (include/clb3d.h):
// D3Q27 flow populations and D3Q7 temperature populations, one fused collide-and-stream kernel per
// time step, CUDA graphs of 32 steps, FP64 field extraction and Nusselt reduction.
//
// Per node the collision runs the moment transforms in factorised form. The raw-moment map of
// D3Q27 (moments e_x^a e_y^b e_z^c, a, b, c <= 2) is the tensor product of the 1-D map
// (f_0, f_+, f_-) -> (f_0 + f_+ + f_-, f_+ - f_-, f_+ + f_-) over the three axes, and the central
// shift N(u) of Eq. (5) is the tensor product of the 1-D shifts (r_0, r_1, r_2) -> (r_0,
// r_1 - u r_0, r_2 - 2 u r_1 + u^2 r_0). So the 27 central moments take three passes of nine
// three-point maps for the raw moments (which also give rho and the momentum of Eq. 13) and three
// passes of nine shifts; the back transform of the relaxed moments runs the inverse 1-D maps
// (uncentral3). About 330 flops for the transforms instead of the ~3,000 of literal 27 x 27
// products.
//
// Storage. FP64 buffers hold the populations. FP32 and FP16 buffers hold deviations from the rest
// state, h_i = f_i - w_i rho0 and t_i = g_i - w^T_i T_ref (w_i = w(a) w(b) w(c), w(0) = 2/3,
// w(+-1) = 1/6), and both compute in FP32.
// The central moments of w_i rho0 about u are rho0 R(a) R(b) R(c) with R = (1, -u, 1/3 + u^2), so
// the collision of Eq. (8) on deviations is k* = k - S (k + E) + (I - S/2) C with
// E = rho0 (R R R - m m m) - (rho - rho0) m m m, m = (1, 0, 1/3); E is formed from per-axis
// differences R - m = (0, -u, u^2) without cancellation. With rho0 = T_ref = 0 the same code is the
// FP64 collision on the populations themselves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>
#include <cstddef>

#include "../../include/clb3d.h"
#include "clb_core.cuh"
#include "clb_host.h"

namespace clb3 {

using namespace clb;

constexpr int NF = 27, NG = 7, NP = NF + NG;
constexpr int kChunk = 32;  // steps per captured graph (even: the buffers return to their roles)
constexpr int kRedThreads = 256;

template <typename A>
struct Lat3 {
    int nx, ny, nz, pitch;
    long long plane;       // elements between planes (< 2^31: 32-bit offsets within a plane)
    int per[3];            // periodic flag per axis
    int kind[6];           // clb_wall per face -x, +x, -y, +y, -z, +z
    A Tw[6];               // anti-bounce-back constant of a Dirichlet face: T_w (cs2_T + u_wn^2) - cs2_T T_b
    int moving;            // some wall face moves: fbb holds its momentum terms
    A fbb[6][27];          // [f^eq_i - f^eq_opp](rho0, u_w) of each face, added on bounce-back
    A s_nu, s_b3, s_3, s_4, s_5, s_6;  // s_b3 = (s_b - s_nu) / 3
    A lambda1, lambda2, cs2T;
    A Fv[3];
    int g_axis;
    A gb, T0;              // buoyancy rho0 g_beta (T - T0) along +g_axis
    A rho_b, T_b;          // rest state of the stored deviations (0 for FP64)
};

__host__ __device__ constexpr int oppd(int d) { return d == 0 ? 0 : 3 - d; }
__host__ __device__ constexpr int vel(int d) { return d == 0 ? 0 : (d == 1 ? 1 : -1); }

// 1-D raw moments (order 0, 1, 2) of (centre, e = +1, e = -1), in place.
template <typename A>
__device__ __forceinline__ void raw3(A& c, A& p, A& m)
{
    const A s = p + m, d = p - m;
    c = c + s;
    p = d;
    m = s;
}

// 1-D shift of raw moments (r0, r1, r2) to central moments about u, in place.
template <typename A>
__device__ __forceinline__ void shift3(A r0, A& r1, A& r2, A u)
{
    r2 = fma_(u * u, r0, fma_(A(-2) * u, r1, r2));
    r1 = fma_(-u, r0, r1);
}

// Moment index k = a + 3 b + 9 c (orders along x, y, z); population index alike with digits.
#define CLB3_LINE_X(b, c) (3 * (b) + 9 * (c))
#define CLB3_LINE_Y(a, c) ((a) + 9 * (c))
#define CLB3_LINE_Z(a, b) ((a) + 3 * (b))

template <typename A>
__device__ __forceinline__ void raw_moments27(A k[NF])
{
#pragma unroll
    for (int t = 0; t < 9; ++t) {  // x lines: (b, c) = (t % 3, t / 3)
        const int o = CLB3_LINE_X(t % 3, t / 3);
        raw3(k[o], k[o + 1], k[o + 2]);
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {  // y lines: (a, c)
        const int o = CLB3_LINE_Y(t % 3, t / 3);
        raw3(k[o], k[o + 3], k[o + 6]);
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {  // z lines: (a, b)
        const int o = CLB3_LINE_Z(t % 3, t / 3);
        raw3(k[o], k[o + 9], k[o + 18]);
    }
}

template <typename A>
__device__ __forceinline__ void central_shift27(A k[NF], A ux, A uy, A uz)
{
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int o = CLB3_LINE_X(t % 3, t / 3);
        shift3(k[o], k[o + 1], k[o + 2], ux);
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int o = CLB3_LINE_Y(t % 3, t / 3);
        shift3(k[o], k[o + 3], k[o + 6], uy);
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int o = CLB3_LINE_Z(t % 3, t / 3);
        shift3(k[o], k[o + 9], k[o + 18], uz);
    }
}

// Populations from central moments about u: the inverse 1-D maps along z, y, x.
template <typename A>
__device__ __forceinline__ void back27(A k[NF], A ux, A uy, A uz)
{
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int o = CLB3_LINE_Z(t % 3, t / 3);
        uncentral3(k[o], k[o + 9], k[o + 18], uz, k[o], k[o + 9], k[o + 18]);
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int o = CLB3_LINE_Y(t % 3, t / 3);
        uncentral3(k[o], k[o + 3], k[o + 6], uy, k[o], k[o + 3], k[o + 6]);
    }
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int o = CLB3_LINE_X(t % 3, t / 3);
        uncentral3(k[o], k[o + 1], k[o + 2], ux, k[o], k[o + 1], k[o + 2]);
    }
}

// Per-axis factors for moment order a: R = central moment of the 1-D rest weights about u,
// m = lattice Maxwellian moment, dl = R - m.
template <typename A>
struct Axis {
    A R[3], m[3], dl[3];
    __device__ __forceinline__ Axis(A u, A cs2)
    {
        const A u2 = u * u;
        R[0] = A(1); R[1] = -u; R[2] = cs2 + u2;
        m[0] = A(1); m[1] = A(0); m[2] = cs2;
        dl[0] = A(0); dl[1] = -u; dl[2] = u2;
    }
};

// E_k of the deviation collision: rho_b (R R R - m m m) - drho m m m. Populations stored as
// themselves (DEV = false, rho_b = 0) need only the last term, which is what the full expression
// evaluates to there (fma(0, d, t) = t). A moment with an order 1 along some axis has no
// Maxwellian part (m(1) = 0): there E is rho_b R R R, a product without cancellation, and zero for
// populations stored as themselves.
template <bool DEV, typename A>
__device__ __forceinline__ A e_term(const Axis<A>& X, const Axis<A>& Y, const Axis<A>& Z, int a, int b,
                                    int c, A rho_b, A drho)
{
    if (a == 1 || b == 1 || c == 1) {
        if constexpr (!DEV) return A(0);
        return rho_b * (X.R[a] * (Y.R[b] * Z.R[c]));
    }
    const A t = -drho * (X.m[a] * Y.m[b] * Z.m[c]);
    if constexpr (!DEV) return t;
    const A d = X.dl[a] * Y.R[b] * Z.R[c] + X.m[a] * (Y.dl[b] * Z.R[c] + Y.m[b] * Z.dl[c]);
    return fma_(rho_b, d, t);
}

// Forcing moment C_k (Eq. 11 on D3Q27): F_d times the Maxwellian moments of the other axes where
// exactly one order is 1.
template <typename A>
__device__ __forceinline__ A c_term(const Axis<A>& X, const Axis<A>& Y, const Axis<A>& Z, int a, int b,
                                    int c, const A F[3])
{
    A v = A(0);
    if (a == 1 && b != 1 && c != 1) v = F[0] * (Y.m[b] * Z.m[c]);
    if (b == 1 && a != 1 && c != 1) v = F[1] * (X.m[a] * Z.m[c]);
    if (c == 1 && a != 1 && b != 1) v = F[2] * (X.m[a] * Y.m[b]);
    return v;
}

template <bool DEV, typename A>
__device__ __forceinline__ void collide_d3q7(const Lat3<A>& P, const A u[3], A dT, A g[NG]);

// One node: Eqs. (3), (13), (23), then the D3Q27 collision (Eq. 8 in 3-D) and the D3Q7 collision
// (Eq. 19 in 3-D), on the stored form (deviations for FP32, populations for FP64). f and g are
// pre-collision on entry and post-collision on return. HIGH1 = true is for s_3 = s_4 = s_5 = s_6 = 1
// (the paper's setting of the high-order rates): there every moment of order 3 or more relaxes to
// its equilibrium plus half its forcing term, k* = -E + C/2, whatever its pre-collision value, so
// those moments need not be formed at all.
template <bool DEV, bool HIGH1 = false, typename A>
__device__ __forceinline__ void collide3(const Lat3<A>& P, A f[NF], A g[NG])
{
    const A cs2 = A(1.0 / 3.0);
    raw_moments27(f);
    const A drho = f[0];
    const A dT = (g[0] + (g[1] + g[2])) + ((g[3] + g[4]) + (g[5] + g[6]));
    const A rho = P.rho_b + drho;
    const A T = P.T_b + dT;
    const A buoy = P.gb * (T - P.T0);
    A F[3];
    F[0] = P.g_axis == 0 ? P.Fv[0] + buoy : P.Fv[0];
    F[1] = P.g_axis == 1 ? P.Fv[1] + buoy : P.Fv[1];
    F[2] = P.g_axis == 2 ? P.Fv[2] + buoy : P.Fv[2];
    const A inv = rcp_(rho);
    const A ux = fma_(A(0.5), F[0], f[1]) * inv;
    const A uy = fma_(A(0.5), F[1], f[3]) * inv;
    const A uz = fma_(A(0.5), F[2], f[9]) * inv;
    central_shift27(f, ux, uy, uz);

    const Axis<A> X(ux, cs2), Y(uy, cs2), Z(uz, cs2);
    // normal second moments: trace with s_b, deviators with s_nu
    const A Xx = f[2] + e_term<DEV>(X, Y, Z, 2, 0, 0, P.rho_b, drho);
    const A Xy = f[6] + e_term<DEV>(X, Y, Z, 0, 2, 0, P.rho_b, drho);
    const A Xz = f[18] + e_term<DEV>(X, Y, Z, 0, 0, 2, P.rho_b, drho);
    const A tr = P.s_b3 * ((Xx + Xy) + Xz);
    f[2] = f[2] - fma_(P.s_nu, Xx, tr);
    f[6] = f[6] - fma_(P.s_nu, Xy, tr);
    f[18] = f[18] - fma_(P.s_nu, Xz, tr);
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        const int a = k % 3, b = (k / 3) % 3, c = k / 9, o = a + b + c;
        if (o == 0 || k == 2 || k == 6 || k == 18) continue;
        if (o == 1) {
            f[k] = f[k] + (a == 1 ? F[0] : b == 1 ? F[1] : F[2]);
            continue;
        }
        const bool forced = ((a == 1) + (b == 1) + (c == 1)) == 1;  // C_k can be non-zero
        if (HIGH1 && o >= 3) {
            const A E = e_term<DEV>(X, Y, Z, a, b, c, P.rho_b, drho);
            f[k] = forced ? fma_(A(0.5), c_term(X, Y, Z, a, b, c, F), -E) : -E;
            continue;
        }
        const A s = o == 2 ? P.s_nu : o == 3 ? P.s_3 : o == 4 ? P.s_4 : o == 5 ? P.s_5 : P.s_6;
        const A x = f[k] + e_term<DEV>(X, Y, Z, a, b, c, P.rho_b, drho);
        const A cf = c_term(X, Y, Z, a, b, c, F);
        f[k] = forced ? fma_(fma_(A(-0.5), s, A(1)), cf, fma_(-s, x, f[k])) : fma_(-s, x, f[k]);
    }
    back27(f, ux, uy, uz);

    const A u[3] = {ux, uy, uz};
    collide_d3q7<DEV>(P, u, dT, g);
}

// D3Q7 collision (Eqs. 16-21 in 3-D) on the stored form with velocity u; dT = sum of the stored
// values (T - T_b). Central moments about u, relaxation, back transform.
template <bool DEV, typename A>
__device__ __forceinline__ void collide_d3q7(const Lat3<A>& P, const A u[3], A dT, A g[NG])
{
    A kd[3], kdd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const A p = g[1 + 2 * d], m = g[2 + 2 * d];
        const A r1 = p - m, r2 = p + m;
        kd[d] = fma_(-u[d], dT, r1);
        kdd[d] = fma_(u[d] * u[d], dT, fma_(A(-2) * u[d], r1, r2));
        // relax: first order towards 0 (deviation term -T_b u), second towards cs2_T T
        const A e1 = DEV ? -P.T_b * u[d] : A(0);
        const A e2 = DEV ? fma_(P.T_b, u[d] * u[d], -P.cs2T * dT) : -P.cs2T * dT;
        kd[d] = fma_(-P.lambda1, DEV ? kd[d] + e1 : kd[d], kd[d]);
        kdd[d] = fma_(-P.lambda2, kdd[d] + e2, kdd[d]);
    }
    A rest = dT;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const A r1 = fma_(u[d], dT, kd[d]);
        const A r2 = fma_(u[d] * u[d], dT, fma_(A(2) * u[d], kd[d], kdd[d]));
        rest = rest - r2;
        half_sum_diff(r2, r1, g[1 + 2 * d], g[2 + 2 * d]);
    }
    g[0] = rest;
}

template <typename A>
__device__ __forceinline__ void equilibrium_d3q7(const Lat3<A>& P, const A u[3], A dT, A g[NG]);

// Equilibrium of one node on the stored form: the back transform of the equilibrium central
// moments minus those of the rest state (-E for D3Q27; (dT, T_b u, cs2_T dT - T_b u^2) for D3Q7).
template <bool DEV, typename A>
__device__ __forceinline__ void equilibrium3(const Lat3<A>& P, A drho, A ux, A uy, A uz, A dT, A f[NF],
                                             A g[NG])
{
    const A cs2 = A(1.0 / 3.0);
    const Axis<A> X(ux, cs2), Y(uy, cs2), Z(uz, cs2);
#pragma unroll
    for (int k = 0; k < NF; ++k) f[k] = -e_term<DEV>(X, Y, Z, k % 3, (k / 3) % 3, k / 9, P.rho_b, drho);
    back27(f, ux, uy, uz);
    const A u[3] = {ux, uy, uz};
    equilibrium_d3q7(P, u, dT, g);
}

// D3Q7 equilibrium on the stored form: the back transform of (dT, T_b u, cs2_T dT - T_b u^2).
template <typename A>
__device__ __forceinline__ void equilibrium_d3q7(const Lat3<A>& P, const A u[3], A dT, A g[NG])
{
    A rest = dT;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const A kd = P.T_b * u[d];
        const A kdd = fma_(P.cs2T, dT, -P.T_b * (u[d] * u[d]));
        const A r1 = fma_(u[d], dT, kd);
        const A r2 = fma_(u[d] * u[d], dT, fma_(A(2) * u[d], kd, kdd));
        rest = rest - r2;
        half_sum_diff(r2, r1, g[1 + 2 * d], g[2 + 2 * d]);
    }
    g[0] = rest;
}

// Source coordinate of the pull along one axis per velocity digit (0: stay, 1: from c - 1,
// 2: from c + 1) and whether it exists (false: the pull crosses a wall).
struct Src {
    int s[3];
    bool ok[3];
    __device__ __forceinline__ Src(int c, int n, int per)
    {
        s[0] = c;
        ok[0] = true;
        ok[1] = c > 0 || per;
        s[1] = c > 0 ? c - 1 : (per ? n - 1 : c);
        ok[2] = c < n - 1 || per;
        s[2] = c < n - 1 ? c + 1 : (per ? 0 : c);
    }
};

// Pull of Eq. (22) for the D3Q7 populations held in planes base .. base + 6 of the buffer.
template <bool NOWALL = false, typename T, typename A>
__device__ __forceinline__ void gather_d3q7(const T* __restrict__ src, const Lat3<A>& P, int x, int y, int z,
                                            int base, A g[NG])
{
    const Src sx(x, P.nx, P.per[0]), sy(y, P.ny, P.per[1]), sz(z, P.nz, P.per[2]);
    const int pl = (int)P.plane;
    const int here = (z * P.ny + y) * P.pitch + x;
    g[0] = to_a(src[base * pl + here]);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int j = 1 + 2 * d + s, jo = 1 + 2 * d + (1 - s);
            const Src& S = d == 0 ? sx : (d == 1 ? sy : sz);
            const int digit = 1 + s;
            const int at = d == 0 ? (z * P.ny + y) * P.pitch + S.s[digit]
                         : d == 1 ? (z * P.ny + S.s[digit]) * P.pitch + x
                                  : (S.s[digit] * P.ny + y) * P.pitch + x;
            if (NOWALL || S.ok[digit]) {
                g[j] = to_a(src[(base + j) * pl + at]);
            } else {
                const int face = 2 * d + s;
                const A bb = to_a(src[(base + jo) * pl + here]);
                g[j] = P.kind[face] == CLB_WALL_DIRICHLET_T ? P.Tw[face] - bb : bb;
            }
        }
}

// Pull of Eqs. (12), (22): population i at the node comes from the node at x - e_i; across a
// wall face f takes the node's own opposite post-collision value, and g the anti-bounce-back
// value on Dirichlet faces. NOWALL = true is for nodes none of whose pulls crosses a wall (every
// source exists, periodic wrap included): the same loads without the wall selects.
template <bool NOWALL = false, typename T, typename A>
__device__ __forceinline__ void gather3(const T* __restrict__ src, const Lat3<A>& P, int x, int y, int z,
                                        A f[NF], A g[NG])
{
    const Src sx(x, P.nx, P.per[0]), sy(y, P.ny, P.per[1]), sz(z, P.nz, P.per[2]);
    const int pl = (int)P.plane;
    const int here = (z * P.ny + y) * P.pitch + x;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int row = (sz.s[c] * P.ny + sy.s[b]) * P.pitch;
            const bool okyz = sy.ok[b] && sz.ok[c];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int i = a + 3 * b + 9 * c;
                const int o = oppd(a) + 3 * oppd(b) + 9 * oppd(c);
                const bool ok = NOWALL || (okyz && sx.ok[a]);
                const int off = ok ? i * pl + row + sx.s[a] : o * pl + here;
                f[i] = to_a(src[off]);
                if (!NOWALL && !ok && P.moving) {
                    // the face crossed; of several (edge, corner), that of the highest axis
                    const int face = !sz.ok[c] ? (c == 1 ? 4 : 5) : !sy.ok[b] ? (b == 1 ? 2 : 3) : (a == 1 ? 0 : 1);
                    f[i] = f[i] + P.fbb[face][i];
                }
            }
        }
    gather_d3q7<NOWALL>(src, P, x, y, z, NF, g);
}

template <typename T, typename A>
__device__ __forceinline__ void store3(T* __restrict__ dst, const Lat3<A>& P, int here, const A f[NF],
                                       const A g[NG])
{
    const int pl = (int)P.plane;
#pragma unroll
    for (int i = 0; i < NF; ++i) dst[i * pl + here] = from_a(f[i], (T*)nullptr);
#pragma unroll
    for (int j = 0; j < NG; ++j) dst[(NF + j) * pl + here] = from_a(g[j], (T*)nullptr);
}

// One node's time step: pull (with the face rules where the node touches a wall face), collision,
// store into the other buffer.
template <int ST, bool HIGH1, typename A>
__device__ __forceinline__ void step3_node(const typename Storage<ST>::T* __restrict__ src,
                                           typename Storage<ST>::T* __restrict__ dst, const Lat3<A>& P,
                                           int x, int y, int z)
{
    A f[NF], g[NG];
    const bool nowall = (P.per[0] || (x > 0 && x < P.nx - 1)) && (P.per[1] || (y > 0 && y < P.ny - 1)) &&
                        (P.per[2] || (z > 0 && z < P.nz - 1));
    if (nowall) gather3<true>(src, P, x, y, z, f, g);
    else gather3(src, P, x, y, z, f, g);
    collide3<Storage<ST>::DEV, HIGH1>(P, f, g);
    store3(dst, P, (z * P.ny + y) * P.pitch + x, f, g);
}

// One time step: thread (tx, ty) of block b updates node x = (b % xblocks) * blockDim.x + tx of
// row r = (b / xblocks) * blockDim.y + ty, row r being (y, z) = (r % ny, r / ny).
template <int ST, bool HIGH1>
__global__ void __launch_bounds__(256) k_step3(const typename Storage<ST>::T* __restrict__ src,
                                               typename Storage<ST>::T* __restrict__ dst,
                                               const Lat3<typename Storage<ST>::A> P, int xblocks)
{
    const int xb = blockIdx.x % xblocks, rb = blockIdx.x / xblocks;
    const int x = xb * blockDim.x + threadIdx.x;
    const int r = rb * blockDim.y + threadIdx.y;
    if (x >= P.nx || r >= P.ny * P.nz) return;
    step3_node<ST, HIGH1>(src, dst, P, x, r % P.ny, r / P.ny);
}

// A lattice of a 3-D batch as the blocks of the batched step see it (each block copies it to
// shared memory).
template <typename A>
struct Member3 {
    Lat3<A> P;
    void* buf[2];
    int xblocks;     // blocks along x
    int tile_begin;  // the lattice's first block
    int flip;        // the lattice's current state is in buf[parity ^ flip]
    int high1;       // s_3 = s_4 = s_5 = s_6 = 1: the collision form that skips those moments
};

// One time step of every lattice of a batch: block b covers tile t = b - tile_begin of lattice
// owner[b], nodes x = (t % xblocks) * blockDim.x + tx of rows (y, z) = (r % ny, r / ny) for
// r = (t / xblocks) * blockDim.y * groups + ty + k blockDim.y, k < groups. The per-node update is
// step3_node, the single-lattice step's. Register cap: the lattice's parameters come from shared
// memory rather than the constant bank, and uncapped the FP32 form takes 128 registers (two
// 256-thread blocks per SM); at 64 it keeps the single-lattice step's four blocks (4 bytes of
// spills), the FP16 form three at 80. FP64 is bound by its arithmetic and takes what it needs.
template <int ST>
__global__ void __maxnreg__(ST == ST_F32 ? 64 : ST == ST_F16DEV ? 80 : 255) k_step3_batched(const Member3<typename Storage<ST>::A>* __restrict__ mem,
                                                       const int* __restrict__ owner, int parity, int groups)
{
    using A = typename Storage<ST>::A;
    using T = typename Storage<ST>::T;
    __shared__ Member3<A> M;
    {
        static_assert(sizeof(Member3<A>) % 4 == 0, "member size");
        const int* s = reinterpret_cast<const int*>(mem + owner[blockIdx.x]);
        int* d = reinterpret_cast<int*>(&M);
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        for (int w = tid; w < (int)(sizeof(Member3<A>) / 4); w += blockDim.x * blockDim.y) d[w] = s[w];
        __syncthreads();
    }
    const int t = blockIdx.x - M.tile_begin;
    const int xb = t % M.xblocks, rb = t / M.xblocks;
    const int x = xb * blockDim.x + threadIdx.x;
    if (x >= M.P.nx) return;
    const int rows = blockDim.y * groups;
    const int r_end = min(M.P.ny * M.P.nz, (rb + 1) * rows);
    const int cur = parity ^ M.flip;
    const T* src = (const T*)M.buf[cur];
    T* dst = (T*)M.buf[cur ^ 1];
    for (int r = rb * rows + threadIdx.y; r < r_end; r += blockDim.y) {
        if (M.high1) step3_node<ST, true>(src, dst, M.P, x, r % M.P.ny, r / M.P.ny);
        else step3_node<ST, false>(src, dst, M.P, x, r % M.P.ny, r / M.P.ny);
    }
}

// The D3Q7 populations of node (x, y, z) written into the slots the next pull reads (planes base ..
// base + 6): across a wall face into the node's own opposite slot, as Tw - value on Dirichlet faces.
template <typename T, typename A>
__device__ __forceinline__ void scatter_d3q7(T* __restrict__ dst, const Lat3<A>& P, int x, int y, int z, int base,
                                             const A g[NG])
{
    const int pl = (int)P.plane;
    const int here = (z * P.ny + y) * P.pitch + x;
    const int n3[3] = {P.nx, P.ny, P.nz};
    dst[base * pl + here] = from_a(g[0], (T*)nullptr);
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
            const int j = 1 + 2 * d + sgn, jo = 1 + 2 * d + (1 - sgn);
            int s[3] = {x, y, z};
            s[d] -= sgn == 0 ? 1 : -1;
            bool ok = true;
            if (s[d] < 0 || s[d] >= n3[d]) {
                if (P.per[d]) s[d] = (s[d] + n3[d]) % n3[d];
                else ok = false;
            }
            if (ok) {
                dst[(base + j) * pl + (s[2] * P.ny + s[1]) * P.pitch + s[0]] = from_a(g[j], (T*)nullptr);
            } else {
                const int face = 2 * d + sgn;
                const A v = P.kind[face] == CLB_WALL_DIRICHLET_T ? P.Tw[face] - g[j] : g[j];
                dst[(base + jo) * pl + here] = from_a(v, (T*)nullptr);
            }
        }
}

// Initial state f = f^eq(rho, u), g = g^eq(T, u), written into the slots the first step's pull
// reads (the inverse of the pull, with the face rules inverted: a value pulled across a wall is
// stored in the node's own opposite slot, for g on Dirichlet faces as Tw - value). Every slot is
// written exactly once.
template <int ST>
__global__ void __launch_bounds__(256) k_init3(typename Storage<ST>::T* __restrict__ dst,
                                               const Lat3<typename Storage<ST>::A> P,
                                               const double* __restrict__ fields, long long n)
{
    using A = typename Storage<ST>::A;
    using T = typename Storage<ST>::T;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int x = int(k % P.nx), y = int((k / P.nx) % P.ny), z = int(k / ((long long)P.nx * P.ny));
    const A drho = A(fields[k] - double(P.rho_b));
    const A ux = A(fields[n + k]), uy = A(fields[2 * n + k]), uz = A(fields[3 * n + k]);
    const A dT = A(fields[4 * n + k] - double(P.T_b));
    A f[NF], g[NG];
    equilibrium3<Storage<ST>::DEV>(P, drho, ux, uy, uz, dT, f, g);
    const int pl = (int)P.plane;
    const int here = (z * P.ny + y) * P.pitch + x;
    // the node's pull of population i reads the node at x - e_i; write there, or in the opposite
    // slot here when x - e_i lies beyond a wall
    const int c3[3] = {x, y, z}, n3[3] = {P.nx, P.ny, P.nz};
#pragma unroll
    for (int i = 0; i < NF; ++i) {
        const int dg[3] = {i % 3, (i / 3) % 3, i / 9};
        int s[3];
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            s[d] = c3[d] - vel(dg[d]);
            if (s[d] < 0 || s[d] >= n3[d]) {
                if (P.per[d]) s[d] = (s[d] + n3[d]) % n3[d];
                else ok = false;
            }
        }
        const int o = oppd(dg[0]) + 3 * oppd(dg[1]) + 9 * oppd(dg[2]);
        const int off = ok ? i * pl + (s[2] * P.ny + s[1]) * P.pitch + s[0] : o * pl + here;
        A v = f[i];
        if (!ok && P.moving) {
            // the pull adds the crossed face's wall term: store the value without it
            int face = -1;
            for (int d = 0; d < 3; ++d) {
                const int sd = c3[d] - vel(dg[d]);
                if (!P.per[d] && (sd < 0 || sd >= n3[d])) face = 2 * d + (sd < 0 ? 0 : 1);
            }
            v = v - P.fbb[face][i];
        }
        dst[off] = from_a(v, (T*)nullptr);
    }
    scatter_d3q7(dst, P, x, y, z, NF, g);
}

// Macroscopic fields (FP64) of the current pre-collision state; with pops != nullptr also the
// populations themselves (deviations plus the rest state).
template <int ST>
__global__ void __launch_bounds__(256) k_fields3(const typename Storage<ST>::T* __restrict__ src,
                                                 const Lat3<typename Storage<ST>::A> P,
                                                 double* __restrict__ out, double* __restrict__ pops,
                                                 long long n)
{
    using A = typename Storage<ST>::A;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int x = int(k % P.nx), y = int((k / P.nx) % P.ny), z = int(k / ((long long)P.nx * P.ny));
    A f[NF], g[NG];
    gather3(src, P, x, y, z, f, g);
    if (pops) {
        const double w1[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};
        const double c2 = double(P.cs2T);
        for (int i = 0; i < NF; ++i)
            pops[i * n + k] = double(f[i]) + double(P.rho_b) * w1[i % 3] * w1[(i / 3) % 3] * w1[i / 9];
        for (int j = 0; j < NG; ++j)
            pops[(NF + j) * n + k] = double(g[j]) + double(P.T_b) * (j == 0 ? 1.0 - 3.0 * c2 : 0.5 * c2);
    }
    // rho, u, T in FP64 from the stored values (Eqs. 3, 13, 23)
    double drho = 0, j[3] = {0, 0, 0}, dT = 0;
    for (int i = 0; i < NF; ++i) {
        const double v = double(f[i]);
        drho += v;
        j[0] += vel(i % 3) * v;
        j[1] += vel((i / 3) % 3) * v;
        j[2] += vel(i / 9) * v;
    }
    for (int q = 0; q < NG; ++q) dT += double(g[q]);
    const double rho = double(P.rho_b) + drho, T = double(P.T_b) + dT;
    double F[3] = {double(P.Fv[0]), double(P.Fv[1]), double(P.Fv[2])};
    F[P.g_axis] += double(P.gb) * (T - double(P.T0));
    out[k] = rho;
    for (int d = 0; d < 3; ++d) out[(1 + d) * n + k] = (j[d] + 0.5 * F[d]) / rho;
    out[4 * n + k] = T;
}

// Per-row FP64 sums of u_axis (T - T0) and of non-finite nodes (block per row (y, z), threads
// striding over x), reduced in shared memory in a fixed order.
template <int ST>
__global__ void __launch_bounds__(kRedThreads) k_nu_rows3(const typename Storage<ST>::T* __restrict__ src,
                                                          const Lat3<typename Storage<ST>::A> P, int axis,
                                                          double* __restrict__ partial)
{
    using A = typename Storage<ST>::A;
    const int r = blockIdx.x;
    const int y = r % P.ny, z = r / P.ny;
    double s = 0.0, bad = 0.0;
    for (int x = threadIdx.x; x < P.nx; x += kRedThreads) {
        A f[NF], g[NG];
        gather3(src, P, x, y, z, f, g);
        double drho = 0, jd = 0, dT = 0;
        for (int i = 0; i < NF; ++i) {
            const int e = axis == 0 ? vel(i % 3) : axis == 1 ? vel((i / 3) % 3) : vel(i / 9);
            drho += double(f[i]);
            jd += e * double(f[i]);
        }
        for (int q = 0; q < NG; ++q) dT += double(g[q]);
        const double rho = double(P.rho_b) + drho, T = double(P.T_b) + dT;
        const double Fd = double(P.Fv[axis]) + (P.g_axis == axis ? double(P.gb) * (T - double(P.T0)) : 0.0);
        const double u = (jd + 0.5 * Fd) / rho;
        s += u * (T - double(P.T0));
        bad += (isfinite(u) && isfinite(T) && isfinite(rho)) ? 0.0 : 1.0;
    }
    __shared__ double sh[2][kRedThreads];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = bad;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * r] = sh[0][0];
        partial[2 * r + 1] = sh[1][0];
    }
}

__global__ void __launch_bounds__(kRedThreads) k_nu_final3(const double* __restrict__ partial, int rows,
                                                           double* __restrict__ out)
{
    double s = 0.0, bad = 0.0;
    for (int r = threadIdx.x; r < rows; r += kRedThreads) {
        s += partial[2 * r];
        bad += partial[2 * r + 1];
    }
    __shared__ double sh[2][kRedThreads];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = bad;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0];
        out[1] = sh[1][0];
    }
}

// Per-row FP64 sums for the steady-state residual: sum |u - u_snap|^2, sum |u|^2,
// sum (T - T_snap)^2, sum T^2 and the count of non-finite nodes (block per row (y, z), threads
// striding over x, a fixed order); with update != 0 the snapshot (u_x, u_y, u_z, T as double
// [4][n]) is replaced by the current fields.
constexpr int kResN = 5;

template <int ST>
__global__ void __launch_bounds__(kRedThreads) k_resid_rows3(const typename Storage<ST>::T* __restrict__ src,
                                                             const Lat3<typename Storage<ST>::A> P,
                                                             double* __restrict__ snap, int update,
                                                             double* __restrict__ partial)
{
    using A = typename Storage<ST>::A;
    const int r = blockIdx.x;
    const int y = r % P.ny, z = r / P.ny;
    const long long n = (long long)P.nx * P.ny * P.nz;
    double v[kResN] = {0, 0, 0, 0, 0};
    for (int x = threadIdx.x; x < P.nx; x += kRedThreads) {
        A f[NF], g[NG];
        gather3(src, P, x, y, z, f, g);
        double drho = 0, j[3] = {0, 0, 0}, dT = 0;
        for (int i = 0; i < NF; ++i) {
            const double w = double(f[i]);
            drho += w;
            j[0] += vel(i % 3) * w;
            j[1] += vel((i / 3) % 3) * w;
            j[2] += vel(i / 9) * w;
        }
        for (int q = 0; q < NG; ++q) dT += double(g[q]);
        const double rho = double(P.rho_b) + drho, T = double(P.T_b) + dT;
        const double buoy = double(P.gb) * (T - double(P.T0));
        double u[3];
        for (int d = 0; d < 3; ++d) u[d] = (j[d] + 0.5 * (double(P.Fv[d]) + (P.g_axis == d ? buoy : 0.0))) / rho;
        const long long k = ((long long)z * P.ny + y) * P.nx + x;
        double du = 0.0, uu = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double e = u[d] - snap[d * n + k];
            du += e * e;
            uu += u[d] * u[d];
        }
        const double eT = T - snap[3 * n + k];
        v[0] += du;
        v[1] += uu;
        v[2] += eT * eT;
        v[3] += T * T;
        v[4] += (isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) && isfinite(T)) ? 0.0 : 1.0;
        if (update) {
            for (int d = 0; d < 3; ++d) snap[d * n + k] = u[d];
            snap[3 * n + k] = T;
        }
    }
    __shared__ double sh[kResN][kRedThreads];
    for (int q = 0; q < kResN; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < kResN; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < kResN; ++q) partial[(long long)kResN * r + q] = sh[q][0];
}

__global__ void __launch_bounds__(kRedThreads) k_resid_final3(const double* __restrict__ partial, int rows,
                                                              double* __restrict__ out)
{
    double v[kResN] = {0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < rows; r += kRedThreads)
        for (int q = 0; q < kResN; ++q) v[q] += partial[(long long)kResN * r + q];
    __shared__ double sh[kResN][kRedThreads];
    for (int q = 0; q < kResN; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < kResN; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < kResN; ++q) out[q] = sh[q][0];
}

// ---------------------------------------------------------------------------------------------
// Thermal-only mode: the D3Q7 equation alone with a prescribed velocity (the 3-D form of the
// Sec. 3.1 set-up). Buffers hold the 7 D3Q7 planes; the velocity is a dense [3][nz][ny][nx] array
// in the arithmetic precision. The pull, collision, equilibrium and initial scatter are the coupled
// step's D3Q7 functions.

template <int ST>
__global__ void __launch_bounds__(256) k_thermal3_step(const typename Storage<ST>::T* __restrict__ src,
                                                       typename Storage<ST>::T* __restrict__ dst,
                                                       const typename Storage<ST>::A* __restrict__ vel,
                                                       const Lat3<typename Storage<ST>::A> P, int xblocks)
{
    using A = typename Storage<ST>::A;
    using T = typename Storage<ST>::T;
    const int xb = blockIdx.x % xblocks, rb = blockIdx.x / xblocks;
    const int x = xb * blockDim.x + threadIdx.x;
    const int r = rb * blockDim.y + threadIdx.y;
    if (x >= P.nx || r >= P.ny * P.nz) return;
    const int y = r % P.ny, z = r / P.ny;
    A g[NG];
    const bool nowall = (P.per[0] || (x > 0 && x < P.nx - 1)) && (P.per[1] || (y > 0 && y < P.ny - 1)) &&
                        (P.per[2] || (z > 0 && z < P.nz - 1));
    if (nowall) gather_d3q7<true>(src, P, x, y, z, 0, g);
    else gather_d3q7(src, P, x, y, z, 0, g);
    const long long n = (long long)P.nx * P.ny * P.nz;
    const long long k = ((long long)z * P.ny + y) * P.nx + x;
    const A u[3] = {vel[k], vel[n + k], vel[2 * n + k]};
    const A dT = (g[0] + (g[1] + g[2])) + ((g[3] + g[4]) + (g[5] + g[6]));
    collide_d3q7<Storage<ST>::DEV>(P, u, dT, g);
    const int pl = (int)P.plane;
    const int here = (z * P.ny + y) * P.pitch + x;
#pragma unroll
    for (int j = 0; j < NG; ++j) dst[j * pl + here] = from_a(g[j], (T*)nullptr);
}

template <int ST>
__global__ void __launch_bounds__(256) k_thermal3_init(typename Storage<ST>::T* __restrict__ dst,
                                                       typename Storage<ST>::A* __restrict__ vel,
                                                       const Lat3<typename Storage<ST>::A> P,
                                                       const double* __restrict__ fields, long long n)
{
    using A = typename Storage<ST>::A;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int x = int(k % P.nx), y = int((k / P.nx) % P.ny), z = int(k / ((long long)P.nx * P.ny));
    const A u[3] = {A(fields[n + k]), A(fields[2 * n + k]), A(fields[3 * n + k])};
    const A dT = A(fields[k] - double(P.T_b));
    A g[NG];
    equilibrium_d3q7(P, u, dT, g);
    scatter_d3q7(dst, P, x, y, z, 0, g);
    for (int d = 0; d < 3; ++d) vel[d * n + k] = u[d];
}

template <int ST>
__global__ void __launch_bounds__(256) k_thermal3_out(const typename Storage<ST>::T* __restrict__ src,
                                                      const Lat3<typename Storage<ST>::A> P,
                                                      double* __restrict__ T, double* __restrict__ pops,
                                                      long long n)
{
    using A = typename Storage<ST>::A;
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int x = int(k % P.nx), y = int((k / P.nx) % P.ny), z = int(k / ((long long)P.nx * P.ny));
    A g[NG];
    gather_d3q7(src, P, x, y, z, 0, g);
    double dT = 0.0;
    for (int j = 0; j < NG; ++j) dT += double(g[j]);
    if (T) T[k] = double(P.T_b) + dT;
    if (pops) {
        const double c2 = double(P.cs2T);
        for (int j = 0; j < NG; ++j) pops[j * n + k] = double(g[j]) + double(P.T_b) * (j == 0 ? 1.0 - 3.0 * c2 : 0.5 * c2);
    }
}

}  // namespace clb3

using namespace clb3;

struct clb3d_lattice {
    int nx = 0, ny = 0, nz = 0;
    clb3d_params p{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    char* mem = nullptr;
    void* buf[2] = {nullptr, nullptr};
    double* stage = nullptr;    // 5 fields (init and extraction)
    double* popst = nullptr;    // populations (allocated on first use)
    double* snap = nullptr;     // u_x, u_y, u_z, T at the last residual check (FP64)
    double* partial = nullptr;  // kResN per row
    double* out = nullptr;      // kResN
    double* host_out = nullptr; // pinned, kResN
    int cur = 0;
    long steps = 0;
    int bx = 128, by = 1;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    Lat3<double> Pd{};
    Lat3<float> Pf{};
    long long plane = 0;
    int pitch = 0;
};

namespace {

long long nodes_of(const clb3d_lattice* h) { return (long long)h->nx * h->ny * h->nz; }

size_t esize(int storage) { return storage == CLB_F64 ? 8 : storage == CLB_F32 ? 4 : 2; }

// Row pitch: rows follow one another without padding (each node is one thread and no access is
// vectorised, so rows need no alignment). A padded row would end mid-sector: the pulls would read
// its padding, and a sector written in part is read back from DRAM when it is written out; for
// short rows (small lattices, batches) that cost a quarter of the read traffic. Planes start on
// 256-byte boundaries.
int pitch3(int nx, int storage)
{
    (void)storage;
    return nx;
}

long long plane3(int nx, int ny, int nz, int storage)
{
    const long long per = 256 / (long long)esize(storage);
    const long long e = (long long)pitch3(nx, storage) * ny * nz;
    return (e + per - 1) / per * per;
}

size_t buf_bytes(int nx, int ny, int nz, int storage)
{
    return align256((size_t)NP * (size_t)plane3(nx, ny, nz, storage) * esize(storage)) + 1024;
}

struct Layout3 {
    size_t buf, stage, snap, partial, out, total;
};

Layout3 layout3(int nx, int ny, int nz, int storage)
{
    Layout3 L;
    const size_t n = (size_t)nx * ny * nz;
    L.buf = buf_bytes(nx, ny, nz, storage);
    L.stage = align256(5 * n * sizeof(double));
    L.snap = align256(4 * n * sizeof(double));
    L.partial = align256((size_t)kResN * ny * nz * sizeof(double));
    L.out = 256;
    L.total = 2 * L.buf + L.stage + L.snap + L.partial + L.out;
    return L;
}

clb_status validate3(int nx, int ny, int nz, const clb3d_params* p)
{
    if (!p) return set_error(CLB_EINVAL, "params must not be NULL");
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxEdge || ny > kMaxEdge || nz > kMaxEdge)
        return set_error(CLB_EINVAL, "lattice %dx%dx%d: each extent must be in [1, %d]", nx, ny, nz, kMaxEdge);
    if ((long long)nx * ny * nz > kMaxNodes)
        return set_error(CLB_EINVAL, "lattice %dx%dx%d exceeds %lld nodes", nx, ny, nz, kMaxNodes);
    if (p->storage != CLB_F64 && p->storage != CLB_F32 && p->storage != CLB_F16DEV)
        return set_error(CLB_EINVAL, "3-D storage must be CLB_F64, CLB_F32 or CLB_F16DEV (got %d)", p->storage);
    if (NP * plane3(nx, ny, nz, p->storage) >= (1LL << 31))
        return set_error(CLB_EINVAL, "lattice %dx%dx%d: a buffer exceeds 2^31 elements", nx, ny, nz);
    for (int f = 0; f < 6; ++f) {
        const int k = p->wall[f];
        if (k != CLB_PERIODIC && k != CLB_WALL_DIRICHLET_T && k != CLB_WALL_ADIABATIC)
            return set_error(CLB_EINVAL, "face %d: wall kind %d is not supported in 3-D", f, k);
    }
    for (int d = 0; d < 3; ++d)
        if ((p->wall[2 * d] == CLB_PERIODIC) != (p->wall[2 * d + 1] == CLB_PERIODIC))
            return set_error(CLB_EINVAL, "axis %d: periodic faces must come in pairs", d);
    if (!(p->nu > 0) || !(p->kappa > 0)) return set_error(CLB_EINVAL, "nu and kappa must be > 0");
    if (!(p->cs2_T > 0) || !(p->cs2_T < 1.0 / 3.0)) return set_error(CLB_EINVAL, "cs2_T must be in (0, 1/3)");
    const double lam1 = rate_kappa(p->kappa, p->cs2_T);
    const double rates[8] = {p->s_b, p->s_3, p->s_4, p->s_5, p->s_6, p->lambda2, rate_nu(p->nu), lam1};
    for (double r : rates)
        if (!(r > 0) || !(r < 2)) return set_error(CLB_EINVAL, "relaxation rates must lie in (0, 2)");
    if (!(p->rho0 > 0)) return set_error(CLB_EINVAL, "rho0 must be > 0");
    if (!(p->g_beta >= 0)) return set_error(CLB_EINVAL, "g_beta must be >= 0");
    if (p->g_axis < 0 || p->g_axis > 2) return set_error(CLB_EINVAL, "g_axis must be 0, 1 or 2");
    for (int f = 0; f < 6; ++f)
        for (int d = 0; d < 3; ++d)
            if (!(std::fabs(p->u_wall[f][d]) <= 0.4))
                return set_error(CLB_EINVAL, "face %d: wall velocity components must lie in [-0.4, 0.4]", f);
    return CLB_OK;
}

template <typename A>
Lat3<A> make_lat3(int nx, int ny, int nz, const clb3d_params& p)
{
    Lat3<A> P;
    std::memset(&P, 0, sizeof(P));
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.pitch = pitch3(nx, p.storage);
    P.plane = plane3(nx, ny, nz, p.storage);
    const bool dev = p.storage != CLB_F64;
    P.rho_b = dev ? A(p.rho0) : A(0);
    P.T_b = dev ? A(p.T_ref) : A(0);
    for (int d = 0; d < 3; ++d) P.per[d] = p.wall[2 * d] == CLB_PERIODIC;
    // Wall terms from the equilibria of the wall state, f^eq_i(rho0, u_w) = rho0 prod_d p1(e_d; u_d)
    // with the 1-D lattice Maxwellian p1(0; u) = 2/3 - u^2, p1(+-1; u) = (1/3 + u^2 +- u)/2, and
    // g^eq_i + g^eq_opp = T_w (cs2_T + u_wn^2) for the pair along the face normal.
    auto p1 = [](int e, double u) { return e == 0 ? 2.0 / 3.0 - u * u : 0.5 * (1.0 / 3.0 + u * u + e * u); };
    P.moving = 0;
    for (int f = 0; f < 6; ++f) {
        P.kind[f] = p.wall[f];
        const bool wall = p.wall[f] != CLB_PERIODIC;
        const double* u = p.u_wall[f];
        const double un = wall ? u[f / 2] : 0.0;
        P.Tw[f] = A(p.T_wall[f] * (p.cs2_T + un * un) - p.cs2_T * (dev ? p.T_ref : 0.0));
        for (int i = 0; i < NF; ++i) {
            const int e[3] = {vel(i % 3), vel((i / 3) % 3), vel(i / 9)};
            double fi = 1.0, fo = 1.0;
            for (int d = 0; d < 3; ++d) {
                fi *= p1(e[d], wall ? u[d] : 0.0);
                fo *= p1(-e[d], wall ? u[d] : 0.0);
            }
            P.fbb[f][i] = A(p.rho0 * (fi - fo));
        }
        if (wall && (u[0] != 0.0 || u[1] != 0.0 || u[2] != 0.0)) P.moving = 1;
    }
    const double s_nu = rate_nu(p.nu);
    P.s_nu = A(s_nu);
    P.s_b3 = A((p.s_b - s_nu) / 3.0);
    P.s_3 = A(p.s_3);
    P.s_4 = A(p.s_4);
    P.s_5 = A(p.s_5);
    P.s_6 = A(p.s_6);
    P.lambda1 = A(rate_kappa(p.kappa, p.cs2_T));
    P.lambda2 = A(p.lambda2);
    P.cs2T = A(p.cs2_T);
    for (int d = 0; d < 3; ++d) P.Fv[d] = A(p.Fv[d]);
    P.g_axis = p.g_axis;
    P.gb = A(p.rho0 * p.g_beta);
    P.T0 = A(p.T0);
    return P;
}

#define CHECK_H3(h) \
    if (!(h)) return set_error(CLB_EINVAL, "lattice handle is NULL")

int xblocks_of(const clb3d_lattice* h) { return (h->nx + h->bx - 1) / h->bx; }

template <int ST, bool HIGH1>
void launch3(const clb3d_lattice* h, int from, cudaStream_t s, unsigned grid, dim3 block, int xb)
{
    using T = typename Storage<ST>::T;
    if constexpr (ST == ST_F64)
        k_step3<ST, HIGH1><<<grid, block, 0, s>>>((const T*)h->buf[from], (T*)h->buf[from ^ 1], h->Pd, xb);
    else
        k_step3<ST, HIGH1><<<grid, block, 0, s>>>((const T*)h->buf[from], (T*)h->buf[from ^ 1], h->Pf, xb);
}

template <int ST>
void launch3_rates(const clb3d_lattice* h, int from, cudaStream_t s, unsigned grid, dim3 block, int xb)
{
    // the high-order rates all 1 (the paper's setting): the form that skips those moments
    const bool high1 = h->p.s_3 == 1.0 && h->p.s_4 == 1.0 && h->p.s_5 == 1.0 && h->p.s_6 == 1.0;
    if (high1) launch3<ST, true>(h, from, s, grid, block, xb);
    else launch3<ST, false>(h, from, s, grid, block, xb);
}

clb_status launch_step3(clb3d_lattice* h, int from, cudaStream_t s)
{
    const int xb = xblocks_of(h);
    const long long rb = ((long long)h->ny * h->nz + h->by - 1) / h->by;
    const dim3 block(h->bx, h->by);
    const unsigned grid = unsigned((long long)xb * rb);
    if (h->p.storage == CLB_F64) launch3_rates<ST_F64>(h, from, s, grid, block, xb);
    else if (h->p.storage == CLB_F32) launch3_rates<ST_F32>(h, from, s, grid, block, xb);
    else launch3_rates<ST_F16DEV>(h, from, s, grid, block, xb);
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

void drop_graphs3(clb3d_lattice* h)
{
    for (auto& g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

clb_status build_graph3(clb3d_lattice* h, int start)
{
    CLB_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    clb_status st = CLB_OK;
    for (int k = 0; k < kChunk && st == CLB_OK; ++k) st = launch_step3(h, start ^ (k & 1), h->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (st != CLB_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return set_error(CLB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&h->graph[start], g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return set_error(CLB_ECUDA, "graph instantiate: %s", cudaGetErrorString(e2));
    return CLB_OK;
}

}  // namespace

extern "C" clb_status clb3d_params_default(clb3d_params* p)
{
    if (!p) return set_error(CLB_EINVAL, "params must not be NULL");
    std::memset(p, 0, sizeof(*p));
    p->nu = 0.02;
    p->kappa = 0.02;
    p->rho0 = 1.0;
    p->s_b = p->s_3 = p->s_4 = p->s_5 = p->s_6 = 1.0;
    p->lambda2 = 1.0;
    p->cs2_T = 0.25;
    p->g_axis = 2;
    p->storage = CLB_F64;
    return CLB_OK;
}

extern "C" clb_status clb3d_footprint(int nx, int ny, int nz, const clb3d_params* p, size_t* bytes)
{
    CLB_TRY(validate3(nx, ny, nz, p));
    if (!bytes) return set_error(CLB_EINVAL, "bytes must not be NULL");
    *bytes = layout3(nx, ny, nz, p->storage).total;
    return CLB_OK;
}

extern "C" clb_status clb3d_create(int nx, int ny, int nz, const clb3d_params* p, void* stream,
                                   clb3d_lattice** out)
{
    if (!out) return set_error(CLB_EINVAL, "out must not be NULL");
    *out = nullptr;
    CLB_TRY(validate3(nx, ny, nz, p));
    clb3d_lattice* h = new (std::nothrow) clb3d_lattice();
    if (!h) return set_error(CLB_ENOMEM, "host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->p = *p;
    h->stream = (cudaStream_t)stream;
    const Layout3 L = layout3(nx, ny, nz, p->storage);
    cudaError_t e = cudaMalloc((void**)&h->mem, L.total);
    if (e != cudaSuccess) {
        delete h;
        return set_error(e == cudaErrorMemoryAllocation ? CLB_ENOMEM : CLB_ECUDA, "cudaMalloc(%zu): %s",
                         L.total, cudaGetErrorString(e));
    }
    char* m = h->mem;
    h->buf[0] = m;
    h->buf[1] = m + L.buf;
    h->stage = (double*)(m + 2 * L.buf);
    h->snap = (double*)(m + 2 * L.buf + L.stage);
    h->partial = (double*)(m + 2 * L.buf + L.stage + L.snap);
    h->out = (double*)(m + 2 * L.buf + L.stage + L.snap + L.partial);
    e = cudaMallocHost((void**)&h->host_out, kResN * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        clb3d_destroy(h);
        return set_error(CLB_ECUDA, "lattice set-up: %s", cudaGetErrorString(e));
    }
    h->Pd = make_lat3<double>(nx, ny, nz, *p);
    h->Pf = make_lat3<float>(nx, ny, nz, *p);
    h->plane = plane3(nx, ny, nz, p->storage);
    h->pitch = pitch3(nx, p->storage);
    h->bx = nx > 128 ? 256 : (nx > 64 ? 128 : (nx > 32 ? 64 : 32));
    h->by = h->bx >= 128 ? 1 : 128 / h->bx;
    *out = h;
    return CLB_OK;
}

extern "C" void clb3d_destroy(clb3d_lattice* h)
{
    if (!h) return;
    if (h->stream || h->mem) cudaStreamSynchronize(h->stream);
    drop_graphs3(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->popst) cudaFree(h->popst);
    if (h->mem) cudaFree(h->mem);
    if (h->host_out) cudaFreeHost(h->host_out);
    delete h;
}

namespace {

// The residual E_R since the last snapshot, with the snapshot replaced by the current fields:
// E_R = max over u (all three components) and T of sqrt(sum |X - X_snap|^2 / max(sum |X|^2,
// N (1e-3 X_ref)^2)) with X_ref = u_ref, dT_ref (the reading of the 2-D form). Synchronises.
clb_status residual3(clb3d_lattice* h, double* er)
{
    const int rows = h->ny * h->nz;
    if (h->p.storage == CLB_F64)
        k_resid_rows3<ST_F64><<<rows, kRedThreads, 0, h->stream>>>((const double*)h->buf[h->cur], h->Pd, h->snap, 1, h->partial);
    else if (h->p.storage == CLB_F32)
        k_resid_rows3<ST_F32><<<rows, kRedThreads, 0, h->stream>>>((const float*)h->buf[h->cur], h->Pf, h->snap, 1, h->partial);
    else
        k_resid_rows3<ST_F16DEV><<<rows, kRedThreads, 0, h->stream>>>((const __half*)h->buf[h->cur], h->Pf, h->snap, 1, h->partial);
    CLB_CUDA(cudaGetLastError());
    k_resid_final3<<<1, kRedThreads, 0, h->stream>>>(h->partial, rows, h->out);
    CLB_CUDA(cudaGetLastError());
    CLB_CUDA(cudaMemcpyAsync(h->host_out, h->out, kResN * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    const double* v = h->host_out;
    if (v[4] > 0) return set_error(CLB_ENAN, "%.0f nodes have non-finite fields after %ld steps", v[4], h->steps);
    const double N = double(nodes_of(h));
    const double fu = N * (1e-3 * h->p.u_ref) * (1e-3 * h->p.u_ref);
    const double fT = N * (1e-3 * h->p.dT_ref) * (1e-3 * h->p.dT_ref);
    const double du = v[1] > fu ? v[1] : fu, dt = v[3] > fT ? v[3] : fT;
    const double ru = v[0] == 0.0 ? 0.0 : (du > 0 ? std::sqrt(v[0] / du) : INFINITY);
    const double rt = v[2] == 0.0 ? 0.0 : (dt > 0 ? std::sqrt(v[2] / dt) : INFINITY);
    *er = ru > rt ? ru : rt;
    return CLB_OK;
}

}  // namespace

extern "C" clb_status clb3d_residual(clb3d_lattice* h, double* er_out)
{
    CHECK_H3(h);
    if (!er_out) return set_error(CLB_EINVAL, "er_out must not be NULL");
    return residual3(h, er_out);
}

extern "C" clb_status clb3d_run(clb3d_lattice* h, double tol, long max_steps, long interval, long* steps_out,
                                double* er_out)
{
    CHECK_H3(h);
    if (interval <= 0 || max_steps < 0) return set_error(CLB_EINVAL, "interval must be > 0 and max_steps >= 0");
    long done = 0;
    double er = INFINITY;
    clb_status st = CLB_OK;
    while (done < max_steps) {
        const long n = std::min(interval, max_steps - done);
        CLB_TRY(clb3d_step(h, n));
        done += n;
        st = residual3(h, &er);
        if (st != CLB_OK || er < tol) break;
    }
    if (steps_out) *steps_out = done;
    if (er_out) *er_out = er;
    return st;
}

extern "C" clb_status clb3d_init_fields(clb3d_lattice* h, const double* rho, const double* ux, const double* uy,
                                        const double* uz, const double* T)
{
    CHECK_H3(h);
    if (!rho || !ux || !uy || !uz || !T) return set_error(CLB_EINVAL, "field pointers must not be NULL");
    const long long n = nodes_of(h);
    const double* src[5] = {rho, ux, uy, uz, T};
    for (int q = 0; q < 5; ++q)
        CLB_CUDA(cudaMemcpyAsync(h->stage + q * n, src[q], n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const unsigned grid = unsigned((n + 255) / 256);
    if (h->p.storage == CLB_F64)
        k_init3<ST_F64><<<grid, 256, 0, h->stream>>>((double*)h->buf[0], h->Pd, h->stage, n);
    else if (h->p.storage == CLB_F32)
        k_init3<ST_F32><<<grid, 256, 0, h->stream>>>((float*)h->buf[0], h->Pf, h->stage, n);
    else
        k_init3<ST_F16DEV><<<grid, 256, 0, h->stream>>>((__half*)h->buf[0], h->Pf, h->stage, n);
    CLB_CUDA(cudaGetLastError());
    h->cur = 0;
    h->steps = 0;
    // the residual's first snapshot: the initial fields
    double er = 0.0;
    CLB_TRY(residual3(h, &er));
    return CLB_OK;
}

extern "C" clb_status clb3d_step(clb3d_lattice* h, long n)
{
    CHECK_H3(h);
    if (n < 0) return set_error(CLB_EINVAL, "n = %ld < 0", n);
    // both parities are captured on the first chunk (no capture later, mid-stepping)
    if (n >= kChunk)
        for (int par = 0; par < 2; ++par)
            if (!h->graph[par]) CLB_TRY(build_graph3(h, par));
    while (n >= kChunk) {
        CLB_CUDA(cudaGraphLaunch(h->graph[h->cur], h->stream));
        n -= kChunk;
        h->steps += kChunk;
    }
    for (; n > 0; --n) {
        CLB_TRY(launch_step3(h, h->cur, h->stream));
        h->cur ^= 1;
        h->steps += 1;
    }
    return CLB_OK;
}

namespace {

clb_status extract3(clb3d_lattice* h, double* pops_dev)
{
    const long long n = nodes_of(h);
    const unsigned grid = unsigned((n + 255) / 256);
    if (h->p.storage == CLB_F64)
        k_fields3<ST_F64><<<grid, 256, 0, h->stream>>>((const double*)h->buf[h->cur], h->Pd, h->stage, pops_dev, n);
    else if (h->p.storage == CLB_F32)
        k_fields3<ST_F32><<<grid, 256, 0, h->stream>>>((const float*)h->buf[h->cur], h->Pf, h->stage, pops_dev, n);
    else
        k_fields3<ST_F16DEV><<<grid, 256, 0, h->stream>>>((const __half*)h->buf[h->cur], h->Pf, h->stage, pops_dev, n);
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

}  // namespace

extern "C" clb_status clb3d_fields(clb3d_lattice* h, double* rho, double* ux, double* uy, double* uz, double* T)
{
    CHECK_H3(h);
    if (!rho || !ux || !uy || !uz || !T) return set_error(CLB_EINVAL, "field pointers must not be NULL");
    CLB_TRY(extract3(h, nullptr));
    const long long n = nodes_of(h);
    double* dst[5] = {rho, ux, uy, uz, T};
    for (int q = 0; q < 5; ++q)
        CLB_CUDA(cudaMemcpyAsync(dst[q], h->stage + q * n, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb3d_populations(clb3d_lattice* h, double* f, double* g)
{
    CHECK_H3(h);
    if (!f || !g) return set_error(CLB_EINVAL, "population pointers must not be NULL");
    const long long n = nodes_of(h);
    if (!h->popst) CLB_CUDA(cudaMalloc((void**)&h->popst, (size_t)NP * n * sizeof(double)));
    CLB_TRY(extract3(h, h->popst));
    CLB_CUDA(cudaMemcpyAsync(f, h->popst, (size_t)NF * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaMemcpyAsync(g, h->popst + (size_t)NF * n, (size_t)NG * n * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb3d_nusselt(clb3d_lattice* h, int axis, double* nu_out)
{
    CHECK_H3(h);
    if (!nu_out) return set_error(CLB_EINVAL, "nu_out must not be NULL");
    if (axis < 0 || axis > 2) return set_error(CLB_EINVAL, "axis must be 0, 1 or 2");
    const int rows = h->ny * h->nz;
    if (h->p.storage == CLB_F64)
        k_nu_rows3<ST_F64><<<rows, kRedThreads, 0, h->stream>>>((const double*)h->buf[h->cur], h->Pd, axis, h->partial);
    else if (h->p.storage == CLB_F32)
        k_nu_rows3<ST_F32><<<rows, kRedThreads, 0, h->stream>>>((const float*)h->buf[h->cur], h->Pf, axis, h->partial);
    else
        k_nu_rows3<ST_F16DEV><<<rows, kRedThreads, 0, h->stream>>>((const __half*)h->buf[h->cur], h->Pf, axis, h->partial);
    CLB_CUDA(cudaGetLastError());
    k_nu_final3<<<1, kRedThreads, 0, h->stream>>>(h->partial, rows, h->out);
    CLB_CUDA(cudaGetLastError());
    CLB_CUDA(cudaMemcpyAsync(h->host_out, h->out, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    if (h->host_out[1] > 0) return set_error(CLB_ENAN, "%.0f nodes have non-finite fields", h->host_out[1]);
    const int n_axis = axis == 0 ? h->nx : axis == 1 ? h->ny : h->nz;
    const double Tl = h->p.T_wall[2 * axis], Th = h->p.T_wall[2 * axis + 1];
    const double dT = std::fabs(Tl - Th) > 0 ? std::fabs(Tl - Th) : 1.0;
    const double sign = Tl >= Th ? 1.0 : -1.0;
    *nu_out = 1.0 + sign * (h->host_out[0] / double(nodes_of(h))) * n_axis / (h->p.kappa * dT);
    return CLB_OK;
}

extern "C" clb_status clb3d_set_launch(clb3d_lattice* h, int block_x, int block_y)
{
    CHECK_H3(h);
    const int bx = block_x ? block_x : h->bx, by = block_y ? block_y : h->by;
    if (bx < 32 || bx > 256 || bx % 32 || by < 1 || bx * by > 256)
        return set_error(CLB_EINVAL, "launch %dx%d: block_x a multiple of 32 in [32, 256], block_x * block_y <= 256",
                         bx, by);
    if (bx != h->bx || by != h->by) {
        CLB_CUDA(cudaStreamSynchronize(h->stream));
        drop_graphs3(h);
        h->bx = bx;
        h->by = by;
    }
    return CLB_OK;
}

extern "C" clb_status clb3d_sync(clb3d_lattice* h)
{
    CHECK_H3(h);
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

namespace {

struct Ckpt3Header {
    char magic[8];
    int nx, ny, nz, storage;
    long long steps;
    unsigned long long bytes;
};

size_t ckpt3_payload(const clb3d_lattice* h)
{
    return (size_t)NP * (size_t)h->plane * esize(h->p.storage);
}

}  // namespace

extern "C" clb_status clb3d_save(clb3d_lattice* h, void* buf, size_t* bytes)
{
    CHECK_H3(h);
    if (!bytes) return set_error(CLB_EINVAL, "bytes must not be NULL");
    const size_t bb = ckpt3_payload(h), need = sizeof(Ckpt3Header) + bb;
    if (!buf) {
        *bytes = need;
        return CLB_OK;
    }
    if (*bytes < need) return set_error(CLB_EINVAL, "checkpoint buffer %zu < %zu bytes", *bytes, need);
    Ckpt3Header hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "CLB3CKP1", 8);
    hd.nx = h->nx;
    hd.ny = h->ny;
    hd.nz = h->nz;
    hd.storage = h->p.storage;
    hd.steps = h->steps;
    hd.bytes = bb;
    std::memcpy(buf, &hd, sizeof(hd));
    CLB_CUDA(cudaMemcpyAsync((char*)buf + sizeof(hd), h->buf[h->cur], bb, cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    *bytes = need;
    return CLB_OK;
}

extern "C" clb_status clb3d_load(clb3d_lattice* h, const void* buf, size_t bytes)
{
    CHECK_H3(h);
    if (!buf || bytes < sizeof(Ckpt3Header)) return set_error(CLB_EINVAL, "checkpoint too small");
    Ckpt3Header hd;
    std::memcpy(&hd, buf, sizeof(hd));
    const size_t bb = ckpt3_payload(h);
    if (std::memcmp(hd.magic, "CLB3CKP1", 8) != 0 || hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz ||
        hd.storage != h->p.storage || hd.bytes != bb || bytes < sizeof(hd) + bb)
        return set_error(CLB_EINVAL, "checkpoint does not match this lattice");
    CLB_CUDA(cudaMemcpyAsync(h->buf[h->cur], (const char*)buf + sizeof(hd), bb, cudaMemcpyHostToDevice, h->stream));
    h->steps = hd.steps;
    // the residual's snapshot restarts from the restored state
    double er = 0.0;
    return residual3(h, &er);
}

extern "C" void* clb3d_stream(clb3d_lattice* h) { return h ? (void*)h->stream : nullptr; }

extern "C" clb_status clb3d_buffers(clb3d_lattice* h, void** current, long long* plane_elems, int* row_pitch)
{
    CHECK_H3(h);
    if (current) *current = h->buf[h->cur];
    if (plane_elems) *plane_elems = h->plane;
    if (row_pitch) *row_pitch = h->pitch;
    return CLB_OK;
}

// ---------------------------------------------------------------------------------------------
// Batches of 3-D lattices: every lattice is an ordinary handle (its own memory, fields, Nusselt
// number, residual); the time steps of all of them go through one k_step3_batched launch per step
// over their concatenated tiles, replayed from CUDA graphs of kChunk steps.

struct clb3d_batch {
    int storage = CLB_F64;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only to capture graphs
    std::vector<clb3d_lattice*> lat;
    std::vector<int> flip;       // lattice k's current state is in buf[parity ^ flip[k]]
    std::vector<char> host_members;
    void* d_members = nullptr;
    int* d_owner = nullptr;
    long long ntiles = 0;
    int bx = 128, by = 2, groups = 1;
    int parity = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

namespace {

// Nodes a block of the batched 3-D step covers at most, and the rounds of resident blocks a
// launch keeps at least (fewer groups of rows per block where the batch is small): the same
// policy as the 2-D batch.
constexpr int kBlockNodes3 = 2048;
constexpr int kMinWaves3 = 8;

template <int ST>
long long resident_blocks3(int threads)
{
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step3_batched<ST>, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return (long long)std::max(1, sms) * std::max(1, per_sm);
}

long long batch3_tiles(const clb3d_batch* b, int g)
{
    long long t = 0;
    for (const clb3d_lattice* h : b->lat)
        t += (long long)((h->nx + b->bx - 1) / b->bx) *
             (((long long)h->ny * h->nz + (long long)b->by * g - 1) / ((long long)b->by * g));
    return t;
}

void drop_batch3_graphs(clb3d_batch* b)
{
    for (auto& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

template <typename A>
Member3<A> member3(const clb3d_batch* b, const clb3d_lattice* h, int flip, int tile_begin, const Lat3<A>& P)
{
    Member3<A> m;
    std::memset(&m, 0, sizeof(m));
    m.P = P;
    m.buf[0] = h->buf[0];
    m.buf[1] = h->buf[1];
    m.xblocks = (h->nx + b->bx - 1) / b->bx;
    m.tile_begin = tile_begin;
    m.flip = flip;
    m.high1 = h->p.s_3 == 1.0 && h->p.s_4 == 1.0 && h->p.s_5 == 1.0 && h->p.s_6 == 1.0;
    return m;
}

// Groups of rows per block and the member and owner tables for the current tile shape; uploads
// them and synchronises the stream.
clb_status batch3_tables(clb3d_batch* b)
{
    drop_batch3_graphs(b);
    const int threads = b->bx * b->by;
    const long long resident = b->storage == CLB_F64   ? resident_blocks3<ST_F64>(threads)
                               : b->storage == CLB_F32 ? resident_blocks3<ST_F32>(threads)
                                                       : resident_blocks3<ST_F16DEV>(threads);
    b->groups = 1;
    for (int g = 2; g * threads <= kBlockNodes3 && batch3_tiles(b, g) >= kMinWaves3 * resident; g *= 2) b->groups = g;
    const long long tiles = batch3_tiles(b, b->groups);
    if (tiles > 0x7fffffffLL) return set_error(CLB_EINVAL, "batch of %lld blocks per step is too large", tiles);
    const size_t msz = b->storage == CLB_F64 ? sizeof(Member3<double>) : sizeof(Member3<float>);
    b->host_members.assign(msz * b->lat.size(), 0);
    std::vector<int> owner((size_t)tiles);
    long long t0 = 0;
    for (size_t k = 0; k < b->lat.size(); ++k) {
        const clb3d_lattice* h = b->lat[k];
        if (b->storage == CLB_F64) {
            const Member3<double> m = member3<double>(b, h, b->flip[k], (int)t0, h->Pd);
            std::memcpy(b->host_members.data() + k * msz, &m, msz);
        } else {
            const Member3<float> m = member3<float>(b, h, b->flip[k], (int)t0, h->Pf);
            std::memcpy(b->host_members.data() + k * msz, &m, msz);
        }
        const long long n = (long long)((h->nx + b->bx - 1) / b->bx) *
                            (((long long)h->ny * h->nz + (long long)b->by * b->groups - 1) / ((long long)b->by * b->groups));
        std::fill(owner.begin() + t0, owner.begin() + t0 + n, (int)k);
        t0 += n;
    }
    cudaFree(b->d_members);
    cudaFree(b->d_owner);
    b->d_members = nullptr;
    b->d_owner = nullptr;
    CLB_CUDA(cudaMalloc(&b->d_members, b->host_members.size()));
    CLB_CUDA(cudaMalloc((void**)&b->d_owner, std::max<size_t>(1, owner.size()) * sizeof(int)));
    CLB_CUDA(cudaMemcpyAsync(b->d_members, b->host_members.data(), b->host_members.size(), cudaMemcpyHostToDevice, b->stream));
    CLB_CUDA(cudaMemcpyAsync(b->d_owner, owner.data(), owner.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CLB_CUDA(cudaStreamSynchronize(b->stream));  // the host vectors are reused or die
    b->ntiles = tiles;
    return CLB_OK;
}

clb_status batch3_launch(clb3d_batch* b, int par, cudaStream_t s)
{
    if (b->ntiles == 0) return CLB_OK;
    const dim3 block(b->bx, b->by);
    const unsigned grid = (unsigned)b->ntiles;
    if (b->storage == CLB_F64)
        k_step3_batched<ST_F64><<<grid, block, 0, s>>>((const Member3<double>*)b->d_members, b->d_owner, par, b->groups);
    else if (b->storage == CLB_F32)
        k_step3_batched<ST_F32><<<grid, block, 0, s>>>((const Member3<float>*)b->d_members, b->d_owner, par, b->groups);
    else
        k_step3_batched<ST_F16DEV><<<grid, block, 0, s>>>((const Member3<float>*)b->d_members, b->d_owner, par, b->groups);
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

clb_status batch3_graph(clb3d_batch* b, int start)
{
    CLB_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    clb_status st = CLB_OK;
    for (int k = 0; k < kChunk && st == CLB_OK; ++k) st = batch3_launch(b, start ^ (k & 1), b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (st != CLB_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return set_error(CLB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaGraphInstantiate(&b->graph[start], g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) return set_error(CLB_ECUDA, "graph instantiate: %s", cudaGetErrorString(e2));
    return CLB_OK;
}

#define CHECK_B3(b) \
    if (!(b)) return set_error(CLB_EINVAL, "batch handle is NULL")
#define CHECK_K3(b, k) \
    if ((k) < 0 || (k) >= (int)(b)->lat.size()) return set_error(CLB_EINVAL, "lattice %d of a batch of %zu", (k), (b)->lat.size())

}  // namespace

extern "C" clb_status clb3d_batch_create(int n, const int* nx, const int* ny, const int* nz, const clb3d_params* p,
                                         void* stream, clb3d_batch** out)
{
    if (!out) return set_error(CLB_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (n < 1 || !nx || !ny || !nz || !p) return set_error(CLB_EINVAL, "a batch needs n >= 1 lattices and their extents and parameters");
    for (int k = 0; k < n; ++k) {
        CLB_TRY(validate3(nx[k], ny[k], nz[k], &p[k]));
        if (p[k].storage != p[0].storage)
            return set_error(CLB_EINVAL, "lattice %d: every lattice of a batch has the same storage", k);
    }
    clb3d_batch* b = new (std::nothrow) clb3d_batch();
    if (!b) return set_error(CLB_ENOMEM, "host allocation failed");
    b->storage = p[0].storage;
    b->stream = (cudaStream_t)stream;
    clb_status st = CLB_OK;
    try {
        b->lat.reserve(n);
        b->flip.reserve(n);
        for (int k = 0; k < n && st == CLB_OK; ++k) {
            clb3d_lattice* h = nullptr;
            st = clb3d_create(nx[k], ny[k], nz[k], &p[k], stream, &h);
            if (st == CLB_OK) {
                b->lat.push_back(h);
                b->flip.push_back(0);
            }
        }
        if (st == CLB_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
            st = set_error(CLB_ECUDA, "batch set-up: %s", cudaGetErrorString(cudaGetLastError()));
        if (st == CLB_OK) st = batch3_tables(b);
    } catch (const std::bad_alloc&) {
        st = set_error(CLB_ENOMEM, "host allocation failed");
    }
    if (st != CLB_OK) {
        clb3d_batch_destroy(b);
        return st;
    }
    *out = b;
    return CLB_OK;
}

extern "C" void clb3d_batch_destroy(clb3d_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_batch3_graphs(b);
    for (clb3d_lattice* h : b->lat) clb3d_destroy(h);
    cudaFree(b->d_members);
    cudaFree(b->d_owner);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

extern "C" clb_status clb3d_batch_lattice(clb3d_batch* b, int k, clb3d_lattice** out)
{
    CHECK_B3(b);
    CHECK_K3(b, k);
    if (!out) return set_error(CLB_EINVAL, "out must not be NULL");
    *out = b->lat[k];
    return CLB_OK;
}

extern "C" clb_status clb3d_batch_init_fields(clb3d_batch* b, int k, const double* rho, const double* ux,
                                              const double* uy, const double* uz, const double* T)
{
    CHECK_B3(b);
    CHECK_K3(b, k);
    const clb_status st = clb3d_init_fields(b->lat[k], rho, ux, uy, uz, T);
    if (st != CLB_OK && st != CLB_ENAN) return st;
    // the lattice's state is now in buf[0]: buf[parity ^ flip] with flip = parity
    b->flip[k] = b->parity;
    const size_t msz = b->storage == CLB_F64 ? sizeof(Member3<double>) : sizeof(Member3<float>);
    const size_t off = msz * k + (b->storage == CLB_F64 ? offsetof(Member3<double>, flip) : offsetof(Member3<float>, flip));
    std::memcpy(b->host_members.data() + off, &b->flip[k], sizeof(int));
    CLB_CUDA(cudaMemcpyAsync((char*)b->d_members + off, b->host_members.data() + off, sizeof(int),
                             cudaMemcpyHostToDevice, b->stream));
    CLB_CUDA(cudaStreamSynchronize(b->stream));
    return st;
}

extern "C" clb_status clb3d_batch_step(clb3d_batch* b, long n)
{
    CHECK_B3(b);
    if (n < 0) return set_error(CLB_EINVAL, "n = %ld < 0", n);
    const long total = n;
    if (n >= kChunk)
        for (int par = 0; par < 2; ++par)
            if (!b->graph[par]) CLB_TRY(batch3_graph(b, par));
    while (n >= kChunk) {
        CLB_CUDA(cudaGraphLaunch(b->graph[b->parity], b->stream));
        n -= kChunk;
    }
    for (; n > 0; --n) {
        CLB_TRY(batch3_launch(b, b->parity, b->stream));
        b->parity ^= 1;
    }
    for (size_t k = 0; k < b->lat.size(); ++k) {
        b->lat[k]->cur = b->parity ^ b->flip[k];
        b->lat[k]->steps += total;
    }
    return CLB_OK;
}

extern "C" clb_status clb3d_batch_set_tile(clb3d_batch* b, int block_x, int block_y)
{
    CHECK_B3(b);
    if (block_x < 32 || block_x > 256 || block_x % 32 || block_y < 1 || block_x * block_y > 256)
        return set_error(CLB_EINVAL, "tile %d x %d: block_x in [32, 256] multiple of 32, block_x * block_y <= 256",
                         block_x, block_y);
    CLB_CUDA(cudaStreamSynchronize(b->stream));
    b->bx = block_x;
    b->by = block_y;
    try {
        return batch3_tables(b);
    } catch (const std::bad_alloc&) {
        return set_error(CLB_ENOMEM, "host allocation failed");
    }
}

extern "C" clb_status clb3d_batch_get_launch(clb3d_batch* b, int* block_x, int* block_y, int* groups,
                                             long long* blocks)
{
    CHECK_B3(b);
    if (block_x) *block_x = b->bx;
    if (block_y) *block_y = b->by;
    if (groups) *groups = b->groups;
    if (blocks) *blocks = b->ntiles;
    return CLB_OK;
}

// ---------------------------------------------------------------------------------------------
// Thermal-only handle.

struct clb3d_thermal {
    int nx = 0, ny = 0, nz = 0;
    clb3d_params p{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    char* mem = nullptr;
    void* buf[2] = {nullptr, nullptr};
    void* vel = nullptr;
    double* stage = nullptr;  // T, ux, uy, uz (init) and T (out)
    double* pops = nullptr;   // populations on demand
    int cur = 0;
    long steps = 0;
    int bx = 128, by = 1;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    Lat3<double> Pd{};
    Lat3<float> Pf{};
};

namespace {

size_t thermal3_buf_bytes(int nx, int ny, int nz, int storage)
{
    return align256((size_t)NG * (size_t)plane3(nx, ny, nz, storage) * esize(storage)) + 1024;
}

size_t thermal3_vel_bytes(long long n, int storage)
{
    return align256((size_t)3 * n * (storage == CLB_F64 ? 8 : 4));
}

clb_status thermal3_launch(clb3d_thermal* h, int from, cudaStream_t s)
{
    const int xb = (h->nx + h->bx - 1) / h->bx;
    const long long rb = ((long long)h->ny * h->nz + h->by - 1) / h->by;
    const dim3 block(h->bx, h->by);
    const unsigned grid = unsigned((long long)xb * rb);
    if (h->p.storage == CLB_F64)
        k_thermal3_step<ST_F64><<<grid, block, 0, s>>>((const double*)h->buf[from], (double*)h->buf[from ^ 1],
                                                       (const double*)h->vel, h->Pd, xb);
    else if (h->p.storage == CLB_F32)
        k_thermal3_step<ST_F32><<<grid, block, 0, s>>>((const float*)h->buf[from], (float*)h->buf[from ^ 1],
                                                       (const float*)h->vel, h->Pf, xb);
    else
        k_thermal3_step<ST_F16DEV><<<grid, block, 0, s>>>((const __half*)h->buf[from], (__half*)h->buf[from ^ 1],
                                                          (const float*)h->vel, h->Pf, xb);
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

#define CHECK_T3(h) \
    if (!(h)) return set_error(CLB_EINVAL, "thermal handle is NULL")

}  // namespace

extern "C" clb_status clb3d_thermal_create(int nx, int ny, int nz, const clb3d_params* p, void* stream,
                                           clb3d_thermal** out)
{
    if (!out) return set_error(CLB_EINVAL, "out must not be NULL");
    *out = nullptr;
    CLB_TRY(validate3(nx, ny, nz, p));
    clb3d_thermal* h = new (std::nothrow) clb3d_thermal();
    if (!h) return set_error(CLB_ENOMEM, "host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->p = *p;
    h->stream = (cudaStream_t)stream;
    const long long n = (long long)nx * ny * nz;
    const size_t bb = thermal3_buf_bytes(nx, ny, nz, p->storage), vb = thermal3_vel_bytes(n, p->storage);
    const size_t sb = align256(4 * (size_t)n * sizeof(double));
    cudaError_t e = cudaMalloc((void**)&h->mem, 2 * bb + vb + sb);
    if (e != cudaSuccess) {
        delete h;
        return set_error(e == cudaErrorMemoryAllocation ? CLB_ENOMEM : CLB_ECUDA, "cudaMalloc: %s",
                         cudaGetErrorString(e));
    }
    h->buf[0] = h->mem;
    h->buf[1] = h->mem + bb;
    h->vel = h->mem + 2 * bb;
    h->stage = (double*)(h->mem + 2 * bb + vb);
    e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        clb3d_thermal_destroy(h);
        return set_error(CLB_ECUDA, "thermal set-up: %s", cudaGetErrorString(e));
    }
    h->Pd = make_lat3<double>(nx, ny, nz, *p);
    h->Pf = make_lat3<float>(nx, ny, nz, *p);
    h->bx = nx > 128 ? 256 : (nx > 64 ? 128 : (nx > 32 ? 64 : 32));
    h->by = h->bx >= 128 ? 1 : 128 / h->bx;
    *out = h;
    return CLB_OK;
}

extern "C" void clb3d_thermal_destroy(clb3d_thermal* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto& g : h->graph)
        if (g) cudaGraphExecDestroy(g);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->pops) cudaFree(h->pops);
    if (h->mem) cudaFree(h->mem);
    delete h;
}

extern "C" clb_status clb3d_thermal_init(clb3d_thermal* h, const double* T, const double* ux, const double* uy,
                                         const double* uz)
{
    CHECK_T3(h);
    if (!T || !ux || !uy || !uz) return set_error(CLB_EINVAL, "field pointers must not be NULL");
    const long long n = (long long)h->nx * h->ny * h->nz;
    const double* src[4] = {T, ux, uy, uz};
    for (int q = 0; q < 4; ++q)
        CLB_CUDA(cudaMemcpyAsync(h->stage + q * n, src[q], n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    const unsigned grid = unsigned((n + 255) / 256);
    if (h->p.storage == CLB_F64)
        k_thermal3_init<ST_F64><<<grid, 256, 0, h->stream>>>((double*)h->buf[0], (double*)h->vel, h->Pd, h->stage, n);
    else if (h->p.storage == CLB_F32)
        k_thermal3_init<ST_F32><<<grid, 256, 0, h->stream>>>((float*)h->buf[0], (float*)h->vel, h->Pf, h->stage, n);
    else
        k_thermal3_init<ST_F16DEV><<<grid, 256, 0, h->stream>>>((__half*)h->buf[0], (float*)h->vel, h->Pf, h->stage, n);
    CLB_CUDA(cudaGetLastError());
    h->cur = 0;
    h->steps = 0;
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb3d_thermal_step(clb3d_thermal* h, long n)
{
    CHECK_T3(h);
    if (n < 0) return set_error(CLB_EINVAL, "n = %ld < 0", n);
    for (int par = 0; n >= kChunk && par < 2; ++par) {
        if (h->graph[par]) continue;
        CLB_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        clb_status st = CLB_OK;
        for (int k = 0; k < kChunk && st == CLB_OK; ++k) st = thermal3_launch(h, par ^ (k & 1), h->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(h->cap, &g);
        if (st != CLB_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return set_error(CLB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        const cudaError_t e2 = cudaGraphInstantiate(&h->graph[par], g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) return set_error(CLB_ECUDA, "graph instantiate: %s", cudaGetErrorString(e2));
    }
    while (n >= kChunk) {
        CLB_CUDA(cudaGraphLaunch(h->graph[h->cur], h->stream));
        n -= kChunk;
        h->steps += kChunk;
    }
    for (; n > 0; --n) {
        CLB_TRY(thermal3_launch(h, h->cur, h->stream));
        h->cur ^= 1;
        h->steps += 1;
    }
    return CLB_OK;
}

namespace {

clb_status thermal3_out(clb3d_thermal* h, double* T_dev, double* pops_dev)
{
    const long long n = (long long)h->nx * h->ny * h->nz;
    const unsigned grid = unsigned((n + 255) / 256);
    if (h->p.storage == CLB_F64)
        k_thermal3_out<ST_F64><<<grid, 256, 0, h->stream>>>((const double*)h->buf[h->cur], h->Pd, T_dev, pops_dev, n);
    else if (h->p.storage == CLB_F32)
        k_thermal3_out<ST_F32><<<grid, 256, 0, h->stream>>>((const float*)h->buf[h->cur], h->Pf, T_dev, pops_dev, n);
    else
        k_thermal3_out<ST_F16DEV><<<grid, 256, 0, h->stream>>>((const __half*)h->buf[h->cur], h->Pf, T_dev, pops_dev, n);
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

}  // namespace

extern "C" clb_status clb3d_thermal_fields(clb3d_thermal* h, double* T)
{
    CHECK_T3(h);
    if (!T) return set_error(CLB_EINVAL, "T must not be NULL");
    const long long n = (long long)h->nx * h->ny * h->nz;
    CLB_TRY(thermal3_out(h, h->stage, nullptr));
    CLB_CUDA(cudaMemcpyAsync(T, h->stage, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb3d_thermal_populations(clb3d_thermal* h, double* g)
{
    CHECK_T3(h);
    if (!g) return set_error(CLB_EINVAL, "g must not be NULL");
    const long long n = (long long)h->nx * h->ny * h->nz;
    if (!h->pops) CLB_CUDA(cudaMalloc((void**)&h->pops, (size_t)NG * n * sizeof(double)));
    CLB_TRY(thermal3_out(h, nullptr, h->pops));
    CLB_CUDA(cudaMemcpyAsync(g, h->pops, (size_t)NG * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb3d_thermal_sync(clb3d_thermal* h)
{
    CHECK_T3(h);
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}
