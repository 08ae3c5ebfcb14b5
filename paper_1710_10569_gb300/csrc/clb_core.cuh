// clb_core.cuh -- per-node device arithmetic of the coupled D2Q9 + D2Q5 central-moment LBM
// (Fei, Luo, Lin & Li, arXiv:1710.10569, Sec. 2).
//
// The moment transforms are applied in factorised form. The raw-moment map M of Eq. (7a) and the
// shift N(u) of Eq. (7b) are tensor products of one-dimensional maps over the velocity components
// (M = M_y (x) M_x, N(u) = N_y(u_y) (x) N_x(u_x)), so the nine central moments follow from two
// passes of three-point sums: x-central moments of each row of equal e_y, then y-central moments
// of those. The back transform f* = M^-1 N(u)^-1 Gamma~* (the sentence after Eq. 12) runs the same
// passes backwards with the 1-D inverse (f_0 = m_0 - m_2, f_+- = (m_2 +- m_1)/2). The D2Q5 part
// (Eqs. 16-21, Appendix A) is the same construction with one row per axis. This is about 200 flops
// per node instead of the ~1,600 of literal 9x9 products, and the result is the same map.
//
// Storage. FP64 buffers hold the populations f_i, g_i themselves. FP32 and FP16 buffers hold
// deviations from a rest state, h_i = f_i - w_i rho0 and t_i = g_i - w^T_i T_b(y), and the
// collision is evaluated on those deviations (collide_dev): every intermediate is then small, so
// FP32 rounding acts on quantities of the size of the non-equilibrium and velocity terms instead
// of on the O(1) populations. The temperature base T_b(y) = T_b + T_dy y is linear in the row: on
// a lattice between two Dirichlet (or wet) y walls with periodic x it is the conduction profile
// between the walls, so that the stored deviations of a layer near its conduction state are the
// small departures from it (a constant base leaves them as large as the wall temperatures, and
// the slow growth of convection near onset is then lost to the rounding of the store). A
// population pulled from the row below (above) was stored against that row's base, so the pull
// corrects it by the constant -w^T T_dy (+w^T T_dy); nothing else depends on the absolute base
// except T in the velocity-dependent terms and in the force.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace clb {

enum { WALL_PERIODIC = 0, WALL_DIRICHLET = 1, WALL_ADIABATIC = 2 };
enum { ST_F64 = 0, ST_F32 = 1, ST_F16DEV = 2 };
enum { NPOP = 14 };  // 9 flow + 5 temperature planes per buffer

// Population layout of a coupled lattice: chunked rows. Row y is cut into chunks of kRowChunk
// consecutive nodes (the last one padded), and a chunk holds its nodes' 14 populations plane after
// plane (kRowChunk consecutive values each), so element (i, x, y) lies at
//   y * P.crow + chunk_off(x) + i * kRowChunk,   P.crow = NPOP * kRowChunk * ceil(nx / kRowChunk).
// A warp's access to one population of 32 V consecutive nodes is 32 V / kRowChunk runs of kRowChunk
// values (one 128-byte line per chunk in FP16), and the 14 populations of a node sit at fixed
// offsets i * kRowChunk from one address, so an access needs no per-population address arithmetic.
constexpr int kRowChunk = 64;
__host__ __device__ __forceinline__ long long chunk_off(int x)
{
    return (long long)((unsigned)x / kRowChunk) * (NPOP * kRowChunk) + (long long)((unsigned)x % kRowChunk);
}

// Storage traits: element type in HBM, arithmetic type in registers, deviation form or not.
template <int ST> struct Storage;
template <> struct Storage<ST_F64> { using T = double; using A = double; static constexpr bool DEV = false; };
template <> struct Storage<ST_F32> { using T = float; using A = float; static constexpr bool DEV = true; };
template <> struct Storage<ST_F16DEV> { using T = __half; using A = float; static constexpr bool DEV = true; };

__device__ __forceinline__ double to_a(double v) { return v; }
__device__ __forceinline__ float to_a(float v) { return v; }
__device__ __forceinline__ float to_a(__half v) { return __half2float(v); }
__device__ __forceinline__ double from_a(double v, double*) { return v; }
__device__ __forceinline__ float from_a(float v, float*) { return v; }
__device__ __forceinline__ __half from_a(float v, __half*) { return __float2half_rn(v); }

// Fused multiply-add written out. The library is compiled without automatic contraction
// (-fmad=false), so every rounding step is the one written here: the per-node arithmetic is the
// same instruction sequence in every kernel and launch shape, which makes results bitwise
// independent of how nodes are assigned to threads.
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rcp_(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double rcp_(double a) { return __drcp_rn(a); }

// Two FP32 lanes (two lattice nodes) in one 64-bit register pair, operated on by the packed
// FP32 instructions of sm_100-class GPUs (add/sub/mul/fma .rn.f32x2). Each lane is rounded exactly
// as the scalar instruction would round it, so a node computed in a pair carries the same bits as
// the same node computed alone.
struct F2 {
    unsigned long long u;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float lo, float hi)
    {
        asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(lo), "f"(hi));
    }
    template <typename T>
    __device__ __forceinline__ explicit F2(T x) : F2(float(x), float(x)) {}
    __device__ __forceinline__ void split(float& lo, float& hi) const
    {
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(u));
    }
};
// Both lanes of a packed pair to storage, each rounded to nearest even (for FP16 one conversion
// instruction packs the two halves).
__device__ __forceinline__ void from_a2(F2 v, float& lo, float& hi) { v.split(lo, hi); }
__device__ __forceinline__ void from_a2(F2 v, __half& lo, __half& hi)
{
    float a, b;
    v.split(a, b);
    unsigned r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));  // b to the upper half
    unsigned short l16, h16;
    asm("mov.b32 {%0, %1}, %2;" : "=h"(l16), "=h"(h16) : "r"(r));
    lo = __ushort_as_half(l16);
    hi = __ushort_as_half(h16);
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.u) : "l"(a.u), "l"(b.u));
    return r;
}
__device__ __forceinline__ F2 operator-(F2 a)
{
    F2 r;
    r.u = a.u ^ 0x8000000080000000ull;  // exact sign flip of both lanes
    return r;
}
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2 fma_(F2 a, F2 b, F2 c)
{
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.u) : "l"(a.u), "l"(b.u), "l"(c.u));
    return r;
}
__device__ __forceinline__ F2 rcp_(F2 a)
{
    float lo, hi;
    a.split(lo, hi);
    return F2(__frcp_rn(lo), __frcp_rn(hi));
}

// Per-lattice constants in the arithmetic precision A.
template <typename A>
struct LatParams {
    int nx, ny;
    long long crow;           // elements per chunked row (coupled lattice: see chunk_off)
    int pitch;                // thermal-only mode (plane-major): elements per row, 128-byte aligned
    long long plane;          // thermal-only mode: elements between population planes
    int per_x, per_y;         // periodic flags
    int kind[4];              // wall kind per side (-x, +x, -y, +y)
    A Tw_c2[4];               // anti-bounce-back constant cs2_T (T_wall - T_b) (= 2 w_i T_w, shifted)
    A s_nu, sp, sm, s_3, s_4; // D2Q9 rates; sp = (s_b + s_nu)/2, sm = (s_b - s_nu)/2
    A lambda1, lambda2, cs2T; // D2Q5 rates and sound speed squared
    A Fvx, Fvy, gb, T0;       // F = (Fvx, Fvy + gb (T - T0)), gb = rho0 * g_beta
    A rho_b, T_b;             // rest state the buffers are stored against (0 for FP64); T_b at row 0
    A T_dy, T_dyw;            // slope of the temperature base along y, and w^T_2 T_dy (pull correction)
    A dTw[4];                 // wall temperature minus the base at the wall's row (wet walls)
    int moving;               // some wall moves: fbb holds its momentum terms
    A fbb[4][9];              // [f^eq_i - f^eq_opp](rho0, u_wall of the side), added on bounce-back
    int wet_x, wet_y;         // both x (y) walls are wet walls (on the end columns / rows of nodes)
    A Twall[4], uwall[4][2];  // wall temperature and velocity (wet walls)
};

// 1-D rest weights of D2Q9 (w(0) = 2/3, w(+-1) = 1/6; w_i = w(e_x) w(e_y)) and D2Q5 weights.
template <typename A>
__device__ __forceinline__ A w9(int i)
{
    const A w1[3] = {A(2) / A(3), A(1) / A(6), A(1) / A(6)};
    const int ax[9] = {0, 1, 0, 2, 0, 1, 2, 2, 1};
    const int ay[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};
    return w1[ax[i]] * w1[ay[i]];
}
template <typename A>
__device__ __forceinline__ A w5(int i, A c2)
{
    return i == 0 ? A(1) - A(2) * c2 : A(0.5) * c2;
}

// Source slots of the 14 pulled populations of node (x, y), Eqs. (12) and (22):
// f_i(x) = f*_i(x - e_i); where x - e_i is beyond a wall the node's own opposite slot is read.
// Velocity order of Eq. (4): 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1)
// 7:(-1,-1) 8:(1,-1). wall_mask bits 0..3: the pull of g1, g3, g2, g4 crossed side -x, +x, -y, +y.
struct Slots {
    long long idx[NPOP];
    int wall_mask;
};

template <typename A>
__device__ __forceinline__ Slots pull_slots(const LatParams<A>& P, int x, int y)
{
    Slots s;
    const bool inL = P.per_x || x > 0;
    const bool inR = P.per_x || x < P.nx - 1;
    const bool inB = P.per_y || y > 0;
    const bool inT = P.per_y || y < P.ny - 1;
    const int xm = x > 0 ? x - 1 : P.nx - 1;
    const int xp = x < P.nx - 1 ? x + 1 : 0;
    const long long r0 = (long long)y * P.crow;
    const long long rm = (long long)(y > 0 ? y - 1 : P.ny - 1) * P.crow;
    const long long rp = (long long)(y < P.ny - 1 ? y + 1 : 0) * P.crow;
    const long long cx = chunk_off(x), cm = chunk_off(xm), cp = chunk_off(xp);
    const long long here = r0 + cx;
    constexpr long long C = kRowChunk;
    s.idx[0] = here;
    s.idx[1] = inL ? r0 + cm + 1 * C : here + 3 * C;
    s.idx[2] = inB ? rm + cx + 2 * C : here + 4 * C;
    s.idx[3] = inR ? r0 + cp + 3 * C : here + 1 * C;
    s.idx[4] = inT ? rp + cx + 4 * C : here + 2 * C;
    s.idx[5] = (inL && inB) ? rm + cm + 5 * C : here + 7 * C;
    s.idx[6] = (inR && inB) ? rm + cp + 6 * C : here + 8 * C;
    s.idx[7] = (inR && inT) ? rp + cp + 7 * C : here + 5 * C;
    s.idx[8] = (inL && inT) ? rp + cm + 8 * C : here + 6 * C;
    const long long g0 = 9 * C;  // g_j lies 9 planes after f_j in the same chunk
    s.idx[9] = g0 + here;
    s.idx[10] = g0 + s.idx[1];
    s.idx[11] = g0 + s.idx[2];
    s.idx[12] = g0 + s.idx[3];
    s.idx[13] = g0 + s.idx[4];
    s.wall_mask = (inL ? 0 : 1) | (inR ? 0 : 2) | (inB ? 0 : 4) | (inT ? 0 : 8);
    return s;
}

template <typename T>
__device__ __forceinline__ void load_slots(const T* __restrict__ src, const Slots& s, T raw[NPOP])
{
#pragma unroll
    for (int i = 0; i < NPOP; ++i) raw[i] = src[s.idx[i]];
}

// Convert the raw loads to arithmetic precision and apply anti-bounce-back on Dirichlet walls:
// g_i = cs2_T T_w - g*_opp (adiabatic walls keep the bounced value g*_opp).
template <typename T, typename A>
__device__ __forceinline__ void finish_pull(const LatParams<A>& P, const T raw[NPOP], int wall_mask,
                                            A f[9], A g[5])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = to_a(raw[i]);
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = to_a(raw[9 + i]);
    // g2 (g4) pulled from the row below (above) is re-based to this row; bounced values are not
    g[2] = (wall_mask & 4) ? g[2] : g[2] - P.T_dyw;
    g[4] = (wall_mask & 8) ? g[4] : g[4] + P.T_dyw;
    if (wall_mask) {
        if ((wall_mask & 1) && P.kind[0] == WALL_DIRICHLET) g[1] = P.Tw_c2[0] - g[1];
        if ((wall_mask & 2) && P.kind[1] == WALL_DIRICHLET) g[3] = P.Tw_c2[1] - g[3];
        if ((wall_mask & 4) && P.kind[2] == WALL_DIRICHLET) g[2] = P.Tw_c2[2] - g[2];
        if ((wall_mask & 8) && P.kind[3] == WALL_DIRICHLET) g[4] = P.Tw_c2[3] - g[4];
        if (P.moving) {
            // moving walls: f_i = f*_opp + [f^eq_i - f^eq_opp](rho0, u_w); a diagonal that crosses
            // both a y wall and an x wall takes the y wall's velocity
            const bool L = wall_mask & 1, R = wall_mask & 2, B = wall_mask & 4, T = wall_mask & 8;
            if (L) f[1] += P.fbb[0][1];
            if (R) f[3] += P.fbb[1][3];
            if (B) f[2] += P.fbb[2][2];
            if (T) f[4] += P.fbb[3][4];
            if (L || B) f[5] += P.fbb[B ? 2 : 0][5];
            if (R || B) f[6] += P.fbb[B ? 2 : 1][6];
            if (R || T) f[7] += P.fbb[T ? 3 : 1][7];
            if (L || T) f[8] += P.fbb[T ? 3 : 0][8];
        }
    }
}

template <typename T, typename A>
__device__ __forceinline__ void gather_pull(const T* __restrict__ src, const LatParams<A>& P, int x, int y,
                                            A f[9], A g[5])
{
    const Slots s = pull_slots(P, x, y);
    T raw[NPOP];
    load_slots(src, s, raw);
    finish_pull(P, raw, s.wall_mask, f, g);
}

template <typename T, typename A>
__device__ __forceinline__ void store_node(T* __restrict__ dst, const LatParams<A>& P, int x, int y,
                                           const A f[9], const A g[5])
{
    T* here = dst + (long long)y * P.crow + chunk_off(x);
#pragma unroll
    for (int i = 0; i < 9; ++i) here[i * kRowChunk] = from_a(f[i], (T*)nullptr);
#pragma unroll
    for (int i = 0; i < 5; ++i) here[(9 + i) * kRowChunk] = from_a(g[i], (T*)nullptr);
}

// Macroscopic fields, Eqs. (3), (13), (23), from stored values (populations, or deviations from
// the rest state: sum w_i e_i = 0, so the momentum needs no correction).
template <typename A>
struct Macro {
    A rho, ux, uy, T, Fx, Fy, drho, dT;  // drho = rho - rho_b, dT = T - T_b
};

// Temperature base of row y (the T_b of deviation storage; 0 for FP64).
template <typename S>
__device__ __forceinline__ S row_base(const LatParams<S>& P, int y)
{
    return fma_(S(y), P.T_dy, P.T_b);
}

// Tb: the temperature base of the node's row (row_base), which the g deviations are taken against.
template <typename A, typename S>
__device__ __forceinline__ Macro<A> macroscopic(const LatParams<S>& P, const A f[9], const A g[5], A Tb)
{
    Macro<A> m;
    // sums over the rows of equal e_y (centre, +x, -x) as central3 forms them, and over the D2Q5
    // axis pairs as the D2Q5 collision forms them, so that the compiler shares them
    m.drho = ((f[0] + (f[1] + f[3])) + (f[2] + (f[5] + f[6]))) + (f[4] + (f[8] + f[7]));
    m.dT = (g[0] + (g[1] + g[3])) + (g[2] + g[4]);
    m.rho = A(P.rho_b) + m.drho;
    m.T = Tb + m.dT;
    m.Fx = A(P.Fvx);
    m.Fy = fma_(A(P.gb), m.T - A(P.T0), A(P.Fvy));
    const A jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const A jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[8] + f[7]);
    const A inv = rcp_(m.rho);
    m.ux = fma_(A(0.5), m.Fx, jx) * inv;
    m.uy = fma_(A(0.5), m.Fy, jy) * inv;
    return m;
}

// Three-point central moments (orders 0, 1, 2) of values c (e = 0), p (e = +1), m (e = -1) about u.
template <typename A>
__device__ __forceinline__ void central3(A c, A p, A m, A u, A& k0, A& k1, A& k2)
{
    const A s = p + m;
    const A s0 = c + s;
    const A d = p - m;
    k0 = s0;
    k1 = fma_(-u, s0, d);
    k2 = fma_(u * u, s0, fma_(A(-2) * u, d, s));
}

// (s + d) / 2 and (s - d) / 2 as two FMAs on the exact half of s: the values of the two sums halved
// (halving is exact and commutes with rounding to nearest outside the subnormal range) in three
// instructions instead of four.
template <typename A>
__device__ __forceinline__ void half_sum_diff(A s, A d, A& plus, A& minus)
{
    const A h = A(0.5) * s;
    plus = fma_(A(0.5), d, h);
    minus = fma_(A(-0.5), d, h);
}
// Packed pairs keep the sums and the halvings (same values): in the FP16 step, issue-limited on the
// FMA pipe, the three-instruction form measured 78.4 against 77.9 us.
__device__ __forceinline__ void half_sum_diff(F2 s, F2 d, F2& plus, F2& minus)
{
    plus = F2(0.5f) * (s + d);
    minus = F2(0.5f) * (s - d);
}

// Inverse of central3: raw moments about 0 (shift back by u), then the 1-D inverse moment map.
template <typename A>
__device__ __forceinline__ void uncentral3(A k0, A k1, A k2, A u, A& c, A& p, A& m)
{
    const A r1 = fma_(u, k0, k1);
    const A r2 = fma_(u * u, k0, fma_(A(2) * u, k1, k2));
    c = k0 - r2;
    half_sum_diff(r2, r1, p, m);  // p = (r2 + r1) / 2, m = (r2 - r1) / 2
}

// f = M^-1 N(u)^-1 k for central moments k[a][b] (a: x order, b: y order).
template <typename A>
__device__ __forceinline__ void back_d2q9(const A k[3][3], A ux, A uy, A f[9])
{
    // y pass: for each x order a, the x-central moment a of the rows e_y = 0, +1, -1
    A r0[3], rp[3], rm[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) uncentral3(k[a][0], k[a][1], k[a][2], uy, r0[a], rp[a], rm[a]);
    // x pass per row: (centre, +x, -x) = (0,1,3), (2,5,6), (4,8,7)
    uncentral3(r0[0], r0[1], r0[2], ux, f[0], f[1], f[3]);
    uncentral3(rp[0], rp[1], rp[2], ux, f[2], f[5], f[6]);
    uncentral3(rm[0], rm[1], rm[2], ux, f[4], f[8], f[7]);
}

template <typename A>
__device__ __forceinline__ void back_d2q5(A T, A k10, A k01, A k20, A k02, A ux, A uy, A g[5])
{
    // Each axis row shares the rest population g0; split the two 1-D inverses over it.
    const A r10 = fma_(ux, T, k10);
    const A r20 = fma_(ux * ux, T, fma_(A(2) * ux, k10, k20));
    const A r01 = fma_(uy, T, k01);
    const A r02 = fma_(uy * uy, T, fma_(A(2) * uy, k01, k02));
    g[0] = T - r20 - r02;
    half_sum_diff(r20, r10, g[1], g[3]);
    half_sum_diff(r02, r01, g[2], g[4]);
}

// D2Q9 central moments k[a][b] = sum f (e_x - u_x)^a (e_y - u_y)^b (Eq. 5b).
template <typename A>
__device__ __forceinline__ void central_d2q9(const A f[9], A ux, A uy, A k[3][3])
{
    A r0[3], rp[3], rm[3];
    central3(f[0], f[1], f[3], ux, r0[0], r0[1], r0[2]);  // row e_y = 0
    central3(f[2], f[5], f[6], ux, rp[0], rp[1], rp[2]);  // row e_y = +1
    central3(f[4], f[8], f[7], ux, rm[0], rm[1], rm[2]);  // row e_y = -1
#pragma unroll
    for (int a = 0; a < 3; ++a) central3(r0[a], rp[a], rm[a], uy, k[a][0], k[a][1], k[a][2]);
}

// D2Q5 collision in populations form (Eqs. 16-21) for temperature T and velocity u. HI1: lambda2 = 1,
// so the second-order central moments relax to equilibrium whatever their value (not formed).
template <bool HI1 = false, typename A>
__device__ __forceinline__ void collide_d2q5(const LatParams<A>& P, A T, A ux, A uy, A g[5])
{
    const A d1 = g[1] - g[3], s1 = g[1] + g[3];
    const A d2 = g[2] - g[4], s2 = g[2] + g[4];
    const A t10 = fma_(-ux, T, d1);
    const A t01 = fma_(-uy, T, d2);
    const A t20 = fma_(ux * ux, T, fma_(A(-2) * ux, d1, s1));
    const A t02 = fma_(uy * uy, T, fma_(A(-2) * uy, d2, s2));
    const A om1 = A(1) - P.lambda1;
    const A om2 = A(1) - P.lambda2;
    const A eqT = P.lambda2 * T * P.cs2T;
    if constexpr (HI1) back_d2q5(T, om1 * t10, om1 * t01, eqT, eqT, ux, uy, g);
    else back_d2q5(T, om1 * t10, om1 * t01, fma_(om2, t20, eqT), fma_(om2, t02, eqT), ux, uy, g);
}

// Collision of one node in place, populations form: Eqs. (6)-(11) for f, Eqs. (16)-(21) for g.
// HI1: the high-order rates are 1 (s_3 = s_4 = lambda2 = 1, the paper's setting, Sec. 3), so k~21,
// k~12, k~22 and the second-order D2Q5 moments relax to their equilibrium and forcing terms
// whatever their value; they are then not formed (the compiler drops that part of the forward
// transforms). The results are the same as with HI1 = false: (1 - s) k is an exact zero for s = 1.
template <bool HI1 = false, typename A>
__device__ __forceinline__ void collide(const LatParams<A>& P, A f[9], A g[5], A Tb)
{
    const Macro<A> m = macroscopic(P, f, g, Tb);
    const A ux = m.ux, uy = m.uy, rho = m.rho, T = m.T;
    const A cs2 = A(1) / A(3);
    A k[3][3];
    central_d2q9(f, ux, uy, k);

    // relaxation, Eq. (8), equilibrium Eq. (9), forcing Eq. (11)
    const A a20 = fma_(-rho, cs2, k[2][0]);
    const A a02 = fma_(-rho, cs2, k[0][2]);
    A q[3][3];
    q[0][0] = rho;
    q[1][0] = k[1][0] + m.Fx;
    q[0][1] = k[0][1] + m.Fy;
    q[2][0] = fma_(-P.sm, a02, fma_(-P.sp, a20, k[2][0]));
    q[0][2] = fma_(-P.sp, a02, fma_(-P.sm, a20, k[0][2]));
    q[1][1] = (A(1) - P.s_nu) * k[1][1];
    const A half3 = (A(1) - A(0.5) * P.s_3) * cs2;
    if constexpr (HI1) {
        q[2][1] = half3 * m.Fy;
        q[1][2] = half3 * m.Fx;
        q[2][2] = P.s_4 * rho * (cs2 * cs2);
    } else {
        q[2][1] = fma_(A(1) - P.s_3, k[2][1], half3 * m.Fy);
        q[1][2] = fma_(A(1) - P.s_3, k[1][2], half3 * m.Fx);
        q[2][2] = fma_(A(1) - P.s_4, k[2][2], P.s_4 * rho * (cs2 * cs2));
    }
    back_d2q9(q, ux, uy, f);

    collide_d2q5<HI1>(P, T, ux, uy, g);
}

// Deviation of the D2Q9 equilibrium from the rest state, f^eq_i(rho, u) - w_i rho_b, written as
// small terms only: f^eq_i = rho p(e_x; u_x) p(e_y; u_y) with the 1-D equilibrium
// p(0) = w(0) - u^2, p(+-1) = w(1) + (u^2 +- u)/2 (the product form of the moments of Eq. 9).
template <typename A>
__device__ __forceinline__ void eq_dev_d2q9(A rho, A drho, A ux, A uy, A f[9])
{
    const A w0 = A(2.0 / 3.0), w1 = A(1.0 / 6.0);
    const A x2 = ux * ux, y2 = uy * uy;
    A dx[3], dy[3];  // e = 0, +1, -1: -u^2, (u^2 + u) / 2, (u^2 - u) / 2
    dx[0] = -x2;
    dy[0] = -y2;
    half_sum_diff(x2, ux, dx[1], dx[2]);
    half_sum_diff(y2, uy, dy[1], dy[2]);
    const A wv[3] = {w0, w1, w1};
    const int ax[9] = {0, 1, 0, 2, 0, 1, 2, 2, 1};
    const int ay[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const A wx = wv[ax[i]], wy = wv[ay[i]], ex = dx[ax[i]], ey = dy[ay[i]];
        f[i] = fma_(drho, wx * wy, rho * fma_(ex, ey, fma_(wx, ey, ex * wy)));
    }
}

// Deviation of the D2Q5 equilibrium from the rest state, g^eq_i(T, u) - w^T_i T_b.
template <typename A>
__device__ __forceinline__ void eq_dev_d2q5(A T, A dT, A ux, A uy, A c2, A g[5])
{
    const A hc = A(0.5) * c2;
    const A hT = A(0.5) * T;
    g[0] = fma_(dT, A(1) - A(2) * c2, -T * fma_(ux, ux, uy * uy));
    g[1] = fma_(dT, hc, hT * fma_(ux, ux, ux));
    g[3] = fma_(dT, hc, hT * fma_(ux, ux, -ux));
    g[2] = fma_(dT, hc, hT * fma_(uy, uy, uy));
    g[4] = fma_(dT, hc, hT * fma_(uy, uy, -uy));
}

// D2Q5 collision on deviations t = g - w^T T_b (Eqs. 16-21) for T = T_b + dT and velocity u (HI1:
// lambda2 = 1, as in collide_d2q5).
template <bool HI1 = false, typename A, typename S>
__device__ __forceinline__ void collide_d2q5_dev(const LatParams<S>& P, A T, A dT, A ux, A uy, A g[5])
{
    const A c2 = A(P.cs2T);
    const A x2 = ux * ux, y2 = uy * uy;
    const A d1 = g[1] - g[3], s1 = g[1] + g[3];
    const A d2 = g[2] - g[4], s2 = g[2] + g[4];
    const A t10 = fma_(-ux, T, d1);
    const A t01 = fma_(-uy, T, d2);
    const A t20 = fma_(-dT, c2, fma_(x2, T, fma_(A(-2) * ux, d1, s1)));
    const A t02 = fma_(-dT, c2, fma_(y2, T, fma_(A(-2) * uy, d2, s2)));
    const A om1 = A(1.0f - P.lambda1);
    const A om2 = A(1.0f - P.lambda2);
    A eT[5], gq[5];
    eq_dev_d2q5(T, dT, ux, uy, c2, eT);
    if constexpr (HI1) back_d2q5(A(0), om1 * t10, om1 * t01, A(0), A(0), ux, uy, gq);
    else back_d2q5(A(0), om1 * t10, om1 * t01, om2 * t20, om2 * t02, ux, uy, gq);
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = gq[i] + eT[i];
}

// Collision of one node in place, deviation form (h = f - w rho_b, t = g - w^T T_b). The same map
// as `collide`: Gamma~* = Gamma~eq + (I - S)(Gamma~ - Gamma~eq) + (I - S/2) C, so
// f* = f^eq + M^-1 N^-1 [(I - S)(Gamma~ - Gamma~eq) + (I - S/2) C]; the non-equilibrium central
// moments are formed from the central moments of h plus those of w rho_b about u
// (1-D: 1, -u, 1/3 + u^2) minus Eq. (9), with the O(1) parts cancelled analytically.
template <bool HI1 = false, typename A, typename S>
__device__ __forceinline__ void collide_dev(const LatParams<S>& P, A f[9], A g[5], A Tb)
{
    const Macro<A> m = macroscopic(P, f, g, Tb);
    const A ux = m.ux, uy = m.uy, rho = m.rho, T = m.T, dr = m.drho, dT = m.dT;
    const A rb = A(P.rho_b);
    const A cs2 = A(1.0 / 3.0), cs4 = A(1.0 / 9.0);
    const A x2 = ux * ux, y2 = uy * uy;
    A k[3][3];
    central_d2q9(f, ux, uy, k);
    // non-equilibrium central moments d = k(h) + rho_b k(w) - Gamma~eq
    const A d10 = fma_(-rb, ux, k[1][0]);
    const A d01 = fma_(-rb, uy, k[0][1]);
    const A d20 = fma_(-dr, cs2, fma_(rb, x2, k[2][0]));
    const A d02 = fma_(-dr, cs2, fma_(rb, y2, k[0][2]));
    const A d11 = fma_(rb * ux, uy, k[1][1]);
    // relaxed non-equilibrium plus forcing, Eqs. (8), (11)
    const A sp = A(P.sp), sm = A(P.sm);
    const A half3 = A((1.0f - 0.5f * P.s_3) * (1.0f / 3.0f));
    A q[3][3];
    q[0][0] = A(0);
    q[1][0] = d10 + m.Fx;
    q[0][1] = d01 + m.Fy;
    q[2][0] = fma_(-sm, d02, fma_(-sp, d20, d20));
    q[0][2] = fma_(-sp, d02, fma_(-sm, d20, d02));
    q[1][1] = A(1.0f - P.s_nu) * d11;
    if constexpr (HI1) {
        // s_3 = s_4 = 1: (1 - s) d is an exact zero (see collide)
        q[2][1] = half3 * m.Fy;
        q[1][2] = half3 * m.Fx;
        q[2][2] = A(0);
    } else {
        const A d21 = fma_(-rb * (cs2 + x2), uy, k[2][1]);
        const A d12 = fma_(-rb * ux, cs2 + y2, k[1][2]);
        const A d22 = fma_(rb, fma_(cs2, x2 + y2, x2 * y2), fma_(-dr, cs4, k[2][2]));
        q[2][1] = fma_(A(1.0f - P.s_3), d21, half3 * m.Fy);
        q[1][2] = fma_(A(1.0f - P.s_3), d12, half3 * m.Fx);
        q[2][2] = A(1.0f - P.s_4) * d22;
    }
    A e[9];
    eq_dev_d2q9(rho, dr, ux, uy, e);
    back_d2q9(q, ux, uy, f);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] += e[i];

    collide_d2q5_dev<HI1>(P, T, dT, ux, uy, g);
}

template <bool DEV, bool HI1 = false, typename A>
__device__ __forceinline__ void collide_any(const LatParams<A>& P, A f[9], A g[5], A Tb)
{
    if constexpr (DEV) collide_dev<HI1>(P, f, g, Tb);
    else collide<HI1>(P, f, g, Tb);
}

// Equilibria in stored form, minus the rest state for deviation storage: f^eq(rho, u) (Eq. 9
// back-transformed), and g^eq(T, u) (Eq. 20) with dT = T - (the temperature base of the row).
template <bool DEV, typename A>
__device__ __forceinline__ void eq_f(const LatParams<A>& P, A rho, A ux, A uy, A f[9])
{
    if (DEV) {
        eq_dev_d2q9(rho, rho - P.rho_b, ux, uy, f);
    } else {
        const A cs2 = A(1) / A(3);
        A k[3][3] = {{rho, A(0), rho * cs2}, {A(0), A(0), A(0)}, {rho * cs2, A(0), rho * cs2 * cs2}};
        back_d2q9(k, ux, uy, f);
    }
}
template <bool DEV, typename A>
__device__ __forceinline__ void eq_g(const LatParams<A>& P, A T, A dT, A ux, A uy, A g[5])
{
    if (DEV) eq_dev_d2q5(T, dT, ux, uy, P.cs2T, g);
    else back_d2q5(T, A(0), A(0), T * P.cs2T, T * P.cs2T, ux, uy, g);
}
template <bool DEV, typename A>
__device__ __forceinline__ void equilibrium(const LatParams<A>& P, A rho, A ux, A uy, A T, A f[9],
                                            A g[5], A Tb)
{
    eq_f<DEV>(P, rho, ux, uy, f);
    eq_g<DEV>(P, T, T - Tb, ux, uy, g);
}

// Wet walls (the paper's own conditions, Sec. 3 first paragraph): the wall lies on the end row
// (column) of nodes. The populations that would come from beyond the wall are set by
// non-equilibrium bounce-back, f_i = f_opp + [f^eq_i - f^eq_opp](rho, u') with u' = u_w - F/(2 rho)
// (so that the force-corrected velocity of Eq. 13 is the wall's), rho from mass and normal
// momentum, and the tangential momentum closed on the two diagonals. g at the wall node is set by
// non-equilibrium extrapolation from the fluid node q next to it: g_i = g^eq_i(T_w, u_w) +
// [g_i(q) - g^eq_i(T(q), u(q))]. A corner node (on an x wall and a y wall) takes the y wall's
// velocity and the mean of the two walls' temperatures, rho from its diagonal neighbour q, the
// unknowns whose opposite is known by non-equilibrium bounce-back and the two buried diagonals
// half the remaining mass each; g by extrapolation from q. All in stored form (the rest state
// cancels in both rules).
template <bool DEV, typename T, typename A>
__device__ __forceinline__ void gather_wet(const T* __restrict__ src, const LatParams<A>& P, int x, int y,
                                           A f[9], A g[5])
{
    const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const bool onx = P.wet_x && (x == 0 || x == P.nx - 1);
    const bool ony = P.wet_y && (y == 0 || y == P.ny - 1);
    const int sx = x == 0 ? 1 : -1, sy = y == 0 ? 1 : -1;  // directions into the fluid
    const int side_x = x == 0 ? 0 : 1, side_y = y == 0 ? 2 : 3;
    const int side = ony ? side_y : side_x;
    A fw[9], gw[5];
    gather_pull(src, P, x, y, fw, gw);
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = fw[i];
    // wall temperature, and its difference from the row's base (a corner has a flat base: the
    // base slopes only between y walls with periodic x)
    const A Tw = (onx && ony) ? A(0.5) * (P.Twall[side_x] + P.Twall[side_y]) : P.Twall[side];
    const A dTw = (onx && ony) ? Tw - P.T_b : P.dTw[side];
    const A uwx = P.uwall[side][0], uwy = P.uwall[side][1];
    const A Fx = P.Fvx, Fy = fma_(P.gb, Tw - P.T0, P.Fvy);
    A fq[9], gq[5];
    gather_pull(src, P, onx ? x + sx : x, ony ? y + sy : y, fq, gq);  // q: never a wall node
    const int qy = ony ? y + sy : y;
    const Macro<A> mq = macroscopic(P, fq, gq, row_base(P, qy));
    A feq[9];
    if (onx && ony) {
        const A rho = mq.rho;
        const A inv = rcp_(rho);
        eq_f<DEV>(P, rho, fma_(A(-0.5) * Fx, inv, uwx), fma_(A(-0.5) * Fy, inv, uwy), feq);
        // unknown: pulled from beyond a wall; buried: unknown with an unknown opposite
        A known = A(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const bool unk = EX[i] == sx || EY[i] == sy;
            const bool unk_o = -EX[i] == sx || -EY[i] == sy;
            if (unk && !unk_o) f[i] = f[OPP[i]] + (feq[i] - feq[OPP[i]]);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const bool buried = (EX[i] == sx || EY[i] == sy) && (-EX[i] == sx || -EY[i] == sy);
            if (!buried) known += f[i];
        }
        const A half = A(0.5) * ((rho - A(P.rho_b)) - known);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            if ((EX[i] == sx || EY[i] == sy) && (-EX[i] == sx || -EY[i] == sy)) f[i] = half;
    } else {
        const int nrm = onx ? sx : sy;
        const A Fa = onx ? Fx : Fy, uwa = onx ? uwx : uwy;
        A Z = A(0), O = A(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ea = onx ? EX[i] : EY[i];
            if (ea == 0) Z += f[i];
            if (ea == -nrm) O += f[i];
        }
        const A num = fma_(-A(nrm) * A(0.5), Fa, fma_(A(2), O, Z) + P.rho_b);
        const A rho = num * rcp_(fma_(-A(nrm), uwa, A(1)));
        const A inv = rcp_(rho);
        const A upx = fma_(A(-0.5) * Fx, inv, uwx), upy = fma_(A(-0.5) * Fy, inv, uwy);
        eq_f<DEV>(P, rho, upx, upy, feq);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            if ((onx ? EX[i] : EY[i]) == nrm) f[i] = f[OPP[i]] + (feq[i] - feq[OPP[i]]);
        A St = A(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int et = onx ? EY[i] : EX[i];
            if (et == 1) St += f[i];
            if (et == -1) St -= f[i];
        }
        const A delta = A(0.5) * fma_(rho, onx ? upy : upx, -St);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int et = onx ? EY[i] : EX[i];
            if ((onx ? EX[i] : EY[i]) == nrm && et != 0) f[i] = et > 0 ? f[i] + delta : f[i] - delta;
        }
    }
    A geqq[5], geqb[5];
    eq_g<DEV>(P, mq.T, mq.dT, mq.ux, mq.uy, geqq);
    eq_g<DEV>(P, Tw, dTw, uwx, uwy, geqb);
#pragma unroll
    for (int i = 0; i < 5; ++i) g[i] = geqb[i] + (gq[i] - geqq[i]);
}

// Pre-collision populations of node (x, y) at the current time, wall rules included.
template <typename T, typename A>
__device__ __forceinline__ void gather(const T* __restrict__ src, const LatParams<A>& P, int x, int y,
                                       A f[9], A g[5])
{
    constexpr bool DEV = sizeof(T) < sizeof(double);
    if ((P.wet_y && (y == 0 || y == P.ny - 1)) || (P.wet_x && (x == 0 || x == P.nx - 1)))
        gather_wet<DEV>(src, P, x, y, f, g);
    else gather_pull(src, P, x, y, f, g);
}

// Weight of node (x, y) in the Eq. 29 average: wet walls lie on the end rows (columns) of nodes,
// so along a wet direction the average over [0, H] is the trapezoid rule (half weight there).
template <typename A>
__device__ __forceinline__ double wet_weight(const LatParams<A>& P, int x, int y)
{
    const double wy = (P.wet_y && (y == 0 || y == P.ny - 1)) ? 0.5 : 1.0;
    const double wx = (P.wet_x && (x == 0 || x == P.nx - 1)) ? 0.5 : 1.0;
    return wx * wy;
}

}  // namespace clb
