// clb_kernels.cuh -- the kernels of one lattice: fused collide-and-stream step (direct and staged
// rows), equilibrium initialisation, field and population extraction. The FP64 diagnostics
// (Nusselt number of Eq. 29 and the steady-state residual) are in clb_diag.cuh.
#pragma once

#include "clb_core.cuh"
#include "clb_host.h"

namespace clb {

// V consecutive elements loaded or stored as one aligned vector access.
template <typename E, int V>
struct alignas(sizeof(E) * V) Pack {
    E e[V];
};

template <typename E>
__device__ __forceinline__ E lane_up(E v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename E>
__device__ __forceinline__ E lane_down(E v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// One time step for V consecutive nodes x0 .. x0+V-1 of row y, called by all 32 lanes of a warp
// on the same row with x0 = (first x of the warp) + lane * V: pull the 14 populations (Eqs. 12,
// 22, with the wall rules), collide (Eqs. 3-11, 13, 16-21, 23), store at the nodes.
// Warps whose 32 * V nodes all lie inside the row take the vector path: per population plane one
// aligned V-wide load of the row the pull comes from; the population pulled from x-1 (x+1) of the
// first (last) node of a thread is the neighbouring lane's last (first) element, passed by a warp
// shuffle, and lane 0 (lane 31) loads the one element beyond the warp. Walls are handled in the
// same path: on a wall row the planes pulled across the wall come from the node's own opposite
// plane (no shift), and at an x wall lane 0 (lane 31) loads its node's own opposite values instead
// of the missing neighbour; the wall terms are then added per node by finish_pull. The ragged end
// of a row gathers node by node. Every path feeds identical values to the identical collision.
//
// warp_vector is the vector body. WALLS = false is the interior of the lattice (no wall next to any node of the
// warp), where every wall term folds away at compile time.
template <int ST, int V, bool WALLS, bool HI1 = false>
__device__ __forceinline__ void warp_vector(const typename Storage<ST>::T* __restrict__ src,
                                            typename Storage<ST>::T* __restrict__ dst,
                                            const LatParams<typename Storage<ST>::A>& P, int x0, int y,
                                            int lane, int keep)
{
    using A = typename Storage<ST>::A;
    using E = typename Storage<ST>::T;
    using PK = Pack<E, V>;
    const int wx0 = x0 - lane * V, wx1 = wx0 + 32 * V - 1;
    {
        const bool wallB = WALLS && !P.per_y && y == 0;
        const bool wallT = WALLS && !P.per_y && y == P.ny - 1;
        const bool wallL = WALLS && !P.per_x && wx0 == 0;
        const bool wallR = WALLS && !P.per_x && wx1 == P.nx - 1;
        const int ym = y > 0 ? y - 1 : P.ny - 1;
        const int yp = y < P.ny - 1 ? y + 1 : 0;
        const long long rc = (long long)y * P.crow, rm = (long long)ym * P.crow, rp = (long long)yp * P.crow;
        const int xl = wx0 > 0 ? wx0 - 1 : P.nx - 1;  // column left of the warp (lane 0)
        const int xr = wx1 < P.nx - 1 ? wx1 + 1 : 0;  // column right of the warp (lane 31)
        // the thread's V nodes lie in one chunk (x0 and kRowChunk are multiples of V), so each
        // population of them is one aligned V-wide vector at a fixed offset from these addresses
        const E* sc = src + rc + chunk_off(x0);
        const E* sm = src + rm + chunk_off(x0);
        const E* sp = src + rp + chunk_off(x0);
        // plane, row (0: y, 1: y-1, 2: y+1) and x shift (+1: pulled from x-1, -1: from x+1)
        const int SHIFT[NPOP] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 0, 1, 0, -1, 0};
        const int ROWSEL[NPOP] = {0, 0, 1, 0, 2, 1, 1, 2, 2, 0, 0, 1, 0, 2};
        const int OPP[NPOP] = {0, 3, 4, 1, 2, 7, 8, 5, 6, 9, 12, 13, 10, 11};
        PK pk[NPOP];
        E edge[NPOP];
#pragma unroll
        for (int i = 0; i < NPOP; ++i) {
            // a pull across the bottom (top) wall reads the node's own opposite plane
            const bool across = (wallB && ROWSEL[i] == 1) || (wallT && ROWSEL[i] == 2);
            const int plane = across ? OPP[i] : i;
            const bool rowc = across || ROWSEL[i] == 0;
            const long long r = rowc ? rc : ROWSEL[i] == 1 ? rm : rp;
            const E* sr = rowc ? sc : ROWSEL[i] == 1 ? sm : sp;
            const int sh = across ? 0 : SHIFT[i];
            pk[i] = *reinterpret_cast<const PK*>(sr + plane * kRowChunk);
            edge[i] = E(0);
            if (sh == 1 && lane == 0)
                edge[i] = wallL ? src[rc + chunk_off(0) + OPP[i] * kRowChunk] : src[r + chunk_off(xl) + plane * kRowChunk];
            if (sh == -1 && lane == 31)
                edge[i] = wallR ? src[rc + chunk_off(P.nx - 1) + OPP[i] * kRowChunk] : src[r + chunk_off(xr) + plane * kRowChunk];
        }
        E raw[V][NPOP];
#pragma unroll
        for (int i = 0; i < NPOP; ++i) {
            const bool across = (wallB && ROWSEL[i] == 1) || (wallT && ROWSEL[i] == 2);
            const int sh = across ? 0 : SHIFT[i];
            // the shuffles run on every lane whatever the shift, so that all lanes take part
            const E up = lane_up(pk[i].e[V - 1]);
            const E dn = lane_down(pk[i].e[0]);
            if (sh == 0) {
#pragma unroll
                for (int k = 0; k < V; ++k) raw[k][i] = pk[i].e[k];
            } else if (sh == 1) {
                raw[0][i] = lane == 0 ? edge[i] : up;
#pragma unroll
                for (int k = 1; k < V; ++k) raw[k][i] = pk[i].e[k - 1];
            } else {
                raw[V - 1][i] = lane == 31 ? edge[i] : dn;
#pragma unroll
                for (int k = 0; k < V - 1; ++k) raw[k][i] = pk[i].e[k + 1];
            }
        }
        const int rowmask = (wallB ? 4 : 0) | (wallT ? 8 : 0);
        int mask[V];
#pragma unroll
        for (int k = 0; k < V; ++k)
            mask[k] = rowmask | ((wallL && lane == 0 && k == 0) ? 1 : 0) | ((wallR && lane == 31 && k == V - 1) ? 2 : 0);
        PK out[NPOP];
        const A Tb = row_base(P, y);
        if constexpr (Storage<ST>::DEV && V % 2 == 0) {
            // FP32 arithmetic: two nodes per packed f32x2 instruction
#pragma unroll
            for (int k = 0; k < V; k += 2) {
                A fa[9], ga[5], fb[9], gb[5];
                finish_pull(P, raw[k], mask[k], fa, ga);
                finish_pull(P, raw[k + 1], mask[k + 1], fb, gb);
                F2 f[9], g[5];
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = F2(fa[i], fb[i]);
#pragma unroll
                for (int i = 0; i < 5; ++i) g[i] = F2(ga[i], gb[i]);
                collide_dev<HI1>(P, f, g, F2(Tb));
#pragma unroll
                for (int i = 0; i < NPOP; ++i) from_a2(i < 9 ? f[i] : g[i - 9], out[i].e[k], out[i].e[k + 1]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                A f[9], g[5];
                finish_pull(P, raw[k], mask[k], f, g);
                collide_any<Storage<ST>::DEV, HI1>(P, f, g, Tb);
#pragma unroll
                for (int i = 0; i < 9; ++i) out[i].e[k] = from_a(f[i], (E*)nullptr);
#pragma unroll
                for (int i = 0; i < 5; ++i) out[9 + i].e[k] = from_a(g[i], (E*)nullptr);
            }
        }
        if (x0 >= keep) {
            E* dc = dst + rc + chunk_off(x0);
#pragma unroll
            for (int i = 0; i < NPOP; ++i) *reinterpret_cast<PK*>(dc + i * kRowChunk) = out[i];
        }
    }
}

// step_warp_nodes picks the path. SPLIT = true compiles the vector body twice, with and without
// the wall terms, and interior warps take the lean copy (fewer instructions; the FP16 form is
// issue-limited). Nodes x < keep are computed but not stored (they belong to another warp: see the
// shifted last tile of a row in the batched kernel).
template <int ST, int V, bool SPLIT = true, bool HI1 = false>
__device__ __forceinline__ void step_warp_nodes(const typename Storage<ST>::T* __restrict__ src,
                                                typename Storage<ST>::T* __restrict__ dst,
                                                const LatParams<typename Storage<ST>::A>& P, int x0,
                                                int y, int lane, int keep = 0)
{
    using A = typename Storage<ST>::A;
    const int wx0 = x0 - lane * V, wx1 = wx0 + 32 * V - 1;
    // warps on a wet row or touching a wet column gather node by node (gather_wet)
    if (wx1 < P.nx && !(P.wet_y && (y == 0 || y == P.ny - 1)) && !(P.wet_x && (wx0 == 0 || wx1 == P.nx - 1))) {
        const bool walls =
            (!P.per_y && (y == 0 || y == P.ny - 1)) || (!P.per_x && (wx0 == 0 || wx1 == P.nx - 1));
        if (!SPLIT || walls) warp_vector<ST, V, true, HI1>(src, dst, P, x0, y, lane, keep);
        else warp_vector<ST, V, false, HI1>(src, dst, P, x0, y, lane, keep);
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int x = x0 + k;
            if (x < P.nx && x >= keep) {
                A f[9], g[5];
                gather(src, P, x, y, f, g);
                collide_any<Storage<ST>::DEV, HI1>(P, f, g, row_base(P, y));
                store_node(dst, P, x, y, f, g);
            }
        }
    }
}

// One time step over the lattice: thread (tx, ty) of block (bx, by) updates nodes
// x0 = (bx * blockDim.x + tx) * V .. x0 + V - 1 of row by * blockDim.y + ty. blockDim.x is a
// multiple of 32, so each warp lies in one row.
// HI1: the form for high-order rates of 1 (see collide), which the host picks when
// s_3 = s_4 = lambda2 = 1.
template <int ST, int V, bool HI1>
__global__ void __launch_bounds__(256) k_step(const typename Storage<ST>::T* __restrict__ src,
                                              typename Storage<ST>::T* __restrict__ dst,
                                              const LatParams<typename Storage<ST>::A> P)
{
    const int lane = threadIdx.x & 31;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (y >= P.ny || x0 - lane * V >= P.nx) return;  // whole warps only
    step_warp_nodes<ST, V, true, HI1>(src, dst, P, x0, y, lane);
}

// Split step. The warps of the interior of the lattice (32 V nodes inside the row, no wall next to
// any of them: not on a wall row, not in a wall column, not at a ragged row end) run in
// k_step_inner, which holds only the wall-free vector body; the other warps run in k_step_edge,
// which holds every path. Compiled into one kernel, the wall and node-by-node paths raise the
// register pressure of the whole kernel and push spills into the interior path (FP16 at 96
// registers: 80 bytes of spills with them, 20 without; 83.1 -> 77.6 us per step on 4096 x 2048).
// The two kernels update disjoint sets of nodes from the same source buffer, so the host runs them
// side by side on two streams. Each node's arithmetic is the same as in k_step.
struct SplitGeom {
    int y0, y1;    // interior rows [y0, y1)
    int c0, c1;    // interior warp columns [c0, c1) (warp column c: nodes c 32 V .. c 32 V + 32 V - 1)
    int nw;        // warp columns per row
    int yb[2], nyb;  // wall rows, every column in k_step_edge
    int cb[2], ncb;  // edge columns of the interior rows
    __host__ __device__ int edge_warps() const { return nyb * nw + (y1 - y0) * ncb; }
};

// Interior warps: thread (tx, ty) of block (bx, by) is lane tx % 32 of warp column
// c0 + (bx blockDim.x + tx) / 32 in row y0 + by blockDim.y + ty.
template <int ST, int V, bool HI1>
__global__ void __launch_bounds__(256) k_step_inner(const typename Storage<ST>::T* __restrict__ src,
                                                    typename Storage<ST>::T* __restrict__ dst,
                                                    const LatParams<typename Storage<ST>::A> P, int y0, int y1,
                                                    int c0, int c1)
{
    const int lane = threadIdx.x & 31;
    const int c = c0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
    if (y >= y1 || c >= c1) return;  // whole warps only
    warp_vector<ST, V, false, HI1>(src, dst, P, c * 32 * V + lane * V, y, lane, 0);
}

// The FP16 form with 4 nodes per thread (its default) and high-order rates of 1, held at 96
// registers: 5 blocks of 128 per SM instead of 4 (120 registers uncapped), 20 bytes of spills.
static __global__ void __maxnreg__(96) k_step_inner_f16x4_hi1(const __half* __restrict__ src, __half* __restrict__ dst,
                                                              const LatParams<float> P, int y0, int y1, int c0, int c1)
{
    const int lane = threadIdx.x & 31;
    const int c = c0 + (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
    if (y >= y1 || c >= c1) return;  // whole warps only
    warp_vector<ST_F16DEV, 4, false, true>(src, dst, P, c * 32 * 4 + lane * 4, y, lane, 0);
}

// Edge warps, one per 32 threads: the wall rows first (every column), then the edge columns of the
// interior rows.
template <int ST, int V, bool HI1>
__global__ void __launch_bounds__(128) k_step_edge(const typename Storage<ST>::T* __restrict__ src,
                                                   typename Storage<ST>::T* __restrict__ dst,
                                                   const LatParams<typename Storage<ST>::A> P, const SplitGeom G)
{
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nr = G.nyb * G.nw;
    int y, c;
    if (w < nr) {
        y = G.yb[w / G.nw];
        c = w % G.nw;
    } else {
        const int v = w - nr;
        if (v >= (G.y1 - G.y0) * G.ncb) return;  // whole warps only
        y = G.y0 + v / G.ncb;
        c = G.cb[v % G.ncb];
    }
    step_warp_nodes<ST, V, true, HI1>(src, dst, P, c * 32 * V + lane * V, y, lane);
}

// ---------------------------------------------------------------------------------------------
// Pipelined variant: each warp marches down R rows of its column segment of 32 * V nodes, staging
// the pulled values of the next rows in shared memory with asynchronous copies (cp.async, tracked
// per thread by commit/wait groups) while it computes the current row. Each thread copies its own
// V-wide vector of every plane; lane 0 and lane 31 also copy the element just outside the warp
// (for FP16 the aligned 4-byte pair that holds it). The values that reach the collision are exactly
// those of step_warp_nodes, so the results are bitwise the same; the staging only keeps more bytes
// in flight per SM than registers allow.

__device__ __forceinline__ void cp_async_bytes(void* smem, const void* gmem, int bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (bytes == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
    else if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename E, int V>
struct StageGeom {
    static constexpr int EDGE = 16 / sizeof(E);      // edge slot: left value(s), then right value(s)
    static constexpr int PS = 32 * V + EDGE;         // elements per plane
    static constexpr int SS = NPOP * PS;             // elements per stage
    static constexpr int RIGHT = EDGE / 2;           // offset of the right edge in the slot
};

constexpr int kPipeWarps = 4;  // warps per block of the pipelined kernel

template <int ST, int V>
__device__ __forceinline__ void stage_issue(const typename Storage<ST>::T* __restrict__ src,
                                            const LatParams<typename Storage<ST>::A>& P, int wx0,
                                            int y, int lane, typename Storage<ST>::T* stage)
{
    using E = typename Storage<ST>::T;
    using G = StageGeom<E, V>;
    const int wx1 = wx0 + 32 * V - 1;
    const int ym = y > 0 ? y - 1 : P.ny - 1;
    const int yp = y < P.ny - 1 ? y + 1 : 0;
    const long long rc = (long long)y * P.crow, rm = (long long)ym * P.crow, rp = (long long)yp * P.crow;
    const int xl = wx0 > 0 ? wx0 - 1 : P.nx - 1;
    const int xr = wx1 < P.nx - 1 ? wx1 + 1 : 0;
    const int SHIFT[NPOP] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 0, 1, 0, -1, 0};
    const int ROWSEL[NPOP] = {0, 0, 1, 0, 2, 1, 1, 2, 2, 0, 0, 1, 0, 2};
    constexpr bool HALF = sizeof(E) == 2;
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const long long r = ROWSEL[i] == 0 ? rc : ROWSEL[i] == 1 ? rm : rp;
        const E* row = src + r + i * kRowChunk;  // population i of the row: at chunk_off(x) from here
        E* sp = stage + i * G::PS;
        constexpr int VB = V * (int)sizeof(E);  // 4, 8, 16 or 32 bytes: copy in pieces of <= 16
#pragma unroll
        for (int c = 0; c < (VB > 16 ? VB / 16 : 1); ++c)
            cp_async_bytes(sp + lane * V + c * (16 / (int)sizeof(E)), row + chunk_off(wx0 + lane * V) + c * (16 / (int)sizeof(E)),
                           VB > 16 ? 16 : VB);
        // an aligned half pair lies inside one chunk (kRowChunk is even)
        if (SHIFT[i] == 1 && lane == 0)
            cp_async_bytes(sp + 32 * V, row + chunk_off(HALF ? (xl & ~1) : xl), HALF ? 4 : (int)sizeof(E));
        if (SHIFT[i] == -1 && lane == 31)
            cp_async_bytes(sp + 32 * V + G::RIGHT, row + chunk_off(HALF ? (xr & ~1) : xr), HALF ? 4 : (int)sizeof(E));
    }
}

template <int ST, int V>
__device__ __forceinline__ void stage_compute(typename Storage<ST>::T* __restrict__ dst,
                                              const LatParams<typename Storage<ST>::A>& P, int wx0,
                                              int y, int lane, const typename Storage<ST>::T* stage)
{
    using A = typename Storage<ST>::A;
    using E = typename Storage<ST>::T;
    using G = StageGeom<E, V>;
    using PK = Pack<E, V>;
    const int wx1 = wx0 + 32 * V - 1;
    const int xl = wx0 > 0 ? wx0 - 1 : P.nx - 1;
    const int xr = wx1 < P.nx - 1 ? wx1 + 1 : 0;
    constexpr bool HALF = sizeof(E) == 2;
    const int il = 32 * V + (HALF ? (xl & 1) : 0);
    const int ir = 32 * V + G::RIGHT + (HALF ? (xr & 1) : 0);
    const int SHIFT[NPOP] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 0, 1, 0, -1, 0};
    E raw[V][NPOP];
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const E* sp = stage + i * G::PS;
        const int b = lane * V;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            int idx = b + k;
            if (SHIFT[i] == 1) idx = (k == 0 && lane == 0) ? il : b + k - 1;
            if (SHIFT[i] == -1) idx = (k == V - 1 && lane == 31) ? ir : b + k + 1;
            raw[k][i] = sp[idx];
        }
    }
    const int x0 = wx0 + lane * V;
    PK out[NPOP];
    const A Tb = row_base(P, y);
    if constexpr (Storage<ST>::DEV && V % 2 == 0) {
#pragma unroll
        for (int k = 0; k < V; k += 2) {
            F2 f[9], g[5];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = F2(to_a(raw[k][i]), to_a(raw[k + 1][i]));
#pragma unroll
            for (int i = 0; i < 5; ++i) g[i] = F2(to_a(raw[k][9 + i]), to_a(raw[k + 1][9 + i]));
            // rows here have no wall: g2 and g4 are pulled from the rows below and above
            g[2] = g[2] - F2(P.T_dyw);
            g[4] = g[4] + F2(P.T_dyw);
            collide_dev(P, f, g, F2(Tb));
#pragma unroll
            for (int i = 0; i < NPOP; ++i) {
                float lo, hi;
                (i < 9 ? f[i] : g[i - 9]).split(lo, hi);
                out[i].e[k] = from_a(lo, (E*)nullptr);
                out[i].e[k + 1] = from_a(hi, (E*)nullptr);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            A f[9], g[5];
            finish_pull(P, raw[k], 0, f, g);
            collide_any<Storage<ST>::DEV>(P, f, g, Tb);
#pragma unroll
            for (int i = 0; i < 9; ++i) out[i].e[k] = from_a(f[i], (E*)nullptr);
#pragma unroll
            for (int i = 0; i < 5; ++i) out[9 + i].e[k] = from_a(g[i], (E*)nullptr);
        }
    }
    E* dc = dst + (long long)y * P.crow + chunk_off(x0);
#pragma unroll
    for (int i = 0; i < NPOP; ++i) *reinterpret_cast<PK*>(dc + i * kRowChunk) = out[i];
}

// Block = kPipeWarps warps side by side along x; block (bx, by) covers columns
// [bx * kPipeWarps * 32 * V, ...) and rows [by * R, by * R + R). S stages of shared memory per warp.
template <int ST, int V, int S>
__global__ void __launch_bounds__(kPipeWarps * 32) k_step_pipe(const typename Storage<ST>::T* __restrict__ src,
                                                               typename Storage<ST>::T* __restrict__ dst,
                                                               const LatParams<typename Storage<ST>::A> P,
                                                               int R)
{
    using E = typename Storage<ST>::T;
    using G = StageGeom<E, V>;
    extern __shared__ __align__(16) unsigned char pipe_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wx0 = (blockIdx.x * kPipeWarps + warp) * 32 * V;
    if (wx0 >= P.nx) return;
    const int y0 = blockIdx.y * R;
    const int rows = min(R, P.ny - y0);
    const int wx1 = wx0 + 32 * V - 1;
    const bool cols_ok = wx1 < P.nx && (P.per_x || (wx0 >= 1 && wx1 <= P.nx - 2));
    if (!cols_ok) {
        for (int j = 0; j < rows; ++j) step_warp_nodes<ST, V>(src, dst, P, wx0 + lane * V, y0 + j, lane);
        return;
    }
    E* ring = reinterpret_cast<E*>(pipe_smem) + warp * S * G::SS;
#pragma unroll
    for (int s = 0; s < S - 1; ++s) {
        const int y = y0 + s;
        if (s < rows && (P.per_y || (y >= 1 && y <= P.ny - 2))) stage_issue<ST, V>(src, P, wx0, y, lane, ring + s * G::SS);
        cp_async_commit();
    }
    for (int j = 0; j < rows; ++j) {
        const int jn = j + S - 1;
        const int yn = y0 + jn;
        if (jn < rows && (P.per_y || (yn >= 1 && yn <= P.ny - 2)))
            stage_issue<ST, V>(src, P, wx0, yn, lane, ring + (jn % S) * G::SS);
        cp_async_commit();
        cp_async_wait<S - 1>();
        __syncwarp();
        const int y = y0 + j;
        if (P.per_y || (y >= 1 && y <= P.ny - 2))
            stage_compute<ST, V>(dst, P, wx0, y, lane, ring + (j % S) * G::SS);
        else
            step_warp_nodes<ST, V>(src, dst, P, wx0 + lane * V, y, lane);
        __syncwarp();
    }
}

template <int ST, int V, int S>
constexpr size_t pipe_smem_bytes()
{
    return (size_t)kPipeWarps * S * StageGeom<typename Storage<ST>::T, V>::SS * sizeof(typename Storage<ST>::T);
}

// Initialisation to f^eq(rho, u), g^eq(T, u) (in stored form). The buffer holds post-collision
// values that the next step pulls, so each equilibrium value is written to the slot its pull
// reads: population i of node x goes to (i, x - e_i), or, when x - e_i is beyond a wall, to the
// node's own opposite slot (with the anti-bounce-back constant removed on Dirichlet walls). Every
// slot is written exactly once. NULL fields mean rho = rho0, u = 0, T = T0.
template <int ST>
__global__ void k_init(typename Storage<ST>::T* __restrict__ dst, const LatParams<typename Storage<ST>::A> P,
                       const double* __restrict__ rho, const double* __restrict__ ux,
                       const double* __restrict__ uy, const double* __restrict__ T, double rho0)
{
    using A = typename Storage<ST>::A;
    using E = typename Storage<ST>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long n = (long long)y * P.nx + x;
    A f[9], g[5];
    equilibrium<Storage<ST>::DEV>(P, rho ? A(rho[n]) : A(rho0), ux ? A(ux[n]) : A(0),
                                  uy ? A(uy[n]) : A(0), T ? A(T[n]) : P.T0, f, g, row_base(P, y));
    const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = x - EX[i], sy = y - EY[i];
        int side = -1;
        if (sx < 0) { if (P.per_x) sx += P.nx; else side = 0; }
        if (sx >= P.nx) { if (P.per_x) sx -= P.nx; else side = 1; }
        if (sy < 0) { if (P.per_y) sy += P.ny; else side = 2; }
        if (sy >= P.ny) { if (P.per_y) sy -= P.ny; else side = 3; }
        long long slot;
        int plane;
        A fv = f[i];
        if (side < 0) {
            plane = i;
            slot = (long long)sy * P.crow + chunk_off(sx);
        } else {
            plane = OPP[i];
            slot = (long long)y * P.crow + chunk_off(x);
            if (P.moving) fv = fv - P.fbb[side][i];
        }
        dst[slot + plane * kRowChunk] = from_a(fv, (E*)nullptr);
        if (i < 5) {
            A v = g[i];
            if (side >= 0 && P.kind[side] == WALL_DIRICHLET) v = P.Tw_c2[side] - v;
            // a value the pull reads from the row below (above) is stored against that row's base
            if (side < 0 && EY[i] == 1) v = v + P.T_dyw;
            if (side < 0 && EY[i] == -1) v = v - P.T_dyw;
            dst[slot + (9 + plane) * kRowChunk] = from_a(v, (E*)nullptr);
        }
    }
}

// rho, u, T at the current time (gathered pre-collision populations), as double [ny][nx].
template <int ST>
__global__ void k_fields(const typename Storage<ST>::T* __restrict__ src,
                         const LatParams<typename Storage<ST>::A> P, double* __restrict__ rho,
                         double* __restrict__ ux, double* __restrict__ uy, double* __restrict__ T)
{
    using A = typename Storage<ST>::A;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    A f[9], g[5];
    gather(src, P, x, y, f, g);
    const Macro<A> m = macroscopic(P, f, g, row_base(P, y));
    const long long n = (long long)y * P.nx + x;
    if (rho) rho[n] = double(P.rho_b) + double(m.drho);
    if (ux) ux[n] = double(m.ux);
    if (uy) uy[n] = double(m.uy);
    if (T) T[n] = fma(double(y), double(P.T_dy), double(P.T_b)) + double(m.dT);
}

// Pre-collision populations at the current time as double f[9][ny][nx], g[5][ny][nx]
// (the rest state added back for deviation storage).
template <int ST>
__global__ void k_pops(const typename Storage<ST>::T* __restrict__ src,
                       const LatParams<typename Storage<ST>::A> P, double* __restrict__ f_out,
                       double* __restrict__ g_out)
{
    using A = typename Storage<ST>::A;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    A f[9], g[5];
    gather(src, P, x, y, f, g);
    const long long n = (long long)y * P.nx + x, N = (long long)P.nx * P.ny;
#pragma unroll
    for (int i = 0; i < 9; ++i) f_out[i * N + n] = double(f[i]) + double(w9<A>(i)) * double(P.rho_b);
#pragma unroll
    for (int i = 0; i < 5; ++i)
        g_out[i * N + n] = double(g[i]) + double(w5<A>(i, P.cs2T)) * fma(double(y), double(P.T_dy), double(P.T_b));
}

}  // namespace clb
