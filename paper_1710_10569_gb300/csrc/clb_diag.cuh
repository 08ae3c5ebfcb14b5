// clb_diag.cuh -- the FP64 diagnostics of one lattice and of batched lattices: the Nusselt number of
// Eq. 29 and the steady-state residual, as fixed-order sums of per-node terms, and the residual's
// snapshot. Kept apart from the step kernels (clb_kernels.cuh), which they only read.
#pragma once

#include "clb_kernels.cuh"

namespace clb {

constexpr int kReduceThreads = 256;

// Fixed-order block sum of RS_N doubles (the same order for every launch shape of the step).
__device__ __forceinline__ void block_sum(double v[RS_N], double* out)
{
    __shared__ double sh[kReduceThreads / 32][RS_N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < RS_N; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < RS_N; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < RS_N; ++k) {
            double s = 0.0;
            for (int w = 0; w < kReduceThreads / 32; ++w) s += sh[w][k];
            out[k] = s;
        }
}

// The Nusselt term u_axis (T - T0) of one node (Eq. 29), in the arithmetic precision A; T is
// returned through T_out.
template <typename A, typename S>
__device__ __forceinline__ A nu_term(const LatParams<S>& P, const Macro<A>& m, int axis, A& T_out)
{
    T_out = m.T;
    return (axis == 0 ? m.ux : m.uy) * (m.T - A(P.T0));
}

// One node's terms of the diagnostics sums, added to v: the fields come from the pulled populations,
// the terms are formed in the arithmetic precision A (FP64 for FP64 storage, FP32 for the FP32 and
// FP16 forms, whose fields are FP32 values) and accumulated in FP64. The residual's snapshot is kept
// in A as well: it holds those same values exactly, and GB300 issues FP64 instructions (the
// conversions included) slowly enough that they bound this pass. With update != 0 the node's
// snapshot entries are replaced by the current fields. The Nusselt term is weighted by wet_weight
// (wet-wall rows and columns count half: the trapezoid rule over [0, H]; 1, 1/2 and 1/4 scale
// exactly in A). Non-finite nodes are counted in nbad.
template <typename E, typename A>
__device__ __forceinline__ void node_diag(const E* __restrict__ src, const LatParams<A>& P, int x, int y,
                                          int axis, A* __restrict__ snap, int update, double v[RS_N], int& nbad)
{
    const long long N = (long long)P.nx * P.ny;
    A f[9], g[5];
    gather(src, P, x, y, f, g);
    const Macro<A> m = macroscopic(P, f, g, row_base(P, y));
    A T;
    const A q = nu_term(P, m, axis, T);
    const long long n = (long long)y * P.nx + x;
    const A dux = m.ux - snap[n], duy = m.uy - snap[N + n], dT = T - snap[2 * N + n];
    v[RS_UT] += double(q * A(wet_weight(P, x, y)));
    v[RS_DU] += double(dux * dux + duy * duy);
    v[RS_U] += double(m.ux * m.ux + m.uy * m.uy);
    v[RS_DT] += double(dT * dT);
    v[RS_T] += double(T * T);
    nbad += (isfinite(m.ux) && isfinite(m.uy) && isfinite(T) && isfinite(m.rho)) ? 0 : 1;
    if (update) {
        snap[n] = m.ux;
        snap[N + n] = m.uy;
        snap[2 * N + n] = T;
    }
}

// The residual's snapshot of the current fields (u_x, u_y, T as A [3][ny][nx]), as node_diag keeps it.
template <int ST>
__global__ void k_snap(const typename Storage<ST>::T* __restrict__ src, const LatParams<typename Storage<ST>::A> P,
                       typename Storage<ST>::A* __restrict__ snap)
{
    using A = typename Storage<ST>::A;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    A f[9], g[5];
    gather(src, P, x, y, f, g);
    const Macro<A> m = macroscopic(P, f, g, row_base(P, y));
    const long long n = (long long)y * P.nx + x, N = (long long)P.nx * P.ny;
    snap[n] = m.ux;
    snap[N + n] = m.uy;
    snap[2 * N + n] = m.T;
}

// Per-row FP64 partial sums for the diagnostics: sum u_axis (T - T0), sum |u - u_snap|^2,
// sum |u|^2, sum (T - T_snap)^2, sum T^2 and the count of non-finite nodes. One block of
// kReduceThreads per row y; threads stride over x in a fixed order, so the sums do not depend on
// how the step kernel is launched. With update != 0 the snapshot (u_x, u_y, T as double
// [3][ny][nx]) is replaced by the current fields. (The batched lattices use this form; a single
// lattice uses the row-segment form below.)
template <typename E, typename A>
__device__ __forceinline__ void reduce_row(const E* __restrict__ src, const LatParams<A>& P, int y,
                                           int axis, A* __restrict__ snap, int update,
                                           double* __restrict__ partial_row)
{
    double v[RS_N] = {0, 0, 0, 0, 0, 0};
    int nbad = 0;
    for (int x = threadIdx.x; x < P.nx; x += kReduceThreads) node_diag(src, P, x, y, axis, snap, update, v, nbad);
    v[RS_BAD] = double(nbad);
    block_sum(v, partial_row);
}

// The same sums over row segments of kDiagNodes = kReduceThreads * 8 nodes: block b covers segment
// seg of row y (b = y * nseg + seg), each thread sums its 8 nodes x = seg * kDiagNodes + t + 256 k in
// order, then the shuffle tree within each warp and the warps in order give partial[b]. The per-node
// sums are FP64 and GB300 issues FP64 slowly, so each thread takes 8 nodes (the warp tree's 30
// FP64 adds per thread are shared by 8 nodes); the register cap keeps 4 blocks per SM so that
// enough gathers are in flight. For nx <= kDiagNodes the order is that of reduce_row.
constexpr int kDiagNodes = kReduceThreads * 8;

template <int ST>
__global__ void __launch_bounds__(kReduceThreads, 4) k_reduce_nodes(
    const typename Storage<ST>::T* __restrict__ src, const LatParams<typename Storage<ST>::A> P,
    int axis, typename Storage<ST>::A* __restrict__ snap, int update, double* __restrict__ partial, int nseg)
{
    const int seg = blockIdx.x % nseg, y = blockIdx.x / nseg;
    const int x0 = seg * kDiagNodes, x1 = min(P.nx, x0 + kDiagNodes);
    double v[RS_N] = {0, 0, 0, 0, 0, 0};
    int nbad = 0;
    for (int x = x0 + threadIdx.x; x < x1; x += kReduceThreads) node_diag(src, P, x, y, axis, snap, update, v, nbad);
    v[RS_BAD] = double(nbad);
    block_sum(v, partial + (long long)blockIdx.x * RS_N);
}

// Sum the per-row partials in row order and finish the diagnostics in FP64: out[0..RS_N-1] = the
// sums, out[RS_N] = Nu (Eq. 29), out[RS_N+1] = E_R.
__device__ __forceinline__ void reduce_final(const double* __restrict__ partial, int rows,
                                             double nodes, double cells, double H, double dT,
                                             double sign, double kappa, double u_ref, double dT_ref,
                                             double* __restrict__ out)
{
    double v[RS_N] = {0, 0, 0, 0, 0, 0};
    for (int r = threadIdx.x; r < rows; r += kReduceThreads)
        for (int k = 0; k < RS_N; ++k) v[k] += partial[(long long)r * RS_N + k];
    __shared__ double tot[RS_N];
    block_sum(v, tot);
    if (threadIdx.x == 0) {
        for (int k = 0; k < RS_N; ++k) out[k] = tot[k];
        finish_diagnostics(tot, nodes, cells, H, dT, sign, kappa, u_ref, dT_ref, &out[RS_N], &out[RS_N + 1]);
    }
}

static __global__ void __launch_bounds__(kReduceThreads) k_reduce_final(const double* __restrict__ partial,
                                                                 int rows, double nodes, double cells,
                                                                 double H, double dT, double sign,
                                                                 double kappa, double u_ref,
                                                                 double dT_ref, double* __restrict__ out)
{
    reduce_final(partial, rows, nodes, cells, H, dT, sign, kappa, u_ref, dT_ref, out);
}

}  // namespace clb
