// clb_thermal.cu -- the D2Q5 central-moment equation alone with a prescribed velocity field
// (include/clb.h: clb_thermal_*). Sec. 3.1 of the paper solves only the D2Q5 equation for a given
// velocity; this is that mode, for convection-diffusion of a passive scalar. Per node and step:
// pull the 5 temperature populations (Eq. 22, the same wall rules as the coupled step), read the
// node's velocity, collide (Eqs. 16-21), store. The collision is the same device function as the
// coupled step's D2Q5 part.
#include <cuda_runtime.h>

#include <algorithm>

#include "clb_kernels.cuh"

using namespace clb;

namespace {

constexpr int NT = 5;  // planes per buffer

// Two consecutive elements loaded or stored as one aligned access.
template <typename E>
struct alignas(2 * sizeof(E)) Pair {
    E e[2];
};

// Velocity storage of the thermal handle: the arithmetic type of the storage.
template <int ST>
using VelT = typename Storage<ST>::A;

template <typename A>
__device__ __forceinline__ void thermal_slots(const LatParams<A>& P, int x, int y, long long idx[NT], int& mask)
{
    const bool inL = P.per_x || x > 0;
    const bool inR = P.per_x || x < P.nx - 1;
    const bool inB = P.per_y || y > 0;
    const bool inT = P.per_y || y < P.ny - 1;
    const int xm = x > 0 ? x - 1 : P.nx - 1;
    const int xp = x < P.nx - 1 ? x + 1 : 0;
    const long long r0 = (long long)y * P.pitch;
    const long long rm = (long long)(y > 0 ? y - 1 : P.ny - 1) * P.pitch;
    const long long rp = (long long)(y < P.ny - 1 ? y + 1 : 0) * P.pitch;
    const long long here = r0 + x;
    const long long pl = P.plane;
    idx[0] = here;
    idx[1] = inL ? 1 * pl + r0 + xm : 3 * pl + here;
    idx[2] = inB ? 2 * pl + rm + x : 4 * pl + here;
    idx[3] = inR ? 3 * pl + r0 + xp : 1 * pl + here;
    idx[4] = inT ? 4 * pl + rp + x : 2 * pl + here;
    mask = (inL ? 0 : 1) | (inR ? 0 : 2) | (inB ? 0 : 4) | (inT ? 0 : 8);
}

template <typename E, typename A>
__device__ __forceinline__ void thermal_gather(const E* __restrict__ src, const LatParams<A>& P, int x, int y, A g[NT])
{
    long long idx[NT];
    int mask;
    thermal_slots(P, x, y, idx, mask);
#pragma unroll
    for (int i = 0; i < NT; ++i) g[i] = to_a(src[idx[i]]);
    // g2 (g4) pulled from the row below (above) is re-based to this row; bounced values are not
    g[2] = (mask & 4) ? g[2] : g[2] - P.T_dyw;
    g[4] = (mask & 8) ? g[4] : g[4] + P.T_dyw;
    if (mask) {
        if ((mask & 1) && P.kind[0] == WALL_DIRICHLET) g[1] = P.Tw_c2[0] - g[1];
        if ((mask & 2) && P.kind[1] == WALL_DIRICHLET) g[3] = P.Tw_c2[1] - g[3];
        if ((mask & 4) && P.kind[2] == WALL_DIRICHLET) g[2] = P.Tw_c2[2] - g[2];
        if ((mask & 8) && P.kind[3] == WALL_DIRICHLET) g[4] = P.Tw_c2[3] - g[4];
    }
}

// D2Q5 equilibrium g^eq(T, u) in stored form (minus w^T T_b(y) for deviation storage; dT = T - T_b(y)).
template <bool DEV, typename A>
__device__ __forceinline__ void thermal_eq(const LatParams<A>& P, A T, A dT, A u, A v, A g[NT])
{
    if constexpr (DEV) eq_dev_d2q5(T, dT, u, v, P.cs2T, g);
    else back_d2q5(T, A(0), A(0), T * P.cs2T, T * P.cs2T, u, v, g);
}

// Pulled populations of node (x, y) with the wall rules, including wet walls: a node on a wet
// wall takes g_i = g^eq_i(T_w, u) + [g_i(q) - g^eq_i(T(q), u(q))] from the fluid node q next to it
// (along the normal; the diagonal neighbour at a corner, where T_w is the mean of the two walls'
// temperatures), u being the prescribed velocity of each node (the paper's non-equilibrium
// extrapolation, Sec. 3).
template <bool DEV, typename E, typename A, typename VT>
__device__ __forceinline__ void thermal_gather_node(const E* __restrict__ src, const LatParams<A>& P,
                                                    const VT* __restrict__ ux, const VT* __restrict__ uy,
                                                    int x, int y, A g[NT])
{
    const bool onx = P.wet_x && (x == 0 || x == P.nx - 1);
    const bool ony = P.wet_y && (y == 0 || y == P.ny - 1);
    if (!onx && !ony) {
        thermal_gather(src, P, x, y, g);
        return;
    }
    const int qx = onx ? (x == 0 ? 1 : x - 1) : x, qy = ony ? (y == 0 ? 1 : y - 1) : y;
    const int side_x = x == 0 ? 0 : 1, side_y = y == 0 ? 2 : 3;
    const A Tw = (onx && ony) ? A(0.5) * (P.Twall[side_x] + P.Twall[side_y]) : P.Twall[ony ? side_y : side_x];
    const A dTw = (onx && ony) ? Tw - P.T_b : P.dTw[ony ? side_y : side_x];
    A gq[NT], eq_q[NT], eq_b[NT];
    thermal_gather(src, P, qx, qy, gq);
    const A dTq = (gq[0] + gq[1]) + (gq[2] + gq[3]) + gq[4];
    const long long nq = (long long)qy * P.nx + qx, nb = (long long)y * P.nx + x;
    thermal_eq<DEV>(P, row_base(P, qy) + dTq, dTq, A(ux[nq]), A(uy[nq]), eq_q);
    thermal_eq<DEV>(P, Tw, dTw, A(ux[nb]), A(uy[nb]), eq_b);
#pragma unroll
    for (int i = 0; i < NT; ++i) g[i] = eq_b[i] + (gq[i] - eq_q[i]);
}

// One node's collision (Eqs. 16-21) with its prescribed velocity.
template <int ST>
__device__ __forceinline__ void thermal_collide(const LatParams<typename Storage<ST>::A>& P,
                                                typename Storage<ST>::A u, typename Storage<ST>::A v,
                                                typename Storage<ST>::A g[NT], typename Storage<ST>::A Tb)
{
    using A = typename Storage<ST>::A;
    const A dT = (g[0] + g[1]) + (g[2] + g[3]) + g[4];
    if constexpr (Storage<ST>::DEV) collide_d2q5_dev(P, Tb + dT, dT, u, v, g);
    else collide_d2q5(P, Tb + dT, u, v, g);
}

// One time step, two neighbouring nodes x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x) and x0 + 1
// of row y = blockIdx.y per thread. A pair whose pulls all stay inside the lattice without wrapping
// reads the planes pulled along y (and the rest plane) as aligned pairs and stores every plane as
// an aligned pair; other pairs (next to a wall or a periodic seam, or the single node at the end of
// an odd row) gather node by node with the wall rules. The values are those of the node-by-node
// path.
template <int ST>
__global__ void __launch_bounds__(128, ST == ST_F64 ? 8 : 12) k_thermal_step(const typename Storage<ST>::T* __restrict__ src,
                                                      typename Storage<ST>::T* __restrict__ dst,
                                                      const VelT<ST>* __restrict__ ux,
                                                      const VelT<ST>* __restrict__ uy,
                                                      const LatParams<typename Storage<ST>::A> P)
{
    using A = typename Storage<ST>::A;
    using E = typename Storage<ST>::T;
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y;
    if (x0 >= P.nx) return;
    const bool two = x0 + 1 < P.nx;
    const long long pl = P.plane;
    const long long here = (long long)y * P.pitch + x0;
    const long long n = (long long)y * P.nx + x0;
    A ga[NT], gb[NT];
    if (two && x0 > 0 && x0 + 2 < P.nx && y > 0 && y + 1 < P.ny) {
        const Pair<E> c0 = *reinterpret_cast<const Pair<E>*>(src + here);
        const Pair<E> c2 = *reinterpret_cast<const Pair<E>*>(src + 2 * pl + here - P.pitch);
        const Pair<E> c4 = *reinterpret_cast<const Pair<E>*>(src + 4 * pl + here + P.pitch);
        ga[0] = to_a(c0.e[0]);
        gb[0] = to_a(c0.e[1]);
        ga[1] = to_a(src[pl + here - 1]);
        gb[1] = to_a(src[pl + here]);
        ga[2] = to_a(c2.e[0]);
        gb[2] = to_a(c2.e[1]);
        ga[3] = to_a(src[3 * pl + here + 1]);
        gb[3] = to_a(src[3 * pl + here + 2]);
        ga[4] = to_a(c4.e[0]);
        gb[4] = to_a(c4.e[1]);
        // re-based to this row (see thermal_gather)
        ga[2] = ga[2] - P.T_dyw;
        gb[2] = gb[2] - P.T_dyw;
        ga[4] = ga[4] + P.T_dyw;
        gb[4] = gb[4] + P.T_dyw;
    } else {
        thermal_gather_node<Storage<ST>::DEV>(src, P, ux, uy, x0, y, ga);
        if (two) thermal_gather_node<Storage<ST>::DEV>(src, P, ux, uy, x0 + 1, y, gb);
    }
    const A Tb = row_base(P, y);
    thermal_collide<ST>(P, A(ux[n]), A(uy[n]), ga, Tb);
    if (two) {
        thermal_collide<ST>(P, A(ux[n + 1]), A(uy[n + 1]), gb, Tb);
        // here is even (x0 and the row pitch are): one aligned pair per plane
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            Pair<E> o;
            o.e[0] = from_a(ga[i], (E*)nullptr);
            o.e[1] = from_a(gb[i], (E*)nullptr);
            *reinterpret_cast<Pair<E>*>(dst + i * pl + here) = o;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NT; ++i) dst[i * pl + here] = from_a(ga[i], (E*)nullptr);
    }
}

// g^eq(T, u) written to the slots the next pull reads (as k_init does for the coupled step), and
// the velocity stored in the handle's precision.
template <int ST>
__global__ void k_thermal_init(typename Storage<ST>::T* __restrict__ dst, VelT<ST>* __restrict__ uxs,
                               VelT<ST>* __restrict__ uys, const LatParams<typename Storage<ST>::A> P,
                               const double* __restrict__ T, const double* __restrict__ ux,
                               const double* __restrict__ uy)
{
    using A = typename Storage<ST>::A;
    using E = typename Storage<ST>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const long long n = (long long)y * P.nx + x;
    const A u = ux ? A(ux[n]) : A(0), v = uy ? A(uy[n]) : A(0);
    const A t = T ? A(T[n]) : P.T0;
    uxs[n] = u;
    uys[n] = v;
    A g[NT];
    if constexpr (Storage<ST>::DEV) {
        eq_dev_d2q5(t, t - row_base(P, y), u, v, P.cs2T, g);
    } else {
        back_d2q5(t, A(0), A(0), t * P.cs2T, t * P.cs2T, u, v, g);
    }
    const int EX[NT] = {0, 1, 0, -1, 0};
    const int EY[NT] = {0, 0, 1, 0, -1};
    const int OPP[NT] = {0, 3, 4, 1, 2};
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        int sx = x - EX[i], sy = y - EY[i];
        int side = -1;
        if (sx < 0) { if (P.per_x) sx += P.nx; else side = 0; }
        if (sx >= P.nx) { if (P.per_x) sx -= P.nx; else side = 1; }
        if (sy < 0) { if (P.per_y) sy += P.ny; else side = 2; }
        if (sy >= P.ny) { if (P.per_y) sy -= P.ny; else side = 3; }
        A val = g[i];
        long long slot;
        int plane;
        if (side < 0) {
            plane = i;
            slot = (long long)sy * P.pitch + sx;
        } else {
            plane = OPP[i];
            slot = (long long)y * P.pitch + x;
            if (P.kind[side] == WALL_DIRICHLET) val = P.Tw_c2[side] - val;
        }
        // a value the pull reads from the row below (above) is stored against that row's base
        if (side < 0 && EY[i] == 1) val = val + P.T_dyw;
        if (side < 0 && EY[i] == -1) val = val - P.T_dyw;
        dst[plane * P.plane + slot] = from_a(val, (E*)nullptr);
    }
}

template <int ST>
__global__ void k_thermal_out(const typename Storage<ST>::T* __restrict__ src,
                              const LatParams<typename Storage<ST>::A> P, const VelT<ST>* __restrict__ ux,
                              const VelT<ST>* __restrict__ uy, double* __restrict__ T, double* __restrict__ pops)
{
    using A = typename Storage<ST>::A;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    A g[NT];
    thermal_gather_node<Storage<ST>::DEV>(src, P, ux, uy, x, y, g);
    const long long n = (long long)y * P.nx + x, N = (long long)P.nx * P.ny;
    const double base = fma(double(y), double(P.T_dy), double(P.T_b));
    if (T) T[n] = base + double((g[0] + g[1]) + (g[2] + g[3]) + g[4]);
    if (pops)
#pragma unroll
        for (int i = 0; i < NT; ++i) pops[i * N + n] = double(g[i]) + double(w5<A>(i, P.cs2T)) * base;
}

constexpr int kChunkT = 32;

}  // namespace

struct clb_thermal {
    int nx = 0, ny = 0;
    clb_params p{};
    int device = 0;
    cudaStream_t stream = nullptr, cap = nullptr;
    char* mem = nullptr;
    void* buf[2] = {nullptr, nullptr};
    void* vel[2] = {nullptr, nullptr};
    double* stage = nullptr;
    int cur = 0;
    long steps = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    LatParams<double> Pd{};
    LatParams<float> Pf{};
};

namespace {

size_t thermal_buffer_bytes(int nx, int ny, int storage)
{
    return align256((size_t)NT * (size_t)plane_elems(nx, ny, storage) * elem_size(storage));
}

size_t thermal_footprint(int nx, int ny, int storage)
{
    const size_t N = (size_t)nx * ny;
    const size_t vb = align256(N * (storage == CLB_F64 ? 8 : 4));
    return 2 * thermal_buffer_bytes(nx, ny, storage) + 2 * vb + align256(5 * N * sizeof(double));
}

clb_status thermal_launch(clb_thermal* h, int from, cudaStream_t s)
{
    const dim3 block(128, 1), grid((h->nx + 255) / 256, h->ny);  // two nodes per thread
    const void* a = h->buf[from];
    void* b = h->buf[from ^ 1];
    switch (h->p.storage) {
    case CLB_F64:
        k_thermal_step<ST_F64><<<grid, block, 0, s>>>((const double*)a, (double*)b, (const double*)h->vel[0], (const double*)h->vel[1], h->Pd);
        break;
    case CLB_F32:
        k_thermal_step<ST_F32><<<grid, block, 0, s>>>((const float*)a, (float*)b, (const float*)h->vel[0], (const float*)h->vel[1], h->Pf);
        break;
    default:
        k_thermal_step<ST_F16DEV><<<grid, block, 0, s>>>((const __half*)a, (__half*)b, (const float*)h->vel[0], (const float*)h->vel[1], h->Pf);
        break;
    }
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

clb_status thermal_out(clb_thermal* h, double* T, double* pops)
{
    const dim3 block(128, 1), grid((h->nx + 127) / 128, h->ny);  // one node per thread
    const void* a = h->buf[h->cur];
    switch (h->p.storage) {
    case CLB_F64:
        k_thermal_out<ST_F64><<<grid, block, 0, h->stream>>>((const double*)a, h->Pd, (const double*)h->vel[0],
                                                             (const double*)h->vel[1], T, pops);
        break;
    case CLB_F32:
        k_thermal_out<ST_F32><<<grid, block, 0, h->stream>>>((const float*)a, h->Pf, (const float*)h->vel[0],
                                                             (const float*)h->vel[1], T, pops);
        break;
    default:
        k_thermal_out<ST_F16DEV><<<grid, block, 0, h->stream>>>((const __half*)a, h->Pf, (const float*)h->vel[0],
                                                                (const float*)h->vel[1], T, pops);
        break;
    }
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

}  // namespace

extern "C" clb_status clb_thermal_create(int nx, int ny, const clb_params* p, void* stream, clb_thermal** out)
{
    if (!out) return set_error(CLB_EINVAL, "out is NULL");
    *out = nullptr;
    CLB_TRY(validate(nx, ny, p));
    auto* h = new (std::nothrow) clb_thermal;
    if (!h) return host_alloc_failed();
    h->nx = nx;
    h->ny = ny;
    h->p = *p;
    h->stream = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    const size_t bb = thermal_buffer_bytes(nx, ny, p->storage);
    const size_t N = (size_t)nx * ny;
    const size_t vb = align256(N * (p->storage == CLB_F64 ? 8 : 4));
    cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->mem, thermal_footprint(nx, ny, p->storage));
    if (e != cudaSuccess) {
        clb_thermal_destroy(h);
        return set_error(e == cudaErrorMemoryAllocation ? CLB_ENOMEM : CLB_ECUDA, "thermal create: %s", cudaGetErrorString(e));
    }
    h->buf[0] = h->mem;
    h->buf[1] = h->mem + bb;
    h->vel[0] = h->mem + 2 * bb;
    h->vel[1] = h->mem + 2 * bb + vb;
    h->stage = (double*)(h->mem + 2 * bb + 2 * vb);
    h->Pd = make_lat_params<double>(nx, ny, *p);
    h->Pf = make_lat_params<float>(nx, ny, *p);
    e = cudaMemsetAsync(h->mem, 0, 2 * bb, h->stream);
    if (e != cudaSuccess) {
        clb_thermal_destroy(h);
        return set_error(CLB_ECUDA, "thermal memset: %s", cudaGetErrorString(e));
    }
    clb_status st = clb_thermal_init(h, nullptr, nullptr, nullptr);
    if (st != CLB_OK) {
        clb_thermal_destroy(h);
        return st;
    }
    *out = h;
    return CLB_OK;
}

extern "C" void clb_thermal_destroy(clb_thermal* h)
{
    if (!h) return;
    if (h->mem) cudaStreamSynchronize(h->stream);
    for (auto& g : h->graph)
        if (g) cudaGraphExecDestroy(g);
    if (h->mem) cudaFree(h->mem);
    if (h->cap) cudaStreamDestroy(h->cap);
    delete h;
}

extern "C" clb_status clb_thermal_init(clb_thermal* h, const double* T, const double* ux, const double* uy)
{
    if (!h) return set_error(CLB_EINVAL, "handle is NULL");
    const size_t N = (size_t)h->nx * h->ny;
    const double* src[3] = {T, ux, uy};
    const double* dev[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k)
        if (src[k]) {
            CLB_CUDA(cudaMemcpyAsync(h->stage + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            dev[k] = h->stage + k * N;
        }
    const dim3 block(128, 1), grid((h->nx + 127) / 128, h->ny);  // one node per thread
    void* d = h->buf[h->cur];
    switch (h->p.storage) {
    case CLB_F64: k_thermal_init<ST_F64><<<grid, block, 0, h->stream>>>((double*)d, (double*)h->vel[0], (double*)h->vel[1], h->Pd, dev[0], dev[1], dev[2]); break;
    case CLB_F32: k_thermal_init<ST_F32><<<grid, block, 0, h->stream>>>((float*)d, (float*)h->vel[0], (float*)h->vel[1], h->Pf, dev[0], dev[1], dev[2]); break;
    default: k_thermal_init<ST_F16DEV><<<grid, block, 0, h->stream>>>((__half*)d, (float*)h->vel[0], (float*)h->vel[1], h->Pf, dev[0], dev[1], dev[2]); break;
    }
    CLB_CUDA(cudaGetLastError());
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    h->steps = 0;
    return CLB_OK;
}

extern "C" clb_status clb_thermal_step(clb_thermal* h, long n)
{
    if (!h) return set_error(CLB_EINVAL, "handle is NULL");
    if (n < 0) return set_error(CLB_EINVAL, "n < 0");
    // both parities are captured on the first chunk (no capture later, mid-stepping)
    for (int par = 0; n >= kChunkT && par < 2; ++par) {
        if (h->graph[par]) continue;
        CLB_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        clb_status st = CLB_OK;
        for (int k = 0; k < kChunkT && st == CLB_OK; ++k) st = thermal_launch(h, par ^ (k & 1), h->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap, &g);
        if (st != CLB_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return set_error(CLB_ECUDA, "capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->graph[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return set_error(CLB_ECUDA, "instantiate: %s", cudaGetErrorString(e));
    }
    while (n >= kChunkT) {
        CLB_CUDA(cudaGraphLaunch(h->graph[h->cur], h->stream));
        n -= kChunkT;
        h->steps += kChunkT;
    }
    for (; n > 0; --n) {
        CLB_TRY(thermal_launch(h, h->cur, h->stream));
        h->cur ^= 1;
        h->steps++;
    }
    return CLB_OK;
}

extern "C" clb_status clb_thermal_fields(clb_thermal* h, double* T)
{
    if (!h || !T) return set_error(CLB_EINVAL, "handle and T must not be NULL");
    const size_t N = (size_t)h->nx * h->ny;
    CLB_TRY(thermal_out(h, h->stage, nullptr));
    CLB_CUDA(cudaMemcpyAsync(T, h->stage, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb_thermal_populations(clb_thermal* h, double* g)
{
    if (!h || !g) return set_error(CLB_EINVAL, "handle and g must not be NULL");
    const size_t N = (size_t)h->nx * h->ny;
    CLB_TRY(thermal_out(h, nullptr, h->stage));
    CLB_CUDA(cudaMemcpyAsync(g, h->stage, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb_thermal_sync(clb_thermal* h)
{
    if (!h) return set_error(CLB_EINVAL, "handle is NULL");
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}
