// clb_lattice.cu -- C ABI of one lattice (include/clb.h): creation, initialisation, the stepping
// loop (CUDA-graph chunks of the fused step kernel), field extraction, FP64 diagnostics,
// checkpoints and the launch-shape autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "clb_diag.cuh"

using namespace clb;

// ------------------------------------------------------------------------------------- errors

namespace clb {
static thread_local std::string g_err;

clb_status set_error(clb_status st, const char* fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}
void clear_error() { g_err.clear(); }

clb_status validate(int nx, int ny, const clb_params* p)
{
    if (!p) return set_error(CLB_EINVAL, "params is NULL");
    if (nx < 2 || ny < 2 || nx > kMaxEdge || ny > kMaxEdge)
        return set_error(CLB_EINVAL, "lattice %d x %d: each edge must be in [2, %d]", nx, ny, kMaxEdge);
    if ((long long)nx * ny > kMaxNodes)
        return set_error(CLB_EINVAL, "lattice %d x %d exceeds %lld nodes", nx, ny, kMaxNodes);
    const double vals[] = {p->nu, p->kappa, p->g_beta, p->T0, p->rho0, p->s_b, p->s_3, p->s_4,
                           p->lambda2, p->cs2_T, p->Fv[0], p->Fv[1], p->T_wall[0], p->T_wall[1],
                           p->T_wall[2], p->T_wall[3], p->T_ref, p->u_ref, p->dT_ref};
    for (double v : vals)
        if (!std::isfinite(v)) return set_error(CLB_EINVAL, "non-finite parameter");
    for (int s = 0; s < 4; ++s)
        for (int c = 0; c < 2; ++c)
            if (!std::isfinite(p->u_wall[s][c]) || std::fabs(p->u_wall[s][c]) > 0.4)
                return set_error(CLB_EINVAL, "u_wall[%d][%d] must be finite with |u| <= 0.4", s, c);
    if (!(p->nu > 0)) return set_error(CLB_EINVAL, "nu must be > 0 (got %g)", p->nu);
    if (!(p->kappa > 0)) return set_error(CLB_EINVAL, "kappa must be > 0 (got %g)", p->kappa);
    if (!(p->rho0 > 0)) return set_error(CLB_EINVAL, "rho0 must be > 0");
    if (!(p->cs2_T > 0 && p->cs2_T < 0.5))
        return set_error(CLB_EINVAL, "cs2_T must be in (0, 1/2) (got %g)", p->cs2_T);
    const double rates[] = {p->s_b, p->s_3, p->s_4, p->lambda2};
    for (double r : rates)
        if (!(r > 0 && r < 2)) return set_error(CLB_EINVAL, "relaxation rates must be in (0, 2) (got %g)", r);
    for (int s = 0; s < 4; ++s)
        if (p->wall[s] < CLB_PERIODIC || p->wall[s] > CLB_WALL_WET)
            return set_error(CLB_EINVAL, "wall[%d] = %d is not a clb_wall", s, p->wall[s]);
    if ((p->wall[0] == CLB_PERIODIC) != (p->wall[1] == CLB_PERIODIC) ||
        (p->wall[2] == CLB_PERIODIC) != (p->wall[3] == CLB_PERIODIC))
        return set_error(CLB_EINVAL, "periodic sides must come in pairs");
    for (int a = 0; a < 2; ++a) {
        const int lo = p->wall[2 * a], hi = p->wall[2 * a + 1], other = p->wall[2 - 2 * a];
        if ((lo == CLB_WALL_WET) != (hi == CLB_WALL_WET))
            return set_error(CLB_EINVAL, "wet walls go on both sides of an axis");
        if (lo == CLB_WALL_WET && (a == 0 ? nx : ny) < 3)
            return set_error(CLB_EINVAL, "wet walls need at least 3 nodes across");
        if (lo == CLB_WALL_WET && other != CLB_PERIODIC && other != CLB_WALL_WET)
            return set_error(CLB_EINVAL, "the sides next to wet walls must be periodic or wet");
    }
    if (p->storage < CLB_F64 || p->storage > CLB_F16DEV)
        return set_error(CLB_EINVAL, "storage %d is not a clb_storage", p->storage);
    return CLB_OK;
}
}  // namespace clb

extern "C" const char* clb_last_error(void) { return g_err.c_str(); }
extern "C" const char* clb_version(void) { return "clb 1.0 (sm_103a)"; }

extern "C" clb_status clb_params_default(clb_params* p)
{
    if (!p) return set_error(CLB_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->nu = 0.02;
    p->kappa = 0.02;
    p->rho0 = 1.0;
    p->s_b = p->s_3 = p->s_4 = p->lambda2 = 1.0;
    p->cs2_T = 0.25;
    p->storage = CLB_F64;
    return CLB_OK;
}

// ------------------------------------------------------------------------------------- handle

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != prev && prev >= 0) cudaSetDevice(prev);
    }
};

// Blocks per row of the diagnostics pass (row segments of kDiagNodes nodes).
int diag_segments(int nx) { return (nx + kDiagNodes - 1) / kDiagNodes; }

struct Layout {
    size_t buf[2], snap, stage, partial, diag, total;
};

Layout layout(int nx, int ny, int storage)
{
    Layout L;
    const size_t N = (size_t)nx * ny;
    size_t off = 0;
    const size_t bb = buffer_slot_bytes(nx, ny, storage);
    L.buf[0] = off; off += bb;
    L.buf[1] = off; off += bb;
    L.snap = off; off += align256(3 * N * sizeof(double));
    L.stage = off; off += align256(4 * N * sizeof(double));
    L.partial = off; off += align256((size_t)ny * diag_segments(nx) * RS_N * sizeof(double));
    L.diag = off; off += align256(16 * sizeof(double));
    L.total = off;
    return L;
}

constexpr int kGraphChunk = 32;  // steps per captured graph (even: the buffers return)

}  // namespace

struct clb_handle {
    int nx = 0, ny = 0;
    clb_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only to capture graphs
    cudaStream_t side = nullptr; // private stream of the split step's edge kernel
    cudaEvent_t fork = nullptr, join = nullptr;  // the split step's fork and join points
    char* mem = nullptr;
    bool own_mem = false;
    Layout L{};
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;  // buffer holding the post-collision populations of the last step
    double* snap = nullptr;
    double* stage = nullptr;
    double* partial = nullptr;
    double* diag = nullptr;
    double* host_diag = nullptr;  // pinned
    long steps = 0;
    int bx = 128, by = 1, npt = 1;
    int pipe_stages = 0, pipe_rows = 8;  // 0 stages: direct kernel
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    LatParams<double> Pd{};
    LatParams<float> Pf{};
};

namespace {

void drop_graphs(clb_handle* h)
{
    for (auto& g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

dim3 grid_for(const clb_handle* h, int bx, int by)
{
    return dim3((h->nx + bx - 1) / bx, (h->ny + by - 1) / by);
}

// The split step (k_step_inner beside k_step_edge) for the FP16 form, which sits at the issue
// limit: 83.0 -> 77.9 us per step on 4096 x 2048. The FP32 form is bound by memory (one kernel:
// 35.0 us, split: 35.2-35.6 us, the fork and join costing more than the registers save) and FP64
// by its arithmetic (602 us either way); they keep the one kernel that holds every path.
template <int ST>
constexpr bool split_step()
{
    return ST == ST_F16DEV;
}

// Interior rows and warp columns of the split step for V nodes per thread: rows next to a y wall
// (or on a wet y wall) and the columns next to an x wall (or on a wet x wall, or holding the ragged
// end of the rows) go to the edge kernel.
SplitGeom split_geom(int nx, int ny, const LatParams<float>& P, int V)
{
    const int W = 32 * V;
    SplitGeom G{};
    G.nw = (nx + W - 1) / W;
    if (!P.per_y || P.wet_y) {
        G.nyb = ny > 1 ? 2 : 1;
        G.yb[0] = 0;
        G.yb[1] = ny - 1;
        G.y0 = 1;
        G.y1 = std::max(1, ny - 1);
    } else {
        G.nyb = 0;
        G.y0 = 0;
        G.y1 = ny;
    }
    const bool xwall = !P.per_x || P.wet_x;
    const bool left = xwall, right = xwall || nx % W != 0;
    G.c0 = left ? 1 : 0;
    G.c1 = std::max(G.c0, right ? G.nw - 1 : G.nw);
    G.ncb = 0;
    if (left) G.cb[G.ncb++] = 0;
    if (right && !(left && G.nw == 1)) G.cb[G.ncb++] = G.nw - 1;
    return G;
}

template <int ST, int NPT>
cudaError_t enqueue_step(const clb_handle* h, const void* a, void* b, cudaStream_t s, int bx, int by)
{
    using E = typename Storage<ST>::T;
    using A = typename Storage<ST>::A;
    const LatParams<A>& P = *reinterpret_cast<const LatParams<A>*>(ST == ST_F64 ? (const void*)&h->Pd : (const void*)&h->Pf);
    const bool hi1 = h->p.s_3 == 1.0 && h->p.s_4 == 1.0 && h->p.lambda2 == 1.0;
    const dim3 block(bx, by);
    if constexpr (!split_step<ST>()) {
        const dim3 grid((h->nx + bx * NPT - 1) / (bx * NPT), (h->ny + by - 1) / by);
        if (hi1) k_step<ST, NPT, true><<<grid, block, 0, s>>>((const E*)a, (E*)b, P);
        else k_step<ST, NPT, false><<<grid, block, 0, s>>>((const E*)a, (E*)b, P);
        return cudaSuccess;
    } else {
        const SplitGeom G = split_geom(h->nx, h->ny, h->Pf, NPT);
        const int ncol = G.c1 - G.c0, nrow = G.y1 - G.y0, nedge = G.edge_warps();
        const bool inner = ncol > 0 && nrow > 0;
        cudaStream_t se = s;
        if (inner && nedge > 0) {
            // fork: the edge warps run on the side stream beside the interior (under graph capture
            // the event pulls the side stream into the capture, and the join closes it)
            cudaError_t e = cudaEventRecord(h->fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->fork, 0);
            if (e != cudaSuccess) return e;
            se = h->side;
        }
        if (nedge > 0) {
            const dim3 ge((nedge * 32 + 127) / 128);
            if (hi1) k_step_edge<ST, NPT, true><<<ge, 128, 0, se>>>((const E*)a, (E*)b, P, G);
            else k_step_edge<ST, NPT, false><<<ge, 128, 0, se>>>((const E*)a, (E*)b, P, G);
        }
        if (inner) {
            const dim3 gi((ncol * 32 + bx - 1) / bx, (nrow + by - 1) / by);
            if (ST == ST_F16DEV && NPT == 4 && hi1)
                k_step_inner_f16x4_hi1<<<gi, block, 0, s>>>((const __half*)a, (__half*)b, h->Pf, G.y0, G.y1, G.c0, G.c1);
            else if (hi1)
                k_step_inner<ST, NPT, true><<<gi, block, 0, s>>>((const E*)a, (E*)b, P, G.y0, G.y1, G.c0, G.c1);
            else
                k_step_inner<ST, NPT, false><<<gi, block, 0, s>>>((const E*)a, (E*)b, P, G.y0, G.y1, G.c0, G.c1);
        }
        if (se != s) {
            cudaError_t e = cudaEventRecord(h->join, se);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->join, 0);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
}

template <int ST>
cudaError_t enqueue_step_npt(const clb_handle* h, const void* a, void* b, cudaStream_t s, int bx, int by, int npt)
{
    if (npt == 4) return enqueue_step<ST, 4>(h, a, b, s, bx, by);
    if (npt == 2) return enqueue_step<ST, 2>(h, a, b, s, bx, by);
    return enqueue_step<ST, 1>(h, a, b, s, bx, by);
}

struct Launch {
    int bx, by, npt, stages, rows;
};

Launch current_launch(const clb_handle* h) { return {h->bx, h->by, h->npt, h->pipe_stages, h->pipe_rows}; }

// Enqueue one step from buffer `from` into the other buffer on stream s.
clb_status launch_step(clb_handle* h, int from, cudaStream_t s, const Launch& L)
{
    void* a = h->buf[from];
    void* b = h->buf[from ^ 1];
    if (L.stages > 0) {
        const cudaError_t e = enqueue_pipe_any(h->p.storage, h->Pd, h->Pf, h->device, h->nx, h->ny, a, b, s, L.npt,
                                               L.stages, L.rows);
        if (e != cudaSuccess) return set_error(CLB_ECUDA, "pipelined step: %s", cudaGetErrorString(e));
    } else {
        cudaError_t e;
        switch (h->p.storage) {
        case CLB_F64: e = enqueue_step_npt<ST_F64>(h, a, b, s, L.bx, L.by, L.npt); break;
        case CLB_F32: e = enqueue_step_npt<ST_F32>(h, a, b, s, L.bx, L.by, L.npt); break;
        default: e = enqueue_step_npt<ST_F16DEV>(h, a, b, s, L.bx, L.by, L.npt); break;
        }
        if (e != cudaSuccess) return set_error(CLB_ECUDA, "step: %s", cudaGetErrorString(e));
    }
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

clb_status build_graph(clb_handle* h, int start)
{
    CLB_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    clb_status st = CLB_OK;
    for (int k = 0; k < kGraphChunk && st == CLB_OK; ++k) st = launch_step(h, start ^ (k & 1), h->cap, current_launch(h));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (st != CLB_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return set_error(CLB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph[start], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_error(CLB_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return CLB_OK;
}

clb_status launch_init(clb_handle* h, const double* rho, const double* ux, const double* uy,
                       const double* T)
{
    const dim3 block(128, 1), grid = grid_for(h, 128, 1);
    void* d = h->buf[h->cur];
    switch (h->p.storage) {
    case CLB_F64: k_init<ST_F64><<<grid, block, 0, h->stream>>>((double*)d, h->Pd, rho, ux, uy, T, h->p.rho0); break;
    case CLB_F32: k_init<ST_F32><<<grid, block, 0, h->stream>>>((float*)d, h->Pf, rho, ux, uy, T, h->p.rho0); break;
    default: k_init<ST_F16DEV><<<grid, block, 0, h->stream>>>((__half*)d, h->Pf, rho, ux, uy, T, h->p.rho0); break;
    }
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

clb_status launch_fields(clb_handle* h, double* rho, double* ux, double* uy, double* T)
{
    const dim3 block(128, 1), grid = grid_for(h, 128, 1);
    const void* s = h->buf[h->cur];
    switch (h->p.storage) {
    case CLB_F64: k_fields<ST_F64><<<grid, block, 0, h->stream>>>((const double*)s, h->Pd, rho, ux, uy, T); break;
    case CLB_F32: k_fields<ST_F32><<<grid, block, 0, h->stream>>>((const float*)s, h->Pf, rho, ux, uy, T); break;
    default: k_fields<ST_F16DEV><<<grid, block, 0, h->stream>>>((const __half*)s, h->Pf, rho, ux, uy, T); break;
    }
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

// Diagnostics into h->diag (device) and h->host_diag (after sync).
clb_status run_diagnostics(clb_handle* h, int axis, int update)
{
    const void* s = h->buf[h->cur];
    const int nseg = diag_segments(h->nx);
    const int rows = h->ny * nseg;  // partial entries
    switch (h->p.storage) {
    case CLB_F64: k_reduce_nodes<ST_F64><<<rows, kReduceThreads, 0, h->stream>>>((const double*)s, h->Pd, axis, h->snap, update, h->partial, nseg); break;
    case CLB_F32: k_reduce_nodes<ST_F32><<<rows, kReduceThreads, 0, h->stream>>>((const float*)s, h->Pf, axis, (float*)h->snap, update, h->partial, nseg); break;
    default: k_reduce_nodes<ST_F16DEV><<<rows, kReduceThreads, 0, h->stream>>>((const __half*)s, h->Pf, axis, (float*)h->snap, update, h->partial, nseg); break;
    }
    CLB_CUDA(cudaGetLastError());
    const NuGeom g = nu_geom(h->nx, h->ny, h->p, axis);
    k_reduce_final<<<1, kReduceThreads, 0, h->stream>>>(h->partial, rows, double(h->nx) * h->ny, g.cells,
                                                        g.H, g.dT, g.sign, h->p.kappa, h->p.u_ref,
                                                        h->p.dT_ref, h->diag);
    CLB_CUDA(cudaGetLastError());
    CLB_CUDA(cudaMemcpyAsync(h->host_diag, h->diag, (RS_N + 2) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    if (h->host_diag[RS_BAD] > 0)
        return set_error(CLB_ENAN, "%.0f nodes have non-finite fields after %ld steps", h->host_diag[RS_BAD], h->steps);
    return CLB_OK;
}

// The residual's snapshot of the current fields, in the arithmetic precision (k_snap).
clb_status take_snapshot(clb_handle* h)
{
    const dim3 block(128, 1), grid = grid_for(h, 128, 1);
    const void* s = h->buf[h->cur];
    switch (h->p.storage) {
    case CLB_F64: k_snap<ST_F64><<<grid, block, 0, h->stream>>>((const double*)s, h->Pd, h->snap); break;
    case CLB_F32: k_snap<ST_F32><<<grid, block, 0, h->stream>>>((const float*)s, h->Pf, (float*)h->snap); break;
    default: k_snap<ST_F16DEV><<<grid, block, 0, h->stream>>>((const __half*)s, h->Pf, (float*)h->snap); break;
    }
    CLB_CUDA(cudaGetLastError());
    return CLB_OK;
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, std::array<int, 5>> g_tune_cache;

}  // namespace

#define CHECK_H(h) \
    do { if (!(h)) return set_error(CLB_EINVAL, "handle is NULL"); } while (0)

extern "C" clb_status clb_footprint(int nx, int ny, const clb_params* p, size_t* bytes)
{
    CLB_TRY(validate(nx, ny, p));
    if (!bytes) return set_error(CLB_EINVAL, "bytes is NULL");
    *bytes = layout(nx, ny, p->storage).total;
    return CLB_OK;
}

extern "C" clb_status clb_create(int nx, int ny, const clb_params* p, void* stream, void* dev_mem,
                                 size_t dev_bytes, clb_handle** out)
{
    try {
        if (!out) return set_error(CLB_EINVAL, "out is NULL");
        *out = nullptr;
        CLB_TRY(validate(nx, ny, p));
        const Layout L = layout(nx, ny, p->storage);
        if (dev_mem && dev_bytes < L.total)
            return set_error(CLB_EINVAL, "dev_bytes %zu < footprint %zu", dev_bytes, L.total);
        if (dev_mem && ((uintptr_t)dev_mem & 255))
            return set_error(CLB_EINVAL, "dev_mem must be 256-byte aligned");
        clb_handle* h = new clb_handle;
        h->nx = nx;
        h->ny = ny;
        h->p = *p;
        h->L = L;
        h->stream = (cudaStream_t)stream;
        cudaGetDevice(&h->device);
        auto fail = [&](clb_status st) {
            clb_destroy(h);
            return st;
        };
        cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(set_error(CLB_ECUDA, "stream: %s", cudaGetErrorString(e)));
        if (dev_mem) {
            h->mem = (char*)dev_mem;
        } else {
            e = cudaMalloc((void**)&h->mem, L.total);
            if (e != cudaSuccess)
                return fail(set_error(e == cudaErrorMemoryAllocation ? CLB_ENOMEM : CLB_ECUDA,
                                      "cudaMalloc(%zu): %s", L.total, cudaGetErrorString(e)));
            h->own_mem = true;
        }
        e = cudaMallocHost((void**)&h->host_diag, 16 * sizeof(double));
        if (e != cudaSuccess) return fail(set_error(CLB_ECUDA, "cudaMallocHost: %s", cudaGetErrorString(e)));
        h->buf[0] = h->mem + L.buf[0];
        h->buf[1] = h->mem + L.buf[1];
        h->snap = (double*)(h->mem + L.snap);
        h->stage = (double*)(h->mem + L.stage);
        h->partial = (double*)(h->mem + L.partial);
        h->diag = (double*)(h->mem + L.diag);
        h->Pd = make_lat_params<double>(nx, ny, *p);
        h->Pf = make_lat_params<float>(nx, ny, *p);
        h->npt = p->storage == CLB_F32 ? 2 : 4;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(std::make_tuple(p->storage, nx, ny));
            if (it != g_tune_cache.end()) {
                h->bx = it->second[0];
                h->by = it->second[1];
                h->npt = it->second[2];
                h->pipe_stages = it->second[3];
                h->pipe_rows = it->second[4];
            }
        }
        // the padding of each row's last chunk is never read, but keep it defined
        e = cudaMemsetAsync(h->mem, 0, L.snap, h->stream);
        if (e != cudaSuccess) return fail(set_error(CLB_ECUDA, "memset: %s", cudaGetErrorString(e)));
        clb_status st = launch_init(h, nullptr, nullptr, nullptr, nullptr);
        if (st == CLB_OK) st = take_snapshot(h);
        if (st == CLB_OK) {
            e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) st = set_error(CLB_ECUDA, "init: %s", cudaGetErrorString(e));
        }
        if (st != CLB_OK) return fail(st);
        *out = h;
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" void clb_destroy(clb_handle* h)
{
    if (!h) return;
    DeviceGuard dg(h->device);
    if (h->stream || h->cap) cudaStreamSynchronize(h->stream);
    drop_graphs(h);
    if (h->own_mem && h->mem) cudaFree(h->mem);
    if (h->host_diag) cudaFreeHost(h->host_diag);
    if (h->side) cudaStreamSynchronize(h->side);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    delete h;
}

extern "C" clb_status clb_init_fields_device(clb_handle* h, const double* rho, const double* ux,
                                             const double* uy, const double* T)
{
    CHECK_H(h);
    DeviceGuard dg(h->device);
    h->steps = 0;
    CLB_TRY(launch_init(h, rho, ux, uy, T));
    return take_snapshot(h);
}

namespace {
// The address at which the current device reads or writes host memory directly: pinned host
// memory (cudaMallocHost, cudaHostAlloc, cudaHostRegister; mapped under unified addressing), over
// the CPU-GPU link. NULL for ordinary pageable memory, which goes through a staging copy instead.
void* device_view(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
}  // namespace

extern "C" clb_status clb_init_fields(clb_handle* h, const double* rho, const double* ux,
                                      const double* uy, const double* T)
{
    TraceRange trace("clb_init_fields");
    CHECK_H(h);
    DeviceGuard dg(h->device);
    const size_t N = (size_t)h->nx * h->ny;
    const double* src[4] = {rho, ux, uy, T};
    const double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k)
        if (src[k]) {
            // pinned host arrays are read by the initialisation kernel itself; pageable ones are staged
            dev[k] = (const double*)device_view(src[k]);
            if (dev[k]) continue;
            CLB_CUDA(cudaMemcpyAsync(h->stage + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
            dev[k] = h->stage + k * N;
        }
    CLB_TRY(clb_init_fields_device(h, dev[0], dev[1], dev[2], dev[3]));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb_step(clb_handle* h, long n)
{
    TraceRange trace("clb_step");
    CHECK_H(h);
    if (n < 0) return set_error(CLB_EINVAL, "n = %ld < 0", n);
    DeviceGuard dg(h->device);
    // Both parities are captured on the first chunk: a later odd number of single launches then
    // switches to the other graph without a capture in the middle of the caller's stepping.
    if (n >= kGraphChunk && (!h->graph[0] || !h->graph[1])) {
        for (int par = 0; par < 2; ++par)
            if (!h->graph[par]) CLB_TRY(build_graph(h, par));
    }
    while (n >= kGraphChunk) {
        CLB_CUDA(cudaGraphLaunch(h->graph[h->cur], h->stream));
        n -= kGraphChunk;
        h->steps += kGraphChunk;
    }
    for (; n > 0; --n) {
        CLB_TRY(launch_step(h, h->cur, h->stream, current_launch(h)));
        h->cur ^= 1;
        h->steps++;
    }
    return CLB_OK;
}

extern "C" clb_status clb_fields_device(clb_handle* h, double* rho, double* ux, double* uy, double* T)
{
    CHECK_H(h);
    DeviceGuard dg(h->device);
    return launch_fields(h, rho, ux, uy, T);
}

extern "C" clb_status clb_fields(clb_handle* h, double* rho, double* ux, double* uy, double* T)
{
    TraceRange trace("clb_fields");
    CHECK_H(h);
    DeviceGuard dg(h->device);
    const size_t N = (size_t)h->nx * h->ny;
    double* host[4] = {rho, ux, uy, T};
    double* dev[4];
    bool staged[4];
    for (int k = 0; k < 4; ++k) {
        // pinned host arrays are written by the field kernel itself; pageable ones through staging
        dev[k] = host[k] ? (double*)device_view(host[k]) : nullptr;
        staged[k] = host[k] && !dev[k];
        if (staged[k]) dev[k] = h->stage + k * N;
    }
    CLB_TRY(launch_fields(h, dev[0], dev[1], dev[2], dev[3]));
    for (int k = 0; k < 4; ++k)
        if (staged[k]) CLB_CUDA(cudaMemcpyAsync(host[k], dev[k], N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

extern "C" clb_status clb_populations(clb_handle* h, double* f, double* g)
{
    CHECK_H(h);
    if (!f || !g) return set_error(CLB_EINVAL, "f and g must not be NULL");
    DeviceGuard dg(h->device);
    const size_t N = (size_t)h->nx * h->ny;
    double* d = nullptr;
    CLB_CUDA(cudaMallocAsync((void**)&d, 14 * N * sizeof(double), h->stream));
    const dim3 block(128, 1), grid = grid_for(h, 128, 1);
    const void* s = h->buf[h->cur];
    switch (h->p.storage) {
    case CLB_F64: k_pops<ST_F64><<<grid, block, 0, h->stream>>>((const double*)s, h->Pd, d, d + 9 * N); break;
    case CLB_F32: k_pops<ST_F32><<<grid, block, 0, h->stream>>>((const float*)s, h->Pf, d, d + 9 * N); break;
    default: k_pops<ST_F16DEV><<<grid, block, 0, h->stream>>>((const __half*)s, h->Pf, d, d + 9 * N); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g, d + 9 * N, 5 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return set_error(CLB_ECUDA, "populations: %s", cudaGetErrorString(e));
    return CLB_OK;
}

extern "C" clb_status clb_nusselt(clb_handle* h, int axis, double* nu_out)
{
    TraceRange trace("clb_nusselt");
    CHECK_H(h);
    if (axis != 0 && axis != 1) return set_error(CLB_EINVAL, "axis must be 0 or 1");
    if (!nu_out) return set_error(CLB_EINVAL, "nu_out is NULL");
    DeviceGuard dg(h->device);
    CLB_TRY(run_diagnostics(h, axis, 0));
    *nu_out = h->host_diag[RS_N];
    return CLB_OK;
}

extern "C" clb_status clb_residual(clb_handle* h, double* er_out)
{
    TraceRange trace("clb_residual");
    CHECK_H(h);
    if (!er_out) return set_error(CLB_EINVAL, "er_out is NULL");
    DeviceGuard dg(h->device);
    CLB_TRY(run_diagnostics(h, 1, 1));
    *er_out = h->host_diag[RS_N + 1];
    return CLB_OK;
}

extern "C" clb_status clb_check(clb_handle* h, int axis, double* nu_out, double* er_out)
{
    TraceRange trace("clb_check");
    CHECK_H(h);
    if (axis != 0 && axis != 1) return set_error(CLB_EINVAL, "axis must be 0 or 1");
    DeviceGuard dg(h->device);
    CLB_TRY(run_diagnostics(h, axis, 1));
    if (nu_out) *nu_out = h->host_diag[RS_N];
    if (er_out) *er_out = h->host_diag[RS_N + 1];
    return CLB_OK;
}

extern "C" clb_status clb_run(clb_handle* h, double tol, long max_steps, long interval,
                              long* steps_out, double* er_out)
{
    TraceRange trace("clb_run");
    CHECK_H(h);
    if (interval <= 0 || max_steps < 0) return set_error(CLB_EINVAL, "interval must be > 0 and max_steps >= 0");
    DeviceGuard dg(h->device);
    long done = 0;
    double er = INFINITY;
    clb_status st = CLB_OK;
    while (done < max_steps) {
        const long n = std::min(interval, max_steps - done);
        CLB_TRY(clb_step(h, n));
        done += n;
        st = run_diagnostics(h, 1, 1);
        if (st != CLB_OK) break;
        er = h->host_diag[RS_N + 1];
        if (er < tol) break;
    }
    if (steps_out) *steps_out = done;
    if (er_out) *er_out = er;
    return st;
}

extern "C" clb_status clb_steps(clb_handle* h, long* steps_out)
{
    CHECK_H(h);
    if (!steps_out) return set_error(CLB_EINVAL, "steps_out is NULL");
    *steps_out = h->steps;
    return CLB_OK;
}

extern "C" clb_status clb_sync(clb_handle* h)
{
    CHECK_H(h);
    DeviceGuard dg(h->device);
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    return CLB_OK;
}

namespace {
struct CkptHeader {
    char magic[8];
    int nx, ny, storage, pad;
    long long steps;
    unsigned long long bytes;
};
}  // namespace

extern "C" clb_status clb_save(clb_handle* h, void* buf, size_t* bytes)
{
    CHECK_H(h);
    if (!bytes) return set_error(CLB_EINVAL, "bytes is NULL");
    const size_t bb = buffer_bytes(h->nx, h->ny, h->p.storage);
    const size_t need = sizeof(CkptHeader) + bb;
    if (!buf) {
        *bytes = need;
        return CLB_OK;
    }
    if (*bytes < need) return set_error(CLB_EINVAL, "checkpoint buffer %zu < %zu", *bytes, need);
    DeviceGuard dg(h->device);
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, "CLBCKPT2", 8);
    hd.nx = h->nx;
    hd.ny = h->ny;
    hd.storage = h->p.storage;
    hd.steps = h->steps;
    hd.bytes = bb;
    std::memcpy(buf, &hd, sizeof(hd));
    CLB_CUDA(cudaMemcpyAsync((char*)buf + sizeof(hd), h->buf[h->cur], bb, cudaMemcpyDeviceToHost, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    *bytes = need;
    return CLB_OK;
}

extern "C" clb_status clb_load(clb_handle* h, const void* buf, size_t bytes)
{
    CHECK_H(h);
    if (!buf || bytes < sizeof(CkptHeader)) return set_error(CLB_EINVAL, "checkpoint too small");
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    const size_t bb = buffer_bytes(h->nx, h->ny, h->p.storage);
    if (std::memcmp(hd.magic, "CLBCKPT2", 8) != 0 || hd.nx != h->nx || hd.ny != h->ny ||
        hd.storage != h->p.storage || hd.bytes != bb || bytes < sizeof(hd) + bb)
        return set_error(CLB_EINVAL, "checkpoint does not match this lattice");
    DeviceGuard dg(h->device);
    CLB_CUDA(cudaMemcpyAsync(h->buf[h->cur], (const char*)buf + sizeof(hd), bb, cudaMemcpyHostToDevice, h->stream));
    CLB_CUDA(cudaStreamSynchronize(h->stream));
    h->steps = hd.steps;
    return CLB_OK;
}

namespace {
clb_status check_launch(const clb_handle* h, const Launch& L)
{
    if (L.bx < 32 || L.bx > 256 || L.bx % 32 || L.by < 1 || L.by > 8 || L.bx * L.by > 256 ||
        (L.npt != 1 && L.npt != 2 && L.npt != 4))
        return set_error(CLB_EINVAL, "launch shape %d x %d x %d: block_x in [32, 256] multiple of 32, "
                                     "block_y in [1, 8], block_x * block_y <= 256, nodes per thread 1, 2 or 4",
                         L.bx, L.by, L.npt);
    if (L.stages != 0 && (L.stages < 2 || L.stages > 4 || L.rows < 1 || L.rows > 256 || L.npt == 1))
        return set_error(CLB_EINVAL, "pipeline %d stages x %d rows: stages 0 (off) or 2..4, rows 1..256, "
                                     "and 2 or 4 nodes per thread", L.stages, L.rows);
    if (L.stages != 0) {
        const size_t e = elem_size(h->p.storage);
        const size_t smem = (size_t)kPipeWarps * L.stages * NPOP * (32 * L.npt + 16 / e) * e;
        if (smem > 227 * 1024)
            return set_error(CLB_EINVAL, "pipeline needs %zu bytes of shared memory per block (max 232448)", smem);
    }
    return CLB_OK;
}

clb_status apply_launch(clb_handle* h, const Launch& L)
{
    CLB_TRY(check_launch(h, L));
    const Launch c = current_launch(h);
    if (c.bx != L.bx || c.by != L.by || c.npt != L.npt || c.stages != L.stages || c.rows != L.rows) {
        DeviceGuard dg(h->device);
        cudaStreamSynchronize(h->stream);
        drop_graphs(h);
        h->bx = L.bx;
        h->by = L.by;
        h->npt = L.npt;
        h->pipe_stages = L.stages;
        h->pipe_rows = L.rows;
    }
    return CLB_OK;
}
}  // namespace

extern "C" clb_status clb_set_launch(clb_handle* h, int block_x, int block_y, int nodes_per_thread)
{
    CHECK_H(h);
    Launch L = current_launch(h);
    if (block_x) L.bx = block_x;
    if (block_y) L.by = block_y;
    if (nodes_per_thread) L.npt = nodes_per_thread;
    if (L.npt == 1) L.stages = 0;
    return apply_launch(h, L);
}

extern "C" clb_status clb_set_pipeline(clb_handle* h, int stages, int rows)
{
    CHECK_H(h);
    Launch L = current_launch(h);
    L.stages = stages;
    if (rows) L.rows = rows;
    return apply_launch(h, L);
}

extern "C" clb_status clb_get_launch(clb_handle* h, int* block_x, int* block_y, int* nodes_per_thread)
{
    CHECK_H(h);
    if (block_x) *block_x = h->bx;
    if (block_y) *block_y = h->by;
    if (nodes_per_thread) *nodes_per_thread = h->npt;
    return CLB_OK;
}

extern "C" clb_status clb_get_pipeline(clb_handle* h, int* stages, int* rows)
{
    CHECK_H(h);
    if (stages) *stages = h->pipe_stages;
    if (rows) *rows = h->pipe_rows;
    return CLB_OK;
}

extern "C" clb_status clb_autotune(clb_handle* h, int* block_x, int* block_y, int* nodes_per_thread)
{
    TraceRange trace("clb_autotune");
    try {
        CHECK_H(h);
        DeviceGuard dg(h->device);
        const size_t bb = buffer_bytes(h->nx, h->ny, h->p.storage);
        void* save = nullptr;
        CLB_CUDA(cudaMallocAsync(&save, bb, h->stream));
        CLB_CUDA(cudaMemcpyAsync(save, h->buf[h->cur], bb, cudaMemcpyDeviceToDevice, h->stream));
        std::vector<Launch> cands;
        const int shapes[][2] = {{64, 1}, {128, 1}, {256, 1}, {32, 4}, {64, 2}, {128, 2}};
        for (int npt : {1, 2, 4})
            for (auto& sh : shapes) cands.push_back({sh[0], sh[1], npt, 0, 8});
        for (int npt : {2, 4})
            for (int st : {2, 3, 4})
                for (int rows : {4, 8, 16}) cands.push_back({128, 1, npt, st, rows});
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        Launch bl = current_launch(h);
        const int reps = 10;
        clb_status st = CLB_OK;
        for (const Launch& c : cands) {
            if (c.bx * c.npt > 2 * h->nx + 64 && c.bx * c.npt > 64) continue;  // far wider than the lattice
            if (c.stages > 0 && check_launch(h, c) != CLB_OK) continue;
            for (int k = 0; k < 4 && st == CLB_OK; ++k) st = launch_step(h, (h->cur + k) & 1, h->stream, c);
            cudaEventRecord(e0, h->stream);
            for (int k = 0; k < reps && st == CLB_OK; ++k) st = launch_step(h, (h->cur + k) & 1, h->stream, c);
            cudaEventRecord(e1, h->stream);
            if (st != CLB_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bl = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaError_t e = cudaMemcpyAsync(h->buf[h->cur], save, bb, cudaMemcpyDeviceToDevice, h->stream);
        cudaFreeAsync(save, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (st != CLB_OK) return st;
        if (e != cudaSuccess) return set_error(CLB_ECUDA, "autotune restore: %s", cudaGetErrorString(e));
        CLB_TRY(apply_launch(h, bl));
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[std::make_tuple(h->p.storage, h->nx, h->ny)] = {bl.bx, bl.by, bl.npt, bl.stages, bl.rows};
        }
        if (block_x) *block_x = bl.bx;
        if (block_y) *block_y = bl.by;
        if (nodes_per_thread) *nodes_per_thread = bl.npt;
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" void* clb_stream(clb_handle* h) { return h ? (void*)h->stream : nullptr; }

extern "C" clb_status clb_step_partition(int nx, int ny, const clb_params* p, int npt, int* geom)
{
    if (!p || !geom) return set_error(CLB_EINVAL, "params or geom is NULL");
    if (npt != 1 && npt != 2 && npt != 4) return set_error(CLB_EINVAL, "nodes per thread %d: 1, 2 or 4", npt);
    const clb_status st = validate(nx, ny, p);
    if (st != CLB_OK) return st;
    try {
        const SplitGeom G = split_geom(nx, ny, make_lat_params<float>(nx, ny, *p), npt);
        const int out[11] = {G.y0, G.y1, G.c0, G.c1, G.nw, G.nyb, G.nyb > 0 ? G.yb[0] : -1, G.nyb > 1 ? G.yb[1] : -1,
                             G.ncb, G.ncb > 0 ? G.cb[0] : -1, G.ncb > 1 ? G.cb[1] : -1};
        std::memcpy(geom, out, sizeof(out));
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_buffers(clb_handle* h, void** cur, void** other, size_t* row_elems, int* chunk)
{
    CHECK_H(h);
    if (cur) *cur = h->buf[h->cur];
    if (other) *other = h->buf[h->cur ^ 1];
    if (row_elems) *row_elems = (size_t)chunked_row_elems(h->nx);
    if (chunk) *chunk = kRowChunk;
    return CLB_OK;
}
