// clb_batch.cu -- many independent lattices stepped together (include/clb.h: clb_batch_*,
// clb_serve_*). An ensemble holds the resident lattices; one launch per time step covers the
// concatenated tiles of all of them (a block finds its lattice through a tile-owner table) and is
// captured in a CUDA graph. The per-node arithmetic is the same device code as the single-lattice
// step, so each lattice evolves exactly as it would alone. Diagnostics run one block per
// (lattice, row) with the same fixed-order sums as a single lattice.
#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "clb_kernels.cuh"

using namespace clb;

namespace {

// Everything a block needs about its lattice (copied to shared memory by the block).
template <typename A>
struct Member {
    LatParams<A> P;
    void* buf[2];
    double* snap;
    double* partial;
    double* diag;
    int tiles_x;
    int tile_begin;
    int row_begin;
    int axis;
    double nodes, cells, H, dT, sign, kappa, u_ref, dT_ref;
};

template <typename A>
__device__ __forceinline__ void load_member(const Member<A>* __restrict__ src, Member<A>& dst)
{
    static_assert(sizeof(Member<A>) % 4 == 0, "member size");
    const int words = sizeof(Member<A>) / 4;
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(&dst);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    for (int w = tid; w < words; w += nt) d[w] = s[w];
    __syncthreads();
}

// One time step of every lattice: block b covers tile (b - tile_begin) of lattice owner[b]; a
// tile is (blockDim.x * V) x (blockDim.y * groups) nodes, V consecutive nodes per thread (the
// same per-warp update as the single-lattice step), each warp stepping `groups` rows.
// Register cap: the FP32 two-nodes-per-thread form (the default tile) is held at 96 registers so
// that five 128-thread blocks stay resident per SM; the other forms take what they need (blocks
// have at most 256 threads).
template <int ST, int V>
__global__ void __maxnreg__((ST == ST_F32 && V == 2) ? 96 : 255) k_step_batched(const Member<typename Storage<ST>::A>* __restrict__ mem,
                                                      const int* __restrict__ owner, int parity, int groups)
{
    using A = typename Storage<ST>::A;
    using E = typename Storage<ST>::T;
    __shared__ Member<A> M;
    load_member(mem + owner[blockIdx.x], M);
    const int t = blockIdx.x - M.tile_begin;
    const int tx = t % M.tiles_x, ty = t / M.tiles_x;
    const int lane = threadIdx.x & 31;
    const int span = blockDim.x * V;
    int xt = tx * span, keep = 0;
    // The last tile of a row that would run past the row's end is moved left to end on the last
    // multiple of V below nx (tail), so that its warps take the vector path (walls included)
    // instead of node-by-node gathers; the nodes it shares with the tile before it are computed
    // alike and stored by that tile only, and the nx % V nodes from tail on are updated node by
    // node by the thread holding the tile's last vector. The moved start stays a multiple of V, so the vector loads stay aligned.
    // A tile that would store no vector node (xt == tail) is not moved.
    const int tail = M.P.nx - M.P.nx % V;
    const bool moved = xt + span > M.P.nx && xt < tail && tail >= span;
    if (moved) {
        keep = xt;
        xt = tail - span;
    }
    const int x0 = xt + threadIdx.x * V;
    if (x0 - lane * V >= M.P.nx) return;  // whole warps only
    const E* src = (const E*)M.buf[parity];
    E* dst = (E*)M.buf[parity ^ 1];
    // The tile's rows: `groups` groups of blockDim.y rows, one group after another, so that the
    // descriptor fetched above serves several rows per warp.
    const int rows = blockDim.y * groups;
    const int y_end = min(M.P.ny, (ty + 1) * rows);
    for (int y = ty * rows + threadIdx.y; y < y_end; y += blockDim.y) {
        step_warp_nodes<ST, V, false>(src, dst, M.P, x0, y, lane, keep);
        if (moved && x0 + V == tail)
            for (int x = tail; x < M.P.nx; ++x) {
                A f[9], g[5];
                gather(src, M.P, x, y, f, g);
                collide_any<Storage<ST>::DEV>(M.P, f, g);
                store_node(dst, M.P, x, y, f, g);
            }
    }
}

// Blocks of k_step_batched<ST, V> resident on the whole device at once.
template <int ST, int V>
long resident_blocks_of(int threads)
{
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_batched<ST, V>, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return (long)std::max(1, sms) * std::max(1, per_sm);
}

template <int ST>
long resident_blocks_npt(int npt, int threads)
{
    return npt == 4 ? resident_blocks_of<ST, 4>(threads)
                    : npt == 2 ? resident_blocks_of<ST, 2>(threads) : resident_blocks_of<ST, 1>(threads);
}

template <int ST>
__global__ void __launch_bounds__(kReduceThreads) k_reduce_rows_batched(
    const Member<typename Storage<ST>::A>* __restrict__ mem, const int* __restrict__ row_owner,
    int parity, int update)
{
    using A = typename Storage<ST>::A;
    using E = typename Storage<ST>::T;
    __shared__ Member<A> M;
    load_member(mem + row_owner[blockIdx.x], M);
    const int y = blockIdx.x - M.row_begin;
    reduce_row((const E*)M.buf[parity], M.P, y, M.axis, M.snap, update, M.partial + (long long)y * RS_N);
}

template <typename A>
__global__ void __launch_bounds__(kReduceThreads) k_reduce_final_batched(const Member<A>* __restrict__ mem)
{
    __shared__ Member<A> M;
    load_member(mem + blockIdx.x, M);
    reduce_final(M.partial, M.P.ny, M.nodes, M.cells, M.H, M.dT, M.sign, M.kappa, M.u_ref, M.dT_ref, M.diag);
}

// A resident lattice (host bookkeeping).
struct Lattice {
    int nx = 0, ny = 0;
    clb_params p{};
    int axis = 1;
    char* mem = nullptr;  // device block: buf0 | buf1 | snap | partial | diag
    size_t bytes = 0;
    void* buf[2] = {nullptr, nullptr};
    double* snap = nullptr;
    double* partial = nullptr;
    double* diag = nullptr;
    long steps = 0;
    double nu = 0, er = INFINITY;
    int status = CLB_OK;
    bool active = true;
};

size_t lattice_bytes(int nx, int ny, int storage)
{
    const size_t N = (size_t)nx * ny;
    return 2 * buffer_slot_bytes(nx, ny, storage) + align256(3 * N * sizeof(double)) +
           align256((size_t)ny * RS_N * sizeof(double)) + align256(16 * sizeof(double));
}

void carve(Lattice& L, char* base)
{
    const size_t N = (size_t)L.nx * L.ny;
    const size_t bb = buffer_slot_bytes(L.nx, L.ny, L.p.storage);
    L.mem = base;
    L.buf[0] = base;
    L.buf[1] = base + bb;
    L.snap = (double*)(base + 2 * bb);
    L.partial = (double*)(base + 2 * bb + align256(3 * N * sizeof(double)));
    L.diag = (double*)((char*)L.partial + align256((size_t)L.ny * RS_N * sizeof(double)));
}

template <typename A>
Member<A> make_member(const Lattice& L, int tile_x, int npt, int tile_begin, int row_begin)
{
    Member<A> m;
    std::memset(&m, 0, sizeof(m));
    m.P = make_lat_params<A>(L.nx, L.ny, L.p);
    m.buf[0] = L.buf[0];
    m.buf[1] = L.buf[1];
    m.snap = L.snap;
    m.partial = L.partial;
    m.diag = L.diag;
    m.tiles_x = (L.nx + tile_x * npt - 1) / (tile_x * npt);
    m.tile_begin = tile_begin;
    m.row_begin = row_begin;
    m.axis = L.axis;
    const NuGeom g = nu_geom(L.nx, L.ny, L.p, L.axis);
    m.nodes = double(L.nx) * L.ny;
    m.cells = g.cells;
    m.H = g.H;
    m.dT = g.dT;
    m.sign = g.sign;
    m.kappa = L.p.kappa;
    m.u_ref = L.p.u_ref;
    m.dT_ref = L.p.dT_ref;
    return m;
}

constexpr int kChunk = 32;  // steps per captured graph (even, so the buffers return)

// Nodes a block of the batched step covers at most: each block first fetches its lattice's
// descriptor (two dependent loads and a barrier), so a block that steps only one group of rows
// spends a large part of its short life waiting on that fetch. On 256 uneven cavities (FP32,
// 32 x 4 threads x 2 nodes) 1, 2, 4, 8 and 16 groups of rows per block gave 42.9, 46.9, 49.2,
// 49.6 and 48.3 GLUPS. Fewer, longer blocks leave a longer tail at the end of the launch, so the
// number of groups is also held where the launch still has kMinWaves rounds of resident blocks.
constexpr int kBlockNodes = 2048;
constexpr int kMinWaves = 8;

// The set of resident lattices and the device tables of the batched launch.
class Ensemble {
public:
    int storage = CLB_F32;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int tile_x = 128, tile_y = 1, npt = 1;
    int groups = 1;  // row groups per block (kBlockNodes): a tile is (tile_x * npt) x (tile_y * groups) nodes
    int parity = 0;  // every resident lattice holds its current data in buf[parity]
    std::vector<Lattice*> members;  // launch order

    ~Ensemble()
    {
        if (graph) cudaGraphExecDestroy(graph);
        cudaFree(d_members);
        cudaFree(d_owner);
        cudaFree(d_row_owner);
        if (h_diag) cudaFreeHost(h_diag);
        if (cap) cudaStreamDestroy(cap);
    }

    clb_status init(int st, cudaStream_t s)
    {
        storage = st;
        stream = s;
        // Default tile: 32 x 4 threads with two nodes per thread (packed f32x2) for the FP32 and
        // FP16 forms, the shape the autotuner picks on uneven batches (43.6 GLUPS on 256 cavities
        // against 31 for one node per thread); the server, which does not autotune, runs on it.
        if (st != CLB_F64) {
            tile_x = 32;
            tile_y = 4;
            npt = 2;
        }
        CLB_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        return CLB_OK;
    }

    void mark_dirty() { dirty = true; }

    // Tiles of the active members when each block steps g groups of tile_y rows.
    long tiles_with(int g) const
    {
        long t = 0;
        for (const Lattice* L : active)
            t += (long)((L->nx + tile_x * npt - 1) / (tile_x * npt)) * ((L->ny + tile_y * g - 1) / (tile_y * g));
        return t;
    }

    // Groups of rows per block: doubled while a block covers at most kBlockNodes nodes and the
    // launch keeps kMinWaves rounds of resident blocks.
    void choose_groups()
    {
        const int threads = tile_x * tile_y;
        const long resident = storage == CLB_F64 ? resident_blocks_npt<ST_F64>(npt, threads)
                              : storage == CLB_F32 ? resident_blocks_npt<ST_F32>(npt, threads)
                                                   : resident_blocks_npt<ST_F16DEV>(npt, threads);
        groups = 1;
        for (int g = 2; g * threads * npt <= kBlockNodes && tiles_with(g) >= kMinWaves * resident; g *= 2) groups = g;
    }

    // Rebuild the tile and row tables for the active members.
    clb_status rebuild()
    {
        if (!dirty) return CLB_OK;
        if (graph) {
            cudaGraphExecDestroy(graph);
            graph = nullptr;
        }
        active.clear();
        for (Lattice* L : members)
            if (L->active) active.push_back(L);
        choose_groups();
        std::vector<int> owner, row_owner;
        const size_t msz = storage == CLB_F64 ? sizeof(Member<double>) : sizeof(Member<float>);
        std::vector<char> host(msz * std::max<size_t>(1, active.size()));
        int tiles = 0, rows = 0;
        for (size_t k = 0; k < active.size(); ++k) {
            const Lattice& L = *active[k];
            const int tx = (L.nx + tile_x * npt - 1) / (tile_x * npt), ty = (L.ny + tile_y * groups - 1) / (tile_y * groups);
            if (storage == CLB_F64) {
                Member<double> m = make_member<double>(L, tile_x, npt, tiles, rows);
                std::memcpy(host.data() + k * msz, &m, msz);
            } else {
                Member<float> m = make_member<float>(L, tile_x, npt, tiles, rows);
                std::memcpy(host.data() + k * msz, &m, msz);
            }
            owner.insert(owner.end(), (size_t)tx * ty, int(k));
            row_owner.insert(row_owner.end(), (size_t)L.ny, int(k));
            tiles += tx * ty;
            rows += L.ny;
        }
        ntiles = tiles;
        nrows = rows;
        CLB_TRY(ensure(d_members, members_cap, host.size()));
        CLB_TRY(ensure(d_owner, owner_cap, std::max<size_t>(1, owner.size()) * sizeof(int)));
        CLB_TRY(ensure(d_row_owner, row_cap, std::max<size_t>(1, row_owner.size()) * sizeof(int)));
        if (!active.empty()) {
            CLB_CUDA(cudaMemcpyAsync(d_members, host.data(), host.size(), cudaMemcpyHostToDevice, stream));
            CLB_CUDA(cudaMemcpyAsync(d_owner, owner.data(), owner.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
            CLB_CUDA(cudaMemcpyAsync(d_row_owner, row_owner.data(), row_owner.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
            // the host vectors die at return: wait for the copies
            CLB_CUDA(cudaStreamSynchronize(stream));
        }
        if (h_diag_cap < active.size()) {
            if (h_diag) cudaFreeHost(h_diag);
            h_diag = nullptr;
            CLB_CUDA(cudaMallocHost((void**)&h_diag, std::max<size_t>(1, active.size()) * 16 * sizeof(double)));
            h_diag_cap = active.size();
        }
        dirty = false;
        return CLB_OK;
    }

    template <int ST>
    void enqueue(cudaStream_t s, int par)
    {
        using A = typename Storage<ST>::A;
        const dim3 block(tile_x, tile_y);
        const Member<A>* m = (const Member<A>*)d_members;
        if (npt == 4) k_step_batched<ST, 4><<<ntiles, block, 0, s>>>(m, d_owner, par, groups);
        else if (npt == 2) k_step_batched<ST, 2><<<ntiles, block, 0, s>>>(m, d_owner, par, groups);
        else k_step_batched<ST, 1><<<ntiles, block, 0, s>>>(m, d_owner, par, groups);
    }

    clb_status launch_step(cudaStream_t s, int par)
    {
        if (ntiles == 0) return CLB_OK;
        switch (storage) {
        case CLB_F64: enqueue<ST_F64>(s, par); break;
        case CLB_F32: enqueue<ST_F32>(s, par); break;
        default: enqueue<ST_F16DEV>(s, par); break;
        }
        CLB_CUDA(cudaGetLastError());
        return CLB_OK;
    }

    clb_status step(long n)
    {
        CLB_TRY(rebuild());
        if (active.empty() || n <= 0) return CLB_OK;
        while (n >= kChunk) {
            if (!graph || graph_parity != parity) {
                if (graph) cudaGraphExecDestroy(graph);
                graph = nullptr;
                CLB_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
                clb_status st = CLB_OK;
                for (int k = 0; k < kChunk && st == CLB_OK; ++k) st = launch_step(cap, parity ^ (k & 1));
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamEndCapture(cap, &g);
                if (st != CLB_OK) {
                    if (g) cudaGraphDestroy(g);
                    return st;
                }
                if (e != cudaSuccess) return set_error(CLB_ECUDA, "capture: %s", cudaGetErrorString(e));
                e = cudaGraphInstantiate(&graph, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return set_error(CLB_ECUDA, "instantiate: %s", cudaGetErrorString(e));
                graph_parity = parity;
            }
            CLB_CUDA(cudaGraphLaunch(graph, stream));
            for (Lattice* L : active) L->steps += kChunk;
            n -= kChunk;
        }
        for (; n > 0; --n) {
            CLB_TRY(launch_step(stream, parity));
            parity ^= 1;
            for (Lattice* L : active) L->steps++;
        }
        return CLB_OK;
    }

    // Nu and E_R (snapshot retaken when update) of every active member; sets L->nu, L->er, status.
    clb_status diagnostics(int update)
    {
        CLB_TRY(rebuild());
        if (active.empty()) return CLB_OK;
        switch (storage) {
        case CLB_F64: k_reduce_rows_batched<ST_F64><<<nrows, kReduceThreads, 0, stream>>>((const Member<double>*)d_members, d_row_owner, parity, update); break;
        case CLB_F32: k_reduce_rows_batched<ST_F32><<<nrows, kReduceThreads, 0, stream>>>((const Member<float>*)d_members, d_row_owner, parity, update); break;
        default: k_reduce_rows_batched<ST_F16DEV><<<nrows, kReduceThreads, 0, stream>>>((const Member<float>*)d_members, d_row_owner, parity, update); break;
        }
        CLB_CUDA(cudaGetLastError());
        if (storage == CLB_F64)
            k_reduce_final_batched<double><<<(int)active.size(), kReduceThreads, 0, stream>>>((const Member<double>*)d_members);
        else
            k_reduce_final_batched<float><<<(int)active.size(), kReduceThreads, 0, stream>>>((const Member<float>*)d_members);
        CLB_CUDA(cudaGetLastError());
        for (size_t k = 0; k < active.size(); ++k)
            CLB_CUDA(cudaMemcpyAsync(h_diag + 16 * k, active[k]->diag, (RS_N + 2) * sizeof(double), cudaMemcpyDeviceToHost, stream));
        CLB_CUDA(cudaStreamSynchronize(stream));
        for (size_t k = 0; k < active.size(); ++k) {
            Lattice* L = active[k];
            const double* d = h_diag + 16 * k;
            L->nu = d[RS_N];
            L->er = d[RS_N + 1];
            if (d[RS_BAD] > 0) L->status = CLB_ENAN;
        }
        return CLB_OK;
    }

    clb_status init_member(Lattice* L, const double* rho, const double* ux, const double* uy,
                           const double* T)
    {
        // fields are device pointers (or NULL); initialise buf[parity] and the snapshot
        const dim3 block(128, 1), grid((L->nx + 127) / 128, L->ny);
        void* d = L->buf[parity];
        const size_t N = (size_t)L->nx * L->ny;
        if (storage == CLB_F64) {
            const LatParams<double> P = make_lat_params<double>(L->nx, L->ny, L->p);
            k_init<ST_F64><<<grid, block, 0, stream>>>((double*)d, P, rho, ux, uy, T, L->p.rho0);
            k_fields<ST_F64><<<grid, block, 0, stream>>>((const double*)d, P, nullptr, L->snap, L->snap + N, L->snap + 2 * N);
        } else {
            const LatParams<float> P = make_lat_params<float>(L->nx, L->ny, L->p);
            if (storage == CLB_F32) {
                k_init<ST_F32><<<grid, block, 0, stream>>>((float*)d, P, rho, ux, uy, T, L->p.rho0);
                k_fields<ST_F32><<<grid, block, 0, stream>>>((const float*)d, P, nullptr, L->snap, L->snap + N, L->snap + 2 * N);
            } else {
                k_init<ST_F16DEV><<<grid, block, 0, stream>>>((__half*)d, P, rho, ux, uy, T, L->p.rho0);
                k_fields<ST_F16DEV><<<grid, block, 0, stream>>>((const __half*)d, P, nullptr, L->snap, L->snap + N, L->snap + 2 * N);
            }
        }
        CLB_CUDA(cudaGetLastError());
        L->steps = 0;
        return CLB_OK;
    }

    clb_status fields(Lattice* L, double* rho, double* ux, double* uy, double* T)
    {
        const dim3 block(128, 1), grid((L->nx + 127) / 128, L->ny);
        const void* d = L->buf[parity];
        if (storage == CLB_F64)
            k_fields<ST_F64><<<grid, block, 0, stream>>>((const double*)d, make_lat_params<double>(L->nx, L->ny, L->p), rho, ux, uy, T);
        else if (storage == CLB_F32)
            k_fields<ST_F32><<<grid, block, 0, stream>>>((const float*)d, make_lat_params<float>(L->nx, L->ny, L->p), rho, ux, uy, T);
        else
            k_fields<ST_F16DEV><<<grid, block, 0, stream>>>((const __half*)d, make_lat_params<float>(L->nx, L->ny, L->p), rho, ux, uy, T);
        CLB_CUDA(cudaGetLastError());
        return CLB_OK;
    }

    int ntiles = 0, nrows = 0;

private:
    clb_status ensure(void*& p, size_t& cap_bytes, size_t need)
    {
        if (cap_bytes >= need) return CLB_OK;
        CLB_CUDA(cudaStreamSynchronize(stream));
        cudaFree(p);
        p = nullptr;
        CLB_CUDA(cudaMalloc(&p, need));
        cap_bytes = need;
        return CLB_OK;
    }
    template <typename P>
    clb_status ensure(P*& p, size_t& cap_bytes, size_t need)
    {
        void* v = p;
        clb_status st = ensure(v, cap_bytes, need);
        p = (P*)v;
        return st;
    }

    bool dirty = true;
    std::vector<Lattice*> active;
    void* d_members = nullptr;
    size_t members_cap = 0;
    int* d_owner = nullptr;
    size_t owner_cap = 0;
    int* d_row_owner = nullptr;
    size_t row_cap = 0;
    double* h_diag = nullptr;
    size_t h_diag_cap = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_parity = 0;
};

// Stage host fields into device memory (double [4][N]) and initialise a member.
clb_status init_from_host(Ensemble& E, Lattice* L, double* stage, const double* rho, const double* ux,
                          const double* uy, const double* T)
{
    const size_t N = (size_t)L->nx * L->ny;
    const double* src[4] = {rho, ux, uy, T};
    const double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k)
        if (src[k]) {
            CLB_CUDA(cudaMemcpyAsync(stage + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, E.stream));
            dev[k] = stage + k * N;
        }
    CLB_TRY(E.init_member(L, dev[0], dev[1], dev[2], dev[3]));
    CLB_CUDA(cudaStreamSynchronize(E.stream));
    return CLB_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------ batches

struct clb_batch {
    Ensemble E;
    std::vector<std::unique_ptr<Lattice>> lat;
    char* mem = nullptr;
    double* stage = nullptr;
    int device = 0;
};

extern "C" clb_status clb_batch_create(int n, const int* nx, const int* ny, const clb_params* p,
                                       void* stream, clb_batch** out)
{
    try {
        if (!out) return set_error(CLB_EINVAL, "out is NULL");
        *out = nullptr;
        if (n <= 0 || !nx || !ny || !p) return set_error(CLB_EINVAL, "need n > 0 and nx, ny, p arrays");
        const int storage = p[0].storage;
        size_t total = 0, max_nodes = 0;
        for (int k = 0; k < n; ++k) {
            CLB_TRY(validate(nx[k], ny[k], &p[k]));
            if (p[k].storage != storage) return set_error(CLB_EINVAL, "instance %d: all instances need the same storage", k);
            total += lattice_bytes(nx[k], ny[k], storage);
            max_nodes = std::max(max_nodes, (size_t)nx[k] * ny[k]);
        }
        auto b = std::make_unique<clb_batch>();
        cudaGetDevice(&b->device);
        CLB_TRY(b->E.init(storage, (cudaStream_t)stream));
        const size_t stage_bytes = align256(4 * max_nodes * sizeof(double));
        CLB_CUDA(cudaMalloc((void**)&b->mem, total + stage_bytes));
        b->stage = (double*)(b->mem + total);
        CLB_CUDA(cudaMemsetAsync(b->mem, 0, total, b->E.stream));
        size_t off = 0;
        for (int k = 0; k < n; ++k) {
            auto L = std::make_unique<Lattice>();
            L->nx = nx[k];
            L->ny = ny[k];
            L->p = p[k];
            L->axis = p[k].wall[0] != CLB_PERIODIC ? 0 : 1;
            carve(*L, b->mem + off);
            off += lattice_bytes(nx[k], ny[k], storage);
            CLB_TRY(b->E.init_member(L.get(), nullptr, nullptr, nullptr, nullptr));
            b->E.members.push_back(L.get());
            b->lat.push_back(std::move(L));
        }
        CLB_CUDA(cudaStreamSynchronize(b->E.stream));
        *out = b.release();
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" void clb_batch_destroy(clb_batch* b)
{
    if (!b) return;
    cudaStreamSynchronize(b->E.stream);
    cudaFree(b->mem);
    delete b;
}

#define CHECK_B(b, k)                                                                      \
    do {                                                                                   \
        if (!(b)) return set_error(CLB_EINVAL, "batch is NULL");                           \
        if ((k) < 0 || (k) >= (int)(b)->lat.size())                                        \
            return set_error(CLB_EINVAL, "instance %d out of range [0, %zu)", (k), (b)->lat.size()); \
    } while (0)

extern "C" clb_status clb_batch_init_fields(clb_batch* b, int k, const double* rho, const double* ux,
                                            const double* uy, const double* T)
{
    try {
        CHECK_B(b, k);
        Lattice* L = b->lat[k].get();
        if (!L->active) {
            L->active = true;
            b->E.mark_dirty();
        }
        L->status = CLB_OK;
        L->er = INFINITY;
        return init_from_host(b->E, L, b->stage, rho, ux, uy, T);
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_batch_step(clb_batch* b, long n)
{
    TraceRange trace("clb_batch_step");
    try {
        if (!b) return set_error(CLB_EINVAL, "batch is NULL");
        if (n < 0) return set_error(CLB_EINVAL, "n < 0");
        return b->E.step(n);
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_batch_fields(clb_batch* b, int k, double* rho, double* ux, double* uy, double* T)
{
    try {
        CHECK_B(b, k);
        Lattice* L = b->lat[k].get();
        const size_t N = (size_t)L->nx * L->ny;
        double* host[4] = {rho, ux, uy, T};
        double* dev[4];
        for (int i = 0; i < 4; ++i) dev[i] = host[i] ? b->stage + i * N : nullptr;
        CLB_TRY(b->E.fields(L, dev[0], dev[1], dev[2], dev[3]));
        for (int i = 0; i < 4; ++i)
            if (host[i]) CLB_CUDA(cudaMemcpyAsync(host[i], dev[i], N * sizeof(double), cudaMemcpyDeviceToHost, b->E.stream));
        CLB_CUDA(cudaStreamSynchronize(b->E.stream));
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_batch_diagnostics(clb_batch* b, const int* axis, double* nu, double* er)
{
    TraceRange trace("clb_batch_diagnostics");
    try {
        if (!b) return set_error(CLB_EINVAL, "batch is NULL");
        bool changed = false;
        for (size_t k = 0; k < b->lat.size(); ++k) {
            const int a = axis ? axis[k] : b->lat[k]->axis;
            if (a != 0 && a != 1) return set_error(CLB_EINVAL, "axis[%zu] must be 0 or 1", k);
            if (a != b->lat[k]->axis) {
                b->lat[k]->axis = a;
                changed = true;
            }
        }
        if (changed) b->E.mark_dirty();
        CLB_TRY(b->E.diagnostics(1));
        clb_status st = CLB_OK;
        for (size_t k = 0; k < b->lat.size(); ++k) {
            const Lattice* L = b->lat[k].get();
            if (nu) nu[k] = L->nu;
            if (er) er[k] = L->er;
            if (L->status == CLB_ENAN) st = set_error(CLB_ENAN, "instance %zu has non-finite fields", k);
        }
        return st;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_batch_run(clb_batch* b, double tol, long max_steps, long interval,
                                    long* steps, double* er, int* status)
{
    TraceRange trace("clb_batch_run");
    try {
        if (!b) return set_error(CLB_EINVAL, "batch is NULL");
        if (interval <= 0 || interval % 2 || max_steps < 0)
            return set_error(CLB_EINVAL, "interval must be even and > 0, max_steps >= 0");
        for (auto& L : b->lat)
            if (L->status != CLB_OK || L->steps >= max_steps) {
                L->active = false;
                b->E.mark_dirty();
            }
        for (;;) {
            bool any = false;
            long n = interval;
            for (auto& L : b->lat)
                if (L->active) {
                    any = true;
                    n = std::min(n, max_steps - L->steps);
                }
            if (!any) break;
            CLB_TRY(b->E.step(n));
            CLB_TRY(b->E.diagnostics(1));
            for (auto& L : b->lat)
                if (L->active && (L->status != CLB_OK || L->er < tol || L->steps >= max_steps)) {
                    L->active = false;
                    b->E.mark_dirty();
                }
        }
        for (size_t k = 0; k < b->lat.size(); ++k) {
            if (steps) steps[k] = b->lat[k]->steps;
            if (er) er[k] = b->lat[k]->er;
            if (status) status[k] = b->lat[k]->status;
        }
        // instances stay retired until re-initialised; re-activate them for further stepping
        for (auto& L : b->lat) L->active = true;
        b->E.mark_dirty();
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_batch_set_tile(clb_batch* b, int tile_x, int tile_y, int nodes_per_thread)
{
    try {
        if (!b) return set_error(CLB_EINVAL, "batch is NULL");
        if (tile_x < 32 || tile_x > 256 || tile_x % 32 || tile_y < 1 || tile_x * tile_y > 256 ||
            (nodes_per_thread != 1 && nodes_per_thread != 2 && nodes_per_thread != 4))
            return set_error(CLB_EINVAL, "tile %d x %d x %d: tile_x in [32, 256] multiple of 32, "
                                         "tile_x * tile_y <= 256, nodes per thread 1, 2 or 4",
                             tile_x, tile_y, nodes_per_thread);
        cudaStreamSynchronize(b->E.stream);
        b->E.tile_x = tile_x;
        b->E.tile_y = tile_y;
        b->E.npt = nodes_per_thread;
        b->E.mark_dirty();
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

// Times candidate tile shapes over the whole batch (10 steps each after 4 warm-up steps) and keeps
// the fastest; the populations of every instance are saved first and restored afterwards.
extern "C" clb_status clb_batch_autotune(clb_batch* b, int* tile_x, int* tile_y, int* nodes_per_thread)
{
    TraceRange trace("clb_batch_autotune");
    try {
        if (!b) return set_error(CLB_EINVAL, "batch is NULL");
        Ensemble& E = b->E;
        CLB_TRY(E.rebuild());
        size_t total = 0;
        for (auto& L : b->lat) total += align256(buffer_bytes(L->nx, L->ny, L->p.storage));
        char* save = nullptr;
        CLB_CUDA(cudaMallocAsync((void**)&save, total, E.stream));
        size_t off = 0;
        for (auto& L : b->lat) {
            const size_t bb = buffer_bytes(L->nx, L->ny, L->p.storage);
            CLB_CUDA(cudaMemcpyAsync(save + off, L->buf[E.parity], bb, cudaMemcpyDeviceToDevice, E.stream));
            off += align256(bb);
        }
        std::vector<long> steps0;
        for (auto& L : b->lat) steps0.push_back(L->steps);
        const int shapes[][3] = {{64, 1, 1}, {128, 1, 1}, {256, 1, 1}, {64, 1, 2}, {128, 1, 2}, {64, 2, 2},
                                 {64, 1, 4}, {128, 1, 4}, {32, 4, 2}, {32, 2, 4}};
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        int bt[3] = {E.tile_x, E.tile_y, E.npt};
        clb_status st = CLB_OK;
        for (auto& sh : shapes) {
            E.tile_x = sh[0];
            E.tile_y = sh[1];
            E.npt = sh[2];
            E.mark_dirty();
            st = E.rebuild();
            for (int k = 0; k < 4 && st == CLB_OK; ++k) st = E.launch_step(E.stream, (E.parity + k) & 1);
            cudaEventRecord(e0, E.stream);
            for (int k = 0; k < 10 && st == CLB_OK; ++k) st = E.launch_step(E.stream, (E.parity + k) & 1);
            cudaEventRecord(e1, E.stream);
            if (st != CLB_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                bt[0] = sh[0];
                bt[1] = sh[1];
                bt[2] = sh[2];
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        off = 0;
        cudaError_t e = cudaSuccess;
        for (auto& L : b->lat) {
            const size_t bb = buffer_bytes(L->nx, L->ny, L->p.storage);
            if (e == cudaSuccess) e = cudaMemcpyAsync(L->buf[E.parity], save + off, bb, cudaMemcpyDeviceToDevice, E.stream);
            off += align256(bb);
        }
        cudaFreeAsync(save, E.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(E.stream);
        for (size_t k = 0; k < b->lat.size(); ++k) b->lat[k]->steps = steps0[k];
        E.tile_x = bt[0];
        E.tile_y = bt[1];
        E.npt = bt[2];
        E.mark_dirty();
        if (st != CLB_OK) return st;
        if (e != cudaSuccess) return set_error(CLB_ECUDA, "batch autotune restore: %s", cudaGetErrorString(e));
        if (tile_x) *tile_x = bt[0];
        if (tile_y) *tile_y = bt[1];
        if (nodes_per_thread) *nodes_per_thread = bt[2];
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_batch_get_launch(clb_batch* b, int* tile_x, int* tile_y, int* nodes_per_thread,
                                           int* groups, long* blocks)
{
    try {
        if (!b) return set_error(CLB_EINVAL, "batch is NULL");
        CLB_TRY(b->E.rebuild());
        if (tile_x) *tile_x = b->E.tile_x;
        if (tile_y) *tile_y = b->E.tile_y;
        if (nodes_per_thread) *nodes_per_thread = b->E.npt;
        if (groups) *groups = b->E.groups;
        if (blocks) *blocks = b->E.ntiles;
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

// ------------------------------------------------------------------------------------ serving

namespace {
struct Request {
    long id;
    std::unique_ptr<Lattice> L;
    std::vector<double> init;  // 4 * N host copy, released at admission
    long cap;
    double tol;
    int done = 0;
    std::vector<double> result;  // 4 * N after retirement
};
}  // namespace

struct clb_server {
    Ensemble E;
    size_t budget = 0, used = 0;
    int max_slots = 0;
    long next_id = 1;
    std::deque<Request*> queue;
    std::map<long, std::unique_ptr<Request>> all;
    std::vector<Request*> running;
    double* stage = nullptr;
    size_t stage_nodes = 0;
};

extern "C" clb_status clb_serve_open(size_t hbm_budget_bytes, int max_slots, int storage, void* stream,
                                     clb_server** out)
{
    try {
        if (!out) return set_error(CLB_EINVAL, "out is NULL");
        *out = nullptr;
        if (max_slots <= 0 || hbm_budget_bytes == 0) return set_error(CLB_EINVAL, "need max_slots > 0 and a budget");
        if (storage < CLB_F64 || storage > CLB_F16DEV) return set_error(CLB_EINVAL, "bad storage");
        auto s = std::make_unique<clb_server>();
        s->budget = hbm_budget_bytes;
        s->max_slots = max_slots;
        CLB_TRY(s->E.init(storage, (cudaStream_t)stream));
        *out = s.release();
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" void clb_serve_close(clb_server* s)
{
    if (!s) return;
    cudaStreamSynchronize(s->E.stream);
    for (Request* r : s->running) cudaFree(r->L->mem);
    if (s->stage) cudaFree(s->stage);
    delete s;
}

extern "C" clb_status clb_serve_submit(clb_server* s, int nx, int ny, const clb_params* p, const double* rho,
                                       const double* ux, const double* uy, const double* T, int nu_axis,
                                       long step_cap, double tol, long* req_id)
{
    TraceRange trace("clb_serve_submit");
    try {
        if (!s) return set_error(CLB_EINVAL, "server is NULL");
        CLB_TRY(validate(nx, ny, p));
        if (p->storage != s->E.storage) return set_error(CLB_EINVAL, "request storage differs from the server's");
        if (nu_axis != 0 && nu_axis != 1) return set_error(CLB_EINVAL, "nu_axis must be 0 or 1");
        if (step_cap < 0) return set_error(CLB_EINVAL, "step_cap < 0");
        const size_t need = lattice_bytes(nx, ny, p->storage);
        if (need > s->budget) return set_error(CLB_ENOMEM, "request needs %zu bytes > budget %zu", need, s->budget);
        auto r = std::make_unique<Request>();
        r->id = s->next_id++;
        r->L = std::make_unique<Lattice>();
        r->L->nx = nx;
        r->L->ny = ny;
        r->L->p = *p;
        r->L->axis = nu_axis;
        r->L->bytes = need;
        r->cap = step_cap;
        r->tol = tol;
        const size_t N = (size_t)nx * ny;
        r->init.assign(4 * N, 0.0);
        const double* src[4] = {rho, ux, uy, T};
        const double dflt[4] = {1.0, 0.0, 0.0, p->T0};
        for (int k = 0; k < 4; ++k) {
            if (src[k]) std::memcpy(r->init.data() + k * N, src[k], N * sizeof(double));
            else std::fill(r->init.begin() + k * N, r->init.begin() + (k + 1) * N, dflt[k]);
        }
        if (req_id) *req_id = r->id;
        s->queue.push_back(r.get());
        s->all[r->id] = std::move(r);
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_serve_progress(clb_server* s, long chunk, int* active, int* queued)
{
    TraceRange trace("clb_serve_progress");
    try {
        if (!s) return set_error(CLB_EINVAL, "server is NULL");
        if (chunk <= 0 || chunk % 2) return set_error(CLB_EINVAL, "chunk must be even and > 0");
        // admission: first fit over the queue in arrival order
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Request* r = *it;
            if ((int)s->running.size() >= s->max_slots) break;
            if (s->used + r->L->bytes > s->budget) {
                ++it;
                continue;
            }
            char* mem = nullptr;
            cudaError_t e = cudaMalloc((void**)&mem, r->L->bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                break;  // device memory is short of the budget; retry next round
            }
            r->L->mem = mem;
            carve(*r->L, mem);
            const size_t N = (size_t)r->L->nx * r->L->ny;
            if (s->stage_nodes < N) {
                cudaStreamSynchronize(s->E.stream);
                cudaFree(s->stage);
                s->stage = nullptr;
                CLB_CUDA(cudaMalloc((void**)&s->stage, 4 * N * sizeof(double)));
                s->stage_nodes = N;
            }
            const double* h = r->init.data();
            CLB_TRY(init_from_host(s->E, r->L.get(), s->stage, h, h + N, h + 2 * N, h + 3 * N));
            std::vector<double>().swap(r->init);
            s->used += r->L->bytes;
            s->running.push_back(r);
            s->E.members.push_back(r->L.get());
            s->E.mark_dirty();
            it = s->queue.erase(it);
        }
        if (!s->running.empty()) {
            CLB_TRY(s->E.step(chunk));
            CLB_TRY(s->E.diagnostics(1));
            std::vector<Request*> keep;
            for (Request* r : s->running) {
                Lattice* L = r->L.get();
                if (L->status != CLB_OK || L->er < r->tol || L->steps >= r->cap) {
                    const size_t N = (size_t)L->nx * L->ny;
                    r->result.assign(4 * N, 0.0);
                    double* dev = nullptr;
                    if (s->stage_nodes < N) return set_error(CLB_ECUDA, "staging buffer too small");
                    dev = s->stage;
                    CLB_TRY(s->E.fields(L, dev, dev + N, dev + 2 * N, dev + 3 * N));
                    CLB_CUDA(cudaMemcpyAsync(r->result.data(), dev, 4 * N * sizeof(double), cudaMemcpyDeviceToHost, s->E.stream));
                    CLB_CUDA(cudaStreamSynchronize(s->E.stream));
                    cudaFree(L->mem);
                    L->mem = nullptr;
                    s->used -= L->bytes;
                    r->done = 1;
                    s->E.members.erase(std::find(s->E.members.begin(), s->E.members.end(), L));
                    s->E.mark_dirty();
                } else {
                    keep.push_back(r);
                }
            }
            s->running.swap(keep);
        }
        if (active) *active = (int)s->running.size();
        if (queued) *queued = (int)s->queue.size();
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_serve_cancel(clb_server* s, long req_id)
{
    try {
        if (!s) return set_error(CLB_EINVAL, "server is NULL");
        auto it = s->all.find(req_id);
        if (it == s->all.end()) return set_error(CLB_EINVAL, "unknown request %ld", req_id);
        Request* r = it->second.get();
        auto q = std::find(s->queue.begin(), s->queue.end(), r);
        if (q != s->queue.end()) s->queue.erase(q);
        auto run = std::find(s->running.begin(), s->running.end(), r);
        if (run != s->running.end()) {
            // no kernel of this server is in flight between calls; release the slot and its memory
            CLB_CUDA(cudaStreamSynchronize(s->E.stream));
            Lattice* L = r->L.get();
            s->E.members.erase(std::find(s->E.members.begin(), s->E.members.end(), L));
            s->E.mark_dirty();
            cudaFree(L->mem);
            L->mem = nullptr;
            s->used -= L->bytes;
            s->running.erase(run);
        }
        s->all.erase(it);
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_serve_poll(clb_server* s, long req_id, int* done, double* nu, long* steps, double* er)
{
    try {
        if (!s) return set_error(CLB_EINVAL, "server is NULL");
        auto it = s->all.find(req_id);
        if (it == s->all.end()) return set_error(CLB_EINVAL, "unknown request %ld", req_id);
        const Request* r = it->second.get();
        if (done) *done = r->done;
        if (nu) *nu = r->L->nu;
        if (steps) *steps = r->L->steps;
        if (er) *er = r->L->er;
        return r->L->status == CLB_ENAN ? set_error(CLB_ENAN, "request %ld blew up", req_id) : CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}

extern "C" clb_status clb_serve_fetch(clb_server* s, long req_id, double* rho, double* ux, double* uy, double* T)
{
    try {
        if (!s) return set_error(CLB_EINVAL, "server is NULL");
        auto it = s->all.find(req_id);
        if (it == s->all.end()) return set_error(CLB_EINVAL, "unknown request %ld", req_id);
        Request* r = it->second.get();
        if (!r->done) return set_error(CLB_EBUSY, "request %ld is still running", req_id);
        const size_t N = (size_t)r->L->nx * r->L->ny;
        double* out[4] = {rho, ux, uy, T};
        for (int k = 0; k < 4; ++k)
            if (out[k]) std::memcpy(out[k], r->result.data() + k * N, N * sizeof(double));
        s->all.erase(it);
        return CLB_OK;
    } catch (const std::bad_alloc&) {
        return host_alloc_failed();
    }
}
