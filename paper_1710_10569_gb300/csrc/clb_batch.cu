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

#include "clb_diag.cuh"

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

// L2 prefetch of the populations that the V nodes x0 .. x0 + V - 1 of row y pull (the vector
// path's 14 loads, without the edge values): a warp that steps several rows one after another
// issues it for its next row before it steps the current one, so that the next row's loads find
// their lines in L2 instead of waiting on DRAM. It holds no registers beyond the addresses.
template <int ST, int V>
__device__ __forceinline__ void prefetch_pulls(const typename Storage<ST>::T* __restrict__ src,
                                               const LatParams<typename Storage<ST>::A>& P, int x0, int y)
{
    using E = typename Storage<ST>::T;
    const int ym = y > 0 ? y - 1 : P.ny - 1;
    const int yp = y < P.ny - 1 ? y + 1 : 0;
    const long long cx = chunk_off(x0);
    const E* sc = src + (long long)y * P.crow + cx;
    const E* sm = src + (long long)ym * P.crow + cx;
    const E* sp = src + (long long)yp * P.crow + cx;
    const int ROWSEL[NPOP] = {0, 0, 1, 0, 2, 1, 1, 2, 2, 0, 0, 1, 0, 2};
#pragma unroll
    for (int i = 0; i < NPOP; ++i) {
        const E* a = (ROWSEL[i] == 0 ? sc : ROWSEL[i] == 1 ? sm : sp) + i * kRowChunk;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// One time step of every lattice: block b covers tile (b - tile_begin) of lattice owner[b]; a
// tile is (blockDim.x * V) x (blockDim.y * groups) nodes, V consecutive nodes per thread (the
// same per-warp update as the single-lattice step), each warp stepping `groups` rows; warps
// clear of every wall take the copy of the vector body without the wall terms.
// Register cap: the FP32 two-nodes-per-thread form (the default tile) is held at 96 registers so
// that five 128-thread blocks stay resident per SM; the other forms take what they need (blocks
// have at most 256 threads).
// HI1: every lattice of the launch has s_3 = s_4 = lambda2 = 1 (the form of collide that does not
// form the moments those rates discard).
template <int ST, int V, bool HI1>
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
    // Columns [xs, xe) of the tile that no warp covers with the vector path: they are updated node
    // by node, one (row, column) pair per thread of the block, so that the lanes of a warp work on
    // different rows at once instead of one lane per row.
    int xs = 0, xe = 0;
    // The last tile of a row that would run past the row's end is moved left to end on the last
    // multiple of V below nx (tail), so that its warps take the vector path (walls included); the
    // nodes it shares with the tile before it are computed alike and stored by that tile only, and
    // the nx % V nodes from tail on go node by node. The moved start stays a multiple of V, so the
    // vector loads stay aligned. A tile that would store no vector node (xt == tail), or a row
    // shorter than a tile, goes node by node as a whole.
    const int tail = M.P.nx - M.P.nx % V;
    bool vector = xt + span <= M.P.nx;
    if (!vector) {
        if (xt < tail && tail >= span) {
            keep = xt;
            xt = tail - span;
            vector = true;
            xs = tail;
        } else {
            xs = xt;
        }
        xe = M.P.nx;
    }
    const E* src = (const E*)M.buf[parity];
    E* dst = (E*)M.buf[parity ^ 1];
    // The tile's rows: `groups` groups of blockDim.y rows, one group after another, so that the
    // descriptor fetched above serves several rows per warp.
    const int rows = blockDim.y * groups;
    const int y0 = ty * rows;
    const int y_end = min(M.P.ny, y0 + rows);
    if (vector) {
        const int x0 = xt + threadIdx.x * V;
        for (int y = y0 + threadIdx.y; y < y_end; y += blockDim.y) {
            // the warp's next row to L2 first (one row ahead: 53.7 -> 55.7 GLUPS on 256 uneven
            // cavities; two rows ahead 53.4)
            if (y + (int)blockDim.y < y_end) prefetch_pulls<ST, V>(src, M.P, x0, y + blockDim.y);
            step_warp_nodes<ST, V, true, HI1>(src, dst, M.P, x0, y, lane, keep);
        }
    }
    const int nrow = y_end - y0;
    const int nodes = nrow * (xe - xs);
    for (int j = threadIdx.y * blockDim.x + threadIdx.x; j < nodes; j += blockDim.x * blockDim.y) {
        const int y = y0 + j % nrow, x = xs + j / nrow;
        A f[9], g[5];
        gather(src, M.P, x, y, f, g);
        collide_any<Storage<ST>::DEV, HI1>(M.P, f, g, row_base(M.P, y));
        store_node(dst, M.P, x, y, f, g);
    }
}

// Blocks of k_step_batched<ST, V, HI1> resident on the whole device at once.
template <int ST, int V, bool HI1>
long resident_blocks_of(int threads)
{
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_batched<ST, V, HI1>, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    return (long)std::max(1, sms) * std::max(1, per_sm);
}

template <int ST, bool HI1>
long resident_blocks_npt(int npt, int threads)
{
    return npt == 4 ? resident_blocks_of<ST, 4, HI1>(threads)
                    : npt == 2 ? resident_blocks_of<ST, 2, HI1>(threads) : resident_blocks_of<ST, 1, HI1>(threads);
}
template <int ST>
long resident_blocks_npt(int npt, int threads, bool hi1)
{
    return hi1 ? resident_blocks_npt<ST, true>(npt, threads) : resident_blocks_npt<ST, false>(npt, threads);
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
    reduce_row((const E*)M.buf[parity], M.P, y, M.axis, (A*)M.snap, update, M.partial + (long long)y * RS_N);
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
Member<A> make_member(const Lattice& L, int tile_x, int npt, int tile_begin, int row_begin, double* diag)
{
    Member<A> m;
    std::memset(&m, 0, sizeof(m));
    m.P = make_lat_params<A>(L.nx, L.ny, L.p);
    m.buf[0] = L.buf[0];
    m.buf[1] = L.buf[1];
    m.snap = L.snap;
    m.partial = L.partial;
    m.diag = diag;
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

// Entries of the tile-owner and row-owner tables a lattice adds to the batched launch at most:
// tiles of one group of rows (more groups per block only merge tiles).
long tiles_of(int nx, int ny, int tile_x, int tile_y, int npt)
{
    return (long)((nx + tile_x * npt - 1) / (tile_x * npt)) * ((ny + tile_y - 1) / tile_y);
}

constexpr int kDiagStride = 16;  // doubles of diagnostics output per member

// The set of resident lattices and the device tables of the batched launch. Every table is
// reserved once (reserve) with a fixed capacity, together with pinned host mirrors; a change of
// membership rewrites the mirrors and copies them to the device in stream order, with no device
// allocation and no synchronisation of the stream.
class Ensemble {
public:
    int storage = CLB_F32;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int tile_x = 128, tile_y = 1, npt = 1;
    int groups = 1;  // row groups per block (kBlockNodes): a tile is (tile_x * npt) x (tile_y * groups) nodes
    bool hi1 = false;  // every active lattice has s_3 = s_4 = 1 (set by rebuild)
    int parity = 0;  // every resident lattice holds its current data in buf[parity]
    std::vector<Lattice*> members;  // launch order

    ~Ensemble()
    {
        drop_graphs();
        cudaFree(d_tables);
        if (h_tables) cudaFreeHost(h_tables);
        if (copied) cudaEventDestroy(copied);
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
        CLB_CUDA(cudaEventCreateWithFlags(&copied, cudaEventDisableTiming));
        return CLB_OK;
    }

    // One device allocation (and one pinned host mirror) for the member descriptors, the
    // diagnostics outputs and the tile- and row-owner tables, at the given capacities.
    clb_status reserve(size_t max_members, size_t max_tiles, size_t max_rows)
    {
        cap_members = std::max<size_t>(1, max_members);
        cap_tiles = std::max<size_t>(1, max_tiles);
        cap_rows = std::max<size_t>(1, max_rows);
        const size_t msz = std::max(sizeof(Member<double>), sizeof(Member<float>));
        off_members = 0;
        off_diag = align256(cap_members * msz);
        off_owner = off_diag + align256(cap_members * kDiagStride * sizeof(double));
        off_rows = off_owner + align256(cap_tiles * sizeof(int));
        table_bytes = off_rows + align256(cap_rows * sizeof(int));
        cudaError_t e = cudaMalloc(&d_tables, table_bytes);
        if (e != cudaSuccess)
            return set_error(e == cudaErrorMemoryAllocation ? CLB_ENOMEM : CLB_ECUDA, "launch tables (%zu bytes): %s",
                             table_bytes, cudaGetErrorString(e));
        e = cudaMallocHost(&h_tables, table_bytes);
        if (e != cudaSuccess) return set_error(CLB_ENOMEM, "pinned launch tables (%zu bytes): %s", table_bytes, cudaGetErrorString(e));
        return CLB_OK;
    }

    size_t capacity_tiles() const { return cap_tiles; }
    size_t capacity_rows() const { return cap_rows; }

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
        const long resident = storage == CLB_F64 ? resident_blocks_npt<ST_F64>(npt, threads, hi1)
                              : storage == CLB_F32 ? resident_blocks_npt<ST_F32>(npt, threads, hi1)
                                                   : resident_blocks_npt<ST_F16DEV>(npt, threads, hi1);
        groups = 1;
        for (int g = 2; g * threads * npt <= kBlockNodes && tiles_with(g) >= kMinWaves * resident; g *= 2) groups = g;
    }

    // Rebuild the tile and row tables for the active members (no allocation, no stream sync).
    clb_status rebuild()
    {
        if (!dirty) return CLB_OK;
        drop_graphs();
        active.clear();
        hi1 = true;
        for (Lattice* L : members)
            if (L->active) {
                active.push_back(L);
                hi1 = hi1 && L->p.s_3 == 1.0 && L->p.s_4 == 1.0 && L->p.lambda2 == 1.0;
            }
        choose_groups();
        const long tiles = tiles_with(groups);
        long rows = 0;
        for (const Lattice* L : active) rows += L->ny;
        if (active.size() > cap_members || (size_t)tiles > cap_tiles || (size_t)rows > cap_rows)
            return set_error(CLB_ENOMEM, "batched launch tables: %zu members, %ld tiles, %ld rows exceed the reserved "
                                         "%zu, %zu, %zu", active.size(), tiles, rows, cap_members, cap_tiles, cap_rows);
        // the mirrors of the previous rebuild may still be in flight to the device
        CLB_CUDA(cudaEventSynchronize(copied));
        const size_t msz = storage == CLB_F64 ? sizeof(Member<double>) : sizeof(Member<float>);
        char* hm = (char*)h_tables + off_members;
        int* owner = (int*)((char*)h_tables + off_owner);
        int* row_owner = (int*)((char*)h_tables + off_rows);
        double* ddiag = (double*)((char*)d_tables + off_diag);
        int t = 0, r = 0;
        for (size_t k = 0; k < active.size(); ++k) {
            const Lattice& L = *active[k];
            const int tx = (L.nx + tile_x * npt - 1) / (tile_x * npt), ty = (L.ny + tile_y * groups - 1) / (tile_y * groups);
            if (storage == CLB_F64) {
                Member<double> m = make_member<double>(L, tile_x, npt, t, r, ddiag + kDiagStride * k);
                std::memcpy(hm + k * msz, &m, msz);
            } else {
                Member<float> m = make_member<float>(L, tile_x, npt, t, r, ddiag + kDiagStride * k);
                std::memcpy(hm + k * msz, &m, msz);
            }
            std::fill(owner + t, owner + t + tx * ty, int(k));
            std::fill(row_owner + r, row_owner + r + L.ny, int(k));
            t += tx * ty;
            r += L.ny;
        }
        ntiles = t;
        nrows = r;
        if (!active.empty()) {
            CLB_CUDA(cudaMemcpyAsync((char*)d_tables + off_members, hm, active.size() * msz, cudaMemcpyHostToDevice, stream));
            CLB_CUDA(cudaMemcpyAsync((char*)d_tables + off_owner, owner, (size_t)t * sizeof(int), cudaMemcpyHostToDevice, stream));
            CLB_CUDA(cudaMemcpyAsync((char*)d_tables + off_rows, row_owner, (size_t)r * sizeof(int), cudaMemcpyHostToDevice, stream));
            CLB_CUDA(cudaEventRecord(copied, stream));
        }
        dirty = false;
        return CLB_OK;
    }

    template <int ST>
    void enqueue(cudaStream_t s, int par)
    {
        using A = typename Storage<ST>::A;
        const dim3 block(tile_x, tile_y);
        const Member<A>* m = (const Member<A>*)((char*)d_tables + off_members);
        const int* owner = (const int*)((char*)d_tables + off_owner);
        if (hi1) {
            if (npt == 4) k_step_batched<ST, 4, true><<<ntiles, block, 0, s>>>(m, owner, par, groups);
            else if (npt == 2) k_step_batched<ST, 2, true><<<ntiles, block, 0, s>>>(m, owner, par, groups);
            else k_step_batched<ST, 1, true><<<ntiles, block, 0, s>>>(m, owner, par, groups);
        } else {
            if (npt == 4) k_step_batched<ST, 4, false><<<ntiles, block, 0, s>>>(m, owner, par, groups);
            else if (npt == 2) k_step_batched<ST, 2, false><<<ntiles, block, 0, s>>>(m, owner, par, groups);
            else k_step_batched<ST, 1, false><<<ntiles, block, 0, s>>>(m, owner, par, groups);
        }
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
        // both parities are captured on the first chunk after a membership change
        for (int par = 0; n >= kChunk && par < 2; ++par) {
            if (graph[par]) continue;
            CLB_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            clb_status st = CLB_OK;
            for (int k = 0; k < kChunk && st == CLB_OK; ++k) st = launch_step(cap, par ^ (k & 1));
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(cap, &g);
            if (st != CLB_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return set_error(CLB_ECUDA, "capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&graph[par], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return set_error(CLB_ECUDA, "instantiate: %s", cudaGetErrorString(e));
        }
        while (n >= kChunk) {
            CLB_CUDA(cudaGraphLaunch(graph[parity], stream));
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
    // The outputs of all members come back in one copy.
    clb_status diagnostics(int update)
    {
        CLB_TRY(rebuild());
        if (active.empty()) return CLB_OK;
        const int* row_owner = (const int*)((char*)d_tables + off_rows);
        const void* m = (char*)d_tables + off_members;
        switch (storage) {
        case CLB_F64: k_reduce_rows_batched<ST_F64><<<nrows, kReduceThreads, 0, stream>>>((const Member<double>*)m, row_owner, parity, update); break;
        case CLB_F32: k_reduce_rows_batched<ST_F32><<<nrows, kReduceThreads, 0, stream>>>((const Member<float>*)m, row_owner, parity, update); break;
        default: k_reduce_rows_batched<ST_F16DEV><<<nrows, kReduceThreads, 0, stream>>>((const Member<float>*)m, row_owner, parity, update); break;
        }
        CLB_CUDA(cudaGetLastError());
        if (storage == CLB_F64)
            k_reduce_final_batched<double><<<(int)active.size(), kReduceThreads, 0, stream>>>((const Member<double>*)m);
        else
            k_reduce_final_batched<float><<<(int)active.size(), kReduceThreads, 0, stream>>>((const Member<float>*)m);
        CLB_CUDA(cudaGetLastError());
        double* hd = (double*)((char*)h_tables + off_diag);
        CLB_CUDA(cudaMemcpyAsync(hd, (char*)d_tables + off_diag, active.size() * kDiagStride * sizeof(double),
                                 cudaMemcpyDeviceToHost, stream));
        CLB_CUDA(cudaStreamSynchronize(stream));
        for (size_t k = 0; k < active.size(); ++k) {
            Lattice* L = active[k];
            const double* d = hd + kDiagStride * k;
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
            k_snap<ST_F64><<<grid, block, 0, stream>>>((const double*)d, P, L->snap);
        } else {
            const LatParams<float> P = make_lat_params<float>(L->nx, L->ny, L->p);
            if (storage == CLB_F32) {
                k_init<ST_F32><<<grid, block, 0, stream>>>((float*)d, P, rho, ux, uy, T, L->p.rho0);
                k_snap<ST_F32><<<grid, block, 0, stream>>>((const float*)d, P, (float*)L->snap);
            } else {
                k_init<ST_F16DEV><<<grid, block, 0, stream>>>((__half*)d, P, rho, ux, uy, T, L->p.rho0);
                k_snap<ST_F16DEV><<<grid, block, 0, stream>>>((const __half*)d, P, (float*)L->snap);
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
    bool dirty = true;
    std::vector<Lattice*> active;
    void* d_tables = nullptr;  // members | diagnostics outputs | tile owners | row owners
    void* h_tables = nullptr;  // pinned mirror of the same layout
    size_t off_members = 0, off_diag = 0, off_owner = 0, off_rows = 0, table_bytes = 0;
    size_t cap_members = 0, cap_tiles = 0, cap_rows = 0;
    cudaEvent_t copied = nullptr;  // recorded after the last copy of the mirrors
    cudaGraphExec_t graph[2] = {nullptr, nullptr};

    void drop_graphs()
    {
        for (auto& g : graph)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }
};

// Device addresses where the four host fields of a member are staged for its initialisation, and
// where its fields are written for the host at retirement: rho, u_x, u_y in the population buffer
// that the next step would write (at least 28 bytes per node in every storage form, 24 needed)
// and T in the T slot of the residual snapshot, which k_fields rewrites only after k_init has read
// it (stream order). No extra device memory is needed.
void own_stage(const Lattice* L, int parity, double* dev[4])
{
    const size_t N = (size_t)L->nx * L->ny;
    double* spare = (double*)L->buf[parity ^ 1];
    dev[0] = spare;
    dev[1] = spare + N;
    dev[2] = spare + 2 * N;
    dev[3] = L->snap + 2 * N;
}

// Copy host fields (any may be NULL) into the member's own staging addresses and initialise it.
// With `wait`, returns after the copies are done (the caller may then reuse its host arrays even
// when they are pinned); otherwise the copies are only ordered on the stream.
clb_status init_from_host(Ensemble& E, Lattice* L, const double* rho, const double* ux, const double* uy,
                          const double* T, bool wait)
{
    const size_t N = (size_t)L->nx * L->ny;
    const double* src[4] = {rho, ux, uy, T};
    double* stage[4];
    own_stage(L, E.parity, stage);
    const double* dev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k)
        if (src[k]) {
            CLB_CUDA(cudaMemcpyAsync(stage[k], src[k], N * sizeof(double), cudaMemcpyHostToDevice, E.stream));
            dev[k] = stage[k];
        }
    CLB_TRY(E.init_member(L, dev[0], dev[1], dev[2], dev[3]));
    if (wait) CLB_CUDA(cudaStreamSynchronize(E.stream));
    return CLB_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------ batches

struct clb_batch {
    Ensemble E;
    std::vector<std::unique_ptr<Lattice>> lat;
    char* mem = nullptr;
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
        size_t total = 0, max_tiles = 0, rows = 0;
        for (int k = 0; k < n; ++k) {
            CLB_TRY(validate(nx[k], ny[k], &p[k]));
            if (p[k].storage != storage) return set_error(CLB_EINVAL, "instance %d: all instances need the same storage", k);
            total += lattice_bytes(nx[k], ny[k], storage);
            max_tiles += tiles_of(nx[k], ny[k], 32, 1, 1);  // the smallest tile clb_batch_set_tile accepts
            rows += ny[k];
        }
        auto b = std::make_unique<clb_batch>();
        cudaGetDevice(&b->device);
        CLB_TRY(b->E.init(storage, (cudaStream_t)stream));
        CLB_TRY(b->E.reserve(n, max_tiles, rows));
        CLB_CUDA(cudaMalloc((void**)&b->mem, total));
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
        return init_from_host(b->E, L, rho, ux, uy, T, true);
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
        // the fields go through the spare population buffer only (the snapshot stays intact)
        double* spare = (double*)L->buf[b->E.parity ^ 1];
        double* dev[4];
        for (int i = 0; i < 4; ++i) dev[i] = nullptr;
        for (int i = 0, slot = 0; i < 4; ++i)
            if (host[i]) dev[i] = spare + (slot++ % 3) * N;
        // at most three fields fit the spare buffer at once: fetch in two rounds when all four are asked
        const int n_asked = (rho != nullptr) + (ux != nullptr) + (uy != nullptr) + (T != nullptr);
        if (n_asked == 4) {
            CLB_TRY(b->E.fields(L, dev[0], dev[1], dev[2], nullptr));
            for (int i = 0; i < 3; ++i)
                CLB_CUDA(cudaMemcpyAsync(host[i], dev[i], N * sizeof(double), cudaMemcpyDeviceToHost, b->E.stream));
            CLB_TRY(b->E.fields(L, nullptr, nullptr, nullptr, spare));
            CLB_CUDA(cudaMemcpyAsync(host[3], spare, N * sizeof(double), cudaMemcpyDeviceToHost, b->E.stream));
            CLB_CUDA(cudaStreamSynchronize(b->E.stream));
            return CLB_OK;
        }
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

extern "C" clb_status clb_batch_status(clb_batch* b, int* status, double* er, long* steps, double* nu)
{
    if (!b) return set_error(CLB_EINVAL, "batch is NULL");
    for (size_t k = 0; k < b->lat.size(); ++k) {
        const Lattice* L = b->lat[k].get();
        if (status) status[k] = L->status;
        if (er) er[k] = L->er;
        if (steps) steps[k] = L->steps;
        if (nu) nu[k] = L->nu;
    }
    return CLB_OK;
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
    long tiles = 0;  // entries of the tile-owner table at one group of rows per block
    int done = 0;
    std::vector<double> result;  // 4 * N after retirement
};

// Best-fit sub-allocation of one device reservation in 256-byte blocks; a released block merges
// with its free neighbours. Host bookkeeping only: taking and giving blocks never calls CUDA.
class Pool {
public:
    ~Pool() { cudaFree(base); }

    clb_status open(size_t bytes)
    {
        size = bytes / 256 * 256;
        const cudaError_t e = cudaMalloc((void**)&base, size);
        if (e != cudaSuccess)
            return set_error(e == cudaErrorMemoryAllocation ? CLB_ENOMEM : CLB_ECUDA, "HBM budget of %zu bytes: %s",
                             size, cudaGetErrorString(e));
        free_[0] = size;
        return CLB_OK;
    }

    // The smallest free block that holds `bytes` (rounded up to 256), or NULL.
    char* take(size_t bytes)
    {
        bytes = align256(bytes);
        auto best = free_.end();
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes && (best == free_.end() || it->second < best->second)) best = it;
        if (best == free_.end()) return nullptr;
        const size_t off = best->first, have = best->second;
        free_.erase(best);
        if (have > bytes) free_[off + bytes] = have - bytes;
        used_[off] = bytes;
        return base + off;
    }

    void give(char* p)
    {
        auto u = used_.find((size_t)(p - base));
        if (u == used_.end()) return;
        size_t off = u->first, bytes = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && next->first == off + bytes) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }

private:
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_, used_;  // offset -> bytes
};
}  // namespace

// The server's device memory is reserved once at clb_serve_open: the whole HBM budget as a pool
// that resident lattices are carved from, and the launch tables at fixed capacities. Admission,
// stepping and retirement then allocate nothing on the device.
struct clb_server {
    Ensemble E;
    Pool pool;
    size_t budget = 0, used = 0;
    long tiles_used = 0, rows_used = 0;
    int max_slots = 0;
    long next_id = 1;
    std::deque<Request*> queue;
    std::map<long, std::unique_ptr<Request>> all;
    std::vector<Request*> running;
};

extern "C" clb_status clb_serve_open(size_t hbm_budget_bytes, int max_slots, int storage, void* stream,
                                     clb_server** out)
{
    try {
        if (!out) return set_error(CLB_EINVAL, "out is NULL");
        *out = nullptr;
        if (max_slots <= 0 || hbm_budget_bytes < 256) return set_error(CLB_EINVAL, "need max_slots > 0 and a budget");
        if (storage < CLB_F64 || storage > CLB_F16DEV) return set_error(CLB_EINVAL, "bad storage");
        auto s = std::make_unique<clb_server>();
        s->budget = hbm_budget_bytes;
        s->max_slots = max_slots;
        CLB_TRY(s->E.init(storage, (cudaStream_t)stream));
        // Table capacities: a resident set this large in tiles or rows is far beyond what the
        // budget holds in lattices of ordinary shape; a request that would overflow them waits.
        const size_t tiles_cap = std::max<size_t>(size_t(1) << 20, hbm_budget_bytes / 16384);
        const size_t rows_cap = std::max<size_t>(size_t(1) << 18, hbm_budget_bytes / 65536);
        CLB_TRY(s->E.reserve(max_slots, tiles_cap, rows_cap));
        CLB_TRY(s->pool.open(hbm_budget_bytes));
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
        const long tiles = tiles_of(nx, ny, s->E.tile_x, s->E.tile_y, s->E.npt);
        if ((size_t)tiles > s->E.capacity_tiles() || (size_t)ny > s->E.capacity_rows())
            return set_error(CLB_ENOMEM, "request of %d x %d exceeds the server's launch tables", nx, ny);
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
        r->tiles = tiles;
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

namespace {
// Return a resident request's memory and table entries to the server.
void release(clb_server* s, Request* r)
{
    Lattice* L = r->L.get();
    s->E.members.erase(std::find(s->E.members.begin(), s->E.members.end(), L));
    s->E.mark_dirty();
    s->pool.give(L->mem);
    L->mem = nullptr;
    s->used -= L->bytes;
    s->tiles_used -= r->tiles;
    s->rows_used -= L->ny;
}
}  // namespace

extern "C" clb_status clb_serve_progress(clb_server* s, long chunk, int* active, int* queued)
{
    TraceRange trace("clb_serve_progress");
    try {
        if (!s) return set_error(CLB_EINVAL, "server is NULL");
        if (chunk <= 0 || chunk % 2) return set_error(CLB_EINVAL, "chunk must be even and > 0");
        // admission: first fit over the queue in arrival order, into the pool and the tables
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Request* r = *it;
            if ((int)s->running.size() >= s->max_slots) break;
            if ((size_t)(s->tiles_used + r->tiles) > s->E.capacity_tiles() ||
                (size_t)(s->rows_used + r->L->ny) > s->E.capacity_rows()) {
                ++it;
                continue;
            }
            char* mem = s->pool.take(r->L->bytes);
            if (!mem) {
                ++it;
                continue;
            }
            r->L->mem = mem;
            carve(*r->L, mem);
            const size_t N = (size_t)r->L->nx * r->L->ny;
            // keep the padding of each row's last chunk defined (it is never read)
            CLB_CUDA(cudaMemsetAsync(mem, 0, 2 * buffer_slot_bytes(r->L->nx, r->L->ny, r->L->p.storage), s->E.stream));
            const double* h = r->init.data();
            // pageable source: the copies have left the host array when they return
            CLB_TRY(init_from_host(s->E, r->L.get(), h, h + N, h + 2 * N, h + 3 * N, false));
            std::vector<double>().swap(r->init);
            s->used += r->L->bytes;
            s->tiles_used += r->tiles;
            s->rows_used += r->L->ny;
            s->running.push_back(r);
            s->E.members.push_back(r->L.get());
            s->E.mark_dirty();
            it = s->queue.erase(it);
        }
        if (!s->running.empty()) {
            CLB_TRY(s->E.step(chunk));
            CLB_TRY(s->E.diagnostics(1));
            std::vector<Request*> keep, leaving;
            for (Request* r : s->running) {
                Lattice* L = r->L.get();
                if (L->status != CLB_OK || L->er < r->tol || L->steps >= r->cap) leaving.push_back(r);
                else keep.push_back(r);
            }
            // fields of every retiring request through its own spare regions, one sync for all
            for (Request* r : leaving) {
                Lattice* L = r->L.get();
                const size_t N = (size_t)L->nx * L->ny;
                double* dev[4];
                own_stage(L, s->E.parity, dev);
                r->result.assign(4 * N, 0.0);
                CLB_TRY(s->E.fields(L, dev[0], dev[1], dev[2], dev[3]));
                for (int k = 0; k < 4; ++k)
                    CLB_CUDA(cudaMemcpyAsync(r->result.data() + k * N, dev[k], N * sizeof(double), cudaMemcpyDeviceToHost,
                                             s->E.stream));
            }
            if (!leaving.empty()) CLB_CUDA(cudaStreamSynchronize(s->E.stream));
            for (Request* r : leaving) {
                release(s, r);
                r->done = 1;
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
            // the slot and its memory return to the server at once; work enqueued later on the
            // server's stream runs after everything that used them
            release(s, r);
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
