// clb_noalloc.cu -- the Nusselt number of a population buffer without any device allocation
// (clb_nusselt_noalloc in include/clb.h).
//
// Why it exists. clb_nusselt works through a handle that owns its scratch, and clb_create obtains
// that memory with cudaMalloc or from the caller. Some callers cannot allocate device memory at
// the moment they want a diagnostic: a progress monitor inside a server that has already handed
// its whole HBM budget to resident lattices (a cudaMalloc there can fail, or take memory the
// admission policy has promised elsewhere), or a latency-sensitive loop that must not call
// cudaMalloc/cudaFree because those calls can synchronise the whole device and stall the other
// streams. Such a caller holds only the population buffer (for example the pointer clb_buffers
// returns) and the lattice's parameters. This entry point serves it with scratch that lives in a
// fixed-size array in the library's own device memory, reserved once when the library is loaded
// on a device and held until the process exits.
//
// Scratch: per-row FP64 partial sums (CLB_NOALLOC_MAX_ROWS rows) and the final sums. Every partial
// is written by its row's block before the final block reads it, and the final block writes
// every output, so nothing has to start at zero. All calls in the process share this one array:
// two calls whose kernels overlap on the GPU (different streams, or different host threads) race
// on it and may return each other's numbers; serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "clb_diag.cuh"

using namespace clb;

namespace {

constexpr int kOut = RS_N + 2;  // final sums, then Nu

__device__ __align__(256) double g_noalloc_scratch[CLB_NOALLOC_MAX_ROWS * RS_N + kOut];

// Address of g_noalloc_scratch on each device, looked up once per device (with it current).
std::mutex g_mu;
double* g_addr[64] = {nullptr};

clb_status scratch_address(double** out)
{
    int dev = 0;
    CLB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(CLB_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_error(CLB_ECUDA, "cudaGetSymbolAddress(noalloc scratch): %s", cudaGetErrorString(e));
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return CLB_OK;
}

// Per-row sums of u_axis (T - T0) and of non-finite nodes (one block of kReduceThreads per row,
// threads striding over x), each node's term formed as in the handle-based diagnostics.
template <int ST>
__global__ void __launch_bounds__(kReduceThreads) k_nusselt_rows_noalloc(
    const typename Storage<ST>::T* __restrict__ src, const LatParams<typename Storage<ST>::A> P,
    int axis, double* __restrict__ scratch)
{
    using A = typename Storage<ST>::A;
    const int y = blockIdx.x;
    double v[RS_N] = {0, 0, 0, 0, 0, 0};
    int nbad = 0;
    for (int x = threadIdx.x; x < P.nx; x += kReduceThreads) {
        A f[9], g[5];
        gather(src, P, x, y, f, g);
        const Macro<A> m = macroscopic(P, f, g, row_base(P, y));
        A T;
        const A q = nu_term(P, m, axis, T);  // the same term as the handle-based diagnostics
        v[RS_UT] += double(q * A(wet_weight(P, x, y)));
        nbad += (isfinite(m.ux) && isfinite(m.uy) && isfinite(T) && isfinite(m.rho)) ? 0 : 1;
    }
    v[RS_BAD] = double(nbad);
    block_sum(v, scratch + (long long)y * RS_N);
}

__global__ void __launch_bounds__(kReduceThreads) k_nusselt_final_noalloc(double* __restrict__ scratch,
                                                                          int rows, double nodes,
                                                                          double cells, double H,
                                                                          double dT, double sign,
                                                                          double kappa)
{
    double* out = scratch + CLB_NOALLOC_MAX_ROWS * RS_N;
    reduce_final(scratch, rows, nodes, cells, H, dT, sign, kappa, 0.0, 0.0, out);
}

}  // namespace

extern "C" clb_status clb_nusselt_noalloc(const void* populations, int nx, int ny, const clb_params* p,
                                          int axis, void* stream, double* nu_out)
{
    CLB_TRY(validate(nx, ny, p));
    if (!populations || !nu_out) return set_error(CLB_EINVAL, "populations and nu_out must not be NULL");
    if (axis != 0 && axis != 1) return set_error(CLB_EINVAL, "axis must be 0 or 1");
    if (ny > CLB_NOALLOC_MAX_ROWS)
        return set_error(CLB_EINVAL, "clb_nusselt_noalloc: ny = %d exceeds the fixed scratch of %d rows "
                                     "(use clb_nusselt on a handle instead)", ny, CLB_NOALLOC_MAX_ROWS);
    double* scratch = nullptr;
    CLB_TRY(scratch_address(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    switch (p->storage) {
    case CLB_F64:
        k_nusselt_rows_noalloc<ST_F64><<<ny, kReduceThreads, 0, s>>>((const double*)populations,
                                                                     make_lat_params<double>(nx, ny, *p), axis, scratch);
        break;
    case CLB_F32:
        k_nusselt_rows_noalloc<ST_F32><<<ny, kReduceThreads, 0, s>>>((const float*)populations,
                                                                     make_lat_params<float>(nx, ny, *p), axis, scratch);
        break;
    default:
        k_nusselt_rows_noalloc<ST_F16DEV><<<ny, kReduceThreads, 0, s>>>((const __half*)populations,
                                                                        make_lat_params<float>(nx, ny, *p), axis, scratch);
        break;
    }
    CLB_CUDA(cudaGetLastError());
    const NuGeom g = nu_geom(nx, ny, *p, axis);
    k_nusselt_final_noalloc<<<1, kReduceThreads, 0, s>>>(scratch, ny, double(nx) * ny, g.cells, g.H, g.dT, g.sign, p->kappa);
    CLB_CUDA(cudaGetLastError());
    double out[kOut];
    CLB_CUDA(cudaMemcpyAsync(out, scratch + CLB_NOALLOC_MAX_ROWS * RS_N, sizeof(out), cudaMemcpyDeviceToHost, s));
    CLB_CUDA(cudaStreamSynchronize(s));
    if (out[RS_BAD] > 0) return set_error(CLB_ENAN, "%.0f nodes have non-finite fields", out[RS_BAD]);
    *nu_out = out[RS_N];
    return CLB_OK;
}
