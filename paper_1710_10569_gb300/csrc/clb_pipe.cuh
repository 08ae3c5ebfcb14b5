// clb_pipe.cuh -- launch templates of the staged-rows step kernel (k_step_pipe in
// clb_kernels.cuh). Each storage form instantiates them in a translation unit of its own
// (clb_pipe_f64.cu, clb_pipe_f32.cu, clb_pipe_f16.cu), so that the 18 heavy instantiations (3
// storage forms x 2 node counts x 3 stage depths) compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "clb_kernels.cuh"

namespace clb {
namespace pipe {


template <int ST, int V, int S>
cudaError_t enqueue_pipe(const LatParams<typename Storage<ST>::A>& P, int device, int nx, int ny, const void* a,
                         void* b, cudaStream_t s, int R)
{
    using E = typename Storage<ST>::T;
    constexpr size_t smem = pipe_smem_bytes<ST, V, S>();
    static bool attr_set[64] = {false};  // per instantiation and device
    const int dev = device >= 0 && device < 64 ? device : 0;
    if (!attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(k_step_pipe<ST, V, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    const int cols = kPipeWarps * 32 * V;
    const dim3 grid((nx + cols - 1) / cols, (ny + R - 1) / R);
    k_step_pipe<ST, V, S><<<grid, kPipeWarps * 32, smem, s>>>((const E*)a, (E*)b, P, R);
    return cudaSuccess;
}

template <int ST, int V>
cudaError_t enqueue_pipe_s(const LatParams<typename Storage<ST>::A>& P, int device, int nx, int ny, const void* a,
                           void* b, cudaStream_t s, int S, int R)
{
    if (S == 2) return enqueue_pipe<ST, V, 2>(P, device, nx, ny, a, b, s, R);
    if (S == 3) return enqueue_pipe<ST, V, 3>(P, device, nx, ny, a, b, s, R);
    return enqueue_pipe<ST, V, 4>(P, device, nx, ny, a, b, s, R);
}

template <int ST>
cudaError_t enqueue_pipe_v(const LatParams<typename Storage<ST>::A>& P, int device, int nx, int ny, const void* a,
                           void* b, cudaStream_t s, int V, int S, int R)
{
    if (V == 4) return enqueue_pipe_s<ST, 4>(P, device, nx, ny, a, b, s, S, R);
    return enqueue_pipe_s<ST, 2>(P, device, nx, ny, a, b, s, S, R);
}


}  // namespace pipe

// One step of the staged-rows kernel for storage form ST (defined in clb_pipe_<form>.cu).
template <int ST>
cudaError_t enqueue_pipe_form(const LatParams<typename Storage<ST>::A>& P, int device, int nx, int ny,
                              const void* a, void* b, cudaStream_t s, int V, int S, int R);

}  // namespace clb
