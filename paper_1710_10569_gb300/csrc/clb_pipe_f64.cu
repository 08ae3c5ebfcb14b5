// clb_pipe_f64.cu -- the staged-rows step kernel's launches for the f64 storage form
// (templates in clb_pipe.cuh).
#include "clb_pipe.cuh"

namespace clb {

template <>
cudaError_t enqueue_pipe_form<ST_F64>(const LatParams<typename Storage<ST_F64>::A>& P, int device, int nx, int ny,
                                    const void* a, void* b, cudaStream_t s, int V, int S, int R)
{
    return pipe::enqueue_pipe_v<ST_F64>(P, device, nx, ny, a, b, s, V, S, R);
}

cudaError_t enqueue_pipe_any(int storage, const LatParams<double>& Pd, const LatParams<float>& Pf, int device,
                             int nx, int ny, const void* a, void* b, cudaStream_t s, int V, int S, int R)
{
    switch (storage) {
    case CLB_F64: return enqueue_pipe_form<ST_F64>(Pd, device, nx, ny, a, b, s, V, S, R);
    case CLB_F32: return enqueue_pipe_form<ST_F32>(Pf, device, nx, ny, a, b, s, V, S, R);
    default: return enqueue_pipe_form<ST_F16DEV>(Pf, device, nx, ny, a, b, s, V, S, R);
    }
}

}  // namespace clb
