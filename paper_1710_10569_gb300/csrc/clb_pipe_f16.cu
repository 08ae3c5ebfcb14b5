// clb_pipe_f16.cu -- the staged-rows step kernel's launches for the f16 storage form
// (templates in clb_pipe.cuh).
#include "clb_pipe.cuh"

namespace clb {

template <>
cudaError_t enqueue_pipe_form<ST_F16DEV>(const LatParams<typename Storage<ST_F16DEV>::A>& P, int device, int nx, int ny,
                                    const void* a, void* b, cudaStream_t s, int V, int S, int R)
{
    return pipe::enqueue_pipe_v<ST_F16DEV>(P, device, nx, ny, a, b, s, V, S, R);
}

}  // namespace clb
