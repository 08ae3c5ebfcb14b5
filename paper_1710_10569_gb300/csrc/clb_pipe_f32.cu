// clb_pipe_f32.cu -- the staged-rows step kernel's launches for the f32 storage form
// (templates in clb_pipe.cuh).
#include "clb_pipe.cuh"

namespace clb {

template <>
cudaError_t enqueue_pipe_form<ST_F32>(const LatParams<typename Storage<ST_F32>::A>& P, int device, int nx, int ny,
                                    const void* a, void* b, cudaStream_t s, int V, int S, int R)
{
    return pipe::enqueue_pipe_v<ST_F32>(P, device, nx, ny, a, b, s, V, S, R);
}

}  // namespace clb
