// Hessian-action launchers for float vectors with float stored data (one
// translation unit per precision so that the kernel variants compile in parallel).
#include "elem_apply_impl.cuh"

namespace tmop {

cudaError_t launch_apply_f32(int d, int p, int q, const ElemParams &P, const void *v, const void *H, void *ev,
               const int *stop, int k, cudaStream_t s, const BatchArgs *B, int64_t ntiles,
               int variant)
{
    return launch_apply_typed<float, float>(d, p, q, P, v, H, ev, stop, k, s, B, ntiles, variant);
}

}  // namespace tmop
