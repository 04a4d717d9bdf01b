// FP32 instantiation of the type-2 score and gradient gather.
#include "grad_impl.cuh"

namespace sd {
template cudaError_t launch_gather<float>(const GatherArgs<float>&, int, cudaStream_t);
template cudaError_t launch_grad_finalize<float>(const double*, const float*, int64_t, int, float*, float*, float*,
                                                 cudaStream_t);
template cudaError_t launch_refine_step<float>(const double*, float*, float*, double*, int64_t, int,
                                                const RefineParams&, int, float*, int, cudaStream_t);
}  // namespace sd
