// FP64 instantiation of the type-2 score and gradient gather.
#include "grad_impl.cuh"

namespace sd {
template cudaError_t launch_gather<double>(const GatherArgs<double>&, int, cudaStream_t);
template cudaError_t launch_grad_finalize<double>(const double*, const double*, int64_t, int, double*, double*,
                                                  double*, cudaStream_t);
template cudaError_t launch_refine_step<double>(const double*, double*, double*, double*, int64_t, int,
                                                const RefineParams&, int, double*, int, cudaStream_t);
}  // namespace sd
