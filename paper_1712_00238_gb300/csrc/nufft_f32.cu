// FP32 instantiation of the nonuniform-FFT passes.
#include "nufft_impl.cuh"
SD_INSTANTIATE_NUFFT(float)
