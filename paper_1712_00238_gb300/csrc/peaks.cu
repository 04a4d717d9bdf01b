// ALU throughput probes: the rates that bound the kernels that are limited by
// arithmetic rather than memory (the SDF sums: FP32 FMA and the special-function
// unit; the FP64 re-score: FP64 FMA) or by shared-memory atomics (the spreading
// tiles), measured on the device they run on.  Each thread runs eight
// independent dependency chains of one instruction class, long enough to hide
// its latency (the atomic kinds: eight adds per iteration to the thread's own
// shared word, the lanes of a warp on distinct banks), over several waves of
// CTAs; the rate is the best of three timed launches after one untimed one.
#include <math.h>

#include <type_traits>

#include "../../include/sdfdock.h"
#include "kernels.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_peak(float* sink, int iters) {
    const float seed = 1e-3f * (float)(threadIdx.x & 31);
    if constexpr (KIND == SD_PEAK_SHARED_ADD32 || KIND == SD_PEAK_SHARED_ADD64) {
        // each thread adds to its own word (consecutive lanes, consecutive words)
        using W = std::conditional_t<KIND == SD_PEAK_SHARED_ADD32, unsigned int, unsigned long long>;
        __shared__ W acc[kThreads];
        acc[threadIdx.x] = 0;
        __syncthreads();
        const W step = (W)(threadIdx.x & 7) + 1;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) atomicAdd(acc + threadIdx.x, step + (W)k);
        __syncthreads();
        if (acc[threadIdx.x] == (W)1) sink[0] = 1.f;  // never true: keeps the adds
    } else if constexpr (KIND == SD_PEAK_FP64_FMA) {
        double v[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) v[k] = 0.5 + seed + 0.01 * k;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) v[k] = fma(v[k], 0.9999, 1e-4);  // fixed point 1
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += v[k];
        if (t == -1.0) sink[0] = (float)t;  // never true: keeps the chains
    } else {
        float v[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) v[k] = 0.5f + seed + 0.01f * k;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if constexpr (KIND == SD_PEAK_FP32_FMA) {
                    v[k] = fmaf(v[k], 0.9999f, 1e-4f);
                } else if constexpr (KIND == SD_PEAK_SFU_EX2) {
                    float e;
                    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(v[k]));
                    v[k] = e - 1.5f;  // stays in (-1, 0)
                } else {
                    float e;
                    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(v[k]));
                    v[k] = e + 0.5f;  // stays near 1.3
                }
            }
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += v[k];
        if (t == -1.0f) sink[0] = t;
    }
}

}  // namespace

int sd_alu_peak(int device, int kind, double* ops_per_s) {
    if (!ops_per_s || kind < 0 || kind > SD_PEAK_SHARED_ADD64) return SD_ERR_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return SD_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return SD_ERR_ARG;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = 8 * (sms > 0 ? sms : 1);
    // enough iterations for a launch of a few to tens of milliseconds
    const int iters = (kind == SD_PEAK_FP64_FMA) ? 2048 : (kind == SD_PEAK_FP32_FMA ? 65536 : 8192);
    void (*kern)(float*, int) = kind == SD_PEAK_FP32_FMA       ? k_peak<SD_PEAK_FP32_FMA>
                                : kind == SD_PEAK_FP64_FMA     ? k_peak<SD_PEAK_FP64_FMA>
                                : kind == SD_PEAK_SFU_EX2      ? k_peak<SD_PEAK_SFU_EX2>
                                : kind == SD_PEAK_SFU_RSQRT    ? k_peak<SD_PEAK_SFU_RSQRT>
                                : kind == SD_PEAK_SHARED_ADD32 ? k_peak<SD_PEAK_SHARED_ADD32>
                                                               : k_peak<SD_PEAK_SHARED_ADD64>;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SD_OK;
    float best = INFINITY;
    if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = SD_ERR_CUDA;
    } else {
        for (int rep = 0; rep < 4 && rc == SD_OK; ++rep) {
            cudaEventRecord(e0, nullptr);
            kern<<<blocks, kThreads>>>(sink, iters);
            sd::note_launch();
            cudaEventRecord(e1, nullptr);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                rc = SD_ERR_CUDA;
            else if (rep > 0 && ms < best)
                best = ms;
        }
    }
    if (rc == SD_OK) {
        // FMA probes count two floating-point operations per instruction
        const double per = (kind == SD_PEAK_FP32_FMA || kind == SD_PEAK_FP64_FMA) ? 2.0 : 1.0;
        const double ops = per * (double)blocks * kThreads * kChains * (double)iters;
        *ops_per_s = ops / (best * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}
