// Top-k selection over per-rotation candidates that allocates no device memory.
//
// Some callers cannot call cudaMalloc while they run: a real-time loop that
// preallocated everything and must not stall on the implicit device
// synchronisation of cudaMalloc/cudaFree, an engine that shares a fixed memory
// pool with other components and forbids growth, or code whose device memory is
// handed out by a foreign allocator.  sd_top_k_poses takes its scratch from the
// context's growable workspace; this entry point instead keeps the selection's
// scratch (one bit per candidate) in a file-scope device array of fixed size.
// Every GPU that loads the library holds that array until the process exits.
#include <mutex>

#include "../../include/sdfdock.h"
#include "kernels.cuh"

// Error reporting and device of a context (defined with the context in api.cu).
int sd_internal_fail(sd_ctx* ctx, int code, const char* fmt, ...);
int sd_internal_device(const sd_ctx* ctx);

namespace {

constexpr int64_t kMaxCandidates = (int64_t)1 << 20;  // SD_TOP_K_STATIC_MAX
constexpr int kMaxDevices = 64;

// Scratch bitset of the selection (128 KiB); the selection kernel clears the
// bits it uses before reading them.
static __device__ __align__(256) unsigned g_topk_flags[kMaxCandidates / 32];

std::mutex g_mu;
void* g_flags_addr[kMaxDevices] = {};

// Device address of the bitset on the current device, looked up once per device.
cudaError_t flags_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_flags_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_topk_flags);
        if (e != cudaSuccess) return e;
        g_flags_addr[device] = p;
    }
    *out = g_flags_addr[device];
    return cudaSuccess;
}

}  // namespace

int sd_top_k_static(sd_ctx* ctx, const sd_cand* cand, int64_t n_cand, int k, sd_cand* out, void* stream) {
    if (!ctx) return SD_ERR_ARG;
    if (!cand || !out) return sd_internal_fail(ctx, SD_ERR_ARG, "top_k_static: NULL pointer");
    if (n_cand < 1 || n_cand > kMaxCandidates)
        return sd_internal_fail(ctx, SD_ERR_ARG, "top_k_static: n_cand must be in [1, 2^20] (got %lld)",
                                (long long)n_cand);
    if (k < 1 || k > 4096) return sd_internal_fail(ctx, SD_ERR_ARG, "top_k_static: k must be in [1, 4096]");
    const int device = sd_internal_device(ctx);
    if (device < 0 || device >= kMaxDevices) return sd_internal_fail(ctx, SD_ERR_ARG, "top_k_static: bad device");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    void* flags = nullptr;
    cudaError_t e = flags_address(device, &flags);
    if (e == cudaSuccess) e = sd::launch_topk(cand, n_cand, k, out, (unsigned*)flags, (cudaStream_t)stream);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess)
        return sd_internal_fail(ctx, SD_ERR_CUDA, "top_k_static: %s", cudaGetErrorString(e));
    return SD_OK;
}
