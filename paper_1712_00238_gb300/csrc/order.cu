// Spatial ordering of a shape's samples.
//
// Samples are kept in Morton (Z-curve) order of their position inside the
// shape's bounding cube [-R, R]^d: consecutive samples are close in space, so
// a CTA that takes a contiguous run of them covers a compact region before and
// after any rotation.  This keeps the spread tiles and gather footprints small
// and lets the re-score skip whole blocks of far pairs.  The order changes
// nothing but the order of floating-point sums.
#include <cub/device/device_radix_sort.cuh>

#include "kernels.cuh"

namespace sd {

__device__ __forceinline__ uint32_t spread_bits10(uint32_t v) {
    // 10 bits -> every third bit of 30
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t spread_bits16(uint32_t v) {
    // 16 bits -> every second bit of 32
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

template <typename T>
__global__ void k_morton_keys(const vec4<T>* pos, int64_t m, double lo, double scale, int dim, uint32_t* keys,
                              int32_t* vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const vec4<T> p = pos[i];
    const double q[3] = {(double)p.x, (double)p.y, (double)p.z};
    const uint32_t top = (dim == 3) ? 1023u : 65535u;
    uint32_t k = 0;
    for (int d = 0; d < dim; ++d) {
        double f = (q[d] - lo) * scale;
        uint32_t v = f <= 0.0 ? 0u : (f >= (double)top ? top : (uint32_t)f);
        k |= (dim == 3 ? spread_bits10(v) : spread_bits16(v)) << d;
    }
    keys[i] = k;
    vals[i] = (int32_t)i;
}

template <typename T>
__global__ void k_permute(const int32_t* perm, const vec4<T>* pin, const cplx<T>* cin, vec4<T>* pout, cplx<T>* cout,
                          int64_t m) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int32_t j = perm[i];
    pout[i] = pin[j];
    cout[i] = cin[j];
}

// perm[i] = index of the sample with the i-th smallest Morton code of pos
// inside the cube [-radius, radius]^d (a stable order).
template <typename T>
cudaError_t morton_order(const vec4<T>* pos, int64_t m, double radius, int dim, int32_t* perm, cudaStream_t st) {
    if (m < 1) return cudaSuccess;
    const double R = radius > 0 ? radius * (1.0 + 1e-6) : 1.0;
    const double scale = ((dim == 3) ? 1024.0 : 65536.0) / (2.0 * R);
    uint32_t *k0 = nullptr, *k1 = nullptr;
    int32_t* v0 = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t e = cudaSuccess;
    auto done = [&](cudaError_t r) {
        pool_free(k0, st); pool_free(k1, st); pool_free(v0, st); pool_free(tmp, st);
        return r;
    };
    if ((e = pool_alloc((void**)&k0, m * sizeof(uint32_t), st)) != cudaSuccess) return done(e);
    if ((e = pool_alloc((void**)&k1, m * sizeof(uint32_t), st)) != cudaSuccess) return done(e);
    if ((e = pool_alloc((void**)&v0, m * sizeof(int32_t), st)) != cudaSuccess) return done(e);
    const unsigned nb = (unsigned)((m + 255) / 256);
    k_morton_keys<T><<<nb, 256, 0, st>>>(pos, m, -R, scale, dim, k0, v0);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
    const int bits = (dim == 3) ? 30 : 32;
    e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k0, k1, v0, perm, (int)m, 0, bits, st);
    if (e != cudaSuccess) return done(e);
    if ((e = pool_alloc(&tmp, tmp_bytes, st)) != cudaSuccess) return done(e);
    e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k0, k1, v0, perm, (int)m, 0, bits, st);
    return done(e);
}

// Reorders pos and c in place (through temporaries) by the Morton code of pos.
template <typename T>
cudaError_t sort_by_morton(vec4<T>* pos, cplx<T>* c, int64_t m, double radius, int dim, cudaStream_t st) {
    if (m < 2) return cudaSuccess;
    int32_t* perm = nullptr;
    vec4<T>* pt = nullptr;
    cplx<T>* ct = nullptr;
    cudaError_t e = cudaSuccess;
    auto done = [&](cudaError_t r) {
        pool_free(perm, st); pool_free(pt, st); pool_free(ct, st);
        return r;
    };
    if ((e = pool_alloc((void**)&perm, m * sizeof(int32_t), st)) != cudaSuccess) return done(e);
    if ((e = pool_alloc((void**)&pt, m * sizeof(vec4<T>), st)) != cudaSuccess) return done(e);
    if ((e = pool_alloc((void**)&ct, m * sizeof(cplx<T>), st)) != cudaSuccess) return done(e);
    if ((e = morton_order<T>(pos, m, radius, dim, perm, st)) != cudaSuccess) return done(e);
    if ((e = cudaMemcpyAsync(pt, pos, m * sizeof(vec4<T>), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return done(e);
    if ((e = cudaMemcpyAsync(ct, c, m * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return done(e);
    k_permute<T><<<(unsigned)((m + 255) / 256), 256, 0, st>>>(perm, pt, ct, pos, c, m);
    note_launch();
    e = cudaGetLastError();
    return done(e);
}

template cudaError_t sort_by_morton<float>(vec4<float>*, cplx<float>*, int64_t, double, int, cudaStream_t);
template cudaError_t sort_by_morton<double>(vec4<double>*, cplx<double>*, int64_t, double, int, cudaStream_t);
template cudaError_t morton_order<float>(const vec4<float>*, int64_t, double, int, int32_t*, cudaStream_t);
template cudaError_t morton_order<double>(const vec4<double>*, int64_t, double, int, int32_t*, cudaStream_t);

}  // namespace sd
