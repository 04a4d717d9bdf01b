// Shared device helpers: complex arithmetic on float2/double2, real-type traits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sd {

// Counts kernel launches made by the library (defined in api.cu).
void note_launch(int n = 1);

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename T> struct vec4_of;
template <> struct vec4_of<float> { using type = float4; };
template <> struct vec4_of<double> { using type = double4_32a; };
template <typename T> using vec4 = typename vec4_of<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) { return mk(a.x * s, a.y * s); }
// a * (-i) for the forward sign, a * (+i) for the inverse sign
template <bool INV, typename C> __host__ __device__ __forceinline__ C mul_mi(C a) {
    return INV ? mk(-a.y, a.x) : mk(a.y, -a.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
// a + (-i) d and a - (-i) d (forward sign; +i for the inverse) without forming the
// rotated operand
template <bool INV, typename C> __host__ __device__ __forceinline__ C add_mi(C a, C d) {
    return INV ? mk(a.x - d.y, a.y + d.x) : mk(a.x + d.y, a.y - d.x);
}
template <bool INV, typename C> __host__ __device__ __forceinline__ C sub_mi(C a, C d) {
    return INV ? mk(a.x + d.y, a.y - d.x) : mk(a.x - d.y, a.y + d.x);
}

// Single-precision pairs: on sm_100+ one paired instruction adds, subtracts or
// scales both components (IEEE round-to-nearest per component, the same values
// as two scalar operations; a - b is the exact product b * -1 plus a, rounded once).
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
#else
    return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
    return __fmul2_rn(a, make_float2(s, s));
#else
    return make_float2(a.x * s, a.y * s);
#endif
}

// Complex accumulation into global memory (atomic).
__device__ __forceinline__ void atomic_cadd(float2* p, float2 v) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    atomicAdd(p, v);  // one vector reduction (sm_90+)
#else
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
#endif
}
__device__ __forceinline__ void atomic_cadd(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

// Rotation matrix of q / |q| (Hamilton, active), row-major 3x3, from doubles.
template <typename T>
__device__ __forceinline__ void quat_to_matrix(const double* q4, T R[9]) {
    double w = q4[0], x = q4[1], y = q4[2], z = q4[3];
    double n = w * w + x * x + y * y + z * z;
    double s = (n > 0.0) ? 2.0 / n : 0.0;
    R[0] = T(1.0 - s * (y * y + z * z)); R[1] = T(s * (x * y - w * z)); R[2] = T(s * (x * z + w * y));
    R[3] = T(s * (x * y + w * z)); R[4] = T(1.0 - s * (x * x + z * z)); R[5] = T(s * (y * z - w * x));
    R[6] = T(s * (x * z - w * y)); R[7] = T(s * (y * z + w * x)); R[8] = T(1.0 - s * (x * x + y * y));
}

}  // namespace sd
