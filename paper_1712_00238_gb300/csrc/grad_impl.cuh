// Score and gradient at arbitrary poses by a type-2 gather (the adjoint of the
// spreading step), for the gradient-driven pose search of Section 6.
//
// The fixed shape's band-limited field Phi(x) = sum_i c1_i K_N(x - p1_i) and its
// gradient are tabulated once on the oversampled periodic grid (inverse FFT of
// the deconvolved spectrum).  For pose (R, t): f = sum_j c2_j Phi(R p2_j + t),
// interpolated with the same exponential-of-semicircle kernel as the spreading.
// With g_j = Re(c2_j grad Phi(y_j)):  d Re f / dt = sum_j g_j, the torque
// tau = sum_j (R p2_j) x g_j is d Re f / d omega for a left perturbation
// R <- exp([omega]x) R, and d Re f / d q = 2 ((0, tau) (x) q/|q|) / |q| through
// R(q/|q|) (a vector orthogonal to q).
#pragma once
#include <math.h>

#include "kernels.cuh"

namespace sd {

constexpr int GA_THREADS = 256;

__device__ __forceinline__ int wrap_n(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

// The four fields of cell i (Phi, d/dx, d/dy, d/dz Phi; 32 bytes for FP32, at a
// 32-byte aligned address) as two 16-byte read-only loads; FP64 cells load
// field by field.
__device__ __forceinline__ void load_cell(const cplx<float>* G, int64_t i, cplx<float> f[4]) {
    const float4* p = reinterpret_cast<const float4*>(G + 4 * i);
    const float4 a = __ldg(p), b = __ldg(p + 1);
    f[0] = mk(a.x, a.y);
    f[1] = mk(a.z, a.w);
    f[2] = mk(b.x, b.y);
    f[3] = mk(b.z, b.w);
}
__device__ __forceinline__ void load_cell(const cplx<double>* G, int64_t i, cplx<double> f[4]) {
    const cplx<double>* p = G + 4 * i;
#pragma unroll
    for (int k = 0; k < 4; ++k) f[k] = p[k];
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(GA_THREADS) k_gather(GatherArgs<T> a) {
    using C = cplx<T>;
    __shared__ T Rm[9], tv[3];
    __shared__ double red[GA_THREADS / 32][7];
    const int pose = blockIdx.y;
    if (threadIdx.x == 0) {
        const T* q = a.quats + 4 * (int64_t)pose;
        const T w = q[0], x = q[1], y = q[2], z = q[3];
        const T n2 = w * w + x * x + y * y + z * z;
        const T s = n2 > T(0) ? T(2) / n2 : T(0);
        Rm[0] = T(1) - s * (y * y + z * z); Rm[1] = s * (x * y - w * z); Rm[2] = s * (x * z + w * y);
        Rm[3] = s * (x * y + w * z); Rm[4] = T(1) - s * (x * x + z * z); Rm[5] = s * (y * z - w * x);
        Rm[6] = s * (x * z - w * y); Rm[7] = s * (y * z + w * x); Rm[8] = T(1) - s * (x * x + y * y);
        const T* t = a.trans + 3 * (int64_t)pose;
        tv[0] = t[0];
        tv[1] = t[1];
        tv[2] = (D == 3) ? t[2] : T(0);
    }
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    T acc[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    if (j < a.m2) {
        const vec4<T> p = a.p2[j];
        const C c = a.c2[j];
        const T pz = (D == 3) ? p.z : T(0);
        T rp[3];
        rp[0] = Rm[0] * p.x + Rm[1] * p.y + Rm[2] * pz;
        rp[1] = Rm[3] * p.x + Rm[4] * p.y + Rm[5] * pz;
        rp[2] = (D == 3) ? Rm[6] * p.x + Rm[7] * p.y + Rm[8] * pz : T(0);
        // x and y weights and indices in registers (their loops are unrolled); the
        // z loop stays rolled and evaluates its weight per iteration, so no array
        // is indexed at run time
        T wt[2][W];
        int ix[2][W];
        const T half = T(W) * T(0.5), inv_half = T(2) / T(W);
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const T g = (rp[d] + tv[d]) * a.inv_h;
            const int u0 = (int)ceil(g - half);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const T zz = (T(u0 + k) - g) * inv_half;
                const T z2 = zz * zz;
                wt[d][k] = (z2 <= T(1)) ? exp(a.beta * (sqrt(T(1) - z2) - T(1))) : T(0);
                ix[d][k] = wrap_n(u0 + k, a.n);
            }
        }
        C phi = mk(T(0), T(0)), g0 = phi, g1 = phi, g2 = phi;
        const int n = a.n;
        if constexpr (D == 2) {
#pragma unroll
            for (int ky = 0; ky < W; ++ky) {
                const int64_t rb = (int64_t)ix[1][ky] * n;
#pragma unroll
                for (int kx = 0; kx < W; ++kx) {
                    const T wgt = wt[1][ky] * wt[0][kx];
                    C f[4];
                    load_cell(a.G, rb + ix[0][kx], f);
                    phi = cadd(phi, cscale(f[0], wgt));
                    g0 = cadd(g0, cscale(f[1], wgt));
                    g1 = cadd(g1, cscale(f[2], wgt));
                }
            }
        } else {
            const T gzc = (rp[2] + tv[2]) * a.inv_h;
            const int uz0 = (int)ceil(gzc - half);
#pragma unroll 1
            for (int kz = 0; kz < W; ++kz) {
                const T zz = (T(uz0 + kz) - gzc) * inv_half;
                const T z2 = zz * zz;
                const T wz = (z2 <= T(1)) ? exp(a.beta * (sqrt(T(1) - z2) - T(1))) : T(0);
                const int64_t zb = (int64_t)wrap_n(uz0 + kz, n) * n;
#pragma unroll
                for (int ky = 0; ky < W; ++ky) {
                    const int64_t rb = (zb + ix[1][ky]) * n;
                    const T wzy = wz * wt[1][ky];
#pragma unroll
                    for (int kx = 0; kx < W; ++kx) {
                        const T wgt = wzy * wt[0][kx];
                        C f[4];
                        load_cell(a.G, rb + ix[0][kx], f);
                        phi = cadd(phi, cscale(f[0], wgt));
                        g0 = cadd(g0, cscale(f[1], wgt));
                        g1 = cadd(g1, cscale(f[2], wgt));
                        g2 = cadd(g2, cscale(f[3], wgt));
                    }
                }
            }
        }
        const T gx = c.x * g0.x - c.y * g0.y;
        const T gy = c.x * g1.x - c.y * g1.y;
        const T gz = (D == 3) ? c.x * g2.x - c.y * g2.y : T(0);
        acc[0] = c.x * phi.x - c.y * phi.y;
        acc[1] = gx;
        acc[2] = gy;
        acc[3] = gz;
        acc[4] = rp[1] * gz - rp[2] * gy;
        acc[5] = rp[2] * gx - rp[0] * gz;
        acc[6] = rp[0] * gy - rp[1] * gx;
    }
    double v[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        v[k] = (double)acc[k];
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 7; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 7) {
        double s = 0.0;
        for (int w = 0; w < GA_THREADS / 32; ++w) s += red[w][threadIdx.x];
        atomicAdd(a.acc + 8 * (int64_t)pose + threadIdx.x, s);
    }
}

template <typename T>
cudaError_t launch_gather(const GatherArgs<T>& a, int dim, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.acc, 0, sizeof(double) * 8 * (a.P > 0 ? a.P : 1), st);
    if (e != cudaSuccess || a.P == 0 || a.m2 == 0) return e;
    const dim3 grid((unsigned)((a.m2 + GA_THREADS - 1) / GA_THREADS), (unsigned)a.P);
#define SD_GATHER_CASE(WW)                                                      \
    case WW:                                                                    \
        if (dim == 2) k_gather<T, 2, WW><<<grid, GA_THREADS, 0, st>>>(a);        \
        else k_gather<T, 3, WW><<<grid, GA_THREADS, 0, st>>>(a);                 \
        note_launch();                                                          \
        return cudaGetLastError();
    switch (a.w) {
        SD_GATHER_CASE(4) SD_GATHER_CASE(5) SD_GATHER_CASE(6) SD_GATHER_CASE(7) SD_GATHER_CASE(8)
        SD_GATHER_CASE(10) SD_GATHER_CASE(12) SD_GATHER_CASE(16)
    }
#undef SD_GATHER_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
__global__ void k_grad_finalize(const double* acc, const T* quats, int64_t P, int dim, T* score, T* dq, T* dt) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double* a = acc + 8 * p;
    score[p] = (T)a[0];
    dt[3 * p + 0] = (T)a[1];
    dt[3 * p + 1] = (T)a[2];
    dt[3 * p + 2] = (T)(dim == 3 ? a[3] : 0.0);
    const double tx = a[4], ty = a[5], tz = a[6];
    const T* q = quats + 4 * p;
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double nq = sqrt(w * w + x * x + y * y + z * z);
    const double inv = nq > 0 ? 1.0 / nq : 0.0;
    const double u0 = w * inv, ux = x * inv, uy = y * inv, uz = z * inv;
    // (0, tau) (x) u = (-tau.u, u0 tau + tau x u)
    const double s0 = -(tx * ux + ty * uy + tz * uz);
    const double sx = u0 * tx + (ty * uz - tz * uy);
    const double sy = u0 * ty + (tz * ux - tx * uz);
    const double sz = u0 * tz + (tx * uy - ty * ux);
    dq[4 * p + 0] = (T)(2.0 * s0 * inv);
    dq[4 * p + 1] = (T)(2.0 * sx * inv);
    dq[4 * p + 2] = (T)(2.0 * sy * inv);
    dq[4 * p + 3] = (T)(2.0 * sz * inv);
}

template <typename T>
cudaError_t launch_grad_finalize(const double* acc, const T* quats, int64_t P, int dim, T* score, T* dq, T* dt,
                                 cudaStream_t st) {
    if (P == 0) return cudaSuccess;
    k_grad_finalize<T><<<(unsigned)((P + 127) / 128), 128, 0, st>>>(acc, quats, P, dim, score, dq, dt);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sd
