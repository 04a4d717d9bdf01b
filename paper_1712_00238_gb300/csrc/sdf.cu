// Skeletal density function of a solid from oriented boundary samples (Section 4).
//
// Pass 1 (per query point p_i): |xi| = min_j ||p_i - q_j|| (Eq. 10A; ties go to the
// lowest j, which does not change the value) and the generalised winding number
// w = sum_j a_j (q_j - p).n_j / (S ||q_j - p||^d), S = 2 pi (2D) or 4 pi (3D); the
// point is inside (pmc = -1) when w > 1/2, a membership derived from the
// consistent outward orientation of the samples.
// Pass 2: rho(p_i) = sum_j phi(zeta_ij) cos(theta_ij) a_j (Eq. 13 as a midpoint
// sum) with zeta = xi + i eta (Eq. 11), cos(theta) = (p - q).n / eta (Eq. 12a),
// phi = lambda / sqrt(2 pi) zeta^-2 g_sigma(eta/|xi| - 1) (Eq. 15),
// lambda = +lambda1 outside / -lambda2 inside (Eq. 16c), and only samples with
// eta/|xi| - 1 <= eps (Eq. 17t).  In 2D every element is weighted by its planar
// angle over 2 pi, i.e. the 3D summand times 2 eta.
// Both passes stage boundary tiles in shared memory; one query point per thread.
#include <math.h>

#include "kernels.cuh"

namespace sd {

constexpr int SDF_TILE = 256;

template <typename T, int D>
__global__ void __launch_bounds__(SDF_TILE) k_sdf_nearest(SdfArgs<T> a) {
    __shared__ vec4<T> sq[SDF_TILE];
    __shared__ vec4<T> sn[SDF_TILE];  // normal with the area in .w
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.m;
    vec4<T> p;
    if (live) p = a.qry[i];
    else { p.x = p.y = p.z = p.w = T(0); }
    T dmin = INFINITY;
    T wind = T(0);
    for (int64_t t0 = 0; t0 < a.n_b; t0 += SDF_TILE) {
        const int64_t j = t0 + threadIdx.x;
        if (j < a.n_b) {
            sq[threadIdx.x] = a.bnd[j];
            vec4<T> nn = a.nrm[j];
            nn.w = a.area[j];
            sn[threadIdx.x] = nn;
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)SDF_TILE, a.n_b - t0);
        for (int k = 0; k < cnt; ++k) {
            const vec4<T> q = sq[k];
            const vec4<T> nn = sn[k];
            const T dx = q.x - p.x, dy = q.y - p.y, dz = (D == 3) ? q.z - p.z : T(0);
            const T d2 = dx * dx + dy * dy + dz * dz;
            dmin = d2 < dmin ? d2 : dmin;
            const T dot = dx * nn.x + dy * nn.y + dz * nn.z;
            if (D == 3) wind += nn.w * dot / (d2 * sqrt(d2));
            else wind += nn.w * dot / d2;
        }
        __syncthreads();
    }
    if (!live) return;
    const T S = (D == 3) ? T(4.0 * M_PI) : T(2.0 * M_PI);
    a.xi_abs[i] = sqrt(dmin);
    int8_t m = (wind / S > T(0.5)) ? int8_t(-1) : int8_t(1);
    if (a.pmc_override) m = a.pmc_override[i] < 0 ? int8_t(-1) : int8_t(1);
    a.pmc[i] = m;
}

// Kahan-compensated accumulation
template <typename T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

template <typename T, int D>
__global__ void __launch_bounds__(SDF_TILE) k_sdf_sum(SdfArgs<T> a) {
    __shared__ vec4<T> sq[SDF_TILE];
    __shared__ vec4<T> sn[SDF_TILE];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.m;
    vec4<T> p;
    T xabs = T(1), xi = T(1);
    if (live) {
        p = a.qry[i];
        xabs = a.xi_abs[i];
        xi = a.pmc[i] < 0 ? -xabs : xabs;
    } else {
        p.x = p.y = p.z = p.w = T(0);
    }
    const T lam = xi > T(0) ? a.lam1 : -a.lam2;
    const T pref = lam / (T(2.0 * M_PI) * a.sigma);  // lambda/sqrt(2 pi) * 1/(sqrt(2 pi) sigma)
    const T inv_xabs = T(1) / xabs;
    const T inv_2s2 = T(1) / (T(2) * a.sigma * a.sigma);
    const T xi2 = xi * xi;
    T sr = 0, cr = 0, si = 0, ci = 0;
    for (int64_t t0 = 0; t0 < a.n_b; t0 += SDF_TILE) {
        const int64_t j = t0 + threadIdx.x;
        if (j < a.n_b) {
            sq[threadIdx.x] = a.bnd[j];
            vec4<T> nn = a.nrm[j];
            nn.w = a.area[j];
            sn[threadIdx.x] = nn;
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)SDF_TILE, a.n_b - t0);
        for (int k = 0; k < cnt; ++k) {
            const vec4<T> q = sq[k];
            const T dx = p.x - q.x, dy = p.y - q.y, dz = (D == 3) ? p.z - q.z : T(0);
            const T d2 = dx * dx + dy * dy + dz * dz;
            const T eta = sqrt(d2);
            const T rm1 = eta * inv_xabs - T(1);
            if (a.eps >= T(0) && rm1 > a.eps) continue;
            const vec4<T> nn = sn[k];
            const T E = exp(-rm1 * rm1 * inv_2s2);
            const T cos_t = (dx * nn.x + dy * nn.y + dz * nn.z) / eta;
            // zeta^-2 = (xi - i eta)^2 / (xi^2 + eta^2)^2
            const T den = xi2 + d2;
            const T inv_den2 = T(1) / (den * den);
            const T zr = (xi2 - d2) * inv_den2;
            const T zi = T(-2) * xi * eta * inv_den2;
            T f = pref * E * cos_t * nn.w;
            if (D == 2) f *= T(2) * eta;  // planar angle measure
            kahan_add(sr, cr, f * zr);
            kahan_add(si, ci, f * zi);
        }
        __syncthreads();
    }
    if (!live) return;
    const T v = a.vol[i];
    a.c_out[i] = mk(sr * v, si * v);
    if (a.rho_out) a.rho_out[i] = mk(sr, si);
    vec4<T> po = p;
    po.w = T(0);
    a.pos_out[i] = po;
}

template <typename T>
cudaError_t launch_sdf(const SdfArgs<T>& a, int dim, cudaStream_t st) {
    if (a.m == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((a.m + SDF_TILE - 1) / SDF_TILE);
    if (dim == 2) {
        k_sdf_nearest<T, 2><<<nb, SDF_TILE, 0, st>>>(a);
        k_sdf_sum<T, 2><<<nb, SDF_TILE, 0, st>>>(a);
    } else {
        k_sdf_nearest<T, 3><<<nb, SDF_TILE, 0, st>>>(a);
        k_sdf_sum<T, 3><<<nb, SDF_TILE, 0, st>>>(a);
    }
    note_launch(2);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_radius(const vec4<T>* p, int64_t m, int dim, double* out) {
    double best = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const vec4<T> v = p[i];
        double r2 = (double)v.x * v.x + (double)v.y * v.y + (dim == 3 ? (double)v.z * v.z : 0.0);
        best = fmax(best, r2);
    }
    for (int off = 16; off > 0; off >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0) {
        // r2 >= 0: ordering of the IEEE bits matches the ordering of the values
        atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(best));
    }
}

template <typename T>
cudaError_t launch_radius(const vec4<T>* p, int64_t m, int dim, double* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    if (m == 0) return cudaSuccess;
    const int nb = (int)((m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024);
    k_radius<T><<<nb, 256, 0, st>>>(p, m, dim, out);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_sdf<float>(const SdfArgs<float>&, int, cudaStream_t);
template cudaError_t launch_sdf<double>(const SdfArgs<double>&, int, cudaStream_t);
template cudaError_t launch_radius<float>(const vec4<float>*, int64_t, int, double*, cudaStream_t);
template cudaError_t launch_radius<double>(const vec4<double>*, int64_t, int, double*, cudaStream_t);

}  // namespace sd
