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
// A block of queries may split its boundary tiles across several CTAs (grid
// y), each writing a partial (nearest distance and winding sum; rho); a
// finishing kernel combines the partials in a fixed order, so the results do
// not depend on how many CTAs shared the work's scheduling.
#include <float.h>
#include <math.h>

#include "kernels.cuh"

namespace sd {

// Queries are processed in Morton order (perm_q) and the boundary samples are
// pre-sorted the same way, so a CTA's 256 queries and a tile's 256 samples are
// each spatially compact.  Pass 2 skips every tile whose bounding box lies
// farther than (1 + eps) max|xi| from the CTA's box: all its pairs would fail
// the truncation test of Eq. 17t anyway (the restriction to eps-approximate
// nearest neighbours of Section 4), so the sum is unchanged.

template <typename T>
__device__ __forceinline__ T recip(T x) { return T(1) / x; }
template <>
__device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }

template <typename T, int D>
__global__ void __launch_bounds__(SDF_TILE) k_sdf_nearest(SdfArgs<T> a, int tiles_per_split, T* part_d2, T* part_w) {
    __shared__ vec4<T> sq[SDF_TILE];
    __shared__ vec4<T> sn[SDF_TILE];  // normal with the area in .w
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.m;
    const int64_t src = live ? (a.perm_q ? (int64_t)a.perm_q[i] : i) : 0;
    vec4<T> p;
    if (live) p = a.qry[src];
    else { p.x = p.y = p.z = p.w = T(0); }
    T dmin = INFINITY;
    T wind = T(0);
    const int64_t t_lo = (int64_t)blockIdx.y * tiles_per_split * SDF_TILE;
    const int64_t t_hi = min(a.n_b, t_lo + (int64_t)tiles_per_split * SDF_TILE);
    for (int64_t t0 = t_lo; t0 < t_hi; t0 += SDF_TILE) {
        const int64_t j = t0 + threadIdx.x;
        if (j < a.n_b) {
            sq[threadIdx.x] = a.bnd[j];
            sn[threadIdx.x] = a.nrm[j];
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
            if (D == 3) {
                const T r = rsqrt(d2);
                wind += nn.w * dot * r * r * r;
            } else {
                wind += nn.w * dot * recip(d2);
            }
        }
        __syncthreads();
    }
    if (!live) return;
    part_d2[(int64_t)blockIdx.y * a.m + i] = dmin;
    part_w[(int64_t)blockIdx.y * a.m + i] = wind;
}

// Nearest distance (the smallest partial) and membership (the partial winding
// sums added in split order) of each query.
template <typename T, int D>
__global__ void k_sdf_nearest_finish(SdfArgs<T> a, int splits, const T* part_d2, const T* part_w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    T dmin = INFINITY, wind = T(0);
    for (int k = 0; k < splits; ++k) {
        const T d = part_d2[(int64_t)k * a.m + i];
        dmin = d < dmin ? d : dmin;
        wind += part_w[(int64_t)k * a.m + i];
    }
    const T S = (D == 3) ? T(4.0 * M_PI) : T(2.0 * M_PI);
    a.xi_abs[i] = sqrt(dmin);
    int8_t m = (wind > T(0.5) * S) ? int8_t(-1) : int8_t(1);
    if (a.pmc_override) {
        const int64_t src = a.perm_q ? (int64_t)a.perm_q[i] : i;
        m = a.pmc_override[src] < 0 ? int8_t(-1) : int8_t(1);
    }
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

template <typename T, int D, int PHI>
__global__ void __launch_bounds__(SDF_TILE) k_sdf_sum(SdfArgs<T> a, int tiles_per_split, cplx<T>* part) {
    __shared__ vec4<T> sq[SDF_TILE];
    __shared__ vec4<T> sn[SDF_TILE];
    __shared__ float wred[SDF_TILE / 32][7];
    __shared__ float box[7];  // lo[3], hi[3], reach
    float wbox[7] = {0, 0, 0, 0, 0, 0, 0};  // the warp's lo[3], hi[3], reach
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.m;
    const int64_t src = live ? (a.perm_q ? (int64_t)a.perm_q[i] : i) : 0;
    vec4<T> p;
    T xabs = T(1), xi = T(1);
    if (live) {
        p = a.qry[src];
        xabs = a.xi_abs[i];
        xi = a.pmc[i] < 0 ? -xabs : xabs;
    } else {
        p.x = p.y = p.z = p.w = T(0);
    }
    // CTA box and cutoff radius (1 + eps) max|xi| for the tile test
    const bool cull = PHI == SD_PHI_SDF && a.tile_box != nullptr && a.eps >= T(0);
    if (cull) {
        float v[7] = {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX, 0.f};
        if (live) {
            v[0] = v[3] = (float)p.x;
            v[1] = v[4] = (float)p.y;
            v[2] = v[5] = (D == 3) ? (float)p.z : 0.f;
            v[6] = (float)xabs;
        }
        for (int off = 16; off > 0; off >>= 1) {
            for (int d = 0; d < 3; ++d) v[d] = fminf(v[d], __shfl_down_sync(0xffffffffu, v[d], off));
            for (int d = 3; d < 7; ++d) v[d] = fmaxf(v[d], __shfl_down_sync(0xffffffffu, v[d], off));
        }
        if ((threadIdx.x & 31) == 0)
            for (int d = 0; d < 7; ++d) wred[threadIdx.x >> 5][d] = v[d];
        // this warp's own box and reach, for the sub-tile test
        for (int d = 0; d < 7; ++d) wbox[d] = __shfl_sync(0xffffffffu, v[d], 0);
        wbox[6] = wbox[6] * (1.f + (float)a.eps) * (1.f + 1e-4f) + 1e-6f;
        __syncthreads();
        if (threadIdx.x < 7) {
            float r = wred[0][threadIdx.x];
            for (int w = 1; w < SDF_TILE / 32; ++w)
                r = threadIdx.x < 3 ? fminf(r, wred[w][threadIdx.x]) : fmaxf(r, wred[w][threadIdx.x]);
            if (threadIdx.x == 6) r = r * (1.f + (float)a.eps) * (1.f + 1e-4f) + 1e-6f;
            box[threadIdx.x] = r;
        }
        __syncthreads();
    }
    const T lam = xi > T(0) ? a.lam1 : -a.lam2;
    // SDF: lambda/sqrt(2 pi) * 1/(sqrt(2 pi) sigma); proximal: lambda/sqrt(2 pi);
    // radial: 1/(sqrt(2 pi) sigma), times lambda1 (real) outside or lambda2 (imaginary) inside
    const T pref = PHI == SD_PHI_SDF      ? lam / (T(2.0 * M_PI) * a.sigma)
                   : PHI == SD_PHI_PROXIMAL ? lam / sqrt(T(2.0 * M_PI))
                                            : T(1) / (sqrt(T(2.0 * M_PI)) * a.sigma);
    const T inv_r = recip(a.radius);
    const T inv_xabs = recip(xabs);
    const T inv_2s2 = recip(T(2) * a.sigma * a.sigma);
    const T xi2 = xi * xi;
    T sr = 0, cr = 0, si = 0, ci = 0;
    const int64_t tile_lo = (int64_t)blockIdx.y * tiles_per_split;
    const int64_t t_hi = min(a.n_b, (tile_lo + tiles_per_split) * SDF_TILE);
    for (int64_t t0 = tile_lo * SDF_TILE, tile = tile_lo; t0 < t_hi; t0 += SDF_TILE, ++tile) {
        if (cull) {
            const float* tb = a.tile_box + tile * 6;
            const float g0 = fmaxf(0.f, fmaxf(tb[0] - box[3], box[0] - tb[3]));
            const float g1 = fmaxf(0.f, fmaxf(tb[1] - box[4], box[1] - tb[4]));
            const float g2 = (D == 3) ? fmaxf(0.f, fmaxf(tb[2] - box[5], box[2] - tb[5])) : 0.f;
            if (g0 * g0 + g1 * g1 + g2 * g2 > box[6] * box[6]) continue;  // same in every thread
        }
        const int64_t j = t0 + threadIdx.x;
        __syncthreads();
        if (j < a.n_b) {
            sq[threadIdx.x] = a.bnd[j];
            sn[threadIdx.x] = a.nrm[j];
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)SDF_TILE, a.n_b - t0);
        for (int k = 0; k < cnt; ++k) {
            if (cull && a.sub_box && (k & 31) == 0) {
                // skip the 32-sample sub-tile when it lies beyond this warp's reach
                const float* sb = a.sub_box + (tile * (SDF_TILE / 32) + (k >> 5)) * 6;
                const float g0 = fmaxf(0.f, fmaxf(sb[0] - wbox[3], wbox[0] - sb[3]));
                const float g1 = fmaxf(0.f, fmaxf(sb[1] - wbox[4], wbox[1] - sb[4]));
                const float g2 = (D == 3) ? fmaxf(0.f, fmaxf(sb[2] - wbox[5], wbox[2] - sb[5])) : 0.f;
                if (g0 * g0 + g1 * g1 + g2 * g2 > wbox[6] * wbox[6]) {  // same in every lane of the warp
                    k += 31;
                    continue;
                }
            }
            const vec4<T> q = sq[k];
            const T dx = p.x - q.x, dy = p.y - q.y, dz = (D == 3) ? p.z - q.z : T(0);
            const T d2 = dx * dx + dy * dy + dz * dz;
            const T eta = sqrt(d2);
            const vec4<T> nn = sn[k];
            if constexpr (PHI == SD_PHI_RADIAL) {
                const T x = eta * inv_r - T(1);
                const T f = pref * exp(-x * x * inv_2s2) * (dx * nn.x + dy * nn.y + dz * nn.z) * recip(eta) * nn.w;
                if (xi > T(0)) kahan_add(sr, cr, a.lam1 * f);
                else kahan_add(si, ci, a.lam2 * f);
                continue;
            }
            const T rm1 = eta * inv_xabs - T(1);
            if (PHI == SD_PHI_SDF && a.eps >= T(0) && rm1 > a.eps) continue;
            const T E = PHI == SD_PHI_SDF ? exp(-rm1 * rm1 * inv_2s2) : T(1);
            const T cos_t = (dx * nn.x + dy * nn.y + dz * nn.z) * recip(eta);
            // zeta^-2 = (xi - i eta)^2 / (xi^2 + eta^2)^2
            const T den = xi2 + d2;
            const T inv_den2 = recip(den * den);
            const T zr = (xi2 - d2) * inv_den2;
            const T zi = T(-2) * xi * eta * inv_den2;
            T f = pref * E * cos_t * nn.w;
            if (D == 2) f *= T(2) * eta;  // planar angle measure
            kahan_add(sr, cr, f * zr);
            kahan_add(si, ci, f * zi);
        }
    }
    if (!live) return;
    part[(int64_t)blockIdx.y * a.m + i] = mk(sr, si);
}

// rho of each query: the partial sums added in split order (compensated), then
// the shape's sample c = rho v and position.
template <typename T>
__global__ void k_sdf_sum_finish(SdfArgs<T> a, int splits, const cplx<T>* part) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    T sr = 0, cr = 0, si = 0, ci = 0;
    for (int k = 0; k < splits; ++k) {
        const cplx<T> v = part[(int64_t)k * a.m + i];
        kahan_add(sr, cr, v.x);
        kahan_add(si, ci, v.y);
    }
    const int64_t src = a.perm_q ? (int64_t)a.perm_q[i] : i;
    const T v = a.vol[src];
    a.c_out[i] = mk(sr * v, si * v);
    if (a.rho_out) a.rho_out[src] = mk(sr, si);
    vec4<T> po = a.qry[src];
    po.w = T(0);
    a.pos_out[i] = po;
}

template <typename T>
__global__ void k_boundary_order(const vec4<T>* bnd, const vec4<T>* nrm, const T* area, const int32_t* perm,
                                 int64_t n_b, int dim, vec4<T>* bnd_s, vec4<T>* nrm_s, float* tile_box,
                                 float* sub_box) {
    __shared__ float wred[SDF_TILE / 32][6];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float v[6] = {FLT_MAX, FLT_MAX, FLT_MAX, -FLT_MAX, -FLT_MAX, -FLT_MAX};
    if (i < n_b) {
        const int32_t j = perm[i];
        const vec4<T> q = bnd[j];
        vec4<T> nn = nrm[j];
        nn.w = area[j];
        bnd_s[i] = q;
        nrm_s[i] = nn;
        v[0] = v[3] = (float)q.x;
        v[1] = v[4] = (float)q.y;
        v[2] = v[5] = (dim == 3) ? (float)q.z : 0.f;
    }
    for (int off = 16; off > 0; off >>= 1) {
        for (int d = 0; d < 3; ++d) v[d] = fminf(v[d], __shfl_down_sync(0xffffffffu, v[d], off));
        for (int d = 3; d < 6; ++d) v[d] = fmaxf(v[d], __shfl_down_sync(0xffffffffu, v[d], off));
    }
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < 6; ++d) wred[threadIdx.x >> 5][d] = v[d];
        // the box of this warp's 32 samples (a sub-tile), widened like the tile's
        float* sb = sub_box + ((int64_t)blockIdx.x * (SDF_TILE / 32) + (threadIdx.x >> 5)) * 6;
        for (int d = 0; d < 6; ++d) {
            const float m = 1e-6f * (fabsf(v[d]) + 1.f);
            sb[d] = v[d] == FLT_MAX || v[d] == -FLT_MAX ? v[d] : (d < 3 ? v[d] - m : v[d] + m);
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float r = wred[0][threadIdx.x];
        for (int w = 1; w < SDF_TILE / 32; ++w)
            r = threadIdx.x < 3 ? fminf(r, wred[w][threadIdx.x]) : fmaxf(r, wred[w][threadIdx.x]);
        // widen by a float ulp-scale margin so the tile test stays conservative
        const float m = 1e-6f * (fabsf(r) + 1.f);
        tile_box[blockIdx.x * 6 + threadIdx.x] = threadIdx.x < 3 ? r - m : r + m;
    }
}

template <typename T>
cudaError_t launch_boundary_order(const vec4<T>* bnd, const vec4<T>* nrm, const T* area, const int32_t* perm,
                                  int64_t n_b, int dim, vec4<T>* bnd_s, vec4<T>* nrm_s, float* tile_box,
                                  cudaStream_t st) {
    if (n_b == 0) return cudaSuccess;
    const int64_t n_tiles = (n_b + SDF_TILE - 1) / SDF_TILE;
    k_boundary_order<T><<<(unsigned)n_tiles, SDF_TILE, 0, st>>>(bnd, nrm, area, perm, n_b, dim, bnd_s, nrm_s, tile_box,
                                                                tile_box + n_tiles * 6);
    note_launch();
    return cudaGetLastError();
}

// Skin / core layers of the signed distance (no boundary sum):
// rho = lambda1 g(xi / R - 1) + i lambda2 g(xi / R + 1), g the normalised Gaussian
// of width sigma.
template <typename T>
__global__ void __launch_bounds__(SDF_TILE) k_sdf_skin(SdfArgs<T> a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    const int64_t src = a.perm_q ? (int64_t)a.perm_q[i] : i;
    const vec4<T> p = a.qry[src];
    const T xi = a.pmc[i] < 0 ? -a.xi_abs[i] : a.xi_abs[i];
    const T inv_r = recip(a.radius);
    const T inv_2s2 = recip(T(2) * a.sigma * a.sigma);
    const T norm = T(1) / (sqrt(T(2.0 * M_PI)) * a.sigma);
    const T xo = xi * inv_r - T(1), xc = xi * inv_r + T(1);
    const T sr = a.lam1 * norm * exp(-xo * xo * inv_2s2);
    const T si = a.lam2 * norm * exp(-xc * xc * inv_2s2);
    const T v = a.vol[src];
    a.c_out[i] = mk(sr * v, si * v);
    if (a.rho_out) a.rho_out[src] = mk(sr, si);
    vec4<T> po = p;
    po.w = T(0);
    a.pos_out[i] = po;
}

// Boundary-tile splits per query block: enough CTAs for about four per SM.
static int sdf_splits(int64_t query_blocks, int64_t tiles) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int64_t s = (4 * (int64_t)sms + query_blocks - 1) / query_blocks;
    s = s < 1 ? 1 : (s > tiles ? tiles : s);
    return (int)(s > 64 ? 64 : s);
}

template <typename T>
cudaError_t launch_sdf(const SdfArgs<T>& a, int dim, cudaStream_t st) {
    if (a.m == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((a.m + SDF_TILE - 1) / SDF_TILE);
    if (a.phi == SD_PHI_SKIN) {
        // membership and distance only (one split), then the pointwise layers
        const int64_t tiles = (a.n_b + SDF_TILE - 1) / SDF_TILE;
        T *d2 = nullptr, *w = nullptr;
        cudaError_t e = pool_alloc((void**)&d2, (size_t)2 * a.m * sizeof(T), st);
        if (e != cudaSuccess) return e;
        w = d2 + a.m;
        if (dim == 2) k_sdf_nearest<T, 2><<<dim3(nb, 1), SDF_TILE, 0, st>>>(a, (int)tiles, d2, w);
        else k_sdf_nearest<T, 3><<<dim3(nb, 1), SDF_TILE, 0, st>>>(a, (int)tiles, d2, w);
        if (dim == 2) k_sdf_nearest_finish<T, 2><<<nb, SDF_TILE, 0, st>>>(a, 1, d2, w);
        else k_sdf_nearest_finish<T, 3><<<nb, SDF_TILE, 0, st>>>(a, 1, d2, w);
        k_sdf_skin<T><<<nb, SDF_TILE, 0, st>>>(a);
        note_launch(3);
        pool_free(d2, st);
        return cudaGetLastError();
    }
    if (a.phi != SD_PHI_SDF && a.phi != SD_PHI_PROXIMAL && a.phi != SD_PHI_RADIAL) return cudaErrorInvalidValue;
    const int64_t tiles = (a.n_b + SDF_TILE - 1) / SDF_TILE;
    const int splits = sdf_splits(nb, tiles < 1 ? 1 : tiles);
    const int tps = (int)((tiles + splits - 1) / splits);
    // partials: nearest distance and winding sum (2 reals), then rho (one complex), per split and query
    char* scratch = nullptr;
    const size_t real_bytes = (size_t)splits * a.m * sizeof(T);
    cudaError_t e = pool_alloc((void**)&scratch, 2 * real_bytes + (size_t)splits * a.m * sizeof(cplx<T>), st);
    if (e != cudaSuccess) return e;
    T* d2 = reinterpret_cast<T*>(scratch);
    T* w = reinterpret_cast<T*>(scratch + real_bytes);
    cplx<T>* part = reinterpret_cast<cplx<T>*>(scratch + 2 * real_bytes);
    const dim3 grid(nb, splits);
    if (dim == 2) k_sdf_nearest<T, 2><<<grid, SDF_TILE, 0, st>>>(a, tps, d2, w);
    else k_sdf_nearest<T, 3><<<grid, SDF_TILE, 0, st>>>(a, tps, d2, w);
    if (dim == 2) k_sdf_nearest_finish<T, 2><<<nb, SDF_TILE, 0, st>>>(a, splits, d2, w);
    else k_sdf_nearest_finish<T, 3><<<nb, SDF_TILE, 0, st>>>(a, splits, d2, w);
#define SD_SUM(DD, PP) k_sdf_sum<T, DD, PP><<<grid, SDF_TILE, 0, st>>>(a, tps, part)
    switch (a.phi) {
        case SD_PHI_SDF:
            if (dim == 2) SD_SUM(2, SD_PHI_SDF);
            else SD_SUM(3, SD_PHI_SDF);
            break;
        case SD_PHI_PROXIMAL:
            if (dim == 2) SD_SUM(2, SD_PHI_PROXIMAL);
            else SD_SUM(3, SD_PHI_PROXIMAL);
            break;
        default:
            if (dim == 2) SD_SUM(2, SD_PHI_RADIAL);
            else SD_SUM(3, SD_PHI_RADIAL);
            break;
    }
#undef SD_SUM
    k_sdf_sum_finish<T><<<nb, SDF_TILE, 0, st>>>(a, splits, part);
    note_launch(4);
    pool_free(scratch, st);
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
template cudaError_t launch_boundary_order<float>(const vec4<float>*, const vec4<float>*, const float*, const int32_t*,
                                                  int64_t, int, vec4<float>*, vec4<float>*, float*, cudaStream_t);
template cudaError_t launch_boundary_order<double>(const vec4<double>*, const vec4<double>*, const double*,
                                                   const int32_t*, int64_t, int, vec4<double>*, vec4<double>*, float*,
                                                   cudaStream_t);

}  // namespace sd
