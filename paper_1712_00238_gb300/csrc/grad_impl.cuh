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

// The fields of cell i, stored as two planes of cells: plane 0 holds (Phi,
// dPhi/dx), plane 1 (dPhi/dy, dPhi/dz) -- 16 bytes per cell and plane for FP32,
// read with one 16-byte read-only load each.
__device__ __forceinline__ void load_cell(const cplx<float>* G, int64_t cells, int64_t i, cplx<float> f[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(G) + i);
    const float4 b = __ldg(reinterpret_cast<const float4*>(G + 2 * cells) + i);
    f[0] = mk(a.x, a.y);
    f[1] = mk(a.z, a.w);
    f[2] = mk(b.x, b.y);
    f[3] = mk(b.z, b.w);
}
__device__ __forceinline__ void load_cell(const cplx<double>* G, int64_t cells, int64_t i, cplx<double> f[4]) {
    f[0] = G[2 * i];
    f[1] = G[2 * i + 1];
    f[2] = G[2 * cells + 2 * i];
    f[3] = G[2 * cells + 2 * i + 1];
}

// One CTA per (pose, chunk of CHUNK samples).  Each thread stages one sample
// (kernel weights, weight value, rotated position, tap-box origin); the warps
// then take the staged samples round-robin and gather each with their lanes on
// consecutive taps, so a load instruction reads a few rows of adjacent cells
// instead of one cell per sample.  A lane keeps, per sample, the weighted sums
// of the four fields over its taps, applies c and the torque arm R p2 to them,
// and accumulates score, force and torque over its samples; lanes and warps are
// summed in FP64 and added to the pose's accumulators.
// Samples per CTA: as many as fit a 40 KiB stage, at most one per thread.
template <typename T, int D, int W>
__host__ __device__ constexpr int gather_chunk() {
    constexpr int rec = D * W + 7;
    constexpr int fit = (40 * 1024) / (rec * (int)sizeof(T)) / 32 * 32;
    return fit < GA_THREADS ? fit : GA_THREADS;
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(GA_THREADS) k_gather(GatherArgs<T> a) {
    using C = cplx<T>;
    constexpr int TAPS = (D == 3) ? W * W * W : W * W;
    constexpr int ROUNDS = (TAPS + 31) / 32;
    constexpr bool TABLE = ROUNDS <= 8;  // per-lane tap table in registers (else derived per round)
    constexpr int CHUNK = gather_chunk<T, D, W>();
    constexpr int NWARP = GA_THREADS / 32;
    constexpr int REC = D * W + 7;  // weights, c (2), R p2 (3), origin cell (wrapped into [0, n)), spare
    __shared__ T stage[CHUNK * REC];
    __shared__ T Rm[9], tv[3];
    __shared__ double red[NWARP][7];
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
    const int n = a.n, pn = a.pn;
    const int64_t cells = (D == 3) ? (int64_t)pn * pn * pn : (int64_t)pn * pn;
    const int64_t j0 = (int64_t)blockIdx.x * CHUNK;
    const int nj = (int)((a.m2 - j0) < (int64_t)CHUNK ? (a.m2 - j0) : (int64_t)CHUNK);
    // stage: one sample per thread
    if ((int)threadIdx.x < nj) {
        const int64_t j = j0 + threadIdx.x;
        const vec4<T> p = a.p2[j];
        const C c = a.c2[j];
        const T pz = (D == 3) ? p.z : T(0);
        T rp[3];
        rp[0] = Rm[0] * p.x + Rm[1] * p.y + Rm[2] * pz;
        rp[1] = Rm[3] * p.x + Rm[4] * p.y + Rm[5] * pz;
        rp[2] = (D == 3) ? Rm[6] * p.x + Rm[7] * p.y + Rm[8] * pz : T(0);
        T* r = stage + threadIdx.x * REC;
        const T half = T(W) * T(0.5), inv_half = T(2) / T(W);
        int base = 0, mul = 1;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const T g = (rp[d] + tv[d]) * a.inv_h;
            const int u0 = (int)ceil(g - half);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const T zz = (T(u0 + k) - g) * inv_half;
                const T z2 = zz * zz;
                r[d * W + k] = (z2 <= T(1)) ? exp(a.beta * (sqrt(T(1) - z2) - T(1))) : T(0);
            }
            base += wrap_n(u0, n) * mul;  // taps reach index n - 1 + W - 1 < pn: no wrapping per tap
            mul *= pn;
        }
        r[D * W] = c.x;
        r[D * W + 1] = c.y;
        r[D * W + 2] = rp[0];
        r[D * W + 3] = rp[1];
        r[D * W + 4] = rp[2];
        // cell indices below 2^31 (pn <= 528 in 3D) travel as the bits of a T
        int* ri = reinterpret_cast<int*>(r + D * W + 5);
        ri[0] = base;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this lane's tap in each round: offset in the grid and (kx, ky, kz)
    constexpr int NT = TABLE ? ROUNDS : 1;
    int toff[NT];  // grid offsets of taps: below pn^3 < 2^28
    int tk[NT];
    auto tap_of = [&](int q, int& kx, int& ky, int& kz) {
        const int tap = min(q * 32 + lane, TAPS - 1);
        kx = tap % W;
        ky = (tap / W) % W;
        kz = (D == 3) ? tap / (W * W) : 0;
    };
    if constexpr (TABLE) {
#pragma unroll
        for (int q = 0; q < ROUNDS; ++q) {
            int kx, ky, kz;
            tap_of(q, kx, ky, kz);
            toff[q] = kx + pn * (ky + pn * kz);
            tk[q] = kx | (ky << 8) | (kz << 16);
        }
    }
    T acc[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int jj = warp; jj < nj; jj += NWARP) {
        const T* r = stage + jj * REC;
        const int base = reinterpret_cast<const int*>(r + D * W + 5)[0];
        C f0 = mk(T(0), T(0)), f1 = f0, f2 = f0, f3 = f0;
#pragma unroll(TABLE ? ROUNDS : 1)
        for (int q = 0; q < ROUNDS; ++q) {
            if (TAPS % 32 == 0 || q * 32 + lane < TAPS) {
                int kx, ky, kz;
                int off;
                if constexpr (TABLE) {
                    kx = tk[q] & 255;
                    ky = (tk[q] >> 8) & 255;
                    kz = tk[q] >> 16;
                    off = toff[q];
                } else {
                    tap_of(q, kx, ky, kz);
                    off = kx + pn * (ky + pn * kz);
                }
                T wgt = r[kx] * r[W + ky];
                if (D == 3) wgt *= r[2 * W + kz];
                const int cell = base + off;
                C f[4];
                load_cell(a.G, cells, cell, f);
                f0 = cadd(f0, cscale(f[0], wgt));
                f1 = cadd(f1, cscale(f[1], wgt));
                f2 = cadd(f2, cscale(f[2], wgt));
                if (D == 3) f3 = cadd(f3, cscale(f[3], wgt));
            }
        }
        const T cx = r[D * W], cy = r[D * W + 1];
        const T rx = r[D * W + 2], ry = r[D * W + 3], rz = r[D * W + 4];
        const T gx = cx * f1.x - cy * f1.y;
        const T gy = cx * f2.x - cy * f2.y;
        const T gz = (D == 3) ? cx * f3.x - cy * f3.y : T(0);
        acc[0] += cx * f0.x - cy * f0.y;
        acc[1] += gx;
        acc[2] += gy;
        acc[3] += gz;
        acc[4] += ry * gz - rz * gy;
        acc[5] += rz * gx - rx * gz;
        acc[6] += rx * gy - ry * gx;
    }
    double v[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        v[k] = (double)acc[k];
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    }
    if (lane == 0)
        for (int k = 0; k < 7; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x < 7) {
        double s = 0.0;
        for (int w = 0; w < NWARP; ++w) s += red[w][threadIdx.x];
        atomicAdd(a.acc + 8 * (int64_t)pose + threadIdx.x, s);
    }
}

template <typename T>
cudaError_t launch_gather(const GatherArgs<T>& a, int dim, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.acc, 0, sizeof(double) * 8 * (a.P > 0 ? a.P : 1), st);
    if (e != cudaSuccess || a.P == 0 || a.m2 == 0) return e;
    auto grid = [&](int chunk) { return dim3((unsigned)((a.m2 + chunk - 1) / chunk), (unsigned)a.P); };
#define SD_GATHER_CASE(WW)                                                                          \
    case WW:                                                                                        \
        if (dim == 2) k_gather<T, 2, WW><<<grid(gather_chunk<T, 2, WW>()), GA_THREADS, 0, st>>>(a); \
        else k_gather<T, 3, WW><<<grid(gather_chunk<T, 3, WW>()), GA_THREADS, 0, st>>>(a);          \
        note_launch();                                                                              \
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

// q <- exp(theta) (x) q / |.| for a rotation vector theta (left multiplication).
__device__ __forceinline__ void rotate_left(double q[4], const double th[3]) {
    const double a = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
    double o[4] = {q[0], q[1], q[2], q[3]};
    if (a > 0.0) {
        const double c = cos(0.5 * a), s = sin(0.5 * a) / a;
        const double ew = c, ex = s * th[0], ey = s * th[1], ez = s * th[2];
        o[0] = ew * q[0] - ex * q[1] - ey * q[2] - ez * q[3];
        o[1] = ew * q[1] + ex * q[0] + ey * q[3] - ez * q[2];
        o[2] = ew * q[2] - ex * q[3] + ey * q[0] + ez * q[1];
        o[3] = ew * q[3] + ex * q[2] - ey * q[1] + ez * q[0];
    }
    const double n = sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2] + o[3] * o[3]);
    for (int k = 0; k < 4; ++k) q[k] = n > 0.0 ? o[k] / n : o[k];
}

// One update of P poses from the gather's accumulators (score, force
// F = d Re f / dt, torque T = sum (R p2) x g): the score goes to hist (if
// given); unless `last` the pose moves by
//   ascent:    t += lr_t F / max|F|, q += lr_q dq / max|dq| (dq = d Re f / dq), q normalised;
//   CG:        Polak-Ribiere directions (beta clipped at 0) kept per block, t moved
//              lr_t along the translation direction, R rotated lr_q radians about
//              the rotation direction;
//   dynamics:  v <- (1 - gamma) v + h F / m, w <- (1 - gamma) w + h T / I,
//              t += h v, q <- exp(h w) q.
// state (P x 12 doubles): CG (gF, gT, dF, dT) of the previous step; dynamics (v, w).
template <typename T>
__global__ void k_refine_step(const double* acc, T* quats, T* trans, double* state, int64_t P, int dim,
                              RefineParams rp, int first, T* hist, int last) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const double* a = acc + 8 * p;
    if (hist) hist[p] = (T)a[0];
    if (last) return;
    T* qo = quats + 4 * p;
    T* to = trans + 3 * p;
    double q[4] = {qo[0], qo[1], qo[2], qo[3]};
    double t[3] = {to[0], to[1], dim == 3 ? (double)to[2] : 0.0};
    const double F[3] = {a[1], a[2], dim == 3 ? a[3] : 0.0};
    const double Tq[3] = {a[4], a[5], a[6]};
    double* st = state ? state + 12 * p : nullptr;
    if (rp.method == SD_REFINE_ASCENT) {
        const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const double inv = nq > 0 ? 1.0 / nq : 0.0;
        const double u0 = q[0] * inv, ux = q[1] * inv, uy = q[2] * inv, uz = q[3] * inv;
        const double tx = Tq[0], ty = Tq[1], tz = Tq[2];
        const double dq[4] = {2.0 * inv * -(tx * ux + ty * uy + tz * uz), 2.0 * inv * (u0 * tx + (ty * uz - tz * uy)),
                              2.0 * inv * (u0 * ty + (tz * ux - tx * uz)), 2.0 * inv * (u0 * tz + (tx * uy - ty * ux))};
        double sf = 1e-30, sq = 1e-30;
        for (int k = 0; k < 3; ++k) sf = fmax(sf, fabs(F[k]));
        for (int k = 0; k < 4; ++k) sq = fmax(sq, fabs(dq[k]));
        for (int k = 0; k < 3; ++k) t[k] += rp.lr_t * F[k] / sf;
        double qn[4];
        for (int k = 0; k < 4; ++k) qn[k] = q[k] + rp.lr_q * dq[k] / sq;
        const double nn = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
        for (int k = 0; k < 4; ++k) q[k] = nn > 0 ? qn[k] / nn : qn[k];
    } else if (rp.method == SD_REFINE_CG) {
        const double* g[2] = {F, Tq};
        double d[2][3];
        for (int b = 0; b < 2; ++b) {
            double beta = 0.0;
            if (!first) {
                const double* gp = st + 3 * b;
                double num = 0.0, den = 0.0;
                for (int k = 0; k < 3; ++k) {
                    num += g[b][k] * (g[b][k] - gp[k]);
                    den += gp[k] * gp[k];
                }
                beta = den > 0.0 ? fmax(0.0, num / den) : 0.0;
            }
            for (int k = 0; k < 3; ++k) d[b][k] = g[b][k] + (first ? 0.0 : beta * st[6 + 3 * b + k]);
        }
        for (int b = 0; b < 2; ++b)
            for (int k = 0; k < 3; ++k) {
                st[3 * b + k] = g[b][k];
                st[6 + 3 * b + k] = d[b][k];
            }
        const double nt = sqrt(d[0][0] * d[0][0] + d[0][1] * d[0][1] + d[0][2] * d[0][2]);
        const double nr = sqrt(d[1][0] * d[1][0] + d[1][1] * d[1][1] + d[1][2] * d[1][2]);
        if (nt > 0.0)
            for (int k = 0; k < 3; ++k) t[k] += rp.lr_t * d[0][k] / nt;
        if (nr > 0.0) {
            const double th[3] = {rp.lr_q * d[1][0] / nr, rp.lr_q * d[1][1] / nr, rp.lr_q * d[1][2] / nr};
            rotate_left(q, th);
        }
    } else {  // SD_REFINE_DYNAMICS
        double v[3], w[3];
        for (int k = 0; k < 3; ++k) {
            v[k] = (first ? 0.0 : (1.0 - rp.damping) * st[k]) + rp.h * F[k] / rp.mass;
            w[k] = (first ? 0.0 : (1.0 - rp.damping) * st[3 + k]) + rp.h * Tq[k] / rp.inertia;
            st[k] = v[k];
            st[3 + k] = w[k];
            t[k] += rp.h * v[k];
        }
        const double th[3] = {rp.h * w[0], rp.h * w[1], rp.h * w[2]};
        rotate_left(q, th);
    }
    for (int k = 0; k < 4; ++k) qo[k] = (T)q[k];
    to[0] = (T)t[0];
    to[1] = (T)t[1];
    if (dim == 3) to[2] = (T)t[2];
}

template <typename T>
cudaError_t launch_refine_step(const double* acc, T* quats, T* trans, double* state, int64_t P, int dim,
                               const RefineParams& rp, int first, T* hist, int last, cudaStream_t st) {
    if (P == 0) return cudaSuccess;
    k_refine_step<T><<<(unsigned)((P + 127) / 128), 128, 0, st>>>(acc, quats, trans, state, P, dim, rp, first, hist,
                                                                  last);
    note_launch();
    return cudaGetLastError();
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
