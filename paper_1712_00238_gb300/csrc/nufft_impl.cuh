// Type-1 nonuniform FFT of rotated samples and the translation-score passes.
//
// Per rotation (Section 5: one FFT over the translations per rotation; the
// scattered samples go through a nonequispaced FFT with oversampling alpha = 2):
//   spread   c_j at y_j = -R p_j onto the oversampled grid with the
//            exponential-of-semicircle kernel psi(z) = exp(beta (sqrt(1 - z^2) - 1))
//            (Barnett, Magland & af Klinteberg 2019), only inside the sub-box that
//            the rotated shape can reach;
//   x pass   forward FFT of length n on the sub-box rows, keep the N central modes;
//   y pass   the same along y (3D);
//   fused    forward FFT along the last axis, keep N modes, multiply by the fixed
//            shape's table W(kappa), inverse FFT of length N along that axis;
//   y pass   inverse along y (3D);
//   x pass   inverse along x, real part, argmax (or the complex map).
#pragma once

#include <float.h>
#include <limits.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <set>
#include <tuple>

#include "fft.cuh"
#include "kernels.cuh"

namespace sd {

struct CandRec {  // same layout as sd_cand
    double score;
    int32_t rot;
    int32_t idx;
};

template <typename T, int LEN>
__host__ __device__ constexpr int lines_per_cta() {
    return (LEN * (int)sizeof(cplx<T>) > 4096) ? 8 : 16;
}

// ---------------------------------------------------------------------------
// spreading
// ---------------------------------------------------------------------------

__device__ __forceinline__ int wrap_index(int a, int s) {
    a %= s;
    return a < 0 ? a + s : a;
}

// Adds the taps of one sample to the sub-box with global atomics.  Along x the
// six (or W) cells of a row are added two at a time with one 16-byte vector
// atomic on an even-aligned cell pair (the out-of-row half of an edge pair adds
// zero), which cuts the L2 atomic operations of a row from W to about W/2 + 1.
// Rows that wrap around a periodic sub-box use one atomic per cell.
__device__ __forceinline__ void add_pair(float2* cell_even, float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    atomicAdd(reinterpret_cast<float4*>(cell_even), make_float4(a.x, a.y, b.x, b.y));
#else
    atomic_cadd(cell_even, a);
    atomic_cadd(cell_even + 1, b);
#endif
}
__device__ __forceinline__ void add_pair(double2* cell_even, double2 a, double2 b) {
    atomic_cadd(cell_even, a);
    atomic_cadd(cell_even + 1, b);
}

template <typename T, int W>
__device__ __forceinline__ void spread_row(cplx<T>* row, int s, int ax0, bool wraps, cplx<T> cy, const T* wx) {
    using C = cplx<T>;
    if (wraps || sizeof(T) == 8) {
#pragma unroll
        for (int kx = 0; kx < W; ++kx) atomic_cadd(row + wrap_index(ax0 + kx, s), cscale(cy, wx[kx]));
        return;
    }
    const C zero = mk(T(0), T(0));
    if ((ax0 & 1) == 0) {
#pragma unroll
        for (int kx = 0; kx < W; kx += 2)
            add_pair(row + ax0 + kx, cscale(cy, wx[kx]), kx + 1 < W ? cscale(cy, wx[kx + 1]) : zero);
    } else {
        add_pair(row + ax0 - 1, zero, cscale(cy, wx[0]));
#pragma unroll
        for (int kx = 1; kx < W; kx += 2)
            add_pair(row + ax0 + kx, cscale(cy, wx[kx]), kx + 1 < W ? cscale(cy, wx[kx + 1]) : zero);
    }
}

template <typename T, int D, int W>
__device__ __forceinline__ void spread_direct(cplx<T>* out, int s, int s_h, const int* u0, const T (*wt)[W],
                                              cplx<T> c) {
    using C = cplx<T>;
    int ax0 = u0[0] + s_h;
    const bool wraps = (ax0 < 0) || (ax0 + W > s);
    ax0 = wrap_index(ax0, s);
    int iy[W];
#pragma unroll
    for (int k = 0; k < W; ++k) iy[k] = wrap_index(u0[1] + k + s_h, s);
    if constexpr (D == 2) {
#pragma unroll
        for (int ky = 0; ky < W; ++ky)
            spread_row<T, W>(out + (int64_t)iy[ky] * s, s, ax0, wraps, cscale(c, wt[1][ky]), wt[0]);
    } else {
#pragma unroll 1
        for (int kz = 0; kz < W; ++kz) {
            const C cz = cscale(c, wt[2][kz]);
            C* plane = out + (int64_t)wrap_index(u0[2] + kz + s_h, s) * s * s;
#pragma unroll
            for (int ky = 0; ky < W; ++ky)
                spread_row<T, W>(plane + (int64_t)iy[ky] * s, s, ax0, wraps, cscale(cz, wt[1][ky]), wt[0]);
        }
    }
}

// One CTA spreads 256 consecutive samples.  Because the samples are stored in
// Morton order, their taps after rotation usually fit a small box: the CTA
// accumulates them there in shared memory (shared atomics) and then adds the
// box's non-zero cells to the sub-box in global memory, one vector atomic per
// cell instead of one per tap.  A box larger than `cap_cells` (or cap_cells = 0)
// falls back to one global atomic per tap.
template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_spread(SpreadArgs<T> a, int cap_cells) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);  // cap_cells x (re, im)
    __shared__ T Rm[9];
    __shared__ int wlo[8][3], whi[8][3];
    __shared__ int box_lo[3], box_ext[3];
    const int b = blockIdx.y;
    if (threadIdx.x == 0) {
        if (a.quats) {
            quat_to_matrix<T>(a.quats + 4 * (a.rot0 + b), Rm);
        } else {
            for (int i = 0; i < 9; ++i) Rm[i] = (i % 4 == 0) ? T(1) : T(0);
        }
    }
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = j < a.m;
    T wt[D][W];
    int u0[D];
    C c = mk(T(0), T(0));
    if (live) {
        const vec4<T> p = a.pos[j];
        c = a.c[j];
        T y[3];
        y[0] = a.sign * (Rm[0] * p.x + Rm[1] * p.y + Rm[2] * p.z);
        y[1] = a.sign * (Rm[3] * p.x + Rm[4] * p.y + Rm[5] * p.z);
        y[2] = a.sign * (Rm[6] * p.x + Rm[7] * p.y + Rm[8] * p.z);
        const T half = T(W) * T(0.5);
        const T inv_half = T(2) / T(W);
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const T g = y[d] * a.inv_h;
            u0[d] = (int)ceil(g - half);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const T z = (T(u0[d] + k) - g) * inv_half;
                const T z2 = z * z;
                wt[d][k] = (z2 <= T(1)) ? exp(a.beta * (sqrt(T(1) - z2) - T(1))) : T(0);
            }
        }
    } else {
#pragma unroll
        for (int d = 0; d < D; ++d) u0[d] = 0;
    }
    // bounding box of the taps of this CTA (unwrapped grid indices)
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (live)
#pragma unroll
        for (int d = 0; d < D; ++d) {
            lo[d] = u0[d];
            hi[d] = u0[d] + W - 1;
        }
#pragma unroll
    for (int d = 0; d < D; ++d)
        for (int off = 16; off > 0; off >>= 1) {
            lo[d] = min(lo[d], __shfl_down_sync(0xffffffffu, lo[d], off));
            hi[d] = max(hi[d], __shfl_down_sync(0xffffffffu, hi[d], off));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) {
            wlo[warp][d] = lo[d];
            whi[warp][d] = hi[d];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) {
            int l = INT_MAX, h = INT_MIN;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                l = min(l, wlo[w][d]);
                h = max(h, whi[w][d]);
            }
            box_lo[d] = l;
            box_ext[d] = (d < D && h >= l) ? h - l + 1 : 1;
        }
    }
    __syncthreads();
    const int ex = box_ext[0], ey = box_ext[1], ez = box_ext[2];
    const int64_t cells = (int64_t)ex * ey * (D == 3 ? ez : 1);
    C* out = a.out + (int64_t)b * a.out_rot_stride;
    const int s = a.s;
    if (cells <= cap_cells) {
        for (int i = threadIdx.x; i < 2 * cells; i += blockDim.x) tile[i] = T(0);
        __syncthreads();
        if (live) {
            const int lx = u0[0] - box_lo[0], ly = u0[1] - box_lo[1], lz = (D == 3) ? u0[2] - box_lo[2] : 0;
#pragma unroll 1
            for (int kz = 0; kz < (D == 3 ? W : 1); ++kz) {
                const C cz = (D == 3) ? cscale(c, wt[D == 3 ? 2 : 0][kz]) : c;
#pragma unroll
                for (int ky = 0; ky < W; ++ky) {
                    const C cy = cscale(cz, wt[1][ky]);
                    T* row = tile + 2 * (((int64_t)(lz + kz) * ey + (ly + ky)) * ex + lx);
#pragma unroll
                    for (int kx = 0; kx < W; ++kx) {
                        atomicAdd(row + 2 * kx, cy.x * wt[0][kx]);
                        atomicAdd(row + 2 * kx + 1, cy.y * wt[0][kx]);
                    }
                }
            }
        }
        __syncthreads();
        for (int64_t li = threadIdx.x; li < cells; li += blockDim.x) {
            const C v = mk(tile[2 * li], tile[2 * li + 1]);
            if (v.x == T(0) && v.y == T(0)) continue;
            const int64_t q = li / ex;
            const int cx = (int)(li - q * ex);
            const int cy = (int)(q % ey);
            const int cz = (int)(q / ey);
            const int ax = wrap_index(box_lo[0] + cx + a.s_h, s);
            const int ay = wrap_index(box_lo[1] + cy + a.s_h, s);
            int64_t off = (int64_t)ay * s + ax;
            if (D == 3) off += (int64_t)wrap_index(box_lo[2] + cz + a.s_h, s) * s * s;
            atomic_cadd(out + off, v);
        }
        return;
    }
    if (!live) return;
    spread_direct<T, D, W>(a.out + (int64_t)b * a.out_rot_stride, s, a.s_h, u0, wt, c);
}

// ---------------------------------------------------------------------------
// spreading by bins (no global atomics, no clearing pass)
// ---------------------------------------------------------------------------
//
// The sub-box is cut into bins of SPREAD_BIN^d cells.  A sample belongs to the
// bin that holds the first cell of its tap box.  Since W - 1 < SPREAD_BIN, the
// taps of a sample only reach its own bin and the next one along each axis, so
// the tile of bin t receives taps only from samples of bins t - {0,1}^d.  One CTA
// per tile gathers those samples, accumulates the taps that fall in its tile in
// shared memory and stores the whole tile (zeros included) once.

constexpr int SPREAD_BIN = 8;

// Tap-box origin (sub-box coordinates, wrapped when the sub-box is the whole
// periodic grid) and kernel weights of sample j under rotation Rm.
template <typename T, int D, int W>
__device__ __forceinline__ void sample_taps(const SpreadArgs<T>& a, const T* Rm, int64_t j, int org[D], T wt[D][W],
                                            cplx<T>& c) {
    const vec4<T> p = a.pos[j];
    c = a.c[j];
    T y[3];
    y[0] = a.sign * (Rm[0] * p.x + Rm[1] * p.y + Rm[2] * p.z);
    y[1] = a.sign * (Rm[3] * p.x + Rm[4] * p.y + Rm[5] * p.z);
    y[2] = a.sign * (Rm[6] * p.x + Rm[7] * p.y + Rm[8] * p.z);
    const T half = T(W) * T(0.5);
    const T inv_half = T(2) / T(W);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const T g = y[d] * a.inv_h;
        const int u0 = (int)ceil(g - half);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const T z = (T(u0 + k) - g) * inv_half;
            const T z2 = z * z;
            wt[d][k] = (z2 <= T(1)) ? exp(a.beta * (sqrt(T(1) - z2) - T(1))) : T(0);
        }
        org[d] = wrap_index(u0 + a.s_h, a.s);
    }
}

template <typename T>
__device__ __forceinline__ void load_rotation(const SpreadArgs<T>& a, int b, T* Rm) {
    if (a.quats) {
        quat_to_matrix<T>(a.quats + 4 * (a.rot0 + b), Rm);
    } else {
        for (int i = 0; i < 9; ++i) Rm[i] = (i % 4 == 0) ? T(1) : T(0);
    }
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_bin_count(SpreadArgs<T> a, BinArgs bn) {
    __shared__ T Rm[9];
    const int b = blockIdx.y;
    if (threadIdx.x == 0) load_rotation(a, b, Rm);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.m) return;
    int org[D];
    T wt[D][W];
    cplx<T> c;
    sample_taps<T, D, W>(a, Rm, j, org, wt, c);
    int bin = 0;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) bin = bin * bn.nb + org[d] / SPREAD_BIN;
    const int64_t o = (int64_t)b * a.m + j;
    bn.bin_of[o] = bin;
    bn.rank[o] = atomicAdd(bn.count + (int64_t)b * bn.nbins + bin, 1);
}

// Exclusive scan of the bin counts of one rotation (one CTA of 1024 threads).
static __global__ void __launch_bounds__(1024) k_bin_scan(BinArgs bn) {
    __shared__ int wsum[32];
    const int b = blockIdx.x;
    const int* cnt = bn.count + (int64_t)b * bn.nbins;
    int* off = bn.offset + (int64_t)b * (bn.nbins + 1);
    const int per = (bn.nbins + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per;
    const int hi = min(bn.nbins, lo + per);
    int local = 0;
    for (int i = lo; i < hi; ++i) local += cnt[i];
    // block exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += v;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int run = incl - local + (warp > 0 ? wsum[warp - 1] : 0);
    for (int i = lo; i < hi; ++i) {
        off[i] = run;
        run += cnt[i];
    }
    if (threadIdx.x == blockDim.x - 1) off[bn.nbins] = run;
}

template <typename T>
__global__ void __launch_bounds__(256) k_bin_scatter(int64_t m, BinArgs bn) {
    const int b = blockIdx.y;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t o = (int64_t)b * m + j;
    const int pos = bn.offset[(int64_t)b * (bn.nbins + 1) + bn.bin_of[o]] + bn.rank[o];
    bn.sorted[(int64_t)b * m + pos] = (int32_t)j;
}

// One CTA per bin: its samples' taps all fall in the bin grown by W - 1 cells,
// accumulated in shared memory (every sample once, taps unrolled), then added to
// the sub-box with one vector atomic per non-zero cell.
template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_spread_tiles(SpreadArgs<T> a, BinArgs bn) {
    using C = cplx<T>;
    constexpr int PS = SPREAD_BIN + W - 1;
    constexpr int CELLS = (D == 3) ? PS * PS * PS : PS * PS;
    __shared__ T tile[2 * CELLS];
    __shared__ T Rm[9];
    const int b = blockIdx.y;
    const int t = blockIdx.x;
    const int* off = bn.offset + (int64_t)b * (bn.nbins + 1);
    const int lo = off[t], hi = off[t + 1];
    if (lo == hi) return;  // empty bin (uniform over the block)
    for (int i = threadIdx.x; i < 2 * CELLS; i += blockDim.x) tile[i] = T(0);
    if (threadIdx.x == 0) load_rotation(a, b, Rm);
    __syncthreads();
    const int nb = bn.nb, s = a.s;
    const int org0[3] = {(t % nb) * SPREAD_BIN, ((t / nb) % nb) * SPREAD_BIN,
                         (D == 3) ? (t / (nb * nb)) * SPREAD_BIN : 0};
    const int32_t* sorted = bn.sorted + (int64_t)b * a.m;
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) {
        int org[D];
        T wt[D][W];
        C c;
        sample_taps<T, D, W>(a, Rm, sorted[p], org, wt, c);
        const int lx = org[0] - org0[0], ly = org[1] - org0[1], lz = (D == 3) ? org[2] - org0[2] : 0;
#pragma unroll 1
        for (int kz = 0; kz < (D == 3 ? W : 1); ++kz) {
            const C cz = (D == 3) ? cscale(c, wt[D == 3 ? 2 : 0][kz]) : c;
#pragma unroll
            for (int ky = 0; ky < W; ++ky) {
                const C cy = cscale(cz, wt[1][ky]);
                T* row = tile + 2 * (((lz + kz) * PS + (ly + ky)) * PS + lx);
#pragma unroll
                for (int kx = 0; kx < W; ++kx) {
                    atomicAdd(row + 2 * kx, cy.x * wt[0][kx]);
                    atomicAdd(row + 2 * kx + 1, cy.y * wt[0][kx]);
                }
            }
        }
    }
    __syncthreads();
    C* out = a.out + (int64_t)b * a.out_rot_stride;
    for (int li = threadIdx.x; li < CELLS; li += blockDim.x) {
        const C v = mk(tile[2 * li], tile[2 * li + 1]);
        if (v.x == T(0) && v.y == T(0)) continue;
        const int x = li % PS, y = (li / PS) % PS, z = li / (PS * PS);
        int64_t o = (int64_t)wrap_index(org0[1] + y, s) * s + wrap_index(org0[0] + x, s);
        if (D == 3) o += (int64_t)wrap_index(org0[2] + z, s) * s * s;
        atomic_cadd(out + o, v);
    }
}

// ---------------------------------------------------------------------------
// row passes (lines contiguous in memory)
// ---------------------------------------------------------------------------

template <typename T, int LEN, int MODE>
__global__ void __launch_bounds__(256) k_rows(RowArgs<T> a) {
    using C = cplx<T>;
    constexpr int TR = lines_per_cta<T, LEN>();
    constexpr int LD = line_pitch(LEN);
    constexpr int NTW = tw_count(LEN);
    constexpr bool INV = (MODE != ROW_FWD);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + TR * LD;
    const int b = blockIdx.y;
    const int row0 = blockIdx.x * TR;
    for (int j = threadIdx.x; j < NTW; j += blockDim.x) tw[j] = a.tw[j];
    const C* in = a.in + (int64_t)b * a.in_rot_stride;
    const C zero = mk(T(0), T(0));
    for (int idx = threadIdx.x; idx < TR * LEN; idx += blockDim.x) {
        const int r = idx / LEN;
        const int pos = idx - r * LEN;
        const int row = row0 + r;
        C v = zero;
        if (row < a.nrows) {
            const C* src = in + (int64_t)row * a.in_row_stride;
            if constexpr (MODE == ROW_FWD) {
                int e = pos + a.s_h;
                if (e >= LEN) e -= LEN;
                if (e < a.len_in) v = src[e];
            } else if constexpr (MODE == ROW_EXPAND) {
                const int hN = a.N >> 1;
                const int e = pos < hN ? pos : (pos >= LEN - hN ? pos - LEN + a.N : -1);
                if (e >= 0) v = src[e];
            } else {
                v = src[pos];
            }
        }
        buf[r * LD + pad(pos)] = v;
    }
    __syncthreads();
    fft_inplace<C, LEN, INV, TR>(buf, LD, tw);
    const C* res = buf;
    C* out = a.out + (int64_t)b * a.out_rot_stride;
    if constexpr (MODE == ROW_FWD) {
        const int N = a.N, hN = N >> 1;
        for (int idx = threadIdx.x; idx < TR * N; idx += blockDim.x) {
            const int r = idx / N;
            const int kp = idx - r * N;
            const int row = row0 + r;
            if (row < a.nrows) {
                const int pos = kp < hN ? kp : kp - N + LEN;
                out[(int64_t)row * a.out_row_stride + kp] = res[r * LD + pad(pos)];
            }
        }
    } else if constexpr (MODE == ROW_INV_MAP || MODE == ROW_EXPAND) {
        for (int idx = threadIdx.x; idx < TR * LEN; idx += blockDim.x) {
            const int r = idx / LEN;
            const int e = idx - r * LEN;
            const int row = row0 + r;
            if (row < a.nrows) out[(int64_t)row * a.out_row_stride + e] = res[r * LD + pad(e)];
        }
    } else {  // ROW_INV_ARGMAX: best (max Re, lowest index) of this tile
        T best = -INFINITY;
        int bidx = INT_MAX;
        for (int idx = threadIdx.x; idx < TR * LEN; idx += blockDim.x) {
            const int r = idx / LEN;
            const int e = idx - r * LEN;
            const int row = row0 + r;
            if (row < a.nrows) {
                const T v = res[r * LD + pad(e)].x;
                const int gi = row * LEN + e;
                if (v > best || (v == best && gi < bidx)) {
                    best = v;
                    bidx = gi;
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const T ob = __shfl_down_sync(0xffffffffu, best, off);
            const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
            if (ob > best || (ob == best && oi < bidx)) {
                best = ob;
                bidx = oi;
            }
        }
        __shared__ T wb[32];
        __shared__ int wi[32];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) {
            wb[warp] = best;
            wi[warp] = bidx;
        }
        __syncthreads();
        if (warp == 0) {
            const int nw = (blockDim.x + 31) >> 5;
            best = lane < nw ? wb[lane] : T(-INFINITY);
            bidx = lane < nw ? wi[lane] : INT_MAX;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ob = __shfl_down_sync(0xffffffffu, best, off);
                const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
                if (ob > best || (ob == best && oi < bidx)) {
                    best = ob;
                    bidx = oi;
                }
            }
            if (lane == 0) {
                const int64_t o = (int64_t)b * gridDim.x + blockIdx.x;
                a.part_score[o] = (double)best;
                a.part_idx[o] = bidx;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// column passes (lines strided; a CTA takes TC adjacent columns)
// ---------------------------------------------------------------------------

template <typename T, int LENF, int LENI, int MODE>
__global__ void __launch_bounds__(256) k_cols(ColArgs<T> a) {
    using C = cplx<T>;
    constexpr int TC = lines_per_cta<T, LENF>();
    constexpr int LD = line_pitch(LENF);
    constexpr int NTWF = tw_count(LENF);
    constexpr int NTWI = (MODE == COL_FUSED) ? tw_count(LENI) : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* twF = buf + TC * LD;
    C* twI = twF + NTWF;
    const int b = blockIdx.z;
    const int outer = blockIdx.y;
    const int col0 = blockIdx.x * TC;
    for (int j = threadIdx.x; j < NTWF; j += blockDim.x) twF[j] = a.twF[j];
    if constexpr (MODE == COL_FUSED)
        for (int j = threadIdx.x; j < NTWI; j += blockDim.x) twI[j] = a.twI[j];
    const int ncols = a.ncols;
    const C* in = a.in + (int64_t)b * a.in_rot_stride + (int64_t)outer * a.in_outer_stride;
    C* out = a.out + (int64_t)b * a.out_rot_stride + (int64_t)outer * a.out_outer_stride;
    const C zero = mk(T(0), T(0));
    const int hN = a.N >> 1;
    for (int idx = threadIdx.x; idx < TC * LENF; idx += blockDim.x) {
        const int col = idx % TC;
        const int pos = idx / TC;
        const int gcol = col0 + col;
        int e;
        if constexpr (MODE == COL_FWD || MODE == COL_FUSED) {
            e = pos + a.s_h;
            if (e >= LENF) e -= LENF;
            if (e >= a.len_in) e = -1;
        } else if constexpr (MODE == COL_EXPAND) {
            e = pos < hN ? pos : (pos >= LENF - hN ? pos - LENF + a.N : -1);
        } else {
            e = pos;
        }
        C v = zero;
        if (e >= 0 && gcol < ncols) v = in[(int64_t)e * ncols + gcol];
        buf[col * LD + pad(pos)] = v;
    }
    __syncthreads();
    constexpr bool INV1 = (MODE == COL_INV || MODE == COL_EXPAND);
    fft_inplace<C, LENF, INV1, TC>(buf, LD, twF);
    C* res = buf;
    if constexpr (MODE == COL_FWD) {
        for (int idx = threadIdx.x; idx < TC * a.N; idx += blockDim.x) {
            const int col = idx % TC;
            const int kp = idx / TC;
            const int gcol = col0 + col;
            if (gcol < ncols) {
                const int pos = kp < hN ? kp : kp - a.N + LENF;
                out[(int64_t)kp * ncols + gcol] = res[col * LD + pad(pos)];
            }
        }
    } else if constexpr (MODE == COL_INV || MODE == COL_EXPAND) {
        for (int idx = threadIdx.x; idx < TC * LENF; idx += blockDim.x) {
            const int col = idx % TC;
            const int e = idx / TC;
            const int gcol = col0 + col;
            if (gcol < ncols) out[(int64_t)e * ncols + gcol] = res[col * LD + pad(e)];
        }
    } else {  // COL_FUSED: keep N modes, multiply by W, inverse of length N (in place)
        constexpr int PERX = (TC * LENI + FFT_THREADS - 1) / FFT_THREADS;
        C v[PERX];
#pragma unroll
        for (int q = 0; q < PERX; ++q) {
            const int idx = threadIdx.x + q * FFT_THREADS;
            v[q] = zero;
            if (idx < TC * LENI) {
                const int col = idx % TC;
                const int kp = idx / TC;
                const int gcol = col0 + col;
                if (gcol < ncols) {
                    const int pos = kp < hN ? kp : kp - LENI + LENF;
                    v[q] = cmul(res[col * LD + pad(pos)], a.W[(int64_t)kp * ncols + gcol]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PERX; ++q) {
            const int idx = threadIdx.x + q * FFT_THREADS;
            if (idx < TC * LENI) buf[(idx % TC) * LD + pad(idx / TC)] = v[q];
        }
        __syncthreads();
        fft_inplace<C, LENI, true, TC>(buf, LD, twI);
        for (int idx = threadIdx.x; idx < TC * LENI; idx += blockDim.x) {
            const int col = idx % TC;
            const int e = idx / TC;
            const int gcol = col0 + col;
            if (gcol < ncols) out[(int64_t)e * ncols + gcol] = buf[col * LD + pad(e)];
        }
    }
}

// ---------------------------------------------------------------------------
// pipelined passes: persistent CTAs that double-buffer their input tiles with
// asynchronous 16-byte copies (cp.async), so the next tile streams in while the
// current one is transformed
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Row passes.  Tile = TR consecutive rows of one rotation; rows are contiguous
// (in_row_stride == len_in), so a tile is one contiguous run of TR*len_in
// elements.  Stage layout: [row][e], dense.
template <typename T, int LEN, int MODE>
__global__ void __launch_bounds__(256) k_rows_p(RowArgs<T> a, int tiles_per_rot, int total_tiles) {
    using C = cplx<T>;
    constexpr int TR = lines_per_cta<T, LEN>();
    constexpr int LD = line_pitch(LEN);
    constexpr int NTW = tw_count(LEN);
    constexpr bool INV = (MODE != ROW_FWD);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + TR * LD;
    C* stage = tw + ((NTW + 1) & ~1);  // 16-byte aligned
    const int stage_elems = TR * a.len_in;
    for (int j = threadIdx.x; j < NTW; j += blockDim.x) tw[j] = a.tw[j];
    constexpr int EPC = 16 / (int)sizeof(C);  // elements per 16-byte chunk

    auto issue = [&](int t, int slot) {
        const int b = t / tiles_per_rot;
        const int row0 = (t - b * tiles_per_rot) * TR;
        const int rows = min(TR, a.nrows - row0);
        const C* src = a.in + (int64_t)b * a.in_rot_stride + (int64_t)row0 * a.len_in;
        C* dst = stage + slot * stage_elems;
        const int chunks = rows * a.len_in / EPC;
        for (int q = threadIdx.x; q < chunks; q += blockDim.x) cp_async16(dst + q * EPC, src + q * EPC);
    };

    int t = blockIdx.x;
    if (t < total_tiles) issue(t, 0);
    cp_async_commit();
    for (int it = 0; t < total_tiles; ++it) {
        const int tn = t + gridDim.x;
        if (tn < total_tiles) issue(tn, (it + 1) & 1);
        cp_async_commit();
        cp_async_wait_1();
        __syncthreads();
        const int b = t / tiles_per_rot;
        const int tl = t - b * tiles_per_rot;
        const int row0 = tl * TR;
        const C* st = stage + (it & 1) * stage_elems;
        const C zero = mk(T(0), T(0));
        for (int idx = threadIdx.x; idx < TR * LEN; idx += blockDim.x) {
            const int r = idx / LEN;
            const int pos = idx - r * LEN;
            C v = zero;
            if (row0 + r < a.nrows) {
                const C* src = st + r * a.len_in;
                if constexpr (MODE == ROW_FWD) {
                    int e = pos + a.s_h;
                    if (e >= LEN) e -= LEN;
                    if (e < a.len_in) v = src[e];
                } else if constexpr (MODE == ROW_EXPAND) {
                    const int hN = a.N >> 1;
                    const int e = pos < hN ? pos : (pos >= LEN - hN ? pos - LEN + a.N : -1);
                    if (e >= 0) v = src[e];
                } else {
                    v = src[pos];
                }
            }
            buf[r * LD + pad(pos)] = v;
        }
        __syncthreads();
        fft_inplace<C, LEN, INV, TR>(buf, LD, tw);
        C* out = a.out + (int64_t)b * a.out_rot_stride;
        if constexpr (MODE == ROW_FWD) {
            const int N = a.N, hN = N >> 1;
            for (int idx = threadIdx.x; idx < TR * N; idx += blockDim.x) {
                const int r = idx / N;
                const int kp = idx - r * N;
                const int row = row0 + r;
                if (row < a.nrows) {
                    const int pos = kp < hN ? kp : kp - N + LEN;
                    out[(int64_t)row * a.out_row_stride + kp] = buf[r * LD + pad(pos)];
                }
            }
        } else if constexpr (MODE == ROW_INV_MAP || MODE == ROW_EXPAND) {
            for (int idx = threadIdx.x; idx < TR * LEN; idx += blockDim.x) {
                const int r = idx / LEN;
                const int e = idx - r * LEN;
                const int row = row0 + r;
                if (row < a.nrows) out[(int64_t)row * a.out_row_stride + e] = buf[r * LD + pad(e)];
            }
        } else {  // ROW_INV_ARGMAX
            T best = -INFINITY;
            int bidx = INT_MAX;
            for (int idx = threadIdx.x; idx < TR * LEN; idx += blockDim.x) {
                const int r = idx / LEN;
                const int e = idx - r * LEN;
                const int row = row0 + r;
                if (row < a.nrows) {
                    const T v = buf[r * LD + pad(e)].x;
                    const int gi = row * LEN + e;
                    if (v > best || (v == best && gi < bidx)) {
                        best = v;
                        bidx = gi;
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ob = __shfl_down_sync(0xffffffffu, best, off);
                const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
                if (ob > best || (ob == best && oi < bidx)) {
                    best = ob;
                    bidx = oi;
                }
            }
            __shared__ T wb[32];
            __shared__ int wi[32];
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            if (lane == 0) {
                wb[warp] = best;
                wi[warp] = bidx;
            }
            __syncthreads();
            if (warp == 0) {
                const int nw = (blockDim.x + 31) >> 5;
                best = lane < nw ? wb[lane] : T(-INFINITY);
                bidx = lane < nw ? wi[lane] : INT_MAX;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const T ob = __shfl_down_sync(0xffffffffu, best, off);
                    const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
                    if (ob > best || (ob == best && oi < bidx)) {
                        best = ob;
                        bidx = oi;
                    }
                }
                if (lane == 0) {
                    const int64_t o = (int64_t)b * tiles_per_rot + tl;
                    a.part_score[o] = (double)best;
                    a.part_idx[o] = bidx;
                }
            }
        }
        __syncthreads();  // buf and this stage slot are reused by the next tile
        t = tn;
    }
}

// Column passes.  Tile = TC adjacent columns of one (rotation, outer) slab; each
// line element row of the tile is TC contiguous elements.  Stage layout: [e][col].
template <typename T, int LENF, int LENI, int MODE>
__global__ void __launch_bounds__(256) k_cols_p(ColArgs<T> a, int col_tiles, int total_tiles) {
    using C = cplx<T>;
    constexpr int TC = lines_per_cta<T, LENF>();
    constexpr int LD = line_pitch(LENF);
    constexpr int NTWF = tw_count(LENF);
    constexpr int NTWI = (MODE == COL_FUSED) ? tw_count(LENI) : 0;
    constexpr int EPC = 16 / (int)sizeof(C);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* twF = buf + TC * LD;
    C* twI = twF + NTWF;
    C* stage = twI + ((NTWI + NTWF + 1) & ~1) - NTWF;  // 16-byte aligned past both tables
    const int L = a.len_in;  // line elements loaded per column
    const int stage_elems = L * TC;
    for (int j = threadIdx.x; j < NTWF; j += blockDim.x) twF[j] = a.twF[j];
    if constexpr (MODE == COL_FUSED)
        for (int j = threadIdx.x; j < NTWI; j += blockDim.x) twI[j] = a.twI[j];
    const int ncols = a.ncols;
    const int per_rot = col_tiles * a.nouter;

    auto issue = [&](int t, int slot) {
        const int b = t / per_rot;
        const int rem = t - b * per_rot;
        const int outer = rem / col_tiles;
        const int col0 = (rem - outer * col_tiles) * TC;
        const int cols = min(TC, ncols - col0);
        const int cpr = cols / EPC;  // 16-byte chunks per line element
        const C* src = a.in + (int64_t)b * a.in_rot_stride + (int64_t)outer * a.in_outer_stride + col0;
        C* dst = stage + slot * stage_elems;
        const int chunks = L * cpr;
        for (int q = threadIdx.x; q < chunks; q += blockDim.x) {
            const int e = q / cpr;
            const int c = (q - e * cpr) * EPC;
            cp_async16(dst + e * TC + c, src + (int64_t)e * ncols + c);
        }
    };

    int t = blockIdx.x;
    if (t < total_tiles) issue(t, 0);
    cp_async_commit();
    const int hN = a.N >> 1;
    const C zero = mk(T(0), T(0));
    for (int it = 0; t < total_tiles; ++it) {
        const int tn = t + gridDim.x;
        if (tn < total_tiles) issue(tn, (it + 1) & 1);
        cp_async_commit();
        cp_async_wait_1();
        __syncthreads();
        const int b = t / per_rot;
        const int rem = t - b * per_rot;
        const int outer = rem / col_tiles;
        const int col0 = (rem - outer * col_tiles) * TC;
        const C* st = stage + (it & 1) * stage_elems;
        for (int idx = threadIdx.x; idx < TC * LENF; idx += blockDim.x) {
            const int col = idx % TC;
            const int pos = idx / TC;
            int e;
            if constexpr (MODE == COL_FWD || MODE == COL_FUSED) {
                e = pos + a.s_h;
                if (e >= LENF) e -= LENF;
                if (e >= L) e = -1;
            } else if constexpr (MODE == COL_EXPAND) {
                e = pos < hN ? pos : (pos >= LENF - hN ? pos - LENF + a.N : -1);
            } else {
                e = pos;
            }
            buf[col * LD + pad(pos)] = (e >= 0 && col0 + col < ncols) ? st[e * TC + col] : zero;
        }
        __syncthreads();
        constexpr bool INV1 = (MODE == COL_INV || MODE == COL_EXPAND);
        fft_inplace<C, LENF, INV1, TC>(buf, LD, twF);
        C* out = a.out + (int64_t)b * a.out_rot_stride + (int64_t)outer * a.out_outer_stride;
        if constexpr (MODE == COL_FWD) {
            for (int idx = threadIdx.x; idx < TC * a.N; idx += blockDim.x) {
                const int col = idx % TC;
                const int kp = idx / TC;
                const int gcol = col0 + col;
                if (gcol < ncols) {
                    const int pos = kp < hN ? kp : kp - a.N + LENF;
                    out[(int64_t)kp * ncols + gcol] = buf[col * LD + pad(pos)];
                }
            }
        } else if constexpr (MODE == COL_INV || MODE == COL_EXPAND) {
            for (int idx = threadIdx.x; idx < TC * LENF; idx += blockDim.x) {
                const int col = idx % TC;
                const int e = idx / TC;
                const int gcol = col0 + col;
                if (gcol < ncols) out[(int64_t)e * ncols + gcol] = buf[col * LD + pad(e)];
            }
        } else {  // COL_FUSED
            constexpr int PERX = (TC * LENI + FFT_THREADS - 1) / FFT_THREADS;
            C v[PERX];
#pragma unroll
            for (int q = 0; q < PERX; ++q) {
                const int idx = threadIdx.x + q * FFT_THREADS;
                v[q] = zero;
                if (idx < TC * LENI) {
                    const int col = idx % TC;
                    const int kp = idx / TC;
                    const int gcol = col0 + col;
                    if (gcol < ncols) {
                        const int pos = kp < hN ? kp : kp - LENI + LENF;
                        v[q] = cmul(buf[col * LD + pad(pos)], a.W[(int64_t)kp * ncols + gcol]);
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < PERX; ++q) {
                const int idx = threadIdx.x + q * FFT_THREADS;
                if (idx < TC * LENI) buf[(idx % TC) * LD + pad(idx / TC)] = v[q];
            }
            __syncthreads();
            fft_inplace<C, LENI, true, TC>(buf, LD, twI);
            for (int idx = threadIdx.x; idx < TC * LENI; idx += blockDim.x) {
                const int col = idx % TC;
                const int e = idx / TC;
                const int gcol = col0 + col;
                if (gcol < ncols) out[(int64_t)e * ncols + gcol] = buf[col * LD + pad(e)];
            }
        }
        __syncthreads();
        t = tn;
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

// Opt a kernel into more than 48 KiB of dynamic shared memory.  The attribute
// is one value per kernel and device, so it only ever grows: a launch with less
// shared memory than the current cap needs no change.
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> cap;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair(dev, (const void*)kernel);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cap.find(key);
    if (it != cap.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cap[key] = bytes;
    return e;
}

// Persistent grid: as many CTAs as fit on the device at once, capped by the tiles.
// A failed query is cleared and falls back to one CTA per SM.
template <typename K>
static int persistent_grid(K kernel, size_t smem, int tiles) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 1;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    return std::max(1, std::min(tiles, sms * per_sm));
}

template <typename T, int LEN, int MODE>
static cudaError_t rows_impl(const RowArgs<T>& a, int batch, int* nparts, cudaStream_t st) {
    using C = cplx<T>;
    if (cudaPeekAtLastError() != cudaSuccess) return cudaErrorUnknown;  // an earlier call left an error
    constexpr int TR = lines_per_cta<T, LEN>();
    const int nb = (a.nrows + TR - 1) / TR;
    if (nparts) *nparts = nb;
    if (nb == 0 || batch == 0) return cudaSuccess;
    const bool aligned = (a.in_row_stride == a.len_in) && ((a.len_in * (int)sizeof(C)) % 16 == 0) &&
                         ((a.in_rot_stride * (int64_t)sizeof(C)) % 16 == 0) &&
                         ((reinterpret_cast<uintptr_t>(a.in) & 15) == 0);
    if (aligned) {
        const int ntw = tw_count(LEN);
        const size_t smem =
            (size_t)(TR * line_pitch(LEN) + ((ntw + 1) & ~1) + 2 * TR * a.len_in) * sizeof(C);
        auto kern = k_rows_p<T, LEN, MODE>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        const int total = nb * batch;
        kern<<<persistent_grid(kern, smem, total), 256, smem, st>>>(a, nb, total);
        note_launch();
        return cudaGetLastError();
    }
    const size_t smem = (size_t)(TR * line_pitch(LEN) + tw_count(LEN)) * sizeof(C);
    auto kern = k_rows<T, LEN, MODE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, batch), 256, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int LENF, int LENI, int MODE>
static cudaError_t cols_impl(const ColArgs<T>& a, int batch, cudaStream_t st) {
    using C = cplx<T>;
    if (cudaPeekAtLastError() != cudaSuccess) return cudaErrorUnknown;  // an earlier call left an error
    constexpr int TC = lines_per_cta<T, LENF>();
    const int nb = (a.ncols + TC - 1) / TC;
    if (nb == 0 || batch == 0 || a.nouter == 0) return cudaSuccess;
    const int epc = 16 / (int)sizeof(C);
    const bool aligned = (a.ncols % TC == 0 || (a.ncols % TC) % epc == 0) && (a.ncols % epc == 0) &&
                         ((a.in_rot_stride * (int64_t)sizeof(C)) % 16 == 0) &&
                         ((a.in_outer_stride * (int64_t)sizeof(C)) % 16 == 0) &&
                         ((reinterpret_cast<uintptr_t>(a.in) & 15) == 0) && a.len_in <= LENF;
    const int ntwf = tw_count(LENF), ntwi = (MODE == COL_FUSED) ? tw_count(LENI) : 0;
    if (aligned) {
        const size_t smem =
            (size_t)(TC * line_pitch(LENF) + ((ntwf + ntwi + 1) & ~1) + 2 * (size_t)a.len_in * TC) * sizeof(C);
        auto kern = k_cols_p<T, LENF, LENI, MODE>;
        cudaError_t e = set_smem(kern, smem);
        if (e != cudaSuccess) return e;
        const int total = nb * a.nouter * batch;
        kern<<<persistent_grid(kern, smem, total), 256, smem, st>>>(a, nb, total);
        note_launch();
        return cudaGetLastError();
    }
    const size_t smem = (size_t)(TC * line_pitch(LENF) + tw_count(LENF) + tw_count(LENI)) * sizeof(C);
    auto kern = k_cols<T, LENF, LENI, MODE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, a.nouter, batch), 256, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rows_t(int mode, const RowArgs<T>& a, int batch, int* nparts, cudaStream_t st) {
    const int len = (mode == ROW_FWD || mode == ROW_EXPAND) ? a.n : a.N;
#define SD_ROW_CASE(L)                                                          \
    case L:                                                                     \
        switch (mode) {                                                         \
            case ROW_FWD: return rows_impl<T, L, ROW_FWD>(a, batch, nparts, st);   \
            case ROW_INV_ARGMAX: return rows_impl<T, L, ROW_INV_ARGMAX>(a, batch, nparts, st); \
            case ROW_INV_MAP: return rows_impl<T, L, ROW_INV_MAP>(a, batch, nparts, st); \
            case ROW_EXPAND: return rows_impl<T, L, ROW_EXPAND>(a, batch, nparts, st); \
        }                                                                       \
        break;
    switch (len) { SD_FOR_EACH_LEN(SD_ROW_CASE) }
#undef SD_ROW_CASE
    return cudaErrorInvalidValue;
}

// n = 2N pairs for the fused pass
template <typename T>
cudaError_t launch_cols_t(int mode, const ColArgs<T>& a, int batch, cudaStream_t st) {
    if (mode == COL_FUSED) {
        switch (a.N) {
#define SD_FUSED_CASE(NN) \
    case NN: return cols_impl<T, 2 * NN, NN, COL_FUSED>(a, batch, st);
            SD_FUSED_CASE(8) SD_FUSED_CASE(16) SD_FUSED_CASE(24) SD_FUSED_CASE(32) SD_FUSED_CASE(48)
            SD_FUSED_CASE(64) SD_FUSED_CASE(96) SD_FUSED_CASE(128) SD_FUSED_CASE(192) SD_FUSED_CASE(256)
#undef SD_FUSED_CASE
        }
        return cudaErrorInvalidValue;
    }
    const int len = (mode == COL_INV) ? a.N : a.n;
#define SD_COL_CASE(L)                                                       \
    case L:                                                                  \
        switch (mode) {                                                      \
            case COL_FWD: return cols_impl<T, L, L, COL_FWD>(a, batch, st);      \
            case COL_INV: return cols_impl<T, L, L, COL_INV>(a, batch, st);      \
            case COL_EXPAND: return cols_impl<T, L, L, COL_EXPAND>(a, batch, st); \
        }                                                                    \
        break;
    switch (len) { SD_FOR_EACH_LEN(SD_COL_CASE) }
#undef SD_COL_CASE
    return cudaErrorInvalidValue;
}

// Shared-memory budget of one spreading CTA (64 KiB of complex cells).
constexpr int kSpreadTileBytes = 64 * 1024;

template <typename T>
cudaError_t launch_spread_t(const SpreadArgs<T>& a, int dim, int batch, cudaStream_t st) {
    if (a.m == 0 || batch == 0) return cudaSuccess;
    const dim3 grid((unsigned)((a.m + 255) / 256), batch);
    const int cap = a.direct ? 0 : kSpreadTileBytes / (int)sizeof(cplx<T>);
    const size_t smem = a.direct ? 0 : (size_t)kSpreadTileBytes;
#define SD_SPREAD_CASE(WW)                                                                   \
    case WW: {                                                                               \
        auto kern = (dim == 2) ? k_spread<T, 2, WW> : k_spread<T, 3, WW>;                    \
        cudaError_t e = set_smem(kern, smem);                                                \
        if (e != cudaSuccess) return e;                                                      \
        kern<<<grid, 256, smem, st>>>(a, cap);                                               \
        note_launch();                                                                       \
        return cudaGetLastError();                                                           \
    }
    switch (a.w) {
        SD_SPREAD_CASE(4) SD_SPREAD_CASE(5) SD_SPREAD_CASE(6) SD_SPREAD_CASE(7) SD_SPREAD_CASE(8)
        SD_SPREAD_CASE(10) SD_SPREAD_CASE(12) SD_SPREAD_CASE(16)
    }
#undef SD_SPREAD_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_spread_bins_t(const SpreadArgs<T>& a, const BinArgs& bn, int dim, int batch, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bn.count, 0, sizeof(int) * (size_t)batch * bn.nbins, st);
    if (e != cudaSuccess) return e;
    const dim3 gpts((unsigned)((a.m + 255) / 256), batch);
    const dim3 gtiles((unsigned)bn.nbins, batch);
#define SD_BIN_CASE(WW)                                                           \
    case WW:                                                                      \
        if (a.m > 0) {                                                            \
            if (dim == 2) k_bin_count<T, 2, WW><<<gpts, 256, 0, st>>>(a, bn);      \
            else k_bin_count<T, 3, WW><<<gpts, 256, 0, st>>>(a, bn);               \
            k_bin_scan<<<batch, 1024, 0, st>>>(bn);                                \
            k_bin_scatter<T><<<gpts, 256, 0, st>>>(a.m, bn);                        \
            note_launch(3);                                                       \
        } else {                                                                  \
            k_bin_scan<<<batch, 1024, 0, st>>>(bn);                                \
            note_launch();                                                        \
        }                                                                         \
        if (dim == 2) k_spread_tiles<T, 2, WW><<<gtiles, 256, 0, st>>>(a, bn);     \
        else k_spread_tiles<T, 3, WW><<<gtiles, 256, 0, st>>>(a, bn);              \
        note_launch();                                                            \
        return cudaGetLastError();
    switch (a.w) {
        SD_BIN_CASE(4) SD_BIN_CASE(5) SD_BIN_CASE(6) SD_BIN_CASE(7)
    }
#undef SD_BIN_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

// Stage-ordered twiddle table of one line length, in FP64 (one thread: at most
// a few hundred entries, built once).
template <typename T>
__global__ void k_twiddles(cplx<T>* tw, int len) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    tw_for_each(len, [&](int j, int r, int k, int P, int R) {
        double s, c;
        sincospi(-2.0 * (double)(r * k) / (double)(P * R), &s, &c);
        tw[j] = mk(T(c), T(s));
    });
}

template <typename T>
__global__ void k_wtable(const cplx<T>* B1, const double* D, int N, int dim, double L, double sigma_g,
                         int shift, int deriv, cplx<T>* W) {
    const int64_t tot = (dim == 2) ? (int64_t)N * N : (int64_t)N * N * N;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tot) return;
    int kp[3];
    int64_t r = i;
    for (int d = 0; d < dim; ++d) {
        kp[d] = (int)(r % N);
        r /= N;
    }
    const int hN = N >> 1;
    double k2 = 0.0, prodD = 1.0, kd = 0.0;
    int ksum = 0;
    bool nyq = false;
    for (int d = 0; d < dim; ++d) {
        const int kap = kp[d] < hN ? kp[d] : kp[d] - N;
        if (kap == -hN) nyq = true;
        const double k = 2.0 * M_PI * (double)kap / L;
        k2 += k * k;
        prodD *= D[kp[d]];
        ksum += kap;
        if (d == deriv) kd = k;
    }
    if (nyq) {
        W[i] = mk(T(0), T(0));
        return;
    }
    double Ld = L * L;
    if (dim == 3) Ld *= L;
    double f = exp(-sigma_g * sigma_g * k2) / (Ld * prodD * prodD);
    if (shift && (ksum & 1)) f = -f;
    const double br = (double)B1[i].x, bi = (double)B1[i].y;
    double vr = f * br, vi = f * bi;
    if (deriv >= 0) {  // times i k
        const double tr = -vi * kd, ti = vr * kd;
        vr = tr;
        vi = ti;
    }
    W[i] = mk(T(vr), T(vi));
}

template <typename T>
__global__ void k_interleave(const cplx<T>* src, cplx<T>* dst, int64_t cells, int f) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cells) dst[4 * i + f] = src[i];
}

template <typename T>
cudaError_t launch_twiddles_t(cplx<T>* tw, int len, cudaStream_t st) {
    k_twiddles<T><<<1, 32, 0, st>>>(tw, len);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wtable_t(const cplx<T>* B1, const double* D, int N, int dim, double L, double sigma_g,
                            int shift, int deriv, cplx<T>* W, cudaStream_t st) {
    const int64_t tot = (dim == 2) ? (int64_t)N * N : (int64_t)N * N * N;
    k_wtable<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(B1, D, N, dim, L, sigma_g, shift, deriv, W);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interleave_t(const cplx<T>* src, cplx<T>* dst, int64_t cells, int f, cudaStream_t st) {
    k_interleave<T><<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(src, dst, cells, f);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sd

#define SD_INSTANTIATE_NUFFT(T)                                                                         \
    namespace sd {                                                                                      \
    template <> cudaError_t launch_spread<T>(const SpreadArgs<T>& a, int dim, int batch, cudaStream_t st) { \
        return launch_spread_t<T>(a, dim, batch, st);                                                   \
    }                                                                                                   \
    template <> cudaError_t launch_rows<T>(int mode, const RowArgs<T>& a, int batch, int* np, cudaStream_t st) { \
        return launch_rows_t<T>(mode, a, batch, np, st);                                                \
    }                                                                                                   \
    template <> cudaError_t launch_cols<T>(int mode, const ColArgs<T>& a, int batch, cudaStream_t st) {   \
        return launch_cols_t<T>(mode, a, batch, st);                                                    \
    }                                                                                                   \
    template <> cudaError_t launch_spread_bins<T>(const SpreadArgs<T>& a, const BinArgs& bn, int dim, int batch, \
                                                  cudaStream_t st) {                                    \
        return launch_spread_bins_t<T>(a, bn, dim, batch, st);                                          \
    }                                                                                                   \
    template <> cudaError_t launch_twiddles<T>(cplx<T>* tw, int len, cudaStream_t st) {                 \
        return launch_twiddles_t<T>(tw, len, st);                                                       \
    }                                                                                                   \
    template <> cudaError_t launch_wtable<T>(const cplx<T>* B1, const double* D, int N, int dim, double L, \
                                             double sg, int shift, int deriv, cplx<T>* W, cudaStream_t st) { \
        return launch_wtable_t<T>(B1, D, N, dim, L, sg, shift, deriv, W, st);                           \
    }                                                                                                   \
    template <> cudaError_t launch_interleave<T>(const cplx<T>* s, cplx<T>* d, int64_t c, int f, cudaStream_t st) { \
        return launch_interleave_t<T>(s, d, c, f, st);                                                  \
    }                                                                                                   \
    }
