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

#include <cooperative_groups.h>

#include "fft.cuh"
#include "fftp.cuh"
#include "kernels.cuh"
#include "topk.cuh"

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

// Threads of a line-pass CTA: the butterflies of the plan's widest stage over
// the CTA's lines (one butterfly per thread per stage), rounded up to whole
// warps, at least 64.  Wider than 384 butterflies (512-point lines) the CTA
// keeps 256 threads with two butterflies each: registers would otherwise allow
// only one CTA per SM.
template <int LEN>
__host__ __device__ constexpr int cta_threads_for(int lines) {
    int most = 0;
    for (int s = 0; plan_radix(LEN, s) != 0; ++s) {
        const int nb = lines * (LEN / plan_radix(LEN, s));
        most = nb > most ? nb : most;
    }
    most = (most + 31) / 32 * 32;
    return most < 64 ? 64 : (most > 384 ? 256 : most);
}

template <typename T, int LEN>
__host__ __device__ constexpr int cta_threads() {
    return cta_threads_for<LEN>(lines_per_cta<T, LEN>());
}

// Resident CTAs per SM that a pass's register allocation is bounded for, 0 for
// the compiler's own choice.  The 384-point FP32 passes (384 threads) take 3
// (at most 56 registers a thread; 66-70 otherwise, which allows two); the
// 512-point FP32 passes take 2 (at most 128; 150-170 otherwise, one CTA); the
// fused 256-point column pass takes 4 (at most 64; it would take 75).  Every
// other pass keeps the compiler's choice, which already allows four or more
// CTAs of 256 threads: an explicit minimum there makes it take more registers
// than it needs.
template <typename T, int LEN>
__host__ __device__ constexpr int min_ctas_per_sm() {
    return sizeof(T) != 4 ? 0 : (LEN == 384 ? 3 : (LEN == 512 ? 2 : 0));
}

// The same for a column pass of MODE (the fused 256-point FP32 pass takes 4).
template <typename T, int LEN, int MODE>
__host__ __device__ constexpr int min_ctas_per_sm_cols() {
    return (sizeof(T) == 4 && LEN == 256 && MODE == COL_FUSED) ? 4 : min_ctas_per_sm<T, LEN>();
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

// Taps of one sample: x/y weights in registers (unrolled loops), the z loop
// rolled with its weight evaluated per iteration (no run-time-indexed arrays).
template <typename T, int D, int W>
__device__ __forceinline__ void spread_direct(cplx<T>* out, int s, int s_h, const int* u0, const T (*wt)[W],
                                              cplx<T> c, T gz, T beta) {
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
        const T inv_half = T(2) / T(W);
        const int uz0 = u0[2];
#pragma unroll 1
        for (int kz = 0; kz < W; ++kz) {
            const T zz = (T(uz0 + kz) - gz) * inv_half;
            const T z2 = zz * zz;
            const T wz = (z2 <= T(1)) ? exp(beta * (sqrt(T(1) - z2) - T(1))) : T(0);
            const C cz = cscale(c, wz);
            C* plane = out + (int64_t)wrap_index(uz0 + kz + s_h, s) * s * s;
#pragma unroll
            for (int ky = 0; ky < W; ++ky)
                spread_row<T, W>(plane + (int64_t)iy[ky] * s, s, ax0, wraps, cscale(cz, wt[1][ky]), wt[0]);
        }
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

// One thread per sample: rotate, evaluate the kernel weights, add the taps to
// the sub-box with global vector atomics (spread_direct).
template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_spread(SpreadArgs<T> a) {
    using C = cplx<T>;
    __shared__ T Rm[9];
    const int b = blockIdx.y;
    if (threadIdx.x == 0) load_rotation(a, b, Rm);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.m) return;
    const vec4<T> p = a.pos[j];
    const C c = a.c[j];
    T y[3];
    y[0] = a.sign * (Rm[0] * p.x + Rm[1] * p.y + Rm[2] * p.z);
    y[1] = a.sign * (Rm[3] * p.x + Rm[4] * p.y + Rm[5] * p.z);
    y[2] = a.sign * (Rm[6] * p.x + Rm[7] * p.y + Rm[8] * p.z);
    const T half = T(W) * T(0.5);
    const T inv_half = T(2) / T(W);
    T wt[2][W];
    int u0[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const T g = y[d] * a.inv_h;
        u0[d] = (int)ceil(g - half);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const T z = (T(u0[d] + k) - g) * inv_half;
            const T z2 = z * z;
            wt[d][k] = (z2 <= T(1)) ? exp(a.beta * (sqrt(T(1) - z2) - T(1))) : T(0);
        }
    }
    const T gz = y[2] * a.inv_h;
    if (D == 3) u0[2] = (int)ceil(gz - half);
    spread_direct<T, D, W>(a.out + (int64_t)b * a.out_rot_stride, a.s, a.s_h, u0, wt, c, gz, a.beta);
}

// ---------------------------------------------------------------------------
// spreading by bins
// ---------------------------------------------------------------------------
//
// The sub-box is cut into bins of TB^d cells (TB = 8, 12 or 16, at least W - 1).
// A sample belongs to the bin that holds the first cell of its tap box, so its
// taps fall in that bin grown by W - 1 cells along each axis: a tile of
// (TB + W - 1)^d cells that one CTA accumulates in shared memory before adding
// it to the sub-box with 16-byte pair atomics (the block-local accumulation
// before the global atomics).

// Tap-box origin (sub-box coordinates, wrapped when the sub-box is the whole
// periodic grid) and kernel weights of sample j under rotation Rm.
// One axis of it: the rotated coordinate d of p, the axis's tap origin and
// its W kernel weights.
template <typename T, int W>
__device__ __forceinline__ int axis_taps(const SpreadArgs<T>& a, const T* Rm, const vec4<T>& p, int d, T wt[W]) {
    const T y = a.sign * (Rm[3 * d] * p.x + Rm[3 * d + 1] * p.y + Rm[3 * d + 2] * p.z);
    const T half = T(W) * T(0.5);
    const T inv_half = T(2) / T(W);
    const T g = y * a.inv_h;
    const int u0 = (int)ceil(g - half);
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const T z = (T(u0 + k) - g) * inv_half;
        const T z2 = z * z;
        wt[k] = (z2 <= T(1)) ? exp(a.beta * (sqrt(T(1) - z2) - T(1))) : T(0);
    }
    return wrap_index(u0 + a.s_h, a.s);
}

template <typename T, int D, int W>
__device__ __forceinline__ void sample_taps(const SpreadArgs<T>& a, const T* Rm, int64_t j, int org[D], T wt[D][W],
                                            cplx<T>& c) {
    const vec4<T> p = a.pos[j];
    c = a.c[j];
#pragma unroll
    for (int d = 0; d < D; ++d) org[d] = axis_taps<T, W>(a, Rm, p, d, wt[d]);
}

// The tap-box origin alone (the same arithmetic as sample_taps).
template <typename T, int D, int W>
__device__ __forceinline__ void sample_origin(const SpreadArgs<T>& a, const T* Rm, int64_t j, int org[D]) {
    const vec4<T> p = a.pos[j];
    T y[3];
    y[0] = a.sign * (Rm[0] * p.x + Rm[1] * p.y + Rm[2] * p.z);
    y[1] = a.sign * (Rm[3] * p.x + Rm[4] * p.y + Rm[5] * p.z);
    y[2] = a.sign * (Rm[6] * p.x + Rm[7] * p.y + Rm[8] * p.z);
    const T half = T(W) * T(0.5);
#pragma unroll
    for (int d = 0; d < D; ++d) org[d] = wrap_index((int)ceil(y[d] * a.inv_h - half) + a.s_h, a.s);
}

// A slot in the sample's bin (bin >= 0; -1 for none): the lanes of a warp with
// the same bin take consecutive slots from one atomic add by the lowest of them
// (a shape's samples are in Morton order, so a warp's samples share few bins).
// Every lane of the warp must call it.
__device__ __forceinline__ int bin_rank(int* count, int bin) {
    const unsigned same = __match_any_sync(0xffffffffu, bin);
    const int lane = (int)(threadIdx.x & 31);
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (lane == leader && bin >= 0) base = atomicAdd(count + bin, __popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(same & ((1u << lane) - 1u));
}

// Raise the bin's largest |component| of c (cmax, float bits: non-negative floats
// order as integers) by the sample's, one atomic per group of lanes with the
// same bin.  Every lane of the warp must call it.
__device__ __forceinline__ void bin_max(int* cmax, int bin, float v) {
    const unsigned same = __match_any_sync(0xffffffffu, bin);
    const unsigned m = __reduce_max_sync(same, (unsigned)__float_as_int(v));
    if ((int)(threadIdx.x & 31) == __ffs(same) - 1 && bin >= 0) atomicMax(cmax + bin, (int)m);
}

// The fixed-point scale of a tile: 2^e with every tap (at most mx, the weights
// being <= 1) below 2^21 and every cell (at most sm, the sum of the tile's |c|)
// below 2^30; x < 2^(biased exponent - 126) for a positive normal x.
__device__ __forceinline__ float tile_scale(float mx, float sm) {
    const int emx = ((__float_as_int(mx) >> 23) & 255) - 126;
    const int esm = ((__float_as_int(sm) >> 23) & 255) - 126;
    const int e = min(21 - emx, 30 - esm);
    const int se = sm > 0.f ? min(max(127 + e, 1), 254) : 127;
    return __int_as_float(se << 23);
}

template <typename T, int D, int W, int TB>
__global__ void __launch_bounds__(256) k_bin_count(SpreadArgs<T> a, BinArgs bn) {
    __shared__ T Rm[9];
    const int b = blockIdx.y;
    if (threadIdx.x == 0) load_rotation(a, b, Rm);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = j < a.m;
    int bin = -1;
    float cm = 0.f;
    if (live) {
        int org[D];
        sample_origin<T, D, W>(a, Rm, j, org);
        bin = 0;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) bin = bin * bn.nb + org[d] / TB;
        const cplx<T> c = a.c[j];
        cm = fmaxf(fabsf((float)c.x), fabsf((float)c.y));
    }
    const int rank = bin_rank(bn.count + (int64_t)b * bn.nbins, bin);
    if (bn.cmax) bin_max(bn.cmax + (int64_t)b * bn.nbins, bin, cm);
    if (live) {
        const int64_t o = (int64_t)b * a.m + j;
        bn.bin_of[o] = bin;
        bn.rank[o] = rank;
    }
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

// Pitches (y, z) of the tile kernel's shared planes, PS = TB + W - 1 cells a
// side.  Lanes take the taps of a sample whose offsets kx + PY ky + PZ kz are
// distinct mod 32, so each atomic instruction touches 32 distinct banks; these
// pitches (the smallest, up to 15 % more cells than dense, found by exhaustive
// search over PY mod 32 and PZ mod 32) let every W^D tap box be covered in the
// minimum ceil(W^D / 32) such rounds, each round's taps lying on rows whose
// staged products c wy wz are read in one shared wavefront.
__host__ __device__ constexpr int tile_pitch(int D, int W, int TB, int axis) {
    // {PY, PZ} per (W, TB); 2D uses PY only
    constexpr int p2[4][3] = {{12, 18, 19}, {13, 19, 26}, {13, 18, 21}, {14, 18, 23}};
    constexpr int p3[4][3][2] = {{{12, 136}, {16, 244}, {20, 392}},
                                 {{13, 165}, {19, 311}, {23, 461}},
                                 {{13, 169}, {18, 314}, {23, 486}},
                                 {{14, 199}, {18, 327}, {23, 510}}};
    const int wi = W - 4, ti = TB == 8 ? 0 : (TB == 12 ? 1 : 2);
    return D == 2 ? (axis == 0 ? p2[wi][ti] : 0) : p3[wi][ti][axis];
}

// Shared-memory layout of the tile kernel: two fixed-point planes of the tile
// (real, imaginary), then the staged sample records.
template <int D, int W, int TB>
struct TileShape {
    static_assert(W >= 4 && W <= 7 && (TB == 8 || TB == 12 || TB == 16), "tile shape not tabulated");
    static constexpr int PS = TB + W - 1;                         // tile side
    static constexpr int PY = tile_pitch(D, W, TB, 0);            // y pitch of the planes
    static constexpr int PZ = tile_pitch(D, W, TB, 1);            // z pitch (3D)
    static_assert(PY >= PS && (D == 2 || PZ >= PY * PS), "pitch below the tile side");
    static constexpr int CELLS = (D == 3) ? PZ * PS : PY * PS;
    static constexpr int ROWS = (D == 3) ? W * W : W;             // (ky, kz) rows of a tap box
    static constexpr int TAPS = ROWS * W;
    static constexpr int CHUNK = 64;                              // samples staged at a time
    // record: wx[W] | c.x c.y (scaled) | base | origin | wy * wz per row
    static constexpr int O_C = W, O_BASE = W + 2, O_ORG = W + 3, O_ROW = W + 4;
    static constexpr int REC = O_ROW + ROWS;
    static constexpr size_t smem = (size_t)2 * CELLS * sizeof(int) + (size_t)CHUNK * REC * sizeof(float);
    __host__ __device__ static constexpr int offset(int tap) {
        return tap % W + PY * ((tap / W) % W) + (D == 3 ? PZ * (tap / (W * W)) : 0);
    }
    // rounds: the most taps whose offsets share a residue mod 32
    __host__ __device__ static constexpr int rounds() {
        int most = 0;
        for (int r = 0; r < 32; ++r) {
            int n = 0;
            for (int t = 0; t < TAPS; ++t) n += (offset(t) & 31) == r;
            most = n > most ? n : most;
        }
        return most;
    }
    static constexpr int ROUNDS = rounds();
    static_assert(ROUNDS == (TAPS + 31) / 32, "pitches leave a bank conflict");
};

// The tap of each (round, lane) of the tile kernel, -1 for an idle lane: the
// q-th tap (in tap order) whose offset is congruent to the lane mod 32.
template <int D, int W, int TB>
struct TapRounds {
    short tap[TileShape<D, W, TB>::ROUNDS * 32];
};
template <int D, int W, int TB>
__host__ __device__ constexpr TapRounds<D, W, TB> make_tap_rounds() {
    using TS = TileShape<D, W, TB>;
    TapRounds<D, W, TB> t{};
    for (int i = 0; i < TS::ROUNDS * 32; ++i) t.tap[i] = -1;
    int used[32] = {};
    for (int k = 0; k < TS::TAPS; ++k) {
        const int r = TS::offset(k) & 31;
        t.tap[used[r]++ * 32 + r] = (short)k;
    }
    return t;
}
template <int D, int W, int TB>
__device__ const TapRounds<D, W, TB> kTapRounds = make_tap_rounds<D, W, TB>();
// Bit q: every lane has a tap in round q.
template <int D, int W, int TB>
__host__ __device__ constexpr unsigned full_rounds_mask() {
    const TapRounds<D, W, TB> t = make_tap_rounds<D, W, TB>();
    unsigned mask = 0;
    for (int q = 0; q < TileShape<D, W, TB>::ROUNDS; ++q) {
        bool full = true;
        for (int l = 0; l < 32; ++l) full = full && t.tap[q * 32 + l] >= 0;
        mask |= (full ? 1u : 0u) << q;
    }
    return mask;
}

// One CTA per (bin, rotation).  The CTA stages CHUNK of the bin's samples at a
// time: one thread per sample evaluates its kernel weights and tile offset, then
// all threads form the products c * scale * wy[ky] * wz[kz] of every row of
// every staged tap box.  The warps then take the staged samples round-robin with
// the lanes on consecutive taps (x fastest), so one shared atomic instruction
// hits up to 32 distinct cells; a tap costs one FFMA per component that both
// multiplies by wx and rounds to the fixed point (the addend 1.5 * 2^23 leaves
// round(v) in the low mantissa bits for |v| < 2^22), an integer subtract and the
// atomic.  The scale is the power of two that keeps every tap below 2^21 and
// every cell (at most the bin's sum of |c|, the weights being <= 1) below 2^30,
// so the integer sums are exact and independent of the order of the adds.
// A sample whose tap box does not lie in the tile (not possible when the
// counting pass and this one agree, as they evaluate the same function) is
// added with global atomics instead.
template <int D, int W, int TB>
__global__ void __launch_bounds__(256, 4) k_spread_tiles(SpreadArgs<float> a, BinArgs bn) {
    using TS = TileShape<D, W, TB>;
    constexpr int PS = TS::PS, PS2 = PS * PS, PY = TS::PY, PZ = TS::PZ, CELLS = TS::CELLS, ROWS = TS::ROWS, TAPS = TS::TAPS;
    constexpr int ROUNDS = TS::ROUNDS;
    constexpr int CHUNK = TS::CHUNK, REC = TS::REC;
    static_assert(4 * CHUNK == 256, "four threads per staged sample");
    constexpr unsigned FULL = full_rounds_mask<D, W, TB>();
    constexpr int NWARP = 8;
    constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23
    constexpr int MAGIC_BITS = 0x4B400000;
    extern __shared__ __align__(16) int tsm[];
    int* tre = tsm;
    int* tim = tsm + CELLS;
    float* stage = reinterpret_cast<float*>(tsm + 2 * CELLS);
    __shared__ float Rm[9];
    const int b = blockIdx.y;
    const int t = blockIdx.x;
    const int* off = bn.offset + (int64_t)b * (bn.nbins + 1);
    const int lo = off[t], hi = off[t + 1];
    if (lo == hi) return;  // empty bin (uniform over the block)
    for (int i = threadIdx.x; i < CELLS; i += blockDim.x) {
        tre[i] = 0;
        tim[i] = 0;
    }
    if (threadIdx.x == 0) load_rotation(a, b, Rm);
    const int32_t* sorted = bn.sorted + (int64_t)b * a.m;
    // the bin's largest |component| of c (from the counting pass) bounds every tap,
    // and the bin's count times it bounds every cell (1e-4 over: float rounding)
    const float mx = __int_as_float(bn.cmax[(int64_t)b * bn.nbins + t]);
    const float scale = tile_scale(mx, (float)(hi - lo) * mx * 1.0001f);
    __syncthreads();  // the zeroed tile and Rm
    const float inv_scale = 1.f / scale;  // a power of two: exact
    const int nb = bn.nb, s = a.s;
    const int org0[3] = {(t % nb) * TB, ((t / nb) % nb) * TB, (D == 3) ? (t / (nb * nb)) * TB : 0};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this lane's tap in each round (the lanes of a round on distinct banks): x
    // weight, row of c * wy * wz, tile offset; bit q of `live`: a tap in round q
    int kx_of[ROUNDS], row_of[ROUNDS], cell_of[ROUNDS];
    unsigned live = 0;
#pragma unroll
    for (int q = 0; q < ROUNDS; ++q) {
        const int tap0 = kTapRounds<D, W, TB>.tap[q * 32 + lane];
        live |= (tap0 >= 0 ? 1u : 0u) << q;
        const int tap = max(tap0, 0);
        const int kx = tap % W, row = tap / W;
        const int ky = row % W, kz = (D == 3) ? row / W : 0;
        kx_of[q] = kx;
        row_of[q] = TS::O_ROW + row;
        cell_of[q] = kx + PY * ky + PZ * kz;
    }
    float2* out = a.out + (int64_t)b * a.out_rot_stride;
    for (int p0 = lo; p0 < hi; p0 += CHUNK) {
        const int nj = min(CHUNK, hi - p0);
        // (1) four threads per sample, lanes 4i..4i+3 of one warp: the kernel
        // weights of one axis each (the fourth: the scaled c); the y and z
        // weights go to the sample's four lanes by shuffles, and each lane stores
        // the products wy * wz of the rows whose kz is its index mod 4
        {
            const int j = (int)threadIdx.x >> 2, part = (int)threadIdx.x & 3;
            const bool act = j < nj;
            float* r = stage + j * REC;
            int contrib = 0, ok = 1, packed = 0;
            float wt[W];
#pragma unroll
            for (int k = 0; k < W; ++k) wt[k] = 1.f;  // 2D: unit z weights in lane 2
            if (act) {
                const int64_t js = sorted[p0 + j];
                if (part < D) {
                    const int o = axis_taps<float, W>(a, Rm, a.pos[js], part, wt);
                    const int l = o - (part == 0 ? org0[0] : (part == 1 ? org0[1] : org0[2]));
                    ok = (l >= 0 && l < TB);
                    contrib = l * (part == 0 ? 1 : (part == 1 ? PY : PZ));
                    packed = o << (10 * part);
                    if (part == 0)
#pragma unroll
                        for (int k = 0; k < W; ++k) r[k] = wt[k];
                } else if (part == 3) {
                    const float2 c = a.c[js];
                    r[TS::O_C] = c.x * scale;
                    r[TS::O_C + 1] = c.y * scale;
                }
            }
            // combine the four lanes of the sample (every lane of the warp takes part)
#pragma unroll
            for (int o = 1; o < 4; o <<= 1) {
                contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
                ok &= __shfl_xor_sync(0xffffffffu, ok, o);
                packed |= __shfl_xor_sync(0xffffffffu, packed, o);
            }
            float wy[W], wz[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                wy[k] = __shfl_sync(0xffffffffu, wt[k], (lane & ~3) | 1);
                wz[k] = __shfl_sync(0xffffffffu, wt[k], (lane & ~3) | 2);
            }
            if (act) {
                if (part == 0) {
                    r[TS::O_BASE] = __int_as_float(ok ? contrib : -1);
                    r[TS::O_ORG] = __int_as_float(packed);
                }
#pragma unroll
                for (int kz = 0; kz < ROWS / W; ++kz)
                    if ((kz & 3) == part)
#pragma unroll
                        for (int ky = 0; ky < W; ++ky) r[TS::O_ROW + ky + W * kz] = wy[ky] * wz[kz];
            }
        }
        __syncthreads();
        // (2) the warps add the staged samples round-robin, one at a time
        for (int j = warp; j < nj; j += NWARP) {
            const float* r = stage + j * REC;
            const int base = __float_as_int(r[TS::O_BASE]);
            if (base >= 0) {  // uniform over the warp
                const float cx = r[TS::O_C], cy = r[TS::O_C + 1];
#pragma unroll
                for (int q = 0; q < ROUNDS; ++q) {
                    if (((FULL >> q) & 1u) || ((live >> q) & 1u)) {
                        const float w = r[kx_of[q]] * r[row_of[q]];
                        const int cell = base + cell_of[q];
                        atomicAdd(tre + cell, __float_as_int(fmaf(cx, w, MAGIC)) - MAGIC_BITS);
                        atomicAdd(tim + cell, __float_as_int(fmaf(cy, w, MAGIC)) - MAGIC_BITS);
                    }
                }
            } else {  // safety net (a tap box outside the tile): global atomics on the sub-box
                const int packed = __float_as_int(r[TS::O_ORG]);
                const float cx = r[TS::O_C] * inv_scale, cy = r[TS::O_C + 1] * inv_scale;
#pragma unroll 1
                for (int q = 0; q < ROUNDS; ++q) {
                    const int tap = q * 32 + lane;
                    if (tap < TAPS) {
                        const int kx = tap % W, ky = (tap / W) % W, kz = (D == 3) ? tap / (W * W) : 0;
                        const float w = r[kx] * r[TS::O_ROW + tap / W];
                        int64_t o = (int64_t)wrap_index(((packed >> 10) & 1023) + ky, s) * s +
                                    wrap_index((packed & 1023) + kx, s);
                        if (D == 3) o += (int64_t)wrap_index(((packed >> 20) & 1023) + kz, s) * s * s;
                        atomic_cadd(out + o, make_float2(cx * w, cy * w));
                    }
                }
            }
        }
        __syncthreads();  // the stage is refilled by the next chunk
    }
    // flush: pairs of x-adjacent tile cells (global x even: bins start at even cells)
    constexpr int XP = (PS + 1) / 2;
    constexpr int PAIRS = (D == 3) ? XP * PS2 : XP * PS;
    bool inner = true;  // the tile does not wrap around the sub-box (no modulo below)
#pragma unroll
    for (int d = 0; d < D; ++d) inner &= (org0[d] + PS <= s);
    for (int i = threadIdx.x; i < PAIRS; i += blockDim.x) {
        const int xp = i % XP, row = i / XP;  // row = y + PS z
        const int x = 2 * xp;
        const int li = (row % PS) * PY + (D == 3 ? (row / PS) * PZ : 0) + x;
        const int r0 = tre[li], i0 = tim[li];
        const int r1 = (x + 1 < PS) ? tre[li + 1] : 0, i1 = (x + 1 < PS) ? tim[li + 1] : 0;
        if ((r0 | i0 | r1 | i1) == 0) continue;
        const float2 v0 = make_float2((float)r0 * inv_scale, (float)i0 * inv_scale);
        const float2 v1 = make_float2((float)r1 * inv_scale, (float)i1 * inv_scale);
        const int y = row % PS, z = row / PS;
        const int gx = org0[0] + x;
        if (inner && gx + 1 < s) {
            int64_t o = (int64_t)(org0[1] + y) * s;
            if (D == 3) o += (int64_t)(org0[2] + z) * s * s;
            add_pair(out + o + gx, v0, v1);
            continue;
        }
        int64_t o = (int64_t)wrap_index(org0[1] + y, s) * s;
        if (D == 3) o += (int64_t)wrap_index(org0[2] + z, s) * s * s;
        if (gx + 1 < s) {
            add_pair(out + o + gx, v0, v1);
        } else {
            atomic_cadd(out + o + wrap_index(gx, s), v0);
            if (x + 1 < PS) atomic_cadd(out + o + wrap_index(gx + 1, s), v1);
        }
    }
}

// ---------------------------------------------------------------------------
// spreading by sample blocks (no sort)
// ---------------------------------------------------------------------------
//
// A shape's samples are stored in Morton order, so a CTA's BOX_SPC consecutive
// samples form a compact patch that, rotated, still fits a small box of the
// sub-box.  The CTA finds that box (block min / max of the tap-box origins),
// accumulates its samples' taps there in a fixed-point shared tile (warps take
// the samples round-robin, lanes on consecutive taps), then adds the box's
// nonzero cells to the sub-box with 16-byte pair atomics: the global atomics
// fall from about W^d / 2 per sample to about one per two cells of the box.  A
// box larger than the tile, or one that wraps around a periodic sub-box, is
// spread with global atomics per tap instead.

constexpr int BOX_SPC = 128;      // samples per CTA
constexpr int BOX_MAXC = 8192;    // cells of the shared tile (2 x 32 KB)

template <int D, int W>
__global__ void __launch_bounds__(BOX_SPC) k_spread_box(SpreadArgs<float> a) {
    constexpr int REC = D * W + 4;  // weights | c.x c.y | packed origin | pad
    constexpr int TAPS = (D == 3) ? W * W * W : W * W;
    constexpr int ROUNDS = (TAPS + 31) / 32;
    constexpr int NWARP = BOX_SPC / 32;
    constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23
    constexpr int MAGIC_BITS = 0x4B400000;
    extern __shared__ __align__(16) int bsm[];
    int* tre = bsm;
    int* tim = bsm + BOX_MAXC;
    __shared__ float stage[BOX_SPC * REC];
    __shared__ float Rm[9];
    __shared__ int wlo[NWARP][3], whi[NWARP][3];
    __shared__ float wmx[NWARP], wsm[NWARP];
    const int b = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) load_rotation(a, b, Rm);
    __syncthreads();
    const int64_t j0 = (int64_t)blockIdx.x * BOX_SPC;
    const int nj = (int)min((int64_t)BOX_SPC, a.m - j0);
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    float mx = 0.f, sm = 0.f;
    if (tid < nj) {
        int org[D];
        float wt[D][W];
        float2 c;
        sample_taps<float, D, W>(a, Rm, j0 + tid, org, wt, c);
        float* r = stage + tid * REC;
#pragma unroll
        for (int d = 0; d < D; ++d) {
#pragma unroll
            for (int k = 0; k < W; ++k) r[d * W + k] = wt[d][k];
            lo[d] = hi[d] = org[d];
        }
        r[D * W] = c.x;
        r[D * W + 1] = c.y;
        r[D * W + 2] = __int_as_float(org[0] | (org[1] << 10) | ((D == 3 ? org[2] : 0) << 20));
        mx = fmaxf(fabsf(c.x), fabsf(c.y));
        sm = mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            lo[d] = min(lo[d], __shfl_down_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_down_sync(0xffffffffu, hi[d], o));
        }
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        sm += __shfl_down_sync(0xffffffffu, sm, o);
    }
    if (lane == 0) {
        for (int d = 0; d < D; ++d) {
            wlo[warp][d] = lo[d];
            whi[warp][d] = hi[d];
        }
        wmx[warp] = mx;
        wsm[warp] = sm;
    }
    __syncthreads();
    int blo[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
    mx = 0.f;
    sm = 0.f;
    for (int w = 0; w < NWARP; ++w) {
        mx = fmaxf(mx, wmx[w]);
        sm += wsm[w];
    }
    bool fits = true;
    int cells = 1;
    for (int d = 0; d < D; ++d) {
        int l = INT_MAX, h = INT_MIN;
        for (int w = 0; w < NWARP; ++w) {
            l = min(l, wlo[w][d]);
            h = max(h, whi[w][d]);
        }
        blo[d] = l;
        ext[d] = h - l + W;
        fits &= (l + ext[d] <= a.s);  // no wrap around a periodic sub-box
        cells *= ext[d];
    }
    fits &= cells <= BOX_MAXC;
    float2* out = a.out + (int64_t)b * a.out_rot_stride;
    const int s = a.s;
    if (!fits) {
        // global atomics per tap (lanes on consecutive taps of one sample)
        for (int jj = warp; jj < nj; jj += NWARP) {
            const float* r = stage + jj * REC;
            const int packed = __float_as_int(r[D * W + 2]);
            const float cx = r[D * W], cy = r[D * W + 1];
            for (int q = 0; q < ROUNDS; ++q) {
                const int tap = q * 32 + lane;
                if (tap < TAPS) {
                    const int kx = tap % W, ky = (tap / W) % W, kz = (D == 3) ? tap / (W * W) : 0;
                    float w = r[kx] * r[W + ky];
                    int64_t o = (int64_t)wrap_index(((packed >> 10) & 1023) + ky, s) * s +
                                wrap_index((packed & 1023) + kx, s);
                    if (D == 3) {
                        w *= r[2 * W + kz];
                        o += (int64_t)wrap_index(((packed >> 20) & 1023) + kz, s) * s * s;
                    }
                    atomic_cadd(out + o, make_float2(cx * w, cy * w));
                }
            }
        }
        return;
    }
    for (int i = tid; i < cells; i += BOX_SPC) {
        tre[i] = 0;
        tim[i] = 0;
    }
    // taps below 2^21, a cell's sum below 2^30 (the weights are <= 1)
    const int emx = ((__float_as_int(mx) >> 23) & 255) - 126;
    const int esm = ((__float_as_int(sm) >> 23) & 255) - 126;
    const int se = sm > 0.f ? min(max(127 + min(21 - emx, 30 - esm), 1), 254) : 127;
    const float scale = __int_as_float(se << 23);
    const float inv_scale = 1.f / scale;
    const int sy = ext[0], sz = ext[0] * ext[1];
    int kx_of[ROUNDS], off_of[ROUNDS];
#pragma unroll
    for (int q = 0; q < ROUNDS; ++q) {
        const int tap = min(q * 32 + lane, TAPS - 1);
        const int kx = tap % W, ky = (tap / W) % W, kz = (D == 3) ? tap / (W * W) : 0;
        kx_of[q] = tap;  // the tap itself: weights are read per axis below
        off_of[q] = kx + ky * sy + kz * sz;
    }
    __syncthreads();
    for (int jj = warp; jj < nj; jj += NWARP) {
        const float* r = stage + jj * REC;
        const int packed = __float_as_int(r[D * W + 2]);
        int base = ((packed & 1023) - blo[0]) + (((packed >> 10) & 1023) - blo[1]) * sy;
        if (D == 3) base += (((packed >> 20) & 1023) - blo[2]) * sz;
        const float cx = r[D * W] * scale, cy = r[D * W + 1] * scale;
#pragma unroll
        for (int q = 0; q < ROUNDS; ++q) {
            if (TAPS % 32 == 0 || q * 32 + lane < TAPS) {
                const int tap = kx_of[q];
                const int kx = tap % W, ky = (tap / W) % W;
                float w = r[kx] * r[W + ky];
                if (D == 3) w *= r[2 * W + tap / (W * W)];
                const int cell = base + off_of[q];
                atomicAdd(tre + cell, __float_as_int(fmaf(cx, w, MAGIC)) - MAGIC_BITS);
                atomicAdd(tim + cell, __float_as_int(fmaf(cy, w, MAGIC)) - MAGIC_BITS);
            }
        }
    }
    __syncthreads();
    // flush: pairs of x-adjacent cells starting at even global x
    const int x0 = blo[0] & ~1;
    const int npair = (blo[0] + ext[0] - x0 + 1) / 2;
    const int rows = ext[1] * (D == 3 ? ext[2] : 1);
    for (int i = tid; i < rows * npair; i += BOX_SPC) {
        const int row = i / npair, k = i - row * npair;
        const int gx = x0 + 2 * k;
        const int lx = gx - blo[0];
        const int li = row * sy + lx;
        const bool in0 = lx >= 0, in1 = lx + 1 < ext[0];
        const int r0 = in0 ? tre[li] : 0, i0 = in0 ? tim[li] : 0;
        const int r1 = in1 ? tre[li + 1] : 0, i1 = in1 ? tim[li + 1] : 0;
        if ((r0 | i0 | r1 | i1) == 0) continue;
        const int gy = blo[1] + row % ext[1];
        int64_t o = (int64_t)gy * s + gx;
        if (D == 3) o += (int64_t)(blo[2] + row / ext[1]) * s * s;
        const float2 v0 = make_float2((float)r0 * inv_scale, (float)i0 * inv_scale);
        const float2 v1 = make_float2((float)r1 * inv_scale, (float)i1 * inv_scale);
        if (gx + 1 < s) {
            add_pair(out + o, v0, v1);
        } else {
            atomic_cadd(out + o, v0);
        }
    }
}

// ---------------------------------------------------------------------------
// spreading fused with the forward x transform (3D, pruned search)
// ---------------------------------------------------------------------------
//
// One CTA owns SX_TY x SX_TZ whole rows (y, z) of the sub-box, all x.  The
// rotated samples are sorted into bins of SX_TY x SX_TZ (y, z) cells by the
// first cell of their tap box, so the rows of bin (by, bz) receive taps only
// from bins {by - 1, by} x {bz - 1, bz} (both sides are at least W - 1).  The
// CTA accumulates those samples' taps, clipped to its rows, in a fixed-point
// shared tile, then runs the pruned forward x transform of its rows straight
// from the tile and writes the N kept modes of each row.  No sub-box is stored,
// cleared or re-read, and no global atomic is issued.

constexpr int SX_W = 6, SX_TY = SPREADX_TY, SX_TZ = SPREADX_TZ, SX_TR = 6, SX_NT = 256, SX_CHUNK = 64;
static_assert(SX_TY >= SX_W - 1 && SX_TZ >= SX_W - 1, "a tap box must meet at most two bins per axis");
static_assert((SX_TY * SX_TZ) % SX_TR == 0, "rows per FFT group must divide the rows of a bin");
// staged record: w[axis][W] | origin[3] | c * scale (pair)
constexpr int SX_O_ORG = 3 * SX_W, SX_O_C = 3 * SX_W + 4;
constexpr int SX_REC = SX_O_C + 2;

// Row pitch of the shared tile (cells): at least s and 6 mod 32, so that the
// lanes of a warp on consecutive taps of one tap box (x fastest) fall in
// distinct banks.
__host__ __device__ inline int spread_x_pitch(int s) { return s + ((6 - s % 32) + 32) % 32; }

template <int LEN>
__host__ __device__ constexpr size_t spread_x_smem_fixed() {
    // twiddles + the larger of the staging records and the FFT line buffer
    return (size_t)tw_count(LEN) * sizeof(float2) +
           ((size_t)SX_CHUNK * SX_REC * sizeof(float) > (size_t)SX_TR * line_pitch(LEN) * sizeof(float2)
                ? (size_t)SX_CHUNK * SX_REC * sizeof(float)
                : (size_t)SX_TR * line_pitch(LEN) * sizeof(float2));
}
__host__ inline size_t spread_x_smem(int len, int px) {
    size_t fixed = 0;
    switch (len) {
#define SD_SXS(L) case L: fixed = spread_x_smem_fixed<L>(); break;
        SD_FOR_EACH_LEN(SD_SXS)
#undef SD_SXS
    }
    return (size_t)2 * SX_TY * SX_TZ * px * sizeof(int) + fixed;
}

template <typename T, int D, int W>
__global__ void __launch_bounds__(256) k_bin_count_yz(SpreadArgs<T> a, BinArgs bn, int ty, int tz) {
    __shared__ T Rm[9];
    const int b = blockIdx.y;
    if (threadIdx.x == 0) load_rotation(a, b, Rm);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = j < a.m;
    int bin = -1, packed = 0;
    float cm = 0.f;
    if (live) {
        int org[D];
        sample_origin<T, D, W>(a, Rm, j, org);
        bin = (org[2] / tz) * bn.nb + org[1] / ty;
        packed = org[0] | (org[1] << 10) | (org[2] << 20);
        const cplx<T> c = a.c[j];
        cm = fmaxf(fabsf((float)c.x), fabsf((float)c.y));
    }
    const int rank = bin_rank(bn.count + (int64_t)b * bn.nbins, bin);
    bin_max(bn.cmax + (int64_t)b * bn.nbins, bin, cm);
    if (live) {
        const int64_t o = (int64_t)b * a.m + j;
        bn.bin_of[o] = bin;
        bn.org[o] = packed;  // the spreading uses this very origin
        bn.rank[o] = rank;
    }
}

template <int LEN>
__global__ void __launch_bounds__(SX_NT, 3) k_spread_x(SpreadArgs<float> a, BinArgs bn, int nbz, int px,
                                                       float2* out, int64_t out_rot_stride, const float2* twg) {
    constexpr int W = SX_W, TY = SX_TY, TZ = SX_TZ, TR = SX_TR, NT = SX_NT, CHUNK = SX_CHUNK, REC = SX_REC;
    constexpr int ROWS = TY * TZ;
    constexpr int LD = line_pitch(LEN);
    constexpr int NTW = tw_count(LEN);
    constexpr int NB1 = LEN / plan_radix(LEN, 0);
    constexpr int NH = LEN / 2;
    constexpr int NWARP = NT / 32;
    constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23
    constexpr int MAGIC_BITS = 0x4B400000;
    extern __shared__ __align__(16) unsigned char sx_raw[];
    int* tre = reinterpret_cast<int*>(sx_raw);
    int* tim = tre + ROWS * px;
    float2* tw = reinterpret_cast<float2*>(tim + ROWS * px);
    float* stage = reinterpret_cast<float*>(tw + NTW);
    float2* buf = reinterpret_cast<float2*>(tw + NTW);  // the same memory, after the accumulation
    __shared__ float Rm[9];
    __shared__ unsigned char divtab[7][W * W];  // (rho / ny) << 4 | rho % ny
    const int b = blockIdx.y;
    const int nby = bn.nb;
    const int by = (int)blockIdx.x % nby, bz = (int)blockIdx.x / nby;
    const int y0 = by * TY, z0 = bz * TZ;
    const int s = a.s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < ROWS * px; i += NT) {
        tre[i] = 0;
        tim[i] = 0;
    }
    for (int j = tid; j < NTW; j += NT) tw[j] = twg[j];
    for (int i = tid; i < 7 * W * W; i += NT) {
        const int ny = i / (W * W), rho = i % (W * W);
        divtab[ny][rho] = ny ? (unsigned char)(((rho / ny) << 4) | (rho % ny)) : 0;
    }
    if (tid == 0) load_rotation(a, b, Rm);
    // the source bins (by - {0, 1}) x (bz - {0, 1}) and their sample ranges
    const int* off = bn.offset + (int64_t)b * (bn.nbins + 1);
    __shared__ int src_lo[4], src_hi[4];
    __shared__ float src_max[4];
    if (tid < 4) {
        const int yy = by - (tid & 1), zz = bz - (tid >> 1);
        src_lo[tid] = src_hi[tid] = 0;
        src_max[tid] = 0.f;
        if (yy >= 0 && zz >= 0) {
            src_lo[tid] = off[zz * nby + yy];
            src_hi[tid] = off[zz * nby + yy + 1];
            src_max[tid] = __int_as_float(bn.cmax[(int64_t)b * bn.nbins + zz * nby + yy]);
        }
    }
    __syncthreads();
    const int32_t* sorted = bn.sorted + (int64_t)b * a.m;
    float2* outb = out + (int64_t)b * out_rot_stride;
    if (src_hi[0] - src_lo[0] + src_hi[1] - src_lo[1] + src_hi[2] - src_lo[2] + src_hi[3] - src_lo[3] == 0) {
        // no sample reaches these rows: their modes are zero
        for (int i = tid; i < ROWS * (NH / 2); i += NT) {
            const int l = i / (NH / 2), k = i % (NH / 2);
            const int y = y0 + l % TY, z = z0 + l / TY;
            if (y < s && z < s)
                reinterpret_cast<float4*>(outb + ((int64_t)z * s + y) * NH)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    // fixed point: taps below 2^21, a cell's sum (at most the sum of |c| over the
    // source samples, the weights being <= 1) below 2^30; each source bin's count
    // times its largest |component| of c (from the binning pass) bounds that sum
    float mx = 0.f, sm = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        mx = fmaxf(mx, src_max[k]);
        sm += (float)(src_hi[k] - src_lo[k]) * src_max[k];
    }
    const float scale = tile_scale(mx, sm * 1.0001f);
    const float inv_scale = 1.f / scale;  // a power of two: exact
    // this lane's tap in each round of a full tap box: x tap and row (ky + ny kz flattened)
    constexpr int ROUNDS = (W * W * W + 31) / 32;
    int kx_of[ROUNDS], rho_of[ROUNDS];
#pragma unroll
    for (int q = 0; q < ROUNDS; ++q) {
        const int tap = min(q * 32 + lane, W * W * W - 1);
        kx_of[q] = tap % W;
        rho_of[q] = tap / W;
    }
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        for (int p0 = src_lo[k]; p0 < src_hi[k]; p0 += CHUNK) {
            const int nj = min(CHUNK, src_hi[k] - p0);
            // four threads per sample: the kernel weights of one axis each, and c
            {
                const int j = tid >> 2, part = tid & 3;
                if (j < nj) {
                    const int64_t js = sorted[p0 + j];
                    float* r = stage + j * REC;
                    if (part < 3) {
                        // the origin the binning pass used, and the weights about it
                        const int o = (bn.org[(int64_t)b * a.m + js] >> (10 * part)) & 1023;
                        const float4 p = a.pos[js];
                        const float y = a.sign * (Rm[3 * part] * p.x + Rm[3 * part + 1] * p.y + Rm[3 * part + 2] * p.z);
                        const float g = y * a.inv_h;
                        const int u0 = o - a.s_h;
#pragma unroll
                        for (int q = 0; q < W; ++q) {
                            const float zz = ((float)(u0 + q) - g) * (2.f / W);
                            const float z2 = zz * zz;
                            r[part * W + q] = (z2 <= 1.f) ? exp(a.beta * (sqrt(1.f - z2) - 1.f)) : 0.f;
                        }
                        r[SX_O_ORG + part] = __int_as_float(o);
                    } else {
                        const float2 c = a.c[js];
                        r[SX_O_C] = c.x * scale;
                        r[SX_O_C + 1] = c.y * scale;
                    }
                }
            }
            __syncthreads();
            // the warps add the staged samples round-robin, lanes on consecutive taps
            // of the sample's tap box clipped to this CTA's rows
            for (int j = warp; j < nj; j += NWARP) {
                const float* r = stage + j * REC;
                const int ox = __float_as_int(r[SX_O_ORG]);
                const int oy = __float_as_int(r[SX_O_ORG + 1]);
                const int oz = __float_as_int(r[SX_O_ORG + 2]);
                const int ly = max(0, y0 - oy), hy = min(W, y0 + TY - oy);
                const int lz = max(0, z0 - oz), hz = min(W, z0 + TZ - oz);
                const int ny = hy - ly, nz = hz - lz;
                if (ny <= 0 || nz <= 0) continue;  // uniform over the warp
                const int ntaps = W * ny * nz;
                const int base = ((oz + lz - z0) * TY + (oy + ly - y0)) * px + ox;
                const float cx = r[SX_O_C], cy = r[SX_O_C + 1];
                const unsigned char* dv = divtab[ny];
#pragma unroll
                for (int q = 0; q < ROUNDS; ++q) {
                    if (q * 32 >= ntaps) break;  // uniform over the warp
                    if (q * 32 + lane < ntaps) {
                        const int d = dv[rho_of[q]];
                        const int ky = d & 15, kz = d >> 4;
                        const int kx = kx_of[q];
                        const int cell = base + kx + (kz * TY + ky) * px;
                        const float w = r[kx] * r[W + ly + ky] * r[2 * W + lz + kz];
                        atomicAdd(tre + cell, __float_as_int(fmaf(cx, w, MAGIC)) - MAGIC_BITS);
                        atomicAdd(tim + cell, __float_as_int(fmaf(cy, w, MAGIC)) - MAGIC_BITS);
                    }
                }
            }
            __syncthreads();  // the stage is refilled by the next chunk
        }
    }
    // forward x transform of the rows, TR at a time (row l: y = y0 + l % TY, z = z0 + l / TY)
    const float2 zero = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int g = 0; g < ROWS / TR; ++g) {
        auto load = [&](int line, int i, int r) -> float2 {
            const int l = g * TR + line;
            const int pos = i + r * NB1;
            const int y = y0 + l % TY, z = z0 + l / TY;
            if (y >= s || z >= s || pos >= s) return zero;
            return make_float2((float)tre[l * px + pos] * inv_scale, (float)tim[l * px + pos] * inv_scale);
        };
        auto emit = [&](int line, int i, int r, float2 v) {
            const int l = g * TR + line;
            const int y = y0 + l % TY, z = z0 + l / TY;
            if (kept_out<LEN>(r) && y < s && z < s)
                outb[((int64_t)z * s + y) * NH + i + kept_slot<LEN>(r)] = v;
        };
        fftp_lines<float2, LEN, false, TR, NT, LAY_ROW, true, false, true>(buf, LD, tw, load, emit);
        __syncthreads();  // buf is rewritten by the next group
    }
}

// ---------------------------------------------------------------------------
// line passes: the first FFT stage reads global memory into registers and the
// last stage writes global memory from registers; stages in between (and the
// product step of the fused pass) go through shared memory
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void argmax_merge(T& best, int& bidx, T v, int i) {
    if (v > best || (v == best && i < bidx)) {
        best = v;
        bidx = i;
    }
}

// Block-wide (max value, lowest index); the result is valid in thread 0.
template <typename T>
__device__ __forceinline__ void block_argmax(T& best, int& bidx) {
    __shared__ T wb[32];
    __shared__ int wi[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const T ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
        argmax_merge(best, bidx, ob, oi);
    }
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
            argmax_merge(best, bidx, ob, oi);
        }
    }
}

// Row passes: TR consecutive rows of one rotation per CTA.
template <typename T, int LEN, int MODE>
__device__ __forceinline__ void rows_body(const RowArgs<T>& a) {
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
    __syncthreads();
    const C* in = a.in + (int64_t)b * a.in_rot_stride;
    C* out = a.out + (int64_t)b * a.out_rot_stride;
    const C zero = mk(T(0), T(0));
    const int N = a.N, hN = N >> 1;
    auto load = [&](int line, int pos) -> C {
        const int row = row0 + line;
        if (row >= a.nrows) return zero;
        const C* src = in + (int64_t)row * a.in_row_stride;
        if constexpr (MODE == ROW_FWD) {
            int e = pos + a.s_h;
            if (e >= LEN) e -= LEN;
            return e < a.len_in ? src[e] : zero;
        } else if constexpr (MODE == ROW_EXPAND) {
            const int e = pos < hN ? pos : (pos >= LEN - hN ? pos - LEN + N : -1);
            return e >= 0 ? src[e] : zero;
        } else {
            return src[pos];
        }
    };
    T best = -INFINITY;
    int bidx = INT_MAX;
    auto emit = [&](int line, int o, C v) {
        const int row = row0 + line;
        if (row >= a.nrows) return;
        if constexpr (MODE == ROW_FWD) {
            const int kp = o < hN ? o : (o >= LEN - hN ? o - LEN + N : -1);
            if (kp >= 0) out[(int64_t)row * a.out_row_stride + kp] = v;
        } else if constexpr (MODE == ROW_INV_ARGMAX) {
            argmax_merge(best, bidx, v.x, row * LEN + o);
        } else {
            out[(int64_t)row * a.out_row_stride + o] = v;
        }
    };
    fft_lines_io<C, LEN, INV, TR, cta_threads<T, LEN>(), LAY_ROW, false>(buf, LD, tw, load, emit);
    if constexpr (MODE == ROW_INV_ARGMAX) {
        block_argmax(best, bidx);
        if (threadIdx.x == 0) {
            const int64_t o = (int64_t)b * gridDim.x + blockIdx.x;
            a.part_score[o] = (double)best;
            a.part_idx[o] = bidx;
        }
    }
}

template <typename T, int LEN, int MODE>
__global__ void __launch_bounds__(cta_threads<T, LEN>()) k_rows(RowArgs<T> a) {
    rows_body<T, LEN, MODE>(a);
}

template <typename T, int LEN, int MODE, int MB>
__global__ void __launch_bounds__(cta_threads<T, LEN>(), MB) k_rows_mb(RowArgs<T> a) {
    rows_body<T, LEN, MODE>(a);
}

// Column passes: TC adjacent columns of one (rotation, outer) slab per CTA.
template <typename T, int LENF, int LENI, int MODE>
__device__ __forceinline__ void cols_body(const ColArgs<T>& a) {
    using C = cplx<T>;
    constexpr int TC = lines_per_cta<T, LENF>();
    constexpr int NT = cta_threads<T, LENF>();
    constexpr int LD = line_pitch(LENF);
    constexpr int NTWF = tw_count(LENF);
    constexpr int NTWI = (MODE == COL_FUSED) ? tw_count(LENI) : 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* twF = buf + TC * LD;
    C* twI = twF + NTWF;
    // a fused pass whose W is too large to stay in L2 runs rotations fastest (grid
    // (batch, column blocks)), so the CTAs that read one block of W for every
    // rotation of a batch run together and W comes from L2; every other pass runs
    // column blocks fastest (grid (blocks, outer, batch))
    const bool rf = MODE == COL_FUSED && a.rot_fastest;
    const int b = rf ? (int)blockIdx.x : (int)blockIdx.z;
    const int outer = rf ? 0 : (int)blockIdx.y;
    const int col0 = (rf ? (int)blockIdx.y : (int)blockIdx.x) * TC;
    for (int j = threadIdx.x; j < NTWF; j += blockDim.x) twF[j] = a.twF[j];
    if constexpr (MODE == COL_FUSED)
        for (int j = threadIdx.x; j < NTWI; j += blockDim.x) twI[j] = a.twI[j];
    __syncthreads();
    const int ncols = a.ncols;
    const C* in = a.in + (int64_t)b * a.in_rot_stride + (int64_t)outer * a.in_outer_stride;
    C* out = a.out + (int64_t)b * a.out_rot_stride + (int64_t)outer * a.out_outer_stride;
    const C zero = mk(T(0), T(0));
    const int N = a.N, hN = N >> 1;
    constexpr bool INV1 = (MODE == COL_INV || MODE == COL_EXPAND);
    auto load = [&](int line, int pos) -> C {
        const int gcol = col0 + line;
        if (gcol >= ncols) return zero;
        int e;
        if constexpr (MODE == COL_FWD || MODE == COL_FUSED) {
            e = pos + a.s_h;
            if (e >= LENF) e -= LENF;
            if (e >= a.len_in) return zero;
        } else if constexpr (MODE == COL_EXPAND) {
            e = pos < hN ? pos : (pos >= LENF - hN ? pos - LENF + N : -1);
            if (e < 0) return zero;
        } else {
            e = pos;
        }
        return in[e * ncols + gcol];  // offsets within one rotation's slab: below 2^31
    };
    if constexpr (MODE == COL_FUSED) {
        // forward: keep the N central modes, multiply by W, place them as the
        // inverse transform's inputs
        auto emit_fwd = [&](int line, int o, C v) {
            const int kp = o < hN ? o : (o >= LENF - hN ? o - LENF + N : -1);
            const int gcol = col0 + line;
            if (kp >= 0 && gcol < ncols) buf[line * LD + pad(kp)] = cmul(v, a.W[kp * ncols + gcol]);
        };
        fft_lines_io<C, LENF, false, TC, NT, LAY_COL, false>(buf, LD, twF, load, emit_fwd);
        __syncthreads();
        auto emit_out = [&](int line, int o, C v) {
            const int gcol = col0 + line;
            if (gcol < ncols) out[o * ncols + gcol] = v;
        };
        fft_lines_io<C, LENI, true, TC, NT, LAY_COL, true>(buf, LD, twI, load, emit_out);
    } else {
        auto emit = [&](int line, int o, C v) {
            const int gcol = col0 + line;
            if (gcol >= ncols) return;
            if constexpr (MODE == COL_FWD) {
                const int kp = o < hN ? o : (o >= LENF - hN ? o - LENF + N : -1);
                if (kp >= 0) out[kp * ncols + gcol] = v;
            } else {
                out[o * ncols + gcol] = v;
            }
        };
        fft_lines_io<C, LENF, INV1, TC, NT, LAY_COL, false>(buf, LD, twF, load, emit);
    }
}

template <typename T, int LENF, int LENI, int MODE>
__global__ void __launch_bounds__(cta_threads<T, LENF>()) k_cols(ColArgs<T> a) {
    cols_body<T, LENF, LENI, MODE>(a);
}

template <typename T, int LENF, int LENI, int MODE, int MB>
__global__ void __launch_bounds__(cta_threads<T, LENF>(), MB) k_cols_mb(ColArgs<T> a) {
    cols_body<T, LENF, LENI, MODE>(a);
}

// ---------------------------------------------------------------------------
// pruned search passes: the sub-box is loaded unshifted (cell a at position a,
// a < s <= n/2) and the forward passes keep only the N = n/2 central modes,
// both decided at compile time (fftp.cuh); the shift of the sub-box to the
// centred grid, exp(2 pi i kappa s_h / n) per axis, is folded into the product
// table of the fused pass (k_wshift)
// ---------------------------------------------------------------------------

// Pitch of an unpadded column line in shared memory (odd: lanes on consecutive
// lines hit distinct banks).
__host__ __device__ constexpr int col_pitch(int len) { return len + 1; }

// x pass: rows of the sub-box -> N modes per row (row stride N = LEN/2).
template <typename T, int LEN>
__device__ __forceinline__ void rows_fwd_p_body(const RowArgs<T>& a) {
    using C = cplx<T>;
    constexpr int TR = lines_per_cta<T, LEN>();
    constexpr int LD = line_pitch(LEN);
    constexpr int NTW = tw_count(LEN);
    constexpr int NB1 = LEN / plan_radix(LEN, 0);
    constexpr int NH = LEN / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + TR * LD;
    const int row0 = blockIdx.x * TR;
    for (int j = threadIdx.x; j < NTW; j += blockDim.x) tw[j] = a.tw[j];
    __syncthreads();
    const int rs = a.in_row_stride;
    const C* in = a.in + (int64_t)blockIdx.y * a.in_rot_stride + (int64_t)row0 * rs;
    C* out = a.out + (int64_t)blockIdx.y * a.out_rot_stride + (int64_t)row0 * NH;
    const int nrows = a.nrows - row0;
    const int s = a.len_in;
    const C zero = mk(T(0), T(0));
    auto load = [&](int line, int i, int r) -> C {
        const int pos = i + r * NB1;
        return (line < nrows && pos < s) ? in[line * rs + pos] : zero;
    };
    auto emit = [&](int line, int i, int r, C v) {
        if (kept_out<LEN>(r) && line < nrows) out[line * NH + i + kept_slot<LEN>(r)] = v;
    };
    fftp_lines<C, LEN, false, TR, cta_threads<T, LEN>(), LAY_ROW, true, false, true>(buf, LD, tw, load, emit);
}

template <typename T, int LEN, int MB>
__global__ void __launch_bounds__(cta_threads<T, LEN>(), MB) k_rows_fwd_p(RowArgs<T> a) {
    rows_fwd_p_body<T, LEN>(a);
}

// y pass (3D): columns (one per kept x mode) of each z plane -> N modes, TC
// columns per CTA.
template <typename T, int LEN, int TC>
__device__ __forceinline__ void cols_fwd_p_body(const ColArgs<T>& a) {
    using C = cplx<T>;
    constexpr int NT = cta_threads_for<LEN>(TC);
    constexpr int LD = col_pitch(LEN);
    constexpr int NTW = tw_count(LEN);
    constexpr int NB1 = LEN / plan_radix(LEN, 0);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + TC * LD;
    const int col0 = blockIdx.x * TC;
    for (int j = threadIdx.x; j < NTW; j += blockDim.x) tw[j] = a.twF[j];
    __syncthreads();
    const int ncols = a.ncols;
    const int ncl = ncols - col0;
    const C* in = a.in + (int64_t)blockIdx.z * a.in_rot_stride + (int64_t)blockIdx.y * a.in_outer_stride + col0;
    C* out = a.out + (int64_t)blockIdx.z * a.out_rot_stride + (int64_t)blockIdx.y * a.out_outer_stride + col0;
    const int s = a.len_in;
    const C zero = mk(T(0), T(0));
    auto load = [&](int line, int i, int r) -> C {
        const int pos = i + r * NB1;
        return (line < ncl && pos < s) ? in[pos * ncols + line] : zero;
    };
    auto emit = [&](int line, int i, int r, C v) {
        if (kept_out<LEN>(r) && line < ncl) out[(i + kept_slot<LEN>(r)) * ncols + line] = v;
    };
    fftp_lines<C, LEN, false, TC, NT, LAY_COL, false, false, true>(buf, LD, tw, load, emit);
}

template <typename T, int LEN, int MB, int TC>
__global__ void __launch_bounds__(cta_threads_for<LEN>(TC), MB) k_cols_fwd_p(ColArgs<T> a) {
    cols_fwd_p_body<T, LEN, TC>(a);
}

// Last axis: pruned forward FFT of length LENF, times the shifted product table
// W' (N x ncols), inverse FFT of length LENF/2 in the same block; TC columns
// per CTA.
template <typename T, int LENF, int TC>
__device__ __forceinline__ void cols_fused_p_body(const ColArgs<T>& a) {
    using C = cplx<T>;
    constexpr int LENI = LENF / 2;
    constexpr int NT = cta_threads_for<LENF>(TC);
    constexpr int LD = col_pitch(LENF);
    constexpr int NTWF = tw_count(LENF);
    constexpr int NTWI = tw_count(LENI);
    constexpr int NB1 = LENF / plan_radix(LENF, 0);
    constexpr int PI = LENI / plan_last_radix(LENI);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* twF = buf + TC * LD;
    C* twI = twF + NTWF;
    const bool rf = a.rot_fastest;
    const int b = rf ? (int)blockIdx.x : (int)blockIdx.z;
    const int col0 = (rf ? (int)blockIdx.y : (int)blockIdx.x) * TC;
    for (int j = threadIdx.x; j < NTWF; j += blockDim.x) twF[j] = a.twF[j];
    for (int j = threadIdx.x; j < NTWI; j += blockDim.x) twI[j] = a.twI[j];
    __syncthreads();
    const int ncols = a.ncols;
    const int ncl = ncols - col0;
    const C* in = a.in + (int64_t)b * a.in_rot_stride + col0;
    C* out = a.out + (int64_t)b * a.out_rot_stride + col0;
    const C* Wc = a.W + col0;
    const int s = a.len_in;
    const C zero = mk(T(0), T(0));
    auto load = [&](int line, int i, int r) -> C {
        const int pos = i + r * NB1;
        return (line < ncl && pos < s) ? in[pos * ncols + line] : zero;
    };
    auto emit_fwd = [&](int line, int i, int r, C v) {
        if (kept_out<LENF>(r) && line < ncl) {
            const int kp = i + kept_slot<LENF>(r);
            buf[line * LD + kp] = cmul(v, Wc[kp * ncols + line]);
        }
    };
    fftp_lines<C, LENF, false, TC, NT, LAY_COL, false, false, true>(buf, LD, twF, load, emit_fwd);
    __syncthreads();
    auto emit_out = [&](int line, int i, int r, C v) {
        if (line < ncl) out[(i + r * PI) * ncols + line] = v;
    };
    fftp_lines<C, LENI, true, TC, NT, LAY_COL, false, true, false>(buf, LD, twI, load, emit_out);
}

template <typename T, int LENF, int MB, int TC>
__global__ void __launch_bounds__(cta_threads_for<LENF>(TC), MB) k_cols_fused_p(ColArgs<T> a) {
    cols_fused_p_body<T, LENF, TC>(a);
}

// Inverse y (3D), in place: columns of N points, full input and output.  Each
// CTA reads its columns completely in the first stage before any write.
// The inverse y and x passes of 192-point FP32 lines are bounded for six CTAs per
// SM (at most 40 registers, no spills; 44 otherwise, which allows five).
template <typename T, int LEN>
__host__ __device__ constexpr int rows_inv_min_ctas() {
    return (sizeof(T) == 4 && (LEN == 192 || LEN == 128)) ? 6 : 0;
}

template <typename T, int LEN>
__device__ __forceinline__ void cols_inv_p_body(const ColArgs<T>& a) {
    using C = cplx<T>;
    constexpr int TC = lines_per_cta<T, LEN>();
    constexpr int NT = cta_threads<T, LEN>();
    constexpr int LD = col_pitch(LEN);
    constexpr int NTW = tw_count(LEN);
    constexpr int NB1 = LEN / plan_radix(LEN, 0);
    constexpr int PL = LEN / plan_last_radix(LEN);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + TC * LD;
    const int col0 = blockIdx.x * TC;
    for (int j = threadIdx.x; j < NTW; j += blockDim.x) tw[j] = a.twF[j];
    __syncthreads();
    const int ncols = a.ncols;
    const int ncl = ncols - col0;
    const C* in = a.in + (int64_t)blockIdx.z * a.in_rot_stride + (int64_t)blockIdx.y * a.in_outer_stride + col0;
    C* out = a.out + (int64_t)blockIdx.z * a.out_rot_stride + (int64_t)blockIdx.y * a.out_outer_stride + col0;
    const C zero = mk(T(0), T(0));
    auto load = [&](int line, int i, int r) -> C { return line < ncl ? in[(i + r * NB1) * ncols + line] : zero; };
    auto emit = [&](int line, int i, int r, C v) {
        if (line < ncl) out[(i + r * PL) * ncols + line] = v;
    };
    fftp_lines<C, LEN, true, TC, NT, LAY_COL, false, false, false>(buf, LD, tw, load, emit);
}

template <typename T, int LEN>
__global__ void __launch_bounds__(cta_threads<T, LEN>(), rows_inv_min_ctas<T, LEN>()) k_cols_inv_p(ColArgs<T> a) {
    cols_inv_p_body<T, LEN>(a);
}

// Inverse x of rows of N points: the per-block argmax of the real part (ties to
// the lowest index) or the complex map.
template <typename T, int LEN, int MODE>
__device__ __forceinline__ void rows_inv_p_body(const RowArgs<T>& a) {
    using C = cplx<T>;
    constexpr int TR = lines_per_cta<T, LEN>();
    constexpr int LD = line_pitch(LEN);
    constexpr int NTW = tw_count(LEN);
    constexpr int NB1 = LEN / plan_radix(LEN, 0);
    constexpr int PL = LEN / plan_last_radix(LEN);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + TR * LD;
    const int row0 = blockIdx.x * TR;
    for (int j = threadIdx.x; j < NTW; j += blockDim.x) tw[j] = a.tw[j];
    __syncthreads();
    const C* in = a.in + (int64_t)blockIdx.y * a.in_rot_stride + (int64_t)row0 * LEN;
    const int nrows = a.nrows - row0;
    const C zero = mk(T(0), T(0));
    auto load = [&](int line, int i, int r) -> C { return line < nrows ? in[line * LEN + i + r * NB1] : zero; };
    T best = -INFINITY;
    int bidx = INT_MAX;
    C* out = (MODE == ROW_INV_MAP) ? a.out + (int64_t)blockIdx.y * a.out_rot_stride + (int64_t)row0 * LEN : nullptr;
    // one last-stage butterfly per thread: its outputs come in increasing index
    // order, so a strict comparison already keeps the lowest index of equal values
    constexpr bool one_bfly = TR * (LEN / plan_last_radix(LEN)) <= cta_threads<T, LEN>();
    auto emit = [&](int line, int i, int r, C v) {
        if (line >= nrows) return;
        if constexpr (MODE == ROW_INV_ARGMAX) {
            if constexpr (one_bfly) {
                if (v.x > best) {
                    best = v.x;
                    bidx = (row0 + line) * LEN + i + r * PL;
                }
            } else {
                argmax_merge(best, bidx, v.x, (row0 + line) * LEN + i + r * PL);
            }
        } else {
            out[line * LEN + i + r * PL] = v;
        }
    };
    fftp_lines<C, LEN, true, TR, cta_threads<T, LEN>(), LAY_ROW, true, false, false>(buf, LD, tw, load, emit);
    if constexpr (MODE == ROW_INV_ARGMAX) {
        block_argmax(best, bidx);
        if (threadIdx.x == 0) {
            const int64_t o = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
            a.part_score[o] = (double)best;
            a.part_idx[o] = bidx;
        }
    }
}


template <typename T, int LEN, int MODE>
__global__ void __launch_bounds__(cta_threads<T, LEN>(), rows_inv_min_ctas<T, LEN>()) k_rows_inv_p(RowArgs<T> a) {
    rows_inv_p_body<T, LEN, MODE>(a);
}

// ---------------------------------------------------------------------------
// inverse y and x of whole z-planes in thread-block clusters (3D search)
// ---------------------------------------------------------------------------
//
// The N x N plane (ky, kx) of one rotation at one z is shared by the IYX_CS CTAs
// of a cluster.  CTA q runs the inverse y transform of the N / IYX_CS columns kx
// in [q N / IYX_CS, (q + 1) N / IYX_CS) in its shared memory, then sends each
// transformed value (y, kx) to the row buffer of the CTA that owns row y
// (distributed shared memory stores); after one cluster barrier every CTA holds
// its N / IYX_CS whole rows and runs the inverse x transform on them from its
// own shared memory.  The plane's intermediate never returns to device memory:
// one read of N^3 per rotation instead of a read, a write and a read.  Both
// buffers take an odd pitch (lanes across lines) and the twiddles are read
// from device memory (L1), which keeps a CTA within a third of an SM's shared
// memory.  Output as the inverse x pass: the map's rows, or each CTA's (max Re,
// lowest index) partial.

constexpr int IYX_CS = 8;  // CTAs per cluster (the portable maximum)

template <typename T, int LEN>
__host__ __device__ constexpr int iyx_lines() { return LEN / IYX_CS; }
template <typename T, int LEN>
__host__ __device__ constexpr int iyx_threads() { return cta_threads_for<LEN>(iyx_lines<T, LEN>()); }
// The register cap of three CTAs per SM where that leaves room for a radix-24
// stage (0: the compiler's choice).
template <typename T, int LEN>
__host__ __device__ constexpr int iyx_min_ctas() {
    return (sizeof(T) == 4 && iyx_threads<T, LEN>() == 384) ? 3 : 0;
}

template <typename T, int LEN, int MODE>
__global__ void __cluster_dims__(IYX_CS, 1, 1) __launch_bounds__(iyx_threads<T, LEN>(), iyx_min_ctas<T, LEN>())
    k_inv_yx(RowArgs<T> a) {
    using C = cplx<T>;
    constexpr int NL = iyx_lines<T, LEN>();  // columns, then rows, of this CTA
    constexpr int NT = iyx_threads<T, LEN>();
    constexpr int LD = col_pitch(LEN);       // both buffers: line * LD + position
    constexpr int NB1 = LEN / plan_radix(LEN, 0);
    constexpr int PL = LEN / plan_last_radix(LEN);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* cols = reinterpret_cast<C*>(smem_raw);  // this CTA's columns: cols[c * LD + y]
    C* rows = cols + NL * LD;                   // this CTA's rows: rows[y_local * LD + kx]
    const C* tw = a.tw;
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    cl.barrier_arrive();  // this CTA runs (its rows may receive remote stores)
    const int q = (int)cl.block_rank();
    const int z = (int)blockIdx.x / IYX_CS;
    const int c0 = q * NL;  // this CTA's first column, then first row
    const C* plane = a.in + (int64_t)blockIdx.y * a.in_rot_stride + (int64_t)z * LEN * LEN;  // [ky][kx]
    // inverse y of columns c0 .. c0 + NL - 1 (lanes across columns: coalesced)
    auto load_y = [&](int line, int i, int r) -> C { return plane[(int64_t)(i + r * NB1) * LEN + c0 + line]; };
    auto emit_y = [&](int line, int i, int r, C v) { cols[line * LD + i + r * PL] = v; };
    fftp_lines<C, LEN, true, NL, NT, LAY_COL, false, false, false>(cols, LD, tw, load_y, emit_y);
    __syncthreads();
    cl.barrier_wait();  // every CTA of the cluster runs
    // send (y, c0 + c) to the owner of row y: lanes on consecutive columns of a row
    for (int e = threadIdx.x; e < NL * LEN; e += NT) {
        const int y = e / NL, c = e - y * NL;
        C* dst = cl.map_shared_rank(rows, y / NL);
        dst[(y % NL) * LD + c0 + c] = cols[c * LD + y];
    }
    cl.sync();  // every row is complete
    // inverse x of rows c0 .. c0 + NL - 1 from this CTA's row buffer
    auto load_none = [&](int, int, int) -> C { return mk(T(0), T(0)); };
    T best = -INFINITY;
    int bidx = INT_MAX;
    const int64_t row0 = (int64_t)z * LEN + c0;  // row (z, y) of the rotation's map
    C* out = (MODE == ROW_INV_MAP) ? a.out + (int64_t)blockIdx.y * a.out_rot_stride + row0 * LEN : nullptr;
    auto emit_x = [&](int line, int i, int r, C v) {
        if constexpr (MODE == ROW_INV_ARGMAX) argmax_merge(best, bidx, v.x, (int)((row0 + line) * LEN) + i + r * PL);
        else out[line * LEN + i + r * PL] = v;
    };
    fftp_lines<C, LEN, true, NL, NT, LAY_COL, false, true, false>(rows, LD, tw, load_none, emit_x);
    if constexpr (MODE == ROW_INV_ARGMAX) {
        block_argmax(best, bidx);
        if (threadIdx.x == 0) {
            const int64_t o = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
            a.part_score[o] = (double)best;
            a.part_idx[o] = bidx;
        }
    }
}

// Inverse x of rows of N points keeping each block's K best translations of the
// real part (score descending, index ascending): a sorted list per thread, merged
// through shared memory after the transform; partials are K per block.
template <typename T, int LEN, int K>
__device__ __forceinline__ void rows_inv_topk_body(const RowArgs<T>& a) {
    using C = cplx<T>;
    constexpr int TR = lines_per_cta<T, LEN>();
    constexpr int NT = cta_threads<T, LEN>();
    constexpr int LD = line_pitch(LEN);
    constexpr int NTW = tw_count(LEN);
    constexpr int NB1 = LEN / plan_radix(LEN, 0);
    constexpr int PL = LEN / plan_last_radix(LEN);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + TR * LD;
    T* sv = reinterpret_cast<T*>(tw + NTW);
    int* si = reinterpret_cast<int*>(sv + NT * K);
    __shared__ T wv[32], bestv[K];
    __shared__ int wi[32], besti[K];
    const int row0 = blockIdx.x * TR;
    for (int j = threadIdx.x; j < NTW; j += blockDim.x) tw[j] = a.tw[j];
    __syncthreads();
    const C* in = a.in + (int64_t)blockIdx.y * a.in_rot_stride + (int64_t)row0 * LEN;
    const int nrows = a.nrows - row0;
    const C zero = mk(T(0), T(0));
    auto load = [&](int line, int i, int r) -> C { return line < nrows ? in[line * LEN + i + r * NB1] : zero; };
    TopK<T, K> top;
    top.init();
    auto emit = [&](int line, int i, int r, C v) {
        if (line < nrows) top.push(v.x, (row0 + line) * LEN + i + r * PL);
    };
    fftp_lines<C, LEN, true, TR, NT, LAY_ROW, true, false, false>(buf, LD, tw, load, emit);
    block_topk_merge<T, K>(top, sv, si, wv, wi, bestv, besti);
    if (threadIdx.x < K) {
        const int64_t o = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * K + threadIdx.x;
        a.part_score[o] = (double)bestv[threadIdx.x];
        a.part_idx[o] = besti[threadIdx.x];
    }
}

template <typename T, int LEN, int K>
__global__ void __launch_bounds__(cta_threads<T, LEN>()) k_rows_inv_topk(RowArgs<T> a) {
    rows_inv_topk_body<T, LEN, K>(a);
}

// Resident CTAs per SM the pruned passes are compiled for (0: the compiler's choice).
// 512-point FP32 lines (256 threads, two butterflies each) take 2 (at most 128
// registers; 146 otherwise); 384-point ones 3 (384 threads: at most 56).
template <typename T, int LEN, int KIND>
__host__ __device__ constexpr int pruned_min_ctas() {
    return sizeof(T) != 4 ? 0 : (LEN == 512 ? 2 : (LEN == 384 ? 3 : 0));
}
// The standard fused pass of 256-point FP32 lines: six CTAs per SM (40 registers,
// no spills; 44 otherwise, which allows five).
template <typename T, int LENF>
__host__ __device__ constexpr int fused_std_min_ctas() {
    return (sizeof(T) == 4 && LENF == 256) ? 6 : pruned_min_ctas<T, LENF, 2>();
}

// Other widths of the pruned column passes (forward y and the fused last axis)
// for FP32 lines of 128 to 384 points: the narrow plan takes half the columns
// per CTA (twice the CTAs, half the shared memory each, 64-byte row segments),
// the wide plan twice (256-byte row segments, up to 99 KB of shared memory).
// Their register bound keeps the per-thread cap of the standard plan.
template <typename T, int LEN>
__host__ __device__ constexpr bool alt_cols_ok() {
    return sizeof(T) == 4 && LEN >= 128 && LEN <= 384;
}
template <typename T, int LEN, int WIDE>
__host__ __device__ constexpr int alt_lines() {
    return WIDE ? 2 * lines_per_cta<T, LEN>() : lines_per_cta<T, LEN>() / 2;
}
template <typename T, int LEN, int KIND, int WIDE>
__host__ __device__ constexpr int alt_min_ctas() {
    return pruned_min_ctas<T, LEN, KIND>() * cta_threads<T, LEN>() / cta_threads_for<LEN>(alt_lines<T, LEN, WIDE>());
}

// W' = W exp(2 pi i s_h (kx + ky [+ kz]) / n) with kappa signed (modes at kappa mod N).
template <typename T>
__global__ void k_wshift(const cplx<T>* W, int N, int dim, int n, int s_h, cplx<T>* out) {
    const int64_t tot = (dim == 2) ? (int64_t)N * N : (int64_t)N * N * N;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tot) return;
    int64_t r = i;
    int64_t ksum = 0;
    for (int d = 0; d < dim; ++d) {
        const int kp = (int)(r % N);
        r /= N;
        ksum += kp < N / 2 ? kp : kp - N;
    }
    // exp(2 pi i ksum s_h / n): reduce the integer ksum * s_h mod n first (exact)
    int64_t e = (ksum * s_h) % n;
    if (e < 0) e += n;
    double sn, cs;
    sincospi(2.0 * (double)e / (double)n, &sn, &cs);
    const double wr = (double)W[i].x, wi = (double)W[i].y;
    out[i] = mk(T(wr * cs - wi * sn), T(wr * sn + wi * cs));
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

template <typename T, int LEN, int MODE>
static cudaError_t rows_impl(const RowArgs<T>& a, int batch, int* nparts, cudaStream_t st) {
    using C = cplx<T>;
    constexpr int TR = lines_per_cta<T, LEN>();
    const int nb = (a.nrows + TR - 1) / TR;
    if (nparts) *nparts = nb;
    if (nb == 0 || batch == 0) return cudaSuccess;
    const size_t smem = (size_t)(TR * line_pitch(LEN) + tw_count(LEN)) * sizeof(C);
    void (*kern)(RowArgs<T>);
    if constexpr (min_ctas_per_sm<T, LEN>() > 0) kern = k_rows_mb<T, LEN, MODE, min_ctas_per_sm<T, LEN>()>;
    else kern = k_rows<T, LEN, MODE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, batch), cta_threads<T, LEN>(), smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int LENF, int LENI, int MODE>
static cudaError_t cols_impl(const ColArgs<T>& a, int batch, cudaStream_t st) {
    using C = cplx<T>;
    constexpr int TC = lines_per_cta<T, LENF>();
    const int nb = (a.ncols + TC - 1) / TC;
    if (nb == 0 || batch == 0 || a.nouter == 0) return cudaSuccess;
    const size_t smem = (size_t)(TC * line_pitch(LENF) + tw_count(LENF) + tw_count(LENI)) * sizeof(C);
    void (*kern)(ColArgs<T>);
    if constexpr (min_ctas_per_sm_cols<T, LENF, MODE>() > 0)
        kern = k_cols_mb<T, LENF, LENI, MODE, min_ctas_per_sm_cols<T, LENF, MODE>()>;
    else kern = k_cols<T, LENF, LENI, MODE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const bool rf = MODE == COL_FUSED && a.rot_fastest;
    const dim3 grid = rf ? dim3(batch, nb, 1) : dim3(nb, a.nouter, batch);
    if (rf && (a.nouter != 1 || nb > 65535)) return cudaErrorInvalidValue;
    kern<<<grid, cta_threads<T, LENF>(), smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

// Lengths the pruned passes are built for (prunable_len).
#define SD_FOR_EACH_PLEN(X) X(16) X(32) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

template <typename T, int LEN>
static cudaError_t rows_fwd_p_impl(const RowArgs<T>& a, int batch, cudaStream_t st) {
    using C = cplx<T>;
    static_assert(prunable_len(LEN), "length not prunable");
    constexpr int TR = lines_per_cta<T, LEN>();
    const int nb = (a.nrows + TR - 1) / TR;
    if (nb == 0 || batch == 0) return cudaSuccess;
    const size_t smem = (size_t)(TR * line_pitch(LEN) + tw_count(LEN)) * sizeof(C);
    auto kern = k_rows_fwd_p<T, LEN, pruned_min_ctas<T, LEN, 0>()>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, batch), cta_threads<T, LEN>(), smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int LEN, int TC, int MB>
static cudaError_t cols_fwd_p_launch(const ColArgs<T>& a, int batch, cudaStream_t st) {
    using C = cplx<T>;
    const int nb = (a.ncols + TC - 1) / TC;
    if (nb == 0 || batch == 0 || a.nouter == 0) return cudaSuccess;
    const size_t smem = (size_t)(TC * col_pitch(LEN) + tw_count(LEN)) * sizeof(C);
    auto kern = k_cols_fwd_p<T, LEN, MB, TC>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, a.nouter, batch), cta_threads_for<LEN>(TC), smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int LEN>
static cudaError_t cols_fwd_p_impl(const ColArgs<T>& a, int batch, cudaStream_t st) {
    static_assert(prunable_len(LEN), "length not prunable");
    if constexpr (alt_cols_ok<T, LEN>()) {
        if (a.lines == LINES_NARROW)
            return cols_fwd_p_launch<T, LEN, alt_lines<T, LEN, 0>(), alt_min_ctas<T, LEN, 1, 0>()>(a, batch, st);
        if (a.lines == LINES_WIDE)
            return cols_fwd_p_launch<T, LEN, alt_lines<T, LEN, 1>(), alt_min_ctas<T, LEN, 1, 1>()>(a, batch, st);
    }
    if (a.lines != LINES_STD) return cudaErrorInvalidValue;
    return cols_fwd_p_launch<T, LEN, lines_per_cta<T, LEN>(), pruned_min_ctas<T, LEN, 1>()>(a, batch, st);
}

template <typename T, int LENF, int TC, int MB>
static cudaError_t cols_fused_p_launch(const ColArgs<T>& a, int batch, cudaStream_t st) {
    using C = cplx<T>;
    const int nb = (a.ncols + TC - 1) / TC;
    if (nb == 0 || batch == 0) return cudaSuccess;
    if (a.nouter != 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(TC * col_pitch(LENF) + tw_count(LENF) + tw_count(LENF / 2)) * sizeof(C);
    auto kern = k_cols_fused_p<T, LENF, MB, TC>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const bool rf = a.rot_fastest;
    if (rf && nb > 65535) return cudaErrorInvalidValue;
    const dim3 grid = rf ? dim3(batch, nb, 1) : dim3(nb, 1, batch);
    kern<<<grid, cta_threads_for<LENF>(TC), smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int LENF>
static cudaError_t cols_fused_p_impl(const ColArgs<T>& a, int batch, cudaStream_t st) {
    static_assert(prunable_len(LENF), "length not prunable");
    if constexpr (alt_cols_ok<T, LENF>()) {
        if (a.lines == LINES_NARROW)
            return cols_fused_p_launch<T, LENF, alt_lines<T, LENF, 0>(), alt_min_ctas<T, LENF, 2, 0>()>(a, batch, st);
        if (a.lines == LINES_WIDE)
            return cols_fused_p_launch<T, LENF, alt_lines<T, LENF, 1>(), alt_min_ctas<T, LENF, 2, 1>()>(a, batch, st);
    }
    if (a.lines != LINES_STD) return cudaErrorInvalidValue;
    return cols_fused_p_launch<T, LENF, lines_per_cta<T, LENF>(), fused_std_min_ctas<T, LENF>()>(a, batch, st);
}

template <typename T, int LEN, int MODE>
static cudaError_t rows_inv_p_impl(const RowArgs<T>& a, int batch, int* nparts, cudaStream_t st) {
    using C = cplx<T>;
    constexpr int TR = lines_per_cta<T, LEN>();
    const int nb = (a.nrows + TR - 1) / TR;
    if (nparts) *nparts = nb;
    if (nb == 0 || batch == 0) return cudaSuccess;
    if (a.in_row_stride != LEN || (MODE == ROW_INV_MAP && a.out_row_stride != LEN)) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(TR * line_pitch(LEN) + tw_count(LEN)) * sizeof(C);
    auto kern = k_rows_inv_p<T, LEN, MODE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, batch), cta_threads<T, LEN>(), smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

// Plane lengths the cluster inverse is built for (FP32; N a multiple of IYX_CS;
// the same list as inv_yx_supported).
#define SD_FOR_EACH_IYX(X) X(32) X(48) X(64) X(96) X(128) X(192) X(256)

template <typename T, int LEN, int MODE>
static cudaError_t inv_yx_impl(const RowArgs<T>& a, int batch, int* nparts, cudaStream_t st) {
    using C = cplx<T>;
    static_assert(LEN % IYX_CS == 0, "plane length not a multiple of the cluster size");
    const int nb = IYX_CS * LEN;  // one cluster per z-plane
    if (nparts) *nparts = nb;
    if (batch == 0) return cudaSuccess;
    if (a.in_row_stride != LEN || (MODE == ROW_INV_MAP && a.out_row_stride != LEN) || a.nrows != LEN * LEN)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * iyx_lines<T, LEN>() * col_pitch(LEN) * sizeof(C);
    auto kern = k_inv_yx<T, LEN, MODE>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, batch), iyx_threads<T, LEN>(), smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_inv_yx_t(int mode, const RowArgs<T>& a, int batch, int* nparts, cudaStream_t st) {
    if constexpr (sizeof(T) != 4) {
        return cudaErrorInvalidValue;
    } else {
        if (mode != ROW_INV_ARGMAX && mode != ROW_INV_MAP) return cudaErrorInvalidValue;
        switch (a.N) {
#define SD_IYX_CASE(L)                                                                       \
    case L:                                                                                  \
        return mode == ROW_INV_ARGMAX ? inv_yx_impl<T, L, ROW_INV_ARGMAX>(a, batch, nparts, st) \
                                      : inv_yx_impl<T, L, ROW_INV_MAP>(a, batch, nparts, st);
            SD_FOR_EACH_IYX(SD_IYX_CASE)
#undef SD_IYX_CASE
        }
        return cudaErrorInvalidValue;
    }
}

template <typename T, int LEN>
static cudaError_t cols_inv_p_impl(const ColArgs<T>& a, int batch, cudaStream_t st) {
    using C = cplx<T>;
    constexpr int TC = lines_per_cta<T, LEN>();
    const int nb = (a.ncols + TC - 1) / TC;
    if (nb == 0 || batch == 0 || a.nouter == 0) return cudaSuccess;
    const size_t smem = (size_t)(TC * col_pitch(LEN) + tw_count(LEN)) * sizeof(C);
    auto kern = k_cols_inv_p<T, LEN>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, a.nouter, batch), cta_threads<T, LEN>(), smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T, int LEN, int K>
static cudaError_t rows_inv_topk_impl(const RowArgs<T>& a, int batch, int* nparts, cudaStream_t st) {
    using C = cplx<T>;
    constexpr int TR = lines_per_cta<T, LEN>();
    constexpr int NT = cta_threads<T, LEN>();
    const int nb = (a.nrows + TR - 1) / TR;
    if (nparts) *nparts = nb * K;
    if (nb == 0 || batch == 0) return cudaSuccess;
    if (a.in_row_stride != LEN) return cudaErrorInvalidValue;
    const size_t smem = (size_t)(TR * line_pitch(LEN) + tw_count(LEN)) * sizeof(C) + (size_t)NT * K * (sizeof(T) + sizeof(int));
    auto kern = k_rows_inv_topk<T, LEN, K>;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nb, batch), NT, smem, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rows_t(int mode, const RowArgs<T>& a, int batch, int* nparts, cudaStream_t st) {
    if (mode >= ROW_INV_TOPK2 && mode <= ROW_INV_TOPK16) {
        switch (a.N) {
#define SD_ROWK_CASE(L)                                                                         \
    case L:                                                                                     \
        switch (mode) {                                                                         \
            case ROW_INV_TOPK2: return rows_inv_topk_impl<T, L, 2>(a, batch, nparts, st);       \
            case ROW_INV_TOPK4: return rows_inv_topk_impl<T, L, 4>(a, batch, nparts, st);       \
            case ROW_INV_TOPK8: return rows_inv_topk_impl<T, L, 8>(a, batch, nparts, st);       \
            default: return rows_inv_topk_impl<T, L, 16>(a, batch, nparts, st);                 \
        }
            SD_ROWK_CASE(8) SD_ROWK_CASE(16) SD_ROWK_CASE(24) SD_ROWK_CASE(32) SD_ROWK_CASE(48) SD_ROWK_CASE(64)
            SD_ROWK_CASE(96) SD_ROWK_CASE(128) SD_ROWK_CASE(192) SD_ROWK_CASE(256)
#undef SD_ROWK_CASE
        }
        return cudaErrorInvalidValue;
    }
    if (mode == ROW_INV_ARGMAX || mode == ROW_INV_MAP) {
        switch (a.N) {
#define SD_ROWI_CASE(L)                                                                                    \
    case L:                                                                                                \
        return mode == ROW_INV_ARGMAX ? rows_inv_p_impl<T, L, ROW_INV_ARGMAX>(a, batch, nparts, st)       \
                                      : rows_inv_p_impl<T, L, ROW_INV_MAP>(a, batch, nparts, st);
            SD_ROWI_CASE(8) SD_ROWI_CASE(16) SD_ROWI_CASE(24) SD_ROWI_CASE(32) SD_ROWI_CASE(48) SD_ROWI_CASE(64)
            SD_ROWI_CASE(96) SD_ROWI_CASE(128) SD_ROWI_CASE(192) SD_ROWI_CASE(256)
#undef SD_ROWI_CASE
        }
        return cudaErrorInvalidValue;
    }
    if (mode == ROW_FWD_P) {
        if (nparts) *nparts = 0;
        switch (a.n) {
#define SD_ROWP_CASE(L) \
    case L: return rows_fwd_p_impl<T, L>(a, batch, st);
            SD_FOR_EACH_PLEN(SD_ROWP_CASE)
#undef SD_ROWP_CASE
        }
        return cudaErrorInvalidValue;
    }
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
    if (mode == COL_FWD_P || mode == COL_FUSED_P) {
        switch (a.n) {
#define SD_COLP_CASE(L)                                                                       \
    case L:                                                                                   \
        return mode == COL_FWD_P ? cols_fwd_p_impl<T, L>(a, batch, st) : cols_fused_p_impl<T, L>(a, batch, st);
            SD_FOR_EACH_PLEN(SD_COLP_CASE)
#undef SD_COLP_CASE
        }
        return cudaErrorInvalidValue;
    }
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
    if (mode == COL_INV) {
        switch (a.N) {
#define SD_COLI_CASE(L) \
    case L: return cols_inv_p_impl<T, L>(a, batch, st);
            SD_COLI_CASE(8) SD_COLI_CASE(16) SD_COLI_CASE(24) SD_COLI_CASE(32) SD_COLI_CASE(48) SD_COLI_CASE(64)
            SD_COLI_CASE(96) SD_COLI_CASE(128) SD_COLI_CASE(192) SD_COLI_CASE(256)
#undef SD_COLI_CASE
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

template <typename T>
cudaError_t launch_spread_t(const SpreadArgs<T>& a, int dim, int batch, cudaStream_t st) {
    if (a.m == 0 || batch == 0) return cudaSuccess;
    const dim3 grid((unsigned)((a.m + 255) / 256), batch);
#define SD_SPREAD_CASE(WW)                                                                   \
    case WW: {                                                                               \
        auto kern = (dim == 2) ? k_spread<T, 2, WW> : k_spread<T, 3, WW>;                    \
        kern<<<grid, 256, 0, st>>>(a);                                                       \
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

template <int D, int W, int TB>
static cudaError_t spread_bins_impl(const SpreadArgs<float>& a, const BinArgs& bn, int batch, cudaStream_t st) {
    const dim3 gpts((unsigned)((a.m + 255) / 256), batch);
    if (a.m > 0) {
        k_bin_count<float, D, W, TB><<<gpts, 256, 0, st>>>(a, bn);
        k_bin_scan<<<batch, 1024, 0, st>>>(bn);
        k_bin_scatter<float><<<gpts, 256, 0, st>>>(a.m, bn);
        note_launch(3);
    } else {
        k_bin_scan<<<batch, 1024, 0, st>>>(bn);
        note_launch();
    }
    auto kern = k_spread_tiles<D, W, TB>;
    const size_t smem = TileShape<D, W, TB>::smem;
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3((unsigned)bn.nbins, batch), 256, smem, st>>>(a, bn);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread_bins_t(const SpreadArgs<T>& a, const BinArgs& bn, int dim, int batch, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    if constexpr (sizeof(T) != 4) {
        return launch_spread_t<T>(a, dim, batch, st);  // binned spreading is FP32 only
    } else {
        // the counts and the bins' largest |c| components, adjacent in the workspace
        cudaError_t e = cudaMemsetAsync(bn.count, 0, 2 * sizeof(int) * (size_t)batch * bn.nbins, st);
        if (e != cudaSuccess) return e;
#define SD_BIN_TB(WW, TBB)                                                                       \
    if (a.w == WW && bn.tb == TBB)                                                               \
        return dim == 2 ? spread_bins_impl<2, WW, TBB>(a, bn, batch, st) : spread_bins_impl<3, WW, TBB>(a, bn, batch, st);
#define SD_BIN_W(WW) SD_BIN_TB(WW, 8) SD_BIN_TB(WW, 12) SD_BIN_TB(WW, 16)
        SD_BIN_W(4) SD_BIN_W(5) SD_BIN_W(6) SD_BIN_W(7)
#undef SD_BIN_W
#undef SD_BIN_TB
        return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_spread_box_t(const SpreadArgs<T>& a, int dim, int batch, cudaStream_t st) {
    if (a.m == 0 || batch == 0) return cudaSuccess;
    if constexpr (sizeof(T) != 4) {
        return launch_spread_t<T>(a, dim, batch, st);
    } else {
        const dim3 grid((unsigned)((a.m + BOX_SPC - 1) / BOX_SPC), batch);
        const size_t smem = (size_t)2 * BOX_MAXC * sizeof(int);
#define SD_BOX_CASE(WW)                                                   \
    case WW: {                                                            \
        auto kern = dim == 2 ? k_spread_box<2, WW> : k_spread_box<3, WW>; \
        cudaError_t e = set_smem(kern, smem);                             \
        if (e != cudaSuccess) return e;                                   \
        kern<<<grid, BOX_SPC, smem, st>>>(a);                             \
        note_launch();                                                    \
        return cudaGetLastError();                                        \
    }
        switch (a.w) { SD_BOX_CASE(4) SD_BOX_CASE(5) SD_BOX_CASE(6) SD_BOX_CASE(7) }
#undef SD_BOX_CASE
        return cudaErrorInvalidValue;
    }
}

// Spreading fused with the forward x transform: bins over (y, z), then one CTA
// per bin writes the kept x modes of its rows (out: batch x s^2 x N).
template <typename T>
cudaError_t launch_spread_x_t(const SpreadArgs<T>& a, const BinArgs& bn, int nbz, cplx<T>* out,
                              int64_t out_rot_stride, const cplx<T>* tw, int batch, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    if constexpr (sizeof(T) != 4) {
        return cudaErrorInvalidValue;
    } else {
        if (a.w != SX_W || 2 * a.s > a.n_full) return cudaErrorInvalidValue;
        // the counts and the bins' largest |c| components, adjacent in the workspace
        cudaError_t e = cudaMemsetAsync(bn.count, 0, 2 * sizeof(int) * (size_t)batch * bn.nbins, st);
        if (e != cudaSuccess) return e;
        const dim3 gpts((unsigned)((a.m + 255) / 256), batch);
        if (a.m > 0) {
            k_bin_count_yz<float, 3, SX_W><<<gpts, 256, 0, st>>>(a, bn, SX_TY, SX_TZ);
            k_bin_scan<<<batch, 1024, 0, st>>>(bn);
            k_bin_scatter<float><<<gpts, 256, 0, st>>>(a.m, bn);
            note_launch(3);
        } else {
            k_bin_scan<<<batch, 1024, 0, st>>>(bn);
            note_launch();
        }
        const int px = spread_x_pitch(a.s);
        const size_t smem = spread_x_smem(a.n_full, px);
        switch (a.n_full) {
#define SD_SX_CASE(L)                                                                                    \
    case L: {                                                                                            \
        auto kern = k_spread_x<L>;                                                                       \
        e = set_smem(kern, smem);                                                                        \
        if (e != cudaSuccess) return e;                                                                  \
        kern<<<dim3((unsigned)bn.nbins, batch), SX_NT, smem, st>>>(a, bn, nbz, px, out, out_rot_stride, tw); \
        note_launch();                                                                                   \
        return cudaGetLastError();                                                                       \
    }
            SD_FOR_EACH_PLEN(SD_SX_CASE)
#undef SD_SX_CASE
        }
        return cudaErrorInvalidValue;
    }
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

// Field f (0: Phi, 1-3: its gradient) of the type-2 tables into its plane:
// plane f / 2 holds fields (2k, 2k + 1) of every cell side by side, on a grid of
// pitch pn >= n per axis whose cells past n repeat the periodic field (a halo,
// so that a tap box starting inside [0, n) never needs wrapping).
template <typename T>
__global__ void k_interleave(const cplx<T>* src, cplx<T>* dst, int n, int pn, int dim, int f) {
    const int64_t cells = (dim == 3) ? (int64_t)pn * pn * pn : (int64_t)pn * pn;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cells) return;
    const int x = (int)(i % pn), y = (int)((i / pn) % pn), z = (dim == 3) ? (int)(i / ((int64_t)pn * pn)) : 0;
    const int sx = x < n ? x : x - n, sy = y < n ? y : y - n, sz = z < n ? z : z - n;
    const int64_t si = (dim == 3) ? ((int64_t)sz * n + sy) * n + sx : (int64_t)sy * n + sx;
    dst[(f >> 1) * 2 * cells + 2 * i + (f & 1)] = src[si];
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
cudaError_t launch_wshift_t(const cplx<T>* W, int N, int dim, int n, int s_h, cplx<T>* out, cudaStream_t st) {
    const int64_t tot = (dim == 2) ? (int64_t)N * N : (int64_t)N * N * N;
    k_wshift<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(W, N, dim, n, s_h, out);
    note_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interleave_t(const cplx<T>* src, cplx<T>* dst, int n, int pn, int dim, int f, cudaStream_t st) {
    const int64_t cells = (dim == 3) ? (int64_t)pn * pn * pn : (int64_t)pn * pn;
    k_interleave<T><<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(src, dst, n, pn, dim, f);
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
    template <> cudaError_t launch_inv_yx<T>(int mode, const RowArgs<T>& a, int batch, int* np, cudaStream_t st) { \
        return launch_inv_yx_t<T>(mode, a, batch, np, st);                                              \
    }                                                                                                   \
    template <> cudaError_t launch_cols<T>(int mode, const ColArgs<T>& a, int batch, cudaStream_t st) {   \
        return launch_cols_t<T>(mode, a, batch, st);                                                    \
    }                                                                                                   \
    template <> cudaError_t launch_spread_bins<T>(const SpreadArgs<T>& a, const BinArgs& bn, int dim, int batch, \
                                                  cudaStream_t st) {                                    \
        return launch_spread_bins_t<T>(a, bn, dim, batch, st);                                          \
    }                                                                                                   \
    template <> cudaError_t launch_spread_x<T>(const SpreadArgs<T>& a, const BinArgs& bn, int nbz, cplx<T>* out, \
                                               int64_t ors, const cplx<T>* tw, int batch, cudaStream_t st) {   \
        return launch_spread_x_t<T>(a, bn, nbz, out, ors, tw, batch, st);                               \
    }                                                                                                   \
    template <> cudaError_t launch_spread_box<T>(const SpreadArgs<T>& a, int dim, int batch, cudaStream_t st) { \
        return launch_spread_box_t<T>(a, dim, batch, st);                                               \
    }                                                                                                   \
    template <> cudaError_t launch_twiddles<T>(cplx<T>* tw, int len, cudaStream_t st) {                 \
        return launch_twiddles_t<T>(tw, len, st);                                                       \
    }                                                                                                   \
    template <> cudaError_t launch_wtable<T>(const cplx<T>* B1, const double* D, int N, int dim, double L, \
                                             double sg, int shift, int deriv, cplx<T>* W, cudaStream_t st) { \
        return launch_wtable_t<T>(B1, D, N, dim, L, sg, shift, deriv, W, st);                           \
    }                                                                                                   \
    template <> cudaError_t launch_wshift<T>(const cplx<T>* W, int N, int dim, int n, int s_h, cplx<T>* out,      \
                                             cudaStream_t st) {                                                \
        return launch_wshift_t<T>(W, N, dim, n, s_h, out, st);                                          \
    }                                                                                                   \
    template <> cudaError_t launch_interleave<T>(const cplx<T>* s, cplx<T>* d, int n, int pn, int dim, int f,       \
                                                 cudaStream_t st) {                                                 \
        return launch_interleave_t<T>(s, d, n, pn, dim, f, st);                                         \
    }                                                                                                   \
    }
