// Pruned line transforms for the search passes.
//
// The forward passes of the search transform lines of the spread sub-box: n
// points of which only the first s <= n/2 can be nonzero (the sub-box is loaded
// unshifted: cell a sits at position a, and the shift to the centred grid is a
// phase applied with the product table), and of whose n outputs only the N = n/2
// central modes are kept.  Both facts are fixed by the plan, not by the data:
//   * the first stage's butterflies read inputs i + r n/R1, r < R1; those with
//     r >= R1/2 lie at or past n/2 and are zero, so the first R1-point DFT runs
//     with its upper half of inputs known to be zero;
//   * the last stage's butterfly i (< P = n/R) writes output i + r P; modes
//     |kappa| < N/2 = n/4 are exactly r < R/4 and r >= 3R/4 when 4 divides R.
// The stage engine below hands the loader (line, i, r) and the emitter
// (line, i, r, value) so that after unrolling r is a compile-time constant:
// dropped outputs are never computed and kept ones land at constant offsets.
#pragma once

#include "fft.cuh"

namespace sd {

// Radix of the last stage of a plan.
__host__ __device__ constexpr int plan_last_radix(int len) {
    int s = 0;
    while (plan_radix(len, s + 1) != 0) ++s;
    return plan_radix(len, s);
}

// A forward pass of length n can prune at compile time when its first radix is
// even (upper half of the first stage's inputs) and 4 divides its last radix.
__host__ __device__ constexpr bool prunable_len(int n) {
    return fft_len_supported(n) && plan_radix(n, 0) % 2 == 0 && plan_last_radix(n) % 4 == 0;
}

// R-point DFT of v whose inputs v[R/2 .. R) are zero (they are not read).
template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_lowhalf(C* v) {
    using T = decltype(C{}.x);
    if constexpr (R == 16) {
        // n = 4 n1 + n2, k = k1 + 4 k2; the first-layer 4-point DFTs see (a0, a1, 0, 0)
        C b[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            const C a0 = v[n2], a1 = v[4 + n2];
            b[n2][0] = cadd(a0, a1);
            b[n2][1] = add_mi<INV>(a0, a1);
            b[n2][2] = csub(a0, a1);
            b[n2][3] = sub_mi<INV>(a0, a1);
        }
#pragma unroll
        for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) b[n2][k1] = cmul(b[n2][k1], w16<INV, C>(n2 * k1));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C x0 = b[0][k1], x1 = b[1][k1], x2 = b[2][k1], x3 = b[3][k1];
            dft4<INV>(x0, x1, x2, x3);
            v[k1] = x0; v[k1 + 4] = x1; v[k1 + 8] = x2; v[k1 + 12] = x3;
        }
    } else if constexpr (R == 8) {
        // even / odd inputs each (a0, a1, 0, 0)
        const T r = T(0.70710678118654752440);
        C e0 = cadd(v[0], v[2]), e1 = add_mi<INV>(v[0], v[2]), e2 = csub(v[0], v[2]), e3 = sub_mi<INV>(v[0], v[2]);
        C o0 = cadd(v[1], v[3]), o1 = add_mi<INV>(v[1], v[3]), o2 = csub(v[1], v[3]), o3 = sub_mi<INV>(v[1], v[3]);
        o1 = cmul(o1, INV ? mk(r, r) : mk(r, -r));
        o2 = mul_mi<INV>(o2);
        o3 = cmul(o3, INV ? mk(-r, r) : mk(-r, -r));
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
    } else {
#pragma unroll
        for (int r = R / 2; r < R; ++r) v[r] = mk(T(0), T(0));
        dft<R, INV>(v);
    }
}

template <bool PAD>
__device__ __forceinline__ int pidx(int j) {
    if constexpr (PAD) return pad(j);
    else return j;
}

// Line transforms of NL lines per block of NT threads (see fft_lines_io for the
// thread layouts).  load(line, i, r) returns first-stage input i + r LEN/R1
// (called for r < R1/2 only when HALF_IN); emit(line, i, r, v) receives output
// i + r P of the last stage.  PAD: in-line padding of the shared buffer (needed
// when a warp's lanes walk one line, LAY_ROW); column layouts use an odd pitch
// and no padding.  SRC_SMEM: the inputs are already in buf.
template <typename C, int LEN, bool INV, int NL, int NT, int LAY, bool PAD, bool SRC_SMEM, bool HALF_IN,
          int S = 0, int P = 1, typename Load, typename Emit>
__device__ __forceinline__ void fftp_lines(C* buf, int ld, const C* tw, Load& load, Emit& emit) {
    constexpr int R = plan_radix(LEN, S);
    constexpr bool first = (S == 0);
    constexpr bool last = (plan_radix(LEN, S + 1) == 0);
    constexpr int NB = LEN / R;
    constexpr int TOT = NL * NB;
    constexpr int PER = (TOT + NT - 1) / NT;
    constexpr bool half = first && HALF_IN;
    C v[PER][R];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int t = threadIdx.x + q * NT;
        if (TOT % NT == 0 || t < TOT) {
            int line, i;
            butterfly_of<LAY, NL, NB>(t, line, i);
            if constexpr (first && !SRC_SMEM) {
#pragma unroll
                for (int r = 0; r < (half ? R / 2 : R); ++r) v[q][r] = load(line, i, r);
            } else {
                const C* ln = buf + line * ld;
#pragma unroll
                for (int r = 0; r < (half ? R / 2 : R); ++r) v[q][r] = ln[pidx<PAD>(i + r * NB)];
                if constexpr (P > 1) {
                    const C* tws = tw + tw_offset(LEN, S) + (i % P) * (R - 1);
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        C w = tws[r - 1];
                        if (INV) w.y = -w.y;
                        v[q][r] = cmul(v[q][r], w);
                    }
                }
            }
            if constexpr (half) dft_lowhalf<R, INV>(v[q]);
            else dft<R, INV>(v[q]);
        }
    }
    if constexpr (!first || SRC_SMEM) __syncthreads();  // every read of buf before any write
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int t = threadIdx.x + q * NT;
        if (TOT % NT == 0 || t < TOT) {
            int line, i;
            butterfly_of<LAY, NL, NB>(t, line, i);
            if constexpr (last) {
#pragma unroll
                for (int r = 0; r < R; ++r) emit(line, i, r, v[q][r]);
            } else {
                C* ln = buf + line * ld;
                const int k = i % P;
                const int j = (i - k) * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) ln[pidx<PAD>(j + r * P)] = v[q][r];
            }
        }
    }
    if constexpr (!last) {
        __syncthreads();
        fftp_lines<C, LEN, INV, NL, NT, LAY, PAD, SRC_SMEM, HALF_IN, S + 1, P * R>(buf, ld, tw, load, emit);
    }
}

// Output r of a last-stage butterfly (output i + r P, P = LEN / RL) kept by a
// forward pass that keeps the N = LEN/2 central modes; its mode slot (kappa mod
// N) is i + r P for the low modes and i + r P - N for the high ones.
template <int LEN>
__device__ __forceinline__ constexpr bool kept_out(int r) {
    constexpr int RL = plan_last_radix(LEN);
    return r < RL / 4 || r >= 3 * RL / 4;
}
template <int LEN>
__device__ __forceinline__ constexpr int kept_slot(int r) {
    constexpr int RL = plan_last_radix(LEN);
    constexpr int PL = LEN / RL;
    return r < RL / 4 ? r * PL : r * PL - LEN / 2;
}

}  // namespace sd
