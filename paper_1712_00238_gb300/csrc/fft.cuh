// Batched line FFTs in shared memory: mixed radix (2, 3, 4, 8, 12, 16, 24) Stockham
// autosort stages (Van Loan, "Computational Frameworks for the FFT", 1992).
//
// Each stage of radix R over a line of LEN points takes, for every butterfly
// index i in [0, LEN/R), the R inputs x[i + r*LEN/R], multiplies input r by the
// twiddle exp(-+2 pi i * r*k / (P*R)) with k = i mod P (P = product of the radices
// of the earlier stages), applies an R-point DFT in registers and stores output r
// at (i - k)*R + k + r*P.  After the last stage the line is in natural order.
// Forward transforms use exp(-2 pi i jk/LEN); inverse ones exp(+2 pi i jk/LEN),
// unnormalised.
//
// Lines live in shared memory with a pitch `ld` (complex elements) and an
// in-line padding of one element per 16 (pad()) so that the strided stores of the
// early stages do not hit one bank.
#pragma once

#include "common.cuh"

namespace sd {

// Radix of stage s for a line of `len` points (0 past the last stage).
__host__ __device__ constexpr int plan_radix(int len, int s) {
    switch (len) {
        case 8: return s == 0 ? 8 : 0;
        case 16: return s == 0 ? 16 : 0;
        case 24: return s == 0 ? 8 : (s == 1 ? 3 : 0);
        case 32: return s == 0 ? 8 : (s == 1 ? 4 : 0);
        case 48: return s == 0 ? 16 : (s == 1 ? 3 : 0);
        case 64: return s == 0 ? 8 : (s == 1 ? 8 : 0);
        case 96: return s == 0 ? 8 : (s == 1 ? 12 : 0);
        case 128: return s == 0 ? 16 : (s == 1 ? 8 : 0);
        case 192: return s == 0 ? 16 : (s == 1 ? 12 : 0);
        case 256: return s == 0 ? 16 : (s == 1 ? 16 : 0);
        case 384: return s == 0 ? 16 : (s == 1 ? 24 : 0);
        case 512: return s == 0 ? 8 : (s == 1 ? 8 : (s == 2 ? 8 : 0));
        default: return 0;
    }
}

__host__ __device__ constexpr bool fft_len_supported(int len) { return plan_radix(len, 0) != 0; }

// Applies X to every supported line length.
#define SD_FOR_EACH_LEN(X) X(8) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

__host__ __device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
// Padded line storage (elements) and an odd pitch for column-wise tile fills.
__host__ __device__ constexpr int line_pitch(int len) { return ((len + (len >> 4)) | 1); }

// ---------------------------------------------------------------------------
// R-point DFTs in registers.  INV selects the +i sign.
// ---------------------------------------------------------------------------

template <bool INV, typename C>
__host__ __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = add_mi<INV>(t1, d);
    a3 = sub_mi<INV>(t1, d);
}

// exp(-+2 pi i m / 16) as constants (cos and sin of multiples of pi/8).
template <bool INV, typename C>
__host__ __device__ __forceinline__ C w16(int m) {
    using T = decltype(C{}.x);
    const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), r = T(0.70710678118654752440);
    T cr, si;  // exp(-i 2 pi m/16) = cr - i si
    switch (m) {
        case 0: cr = 1; si = 0; break;
        case 1: cr = c1; si = s1; break;
        case 2: cr = r; si = r; break;
        case 3: cr = s1; si = c1; break;
        case 4: cr = 0; si = 1; break;
        case 6: cr = -r; si = r; break;
        case 9: cr = -c1; si = -s1; break;
        default: cr = 1; si = 0; break;  // not used by dft16
    }
    return INV ? mk(cr, si) : mk(cr, -si);
}

// exp(-+2 pi i m / 24), m in [0, 24): the angle r * 15 degrees of its quadrant
// (r = m mod 6) rotated by -+i per quadrant.  cos 15 = (sqrt 6 + sqrt 2) / 4,
// sin 15 = (sqrt 6 - sqrt 2) / 4.
template <bool INV, typename C>
__host__ __device__ __forceinline__ C w24(int m) {
    using T = decltype(C{}.x);
    const T c15 = T(0.96592582628906828675), s15 = T(0.25881904510252076235);
    const T c30 = T(0.86602540378443864676), r = T(0.70710678118654752440);
    T c, s;  // cos and sin of (m mod 6) * 15 degrees
    switch (m % 6) {
        case 0: c = 1; s = 0; break;
        case 1: c = c15; s = s15; break;
        case 2: c = c30; s = T(0.5); break;
        case 3: c = r; s = r; break;
        case 4: c = T(0.5); s = c30; break;
        default: c = s15; s = c15; break;
    }
    T x, y;  // exp(-i theta) rotated by (-i)^quadrant
    switch ((m / 6) & 3) {
        case 0: x = c; y = -s; break;
        case 1: x = -s; y = -c; break;
        case 2: x = -c; y = s; break;
        default: x = s; y = c; break;
    }
    return INV ? mk(x, -y) : mk(x, y);
}

template <int R, bool INV, typename C>
__host__ __device__ __forceinline__ void dft(C* v);

// R = 3 Q points (Q = 4 or 8) by one Cooley-Tukey split: input n = Q n1 + n2,
// output k = k1 + 3 k2; 3-point DFTs over n1, twiddles w_R^(n2 k1), Q-point
// DFTs over n2.
template <int Q, bool INV, typename C>
__host__ __device__ __forceinline__ void dft3q(C* v) {
    constexpr int R = 3 * Q;
    C b[3][Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
        C t[3] = {v[n2], v[Q + n2], v[2 * Q + n2]};
        dft<3, INV>(t);
        b[0][n2] = t[0];
#pragma unroll
        for (int k1 = 1; k1 < 3; ++k1) b[k1][n2] = n2 == 0 ? t[k1] : cmul(t[k1], w24<INV, C>((24 / R) * n2 * k1));
    }
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        dft<Q, INV>(b[k1]);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[k1 + 3 * k2] = b[k1][k2];
    }
}

template <int R, bool INV, typename C>
__host__ __device__ __forceinline__ void dft(C* v) {
    using T = decltype(C{}.x);
    if constexpr (R == 2) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        const T s3 = T(0.86602540378443864676);
        C t = cadd(v[1], v[2]), u = csub(v[1], v[2]);
        C m = csub(v[0], cscale(t, T(0.5)));
        v[0] = cadd(v[0], t);
        C d = cscale(mul_mi<INV>(u), s3);
        v[1] = cadd(m, d);
        v[2] = csub(m, d);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        const T r = T(0.70710678118654752440);
        C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4<INV>(e0, e1, e2, e3);
        dft4<INV>(o0, o1, o2, o3);
        // o_k *= exp(-+2 pi i k/8)
        o1 = cmul(o1, INV ? mk(r, r) : mk(r, -r));
        o2 = mul_mi<INV>(o2);
        o3 = cmul(o3, INV ? mk(-r, r) : mk(-r, -r));
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
    } else if constexpr (R == 16) {
        // n = 4 n1 + n2, k = k1 + 4 k2
        C b[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            b[n2][0] = v[n2]; b[n2][1] = v[4 + n2]; b[n2][2] = v[8 + n2]; b[n2][3] = v[12 + n2];
            dft4<INV>(b[n2][0], b[n2][1], b[n2][2], b[n2][3]);
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
    } else if constexpr (R == 12) {
        dft3q<4, INV>(v);
    } else if constexpr (R == 24) {
        dft3q<8, INV>(v);
    }
}

// Twiddles are stored stage by stage: for a stage of radix R after stages of
// product P > 1, the block of P*(R-1) entries tw[off + k*(R-1) + (r-1)] =
// exp(-2 pi i r k / (P R)), k in [0, P), r in [1, R).  Consecutive butterflies
// (consecutive k) read entries R-1 apart (an odd stride): no bank conflicts.
__host__ __device__ constexpr int tw_offset(int len, int s) {
    int off = 0, p = 1;
    for (int q = 0; q < s; ++q) {
        const int r = plan_radix(len, q);
        if (p > 1) off += p * (r - 1);
        p *= r;
    }
    return off;
}
__host__ __device__ constexpr int tw_count(int len) {
    int s = 0;
    while (plan_radix(len, s) != 0) ++s;
    return tw_offset(len, s);
}

// Fills the stage-ordered table of one length (host or device, any precision);
// `f(j, r, k, P, R)` stores exp(-2 pi i r k / (P R)) at entry j.
template <typename F>
__host__ __device__ inline void tw_for_each(int len, F f) {
    int off = 0, p = 1;
    for (int s = 0; plan_radix(len, s) != 0; ++s) {
        const int R = plan_radix(len, s);
        if (p > 1)
            for (int k = 0; k < p; ++k)
                for (int r = 1; r < R; ++r) f(off + k * (R - 1) + (r - 1), r, k, p, R);
        if (p > 1) off += p * (R - 1);
        p *= R;
    }
}

// Load, twiddle and transform one butterfly of a Stockham stage into v[].
template <typename C, int LEN, int R, int P, bool INV>
__host__ __device__ __forceinline__ void stockham_load(const C* __restrict__ line, int i, const C* __restrict__ tw,
                                                       C v[R]) {
    constexpr int NB = LEN / R;
    const int k = i % P;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = line[pad(i + r * NB)];
    if constexpr (P > 1) {
        const C* t = tw + k * (R - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) {
            C w = t[r - 1];
            if (INV) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
    }
    dft<R, INV>(v);
}

template <typename C, int LEN, int R, int P>
__host__ __device__ __forceinline__ void stockham_store(C* __restrict__ line, int i, const C v[R]) {
    const int k = i % P;
    const int j = (i - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) line[pad(j + r * P)] = v[r];
}

#ifdef __CUDACC__
// Line transforms whose first stage reads its inputs through a loader (global
// memory, registers in flight) and whose last stage hands its outputs to an
// emitter (global memory or the next step), so only the stages in between go
// through shared memory: one round trip for two-stage lengths.
//
// LAY_ROW: lines are contiguous (a warp's lanes take consecutive butterflies of
// one line); LAY_COL: lines are columns (lanes take consecutive lines).  NL lines
// per block of NT threads; a stage with fewer butterflies than NT leaves the
// rest of the threads idle until its barrier.  load(line, pos) returns input `pos`;
// emit(line, o, v) receives output `o` (natural order).  SRC_SMEM: the inputs
// are already in `buf` (pitch ld, padded) and are read from there.
enum { LAY_ROW = 0, LAY_COL = 1 };

template <int LAY, int NL, int NB>
__device__ __forceinline__ void butterfly_of(int t, int& line, int& i) {
    if constexpr (LAY == LAY_ROW) {
        line = t / NB;
        i = t - line * NB;
    } else {
        i = t / NL;
        line = t - i * NL;
    }
}

template <typename C, int LEN, bool INV, int NL, int NT, int LAY, bool SRC_SMEM, int S = 0, int P = 1,
          typename Load, typename Emit>
__device__ __forceinline__ void fft_lines_io(C* buf, int ld, const C* tw, Load& load, Emit& emit) {
    constexpr int R = plan_radix(LEN, S);
    constexpr bool first = (S == 0);
    constexpr bool last = (plan_radix(LEN, S + 1) == 0);
    constexpr int NB = LEN / R;
    constexpr int TOT = NL * NB;
    constexpr int PER = (TOT + NT - 1) / NT;
    C v[PER][R];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int t = threadIdx.x + q * NT;
        if (TOT % NT == 0 || t < TOT) {
            int line, i;
            butterfly_of<LAY, NL, NB>(t, line, i);
            if constexpr (first && !SRC_SMEM) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[q][r] = load(line, i + r * NB);
                dft<R, INV>(v[q]);
            } else {
                stockham_load<C, LEN, R, P, INV>(buf + line * ld, i, tw + tw_offset(LEN, S), v[q]);
            }
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
                for (int r = 0; r < R; ++r) emit(line, i + r * P, v[q][r]);  // P = NB here
            } else {
                stockham_store<C, LEN, R, P>(buf + line * ld, i, v[q]);
            }
        }
    }
    if constexpr (!last) {
        __syncthreads();
        fft_lines_io<C, LEN, INV, NL, NT, LAY, SRC_SMEM, S + 1, P * R>(buf, ld, tw, load, emit);
    }
}
#endif

// Host execution of the same stage sequence on one line, in place (used by the
// library's self-test of the index arithmetic).
template <typename C, int LEN, bool INV, int S = 0, int P = 1>
inline void fft_line_host(C* line, const C* tw) {
    constexpr int R = plan_radix(LEN, S);
    if constexpr (R != 0) {
        constexpr int NB = LEN / R;
        C v[NB][R];
        for (int i = 0; i < NB; ++i) stockham_load<C, LEN, R, P, INV>(line, i, tw + tw_offset(LEN, S), v[i]);
        for (int i = 0; i < NB; ++i) stockham_store<C, LEN, R, P>(line, i, v[i]);
        fft_line_host<C, LEN, INV, S + 1, P * R>(line, tw);
    }
}

}  // namespace sd
