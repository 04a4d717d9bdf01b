// The k best (value, index) pairs of a block: each thread keeps a sorted list in
// registers, then the block merges the lists through shared memory.  Order:
// value descending, then index ascending (NaN values are never kept).
#pragma once

#include <limits.h>
#include <math.h>

namespace sd {

template <typename V>
__device__ __forceinline__ bool topk_better(V a, int ia, V b, int ib) {
    return a > b || (a == b && ia < ib);
}

template <typename V, int K>
struct TopK {
    V v[K];
    int i[K];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            v[k] = -INFINITY;
            i[k] = INT_MAX;
        }
    }
    // Bubbles (x, ix) into place; the last entry falls off.  Static indices only.
    __device__ __forceinline__ void push(V x, int ix) {
        if (!topk_better(x, ix, v[K - 1], i[K - 1])) return;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (topk_better(x, ix, v[k], i[k])) {
                const V tv = v[k];
                const int ti = i[k];
                v[k] = x;
                i[k] = ix;
                x = tv;
                ix = ti;
            }
        }
    }
};

// Merges every thread's list into the block's first K entries (out_v / out_i,
// written by thread 0).  sv / si: shared scratch of blockDim.x * K entries; wv /
// wi: shared scratch of 32 entries.  Every thread of the block must call it.
template <typename V, int K>
__device__ void block_topk_merge(const TopK<V, K>& t, V* sv, int* si, V* wv, int* wi, V* out_v, int* out_i) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        sv[tid * K + k] = t.v[k];
        si[tid * K + k] = t.i[k];
    }
    __shared__ int won;
    int h = 0;  // this thread's next unmerged entry
    __syncthreads();
    for (int k = 0; k < K; ++k) {
        V b = h < K ? sv[tid * K + h] : V(-INFINITY);
        int bi = h < K ? si[tid * K + h] : INT_MAX;
        for (int off = 16; off > 0; off >>= 1) {
            const V ob = __shfl_down_sync(0xffffffffu, b, off);
            const int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (topk_better(ob, oi, b, bi)) {
                b = ob;
                bi = oi;
            }
        }
        if (lane == 0) {
            wv[warp] = b;
            wi[warp] = bi;
        }
        __syncthreads();
        if (warp == 0) {
            b = lane < nw ? wv[lane] : V(-INFINITY);
            bi = lane < nw ? wi[lane] : INT_MAX;
            for (int off = 16; off > 0; off >>= 1) {
                const V ob = __shfl_down_sync(0xffffffffu, b, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (topk_better(ob, oi, b, bi)) {
                    b = ob;
                    bi = oi;
                }
            }
            if (lane == 0) {
                out_v[k] = b;
                out_i[k] = bi;
                won = bi;
            }
        }
        __syncthreads();
        // indices are distinct among real entries: the owner of the winner advances
        if (h < K && si[tid * K + h] == won && won != INT_MAX) ++h;
        __syncthreads();
    }
}

}  // namespace sd
