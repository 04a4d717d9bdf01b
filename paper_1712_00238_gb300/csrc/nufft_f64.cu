// FP64 instantiation of the nonuniform-FFT passes, plus the FP64 tables and the
// per-rotation argmax reduction shared by both precisions.
#include "nufft_impl.cuh"
#include "topk.cuh"
SD_INSTANTIATE_NUFFT(double)

namespace sd {

// D[kappa'] = (w/2) * psihat(pi kappa w / n), psihat(xi) = int_{-1}^{1} psi(z) e^{-i xi z} dz
//          = 2 int_0^{pi/2} exp(beta (cos th - 1)) cos(xi sin th) cos th dth   (z = sin th),
// a smooth integrand, by Gauss-Legendre nodes on [0, pi/2].
__global__ void k_deconv(double* D, int N, int n, int w, double beta, const double* gx, const double* gw,
                         int nq) {
    const int kp = blockIdx.x * blockDim.x + threadIdx.x;
    if (kp >= N) return;
    const int kap = kp < N / 2 ? kp : kp - N;
    const double xi = M_PI * (double)kap * (double)w / (double)n;
    double acc = 0.0;
    for (int q = 0; q < nq; ++q) {
        const double th = gx[q];
        double s, c;
        sincos(th, &s, &c);
        acc += gw[q] * exp(beta * (c - 1.0)) * cos(xi * s) * c;
    }
    D[kp] = 0.5 * (double)w * 2.0 * acc;
}

cudaError_t launch_deconv(double* D, int N, int n, int w, double beta, const double* gx, const double* gw,
                          int nq, cudaStream_t st) {
    k_deconv<<<(N + 127) / 128, 128, 0, st>>>(D, N, n, w, beta, gx, gw, nq);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_reduce_argmax(const double* ps, const int* pi, int nparts, int64_t rot0, CandRec* cand) {
    const int b = blockIdx.x;
    double best = -INFINITY;
    int bidx = INT_MAX;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
        const double v = ps[(int64_t)b * nparts + p];
        const int i = pi[(int64_t)b * nparts + p];
        if (v > best || (v == best && i < bidx)) {
            best = v;
            bidx = i;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
        if (ob > best || (ob == best && oi < bidx)) {
            best = ob;
            bidx = oi;
        }
    }
    __shared__ double wb[32];
    __shared__ int wi[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wb[warp] = best;
        wi[warp] = bidx;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        best = lane < nw ? wb[lane] : -INFINITY;
        bidx = lane < nw ? wi[lane] : INT_MAX;
        for (int off = 16; off > 0; off >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, off);
            const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
            if (ob > best || (ob == best && oi < bidx)) {
                best = ob;
                bidx = oi;
            }
        }
        if (lane == 0) {
            CandRec r;
            r.score = best;
            r.rot = (int32_t)(rot0 + b);
            r.idx = bidx == INT_MAX ? -1 : bidx;
            cand[rot0 + b] = r;
        }
    }
}

cudaError_t launch_reduce_argmax(const double* ps, const int* pi, int nparts, int batch, int64_t rot0,
                                 void* cand, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    k_reduce_argmax<<<batch, 256, 0, st>>>(ps, pi, nparts, rot0, reinterpret_cast<CandRec*>(cand));
    note_launch();
    return cudaGetLastError();
}

template <int K>
__global__ void k_reduce_topk(const double* ps, const int* pi, int nparts, int k_r, int64_t rot0, CandRec* cand) {
    extern __shared__ __align__(16) unsigned char rk_raw[];
    double* sv = reinterpret_cast<double*>(rk_raw);
    int* si = reinterpret_cast<int*>(sv + blockDim.x * K);
    __shared__ double wv[32], bestv[K];
    __shared__ int wi[32], besti[K];
    const int b = blockIdx.x;
    TopK<double, K> top;
    top.init();
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) top.push(ps[(int64_t)b * nparts + p], pi[(int64_t)b * nparts + p]);
    block_topk_merge<double, K>(top, sv, si, wv, wi, bestv, besti);
    if (threadIdx.x < k_r) {
        CandRec c;
        const bool real = besti[threadIdx.x] != INT_MAX;
        c.score = real ? bestv[threadIdx.x] : -INFINITY;
        c.rot = (int32_t)(rot0 + b);
        c.idx = real ? besti[threadIdx.x] : -1;
        cand[(rot0 + b) * (int64_t)k_r + threadIdx.x] = c;
    }
}

cudaError_t launch_reduce_topk(const double* ps, const int* pi, int nparts, int K, int k_r, int batch, int64_t rot0,
                               void* cand, cudaStream_t st) {
    if (batch == 0) return cudaSuccess;
    CandRec* c = reinterpret_cast<CandRec*>(cand);
    const size_t smem = (size_t)128 * K * (sizeof(double) + sizeof(int));
    switch (K) {
        case 2: k_reduce_topk<2><<<batch, 128, smem, st>>>(ps, pi, nparts, k_r, rot0, c); break;
        case 4: k_reduce_topk<4><<<batch, 128, smem, st>>>(ps, pi, nparts, k_r, rot0, c); break;
        case 8: k_reduce_topk<8><<<batch, 128, smem, st>>>(ps, pi, nparts, k_r, rot0, c); break;
        case 16: k_reduce_topk<16><<<batch, 128, smem, st>>>(ps, pi, nparts, k_r, rot0, c); break;
        default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace sd
