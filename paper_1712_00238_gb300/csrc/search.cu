// Search over the per-rotation maxima (the argmax over T of Section 4) and the
// FP64 re-score of the best poses.
//
// top-k: one CTA selects k candidates in order (score descending, rotation
// ascending, translation index ascending), k rounds of a block-wide arg-best
// over the candidates not yet taken (flags in a bitset).
// re-score: f_c(R, t) = sum_ij c1_i c2_j G_{sigma_g sqrt 2}(R p2_j + t - p1_i) in
// FP64 (the continuous score of Eq. 8 for Gaussian-represented SDFs).  Pairs
// are screened in FP32 against a cutoff of 8 sigma_g sqrt 2 (with a margin), and
// CTA / tile bounding boxes skip whole blocks of far pairs.
#include <algorithm>
#include <float.h>
#include <limits.h>
#include <math.h>

#include "kernels.cuh"

namespace sd {

struct Cand {
    double score;
    int32_t rot;
    int32_t idx;
};

__device__ __forceinline__ bool cand_better(double s, int r, int i, int64_t p, double s2, int r2, int i2, int64_t p2) {
    if (s != s2) return s > s2;
    if (r != r2) return r < r2;
    if (i != i2) return i < i2;
    return p < p2;
}

__global__ void __launch_bounds__(1024) k_topk(const Cand* cand, int64_t n, int k, Cand* out, unsigned* flags) {
    const int64_t nw = (n + 31) / 32;
    for (int64_t i = threadIdx.x; i < nw; i += blockDim.x) flags[i] = 0u;
    __syncthreads();
    __shared__ double ws[32];
    __shared__ int wr[32], wi[32];
    __shared__ long long wp[32];
    for (int it = 0; it < k; ++it) {
        double bs = -INFINITY;
        int br = INT_MAX, bi = INT_MAX;
        long long bp = LLONG_MAX;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
            if (flags[p >> 5] & (1u << (p & 31))) continue;
            const Cand c = cand[p];
            const double s = (c.score == c.score) ? c.score : -INFINITY;  // NaN ranks last
            if (bp == LLONG_MAX || cand_better(s, c.rot, c.idx, p, bs, br, bi, bp)) {
                bs = s; br = c.rot; bi = c.idx; bp = p;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            const double os = __shfl_down_sync(0xffffffffu, bs, off);
            const int orr = __shfl_down_sync(0xffffffffu, br, off);
            const int oi = __shfl_down_sync(0xffffffffu, bi, off);
            const long long op = __shfl_down_sync(0xffffffffu, bp, off);
            if (op != LLONG_MAX && (bp == LLONG_MAX || cand_better(os, orr, oi, op, bs, br, bi, bp))) {
                bs = os; br = orr; bi = oi; bp = op;
            }
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) { ws[warp] = bs; wr[warp] = br; wi[warp] = bi; wp[warp] = bp; }
        __syncthreads();
        if (warp == 0) {
            const int nwarp = (blockDim.x + 31) >> 5;
            bs = lane < nwarp ? ws[lane] : -INFINITY;
            br = lane < nwarp ? wr[lane] : INT_MAX;
            bi = lane < nwarp ? wi[lane] : INT_MAX;
            bp = lane < nwarp ? wp[lane] : LLONG_MAX;
            for (int off = 16; off > 0; off >>= 1) {
                const double os = __shfl_down_sync(0xffffffffu, bs, off);
                const int orr = __shfl_down_sync(0xffffffffu, br, off);
                const int oi = __shfl_down_sync(0xffffffffu, bi, off);
                const long long op = __shfl_down_sync(0xffffffffu, bp, off);
                if (op != LLONG_MAX && (bp == LLONG_MAX || cand_better(os, orr, oi, op, bs, br, bi, bp))) {
                    bs = os; br = orr; bi = oi; bp = op;
                }
            }
            if (lane == 0) {
                Cand c;
                if (bp == LLONG_MAX) {
                    c.score = -INFINITY; c.rot = -1; c.idx = -1;
                } else {
                    c = cand[bp];
                    flags[bp >> 5] |= (1u << (bp & 31));
                }
                out[it] = c;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_topk(const void* cand, int64_t n, int k, void* out, unsigned* flags, cudaStream_t st) {
    k_topk<<<1, 1024, 0, st>>>(reinterpret_cast<const Cand*>(cand), n, k, reinterpret_cast<Cand*>(out), flags);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------

constexpr int RS_TILE = 256;
constexpr int RS_WARPS = RS_TILE / 32;

// Block-wide bounding box of one point per thread (dead threads pass +inf/-inf);
// the result is valid in out_lo/out_hi (shared) after the call.
__device__ __forceinline__ void block_bbox(float lo[3], float hi[3], float (*wlo)[3], float (*whi)[3],
                                           float out_lo[3], float out_hi[3]) {
    for (int d = 0; d < 3; ++d)
        for (int off = 16; off > 0; off >>= 1) {
            lo[d] = fminf(lo[d], __shfl_down_sync(0xffffffffu, lo[d], off));
            hi[d] = fmaxf(hi[d], __shfl_down_sync(0xffffffffu, hi[d], off));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int d = 0; d < 3; ++d) { wlo[warp][d] = lo[d]; whi[warp][d] = hi[d]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) {
            float a = FLT_MAX, b = -FLT_MAX;
            for (int w = 0; w < RS_WARPS; ++w) { a = fminf(a, wlo[w][d]); b = fmaxf(b, whi[w][d]); }
            out_lo[d] = a;
            out_hi[d] = b;
        }
    }
    __syncthreads();
}

// Pose (R, t) of a candidate: rotation matrix (FP64) and translation of its grid index.
__device__ void pose_of(const Cand& cd, const double* quats, int N, double L, int dim, double Rm[9], double tv[3]) {
    const double h = L / N;
    int idx = cd.idx < 0 ? 0 : cd.idx;
    for (int d = 0; d < 3; ++d) {
        if (d < dim) {
            tv[d] = (double)(idx % N - N / 2) * h;
            idx /= N;
        } else {
            tv[d] = 0.0;
        }
    }
    const double* q = quats + 4 * (int64_t)cd.rot;
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double n2 = w * w + x * x + y * y + z * z;
    const double s = n2 > 0 ? 2.0 / n2 : 0.0;
    Rm[0] = 1 - s * (y * y + z * z); Rm[1] = s * (x * y - w * z); Rm[2] = s * (x * z + w * y);
    Rm[3] = s * (x * y + w * z); Rm[4] = 1 - s * (x * x + z * z); Rm[5] = s * (y * z - w * x);
    Rm[6] = s * (x * z - w * y); Rm[7] = s * (y * z + w * x); Rm[8] = 1 - s * (x * x + y * y);
}

// Per pose: the moved samples y_j = R p2_j + t in FP64 and the float bounding box
// of every tile of RS_TILE consecutive samples.
template <typename T>
__global__ void __launch_bounds__(RS_TILE) k_rescore_move(RescoreArgs<T> a) {
    __shared__ double Rm[9], tv[3];
    __shared__ float wlo[RS_WARPS][3], whi[RS_WARPS][3];
    __shared__ float blo[3], bhi[3];
    const int pose = blockIdx.y;
    const Cand cd = reinterpret_cast<const Cand*>(a.top)[pose];
    const int ntiles = gridDim.x;
    float* tb = a.tile_box + ((int64_t)pose * ntiles + blockIdx.x) * 6;
    if (cd.rot < 0) {
        if (threadIdx.x < 3) { tb[threadIdx.x] = FLT_MAX; tb[3 + threadIdx.x] = -FLT_MAX; }
        return;
    }
    if (threadIdx.x == 0) pose_of(cd, a.quats, a.N, a.L, a.dim, Rm, tv);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * RS_TILE + threadIdx.x;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    if (j < a.m2) {
        const vec4<T> p = a.p2[j];
        const double qx = p.x, qy = p.y, qz = (a.dim == 3) ? (double)p.z : 0.0;
        double4 y;
        y.x = Rm[0] * qx + Rm[1] * qy + Rm[2] * qz + tv[0];
        y.y = Rm[3] * qx + Rm[4] * qy + Rm[5] * qz + tv[1];
        y.z = (a.dim == 3) ? Rm[6] * qx + Rm[7] * qy + Rm[8] * qz + tv[2] : 0.0;
        y.w = 0.0;
        reinterpret_cast<double4*>(a.moved)[(int64_t)pose * a.m2 + j] = y;
        lo[0] = hi[0] = (float)y.x; lo[1] = hi[1] = (float)y.y; lo[2] = hi[2] = (float)y.z;
    }
    block_bbox(lo, hi, wlo, whi, blo, bhi);
    if (threadIdx.x < 3) { tb[threadIdx.x] = blo[threadIdx.x]; tb[3 + threadIdx.x] = bhi[threadIdx.x]; }
}

// Pairs that pass the FP32 screen are queued per warp and evaluated 32 at a
// time in FP64 with every lane busy: only the pose's total is needed, so any
// lane may take any pair.
constexpr int RS_QUEUE = 256;  // pair slots per warp

template <typename T>
__global__ void __launch_bounds__(RS_TILE) k_rescore(RescoreArgs<T> a) {
    __shared__ double yx[RS_TILE], yy[RS_TILE], yz[RS_TILE], cr[RS_TILE], ci[RS_TILE];
    __shared__ double qx1[RS_TILE], qy1[RS_TILE], qz1[RS_TILE], ar1[RS_TILE], ai1[RS_TILE];
    __shared__ float4 fxyz[RS_TILE];  // FP32 copies of the moved samples for the screen (one load each)
    __shared__ unsigned short qpair[RS_WARPS][RS_QUEUE][2];  // (fixed slot, moving slot)
    __shared__ float wlo[RS_WARPS][3], whi[RS_WARPS][3];
    __shared__ float blo[3], bhi[3];
    __shared__ float slo[RS_WARPS][3], shi[RS_WARPS][3];  // boxes of the 32-sample slices of a moving tile
    __shared__ double tv[3];
    __shared__ int skip;
    const int pose = blockIdx.y;
    const Cand cd = reinterpret_cast<const Cand*>(a.top)[pose];
    if (cd.rot < 0) return;  // uniform over the block
    if (threadIdx.x == 0) {
        double Rm[9], t3[3];
        pose_of(cd, a.quats, a.N, a.L, a.dim, Rm, t3);
        tv[0] = t3[0]; tv[1] = t3[1]; tv[2] = t3[2];
    }
    const double sg2 = 2.0 * a.sigma_g * a.sigma_g;  // (sigma_g sqrt 2)^2
    const double inv_2sg2 = 1.0 / (2.0 * sg2);
    const double cut = 8.0 * sqrt(sg2);
    const float cut2f = (float)(cut * cut) * 1.001f;
    const double norm = (a.dim == 3) ? pow(2.0 * M_PI * sg2, -1.5) : 1.0 / (2.0 * M_PI * sg2);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.m1;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    float pxf = 0.f, pyf = 0.f, pzf = 0.f;
    {
        double px = 0, py = 0, pz = 0, ar = 0, ai = 0;
        if (live) {
            const vec4<T> p = a.p1[i];
            px = p.x; py = p.y; pz = (a.dim == 3) ? (double)p.z : 0.0;
            ar = a.c1[i].x; ai = a.c1[i].y;
            pxf = (float)px; pyf = (float)py; pzf = (float)pz;
            lo[0] = hi[0] = pxf; lo[1] = hi[1] = pyf; lo[2] = hi[2] = pzf;
        }
        qx1[threadIdx.x] = px; qy1[threadIdx.x] = py; qz1[threadIdx.x] = pz;
        ar1[threadIdx.x] = ar; ai1[threadIdx.x] = ai;
    }
    // this warp's box of fixed samples (every lane holds it)
    float flo[3], fhi[3];
    for (int d = 0; d < 3; ++d) {
        flo[d] = lo[d];
        fhi[d] = hi[d];
        for (int off = 16; off > 0; off >>= 1) {
            flo[d] = fminf(flo[d], __shfl_xor_sync(0xffffffffu, flo[d], off));
            fhi[d] = fmaxf(fhi[d], __shfl_xor_sync(0xffffffffu, fhi[d], off));
        }
    }
    block_bbox(lo, hi, wlo, whi, blo, bhi);
    // the moved samples lie in a ball of radius sqrt(r2max) around t
    if (threadIdx.x == 0) {
        double dd = 0.0;
        for (int d = 0; d < a.dim; ++d) {
            const double c = tv[d];
            const double e = c < blo[d] ? blo[d] - c : (c > bhi[d] ? c - bhi[d] : 0.0);
            dd += e * e;
        }
        const double reach = sqrt(a.r2max) * (1.0 + 1e-5) + cut * (1.0 + 1e-4) + 1e-6;
        skip = dd > reach * reach;
    }
    __syncthreads();
    if (skip) return;
    // tile test margin: float rounding of both boxes
    const double mag = fabs(tv[0]) + fabs(tv[1]) + fabs(tv[2]) + sqrt(a.r2max) + 1.0;
    const float cmarg = (float)(cut * (1.0 + 1e-4) + 1e-6 * mag);
    const float cm2 = cmarg * cmarg;
    const float blo0 = blo[0], blo1 = blo[1], blo2 = blo[2], bhi0 = bhi[0], bhi1 = bhi[1], bhi2 = bhi[2];
    const int ntiles = (int)((a.m2 + RS_TILE - 1) / RS_TILE);
    const float* tbase = a.tile_box + (int64_t)pose * ntiles * 6;
    const double4* moved = reinterpret_cast<const double4*>(a.moved) + (int64_t)pose * a.m2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned short(*queue)[2] = qpair[warp];
    int qn = 0;  // entries in this warp's queue (same value in every lane)
    double sr = 0.0, si = 0.0;
    auto drain = [&](int upto) {  // evaluate queue entries [0, upto) in FP64
        for (int q0 = 0; q0 < upto; q0 += 32) {
            const int q = q0 + lane;
            if (q < upto) {
                const int fi = queue[q][0], mj = queue[q][1];
                const double dx = yx[mj] - qx1[fi], dy = yy[mj] - qy1[fi], dz = yz[mj] - qz1[fi];
                const double g = norm * exp(-(dx * dx + dy * dy + dz * dz) * inv_2sg2);
                const double br = cr[mj] * g, bi = ci[mj] * g;
                sr += ar1[fi] * br - ai1[fi] * bi;
                si += ar1[fi] * bi + ai1[fi] * br;
            }
        }
    };
    // this CTA's share of the moving tiles (grid z splits them, so that the few
    // fixed blocks near the contact are spread over more CTAs)
    const int per = (ntiles + (int)gridDim.z - 1) / (int)gridDim.z;
    const int t_lo = (int)blockIdx.z * per, t_hi = min(ntiles, t_lo + per);
    for (int tile = t_lo; tile < t_hi; ++tile) {
        const float* tb = tbase + tile * 6;
        const float g0 = fmaxf(0.f, fmaxf(tb[0] - bhi0, blo0 - tb[3]));
        const float g1 = fmaxf(0.f, fmaxf(tb[1] - bhi1, blo1 - tb[4]));
        const float g2 = (a.dim == 3) ? fmaxf(0.f, fmaxf(tb[2] - bhi2, blo2 - tb[5])) : 0.f;
        if (g0 * g0 + g1 * g1 + g2 * g2 > cm2) continue;  // same decision in every thread
        const int64_t j = (int64_t)tile * RS_TILE + threadIdx.x;
        __syncthreads();
        {
            float mlo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mhi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
            if (j < a.m2) {
                const double4 y = moved[j];
                yx[threadIdx.x] = y.x; yy[threadIdx.x] = y.y; yz[threadIdx.x] = y.z;
                fxyz[threadIdx.x] = make_float4((float)y.x, (float)y.y, (float)y.z, 0.f);
                cr[threadIdx.x] = a.c2[j].x; ci[threadIdx.x] = a.c2[j].y;
                mlo[0] = mhi[0] = (float)y.x;
                mlo[1] = mhi[1] = (float)y.y;
                mlo[2] = mhi[2] = (float)y.z;
            }
            for (int d = 0; d < 3; ++d)
                for (int off = 16; off > 0; off >>= 1) {
                    mlo[d] = fminf(mlo[d], __shfl_down_sync(0xffffffffu, mlo[d], off));
                    mhi[d] = fmaxf(mhi[d], __shfl_down_sync(0xffffffffu, mhi[d], off));
                }
            if (lane == 0)
                for (int d = 0; d < 3; ++d) { slo[warp][d] = mlo[d]; shi[warp][d] = mhi[d]; }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)RS_TILE, a.m2 - (int64_t)tile * RS_TILE);
        for (int k = 0; k < cnt; ++k) {
            if ((k & 31) == 0) {  // skip a slice whose box is beyond the cutoff of this warp's box
                const int sl = k >> 5;
                const float h0 = fmaxf(0.f, fmaxf(slo[sl][0] - fhi[0], flo[0] - shi[sl][0]));
                const float h1 = fmaxf(0.f, fmaxf(slo[sl][1] - fhi[1], flo[1] - shi[sl][1]));
                const float h2 = (a.dim == 3) ? fmaxf(0.f, fmaxf(slo[sl][2] - fhi[2], flo[2] - shi[sl][2])) : 0.f;
                if (h0 * h0 + h1 * h1 + h2 * h2 > cm2) {  // same decision in every lane of the warp
                    k += 31;
                    continue;
                }
            }
            bool pass = false;
            if (live) {
                const float4 f = fxyz[k];
                const float dxf = f.x - pxf, dyf = f.y - pyf, dzf = f.z - pzf;
                pass = dxf * dxf + dyf * dyf + dzf * dzf <= cut2f;
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            if (m) {
                if (pass) {
                    const int slot = qn + __popc(m & ((1u << lane) - 1u));
                    queue[slot][0] = (unsigned short)threadIdx.x;
                    queue[slot][1] = (unsigned short)k;
                }
                qn += __popc(m);
                if (qn > RS_QUEUE - 32) {
                    __syncwarp();
                    drain(qn);
                    __syncwarp();
                    qn = 0;
                }
            }
        }
        __syncwarp();
        drain(qn);  // the tile's smem is overwritten by the next tile
        __syncwarp();
        qn = 0;
    }
    for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, off);
        si += __shfl_down_sync(0xffffffffu, si, off);
    }
    if (lane == 0) {
        atomicAdd(a.out + 2 * pose, sr);
        atomicAdd(a.out + 2 * pose + 1, si);
    }
}

template <typename T>
cudaError_t launch_rescore(const RescoreArgs<T>& a, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.out, 0, sizeof(double) * 2 * (a.k > 0 ? a.k : 1), st);
    if (e != cudaSuccess || a.k == 0 || a.m1 == 0 || a.m2 == 0) return e;
    const unsigned ntiles = (unsigned)((a.m2 + RS_TILE - 1) / RS_TILE);
    k_rescore_move<T><<<dim3(ntiles, a.k), RS_TILE, 0, st>>>(a);
    note_launch();
    // split the moving tiles over grid z until there are about 64 CTAs per SM
    // (most CTAs find their fixed block beyond reach of the pose and return)
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
    }
    const int64_t fixed_tiles = (a.m1 + RS_TILE - 1) / RS_TILE;
    const int64_t want = ((int64_t)64 * sms + fixed_tiles * a.k - 1) / (fixed_tiles * a.k);
    const unsigned groups = (unsigned)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)ntiles, 16}));
    const dim3 grid((unsigned)fixed_tiles, a.k, groups);
    k_rescore<T><<<grid, RS_TILE, 0, st>>>(a);
    note_launch();
    return cudaGetLastError();
}

template cudaError_t launch_rescore<float>(const RescoreArgs<float>&, cudaStream_t);
template cudaError_t launch_rescore<double>(const RescoreArgs<double>&, cudaStream_t);

int rescore_tiles(int64_t m2) { return (int)((m2 + RS_TILE - 1) / RS_TILE); }

}  // namespace sd
