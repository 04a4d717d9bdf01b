// Kernel argument blocks and host-side launchers of every device step.
//
// Layout conventions (all arrays complex, row-major, x fastest):
//   sub-box   : the spread target, s^d cells; cell a along an axis stands for the
//               oversampled-grid index u = a - s_h (mod n).  s = 2 s_h <= n.
//   modes     : kappa in [-N/2, N/2) stored at kappa mod N along each axis.
//   score map : t index i in [0, N) per axis, t = (i - N/2) h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "../../include/sdfdock.h"

namespace sd {

// Stream-ordered allocation from the device's memory pool (defined in api.cu).
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);
void pool_free(void* p, cudaStream_t st);

// ---- SDF (Eq. 10A-17t) ------------------------------------------------------
template <typename T>
struct SdfArgs {
    const vec4<T>* bnd;   // n_b boundary positions
    const vec4<T>* nrm;   // n_b unit outward normals
    const T* area;        // n_b
    int64_t n_b;
    const vec4<T>* qry;   // m query points
    const T* vol;         // m
    int64_t m;
    const int8_t* pmc_override;  // m or null
    T lam1, lam2, sigma, eps;    // eps < 0 disables truncation
    int phi;                     // SD_PHI_* (kernel of Eq. 13)
    T radius;                    // R of the radial and skin / core kernels
    // outputs / intermediates
    T* xi_abs;            // m: nearest distance
    int8_t* pmc;          // m: +1 / -1
    cplx<T>* c_out;       // m: rho * vol
    cplx<T>* rho_out;     // m or null (caller order)
    vec4<T>* pos_out;     // m: copy of the query points for the shape (processing order)
    const int32_t* perm_q;  // processing order of the queries (caller index), or null
    const float* tile_box;  // boundary tile boxes (n_tiles x 6: lo, hi), or null
    const float* sub_box;   // boxes of 32-sample sub-tiles (n_tiles * SDF_TILE / 32 x 6), or null
    int64_t n_tiles;        // boundary tiles of SDF_TILE samples
};
// Boundary samples gathered into Morton order: positions, normals with the
// area in .w, the bounding box of every tile of SDF_TILE samples (tile_box,
// n_tiles x 6) followed by those of its 32-sample sub-tiles
// (n_tiles * SDF_TILE / 32 x 6 more floats).
template <typename T>
cudaError_t launch_boundary_order(const vec4<T>* bnd, const vec4<T>* nrm, const T* area, const int32_t* perm,
                                  int64_t n_b, int dim, vec4<T>* bnd_s, vec4<T>* nrm_s, float* tile_box,
                                  cudaStream_t st);
constexpr int SDF_TILE = 256;
template <typename T> cudaError_t launch_sdf(const SdfArgs<T>& a, int dim, cudaStream_t st);

// max |p| over m points (result in *out, device double)
template <typename T> cudaError_t launch_radius(const vec4<T>* p, int64_t m, int dim, double* out,
                                                cudaStream_t st);

// ---- type-1 spreading -------------------------------------------------------
template <typename T>
struct SpreadArgs {
    const vec4<T>* pos;   // m sample positions
    const cplx<T>* c;     // m sample weights
    int64_t m;
    const double* quats;  // rotation list (w, x, y, z); null = identity
    int64_t rot0;         // first rotation of this batch
    T sign;               // spread at sign * R p
    T inv_h;              // 1 / h' (oversampled spacing)
    T beta;               // ES kernel shape
    int w;                // kernel width (cells)
    int s, s_h;           // sub-box side and half-side
    cplx<T>* out;         // batch x s^d
    int64_t out_rot_stride;
    int n_full;           // oversampled grid length n (s == n means periodic wrap)
};
template <typename T> cudaError_t launch_spread(const SpreadArgs<T>& a, int dim, int batch, cudaStream_t st);

// Bins of the spread sub-box (tb^d cells each) and the per-rotation sample order.
struct BinArgs {
    int tb;               // cells per bin along an axis: 8, 12 or 16
    int nb;               // bins per axis = ceil(s / tb)
    int nbins;            // nb^d
    int* count;           // batch x nbins
    int* cmax;            // batch x nbins, right after count: each bin's largest |component| of c
                          // (float bits), for the fixed-point scale of its tile
    int* offset;          // batch x (nbins + 1)
    int* bin_of;          // batch x m
    int* rank;            // batch x m
    int32_t* sorted;      // batch x m: sample indices in bin order
    int32_t* org;         // batch x m: packed tap-box origin (x | y << 10 | z << 20), fused spreading only
};
// Spread by bins; accumulates into the batch's sub-boxes, which must be cleared first.
// Supports w = 4..7 and tb = 8, 12, 16 (shared tile of (tb + w - 1)^d cells).
template <typename T>
cudaError_t launch_spread_bins(const SpreadArgs<T>& a, const BinArgs& bn, int dim, int batch, cudaStream_t st);

// Spread by blocks of Morton-consecutive samples: each CTA accumulates its
// samples' taps in a shared box and adds the box to the sub-box (which must be
// cleared first).  FP32, w = 4..7; other precisions spread directly.
template <typename T> cudaError_t launch_spread_box(const SpreadArgs<T>& a, int dim, int batch, cudaStream_t st);

// Spreading fused with the forward x transform of the pruned 3D search (FP32,
// w = 6, 2 s <= n): the samples are binned by the (y, z) of their tap box in
// bins of SPREADX_TY x SPREADX_TZ cells (bn.nb = bins along y, nbz along z,
// bn.nbins = nb * nbz), then each bin's CTA writes the N kept x modes of its
// rows to out (batch x s^2 rows x N, row (y, z) at z s + y).  No sub-box.  Both
// sides are at least w - 1, so a tap box meets at most 2 x 2 bins; 6 x 6 rows
// keep a CTA's shared memory to three CTAs per SM at n = 384 (measured faster
// than 5 x 6).
constexpr int SPREADX_TY = 6, SPREADX_TZ = 6;
template <typename T>
cudaError_t launch_spread_x(const SpreadArgs<T>& a, const BinArgs& bn, int nbz, cplx<T>* out, int64_t out_rot_stride,
                            const cplx<T>* tw, int batch, cudaStream_t st);

// ---- line passes ------------------------------------------------------------
// *_P modes are the pruned forward passes of the search: the sub-box is read
// unshifted (cell a at position a, a < s <= n/2; the shift is a phase folded
// into W, see launch_wshift), and only the N = n/2 central modes are computed.
// ROW_INV_TOPK*: inverse x keeping each block's 2 / 4 / 8 / 16 best translations.
enum RowMode {
    ROW_FWD = 0, ROW_INV_ARGMAX = 1, ROW_INV_MAP = 2, ROW_EXPAND = 3, ROW_FWD_P = 4,
    ROW_INV_TOPK2 = 8, ROW_INV_TOPK4 = 9, ROW_INV_TOPK8 = 10, ROW_INV_TOPK16 = 11
};
enum ColMode { COL_FWD = 0, COL_INV = 1, COL_FUSED = 2, COL_EXPAND = 3, COL_FWD_P = 4, COL_FUSED_P = 5 };

// Whether the pruned passes serve an oversampled length n (a host-side copy of
// prunable_len for the lengths the library builds).
inline bool pruned_len_ok(int n) {
    switch (n) {
        case 16: case 32: case 64: case 96: case 128: case 192: case 256: case 384: case 512: return true;
        default: return false;
    }
}

template <typename T>
struct RowArgs {
    const cplx<T>* in;
    cplx<T>* out;
    int64_t in_rot_stride, out_rot_stride;
    int nrows, in_row_stride, out_row_stride;
    int len_in;   // ROW_FWD: s (data at u = e - s_h); others: N
    int s_h;
    int N;        // modes / outputs per line
    int n;        // oversampled length (ROW_FWD, ROW_EXPAND)
    const cplx<T>* tw;        // twiddles of the transform length
    double* part_score;       // ROW_INV_ARGMAX: batch x gridDim.x
    int* part_idx;
};
template <typename T> cudaError_t launch_rows(int mode, const RowArgs<T>& a, int batch, int* nparts,
                                              cudaStream_t st);
// Inverse y and x of whole z-planes in thread-block clusters (3D, FP32, modes
// ROW_INV_ARGMAX / ROW_INV_MAP): a.in is the rotation's N^3 volume (z, ky, kx)
// after the last-axis pass, a.nrows = N^2, row strides N; *nparts receives the
// argmax partials per rotation (N times the cluster size).
template <typename T> cudaError_t launch_inv_yx(int mode, const RowArgs<T>& a, int batch, int* nparts,
                                                cudaStream_t st);
inline bool inv_yx_supported(int N) {
    return N == 32 || N == 48 || N == 64 || N == 96 || N == 128 || N == 192 || N == 256;
}

template <typename T>
struct ColArgs {
    const cplx<T>* in;
    cplx<T>* out;
    int64_t in_rot_stride, out_rot_stride;
    int ncols;                          // contiguous columns; element stride along the axis
    int nouter;
    int64_t in_outer_stride, out_outer_stride;
    int len_in;                         // COL_FWD / COL_FUSED: s; others N
    int s_h;
    int N, n;
    const cplx<T>* twF;                 // twiddles of n (forward / expand)
    const cplx<T>* twI;                 // twiddles of N (inverse)
    const cplx<T>* W;                   // COL_FUSED: N x ncols table
    int rot_fastest;                    // COL_FUSED: grid (batch, column blocks), W reused from L2
    int lines;                          // COL_FWD_P / COL_FUSED_P: columns per CTA (LINES_*)
};
enum { LINES_STD = 0, LINES_NARROW = 1, LINES_WIDE = 2 };  // standard, half, twice
template <typename T> cudaError_t launch_cols(int mode, const ColArgs<T>& a, int batch, cudaStream_t st);

// twiddles exp(-2 pi i j / len), computed in FP64
template <typename T> cudaError_t launch_twiddles(cplx<T>* tw, int len, cudaStream_t st);

// ---- tables (FP64) ------------------------------------------------------------
// D[kappa'] = (w/2) * psihat(pi * kappa * w / n), kappa' in [0, N), by Gauss-Legendre
// quadrature of the ES kernel (nodes/weights on [0, pi/2] after z = sin(theta)).
cudaError_t launch_deconv(double* D, int N, int n, int w, double beta, const double* gl_x,
                          const double* gl_w, int nq, cudaStream_t st);

// W = (-1)^{sum kappa} exp(-sg^2 |k|^2) B1 / (L^d prod D^2); zero on Nyquist.
// shift = 0 drops the (-1)^{sum kappa} factor; deriv = -1 (none) or axis a
// multiplies by i k_a.
template <typename T>
cudaError_t launch_wtable(const cplx<T>* B1, const double* D, int N, int dim, double L, double sigma_g,
                          int shift, int deriv, cplx<T>* W, cudaStream_t st);

// W' = W exp(2 pi i s_h sum_d kappa_d / n): the product table of a search whose
// forward passes read the sub-box unshifted (the *_P modes).
template <typename T>
cudaError_t launch_wshift(const cplx<T>* W, int N, int dim, int n, int s_h, cplx<T>* out, cudaStream_t st);

// top-K partials (K per block, K in {2, 4, 8, 16}) -> the k_r <= K best
// candidates of each rotation (score descending, index ascending)
cudaError_t launch_reduce_topk(const double* part_score, const int* part_idx, int nparts, int K, int k_r, int batch,
                               int64_t rot0, void* cand, cudaStream_t st);

// argmax partials -> one candidate per rotation
cudaError_t launch_reduce_argmax(const double* part_score, const int* part_idx, int nparts, int batch,
                                 int64_t rot0, void* cand, cudaStream_t st);

// field f of 4 into its plane of the halo-padded type-2 tables
template <typename T>
cudaError_t launch_interleave(const cplx<T>* src, cplx<T>* dst, int n, int pn, int dim, int f, cudaStream_t st);

// ---- search -----------------------------------------------------------------
cudaError_t launch_topk(const void* cand, int64_t n, int k, void* out_cand, unsigned* flags,
                        cudaStream_t st);
template <typename T>
struct RescoreArgs {
    const vec4<T>* p1; const cplx<T>* c1; int64_t m1;
    const vec4<T>* p2; const cplx<T>* c2; int64_t m2;
    const void* top;          // k sd_cand
    int k;
    const double* quats;
    int N; double L; double sigma_g; int dim;
    double r2max;             // squared bounding radius of the moving samples
    double* out;              // k x 2 (re, im)
    void* moved;              // scratch: k x m2 double4 (moved samples)
    float* tile_box;          // scratch: k x rescore_tiles(m2) x 6 (lo, hi)
};
template <typename T> cudaError_t launch_rescore(const RescoreArgs<T>& a, cudaStream_t st);
int rescore_tiles(int64_t m2);

// Morton order (permutation) of points inside the cube [-radius, radius]^d.
template <typename T>
cudaError_t morton_order(const vec4<T>* pos, int64_t m, double radius, int dim, int32_t* perm, cudaStream_t st);

// Reorder a shape's samples by the Morton code of their position (in place).
template <typename T>
cudaError_t sort_by_morton(vec4<T>* pos, cplx<T>* c, int64_t m, double radius, int dim, cudaStream_t st);

// ---- type-2 gather: score and gradient ---------------------------------------
template <typename T>
struct GatherArgs {
    const vec4<T>* p2; const cplx<T>* c2; int64_t m2;
    const T* quats;           // P x 4
    const T* trans;           // P x 3
    int64_t P;
    const cplx<T>* G;         // two planes of pn^d cells: (Phi, dPhi/dx), (dPhi/dy, dPhi/dz)
    int n;                    // periodic grid size per axis
    int pn;                   // pitch of the planes: n plus a halo of w cells repeating the field
    T inv_h, beta;
    int w;
    double* acc;              // P x 8
};
template <typename T> cudaError_t launch_gather(const GatherArgs<T>& a, int dim, cudaStream_t st);
template <typename T> cudaError_t launch_grad_finalize(const double* acc, const T* quats, int64_t P, int dim,
                                                       T* score, T* dq, T* dt, cudaStream_t st);
// Pose-update rule of the refinement loop (values of sd_refine_params.method).
struct RefineParams {
    int method;
    double lr_t, lr_q, mass, inertia, damping, h;
};
template <typename T> cudaError_t launch_refine_step(const double* acc, T* quats, T* trans, double* state, int64_t P,
                                                     int dim, const RefineParams& rp, int first, T* hist, int last,
                                                     cudaStream_t st);

}  // namespace sd
