// C ABI of the SDF complementarity library: contexts, shapes, plans and the
// per-call pipelines.  See include/sdfdock.h for the contract of every entry.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <atomic>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sdfdock.h"
#include "fft.cuh"
#include "kernels.cuh"

using namespace sd;

// ---------------------------------------------------------------------------
// context and shapes
// ---------------------------------------------------------------------------

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Prep {  // fixed-shape tables for one grid
    int N = 0;
    double L = 0;
    void* B1 = nullptr;  // N^d: spread + forward FFT of the fixed samples (deconvolution pending)
    void* W = nullptr;   // N^d: the product table of the search
    void* G = nullptr;   // n^d x 4: Phi and its gradient on the oversampled grid
    // W times the phase of an unshifted sub-box of half-side s_h (the pruned
    // passes), one per s_h met: (s_h, table)
    std::vector<std::pair<int, void*>> Wsh;
};

struct TimerRec {
    int kind;
    cudaEvent_t a, b;
    bool pooled = true;  // false: the events belong to a captured graph
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> events;  // event nodes of a multi-job graph (owned)
    std::vector<TimerRec> timers;     // pass-timing event nodes (owned), read back after each replay
    long long kernels = 0;            // kernel launches captured (counted again at every replay)
};

// Bin side of binned spreading when it is asked for without the autotuner.
constexpr int DEFAULT_BIN = 16;

struct Plan {      // launch plan of one scoring job
    int B = 1;     // rotations per launch sequence
    int bins = 0;  // bin side (8, 12, 16) of bin-sorted spreading, 0: direct,
                   // 1: spreading fused with the forward x transform (SPREAD_X),
                   // 2: shared boxes of sample blocks (SPREAD_BOX)
    int fft = SD_FFT_PRUNED;  // forward-pass plan (SD_FFT_FULL / _PRUNED / _PRUNED_NARROW / _PRUNED_WIDE)
};

struct sd_ctx {
    int device = 0;
    int opt_timing = 0;
    std::vector<TimerRec> pending;       // event pairs not yet read back
    std::vector<TimerRec>* capture_timers = nullptr;  // while capturing a graph with "timing" on
    std::vector<cudaEvent_t> event_pool;
    double pass_ms[SD_PASS_COUNT] = {};
    int64_t pass_n[SD_PASS_COUNT] = {};
    sd_params p{};
    std::string err;
    int64_t opt_batch = 0;
    int opt_graph = 0;
    int opt_plain = 0;
    int opt_spread_direct = 1;  // 0: spread by bins
    int opt_pruned = 1;         // 0: forward passes read the shifted sub-box and compute every mode
    int opt_fft_plan = -1;      // >= 0: this SD_FFT_* plan wherever it applies (not tuned)
    int opt_inv_cluster = 0;    // 1: inverse y and x of whole z-planes in thread-block clusters (3D FP32)
    int opt_bin_side = DEFAULT_BIN;  // bin side of binned spreading when it is not tuned
    int opt_spread_fused = 0;   // 1: spreading fused with the forward x transform where available
    int opt_spread_box = 0;     // 1: spreading by shared boxes of sample blocks
    int opt_sdf_cull = 2;       // 0: SDF sums over every boundary tile; 1: skip far tiles; 2: and far sub-tiles per warp
    int opt_autotune = 0;       // 1: time candidate plans per job geometry
    std::map<std::string, Plan> tuned;
    DevBuf ws[8];
    std::map<std::pair<int, int>, void*> twiddles;  // (len, precision)
    std::map<std::tuple<int, int, int, double>, double*> deconv;
    double* gl_x = nullptr;
    double* gl_w = nullptr;
    int nq = 0;
    std::map<std::string, GraphEntry> graphs;
    std::deque<std::string> graph_order;  // keys of `graphs`, oldest first
    std::map<std::string, int> seen;
};

struct sd_shape {
    sd_ctx* ctx = nullptr;
    int64_t m = 0;
    void* pos = nullptr;  // m x 4 real
    void* c = nullptr;    // m x 2 real
    double radius = 0.0;
    std::vector<Prep> preps;
};

static std::string g_create_err;
static std::atomic<long long> g_launches{0};

void sd::note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// CUDA-event timing of one pass launch on the stream (when the context's
// "timing" option is on).  While a graph is captured the two events become
// event-record nodes of the graph, read back after each of its replays.
static cudaEvent_t pool_event(sd_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

struct PassTimer {
    sd_ctx* ctx;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    PassTimer(sd_ctx* c, int k, cudaStream_t s, bool on) : ctx(c), kind(k), st(s) {
        if (!on || !c->opt_timing) return;
        if (c->capture_timers) {
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventRecordWithFlags(a, s, cudaEventRecordExternal) != cudaSuccess) {
                if (a) cudaEventDestroy(a);
                a = nullptr;
                cudaGetLastError();
            }
            return;
        }
        a = pool_event(c);
        if (a) cudaEventRecord(a, s);
    }
    ~PassTimer() {
        if (!a) return;
        if (ctx->capture_timers) {
            cudaEvent_t b = nullptr;
            if (cudaEventCreate(&b) != cudaSuccess || cudaEventRecordWithFlags(b, st, cudaEventRecordExternal) != cudaSuccess) {
                if (b) cudaEventDestroy(b);
                cudaEventDestroy(a);
                cudaGetLastError();
                return;
            }
            ctx->capture_timers->push_back({kind, a, b, false});
            return;
        }
        cudaEvent_t b = pool_event(ctx);
        if (!b) return;
        cudaEventRecord(b, st);
        ctx->pending.push_back({kind, a, b});
    }
};

static void harvest_timers(sd_ctx* ctx) {
    for (auto& r : ctx->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            ctx->pass_ms[r.kind] += ms;
            ctx->pass_n[r.kind] += 1;
        } else {
            cudaGetLastError();
        }
        if (r.pooled) {
            ctx->event_pool.push_back(r.a);
            ctx->event_pool.push_back(r.b);
        }
    }
    ctx->pending.clear();
}

static int fail(sd_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_err = buf;
    return code;
}

#define CK(ctx, x)                                                                            \
    do {                                                                                      \
        cudaError_t e_ = (x);                                                                 \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SD_ERR_OOM : SD_ERR_CUDA,      \
                        "%s failed: %s", #x, cudaGetErrorString(e_));                         \
    } while (0)

#define CKI(x)                  \
    do {                        \
        int r_ = (x);           \
        if (r_ != SD_OK) return r_; \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static size_t real_size(const sd_ctx* ctx) { return ctx->p.precision == SD_F64 ? 8 : 4; }

// Per-call and per-shape buffers come from the device's stream-ordered memory
// pool (its release threshold is raised when a context is created), so repeated
// shape builds and table preparations reuse memory instead of paying for
// cudaMalloc/cudaFree and their device synchronisation.
cudaError_t sd::pool_alloc(void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    return cudaMallocAsync(p, bytes ? bytes : 1, st);
}
void sd::pool_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

// Captured graphs hold raw workspace and table pointers: drop them before any
// of those buffers is freed.
static void release_graph(GraphEntry& g) {
    cudaGraphExecDestroy(g.exec);
    for (auto e : g.events) cudaEventDestroy(e);
    for (auto& t : g.timers) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
}

static void drop_graphs(sd_ctx* ctx) {
    harvest_timers(ctx);  // pending reads may name a graph's timing events
    for (auto& kv : ctx->graphs) release_graph(kv.second);
    ctx->graph_order.clear();
    ctx->graphs.clear();
    ctx->seen.clear();
}

// Keeps a newly captured graph; the cache holds at most 64, the oldest going
// first (an executable graph or event still in flight is released when it
// completes).  The first-call markers are bounded too.
static std::map<std::string, GraphEntry>::iterator keep_graph(sd_ctx* ctx, const std::string& k,
                                                             const GraphEntry& ge) {
    constexpr size_t kMaxGraphs = 64;
    while (ctx->graphs.size() >= kMaxGraphs && !ctx->graph_order.empty()) {
        auto old = ctx->graphs.find(ctx->graph_order.front());
        if (old != ctx->graphs.end()) {
            if (!old->second.timers.empty()) harvest_timers(ctx);
            release_graph(old->second);
            ctx->graphs.erase(old);
        }
        ctx->graph_order.pop_front();
    }
    if (ctx->seen.size() > 4096) ctx->seen.clear();
    ctx->graph_order.push_back(k);
    return ctx->graphs.emplace(k, ge).first;
}

static int ws_get(sd_ctx* ctx, int slot, size_t bytes, void** out) {
    DevBuf& b = ctx->ws[slot];
    if (b.bytes < bytes) {
        drop_graphs(ctx);
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        size_t want = bytes + bytes / 8 + 256;
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, SD_ERR_OOM, "workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
        }
        b.bytes = want;
    }
    *out = b.p;
    return SD_OK;
}

static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    // roots of P_n by Newton's method; weights 2 / ((1 - x^2) P_n'(x)^2)
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p2 = p1;
                p1 = p0;
                p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
            }
            dp = n * (z * p0 - p1) / (z * z - 1.0);
            const double dz = p0 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = 0.0;
        for (int j = 1; j <= n; ++j) {
            const double p2 = p1;
            p1 = p0;
            p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
        }
        dp = n * (z * p0 - p1) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static int get_twiddles(sd_ctx* ctx, int len, void** out, cudaStream_t st) {
    auto key = std::make_pair(len, ctx->p.precision);
    auto it = ctx->twiddles.find(key);
    if (it != ctx->twiddles.end()) {
        *out = it->second;
        return SD_OK;
    }
    void* p = nullptr;
    CK(ctx, cudaMalloc(&p, (size_t)len * 2 * real_size(ctx)));
    if (ctx->p.precision == SD_F64) CK(ctx, launch_twiddles<double>((double2*)p, len, st));
    else CK(ctx, launch_twiddles<float>((float2*)p, len, st));
    ctx->twiddles[key] = p;
    *out = p;
    return SD_OK;
}

static int get_deconv(sd_ctx* ctx, int N, int n, double** out, cudaStream_t st) {
    auto key = std::make_tuple(N, n, ctx->p.w, ctx->p.beta);
    auto it = ctx->deconv.find(key);
    if (it != ctx->deconv.end()) {
        *out = it->second;
        return SD_OK;
    }
    if (!ctx->gl_x) {
        std::vector<double> x, w;
        const int nq = 96;
        gauss_legendre(nq, x, w);
        for (int i = 0; i < nq; ++i) {  // map [-1, 1] -> [0, pi/2]
            x[i] = (x[i] + 1.0) * (M_PI / 4.0);
            w[i] *= M_PI / 4.0;
        }
        CK(ctx, cudaMalloc(&ctx->gl_x, nq * sizeof(double)));
        CK(ctx, cudaMalloc(&ctx->gl_w, nq * sizeof(double)));
        CK(ctx, cudaMemcpy(ctx->gl_x, x.data(), nq * sizeof(double), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(ctx->gl_w, w.data(), nq * sizeof(double), cudaMemcpyHostToDevice));
        ctx->nq = nq;
    }
    double* D = nullptr;
    CK(ctx, cudaMalloc(&D, N * sizeof(double)));
    CK(ctx, launch_deconv(D, N, n, ctx->p.w, ctx->p.beta, ctx->gl_x, ctx->gl_w, ctx->nq, st));
    ctx->deconv[key] = D;
    *out = D;
    return SD_OK;
}

// ---------------------------------------------------------------------------
// geometry of one search: grid sizes and the moving shape's sub-box
// ---------------------------------------------------------------------------

struct Geo {
    int dim, N, n;
    double L, inv_h;
    int s, s_h;
    int64_t cells_box;  // s^d
};

static bool grid_ok(int N) {
    switch (N) {
        case 8: case 16: case 24: case 32: case 48: case 64: case 96: case 128: case 192: case 256: return true;
        default: return false;
    }
}

static int make_geo(sd_ctx* ctx, const sd_grid* g, double radius, Geo* out) {
    if (!g) return fail(ctx, SD_ERR_ARG, "grid is NULL");
    if (!grid_ok(g->N)) return fail(ctx, SD_ERR_ARG, "unsupported grid size N=%d", g->N);
    if (!(g->L > 0.0) || !isfinite(g->L)) return fail(ctx, SD_ERR_ARG, "box side L must be positive and finite");
    Geo G;
    G.dim = ctx->p.dim;
    G.N = g->N;
    G.n = ctx->p.alpha * g->N;
    G.L = g->L;
    G.inv_h = (double)G.n / g->L;
    const double reach = radius * G.inv_h + 0.5 * ctx->p.w;
    if (reach > 1.5 * G.n) return fail(ctx, SD_ERR_ARG, "shape radius %.6g exceeds the periodic box", radius);
    int s_h = (int)floor(reach) + 2;
    if (2 * s_h >= G.n) s_h = G.n / 2;
    G.s_h = s_h;
    G.s = 2 * s_h;
    G.cells_box = (G.dim == 2) ? (int64_t)G.s * G.s : (int64_t)G.s * G.s * G.s;
    *out = G;
    return SD_OK;
}

// ---------------------------------------------------------------------------
// forward transform of a spread sub-box: box -> N^d modes (kappa mod N order)
// ---------------------------------------------------------------------------
//
// 3D: box (s,s,s) -x-> (s,s,N) -y-> (s,N,N) -z-> (N,N,N)   (last step FWD or FUSED)
// 2D: box (s,s)   -x-> (s,N)   -y-> (N,N)

template <typename T>
struct Tw {
    const cplx<T>* n;
    const cplx<T>* N;
};

template <typename T>
static int get_tw(sd_ctx* ctx, const Geo& G, Tw<T>* tw, cudaStream_t st) {
    void *a, *b;
    CKI(get_twiddles(ctx, G.n, &a, st));
    CKI(get_twiddles(ctx, G.N, &b, st));
    tw->n = (const cplx<T>*)a;
    tw->N = (const cplx<T>*)b;
    return SD_OK;
}

// x pass: rows of the box
template <typename T>
static cudaError_t pass_x_fwd(const Geo& G, const Tw<T>& tw, const cplx<T>* in, int64_t in_rs, cplx<T>* out,
                              int64_t out_rs, int batch, cudaStream_t st, int mode = ROW_FWD) {
    RowArgs<T> r{};
    r.in = in;
    r.out = out;
    r.in_rot_stride = in_rs;
    r.out_rot_stride = out_rs;
    r.nrows = (G.dim == 2) ? G.s : G.s * G.s;
    r.in_row_stride = G.s;
    r.out_row_stride = G.N;
    r.len_in = G.s;
    r.s_h = G.s_h;
    r.N = G.N;
    r.n = G.n;
    r.tw = tw.n;
    return launch_rows<T>(mode, r, batch, nullptr, st);
}

// y pass (3D): (s,s,N) -> (s,N,N)
template <typename T>
static cudaError_t pass_y_fwd(const Geo& G, const Tw<T>& tw, const cplx<T>* in, int64_t in_rs, cplx<T>* out,
                              int64_t out_rs, int batch, cudaStream_t st, int mode = COL_FWD, int lines = LINES_STD) {
    ColArgs<T> c{};
    c.lines = lines;
    c.in = in;
    c.out = out;
    c.in_rot_stride = in_rs;
    c.out_rot_stride = out_rs;
    c.ncols = G.N;
    c.nouter = G.s;
    c.in_outer_stride = (int64_t)G.s * G.N;
    c.out_outer_stride = (int64_t)G.N * G.N;
    c.len_in = G.s;
    c.s_h = G.s_h;
    c.N = G.N;
    c.n = G.n;
    c.twF = tw.n;
    c.twI = tw.N;
    return launch_cols<T>(mode, c, batch, st);
}

// last axis (z in 3D, y in 2D): FWD (modes) or FUSED (product with W, inverse)
template <typename T>
static cudaError_t pass_last(int mode, const Geo& G, const Tw<T>& tw, const cplx<T>* in, int64_t in_rs,
                             cplx<T>* out, int64_t out_rs, const cplx<T>* W, int batch, cudaStream_t st,
                             int lines = LINES_STD) {
    ColArgs<T> c{};
    c.lines = lines;
    c.in = in;
    c.out = out;
    c.in_rot_stride = in_rs;
    c.out_rot_stride = out_rs;
    c.ncols = (G.dim == 2) ? G.N : G.N * G.N;
    c.nouter = 1;
    c.in_outer_stride = 0;
    c.out_outer_stride = 0;
    c.len_in = G.s;
    c.s_h = G.s_h;
    c.N = G.N;
    c.n = G.n;
    c.twF = tw.n;
    c.twI = tw.N;
    c.W = W;
    // W larger than a quarter of the 129 MB L2 would be evicted between rotations
    // by the streaming data: let the batch's rotations share each block of it
    const int64_t w_bytes = (int64_t)c.ncols * G.N * (int64_t)sizeof(cplx<T>);
    c.rot_fastest = ((mode == COL_FUSED || mode == COL_FUSED_P) && w_bytes > ((int64_t)32 << 20)) ? 1 : 0;
    return launch_cols<T>(mode, c, batch, st);
}

// inverse y (3D): (N,N,N) in place
template <typename T>
static cudaError_t pass_y_inv(const Geo& G, const Tw<T>& tw, cplx<T>* buf, int64_t rs, int batch, cudaStream_t st) {
    ColArgs<T> c{};
    c.in = buf;
    c.out = buf;
    c.in_rot_stride = rs;
    c.out_rot_stride = rs;
    c.ncols = G.N;
    c.nouter = G.N;
    c.in_outer_stride = (int64_t)G.N * G.N;
    c.out_outer_stride = (int64_t)G.N * G.N;
    c.len_in = G.N;
    c.s_h = 0;
    c.N = G.N;
    c.n = G.n;
    c.twF = tw.N;
    c.twI = tw.N;
    return launch_cols<T>(COL_INV, c, batch, st);
}

// Bin workspace of one spread batch (slot 6) with bins of tb^d cells: its size
// and its layout.
static size_t bins_bytes(int s, int dim, int64_t m, int batch, int tb) {
    const int nb = (s + tb - 1) / tb;
    const int nbins = (dim == 2) ? nb * nb : nb * nb * nb;
    const size_t ints = (size_t)batch * (3 * (size_t)nbins + 1) + 3 * (size_t)batch * (size_t)m;
    return ints * sizeof(int);
}

static void bins_layout(void* p, int s, int dim, int64_t m, int batch, int tb, BinArgs* bn) {
    const int nb = (s + tb - 1) / tb;
    const int nbins = (dim == 2) ? nb * nb : nb * nb * nb;
    int* q = (int*)p;
    bn->tb = tb;
    bn->nb = nb;
    bn->nbins = nbins;
    bn->count = q;
    q += (size_t)batch * nbins;
    bn->cmax = q;
    q += (size_t)batch * nbins;
    bn->offset = q;
    q += (size_t)batch * (nbins + 1);
    bn->bin_of = q;
    q += (size_t)batch * m;
    bn->rank = q;
    q += (size_t)batch * m;
    bn->sorted = q;
    bn->org = nullptr;  // tiles re-evaluate the origin (with a safety net)
}

static int bins_for(sd_ctx* ctx, int s, int dim, int64_t m, int batch, int tb, BinArgs* bn) {
    void* p = nullptr;
    CKI(ws_get(ctx, 6, bins_bytes(s, dim, m, batch, tb), &p));
    bins_layout(p, s, dim, m, batch, tb, bn);
    return SD_OK;
}

// Plan.bins value of spreading fused with the forward x transform.
constexpr int SPREAD_X = 1;
// Plan.bins value of spreading by blocks of Morton-consecutive samples.
constexpr int SPREAD_BOX = 2;

// Bin workspace of the fused spreading (bins over (y, z)).
static int spread_x_bins(int s, int* nby, int* nbz) {
    *nby = (s + SPREADX_TY - 1) / SPREADX_TY;
    *nbz = (s + SPREADX_TZ - 1) / SPREADX_TZ;
    return *nby * *nbz;
}
static size_t bins_bytes_x(int s, int64_t m, int batch) {
    int nby, nbz;
    const int nbins = spread_x_bins(s, &nby, &nbz);
    return ((size_t)batch * (3 * (size_t)nbins + 1) + 4 * (size_t)batch * (size_t)m) * sizeof(int);
}
static void bins_layout_x(void* p, int s, int64_t m, int batch, BinArgs* bn, int* nbz) {
    int nby;
    const int nbins = spread_x_bins(s, &nby, nbz);
    int* q = (int*)p;
    bn->tb = SPREADX_TY;
    bn->nb = nby;
    bn->nbins = nbins;
    bn->count = q;
    q += (size_t)batch * nbins;
    bn->cmax = q;
    q += (size_t)batch * nbins;
    bn->offset = q;
    q += (size_t)batch * (nbins + 1);
    bn->bin_of = q;
    q += (size_t)batch * m;
    bn->rank = q;
    q += (size_t)batch * m;
    bn->sorted = q;
    q += (size_t)batch * m;
    bn->org = q;
}

// Binned spreading exists for FP32 and kernel widths 4-7 (tiles of tb + w - 1 cells).
static bool bins_supported(const sd_ctx* ctx) { return ctx->p.precision == SD_F32 && ctx->p.w >= 4 && ctx->p.w <= 7; }

// ---------------------------------------------------------------------------
// fixed-shape preparation for a grid
// ---------------------------------------------------------------------------

template <typename T>
static int prep_fixed(sd_ctx* ctx, sd_shape* fx, const sd_grid* g, Prep** out, cudaStream_t st) {
    for (auto& p : fx->preps)
        if (p.N == g->N && p.L == g->L) {
            *out = &p;
            return SD_OK;
        }
    using C = cplx<T>;
    Geo G;
    CKI(make_geo(ctx, g, fx->radius, &G));
    Tw<T> tw;
    CKI(get_tw<T>(ctx, G, &tw, st));
    double* D = nullptr;
    CKI(get_deconv(ctx, G.N, G.n, &D, st));
    const int64_t Nd = (G.dim == 2) ? (int64_t)G.N * G.N : (int64_t)G.N * G.N * G.N;
    const int64_t sz0 = G.cells_box;
    const int64_t sz1 = (G.dim == 2) ? (int64_t)G.s * G.N : (int64_t)G.s * G.s * G.N;
    const int64_t sz2 = (G.dim == 2) ? 0 : (int64_t)G.s * G.N * G.N;
    C *b0 = nullptr, *b1 = nullptr, *b2 = nullptr, *B1 = nullptr, *W = nullptr;
    CK(ctx, pool_alloc((void**)&b0, sz0 * sizeof(C), st));
    CK(ctx, pool_alloc((void**)&b1, sz1 * sizeof(C), st));
    if (sz2) CK(ctx, pool_alloc((void**)&b2, sz2 * sizeof(C), st));
    CK(ctx, pool_alloc((void**)&B1, Nd * sizeof(C), st));
    CK(ctx, pool_alloc((void**)&W, Nd * sizeof(C), st));
    SpreadArgs<T> sa{};
    sa.pos = (const vec4<T>*)fx->pos;
    sa.c = (const C*)fx->c;
    sa.m = fx->m;
    sa.quats = nullptr;
    sa.rot0 = 0;
    sa.sign = T(1);
    sa.inv_h = (T)G.inv_h;
    sa.beta = (T)ctx->p.beta;
    sa.w = ctx->p.w;
    sa.s = G.s;
    sa.s_h = G.s_h;
    sa.out = b0;
    sa.out_rot_stride = 0;
    sa.n_full = G.n;
    CK(ctx, cudaMemsetAsync(b0, 0, sz0 * sizeof(C), st));
    if (ctx->opt_spread_direct || !bins_supported(ctx)) {
        CK(ctx, launch_spread<T>(sa, G.dim, 1, st));
    } else {
        BinArgs bn;
        CKI(bins_for(ctx, G.s, G.dim, fx->m, 1, DEFAULT_BIN, &bn));
        CK(ctx, launch_spread_bins<T>(sa, bn, G.dim, 1, st));
    }
    CK(ctx, pass_x_fwd<T>(G, tw, b0, 0, b1, 0, 1, st));
    if (G.dim == 3) {
        CK(ctx, pass_y_fwd<T>(G, tw, b1, 0, b2, 0, 1, st));
        CK(ctx, pass_last<T>(COL_FWD, G, tw, b2, 0, B1, 0, nullptr, 1, st));
    } else {
        CK(ctx, pass_last<T>(COL_FWD, G, tw, b1, 0, B1, 0, nullptr, 1, st));
    }
    CK(ctx, launch_wtable<T>(B1, D, G.N, G.dim, G.L, ctx->p.sigma_g, 1, -1, W, st));
    pool_free(b0, st);
    pool_free(b1, st);
    pool_free(b2, st);
    CK(ctx, cudaStreamSynchronize(st));
    Prep p;
    p.N = g->N;
    p.L = g->L;
    p.B1 = B1;
    p.W = W;
    fx->preps.push_back(p);
    *out = &fx->preps.back();
    return SD_OK;
}

// Phi and its gradient on the oversampled grid (type-2 tables)
template <typename T>
static int prep_fields(sd_ctx* ctx, sd_shape* fx, const sd_grid* g, Prep** out, cudaStream_t st) {
    Prep* p = nullptr;
    CKI(prep_fixed<T>(ctx, fx, g, &p, st));
    if (p->G) {
        *out = p;
        return SD_OK;
    }
    using C = cplx<T>;
    Geo G;
    CKI(make_geo(ctx, g, fx->radius, &G));
    Tw<T> tw;
    CKI(get_tw<T>(ctx, G, &tw, st));
    double* D = nullptr;
    CKI(get_deconv(ctx, G.N, G.n, &D, st));
    const int N = G.N, n = G.n;
    const int64_t Nd = (G.dim == 2) ? (int64_t)N * N : (int64_t)N * N * N;
    const int64_t nd = (G.dim == 2) ? (int64_t)n * n : (int64_t)n * n * n;
    const int64_t sx = (G.dim == 2) ? (int64_t)N * n : (int64_t)N * N * n;
    const int64_t sy = (G.dim == 2) ? 0 : (int64_t)N * n * n;
    C *F = nullptr, *X = nullptr, *Y = nullptr, *Z = nullptr, *Gf = nullptr;
    CK(ctx, pool_alloc((void**)&F, Nd * sizeof(C), st));
    CK(ctx, pool_alloc((void**)&X, sx * sizeof(C), st));
    if (sy) CK(ctx, pool_alloc((void**)&Y, sy * sizeof(C), st));
    CK(ctx, pool_alloc((void**)&Z, nd * sizeof(C), st));
    // type-2 tables on a grid of pitch n + w: the cells past n repeat the periodic field
    const int pn = n + ctx->p.w;
    const int64_t pd = (G.dim == 2) ? (int64_t)pn * pn : (int64_t)pn * pn * pn;
    CK(ctx, pool_alloc((void**)&Gf, 4 * pd * sizeof(C), st));
    CK(ctx, cudaMemsetAsync(Gf, 0, 4 * pd * sizeof(C), st));
    for (int f = 0; f <= G.dim; ++f) {
        CK(ctx, launch_wtable<T>((const C*)p->B1, D, N, G.dim, G.L, ctx->p.sigma_g, 0, f - 1, F, st));
        RowArgs<T> r{};
        r.in = F;
        r.out = X;
        r.nrows = (G.dim == 2) ? N : N * N;
        r.in_row_stride = N;
        r.out_row_stride = n;
        r.len_in = N;
        r.N = N;
        r.n = n;
        r.tw = tw.n;
        CK(ctx, launch_rows<T>(ROW_EXPAND, r, 1, nullptr, st));
        ColArgs<T> c{};
        c.N = N;
        c.n = n;
        c.twF = tw.n;
        c.twI = tw.n;
        c.len_in = N;
        if (G.dim == 3) {
            c.in = X;
            c.out = Y;
            c.ncols = n;
            c.nouter = N;
            c.in_outer_stride = (int64_t)N * n;
            c.out_outer_stride = (int64_t)n * n;
            CK(ctx, launch_cols<T>(COL_EXPAND, c, 1, st));
            c.in = Y;
            c.out = Z;
            c.ncols = n * n;
            c.nouter = 1;
            c.in_outer_stride = 0;
            c.out_outer_stride = 0;
            CK(ctx, launch_cols<T>(COL_EXPAND, c, 1, st));
        } else {
            c.in = X;
            c.out = Z;
            c.ncols = n;
            c.nouter = 1;
            CK(ctx, launch_cols<T>(COL_EXPAND, c, 1, st));
        }
        CK(ctx, launch_interleave<T>(Z, Gf, n, pn, G.dim, f, st));
    }
    pool_free(F, st);
    pool_free(X, st);
    pool_free(Y, st);
    pool_free(Z, st);
    CK(ctx, cudaStreamSynchronize(st));
    p->G = Gf;
    *out = p;
    return SD_OK;
}

// ---------------------------------------------------------------------------
// search pipeline
// ---------------------------------------------------------------------------

template <typename T>
static int64_t per_rot_elems(const Geo& G, int64_t* e0, int64_t* e1) {
    const int64_t N = G.N, s = G.s;
    if (G.dim == 2) {
        *e0 = std::max(s * s, N * N);
        *e1 = s * N;
    } else {
        *e0 = std::max(s * s * s, s * N * N);
        *e1 = std::max(s * s * N, N * N * N);
    }
    return *e0 + *e1;
}

template <typename T>
static int choose_batch(sd_ctx* ctx, const Geo& G, int64_t n_r) {
    int64_t e0, e1;
    const int64_t per = per_rot_elems<T>(G, &e0, &e1) * (int64_t)sizeof(cplx<T>);
    int64_t b = ctx->opt_batch > 0 ? ctx->opt_batch : std::max<int64_t>(1, ((int64_t)1 << 30) / per);
    if (ctx->opt_plain) b = 1;
    b = std::min<int64_t>(b, 64);
    b = std::min<int64_t>(b, std::max<int64_t>(n_r, 1));
    return (int)b;
}

// One scoring job (a fixed shape, a moving shape, a grid and a rotation list)
// with its launch plan and, once bound, its workspace pointers.
template <typename T>
struct Search {
    const sd_shape* moving = nullptr;
    const double* quats = nullptr;
    int64_t n_r = 0;
    Geo G{};
    Tw<T> tw{};
    const cplx<T>* W = nullptr;
    void* out = nullptr;
    int maps = 0;
    Plan plan{};
    bool prunable = false;          // pruned forward passes apply (sub-box in the low half of a line)
    bool alt_cols = false;          // and their narrow / wide column plans exist (FP32, n 128..384)
    const cplx<T>* Wsh = nullptr;   // the shifted table W' of the pruned passes
    bool iyx = false;               // inverse y + x in clusters (maps, or one candidate per rotation)
    int k_r = 1;          // candidates per rotation (argmax output)
    int64_t e0 = 0, e1 = 0, rows_last = 0, Nd = 0;
    cplx<T>* b0 = nullptr;
    cplx<T>* b1 = nullptr;
    double* ps = nullptr;
    int* pi = nullptr;
    BinArgs bn{};
    int nbz = 0;  // SPREAD_X: bins along z
};

// Spreading fused with the x transform: pruned 3D FP32 searches with w = 6.
template <typename T>
static bool spread_x_ok(const sd_ctx* ctx, const Search<T>& S) {
    return sizeof(T) == 4 && S.G.dim == 3 && ctx->p.w == 6 && S.plan.fft != SD_FFT_FULL;
}

// The forward-pass plans a job can run: FULL always, the pruned ones where the
// sub-box fits.
template <typename T>
static bool fft_plan_ok(const Search<T>& S, int fft) {
    return fft == SD_FFT_FULL || (fft == SD_FFT_PRUNED && S.prunable) ||
           ((fft == SD_FFT_PRUNED_NARROW || fft == SD_FFT_PRUNED_WIDE) && S.alt_cols);
}

// The plan a job starts from: the forced one if it applies, else pruned where
// possible.
template <typename T>
static int fft_plan_default(const sd_ctx* ctx, const Search<T>& S) {
    if (ctx->opt_fft_plan >= 0 && fft_plan_ok(S, ctx->opt_fft_plan)) return ctx->opt_fft_plan;
    return S.prunable ? SD_FFT_PRUNED : SD_FFT_FULL;
}

// Fixed-shape tables, geometry, twiddles and the default plan of a job (may
// synchronise the stream the first time a fixed shape meets a grid).
template <typename T>
static int search_setup(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const double* quats, int64_t n_r,
                        const sd_grid* g, void* out, int maps, cudaStream_t st, Search<T>* S) {
    Prep* prep = nullptr;
    CKI(prep_fixed<T>(ctx, const_cast<sd_shape*>(fixed), g, &prep, st));
    CKI(make_geo(ctx, g, moving->radius, &S->G));
    CKI(get_tw<T>(ctx, S->G, &S->tw, st));
    S->moving = moving;
    S->quats = quats;
    S->n_r = n_r;
    S->W = (const cplx<T>*)prep->W;
    S->out = out;
    S->maps = maps;
    S->plan.B = choose_batch<T>(ctx, S->G, n_r);
    S->plan.bins = (!ctx->opt_spread_direct && bins_supported(ctx)) ? ctx->opt_bin_side : 0;
    per_rot_elems<T>(S->G, &S->e0, &S->e1);
    S->rows_last = (S->G.dim == 2) ? S->G.N : (int64_t)S->G.N * S->G.N;
    S->Nd = (S->G.dim == 2) ? (int64_t)S->G.N * S->G.N : (int64_t)S->G.N * S->G.N * S->G.N;
    // pruned forward passes: the sub-box must fit in the low half of a line
    S->prunable = ctx->opt_pruned && pruned_len_ok(S->G.n) && S->G.s <= S->G.N;
    S->alt_cols = S->prunable && sizeof(T) == 4 && S->G.n >= 128 && S->G.n <= 384;
    if (S->prunable) {
        void* ws = nullptr;
        for (auto& w : prep->Wsh)
            if (w.first == S->G.s_h) ws = w.second;
        if (!ws) {
            CK(ctx, pool_alloc(&ws, (size_t)S->Nd * sizeof(cplx<T>), st));
            CK(ctx, launch_wshift<T>((const cplx<T>*)prep->W, S->G.N, S->G.dim, S->G.n, S->G.s_h, (cplx<T>*)ws, st));
            prep->Wsh.emplace_back(S->G.s_h, ws);
        }
        S->Wsh = (const cplx<T>*)ws;
    }
    S->plan.fft = fft_plan_default(ctx, *S);
    S->iyx = ctx->opt_inv_cluster && sizeof(T) == 4 && S->G.dim == 3 && inv_yx_supported(S->G.N);
    if (ctx->opt_spread_box && bins_supported(ctx)) S->plan.bins = SPREAD_BOX;
    if (ctx->opt_spread_fused && spread_x_ok(ctx, *S)) S->plan.bins = SPREAD_X;
    return SD_OK;
}

// Workspace bytes per slot of a job under its plan (maximum into need[]).
template <typename T>
static void search_need(const Search<T>& S, size_t need[8]) {
    const size_t B = (size_t)S.plan.B;
    need[0] = std::max(need[0], B * S.e0 * sizeof(cplx<T>));
    need[1] = std::max(need[1], B * S.e1 * sizeof(cplx<T>));
    // argmax partials: one per block of rows, or up to 16 per block (k_r > 1):
    // blocks hold at least 8 rows, so twice the rows rounded up to 16 bounds both
    const size_t parts = 2 * (((size_t)S.rows_last + 15) / 16) * 16;
    need[2] = std::max(need[2], B * parts * sizeof(double));
    need[3] = std::max(need[3], B * parts * sizeof(int));
    if (S.plan.bins == SPREAD_X) need[6] = std::max(need[6], bins_bytes_x(S.G.s, S.moving->m, S.plan.B));
    else if (S.plan.bins > SPREAD_BOX)
        need[6] = std::max(need[6], bins_bytes(S.G.s, S.G.dim, S.moving->m, S.plan.B, S.plan.bins));
}

static int ws_reserve(sd_ctx* ctx, const size_t need[8]) {
    void* p;
    for (int k = 0; k < 8; ++k)
        if (need[k]) CKI(ws_get(ctx, k, need[k], &p));
    return SD_OK;
}

// Points a job at the (reserved) workspace.
template <typename T>
static void search_bind(sd_ctx* ctx, Search<T>* S) {
    S->b0 = (cplx<T>*)ctx->ws[0].p;
    S->b1 = (cplx<T>*)ctx->ws[1].p;
    S->ps = (double*)ctx->ws[2].p;
    S->pi = (int*)ctx->ws[3].p;
    if (S->plan.bins == SPREAD_X) bins_layout_x(ctx->ws[6].p, S->G.s, S->moving->m, S->plan.B, &S->bn, &S->nbz);
    else if (S->plan.bins > SPREAD_BOX)
        bins_layout(ctx->ws[6].p, S->G.s, S->G.dim, S->moving->m, S->plan.B, S->plan.bins, &S->bn);
}

// Launch sequence of rotations [r_lo, r_hi), plan.B rotations at a time.
// mode 0 writes per-rotation argmax candidates, mode 1 whole maps.
template <typename T>
static int search_enqueue(sd_ctx* ctx, const Search<T>& S, int64_t r_lo, int64_t r_hi, cudaStream_t s, bool timed) {
    using C = cplx<T>;
    const Geo& G = S.G;
    const int B = S.plan.B;
    const bool fused_x = S.plan.bins == SPREAD_X;
    // the cluster inverse ends with one candidate per rotation (or the map)
    const bool iyx = S.iyx && (S.maps || S.k_r <= 1);
    for (int64_t r0 = r_lo; r0 < r_hi; r0 += B) {
        const int b = (int)std::min<int64_t>(B, r_hi - r0);
        if (!fused_x) {
            PassTimer pt(ctx, SD_PASS_CLEAR, s, timed);
            CK(ctx, cudaMemsetAsync(S.b0, 0, (size_t)b * S.e0 * sizeof(C), s));
        }
        SpreadArgs<T> sa{};
        sa.pos = (const vec4<T>*)S.moving->pos;
        sa.c = (const C*)S.moving->c;
        sa.m = S.moving->m;
        sa.quats = S.quats;
        sa.rot0 = r0;
        sa.sign = T(-1);
        sa.inv_h = (T)G.inv_h;
        sa.beta = (T)ctx->p.beta;
        sa.w = ctx->p.w;
        sa.s = G.s;
        sa.s_h = G.s_h;
        sa.out = S.b0;
        sa.out_rot_stride = S.e0;
        sa.n_full = G.n;
        const bool pruned = S.plan.fft != SD_FFT_FULL;
        const int lines = S.plan.fft == SD_FFT_PRUNED_NARROW ? LINES_NARROW
                          : (S.plan.fft == SD_FFT_PRUNED_WIDE ? LINES_WIDE : LINES_STD);
        const int mx = pruned ? ROW_FWD_P : ROW_FWD;
        const int my = pruned ? COL_FWD_P : COL_FWD;
        const int mf = pruned ? COL_FUSED_P : COL_FUSED;
        const C* Wp = pruned ? S.Wsh : S.W;
        if (fused_x) {
            // spreading and the forward x transform in one pass: no sub-box
            PassTimer pt(ctx, SD_PASS_SPREAD_X, s, timed);
            CK(ctx, launch_spread_x<T>(sa, S.bn, S.nbz, S.b1, S.e1, S.tw.n, b, s));
        } else {
            {
                PassTimer pt(ctx, SD_PASS_SPREAD, s, timed);
                if (S.plan.bins == SPREAD_BOX) CK(ctx, launch_spread_box<T>(sa, G.dim, b, s));
                else if (S.plan.bins) CK(ctx, launch_spread_bins<T>(sa, S.bn, G.dim, b, s));
                else CK(ctx, launch_spread<T>(sa, G.dim, b, s));
            }
            PassTimer pt(ctx, SD_PASS_FWD_X, s, timed);
            CK(ctx, pass_x_fwd<T>(G, S.tw, S.b0, S.e0, S.b1, S.e1, b, s, mx));
        }
        C* fin;
        int64_t fin_rs;
        if (G.dim == 3) {
            {
                PassTimer pt(ctx, SD_PASS_FWD_Y, s, timed);
                CK(ctx, pass_y_fwd<T>(G, S.tw, S.b1, S.e1, S.b0, S.e0, b, s, my, lines));
            }
            {
                PassTimer pt(ctx, SD_PASS_FUSED, s, timed);
                CK(ctx, pass_last<T>(mf, G, S.tw, S.b0, S.e0, S.b1, S.e1, Wp, b, s, lines));
            }
            if (!iyx) {
                PassTimer pt(ctx, SD_PASS_INV_Y, s, timed);
                CK(ctx, pass_y_inv<T>(G, S.tw, S.b1, S.e1, b, s));
            }
            fin = S.b1;
            fin_rs = S.e1;
        } else {
            PassTimer pt(ctx, SD_PASS_FUSED, s, timed);
            CK(ctx, pass_last<T>(mf, G, S.tw, S.b1, S.e1, S.b0, S.e0, Wp, b, s, lines));
            fin = S.b0;
            fin_rs = S.e0;
        }
        RowArgs<T> r{};
        r.in = fin;
        r.in_rot_stride = fin_rs;
        r.nrows = (int)S.rows_last;
        r.in_row_stride = G.N;
        r.out_row_stride = G.N;
        r.len_in = G.N;
        r.N = G.N;
        r.n = G.n;
        r.tw = S.tw.N;
        if (S.maps) {
            r.out = (C*)S.out + r0 * S.Nd;
            r.out_rot_stride = S.Nd;
            PassTimer pt(ctx, iyx ? SD_PASS_INV_YX : SD_PASS_INV_X, s, timed);
            if (iyx) CK(ctx, launch_inv_yx<T>(ROW_INV_MAP, r, b, nullptr, s));
            else CK(ctx, launch_rows<T>(ROW_INV_MAP, r, b, nullptr, s));
        } else {
            int nparts = 0;
            r.part_score = S.ps;
            r.part_idx = S.pi;
            // k_r > 1: each block keeps its K >= k_r best (K a power of two, <= 16)
            const int K = S.k_r <= 1 ? 1 : (S.k_r <= 2 ? 2 : (S.k_r <= 4 ? 4 : (S.k_r <= 8 ? 8 : 16)));
            const int mode = K == 1 ? ROW_INV_ARGMAX
                                    : (K == 2 ? ROW_INV_TOPK2 : (K == 4 ? ROW_INV_TOPK4 : (K == 8 ? ROW_INV_TOPK8 : ROW_INV_TOPK16)));
            {
                PassTimer pt(ctx, iyx ? SD_PASS_INV_YX : SD_PASS_INV_X, s, timed);
                if (iyx) CK(ctx, launch_inv_yx<T>(mode, r, b, &nparts, s));
                else CK(ctx, launch_rows<T>(mode, r, b, &nparts, s));
            }
            PassTimer pt(ctx, SD_PASS_REDUCE, s, timed);
            if (K == 1) CK(ctx, launch_reduce_argmax(S.ps, S.pi, nparts, b, r0, S.out, s));
            else CK(ctx, launch_reduce_topk(S.ps, S.pi, nparts, K, S.k_r, b, r0, S.out, s));
        }
    }
    return SD_OK;
}

// ---------------------------------------------------------------------------
// autotuner: per job geometry, the plan (rotations per launch, spreading
// variant, forward-pass FFT plan) with the lowest measured time per rotation
// ---------------------------------------------------------------------------

template <typename T>
static std::string plan_key(sd_ctx* ctx, const Search<T>& S) {
    // jobs of one grid whose sub-boxes and sample counts are close share a plan
    int lg = 0;
    for (int64_t m = S.moving->m; m > 1; m >>= 1) ++lg;
    char key[128];
    snprintf(key, sizeof key, "%d|%d|%d|%d|%d|%d", ctx->p.precision, S.G.dim, S.G.N, S.G.n, S.G.s / 16, lg);
    return key;
}

// Times each candidate plan on the job's own first rotations (CUDA events on
// the stream, after one untimed run) and keeps the fastest per rotation.  The
// job's outputs for those rotations are overwritten when it runs.
template <typename T>
static int autotune(sd_ctx* ctx, Search<T>* S, cudaStream_t st) {
    const std::string key = plan_key(ctx, *S);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        S->plan.B = (int)std::min<int64_t>(it->second.B, std::max<int64_t>(S->n_r, 1));
        S->plan.bins = it->second.bins;
        if (ctx->opt_fft_plan < 0 && fft_plan_ok(*S, it->second.fft)) S->plan.fft = it->second.fft;
        return SD_OK;
    }
    // first stage: batch x spreading under the job's default FFT plan; second
    // stage: the other FFT plans under the best of the first
    const int b0 = S->plan.B, f0 = S->plan.fft;
    std::vector<Plan> cand;
    for (int B : {b0 / 4, b0 / 2, b0, 2 * b0}) {
        if (B < 1 || B > 64 || (B > S->n_r && B != b0)) continue;
        for (int bins : {0, SPREAD_BOX, SPREAD_X, 8, 12, 16}) {
            if (bins == SPREAD_X ? !spread_x_ok(ctx, *S) : (bins && !bins_supported(ctx))) continue;
            bool dup = false;
            for (auto& c : cand) dup |= (c.B == B && c.bins == bins);
            if (!dup) cand.push_back(Plan{B, bins, f0});
        }
    }
    int most = 1;
    for (auto& c : cand) most = std::max(most, c.B);
    const int64_t n_trial = std::min<int64_t>(S->n_r, 2 * (int64_t)most);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(ctx, cudaEventCreate(&e0));
    CK(ctx, cudaEventCreate(&e1));
    Plan best = S->plan;
    double best_ms = INFINITY;
    int rc = SD_OK;
    auto trial = [&](const Plan& c) -> int {
        Search<T> t = *S;
        t.plan = c;
        size_t need[8] = {};
        search_need(t, need);
        CKI(ws_reserve(ctx, need));
        search_bind(ctx, &t);
        CKI(search_enqueue(ctx, t, 0, std::min<int64_t>(n_trial, c.B), st, false));
        cudaEventRecord(e0, st);
        CKI(search_enqueue(ctx, t, 0, n_trial, st, false));
        cudaEventRecord(e1, st);
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return fail(ctx, SD_ERR_CUDA, "autotune timing failed: %s", cudaGetErrorString(e));
        const double per = ms / (double)n_trial;
        if (per < best_ms) {
            best_ms = per;
            best = c;
        }
        return SD_OK;
    };
    for (auto& c : cand)
        if ((rc = trial(c)) != SD_OK) break;
    if (rc == SD_OK && ctx->opt_fft_plan < 0) {
        const Plan first = best;
        for (int f : {SD_FFT_PRUNED, SD_FFT_PRUNED_NARROW, SD_FFT_PRUNED_WIDE, SD_FFT_FULL}) {
            Plan c = first;
            c.fft = f;
            // spreading fused with the x pass exists only under the pruned plans
            if (f == first.fft || !fft_plan_ok(*S, f) || (f == SD_FFT_FULL && c.bins == SPREAD_X)) continue;
            if ((rc = trial(c)) != SD_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SD_OK) return rc;
    ctx->tuned[key] = best;
    S->plan = best;
    return SD_OK;
}

// Runs one job: workspace, then the launch sequence (eager, or replayed from a
// captured graph when the "graph" option is on).
template <typename T>
static int run_search(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const double* quats, int64_t n_r,
                      const sd_grid* g, void* out, int maps, cudaStream_t st, int k_r = 1) {
    Search<T> S;
    CKI(search_setup<T>(ctx, fixed, moving, quats, n_r, g, out, maps, st, &S));
    S.k_r = k_r;
    if (ctx->opt_autotune && !ctx->opt_plain && ctx->opt_batch <= 0) CKI(autotune<T>(ctx, &S, st));
    size_t need[8] = {};
    search_need(S, need);
    CKI(ws_reserve(ctx, need));
    search_bind(ctx, &S);

    if (ctx->opt_graph && !ctx->opt_plain && st != nullptr) {
        char key[256];
        snprintf(key, sizeof key, "%p|%p|%p|%lld|%d|%.17g|%p|%d|%p|%d|%d|%d|%d|%d", (const void*)fixed,
                 (const void*)moving, (const void*)quats, (long long)n_r, g->N, g->L, out, maps, (void*)st, S.plan.B,
                 S.plan.bins, S.plan.fft, ctx->opt_timing, S.k_r * 2 + (int)S.iyx);
        std::string k(key);
        auto it = ctx->graphs.find(k);
        if (it == ctx->graphs.end()) {
            if (ctx->seen[k]++ == 0) return search_enqueue(ctx, S, 0, n_r, st, true);  // first call runs eagerly
            cudaGraph_t graph;
            const long long l0 = g_launches.load();
            std::vector<TimerRec> timers;  // with "timing" on: pass events as graph nodes
            CK(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            ctx->capture_timers = ctx->opt_timing ? &timers : nullptr;
            int rc = search_enqueue(ctx, S, 0, n_r, st, ctx->opt_timing != 0);
            ctx->capture_timers = nullptr;
            cudaError_t ec = cudaStreamEndCapture(st, &graph);
            GraphEntry ge;
            ge.timers = timers;
            if (rc != SD_OK || ec != cudaSuccess) {
                ge.exec = nullptr;
                for (auto& t : ge.timers) {
                    cudaEventDestroy(t.a);
                    cudaEventDestroy(t.b);
                }
                if (ec == cudaSuccess) cudaGraphDestroy(graph);
                if (rc != SD_OK) return rc;
                CK(ctx, ec);
            }
            ge.kernels = g_launches.load() - l0;
            g_launches.fetch_sub(ge.kernels);  // counted when the graph runs
            ec = cudaGraphInstantiate(&ge.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ec != cudaSuccess)
                for (auto& t : ge.timers) {
                    cudaEventDestroy(t.a);
                    cudaEventDestroy(t.b);
                }
            CK(ctx, ec);
            it = keep_graph(ctx, k, ge);
        }
        // the graph's pass events still hold its previous replay: read them first
        if (!it->second.timers.empty()) harvest_timers(ctx);
        {
            PassTimer pt(ctx, SD_PASS_GRAPH, st, true);
            CK(ctx, cudaGraphLaunch(it->second.exec, st));
        }
        for (auto& t : it->second.timers) ctx->pending.push_back(t);
        note_launch((int)it->second.kernels);
        return SD_OK;
    }
    return search_enqueue(ctx, S, 0, n_r, st, true);
}

// Many jobs in one launch sequence.  Each job gets its own plan (tuned when the
// "autotune" option is on); the workspace is reserved once for the largest.
// The first call with a given job list runs eagerly, later calls replay one
// captured CUDA graph that holds every job, with an event node between jobs
// for the per-job device times.
template <typename T>
static int run_pairs(sd_ctx* ctx, const sd_pair_job* jobs, int64_t n_jobs, sd_pair_stat* stats, cudaStream_t st) {
    std::vector<Search<T>> S((size_t)n_jobs);
    std::string k = "pairs";
    for (int64_t j = 0; j < n_jobs; ++j) {
        const sd_pair_job& J = jobs[j];
        CKI(search_setup<T>(ctx, J.fixed, J.moving, J.quats, J.n_r, &J.grid, J.cand_out, 0, st, &S[j]));
        if (ctx->opt_autotune && !ctx->opt_plain && ctx->opt_batch <= 0) CKI(autotune<T>(ctx, &S[j], st));
        char part[256];
        snprintf(part, sizeof part, "|%p,%p,%p,%lld,%d,%.17g,%p,%d,%d,%d", (const void*)J.fixed,
                 (const void*)J.moving, (const void*)J.quats, (long long)J.n_r, J.grid.N, J.grid.L,
                 (void*)J.cand_out, S[j].plan.B, S[j].plan.bins, S[j].plan.fft * 2 + (int)S[j].iyx);
        k += part;
    }
    char tail[64];
    snprintf(tail, sizeof tail, "|%p", (void*)st);
    k += tail;
    size_t need[8] = {};
    for (auto& x : S) search_need(x, need);
    CKI(ws_reserve(ctx, need));
    for (auto& x : S) search_bind(ctx, &x);

    // events around every job: eager records, or event nodes of the graph
    auto it = ctx->graphs.find(k);
    const bool replay = it != ctx->graphs.end();
    const bool capture = !replay && st != nullptr && ctx->seen[k]++ > 0;
    std::vector<cudaEvent_t> evs;
    if (replay) {
        evs = it->second.events;
    } else {
        evs.resize((size_t)n_jobs + 1, nullptr);
        for (auto& e : evs) CK(ctx, cudaEventCreate(&e));
    }
    int rc = SD_OK;
    if (!replay) {
        cudaGraph_t graph = nullptr;
        const long long l0 = g_launches.load();
        if (capture) CK(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int64_t j = 0; j < n_jobs && rc == SD_OK; ++j) {
            cudaError_t e = capture ? cudaEventRecordWithFlags(evs[j], st, cudaEventRecordExternal)
                                    : cudaEventRecord(evs[j], st);
            if (e != cudaSuccess) rc = fail(ctx, SD_ERR_CUDA, "event record failed: %s", cudaGetErrorString(e));
            if (rc == SD_OK) rc = search_enqueue(ctx, S[j], 0, S[j].n_r, st, !capture);
        }
        if (rc == SD_OK) {
            cudaError_t e = capture ? cudaEventRecordWithFlags(evs[n_jobs], st, cudaEventRecordExternal)
                                    : cudaEventRecord(evs[n_jobs], st);
            if (e != cudaSuccess) rc = fail(ctx, SD_ERR_CUDA, "event record failed: %s", cudaGetErrorString(e));
        }
        if (capture) {
            cudaError_t ec = cudaStreamEndCapture(st, &graph);
            if (rc == SD_OK && ec != cudaSuccess)
                rc = fail(ctx, SD_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ec));
            GraphEntry ge;
            if (rc == SD_OK) {
                ec = cudaGraphInstantiate(&ge.exec, graph, 0);
                if (ec != cudaSuccess) rc = fail(ctx, SD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ec));
            }
            if (graph) cudaGraphDestroy(graph);
            ge.kernels = g_launches.load() - l0;
            g_launches.fetch_sub(ge.kernels);  // counted when the graph runs
            if (rc == SD_OK) {
                ge.events = evs;
                it = keep_graph(ctx, k, ge);
            }
        }
        if (rc != SD_OK) {
            for (auto e : evs) cudaEventDestroy(e);
            return rc;
        }
    }
    if (replay || capture) {
        {
            PassTimer pt(ctx, SD_PASS_GRAPH, st, true);
            CK(ctx, cudaGraphLaunch(it->second.exec, st));
        }
        note_launch((int)it->second.kernels);
    }
    if (stats) {
        CK(ctx, cudaEventSynchronize(evs[n_jobs]));
        for (int64_t j = 0; j < n_jobs; ++j) {
            float ms = NAN;
            if (cudaEventElapsedTime(&ms, evs[j], evs[j + 1]) != cudaSuccess) {
                cudaGetLastError();
                ms = NAN;
            }
            stats[j].ms = ms;
            stats[j].batch = S[j].plan.B;
            stats[j].spread_bins = S[j].plan.bins;
            stats[j].fft_plan = S[j].plan.fft;
            stats[j].n = S[j].G.n;
            stats[j].s = S[j].G.s;
        }
    }
    if (!replay && !capture)  // eager events are not kept (released once they complete)
        for (auto e : evs) cudaEventDestroy(e);
    return SD_OK;
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------

// Entry points (C linkage from the declarations in sdfdock.h).

int sd_default_params(sd_params* p, int dim, int precision) {
    if (!p) return SD_ERR_ARG;
    memset(p, 0, sizeof *p);
    p->dim = dim;
    p->precision = precision;
    p->lambda1 = 1.0;
    p->lambda2 = 3.0;
    p->sigma_t = 0.5;
    p->eps = 1.5;
    p->sigma_g = 0.03;
    p->w = 6;
    p->alpha = 2;
    p->beta = 0.0;
    p->phi = SD_PHI_SDF;
    p->phi_radius = 1.0;
    return SD_OK;
}

int sd_create(sd_ctx** out, int device, const sd_params* p) {
    if (!out || !p) return fail(nullptr, SD_ERR_ARG, "sd_create: NULL argument");
    *out = nullptr;
    if (p->dim != 2 && p->dim != 3) return fail(nullptr, SD_ERR_ARG, "dim must be 2 or 3");
    if (p->precision != SD_F32 && p->precision != SD_F64) return fail(nullptr, SD_ERR_ARG, "bad precision");
    if (p->alpha != 2) return fail(nullptr, SD_ERR_UNIMPLEMENTED, "only oversampling alpha = 2 is supported");
    const int ws[] = {4, 5, 6, 7, 8, 10, 12, 16};
    bool wok = false;
    for (int w : ws) wok |= (p->w == w);
    if (!wok) return fail(nullptr, SD_ERR_ARG, "spreading width w=%d not supported (4-8, 10, 12, 16)", p->w);
    if (!(p->sigma_t > 0) || !(p->sigma_g > 0) || !(p->lambda1 >= 0) || !(p->lambda2 >= 0) || isnan(p->eps))
        return fail(nullptr, SD_ERR_ARG, "sigma_t, sigma_g must be > 0; lambdas >= 0; eps not NaN");
    if (p->phi < SD_PHI_SDF || p->phi > SD_PHI_SKIN) return fail(nullptr, SD_ERR_ARG, "unknown phi-kernel %d", p->phi);
    if (!(p->phi_radius > 0) || !isfinite(p->phi_radius))
        return fail(nullptr, SD_ERR_ARG, "phi_radius must be positive and finite");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, SD_ERR_CUDA, "CUDA device %d not available", device);
    }
    {
        // keep freed pool memory for reuse by later calls on this device
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(device);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
        if (prev >= 0 && prev != device) cudaSetDevice(prev);
    }
    sd_ctx* c = new sd_ctx();
    c->device = device;
    c->p = *p;
    if (!(c->p.beta > 0)) c->p.beta = 2.30 * c->p.w;
    *out = c;
    return SD_OK;
}

int sd_destroy(sd_ctx* ctx) {
    if (!ctx) return SD_OK;
    DeviceGuard dg(ctx->device);
    for (auto& b : ctx->ws)
        if (b.p) cudaFree(b.p);
    for (auto& kv : ctx->twiddles) cudaFree(kv.second);
    for (auto& kv : ctx->deconv) cudaFree(kv.second);
    drop_graphs(ctx);
    harvest_timers(ctx);
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->gl_x) cudaFree(ctx->gl_x);
    if (ctx->gl_w) cudaFree(ctx->gl_w);
    delete ctx;
    return SD_OK;
}

const char* sd_last_error(const sd_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int sd_set_option(sd_ctx* ctx, const char* key, int64_t value) {
    if (!ctx || !key) return SD_ERR_ARG;
    if (!strcmp(key, "batch")) ctx->opt_batch = value;
    else if (!strcmp(key, "graph")) ctx->opt_graph = (int)value;
    else if (!strcmp(key, "plain")) ctx->opt_plain = (int)value;
    else if (!strcmp(key, "timing")) ctx->opt_timing = (int)value;
    else if (!strcmp(key, "spread_direct")) ctx->opt_spread_direct = (int)value;
    else if (!strcmp(key, "pruned")) ctx->opt_pruned = (int)value;
    else if (!strcmp(key, "inverse_cluster")) ctx->opt_inv_cluster = (int)value;
    else if (!strcmp(key, "spread_bin_side")) {
        if (value != 8 && value != 12 && value != 16) return fail(ctx, SD_ERR_ARG, "spread_bin_side: 8, 12 or 16");
        ctx->opt_bin_side = (int)value;
    } else if (!strcmp(key, "fft_plan")) {
        if (value < -1 || value > SD_FFT_PRUNED_WIDE) return fail(ctx, SD_ERR_ARG, "fft_plan: -1 to 3");
        ctx->opt_fft_plan = (int)value;
    }
    else if (!strcmp(key, "spread_fused")) ctx->opt_spread_fused = (int)value;
    else if (!strcmp(key, "spread_box")) ctx->opt_spread_box = (int)value;
    else if (!strcmp(key, "sdf_cull")) ctx->opt_sdf_cull = (int)value;
    else if (!strcmp(key, "autotune")) ctx->opt_autotune = (int)value;
    else return fail(ctx, SD_ERR_ARG, "unknown option '%s'", key);
    return SD_OK;
}

template <typename T>
static int sdf_build_t(sd_ctx* ctx, const void* bnd, const void* nrm, const void* area, int64_t n_b, const void* qry,
                       const void* vol, int64_t m, const int8_t* pmc_override, sd_shape** out, void* rho_out,
                       cudaStream_t st) {
    sd_shape* s = new sd_shape();
    s->ctx = ctx;
    s->m = m;
    std::unique_ptr<sd_shape> guard(s);
    // temporaries: nearest distances, memberships, radii, Morton orders, the
    // sorted boundary and its tile boxes
    T* xi = nullptr;
    int8_t* pm = nullptr;
    double* rad = nullptr;
    int32_t *perm_q = nullptr, *perm_b = nullptr;
    vec4<T>*bnd_s = nullptr, *nrm_s = nullptr;
    float* tbox = nullptr;
    const int64_t n_tiles = (n_b + SDF_TILE - 1) / SDF_TILE;
    auto cleanup = [&]() {
        pool_free(xi, st); pool_free(pm, st); pool_free(rad, st); pool_free(perm_q, st); pool_free(perm_b, st);
        pool_free(bnd_s, st); pool_free(nrm_s, st); pool_free(tbox, st);
    };
    auto fail_free = [&](int code, const char* what, cudaError_t e) {
        cleanup();
        pool_free(s->pos, st);
        pool_free(s->c, st);
        s->pos = s->c = nullptr;
        return fail(ctx, code, "sdf_build: %s: %s", what, cudaGetErrorString(e));
    };
    const size_t mm = (size_t)std::max<int64_t>(m, 1);
    cudaError_t e = cudaSuccess;
    if ((e = pool_alloc(&s->pos, mm * sizeof(vec4<T>), st)) != cudaSuccess ||
        (e = pool_alloc(&s->c, mm * sizeof(cplx<T>), st)) != cudaSuccess ||
        (e = pool_alloc((void**)&xi, mm * sizeof(T), st)) != cudaSuccess ||
        (e = pool_alloc((void**)&pm, mm, st)) != cudaSuccess ||
        (e = pool_alloc((void**)&rad, 2 * sizeof(double), st)) != cudaSuccess ||
        (e = pool_alloc((void**)&perm_q, mm * sizeof(int32_t), st)) != cudaSuccess ||
        (e = pool_alloc((void**)&perm_b, (size_t)n_b * sizeof(int32_t), st)) != cudaSuccess ||
        (e = pool_alloc((void**)&bnd_s, (size_t)n_b * sizeof(vec4<T>), st)) != cudaSuccess ||
        (e = pool_alloc((void**)&nrm_s, (size_t)n_b * sizeof(vec4<T>), st)) != cudaSuccess ||
        (e = pool_alloc((void**)&tbox, (size_t)n_tiles * (1 + SDF_TILE / 32) * 6 * sizeof(float), st)) != cudaSuccess)
        return fail_free(SD_ERR_OOM, "allocation failed", e);
    // bounding radii of the queries and of the boundary samples
    double r2[2] = {0.0, 0.0};
    e = launch_radius<T>((const vec4<T>*)qry, m, ctx->p.dim, rad, st);
    if (e == cudaSuccess) e = launch_radius<T>((const vec4<T>*)bnd, n_b, ctx->p.dim, rad + 1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r2, rad, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_free(SD_ERR_CUDA, "radius", e);
    if (!isfinite(r2[0]) || !isfinite(r2[1])) {
        cleanup();
        pool_free(s->pos, st);
        pool_free(s->c, st);
        s->pos = s->c = nullptr;
        return fail(ctx, SD_ERR_NONFINITE, "sdf_build: non-finite query or boundary point");
    }
    // Morton orders: queries are processed (and the shape stored) in that order
    e = morton_order<T>((const vec4<T>*)qry, m, sqrt(r2[0]), ctx->p.dim, perm_q, st);
    if (e == cudaSuccess) e = morton_order<T>((const vec4<T>*)bnd, n_b, sqrt(r2[1]), ctx->p.dim, perm_b, st);
    if (e == cudaSuccess)
        e = launch_boundary_order<T>((const vec4<T>*)bnd, (const vec4<T>*)nrm, (const T*)area, perm_b, n_b,
                                     ctx->p.dim, bnd_s, nrm_s, tbox, st);
    if (e != cudaSuccess) return fail_free(SD_ERR_CUDA, "ordering", e);
    SdfArgs<T> a{};
    a.bnd = bnd_s;
    a.nrm = nrm_s;
    a.area = nullptr;
    a.n_b = n_b;
    a.qry = (const vec4<T>*)qry;
    a.vol = (const T*)vol;
    a.m = m;
    a.pmc_override = pmc_override;
    a.lam1 = (T)ctx->p.lambda1;
    a.lam2 = (T)ctx->p.lambda2;
    a.sigma = (T)ctx->p.sigma_t;
    a.eps = isinf(ctx->p.eps) ? T(-1) : (T)ctx->p.eps;
    a.phi = ctx->p.phi;
    a.radius = (T)ctx->p.phi_radius;
    a.xi_abs = xi;
    a.pmc = pm;
    a.c_out = (cplx<T>*)s->c;
    a.rho_out = (cplx<T>*)rho_out;
    a.pos_out = (vec4<T>*)s->pos;
    a.perm_q = perm_q;
    a.tile_box = ctx->opt_sdf_cull ? tbox : nullptr;
    a.sub_box = ctx->opt_sdf_cull >= 2 ? tbox + n_tiles * 6 : nullptr;
    a.n_tiles = n_tiles;
    e = launch_sdf<T>(a, ctx->p.dim, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_free(SD_ERR_CUDA, "kernels", e);
    cleanup();
    CK(ctx, cudaStreamSynchronize(st));
    s->radius = sqrt(r2[0]);
    *out = guard.release();
    return SD_OK;
}

int sd_sdf_build(sd_ctx* ctx, const void* bnd, const void* nrm, const void* area, int64_t n_b, const void* qry,
                 const void* vol, int64_t m, const int8_t* pmc_override, sd_shape** out, void* rho_out,
                 void* stream) {
    if (!ctx) return SD_ERR_ARG;
    if (!out) return fail(ctx, SD_ERR_ARG, "sdf_build: out is NULL");
    *out = nullptr;
    if (n_b <= 0 || m < 0) return fail(ctx, SD_ERR_ARG, "sdf_build: need n_b > 0 and m >= 0");
    if (!bnd || !nrm || !area || (m > 0 && (!qry || !vol)))
        return fail(ctx, SD_ERR_ARG, "sdf_build: NULL input pointer");
    if (m > (int64_t)INT32_MAX || n_b > (int64_t)INT32_MAX) return fail(ctx, SD_ERR_ARG, "sdf_build: size too large");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->p.precision == SD_F64)
        return sdf_build_t<double>(ctx, bnd, nrm, area, n_b, qry, vol, m, pmc_override, out, rho_out, st);
    return sdf_build_t<float>(ctx, bnd, nrm, area, n_b, qry, vol, m, pmc_override, out, rho_out, st);
}

int sd_shape_from_samples(sd_ctx* ctx, const void* pos, const void* c, int64_t m, sd_shape** out, void* stream) {
    if (!ctx) return SD_ERR_ARG;
    if (!out || (m > 0 && (!pos || !c)) || m < 0) return fail(ctx, SD_ERR_ARG, "shape_from_samples: bad arguments");
    *out = nullptr;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rs = real_size(ctx);
    sd_shape* s = new sd_shape();
    s->ctx = ctx;
    s->m = m;
    std::unique_ptr<sd_shape> guard(s);
    double* rad = nullptr;
    cudaError_t e;
    if ((e = pool_alloc(&s->pos, std::max<int64_t>(m, 1) * 4 * rs, st)) != cudaSuccess ||
        (e = pool_alloc(&s->c, std::max<int64_t>(m, 1) * 2 * rs, st)) != cudaSuccess ||
        (e = pool_alloc((void**)&rad, sizeof(double), st)) != cudaSuccess) {
        pool_free(s->pos, st);
        pool_free(s->c, st);
        pool_free(rad, st);
        s->pos = s->c = nullptr;
        return fail(ctx, SD_ERR_OOM, "shape_from_samples: %s", cudaGetErrorString(e));
    }
    double r2 = 0.0;
    e = cudaMemcpyAsync(s->pos, pos, m * 4 * rs, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->c, c, m * 2 * rs, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = (ctx->p.precision == SD_F64) ? launch_radius<double>((const double4_32a*)s->pos, m, ctx->p.dim, rad, st)
                                         : launch_radius<float>((const float4*)s->pos, m, ctx->p.dim, rad, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&r2, rad, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    pool_free(rad, st);
    if (e != cudaSuccess) {
        pool_free(s->pos, st);
        pool_free(s->c, st);
        s->pos = s->c = nullptr;
        return fail(ctx, SD_ERR_CUDA, "shape_from_samples: %s", cudaGetErrorString(e));
    }
    if (!isfinite(r2)) return fail(ctx, SD_ERR_NONFINITE, "shape_from_samples: non-finite position");
    s->radius = sqrt(r2);
    e = (ctx->p.precision == SD_F64)
            ? sort_by_morton<double>((double4_32a*)s->pos, (double2*)s->c, m, s->radius, ctx->p.dim, st)
            : sort_by_morton<float>((float4*)s->pos, (float2*)s->c, m, s->radius, ctx->p.dim, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(ctx, SD_ERR_CUDA, "shape_from_samples: ordering failed: %s", cudaGetErrorString(e));
    *out = guard.release();
    return SD_OK;
}

int sd_shape_info(const sd_shape* s, int64_t* m, double* radius) {
    if (!s) return SD_ERR_ARG;
    if (m) *m = s->m;
    if (radius) *radius = s->radius;
    return SD_OK;
}

int sd_shape_free(sd_shape* s) {
    if (!s) return SD_OK;
    DeviceGuard dg(s->ctx ? s->ctx->device : 0);
    if (s->ctx) drop_graphs(s->ctx);
    // the shape's buffers may still be read by work on any stream: wait for the
    // device, then hand them back to the pool
    cudaDeviceSynchronize();
    pool_free(s->pos, nullptr);
    pool_free(s->c, nullptr);
    for (auto& p : s->preps) {
        pool_free(p.B1, nullptr);
        pool_free(p.W, nullptr);
        pool_free(p.G, nullptr);
        for (auto& w : p.Wsh) pool_free(w.second, nullptr);
    }
    delete s;
    return SD_OK;
}

static int check_pair(sd_ctx* ctx, const sd_shape* a, const sd_shape* b) {
    if (!a || !b) return fail(ctx, SD_ERR_ARG, "shape is NULL");
    if (a->ctx != ctx || b->ctx != ctx) return fail(ctx, SD_ERR_ARG, "shape belongs to another context");
    if (a->m == 0 || b->m == 0) return fail(ctx, SD_ERR_ARG, "shape has no samples");
    return SD_OK;
}

int sd_score_rotations(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const double* quats, int64_t n_r,
                       const sd_grid* g, int k_r, sd_cand* cand_out, void* stream) {
    if (!ctx) return SD_ERR_ARG;
    CKI(check_pair(ctx, fixed, moving));
    if (n_r < 0 || n_r > (int64_t)INT32_MAX) return fail(ctx, SD_ERR_ARG, "score_rotations: bad rotation count");
    if (n_r == 0) return SD_OK;
    if (!quats || !cand_out) return fail(ctx, SD_ERR_ARG, "score_rotations: NULL pointer");
    if (k_r < 1 || k_r > 16) return fail(ctx, SD_ERR_ARG, "score_rotations: k_r must be in [1, 16] (got %d)", k_r);
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->p.precision == SD_F64)
        return run_search<double>(ctx, fixed, moving, quats, n_r, g, cand_out, 0, st, k_r);
    return run_search<float>(ctx, fixed, moving, quats, n_r, g, cand_out, 0, st, k_r);
}

int sd_score_maps(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const double* quats, int64_t n_r,
                  const sd_grid* g, void* map_out, void* stream) {
    if (!ctx) return SD_ERR_ARG;
    CKI(check_pair(ctx, fixed, moving));
    if (n_r < 0 || n_r > (int64_t)INT32_MAX) return fail(ctx, SD_ERR_ARG, "score_maps: bad rotation count");
    if (n_r == 0) return SD_OK;
    if (!quats || !map_out) return fail(ctx, SD_ERR_ARG, "score_maps: NULL pointer");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->p.precision == SD_F64) return run_search<double>(ctx, fixed, moving, quats, n_r, g, map_out, 1, st);
    return run_search<float>(ctx, fixed, moving, quats, n_r, g, map_out, 1, st);
}

int sd_tune_export(sd_ctx* ctx, char* buf, int64_t cap, int64_t* len) {
    if (!ctx) return SD_ERR_ARG;
    std::string js = "{\"sdfdock_plans\": 1, \"plans\": [";
    bool first = true;
    for (const auto& kv : ctx->tuned) {
        char e[256];
        snprintf(e, sizeof e, "%s{\"key\": \"%s\", \"batch\": %d, \"spread_bins\": %d, \"fft\": %d}",
                 first ? "" : ", ", kv.first.c_str(), kv.second.B, kv.second.bins, kv.second.fft);
        js += e;
        first = false;
    }
    js += "]}";
    const int64_t need = (int64_t)js.size() + 1;
    if (len) *len = need;
    if (!buf) return SD_OK;
    if (cap < need) return fail(ctx, SD_ERR_ARG, "tune_export: buffer of %lld bytes, %lld needed", (long long)cap,
                                (long long)need);
    memcpy(buf, js.c_str(), (size_t)need);
    return SD_OK;
}

int sd_tune_import(sd_ctx* ctx, const char* json) {
    if (!ctx) return SD_ERR_ARG;
    if (!json || !strstr(json, "\"sdfdock_plans\"")) return fail(ctx, SD_ERR_ARG, "tune_import: not a plan table");
    std::map<std::string, Plan> got;
    const char* p = json;
    while ((p = strstr(p, "{\"key\": \"")) != nullptr) {
        p += strlen("{\"key\": \"");
        const char* q = strchr(p, '"');
        if (!q || q - p > 120) return fail(ctx, SD_ERR_ARG, "tune_import: malformed key");
        std::string key(p, (size_t)(q - p));
        int B = 0, bins = -1, fft = SD_FFT_PRUNED;
        const int nf = sscanf(q, "\", \"batch\": %d, \"spread_bins\": %d, \"fft\": %d}", &B, &bins, &fft);
        if (nf < 2 || B < 1 || B > 64 ||
            (bins != 0 && bins != SPREAD_X && bins != SPREAD_BOX && bins != 8 && bins != 12 && bins != 16) ||
            fft < SD_FFT_FULL || fft > SD_FFT_PRUNED_WIDE)
            return fail(ctx, SD_ERR_ARG, "tune_import: malformed entry for key %s", key.c_str());
        got[key] = Plan{B, bins, fft};
        p = q;
    }
    for (auto& kv : got) ctx->tuned[kv.first] = kv.second;
    return SD_OK;
}

int sd_search_plan(sd_ctx* ctx, const sd_shape* moving, const sd_grid* g, int64_t n_r, int32_t* batch,
                   int32_t* spread_bins, int32_t* fft_plan) {
    if (!ctx) return SD_ERR_ARG;
    if (!moving || moving->ctx != ctx) return fail(ctx, SD_ERR_ARG, "search_plan: bad moving shape");
    if (n_r < 1) return fail(ctx, SD_ERR_ARG, "search_plan: bad rotation count");
    auto plan = [&](auto tag) -> int {
        using T = decltype(tag);
        Search<T> S;
        CKI(make_geo(ctx, g, moving->radius, &S.G));
        S.moving = moving;
        S.n_r = n_r;
        S.plan.B = choose_batch<T>(ctx, S.G, n_r);
        S.plan.bins = (!ctx->opt_spread_direct && bins_supported(ctx)) ? ctx->opt_bin_side : 0;
        S.prunable = ctx->opt_pruned && pruned_len_ok(S.G.n) && S.G.s <= S.G.N;
        S.alt_cols = S.prunable && sizeof(T) == 4 && S.G.n >= 128 && S.G.n <= 384;
        S.plan.fft = fft_plan_default(ctx, S);
        if (ctx->opt_spread_box && bins_supported(ctx)) S.plan.bins = SPREAD_BOX;
        if (ctx->opt_spread_fused && spread_x_ok(ctx, S)) S.plan.bins = SPREAD_X;
        if (ctx->opt_autotune && !ctx->opt_plain && ctx->opt_batch <= 0) {
            auto it = ctx->tuned.find(plan_key(ctx, S));
            if (it != ctx->tuned.end()) {
                S.plan.B = (int)std::min<int64_t>(it->second.B, n_r);
                S.plan.bins = it->second.bins;
                if (ctx->opt_fft_plan < 0 && fft_plan_ok(S, it->second.fft)) S.plan.fft = it->second.fft;
            }
        }
        if (batch) *batch = S.plan.B;
        if (spread_bins) *spread_bins = S.plan.bins;
        if (fft_plan) *fft_plan = S.plan.fft;
        return SD_OK;
    };
    if (ctx->p.precision == SD_F64) return plan(double{});
    return plan(float{});
}

int sd_score_pairs(sd_ctx* ctx, const sd_pair_job* jobs, int64_t n_jobs, sd_pair_stat* stats, void* stream) {
    if (!ctx) return SD_ERR_ARG;
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(ctx, SD_ERR_ARG, "score_pairs: bad job list");
    if (n_jobs == 0) return SD_OK;
    for (int64_t j = 0; j < n_jobs; ++j) {
        CKI(check_pair(ctx, jobs[j].fixed, jobs[j].moving));
        if (jobs[j].n_r < 1 || jobs[j].n_r > (int64_t)INT32_MAX)
            return fail(ctx, SD_ERR_ARG, "score_pairs: job %lld has a bad rotation count", (long long)j);
        if (!jobs[j].quats || !jobs[j].cand_out)
            return fail(ctx, SD_ERR_ARG, "score_pairs: job %lld has a NULL pointer", (long long)j);
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->p.precision == SD_F64) return run_pairs<double>(ctx, jobs, n_jobs, stats, st);
    return run_pairs<float>(ctx, jobs, n_jobs, stats, st);
}

template <typename T>
static int top_k_t(sd_ctx* ctx, const sd_cand* cand, int64_t n_cand, int k, int rescore, const sd_shape* fixed,
                   const sd_shape* moving, const double* quats, const sd_grid* g, sd_pose* out, cudaStream_t st) {
    void *flags, *top, *res;
    CKI(ws_get(ctx, 4, (size_t)((n_cand + 31) / 32) * 4 + 256, &flags));
    const size_t moved_bytes = rescore ? (size_t)k * moving->m * 4 * sizeof(double) : 0;
    const size_t box_bytes = rescore ? (size_t)k * rescore_tiles(moving->m) * 6 * sizeof(float) : 0;
    // layout: [top k sd_cand][re-scores 2k doubles][moved samples][tile boxes], 256-byte aligned
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t res_off = up((size_t)k * sizeof(sd_cand));
    const size_t head = up(res_off + (size_t)k * 2 * sizeof(double));
    CKI(ws_get(ctx, 5, head + up(moved_bytes) + box_bytes + 256, &top));
    res = (char*)top + res_off;
    void* moved = (char*)top + head;
    float* tile_box = (float*)((char*)moved + ((moved_bytes + 255) / 256) * 256);
    CK(ctx, launch_topk(cand, n_cand, k, top, (unsigned*)flags, st));
    if (rescore) {
        RescoreArgs<T> a{};
        a.p1 = (const vec4<T>*)fixed->pos;
        a.c1 = (const cplx<T>*)fixed->c;
        a.m1 = fixed->m;
        a.p2 = (const vec4<T>*)moving->pos;
        a.c2 = (const cplx<T>*)moving->c;
        a.m2 = moving->m;
        a.top = top;
        a.k = k;
        a.quats = quats;
        a.N = g->N;
        a.L = g->L;
        a.sigma_g = ctx->p.sigma_g;
        a.dim = ctx->p.dim;
        a.r2max = moving->radius * moving->radius;
        a.out = (double*)res;
        a.moved = moved;
        a.tile_box = tile_box;
        CK(ctx, launch_rescore<T>(a, st));
    }
    std::vector<sd_cand> hc(k);
    std::vector<double> hr(2 * (size_t)k, 0.0);
    CK(ctx, cudaMemcpyAsync(hc.data(), top, k * sizeof(sd_cand), cudaMemcpyDeviceToHost, st));
    if (rescore) CK(ctx, cudaMemcpyAsync(hr.data(), res, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(ctx, cudaStreamSynchronize(st));
    const double h = g->L / g->N;
    for (int i = 0; i < k; ++i) {
        sd_pose& p = out[i];
        memset(&p, 0, sizeof p);
        p.score = hc[i].score;
        p.rot = hc[i].rot;
        p.idx = hc[i].idx;
        int idx = hc[i].idx < 0 ? 0 : hc[i].idx;
        for (int d = 0; d < ctx->p.dim; ++d) {
            p.t[d] = (double)(idx % g->N - g->N / 2) * h;
            idx /= g->N;
        }
        p.score_fp64 = hr[2 * i];
        p.score_fp64_im = hr[2 * i + 1];
    }
    return SD_OK;
}

int sd_top_k_poses(sd_ctx* ctx, const sd_cand* cand, int64_t n_cand, int k, int rescore_fp64, const sd_shape* fixed,
                   const sd_shape* moving, const double* quats, const sd_grid* g, sd_pose* out, void* stream) {
    if (!ctx) return SD_ERR_ARG;
    if (!cand || !out || n_cand < 1 || n_cand > ((int64_t)1 << 22) || k < 1 || k > 4096)
        return fail(ctx, SD_ERR_ARG, "top_k_poses: need 1 <= n_cand <= 2^22, 1 <= k <= 4096 and buffers");
    if (!g || !grid_ok(g->N)) return fail(ctx, SD_ERR_ARG, "top_k_poses: bad grid");
    if (rescore_fp64) {
        CKI(check_pair(ctx, fixed, moving));
        if (!quats) return fail(ctx, SD_ERR_ARG, "top_k_poses: quats needed for the re-score");
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->p.precision == SD_F64)
        return top_k_t<double>(ctx, cand, n_cand, k, rescore_fp64, fixed, moving, quats, g, out, st);
    return top_k_t<float>(ctx, cand, n_cand, k, rescore_fp64, fixed, moving, quats, g, out, st);
}

template <typename T>
static int score_grad_t(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const sd_grid* g,
                        const void* quats, const void* trans, int64_t P, void* score, void* dq, void* dt,
                        cudaStream_t st) {
    Prep* p = nullptr;
    CKI(prep_fields<T>(ctx, const_cast<sd_shape*>(fixed), g, &p, st));
    void* acc;
    CKI(ws_get(ctx, 4, (size_t)P * 8 * sizeof(double) + 256, &acc));
    GatherArgs<T> a{};
    a.p2 = (const vec4<T>*)moving->pos;
    a.c2 = (const cplx<T>*)moving->c;
    a.m2 = moving->m;
    a.quats = (const T*)quats;
    a.trans = (const T*)trans;
    a.P = P;
    a.G = (const cplx<T>*)p->G;
    a.n = ctx->p.alpha * g->N;
    a.pn = a.n + ctx->p.w;
    a.inv_h = (T)(a.n / g->L);
    a.beta = (T)ctx->p.beta;
    a.w = ctx->p.w;
    a.acc = (double*)acc;
    CK(ctx, launch_gather<T>(a, ctx->p.dim, st));
    CK(ctx, launch_grad_finalize<T>((const double*)acc, (const T*)quats, P, ctx->p.dim, (T*)score, (T*)dq, (T*)dt, st));
    return SD_OK;
}

template <typename T>
static int refine_t(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const sd_grid* g, void* quats,
                    void* trans, int64_t P, int steps, const RefineParams& rp, void* hist, cudaStream_t st) {
    Prep* p = nullptr;
    CKI(prep_fields<T>(ctx, const_cast<sd_shape*>(fixed), g, &p, st));
    void *acc, *state = nullptr;
    CKI(ws_get(ctx, 4, (size_t)P * 8 * sizeof(double) + 256, &acc));
    if (rp.method != SD_REFINE_ASCENT) CKI(ws_get(ctx, 7, (size_t)P * 12 * sizeof(double) + 256, &state));
    GatherArgs<T> a{};
    a.p2 = (const vec4<T>*)moving->pos;
    a.c2 = (const cplx<T>*)moving->c;
    a.m2 = moving->m;
    a.quats = (const T*)quats;
    a.trans = (const T*)trans;
    a.P = P;
    a.G = (const cplx<T>*)p->G;
    a.n = ctx->p.alpha * g->N;
    a.pn = a.n + ctx->p.w;
    a.inv_h = (T)(a.n / g->L);
    a.beta = (T)ctx->p.beta;
    a.w = ctx->p.w;
    a.acc = (double*)acc;
    for (int k = 0; k <= steps; ++k) {
        CK(ctx, launch_gather<T>(a, ctx->p.dim, st));
        T* h = hist ? (T*)hist + (int64_t)k * P : nullptr;
        CK(ctx, launch_refine_step<T>((const double*)acc, (T*)quats, (T*)trans, (double*)state, P, ctx->p.dim, rp,
                                      k == 0, h, k == steps, st));
    }
    return SD_OK;
}

int sd_refine(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const sd_grid* g, void* quats,
              void* trans, int64_t P, int steps, const sd_refine_params* params, void* hist, void* stream) {
    if (!ctx) return SD_ERR_ARG;
    CKI(check_pair(ctx, fixed, moving));
    if (!params) return fail(ctx, SD_ERR_ARG, "refine: params is NULL");
    if (P < 0 || steps < 0) return fail(ctx, SD_ERR_ARG, "refine: negative pose or step count");
    if (P == 0) return SD_OK;
    if (!quats || !trans) return fail(ctx, SD_ERR_ARG, "refine: NULL pointer");
    RefineParams rp{params->method, params->lr_t, params->lr_q, params->mass, params->inertia, params->damping,
                    params->dt};
    auto finite_nonneg = [](double x) { return isfinite(x) && x >= 0.0; };
    if (rp.method == SD_REFINE_ASCENT || rp.method == SD_REFINE_CG) {
        if (!finite_nonneg(rp.lr_t) || !finite_nonneg(rp.lr_q))
            return fail(ctx, SD_ERR_ARG, "refine: step sizes must be finite and non-negative");
    } else if (rp.method == SD_REFINE_DYNAMICS) {
        if (!(isfinite(rp.mass) && rp.mass > 0.0) || !(isfinite(rp.inertia) && rp.inertia > 0.0) ||
            !(rp.damping >= 0.0 && rp.damping <= 1.0) || !finite_nonneg(rp.h))
            return fail(ctx, SD_ERR_ARG, "refine: dynamics needs mass, inertia > 0, damping in [0, 1], dt >= 0");
    } else {
        return fail(ctx, SD_ERR_ARG, "refine: unknown method %d", rp.method);
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->p.precision == SD_F64) return refine_t<double>(ctx, fixed, moving, g, quats, trans, P, steps, rp, hist, st);
    return refine_t<float>(ctx, fixed, moving, g, quats, trans, P, steps, rp, hist, st);
}

int sd_refine_poses(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const sd_grid* g, void* quats,
                    void* trans, int64_t P, int steps, double lr_t, double lr_q, void* hist, void* stream) {
    sd_refine_params rp{SD_REFINE_ASCENT, lr_t, lr_q, 1.0, 1.0, 0.0, 0.0};
    return sd_refine(ctx, fixed, moving, g, quats, trans, P, steps, &rp, hist, stream);
}

int sd_score_grad(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const sd_grid* g, const void* quats,
                  const void* trans, int64_t P, void* score, void* dq, void* dt, void* stream) {
    if (!ctx) return SD_ERR_ARG;
    CKI(check_pair(ctx, fixed, moving));
    if (P < 0 || P > 65535) return fail(ctx, SD_ERR_ARG, "score_grad: 0 <= P <= 65535");
    if (P == 0) return SD_OK;
    if (!quats || !trans || !score || !dq || !dt) return fail(ctx, SD_ERR_ARG, "score_grad: NULL pointer");
    if (!g || !grid_ok(g->N)) return fail(ctx, SD_ERR_ARG, "score_grad: bad grid");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->p.precision == SD_F64)
        return score_grad_t<double>(ctx, fixed, moving, g, quats, trans, P, score, dq, dt, st);
    return score_grad_t<float>(ctx, fixed, moving, g, quats, trans, P, score, dq, dt, st);
}

// Host execution of the line-FFT stage sequence used by every pass kernel, in
// FP64: lets the index arithmetic be checked without a GPU.  in/out: len x 2.
int sd_host_line_fft(int len, int inverse, const double* in, double* out) {
    if (!in || !out || !fft_len_supported(len)) return SD_ERR_ARG;
    std::vector<double2> a(pad(len) + 2), tw(std::max(tw_count(len), 1));
    tw_for_each(len, [&](int j, int r, int k, int P, int R) {
        const double ang = -2.0 * M_PI * (double)(r * k) / (double)(P * R);
        tw[j] = make_double2(cos(ang), sin(ang));
    });
    for (int j = 0; j < len; ++j) a[pad(j)] = make_double2(in[2 * j], in[2 * j + 1]);
#define SD_HOST_CASE(L)                                                 \
    case L:                                                             \
        if (inverse) fft_line_host<double2, L, true>(a.data(), tw.data()); \
        else fft_line_host<double2, L, false>(a.data(), tw.data());        \
        break;
    switch (len) { SD_FOR_EACH_LEN(SD_HOST_CASE) }
#undef SD_HOST_CASE
    for (int j = 0; j < len; ++j) {
        out[2 * j] = a[pad(j)].x;
        out[2 * j + 1] = a[pad(j)].y;
    }
    return SD_OK;
}

const char* sd_version(void) { return "sdfdock 0.1 (sm_103a)"; }

int64_t sd_launch_count(void) { return (int64_t)g_launches.load(); }

// Helpers for entry points defined in other translation units.
int sd_internal_fail(sd_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return fail(ctx, code, "%s", buf);
}

int sd_internal_device(const sd_ctx* ctx) { return ctx ? ctx->device : -1; }

int sd_pass_times(sd_ctx* ctx, int kind, int64_t* launches, double* ms) {
    if (!ctx) return SD_ERR_ARG;
    DeviceGuard dg(ctx->device);
    harvest_timers(ctx);
    if (kind < 0) {
        for (int k = 0; k < SD_PASS_COUNT; ++k) {
            ctx->pass_ms[k] = 0.0;
            ctx->pass_n[k] = 0;
        }
        return SD_OK;
    }
    if (kind >= SD_PASS_COUNT) return fail(ctx, SD_ERR_ARG, "pass kind out of range");
    if (launches) *launches = ctx->pass_n[kind];
    if (ms) *ms = ctx->pass_ms[kind];
    return SD_OK;
}
