/*
 * sdfdock.h - C ABI of the skeletal-density (SDF) shape-complementarity library.
 *
 * The library scores rigid poses of a moving solid S2 against a fixed solid S1
 * (Behandish & Ilies, "Shape Complementarity Analysis for Objects of Arbitrary
 * Shape"): each solid's skeletal density function rho (Section 4, Eq. 13 with
 * the kernel of Eq. 15) is sampled at query points, the samples carry Gaussians,
 * and the score f(tau) = integral of rho1(p) rho2(tau^-1 p) dv (Eq. 1 / Eq. 8)
 * is searched over rotations x translations with one FFT per rotation
 * (Section 5), using a nonequispaced FFT for the scattered samples.
 *
 * Conventions shared by every call
 * --------------------------------
 * - All functions return an int: SD_OK (0) or a negative SD_ERR_* code.  The
 *   message of the last failure is in sd_last_error(ctx).  No call aborts the
 *   process or throws across the ABI.
 * - "real" means float for a context created with precision SD_F32 and double
 *   for SD_F64.  Complex numbers are (re, im) pairs of real.
 * - Points are stored as 4 reals (x, y, z, unused); 2D contexts ignore z.
 * - Pointers marked "device" are CUDA device pointers on the context's device;
 *   "host" pointers are ordinary memory.  The caller keeps ownership of every
 *   buffer it passes.  Calls are asynchronous on `stream` (a cudaStream_t, NULL
 *   for the legacy default stream) unless stated otherwise.
 * - Quaternions are (w, x, y, z), Hamilton product, acting as the active
 *   rotation p -> q p q*; they need not be normalised.  A pose (R, t) moves S2 as
 *   x -> R x + t about S2's frame origin.
 * - Translations of the score grid are t_m = (i - N/2) * h, h = L / N, for
 *   i in [0, N) per axis; the flat index of a translation is
 *   (iz * N + iy) * N + ix (3D) or iy * N + ix (2D).
 */
#ifndef SDFDOCK_H
#define SDFDOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SD_OK 0
#define SD_ERR_ARG (-1)           /* invalid argument or unsupported size           */
#define SD_ERR_OOM (-2)           /* device allocation failed                       */
#define SD_ERR_CUDA (-3)          /* a CUDA runtime call or kernel launch failed    */
#define SD_ERR_TIMEOUT (-4)       /* reserved: a bounded device wait gave up        */
#define SD_ERR_UNIMPLEMENTED (-5) /* a valid request this library does not support  */
#define SD_ERR_NONFINITE (-6)     /* a result was NaN or infinite                   */

#define SD_F32 0
#define SD_F64 1

typedef struct sd_ctx sd_ctx;
typedef struct sd_shape sd_shape;

/* Parameters of a context.  sd_default_params() fills the paper's validation
 * values (Section 6): lambda1 = 1, lambda2 = 3, sigma_t = 0.5, eps = 1.5. */
typedef struct sd_params {
    int dim;          /* 2 or 3                                                        */
    int precision;    /* SD_F32 or SD_F64: the arithmetic of every kernel              */
    double lambda1;   /* Eq. 16c: weight outside the solid (+lambda1)                  */
    double lambda2;   /* Eq. 16c: weight inside the solid (-lambda2)                   */
    double sigma_t;   /* Eq. 15: thickness factor of the medial Gaussian               */
    double eps;       /* Eq. 17t: truncation; INFINITY keeps every boundary sample     */
    double sigma_g;   /* width of the Gaussian carried by each SDF sample              */
    int w;            /* spreading width in grid cells of the oversampled grid (2..16) */
    int alpha;        /* oversampling factor of the nonequispaced FFT (only 2)         */
    double beta;      /* shape of the exponential-of-semicircle kernel; <= 0: 2.30*w   */
    int phi;          /* SD_PHI_*: the phi-kernel of Eq. 13 (default SD_PHI_SDF)        */
    double phi_radius;/* characteristic radius R of SD_PHI_RADIAL / SD_PHI_SKIN (> 0)   */
} sd_params;

/* phi-kernels (Section 4: Eq. 13 holds for any phi, each giving an affinity).  g is
 * the normalised Gaussian of width sigma_t, R = phi_radius, lambda = +lambda1
 * outside and -lambda2 inside (Eq. 16c).
 *   SD_PHI_SDF       Eq. 15 with the truncation of Eq. 17t: the skeletal density.
 *   SD_PHI_PROXIMAL  phi = lambda zeta^-2 / sqrt(2 pi): the proximal factor alone
 *                    (inverse-square, no characteristic size; eps is ignored).
 *   SD_PHI_RADIAL    phi = c g(eta / R - 1) with c = lambda1 outside, i lambda2
 *                    inside: uses eta = Im zeta only, like a radial-basis
 *                    double-skin affinity (eps is ignored).
 *   SD_PHI_SKIN      rho = lambda1 g(xi / R - 1) + i lambda2 g(xi / R + 1): the
 *                    skin / core layers of the signed distance (no boundary sum).
 * In 2D the inverse-square kernels take the planar angle measure as Eq. 15 does. */
#define SD_PHI_SDF 0
#define SD_PHI_PROXIMAL 1
#define SD_PHI_RADIAL 2
#define SD_PHI_SKIN 3

/* Translation grid: N points per axis on a periodic box of side L. */
typedef struct sd_grid {
    int N;            /* one of 8, 16, 24, 32, 48, 64, 96, 128, 192, 256 */
    double L;
} sd_grid;

/* Per-rotation best translation (16 bytes). */
typedef struct sd_cand {
    double score;     /* Re f_N at the best translation of this rotation */
    int32_t rot;      /* rotation index in the call's quaternion list    */
    int32_t idx;      /* flat translation index                          */
} sd_cand;

/* A ranked pose. */
typedef struct sd_pose {
    double score;         /* Re f_N from the FFT search                          */
    double score_fp64;    /* Re f_c from FP64 direct pair sums (0 if not asked)  */
    double score_fp64_im; /* Im f_c, a diagnostic                                */
    int32_t rot;
    int32_t idx;
    double t[3];          /* translation of the pose (t[2] = 0 in 2D)            */
} sd_pose;

/* ---- context ------------------------------------------------------------ */

/* Fill *p with defaults for the given dimension and precision. */
int sd_default_params(sd_params* p, int dim, int precision);

/* Create a context on CUDA device `device`.  Validates *p (SD_ERR_ARG). */
int sd_create(sd_ctx** out, int device, const sd_params* p);

/* Free a context, its workspace and its cached plans.  Shapes made with it
 * must be freed first; NULL is accepted. */
int sd_destroy(sd_ctx* ctx);

/* Message of the last failure on this context ("" if none).  Valid until the
 * next call on the context.  A NULL ctx returns the message of the last failed
 * sd_create. */
const char* sd_last_error(const sd_ctx* ctx);

/* A context serves one host thread at a time: calls on one context from
 * several threads must be serialised by the caller.
 *
 * Set a tuning option: "batch" (rotations per batch, 0 = automatic),
 * "graph" (1: replay the batched launch sequence from a captured CUDA graph;
 * needs a non-NULL stream; the first call with given arguments runs eagerly,
 * later ones capture once and replay), "plain" (1: one rotation per batch, no
 * graph), "timing" (1: CUDA-event timing of every pass, see sd_pass_times),
 * "spread_direct" (1, the default: spread with global vector atomics per kernel
 * row; 0: sort the samples into 16^d-cell bins and accumulate each bin's taps in
 * shared memory first), "spread_bin_side" (8, 12 or 16, default 16: the bin
 * side of binned spreading when the autotuner does not choose it), "pruned"
 * (1, the default: the forward FFT passes of the
 * search read the spread sub-box unshifted and compute only the kept modes, with
 * the shift applied as a phase in the product table; 0: the shifted sub-box and
 * every mode; results are the same up to FP rounding), "fft_plan" (-1, the
 * default: the autotuner's choice, else SD_FFT_PRUNED where the pruned passes
 * apply; 0..3: that SD_FFT_* plan wherever it applies, never tuned),
 * "inverse_cluster" (1: in 3D FP32 searches with N in {32, 48, 64, 96, 128,
 * 192, 256} returning maps or one candidate per rotation, the inverse y and x
 * transforms of each z-plane run in one kernel, a cluster of 8 CTAs per plane
 * holding the plane in distributed shared memory between the two axes; 0, the
 * default: two passes through device memory, measured faster; same results up
 * to FP rounding),
 * "spread_box" (1: each
 * CTA spreads a block of Morton-consecutive samples into a shared box of the
 * sub-box and adds the box's nonzero cells with 16-byte atomics; FP32, w 4-7;
 * default 0), "spread_fused" (1: in
 * pruned 3D FP32 searches with w = 6, spread each rotation's samples straight
 * into whole rows held in shared memory and run the forward x transform there,
 * with no sub-box in device memory; default 0), "sdf_cull" (2, the default:
 * the SDF sums skip every 256-sample boundary tile that lies beyond the
 * truncation radius (1 + eps)|xi| of every query of a block, and each warp skips
 * the 32-sample sub-tiles beyond that radius of its own 32 queries -- the
 * restriction of Eq. 13's sum to the eps-approximate neighbours of Section 4
 * through the Morton-ordered samples; 1: tiles only; 0: sum over every tile;
 * results are the same), "autotune" (1: before a scoring job
 * runs, time its candidate plans -- rotations per batch from a quarter to
 * twice the automatic choice, direct spreading, shared boxes of sample blocks,
 * bins of 8, 12 or 16 cells, or
 * (pruned 3D FP32 searches with w = 6) spreading fused with the forward x
 * transform -- on its first
 * rotations and keep the fastest, then time the other forward-pass FFT plans
 * (SD_FFT_*) under that choice and keep the fastest of those; the choice is
 * cached per precision, grid,
 * sub-box size and sample-count octave; ignored when "batch" or "plain" is
 * set; results do not depend on the plan beyond FP32 rounding). */
int sd_set_option(sd_ctx* ctx, const char* key, int64_t value);

/* ---- shapes: the sampled SDF (Section 4, Eq. 10A-17t) ------------------- */

/* Build a shape's sampled SDF from oriented boundary samples.
 *   bnd   device, n_b x 4 real: boundary sample positions q_j
 *   nrm   device, n_b x 4 real: unit outward normals n_j
 *   area  device, n_b real: boundary measure a_j carried by each sample
 *   qry   device, m x 4 real: query points p_i
 *   vol   device, m real: cell volume v_i of each query point
 *   pmc_override  device, m int8 (+1 outside, -1 inside) or NULL to use the
 *         winding-number membership of the samples
 *   out   receives a new shape holding p_i and c_i = rho(p_i) v_i
 *   rho_out  device, m x 2 real, or NULL: receives rho(p_i)
 * rho follows Eq. 13 with Eq. 15/16c and the truncation of Eq. 17t, xi from
 * Eq. 10A (nearest sample), zeta = xi + i eta (Eq. 11),
 * cos(theta) from Eq. 12a; in 2D each element is weighted by its planar angle
 * over 2 pi.  The shape stores its samples in Morton (Z-curve) order of
 * position; rho_out is in the caller's order.  Synchronises `stream`. */
int sd_sdf_build(sd_ctx* ctx, const void* bnd, const void* nrm, const void* area, int64_t n_b,
                 const void* qry, const void* vol, int64_t m, const int8_t* pmc_override,
                 sd_shape** out, void* rho_out, void* stream);

/* Make a shape directly from weighted samples (p_i device m x 4 real,
 * c_i device m x 2 real).  Copies them, stored in Morton order of position.
 * Synchronises `stream`. */
int sd_shape_from_samples(sd_ctx* ctx, const void* pos, const void* c, int64_t m,
                          sd_shape** out, void* stream);

/* Number of samples and the largest |p_i| of a shape. */
int sd_shape_info(const sd_shape* s, int64_t* m, double* radius);

/* Free a shape and its cached spectra; NULL is accepted. */
int sd_shape_free(sd_shape* s);

/* ---- adaptive sampling of the SDF (Section 5, octree) ------------------ */

/* Section 5 proposes sampling the SDF on a tree subdivided deepest where the
 * skeletal density is high, instead of a uniform grid, and scoring the
 * nonequispaced samples with a nonequispaced FFT (what sd_score_rotations runs).
 * sd_octree builds such a tree (a quadtree in 2D) on the HOST, one level at a
 * time, from SDF values the caller evaluates -- normally with sd_sdf_build's
 * rho_out at the centres sd_octree_pending lists.  Needs no GPU.
 *
 * Rule: the root is the cube [lo, lo + size]^dim, cut uniformly into
 * 2^depth_min cells per axis.  A cell of side h = size / 2^D at depth
 * D < depth_max, centre c, is split into its 2^dim children when the boundary
 * sample nearest c lies closer than half the cell's diagonal (0.5 h sqrt(dim)),
 * or else when |rho(c)| h^dim >= tau.  Cells not split are leaves (position c,
 * volume h^dim), except that a leaf whose centre lies closer than `clearance`
 * to a boundary sample is dropped, and so is a leaf whose centre lies farther
 * than `band` from it; a cell whose centre lies farther than band + 0.5 h sqrt(dim)
 * lies wholly beyond the band and is dropped without being split or evaluated
 * (band = INFINITY keeps everything).  Leaves are listed by depth, then by the
 * linear index k_x + 2^D (k_y + 2^D k_z) of their integer coordinates
 * k = (c - lo) / h - 1/2.  tau = 0 gives the uniform grid at depth_max.
 *
 *   bnd        host, n_b x 4 double: boundary sample positions (x, y, z, pad);
 *              n_b = 0 (bnd may be NULL) means no boundary; copied
 *   lo         host, dim doubles: the root's lowest corner
 *   depth_min <= depth_max <= 20
 * Errors: SD_ERR_ARG for bad arguments, SD_ERR_NONFINITE for a non-finite
 * boundary position, SD_ERR_OOM when a level would exceed 2^27 cells or memory
 * runs out; *out is NULL then.  Not thread-safe per tree. */
typedef struct sd_octree sd_octree;
int sd_octree_create(int dim, const double* bnd, int64_t n_b, const double* lo, double size, int depth_min,
                     int depth_max, double tau, double clearance, double band, sd_octree** out);

/* The cells of the current level that need rho: *n of them (0 once the tree
 * is complete).  centres (host, n x 4 double, or NULL) receives their centres
 * (x, y, z, 0), vol (host, n double, or NULL) their volumes h^dim. */
int sd_octree_pending(const sd_octree* t, int64_t* n, double* centres, double* vol);

/* Feed rho at the pending centres (host, n x 2 double: re, im, in the order
 * sd_octree_pending listed them) and resolve levels until rho is needed again
 * or the tree is complete.  n must equal the pending count (SD_ERR_ARG);
 * a non-finite value returns SD_ERR_NONFINITE and leaves the tree unchanged;
 * SD_ERR_OOM (level too large) leaves the tree unusable. */
int sd_octree_feed(sd_octree* t, const double* rho, int64_t n);

/* The leaves of a complete tree (SD_ERR_ARG before): *m of them; centres
 * (host, m x 4 double), vol (host, m double) and coords (host, m x 4 int32:
 * k_x, k_y, k_z, depth) may each be NULL. */
int sd_octree_leaves(const sd_octree* t, int64_t* m, double* centres, double* vol, int32_t* coords);

/* Free a tree; NULL is accepted. */
int sd_octree_free(sd_octree* t);

/* ---- search over rotations x translations (Section 5) ------------------ */

/* For each rotation r, the best translation of Re f_N(R_r, t) over the grid.
 *   quats     device, n_r x 4 double
 *   k_r       candidates per rotation, 1 <= k_r <= 16: the k_r best translations
 *             of each rotation (score descending, index ascending)
 *   cand_out  device, n_r x k_r sd_cand, ordered by rotation, then rank
 * f_N is the band-limited periodic score: the pair sum of c1_i c2_j times the
 * Fourier series of the Gaussian of width sigma_g*sqrt(2) on the box, modes
 * |kappa_d| < N/2.  Computed per rotation as: rotate S2's samples, spread them
 * onto the oversampled grid, forward FFT (type-1 nonuniform FFT), multiply by
 * the fixed shape's table, inverse FFT, argmax (ties to the lowest index). */
int sd_score_rotations(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving,
                       const double* quats, int64_t n_r, const sd_grid* g, int k_r,
                       sd_cand* cand_out, void* stream);

/* The complex score maps f_N for each rotation, for inspection and testing.
 *   map_out   device, n_r x N^dim x 2 real, flat translation order. */
int sd_score_maps(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving,
                  const double* quats, int64_t n_r, const sd_grid* g, void* map_out,
                  void* stream);

/* One scoring job of sd_score_pairs: a pair of shapes of this context, its
 * grid, its rotations (device, n_r x 4 double) and its per-rotation argmax
 * output (device, n_r sd_cand), as for sd_score_rotations with k_r = 1. */
typedef struct sd_pair_job {
    const sd_shape* fixed;
    const sd_shape* moving;
    const double* quats;
    int64_t n_r;
    sd_grid grid;
    sd_cand* cand_out;
} sd_pair_job;

/* Per-job report of sd_score_pairs. */
typedef struct sd_pair_stat {
    double ms;            /* device time of the job within the call */
    int32_t batch;        /* rotations per batch of its plan */
    int32_t spread_bins;  /* bin side of its plan's binned spreading, 0: direct,
                             1: spreading fused with the forward x transform,
                             2: shared boxes of sample blocks */
    int32_t n;            /* oversampled grid size per axis */
    int32_t s;            /* sub-box side of its moving shape */
    int32_t fft_plan;     /* forward-pass plan of its search (SD_FFT_*) */
} sd_pair_stat;

/* Score many shape pairs, each on its own grid and rotation list, in one
 * launch sequence on `stream` (Section 5's search applied to a batch of
 * problems).  Each job runs with its own plan (autotuned when the "autotune"
 * option is on); the workspace is sized once for the largest job.  The first
 * call with a given job list runs eagerly; later calls with the same list
 * replay one captured CUDA graph holding every job.  Each job's candidates
 * are those of sd_score_rotations on it, up to the FP32 rounding of the
 * spreading's atomic order (its plan may differ).
 *   jobs   host, n_jobs sd_pair_job; pointers inside stay valid while the
 *          context may replay the graph (until sd_shape_free or sd_destroy)
 *   stats  host, n_jobs sd_pair_stat, or NULL.  When given, the call
 *          synchronises on the end of the sequence and fills each job's time
 *          (from events around each job) and plan; otherwise it is
 *          asynchronous.
 * Errors: SD_ERR_ARG for a bad job (NULL pointer, n_r < 1, a shape of another
 * context), as sd_score_rotations otherwise. */
int sd_score_pairs(sd_ctx* ctx, const sd_pair_job* jobs, int64_t n_jobs, sd_pair_stat* stats,
                   void* stream);

/* Forward-pass FFT plans of a search (Section 5's transform over the
 * translations, computed axis by axis):
 *   SD_FFT_FULL           every pass reads the shifted sub-box padded to n and
 *                         computes all n outputs of each line
 *   SD_FFT_PRUNED         the passes skip the zero upper half of each line and
 *                         compute only the N kept modes; the sub-box shift is a
 *                         phase folded into the product table
 *   SD_FFT_PRUNED_NARROW  as PRUNED, with half the columns per CTA in the
 *                         forward y and fused last-axis passes (FP32, n 128..384)
 *   SD_FFT_PRUNED_WIDE    as PRUNED, with twice the columns per CTA there
 *                         (FP32, n 128..384) */
#define SD_FFT_FULL 0
#define SD_FFT_PRUNED 1
#define SD_FFT_PRUNED_NARROW 2
#define SD_FFT_PRUNED_WIDE 3

/* The plan a search of n_r rotations of `moving` on grid g would run with now:
 * rotations per batch, the bin side of binned spreading (0: direct; 1:
 * spreading fused with the forward x transform; 2: shared boxes of sample
 * blocks) and the forward-pass FFT plan (SD_FFT_*).  Each output pointer may
 * be NULL.  With the
 * "autotune" option it is the cached choice for this geometry if there is one
 * (the first search of a geometry makes it), else the default.  No device work. */
int sd_search_plan(sd_ctx* ctx, const sd_shape* moving, const sd_grid* g, int64_t n_r, int32_t* batch,
                   int32_t* spread_bins, int32_t* fft_plan);

/* The autotuner's cached plans as JSON text,
 *   {"sdfdock_plans": 1, "plans": [{"key": K, "batch": B, "spread_bins": S, "fft": F}, ...]}
 * (K: precision|dim|N|n|sub-box/16|log2 of the moving sample count).  *len
 * receives the size including the terminating NUL; with buf NULL only the size
 * is returned; a smaller cap is SD_ERR_ARG. */
int sd_tune_export(sd_ctx* ctx, char* buf, int64_t cap, int64_t* len);

/* Add the plans of a JSON text written by sd_tune_export to this context's
 * cache (entries with a key already present are replaced), so searches of those
 * geometries skip the timing trials (an entry without "fft" takes
 * SD_FFT_PRUNED; a plan that does not apply to a job is replaced by the job's
 * default there).  A text that is not such a table, or an entry with batch
 * outside [1, 64], spread_bins not 0, 1, 2, 8, 12 or 16, or fft not 0 to 3,
 * is SD_ERR_ARG and leaves the cache unchanged. */
int sd_tune_import(sd_ctx* ctx, const char* json);

/* Global top-k over per-rotation candidates, ordered by score descending,
 * then rotation ascending, then translation index ascending; optionally each
 * pose is re-scored in FP64 by direct pair sums of the continuous score
 * f_c = sum_ij c1_i c2_j G_{sigma_g sqrt 2}(R p2_j + t - p1_i) (pairs farther
 * than 8 sigma_g sqrt 2 are skipped).
 *   cand   device, n_cand sd_cand (1 <= n_cand <= 2^22)
 *   quats  device, the quaternion list the candidates index
 *   out    host, k sd_pose
 * Synchronises `stream`. */
int sd_top_k_poses(sd_ctx* ctx, const sd_cand* cand, int64_t n_cand, int k, int rescore_fp64,
                   const sd_shape* fixed, const sd_shape* moving, const double* quats,
                   const sd_grid* g, sd_pose* out, void* stream);

/* ---- score and gradient at arbitrary poses (Section 6, gradient search) -- */

/* Re f_N and its gradient at P poses, by a type-2 gather of the band-limited
 * field Phi(x) = sum_i c1_i K_N(x - p1_i) and its gradient at R p2_j + t.
 *   quats  device, P x 4 real (raw quaternions)
 *   trans  device, P x 3 real (2D: z ignored)
 *   score  device, P real
 *   dq     device, P x 4 real: d score / d q through R(q/|q|) (orthogonal to q)
 *   dt     device, P x 3 real: d score / d t (2D: dt[2] = 0) */
int sd_score_grad(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const sd_grid* g,
                  const void* quats, const void* trans, int64_t P, void* score, void* dq,
                  void* dt, void* stream);

/* Gradient ascent on Re f_N from P starting poses, all on the device (the
 * gradient-driven search of Section 6): each of `steps` steps evaluates the
 * score and gradient as sd_score_grad does, then moves each translation by
 * lr_t * dt / max|dt| and each quaternion by lr_q * dq / max|dq| (so a pose's
 * largest move per step is lr_t, resp. lr_q, in its own units) and normalises
 * the quaternion.
 *   quats  device, P x 4 real (raw quaternions, updated in place)
 *   trans  device, P x 3 real (updated in place; 2D: z ignored)
 *   hist   device, (steps + 1) x P real, or NULL: the score before each step
 *          and after the last
 * Asynchronous on `stream`; one gather and one small kernel per step. */
int sd_refine_poses(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const sd_grid* g,
                    void* quats, void* trans, int64_t P, int steps, double lr_t, double lr_q, void* hist,
                    void* stream);

/* Pose-update rules of sd_refine (Section 6: the score as a virtual energy
 * E ~ -f with force F = d Re f / dt and torque T = sum_j (R p2_j) x g_j, the
 * derivative for a left rotation R <- exp([omega]x) R). */
#define SD_REFINE_ASCENT 0    /* t += lr_t F / max|F|; q += lr_q dq / max|dq|, normalised */
#define SD_REFINE_CG 1        /* Polak-Ribiere (beta clipped at 0) per translation / rotation block;
                                 t moves lr_t along its direction, R turns lr_q radians */
#define SD_REFINE_DYNAMICS 2  /* damped rigid body from rest: v <- (1-damping) v + dt F / mass,
                                 w <- (1-damping) w + dt T / inertia, t += dt v, q <- exp(dt w) q */

typedef struct sd_refine_params {
    int method;      /* SD_REFINE_* */
    double lr_t;     /* ascent, CG: largest translation per step */
    double lr_q;     /* ascent: largest quaternion change per step; CG: rotation per step (radians) */
    double mass;     /* dynamics: mass (> 0) */
    double inertia;  /* dynamics: scalar moment of inertia (> 0) */
    double damping;  /* dynamics: velocity damping factor per step, in [0, 1] */
    double dt;       /* dynamics: time step (>= 0) */
} sd_refine_params;

/* Local maximisation of Re f_N from P starting poses on the device with one of
 * the SD_REFINE_* rules: `steps` updates, each after a type-2 gather of the
 * score, force and torque (as sd_score_grad).  quats / trans / hist as for
 * sd_refine_poses; per-pose state (CG directions, velocities) lives in the
 * context's workspace.  SD_ERR_ARG for an unknown method or out-of-range
 * parameter.  Asynchronous on `stream`. */
int sd_refine(sd_ctx* ctx, const sd_shape* fixed, const sd_shape* moving, const sd_grid* g, void* quats,
              void* trans, int64_t P, int steps, const sd_refine_params* params, void* hist, void* stream);

/* ---- allocation-free variant ------------------------------------------------- */

/* Largest candidate count accepted by sd_top_k_static. */
#define SD_TOP_K_STATIC_MAX (1 << 20)

/* Top-k selection over per-rotation candidates, ordered like sd_top_k_poses
 * (score descending, rotation ascending, index ascending; no FP64 re-score),
 * that allocates no device memory.  The paper has no counterpart of this entry:
 * it exists for callers that cannot allocate while they run (real-time loops
 * that must not stall on cudaMalloc's implicit synchronisation, engines bound
 * to a fixed shared memory pool, device memory owned by a foreign allocator).
 *   cand   device, n_cand sd_cand, 1 <= n_cand <= SD_TOP_K_STATIC_MAX
 *   out    device, k sd_cand (1 <= k <= 4096), best first; entries past the
 *          number of candidates have rot = idx = -1
 * Scratch: a 128 KiB bitset in a fixed device array that every GPU which loads
 * the library keeps until the process exits; each call clears the bits it uses.
 * The first call on a device looks up the array's device address (set-up):
 * make that first call before any stream capture.  The address stays cached for
 * the process, so a cudaDeviceReset (or anything else that destroys the
 * device's primary context) invalidates it together with every context and
 * shape on that device: do not call this entry on a device after such a reset.
 * All calls share the one array, so calls whose kernels can overlap on the GPU
 * (other streams, other host threads) race; serialise them.  Larger inputs
 * return SD_ERR_ARG.
 * Cost: one CTA makes k passes over the candidates, O(k n_cand) reads (the same
 * selection as sd_top_k_poses); at k = 4096 and n_cand = 2^20 that is 64 GiB of
 * reads by one SM.
 * Asynchronous on `stream`. */
int sd_top_k_static(sd_ctx* ctx, const sd_cand* cand, int64_t n_cand, int k, sd_cand* out, void* stream);

/* ---- diagnostics ----------------------------------------------------------- */

/* Runs, on the host in FP64, the same sequence of mixed-radix Stockham stages
 * that the device line FFTs execute, for one line of `len` points (a supported
 * length: 8, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512).  Forward
 * (inverse = 0) is X_k = sum_j x_j exp(-2 pi i jk/len); inverse uses +i and is
 * unnormalised.  in, out: host, len x 2 double.  Needs no GPU. */
int sd_host_line_fft(int len, int inverse, const double* in, double* out);

/* Probe of an arithmetic rate of this GPU, for the rooflines of the kernels
 * bound by arithmetic rather than memory (the SDF sums: FP32 FMA and the
 * special-function unit; the FP64 re-score: FP64 FMA) or by shared-memory
 * atomics (the spreading tiles).  The paper has no counterpart.  Runs a probe
 * kernel (eight independent dependency chains per thread, or for the atomic
 * kinds each lane adding to its own shared word, so that the lanes of a warp
 * hit distinct banks; eight CTAs of 256 threads per SM) on `device` for a few
 * to tens of milliseconds, synchronously on the legacy default stream, and
 * stores the best of three timed launches in *ops_per_s: floating-point
 * operations per second for the FMA kinds (two per FMA), instructions (atomic
 * adds) per second for the others.  Allocates 4 bytes of device memory for the
 * duration of the call.  SD_ERR_ARG for an unknown kind or device, SD_ERR_CUDA
 * if a CUDA call fails. */
#define SD_PEAK_FP32_FMA 0
#define SD_PEAK_FP64_FMA 1
#define SD_PEAK_SFU_EX2 2    /* ex2.approx.f32 (the exponential's special-function step) */
#define SD_PEAK_SFU_RSQRT 3  /* rsqrt.approx.f32 */
#define SD_PEAK_SHARED_ADD32 4 /* 32-bit integer atomic add to shared memory */
#define SD_PEAK_SHARED_ADD64 5 /* 64-bit integer atomic add to shared memory */
int sd_alu_peak(int device, int kind, double* ops_per_s);

/* Library version string (static storage). */
const char* sd_version(void);

/* Number of kernels the library has launched in this process. */
int64_t sd_launch_count(void);

/* Pass kinds of the search pipeline, for sd_pass_times. */
#define SD_PASS_CLEAR 0   /* zeroing of the spread sub-box                    */
#define SD_PASS_SPREAD 1  /* rotate + spread (type-1, first half)             */
#define SD_PASS_FWD_X 2   /* forward FFT along x, N of n modes kept           */
#define SD_PASS_FWD_Y 3   /* forward FFT along y (3D)                         */
#define SD_PASS_FUSED 4   /* last axis: forward FFT, product, inverse FFT     */
#define SD_PASS_INV_Y 5   /* inverse FFT along y (3D)                         */
#define SD_PASS_INV_X 6   /* inverse FFT along x with argmax (or the map)     */
#define SD_PASS_REDUCE 7  /* per-rotation argmax reduction                    */
#define SD_PASS_GRAPH 8   /* one replay of a captured search graph            */
#define SD_PASS_SPREAD_X 9  /* rotate + spread fused with the forward x FFT   */
#define SD_PASS_INV_YX 10   /* inverse y and x of whole z-planes in clusters  */
#define SD_PASS_COUNT 11

/* With the context option "timing" = 1, every pass launch of the search is
 * bracketed by CUDA events on its stream; a search replayed from a captured
 * graph (option "graph") carries those events as event-record nodes of the
 * graph, and each replay's times are read back before the graph's next replay
 * (the graph is captured separately with and without timing).  Returns the
 * number of timed launches and their summed device time (ms) for `kind`;
 * synchronises on the recorded events.  kind < 0 resets the totals. */
int sd_pass_times(sd_ctx* ctx, int kind, int64_t* launches, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* SDFDOCK_H */
