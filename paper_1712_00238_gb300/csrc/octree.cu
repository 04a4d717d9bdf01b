// Adaptive octree (quadtree in 2D) of SDF sample cells (Section 5).
//
// Section 5 notes that the skeletal density varies most near the skeleton and
// proposes sampling it on a tree subdivided deepest there, feeding the
// nonequispaced samples to a nonequispaced FFT.  The tree is built here on the
// host, one level at a time: cells whose centre lies within half a diagonal of
// the nearest boundary sample are split outright; the others ask the caller for
// rho at their centres (evaluated on the device by sd_sdf_build) and are split
// when their weight |rho| h^d reaches tau.  Leaves become the SDF samples;
// optionally only those within a band around the boundary.
//
// Nearest boundary distances come from a uniform bucket grid over the boundary
// samples searched in growing Chebyshev shells, exact below the radius a level
// needs.  Cells of a level are kept as sorted linear keys
// k_x + 2^D (k_y + 2^D k_z), which is also the order leaves are listed in.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "../../include/sdfdock.h"

namespace {

constexpr int kMaxDepth = 20;
constexpr int kMaxCellsLog2 = 27;
constexpr int64_t kMaxCells = int64_t(1) << kMaxCellsLog2;  // cells of one level

struct BucketGrid {
    int dim = 3;
    double lo[3] = {0, 0, 0};
    double b = 1.0;
    int64_t g[3] = {1, 1, 1};
    std::vector<int64_t> start;  // bucket b holds pts[start[b] .. start[b+1])
    std::vector<double> pts;     // 3 per sample, grouped by bucket

    int64_t flat(const int64_t* j) const { return j[0] + g[0] * (j[1] + g[1] * j[2]); }

    void build(const double* bnd, int64_t n, int d) {
        dim = d;
        double hi[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) lo[a] = hi[a] = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < dim; ++a) {
                const double x = bnd[4 * i + a];
                if (i == 0 || x < lo[a]) lo[a] = x;
                if (i == 0 || x > hi[a]) hi[a] = x;
            }
        double ext = 0.0;
        for (int a = 0; a < dim; ++a) ext = std::max(ext, hi[a] - lo[a]);
        // about 4 n buckets over the box: a few samples per bucket on a surface
        const double side = std::max(1.0, std::floor(std::pow(4.0 * (double)std::max<int64_t>(n, 1), 1.0 / dim)));
        b = ext > 0.0 ? ext / side : 1.0;
        for (int a = 0; a < 3; ++a) g[a] = a < dim ? (int64_t)std::floor((hi[a] - lo[a]) / b) + 1 : 1;
        const int64_t nb = g[0] * g[1] * g[2];
        std::vector<int64_t> idx((size_t)n);
        start.assign((size_t)nb + 1, 0);
        for (int64_t i = 0; i < n; ++i) {
            int64_t j[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a)
                j[a] = std::min(g[a] - 1, std::max<int64_t>(0, (int64_t)std::floor((bnd[4 * i + a] - lo[a]) / b)));
            idx[(size_t)i] = flat(j);
            ++start[(size_t)idx[(size_t)i] + 1];
        }
        for (int64_t k = 0; k < nb; ++k) start[(size_t)k + 1] += start[(size_t)k];
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        pts.assign((size_t)n * 3, 0.0);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t at = fill[(size_t)idx[(size_t)i]]++;
            for (int a = 0; a < dim; ++a) pts[(size_t)(3 * at + a)] = bnd[4 * i + a];
        }
    }

    // distance from p to the nearest sample; exact when it is below `cap`,
    // otherwise some value >= cap (infinity when there are no samples)
    double nearest(const double* p, double cap) const {
        if (pts.empty()) return INFINITY;
        int64_t kp[3] = {0, 0, 0};
        int64_t s0 = 0, smax = 0;
        for (int a = 0; a < dim; ++a) {
            const double f = std::floor((p[a] - lo[a]) / b);
            kp[a] = (int64_t)std::max(-1e15, std::min(1e15, f));
            s0 = std::max(s0, std::max(-kp[a], kp[a] - (g[a] - 1)));
            smax = std::max(smax, std::max(kp[a], g[a] - 1 - kp[a]));
        }
        double best2 = INFINITY;
        for (int64_t s = s0; s <= smax; ++s) {
            // samples in shells >= s lie at least (s - 1) b away
            if (s >= 1) {
                const double lim = (double)(s - 1) * b;
                if (best2 <= lim * lim || lim >= cap) break;
            }
            int64_t jlo[3] = {0, 0, 0}, jhi[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) {
                jlo[a] = std::max<int64_t>(0, kp[a] - s);
                jhi[a] = std::min<int64_t>(g[a] - 1, kp[a] + s);
            }
            int64_t j[3];
            for (j[2] = jlo[2]; j[2] <= jhi[2]; ++j[2])
                for (j[1] = jlo[1]; j[1] <= jhi[1]; ++j[1])
                    for (j[0] = jlo[0]; j[0] <= jhi[0]; ++j[0]) {
                        int64_t cheb = 0;
                        for (int a = 0; a < dim; ++a) cheb = std::max(cheb, j[a] > kp[a] ? j[a] - kp[a] : kp[a] - j[a]);
                        if (cheb != s) {
                            // interior of the shell: jump to its far face along x
                            if (j[0] > kp[0] - s && j[0] < kp[0] + s && cheb < s) j[0] = std::max(j[0], kp[0] + s - 1);
                            continue;
                        }
                        const int64_t f = flat(j);
                        for (int64_t i = start[(size_t)f]; i < start[(size_t)f + 1]; ++i) {
                            double d2 = 0.0;
                            for (int a = 0; a < dim; ++a) {
                                const double d = p[a] - pts[(size_t)(3 * i + a)];
                                d2 += d * d;
                            }
                            best2 = std::min(best2, d2);
                        }
                    }
        }
        return std::sqrt(best2);
    }
};

}  // namespace

struct sd_octree {
    int dim = 3, d_min = 0, d_max = 0, D = 0;
    double lo[3] = {0, 0, 0};
    double size = 1.0, tau = 0.0, clear = 0.0, band = INFINITY;
    bool done = false, failed = false;
    BucketGrid grid;
    std::vector<int64_t> keys;   // cells of level D, sorted
    std::vector<double> xi;      // nearest boundary distance per cell
    std::vector<uint8_t> split;  // split decision per cell
    std::vector<uint8_t> beyond; // cell lies wholly beyond the band
    std::vector<int64_t> ask;    // cells of level D that need rho
    std::vector<double> leaf_c, leaf_v;
    std::vector<int32_t> leaf_k;

    double side() const { return size / (double)(int64_t(1) << D); }

    void coords(int64_t key, int64_t* k) const {
        const int64_t m = (int64_t(1) << D) - 1;
        k[0] = key & m;
        k[1] = dim > 1 ? (key >> D) & m : 0;
        k[2] = dim > 2 ? (key >> (2 * D)) : 0;
    }

    void centre(int64_t key, double* c) const {
        int64_t k[3];
        coords(key, k);
        const double h = side();
        for (int a = 0; a < 3; ++a) c[a] = a < dim ? lo[a] + ((double)k[a] + 0.5) * h : 0.0;
    }

    // distances, outright splits and cells beyond the band of the current level;
    // records which cells need rho.  The distance to the boundary is 1-Lipschitz,
    // so a cell whose centre lies farther than band + r holds no point within the band.
    void examine() {
        const double h = side();
        const double r = 0.5 * h * std::sqrt((double)dim);
        double cap = std::max(r, clear);
        if (std::isfinite(band)) cap = std::max(cap, band + r);
        cap = cap * (1.0 + 1e-12) + 1e-300;
        xi.assign(keys.size(), 0.0);
        split.assign(keys.size(), 0);
        beyond.assign(keys.size(), 0);
        ask.clear();
        for (size_t i = 0; i < keys.size(); ++i) {
            double c[3];
            centre(keys[i], c);
            xi[i] = grid.nearest(c, cap);
            beyond[i] = xi[i] - r > band ? 1 : 0;
            if (D < d_max) {
                if (xi[i] < r)
                    split[i] = 1;
                else if (!beyond[i])
                    ask.push_back((int64_t)i);
            }
        }
    }

    // emit the level's leaves and move to the children of its split cells
    int advance() {
        const double h = side();
        const double v = std::pow(h, (double)dim);
        int64_t n_split = 0;
        for (size_t i = 0; i < keys.size(); ++i) {
            if (split[i]) {
                ++n_split;
                continue;
            }
            if (beyond[i] || !(xi[i] >= clear) || !(xi[i] <= band)) continue;
            double c[3];
            centre(keys[i], c);
            int64_t k[3];
            coords(keys[i], k);
            leaf_c.insert(leaf_c.end(), {c[0], c[1], c[2], 0.0});
            leaf_v.push_back(v);
            leaf_k.insert(leaf_k.end(), {(int32_t)k[0], (int32_t)k[1], (int32_t)k[2], (int32_t)D});
        }
        if (n_split == 0 || D == d_max) {
            keys.clear();
            done = true;
            return SD_OK;
        }
        if (n_split > (kMaxCells >> dim)) return SD_ERR_OOM;
        std::vector<int64_t> next;
        next.reserve((size_t)(n_split << dim));
        const int D1 = D + 1;
        for (size_t i = 0; i < keys.size(); ++i) {
            if (!split[i]) continue;
            int64_t k[3];
            coords(keys[i], k);
            for (int o = 0; o < (1 << dim); ++o) {
                int64_t key = 0;
                for (int a = dim - 1; a >= 0; --a) key = (key << D1) | (2 * k[a] + ((o >> a) & 1));
                next.push_back(key);
            }
        }
        std::sort(next.begin(), next.end());
        keys.swap(next);
        D = D1;
        return SD_OK;
    }

    // examine levels until one needs rho or the tree is complete
    int settle() {
        while (!done) {
            examine();
            if (!ask.empty()) return SD_OK;
            const int rc = advance();
            if (rc != SD_OK) return rc;
        }
        return SD_OK;
    }
};

extern "C" {

int sd_octree_create(int dim, const double* bnd, int64_t n_b, const double* lo, double size, int depth_min,
                     int depth_max, double tau, double clearance, double band, sd_octree** out) {
    if (!out) return SD_ERR_ARG;
    *out = nullptr;
    if ((dim != 2 && dim != 3) || n_b < 0 || (n_b > 0 && !bnd) || !lo) return SD_ERR_ARG;
    if (!(size > 0.0) || !std::isfinite(size) || !(tau >= 0.0) || !(clearance >= 0.0) || !std::isfinite(clearance) ||
        !(band >= 0.0))
        return SD_ERR_ARG;
    if (depth_min < 0 || depth_max < depth_min || depth_max > kMaxDepth) return SD_ERR_ARG;
    if ((int64_t)depth_min * dim > kMaxCellsLog2) return SD_ERR_OOM;
    for (int a = 0; a < dim; ++a)
        if (!std::isfinite(lo[a])) return SD_ERR_ARG;
    for (int64_t i = 0; i < n_b; ++i)
        for (int a = 0; a < dim; ++a)
            if (!std::isfinite(bnd[4 * i + a])) return SD_ERR_NONFINITE;
    try {
        std::unique_ptr<sd_octree> t(new sd_octree());
        t->dim = dim;
        t->d_min = depth_min;
        t->d_max = depth_max;
        t->D = depth_min;
        for (int a = 0; a < 3; ++a) t->lo[a] = a < dim ? lo[a] : 0.0;
        t->size = size;
        t->tau = tau;
        t->clear = clearance;
        t->band = band;
        t->grid.build(bnd, n_b, dim);
        const int64_t n0 = int64_t(1) << (depth_min * dim);
        t->keys.resize((size_t)n0);
        for (int64_t i = 0; i < n0; ++i) t->keys[(size_t)i] = i;  // the uniform level is already in key order
        const int rc = t->settle();
        if (rc != SD_OK) return rc;
        *out = t.release();
        return SD_OK;
    } catch (const std::bad_alloc&) {
        return SD_ERR_OOM;
    }
}

int sd_octree_pending(const sd_octree* t, int64_t* n, double* centres, double* vol) {
    if (!t || !n) return SD_ERR_ARG;
    if (t->failed) return SD_ERR_ARG;
    *n = t->done ? 0 : (int64_t)t->ask.size();
    if (t->done) return SD_OK;
    const double v = std::pow(t->side(), (double)t->dim);
    for (size_t j = 0; j < t->ask.size(); ++j) {
        if (centres) {
            t->centre(t->keys[(size_t)t->ask[j]], centres + 4 * j);
            centres[4 * j + 3] = 0.0;
        }
        if (vol) vol[j] = v;
    }
    return SD_OK;
}

int sd_octree_feed(sd_octree* t, const double* rho, int64_t n) {
    if (!t || t->failed || t->done) return SD_ERR_ARG;
    if (n != (int64_t)t->ask.size() || (n > 0 && !rho)) return SD_ERR_ARG;
    for (int64_t j = 0; j < n; ++j)
        if (!std::isfinite(rho[2 * j]) || !std::isfinite(rho[2 * j + 1])) return SD_ERR_NONFINITE;
    const double v = std::pow(t->side(), (double)t->dim);
    for (int64_t j = 0; j < n; ++j)
        t->split[(size_t)t->ask[(size_t)j]] = std::hypot(rho[2 * j], rho[2 * j + 1]) * v >= t->tau ? 1 : 0;
    try {
        int rc = t->advance();
        if (rc == SD_OK) rc = t->settle();
        if (rc != SD_OK) t->failed = true;
        return rc;
    } catch (const std::bad_alloc&) {
        t->failed = true;
        return SD_ERR_OOM;
    }
}

int sd_octree_leaves(const sd_octree* t, int64_t* m, double* centres, double* vol, int32_t* coords) {
    if (!t || !m || t->failed) return SD_ERR_ARG;
    if (!t->done) return SD_ERR_ARG;
    const size_t n = t->leaf_v.size();
    *m = (int64_t)n;
    if (centres && n) std::memcpy(centres, t->leaf_c.data(), n * 4 * sizeof(double));
    if (vol && n) std::memcpy(vol, t->leaf_v.data(), n * sizeof(double));
    if (coords && n) std::memcpy(coords, t->leaf_k.data(), n * 4 * sizeof(int32_t));
    return SD_OK;
}

int sd_octree_free(sd_octree* t) {
    delete t;
    return SD_OK;
}

}  // extern "C"
