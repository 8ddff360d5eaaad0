// FP64 CPU oracle for the SPH neighbour search and the density / hydro-force loops.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call, link or
// load this file: only the tests, the package's smoke check and the CPU-baseline arm
// of the benchmark use it.  It shares no code, header or table with the CUDA path.
//
// Everything here is the plain definition, in FP64, compiled with -ffp-contract=off so
// that every product and sum is rounded exactly as written:
//
//  * Peano-Hilbert keys (Sec. 1: Gadget3 orders particles along the Hilbert curve;
//    the curve variant is not stated, the reading taken is Skilling's transpose
//    construction, "Programming the Hilbert curve", AIP Conf. Proc. 707 (2004), on a
//    2^21 grid per axis, axis order x, y, z, interleaved most significant bit first).
//  * stable order by key (ties keep the input order).
//  * neighbour sets (Sec. 1.1): density  N_i = { j : |r_ij| < h_i },
//                               hydro    N_i = { j : |r_ij| < max(h_i, h_j) },
//    minimum-image distances in the periodic unit cube, r^2 = dx*dx + dy*dy + dz*dz.
//  * M4 cubic-spline kernel with compact support h (the paper fixes no kernel; this is
//    the Gadget convention), the SPH density with its h-derivative, the grad-h
//    correction f_i, and the smoothing-length iteration to a fixed effective
//    neighbour number N_ngb = 4 pi rho h^3 / (3 m) (Sec. 2.2, the relation above Eq. 1).
//  * SPH hydro accelerations and du/dt (grad-h pressure term plus Monaghan
//    artificial viscosity, optionally limited by Balsara's switch); the paper only
//    cites its hydro scheme, the reading is the standard energy-conserving form.
//  * velocity divergence and curl over the density sets (no formula in the paper; the
//    standard SPH estimates from the velocity gradient at h_i).
//  * the backward (adjoint) of the density and the accelerations with respect to
//    positions, velocities and masses, h tied to them by the neighbour-number relation
//    (the paper has no backward pass), and a forward-mode dual-number check of it.
//
// A pointer octree is used only to prune the candidate set; every candidate is still
// tested with the exact definition above, and the pruned sets are pinned against the
// brute-force O(N^2) sets in the tests.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -pthread

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <limits>
#include <thread>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;

int n_threads() {
    const char* e = std::getenv("ORACLE_THREADS");
    if (e && std::atoi(e) > 0) return std::atoi(e);
    unsigned t = std::thread::hardware_concurrency();
    return t ? (int)t : 1;
}

// Runs body(i) for i in [0, n) on a pool of threads, dynamic chunks.
template <class F>
void parallel_for(int64_t n, F body) {
    int nt = n_threads();
    if (n < 64 || nt == 1) {
        for (int64_t i = 0; i < n; ++i) body(i);
        return;
    }
    std::atomic<int64_t> next{0};
    const int64_t chunk = 16;
    auto work = [&]() {
        for (;;) {
            int64_t b = next.fetch_add(chunk);
            if (b >= n) break;
            int64_t e = std::min(n, b + chunk);
            for (int64_t i = b; i < e; ++i) body(i);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) pool.emplace_back(work);
    for (auto& th : pool) th.join();
}

// ---------------------------------------------------------------------------------
// Peano-Hilbert index of a cell of a 2^bits grid (Skilling's construction).
// The coordinates are first brought into "transposed Hilbert" form, level by level
// from the coarsest bit: at each level Q, for every axis a, if bit Q of axis a is set
// the lower bits of axis 0 are complemented, otherwise the lower bits of axis 0 and
// axis a are exchanged.  A Gray code along the axes follows, then a common correction
// mask.  The index bits are the transposed coordinates read level by level, axis 0
// most significant.
uint64_t hilbert_index(uint32_t cx, uint32_t cy, uint32_t cz, int bits) {
    uint32_t a[3] = {cx, cy, cz};
    const uint32_t top = 1u << (bits - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        const uint32_t below = q - 1;
        for (int ax = 0; ax < 3; ++ax) {
            if (a[ax] & q) {
                a[0] ^= below;
            } else {
                uint32_t diff = (a[0] ^ a[ax]) & below;
                a[0] ^= diff;
                a[ax] ^= diff;
            }
        }
    }
    for (int ax = 1; ax < 3; ++ax) a[ax] ^= a[ax - 1];
    uint32_t fix = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (a[2] & q) fix ^= (q - 1);
    for (int ax = 0; ax < 3; ++ax) a[ax] ^= fix;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b) {
        key = (key << 3) | ((uint64_t)((a[0] >> b) & 1u) << 2) |
              ((uint64_t)((a[1] >> b) & 1u) << 1) | (uint64_t)((a[2] >> b) & 1u);
    }
    return key;
}

constexpr int kKeyBits = 21;

uint32_t grid_cell(double x) {
    // x is in [0, 1); x * 2^21 is exact, floor is exact.
    double s = std::floor(x * 2097152.0);
    if (s < 0.0) s = 0.0;
    if (s > 2097151.0) s = 2097151.0;
    return (uint32_t)s;
}

// ---------------------------------------------------------------------------------
// Distances in the periodic unit cube.  d = x_j - x_i, brought to the nearest image
// with round-half-even (so that d_ij == -d_ji bit for bit).
inline double min_image(double d) { return d - std::nearbyint(d); }

inline double dist2(const double* x, const double* y, const double* z, int64_t i, int64_t j,
                    double& dx, double& dy, double& dz) {
    dx = min_image(x[j] - x[i]);
    dy = min_image(y[j] - y[i]);
    dz = min_image(z[j] - z[i]);
    double sx = dx * dx;
    double sy = dy * dy;
    double sz = dz * dz;
    return (sx + sy) + sz;
}

// ---------------------------------------------------------------------------------
// M4 cubic spline with support radius h:
//   W(r,h) = 8/(pi h^3) * { 1 - 6 q^2 + 6 q^3      0   <= q <= 1/2
//                         { 2 (1 - q)^3           1/2 <  q <= 1
//                         { 0                     q > 1,          q = r / h.
// dW/dr and dW/dh = -(3 W + r dW/dr) / h follow by differentiation.
void m4_kernel(double r, double h, double& w, double& dwdr) {
    double q = r / h;
    double sigma = 8.0 / (kPi * h * h * h);
    if (q <= 0.5) {
        w = sigma * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
        dwdr = sigma / h * (-12.0 * q + 18.0 * q * q);
    } else if (q <= 1.0) {
        double u = 1.0 - q;
        w = sigma * 2.0 * u * u * u;
        dwdr = sigma / h * (-6.0 * u * u);
    } else {
        w = 0.0;
        dwdr = 0.0;
    }
}

// ---------------------------------------------------------------------------------
// Pruning octree (an accelerator only; correctness comes from the exact test).
struct Tree {
    struct Node {
        double lo[3], hi[3];
        double hmax;
        int32_t first, count;
        int32_t child[8];
        int nchild;
    };
    std::vector<Node> nodes;
    std::vector<int32_t> order;
};

constexpr int kLeafMax = 16;

void build_node(Tree& t, const double* x, const double* y, const double* z, const double* h,
                int32_t first, int32_t count, double cx, double cy, double cz, double half,
                int depth, std::vector<int32_t>& scratch) {
    int idx = (int)t.nodes.size();
    t.nodes.push_back(Tree::Node());
    Tree::Node nd;
    nd.first = first;
    nd.count = count;
    nd.nchild = 0;
    nd.hmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        nd.lo[a] = std::numeric_limits<double>::infinity();
        nd.hi[a] = -std::numeric_limits<double>::infinity();
    }
    for (int32_t k = first; k < first + count; ++k) {
        int32_t p = t.order[k];
        double c[3] = {x[p], y[p], z[p]};
        for (int a = 0; a < 3; ++a) {
            nd.lo[a] = std::min(nd.lo[a], c[a]);
            nd.hi[a] = std::max(nd.hi[a], c[a]);
        }
        if (h) nd.hmax = std::max(nd.hmax, h[p]);
    }
    if (count > kLeafMax && depth < 48) {
        // split the range into the 8 octants of the cell
        int32_t cnt[8] = {0};
        auto octant = [&](int32_t p) {
            return (x[p] >= cx ? 1 : 0) | (y[p] >= cy ? 2 : 0) | (z[p] >= cz ? 4 : 0);
        };
        for (int32_t k = first; k < first + count; ++k) cnt[octant(t.order[k])]++;
        int32_t start[8];
        int32_t s = first;
        for (int o = 0; o < 8; ++o) { start[o] = s; s += cnt[o]; }
        int32_t fill[8];
        for (int o = 0; o < 8; ++o) fill[o] = start[o];
        scratch.resize(count);
        for (int32_t k = first; k < first + count; ++k) {
            int32_t p = t.order[k];
            scratch[fill[octant(p)]++ - first] = p;
        }
        for (int32_t k = 0; k < count; ++k) t.order[first + k] = scratch[k];
        double q = half * 0.5;
        for (int o = 0; o < 8; ++o) {
            if (cnt[o] == 0) continue;
            double ox = cx + ((o & 1) ? q : -q);
            double oy = cy + ((o & 2) ? q : -q);
            double oz = cz + ((o & 4) ? q : -q);
            int child = (int)t.nodes.size();
            nd.child[nd.nchild++] = child;
            build_node(t, x, y, z, h, start[o], cnt[o], ox, oy, oz, q, depth + 1, scratch);
        }
    }
    t.nodes[idx] = nd;
}

void build_tree(Tree& t, int64_t n, const double* x, const double* y, const double* z,
                const double* h) {
    t.nodes.clear();
    t.order.resize(n);
    for (int64_t i = 0; i < n; ++i) t.order[i] = (int32_t)i;
    std::vector<int32_t> scratch;
    if (n > 0) build_node(t, x, y, z, h, 0, (int32_t)n, 0.5, 0.5, 0.5, 0.5, 0, scratch);
}

// squared periodic distance from a point to an axis-aligned box inside the unit cube
double box_dist2(const double p[3], const double lo[3], const double hi[3]) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double best = std::numeric_limits<double>::infinity();
        for (int sh = -1; sh <= 1; ++sh) {
            double q = p[a] + (double)sh;
            double d = std::max(0.0, std::max(lo[a] - q, q - hi[a]));
            best = std::min(best, d);
        }
        s += best * best;
    }
    return s;
}

// All particles in leaves whose box lies within the opening radius of p.  With
// use_hmax the radius of a node is max(radius, node hmax) (the hydro criterion).
void tree_candidates(const Tree& t, const double p[3], double radius, bool use_hmax,
                     std::vector<int32_t>& out) {
    out.clear();
    if (t.nodes.empty()) return;
    std::vector<int32_t> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        const Tree::Node& nd = t.nodes[stack.back()];
        stack.pop_back();
        double r = use_hmax ? std::max(radius, nd.hmax) : radius;
        double lim = r * r * (1.0 + 1e-9) + 1e-300;
        if (box_dist2(p, nd.lo, nd.hi) > lim) continue;
        if (nd.nchild == 0) {
            for (int32_t k = nd.first; k < nd.first + nd.count; ++k) out.push_back(t.order[k]);
        } else {
            for (int c = 0; c < nd.nchild; ++c) stack.push_back(nd.child[c]);
        }
    }
}

struct Particles {
    int64_t n;
    const double *x, *y, *z;
};

// Neighbour indices of target i, ascending.  kind 0 = density, 1 = hydro.
void neighbours(const Particles& P, const double* h, const Tree* tree, int64_t i, int kind,
                std::vector<int32_t>& cand, std::vector<int32_t>& out) {
    out.clear();
    double hi2 = h[i] * h[i];
    auto test = [&](int64_t j) {
        double dx, dy, dz;
        double r2 = dist2(P.x, P.y, P.z, i, j, dx, dy, dz);
        if (kind == 0) return r2 < hi2;
        if (j == i) return false;
        double hj2 = h[j] * h[j];
        return r2 < std::max(hi2, hj2);
    };
    if (tree) {
        double p[3] = {P.x[i], P.y[i], P.z[i]};
        tree_candidates(*tree, p, h[i], kind == 1, cand);
        for (int32_t j : cand)
            if (test(j)) out.push_back(j);
        std::sort(out.begin(), out.end());
    } else {
        for (int64_t j = 0; j < P.n; ++j)
            if (test(j)) out.push_back((int32_t)j);
    }
}

struct DensityOut {
    double rho, drhodh;
    int32_t n;
};

// Grouped search (Sec. 2.1, Neighbour Recycling): the members of a group share one
// tree walk around a centre c, the group's first member as in the paper.  Density:
// every neighbour j of member k has |x_j - c| <= |x_j - x_k| + |x_k - c| < h_k + d_k
// with d_k = |x_k - c|, so the walk radius R = max_k (d_k + h_k) covers every member's
// sphere.  Hydro: j is a neighbour of k through max(h_k, h_j), so the walk opens a node
// when its box is within R_g + max(hmax_g, node hmax), R_g = max_k d_k,
// hmax_g = max_k h_k.  Every member then applies its own exact test to the superset.
double periodic_dist(const Particles& P, int64_t a, int64_t b) {
    double dx, dy, dz;
    return std::sqrt(dist2(P.x, P.y, P.z, a, b, dx, dy, dz));
}

void tree_candidates_sym(const Tree& t, const double p[3], double rg, double hmax_g,
                         std::vector<int32_t>& out) {
    out.clear();
    if (t.nodes.empty()) return;
    std::vector<int32_t> stack;
    stack.push_back(0);
    while (!stack.empty()) {
        const Tree::Node& nd = t.nodes[stack.back()];
        stack.pop_back();
        double r = rg + std::max(hmax_g, nd.hmax);
        double lim = r * r * (1.0 + 1e-9) + 1e-300;
        if (box_dist2(p, nd.lo, nd.hi) > lim) continue;
        if (nd.nchild == 0) {
            for (int32_t k = nd.first; k < nd.first + nd.count; ++k) out.push_back(t.order[k]);
        } else {
            for (int c = 0; c < nd.nchild; ++c) stack.push_back(nd.child[c]);
        }
    }
}

// The superset of the group members[0 .. cnt) (kind 0 density, 1 hydro).
void group_superset(const Tree& t, const Particles& P, const double* h, const int32_t* members, int cnt,
                    int kind, std::vector<int32_t>& cand) {
    const int64_t c = members[0];
    const double p[3] = {P.x[c], P.y[c], P.z[c]};
    double rs = 0.0, rg = 0.0, hmax_g = 0.0;
    for (int k = 0; k < cnt; ++k) {
        const double d = periodic_dist(P, c, members[k]);
        rs = std::max(rs, d + h[members[k]]);
        rg = std::max(rg, d);
        hmax_g = std::max(hmax_g, h[members[k]]);
    }
    if (kind == 0) tree_candidates(t, p, rs, false, cand);
    else tree_candidates_sym(t, p, rg, hmax_g, cand);
}

// Member i's own neighbours among the candidates (the same test as the per-particle
// search), ascending.
void filter_superset(const Particles& P, const double* h, int64_t i, int kind, const std::vector<int32_t>& cand,
                     std::vector<int32_t>& out) {
    out.clear();
    const double hi2 = h[i] * h[i];
    for (int32_t j : cand) {
        double dx, dy, dz;
        const double r2 = dist2(P.x, P.y, P.z, i, j, dx, dy, dz);
        if (kind == 0) {
            if (r2 < hi2) out.push_back(j);
        } else if (j != i && r2 < std::max(hi2, h[j] * h[j])) {
            out.push_back(j);
        }
    }
    std::sort(out.begin(), out.end());
}

// rho_i and dRho_i/dh_i over the neighbour list nb (ascending indices), in that order
DensityOut density_sum(const Particles& P, const double* m, double hi, int64_t i,
                       const std::vector<int32_t>& nb) {
    DensityOut o{0.0, 0.0, (int32_t)nb.size()};
    for (int32_t j : nb) {
        double dx, dy, dz;
        double r = std::sqrt(dist2(P.x, P.y, P.z, i, j, dx, dy, dz));
        double w, dwdr;
        m4_kernel(r, hi, w, dwdr);
        o.rho += m[j] * w;
        o.drhodh += m[j] * (-(3.0 * w + r * dwdr) / hi);
    }
    return o;
}

DensityOut density_at(const Particles& P, const double* m, double hi, const Tree* tree,
                      int64_t i, std::vector<int32_t>& cand, std::vector<int32_t>& nb) {
    nb.clear();
    double hi2 = hi * hi;
    if (tree) {
        double p[3] = {P.x[i], P.y[i], P.z[i]};
        tree_candidates(*tree, p, hi, false, cand);
        for (int32_t j : cand) {
            double dx, dy, dz;
            if (dist2(P.x, P.y, P.z, i, j, dx, dy, dz) < hi2) nb.push_back(j);
        }
        std::sort(nb.begin(), nb.end());
    } else {
        for (int64_t j = 0; j < P.n; ++j) {
            double dx, dy, dz;
            if (dist2(P.x, P.y, P.z, i, j, dx, dy, dz) < hi2) nb.push_back((int32_t)j);
        }
    }
    return density_sum(P, m, hi, i, nb);
}

// Inputs of the hydro sums, indexed by particle.  fbal: the viscosity limiter of every
// particle (NULL: 1, the plain Monaghan viscosity).
struct HydroIn {
    const double *x, *y, *z, *vx, *vy, *vz, *m, *h, *rho, *fgrad, *u;
    double gamma, alpha, beta, eps;
    const double* fbal;
};

// a_i and du_i/dt over the hydro neighbour list nb (ascending indices), in that order.
void hydro_sum(const HydroIn& H, int64_t i, const std::vector<int32_t>& nb, double acc[3], double& du) {
    const double gamma = H.gamma, alpha = H.alpha, beta = H.beta, eps = H.eps;
    const double *x = H.x, *y = H.y, *z = H.z, *vx = H.vx, *vy = H.vy, *vz = H.vz;
    const double *m = H.m, *h = H.h, *rho = H.rho, *fgrad = H.fgrad, *u = H.u;
    double Pi = (gamma - 1.0) * rho[i] * u[i];
    double ci = std::sqrt(gamma * Pi / rho[i]);
    double Ai = fgrad[i] * Pi / (rho[i] * rho[i]);
    acc[0] = acc[1] = acc[2] = 0.0;
    du = 0.0;
    for (int32_t j : nb) {
        double dx, dy, dz;
        double r2 = dist2(x, y, z, i, j, dx, dy, dz);
        if (r2 == 0.0) continue;
        double r = std::sqrt(r2);
        double rij[3] = {-dx, -dy, -dz};
        double wi, dwi, wj, dwj;
        m4_kernel(r, h[i], wi, dwi);
        m4_kernel(r, h[j], wj, dwj);
        double Pj = (gamma - 1.0) * rho[j] * u[j];
        double cj = std::sqrt(gamma * Pj / rho[j]);
        double Aj = fgrad[j] * Pj / (rho[j] * rho[j]);
        double vij[3] = {vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]};
        double vr = vij[0] * rij[0] + vij[1] * rij[1] + vij[2] * rij[2];
        double visc = 0.0;
        if (vr < 0.0) {
            double hb = 0.5 * (h[i] + h[j]);
            double mu = hb * vr / (r2 + eps * hb * hb);
            double cb = 0.5 * (ci + cj);
            double rb = 0.5 * (rho[i] + rho[j]);
            visc = (-alpha * cb * mu + beta * mu * mu) / rb;
            if (H.fbal) visc *= 0.5 * (H.fbal[i] + H.fbal[j]);
        }
        double gi[3], gj[3], gb[3];
        for (int a = 0; a < 3; ++a) {
            gi[a] = dwi * rij[a] / r;
            gj[a] = dwj * rij[a] / r;
            gb[a] = 0.5 * (gi[a] + gj[a]);
        }
        for (int a = 0; a < 3; ++a) acc[a] -= m[j] * (Ai * gi[a] + Aj * gj[a] + visc * gb[a]);
        double vgi = vij[0] * gi[0] + vij[1] * gi[1] + vij[2] * gi[2];
        double vgb = vij[0] * gb[0] + vij[1] * gb[1] + vij[2] * gb[2];
        du += m[j] * (Ai * vgi + 0.5 * visc * vgb);
    }
}

double neff_of(double h, double rho, double m) { return 4.0 * kPi / 3.0 * h * h * h * rho / m; }
double fgrad_of(double h, double rho, double drhodh) {
    return 1.0 / (1.0 + h / (3.0 * rho) * drhodh);
}

}  // namespace

extern "C" {

// Keys of cells (for the tests on small grids): bits per axis <= 21.
int orc_hilbert_cells(int64_t n, const uint32_t* cx, const uint32_t* cy, const uint32_t* cz,
                      int bits, uint64_t* keys) {
    if (bits < 1 || bits > 21) return -1;
    for (int64_t i = 0; i < n; ++i) keys[i] = hilbert_index(cx[i], cy[i], cz[i], bits);
    return 0;
}

// 63-bit keys of positions in [0,1)^3 on the 2^21 grid.
int orc_hilbert_keys(int64_t n, const double* x, const double* y, const double* z,
                     uint64_t* keys) {
    for (int64_t i = 0; i < n; ++i) {
        if (!(x[i] >= 0.0 && x[i] < 1.0 && y[i] >= 0.0 && y[i] < 1.0 && z[i] >= 0.0 &&
              z[i] < 1.0))
            return -1;
        keys[i] = hilbert_index(grid_cell(x[i]), grid_cell(y[i]), grid_cell(z[i]), kKeyBits);
    }
    return 0;
}

// perm[r] = input index of the particle with rank r (stable by key).
int orc_stable_order(int64_t n, const uint64_t* keys, int32_t* perm) {
    std::vector<int32_t> p(n);
    for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
    std::stable_sort(p.begin(), p.end(), [&](int32_t a, int32_t b) { return keys[a] < keys[b]; });
    for (int64_t i = 0; i < n; ++i) perm[i] = p[i];
    return 0;
}

void orc_kernel(int64_t n, const double* r, const double* h, double* w, double* dwdr,
                double* dwdh) {
    for (int64_t i = 0; i < n; ++i) {
        double a, b;
        m4_kernel(r[i], h[i], a, b);
        w[i] = a;
        dwdr[i] = b;
        dwdh[i] = -(3.0 * a + r[i] * b) / h[i];
    }
}

// Minimum-image squared distances for index pairs (used by the symmetry tests).
void orc_pair_r2(int64_t n, const double* x, const double* y, const double* z, int64_t npairs,
                 const int32_t* pi, const int32_t* pj, double* r2) {
    (void)n;
    for (int64_t k = 0; k < npairs; ++k) {
        double dx, dy, dz;
        r2[k] = dist2(x, y, z, pi[k], pj[k], dx, dy, dz);
    }
}

// Neighbour sets of the targets.  With idx == nullptr only offsets are written
// (offsets[0] = 0, offsets[t+1] = offsets[t] + |N_t|); otherwise idx receives the
// ascending neighbour indices of every target at those offsets.
int orc_ngb_sets(int64_t n, const double* x, const double* y, const double* z,
                 const double* h, int kind, int64_t nt, const int32_t* targets, int use_tree,
                 int64_t* offsets, int32_t* idx) {
    Particles P{n, x, y, z};
    Tree tree;
    if (use_tree) build_tree(tree, n, x, y, z, h);
    std::vector<int64_t> cnt(nt, 0);
    std::vector<std::vector<int32_t>> lists(idx ? nt : 0);
    parallel_for(nt, [&](int64_t t) {
        std::vector<int32_t> cand, out;
        neighbours(P, h, use_tree ? &tree : nullptr, targets[t], kind, cand, out);
        cnt[t] = (int64_t)out.size();
        if (idx) lists[t] = out;
    });
    if (!idx) {
        offsets[0] = 0;
        for (int64_t t = 0; t < nt; ++t) offsets[t + 1] = offsets[t] + cnt[t];
    } else {
        for (int64_t t = 0; t < nt; ++t)
            std::copy(lists[t].begin(), lists[t].end(), idx + offsets[t]);
    }
    return 0;
}

// Density, dRho/dh, grad-h factor f, effective neighbour number and neighbour count of
// the targets at the given smoothing lengths (h is indexed by particle).
int orc_density(int64_t n, const double* x, const double* y, const double* z, const double* m,
                const double* h, int64_t nt, const int32_t* targets, int use_tree, double* rho,
                double* drhodh, double* fgrad, double* neff, int32_t* nngb) {
    Particles P{n, x, y, z};
    Tree tree;
    if (use_tree) build_tree(tree, n, x, y, z, nullptr);
    parallel_for(nt, [&](int64_t t) {
        std::vector<int32_t> cand, nb;
        int64_t i = targets[t];
        DensityOut o = density_at(P, m, h[i], use_tree ? &tree : nullptr, i, cand, nb);
        rho[t] = o.rho;
        drhodh[t] = o.drhodh;
        fgrad[t] = fgrad_of(h[i], o.rho, o.drhodh);
        neff[t] = neff_of(h[i], o.rho, m[i]);
        nngb[t] = o.n;
    });
    return 0;
}

// Smoothing-length iteration of every target to |N_eff - nngb| <= dn.  h (length n) is
// read as the initial guess and overwritten for the targets.  Per target: bracket
// [lo, hi) starting at (0, inf); each pass evaluates rho(h) and dRho/dh, stops when
// converged, otherwise narrows the bracket and takes the Newton step on
// g(h) = (4 pi / 3) h^3 rho(h) - nngb m; a step outside the bracket (or not finite)
// is replaced by a bisection in volume (h * 2^(1/3) or h / 2^(1/3) while one side is
// open, else the cube root of the mean of the bracket's cubes).
// Returns the number of targets that did not converge within max_iter passes.
int64_t orc_density_iterate(int64_t n, const double* x, const double* y, const double* z,
                            const double* m, double* h, int64_t nt, const int32_t* targets,
                            double nngb_target, double dn, int max_iter, int use_tree,
                            double* rho, double* drhodh, double* fgrad, double* neff,
                            int32_t* nngb, int32_t* iters) {
    Particles P{n, x, y, z};
    Tree tree;
    if (use_tree) build_tree(tree, n, x, y, z, nullptr);
    const double cbrt2 = 1.2599210498948731647672106;
    std::atomic<int64_t> failed{0};
    std::vector<double> hnew(nt);
    parallel_for(nt, [&](int64_t t) {
        std::vector<int32_t> cand, nb;
        int64_t i = targets[t];
        double hh = h[i];
        double lo = 0.0, hi = std::numeric_limits<double>::infinity();
        bool ok = false;
        DensityOut o{0, 0, 0};
        int it = 0;
        for (it = 1; it <= max_iter; ++it) {
            o = density_at(P, m, hh, use_tree ? &tree : nullptr, i, cand, nb);
            double ne = neff_of(hh, o.rho, m[i]);
            if (std::fabs(ne - nngb_target) <= dn) { ok = true; break; }
            if (it == max_iter) break;
            if (ne < nngb_target) lo = hh; else hi = hh;
            double g = 4.0 * kPi / 3.0 * hh * hh * hh * o.rho - nngb_target * m[i];
            double gp = 4.0 * kPi * hh * hh * o.rho + 4.0 * kPi / 3.0 * hh * hh * hh * o.drhodh;
            double hn = hh - g / gp;
            if (!(hn > lo && hn < hi) || !std::isfinite(hn)) {
                if (std::isinf(hi)) hn = hh * cbrt2;
                else if (lo == 0.0) hn = hh / cbrt2;
                else hn = std::cbrt(0.5 * (lo * lo * lo + hi * hi * hi));
            }
            hh = hn;
        }
        if (!ok) failed.fetch_add(1);
        hnew[t] = hh;
        rho[t] = o.rho;
        drhodh[t] = o.drhodh;
        fgrad[t] = fgrad_of(hh, o.rho, o.drhodh);
        neff[t] = neff_of(hh, o.rho, m[i]);
        nngb[t] = o.n;
        iters[t] = std::min(it, max_iter);
    });
    for (int64_t t = 0; t < nt; ++t) h[targets[t]] = hnew[t];
    return failed.load();
}

// Velocity divergence and curl of the targets over their density sets (the other
// quantities a Gadget density pass hands to the hydro loop; not in the paper).  With
// the SPH velocity gradient at h_i,
//   G_ab(i) = -(1 / rho_i) sum_{j in N_i} m_j (v_i - v_j)_a (grad_i W(r_ij, h_i))_b,
//   grad_i W = W'(r) (x_i - x_j) / r,
// the divergence is tr G and the curl is (G_zy - G_yz, G_xz - G_zx, G_yx - G_xy).
// A linear field v = A x gives G = c A with a scalar c near 1 on a uniform set.
int orc_velocity_derivs(int64_t n, const double* x, const double* y, const double* z, const double* vel,
                        const double* m, const double* h, const double* rho, int64_t nt,
                        const int32_t* targets, int use_tree, double* divv, double* curl) {
    Particles P{n, x, y, z};
    Tree tree;
    if (use_tree) build_tree(tree, n, x, y, z, nullptr);
    parallel_for(nt, [&](int64_t t) {
        std::vector<int32_t> cand, nb;
        const int64_t i = targets[t];
        density_at(P, m, h[i], use_tree ? &tree : nullptr, i, cand, nb);
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int32_t j : nb) {
            double dx, dy, dz;
            const double r2 = dist2(x, y, z, i, j, dx, dy, dz);
            if (r2 == 0.0) continue;
            const double r = std::sqrt(r2);
            double w, dwdr;
            m4_kernel(r, h[i], w, dwdr);
            const double g[3] = {-dx / r * dwdr, -dy / r * dwdr, -dz / r * dwdr};   // x_i - x_j = -d
            const double v[3] = {vel[3 * i] - vel[3 * j], vel[3 * i + 1] - vel[3 * j + 1],
                                 vel[3 * i + 2] - vel[3 * j + 2]};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) G[a][b] -= m[j] * v[a] * g[b];
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] /= rho[i];
        divv[t] = G[0][0] + G[1][1] + G[2][2];
        curl[3 * t] = G[2][1] - G[1][2];
        curl[3 * t + 1] = G[0][2] - G[2][0];
        curl[3 * t + 2] = G[1][0] - G[0][1];
    });
    return 0;
}

// SPH accelerations and du/dt of the targets.  Per-particle inputs are indexed by
// particle: positions, velocities, masses m, smoothing lengths h, densities rho,
// grad-h factors f, specific internal energies u.  P = (gamma - 1) rho u,
// c = sqrt(gamma P / rho).  For j in the hydro set of i (j != i):
//   a_i   -= m_j [ f_i P_i/rho_i^2 gW_i + f_j P_j/rho_j^2 gW_j + Pi_ij (gW_i + gW_j)/2 ]
//   du_i  += m_j [ f_i P_i/rho_i^2 v_ij . gW_i + Pi_ij v_ij . (gW_i + gW_j)/4 ]
// with gW_k = dW/dr(r, h_k) r_ij / r, r_ij = x_i - x_j, v_ij = v_i - v_j and the
// Monaghan viscosity Pi_ij = (-alpha cbar mu + beta mu^2) / rhobar for v_ij . r_ij < 0
// (else 0), mu = hbar v_ij.r_ij / (r^2 + eps hbar^2), bars = pair means.
// Coincident pairs (r = 0) contribute nothing (the kernel gradient vanishes there).
// With fbal (not NULL) the viscosity of every pair is scaled by the pair mean of the
// limiter, Pi_ij (fbal_i + fbal_j) / 2 (Balsara's switch; orc_balsara gives fbal).
int orc_hydro(int64_t n, const double* x, const double* y, const double* z,
              const double* vx, const double* vy, const double* vz, const double* m,
              const double* h, const double* rho, const double* fgrad, const double* u,
              int64_t nt, const int32_t* targets, double gamma, double alpha, double beta,
              double eps, int use_tree, double* ax, double* ay, double* az, double* dudt,
              int32_t* nngb, const double* fbal) {
    Particles P{n, x, y, z};
    const HydroIn H{x, y, z, vx, vy, vz, m, h, rho, fgrad, u, gamma, alpha, beta, eps, fbal};
    Tree tree;
    if (use_tree) build_tree(tree, n, x, y, z, h);
    parallel_for(nt, [&](int64_t t) {
        std::vector<int32_t> cand, nb;
        int64_t i = targets[t];
        neighbours(P, h, use_tree ? &tree : nullptr, i, 1, cand, nb);
        double acc[3];
        hydro_sum(H, i, nb, acc, dudt[t]);
        ax[t] = acc[0];
        ay[t] = acc[1];
        az[t] = acc[2];
        nngb[t] = (int32_t)nb.size();
    });
    return 0;
}

// Grouped density and hydro (Sec. 2.1): the targets, given in the order of the curve,
// are cut into groups of g consecutive entries; each group walks the tree once for its
// superset and each member filters it.  Outputs are indexed like the targets and are
// those of orc_density / orc_hydro bit for bit (same sets, same summation order).
// stats[0..2] = walks, candidates (sum of superset sizes), member x candidate tests.
int orc_density_grouped(int64_t n, const double* x, const double* y, const double* z, const double* m,
                        const double* h, int64_t nt, const int32_t* ordered, int g, double* rho,
                        double* drhodh, double* fgrad, double* neff, int32_t* nngb, int64_t* stats) {
    if (g < 1) return -1;
    Particles P{n, x, y, z};
    Tree tree;
    build_tree(tree, n, x, y, z, nullptr);
    const int64_t ngroups = (nt + g - 1) / g;
    std::atomic<int64_t> cands{0}, tests{0};
    parallel_for(ngroups, [&](int64_t G) {
        const int64_t b = G * g;
        const int cnt = (int)std::min<int64_t>(g, nt - b);
        std::vector<int32_t> cand, nb;
        group_superset(tree, P, h, ordered + b, cnt, 0, cand);
        cands.fetch_add((int64_t)cand.size());
        tests.fetch_add((int64_t)cand.size() * cnt);
        for (int k = 0; k < cnt; ++k) {
            const int64_t t = b + k, i = ordered[t];
            filter_superset(P, h, i, 0, cand, nb);
            const DensityOut o = density_sum(P, m, h[i], i, nb);
            rho[t] = o.rho;
            drhodh[t] = o.drhodh;
            fgrad[t] = fgrad_of(h[i], o.rho, o.drhodh);
            neff[t] = neff_of(h[i], o.rho, m[i]);
            nngb[t] = o.n;
        }
    });
    stats[0] = ngroups;
    stats[1] = cands.load();
    stats[2] = tests.load();
    return 0;
}

int orc_hydro_grouped(int64_t n, const double* x, const double* y, const double* z, const double* vx,
                      const double* vy, const double* vz, const double* m, const double* h, const double* rho,
                      const double* fgrad, const double* u, int64_t nt, const int32_t* ordered, int g,
                      double gamma, double alpha, double beta, double eps, double* ax, double* ay, double* az,
                      double* dudt, int32_t* nngb, int64_t* stats) {
    if (g < 1) return -1;
    Particles P{n, x, y, z};
    const HydroIn H{x, y, z, vx, vy, vz, m, h, rho, fgrad, u, gamma, alpha, beta, eps, nullptr};
    Tree tree;
    build_tree(tree, n, x, y, z, h);
    const int64_t ngroups = (nt + g - 1) / g;
    std::atomic<int64_t> cands{0}, tests{0};
    parallel_for(ngroups, [&](int64_t G) {
        const int64_t b = G * g;
        const int cnt = (int)std::min<int64_t>(g, nt - b);
        std::vector<int32_t> cand, nb;
        group_superset(tree, P, h, ordered + b, cnt, 1, cand);
        cands.fetch_add((int64_t)cand.size());
        tests.fetch_add((int64_t)cand.size() * cnt);
        for (int k = 0; k < cnt; ++k) {
            const int64_t t = b + k, i = ordered[t];
            filter_superset(P, h, i, 1, cand, nb);
            double acc[3];
            hydro_sum(H, i, nb, acc, dudt[t]);
            ax[t] = acc[0];
            ay[t] = acc[1];
            az[t] = acc[2];
            nngb[t] = (int32_t)nb.size();
        }
    });
    stats[0] = ngroups;
    stats[1] = cands.load();
    stats[2] = tests.load();
    return 0;
}

// Balsara's viscosity limiter of every particle from its velocity divergence and curl
// (Balsara 1995, in the form used with Gadget's SPH):
//   fbal_i = |div v_i| / (|div v_i| + |curl v_i| + 1e-4 c_i / h_i),
// c_i = sqrt(gamma (gamma - 1) u_i) the sound speed, h_i the smoothing length.  It is
// near 1 in compression (no curl) and near 0 in shear (no divergence).
int orc_balsara(int64_t n, const double* divv, const double* curl, const double* u, const double* h,
                double gamma, double* fbal) {
    for (int64_t i = 0; i < n; ++i) {
        const double c = std::sqrt(gamma * (gamma - 1.0) * u[i]);
        const double ad = std::fabs(divv[i]);
        const double ac = std::sqrt(curl[3 * i] * curl[3 * i] + curl[3 * i + 1] * curl[3 * i + 1] +
                                    curl[3 * i + 2] * curl[3 * i + 2]);
        fbal[i] = ad / (ad + ac + 1e-4 * c / h[i]);
    }
    return 0;
}

int orc_threads(void) { return n_threads(); }

}  // extern "C"

// =================================================================================
// Backward (adjoint) of L = sum_i w_i . a_i + sum_i s_i rho_i with respect to the
// positions, velocities and masses (the method's differentiated form; the paper has
// no backward pass).  Neighbour sets are those of the given state; the smoothing
// lengths are defined by the exact constraint G_i = (4 pi / 3) h_i^3 rho_i - N m_i = 0
// (solved here to |G| <= 1e-13 N m), so h_i(x, m) enters through the implicit
// function theorem; f_i enters through rho_i, dRho_i/dh_i and h_i.
// =================================================================================

namespace {

// M4 kernel with the derivatives the adjoint needs:
//   W, W_r, W_rr, W_h, W_rh, W_hh  (r = distance, h = support)
struct K2 { double w, wr, wrr, wh, wrh, whh; };

K2 m4_full(double r, double h) {
    K2 k{0, 0, 0, 0, 0, 0};
    double q = r / h;
    if (q >= 1.0) return k;
    double sigma = 8.0 / (kPi * h * h * h);
    double w, w1, w2;  // w(q), w'(q), w''(q)
    if (q <= 0.5) {
        w = 1.0 - 6.0 * q * q + 6.0 * q * q * q;
        w1 = -12.0 * q + 18.0 * q * q;
        w2 = -12.0 + 36.0 * q;
    } else {
        double u = 1.0 - q;
        w = 2.0 * u * u * u;
        w1 = -6.0 * u * u;
        w2 = 12.0 * u;
    }
    k.w = sigma * w;
    k.wr = sigma * w1 / h;
    k.wrr = sigma * w2 / (h * h);
    k.wh = -sigma / h * (3.0 * w + q * w1);
    k.wrh = -sigma / (h * h) * (4.0 * w1 + q * w2);
    k.whh = sigma / (h * h) * (12.0 * w + 8.0 * q * w1 + q * q * w2);
    return k;
}

struct PairList {
    std::vector<int64_t> off;
    std::vector<int32_t> idx;
};

// hydro neighbour lists of all particles (j != i, |r| < max(h_i, h_j)), ascending
PairList hydro_lists(const Particles& P, const double* h, bool use_tree) {
    Tree tree;
    if (use_tree) build_tree(tree, P.n, P.x, P.y, P.z, h);
    std::vector<std::vector<int32_t>> lists(P.n);
    parallel_for(P.n, [&](int64_t i) {
        std::vector<int32_t> cand, out;
        neighbours(P, h, use_tree ? &tree : nullptr, i, 1, cand, out);
        lists[i] = out;
    });
    PairList L;
    L.off.assign(P.n + 1, 0);
    for (int64_t i = 0; i < P.n; ++i) L.off[i + 1] = L.off[i] + (int64_t)lists[i].size();
    L.idx.resize(L.off[P.n]);
    for (int64_t i = 0; i < P.n; ++i) std::copy(lists[i].begin(), lists[i].end(), L.idx.begin() + L.off[i]);
    return L;
}

// rho, dRho/dh, d2Rho/dh2 at h_i over the density set (j with |r| < h_i, i included);
// every such j is i itself or in i's hydro list.
void density3(const Particles& P, const double* m, const double* h, const PairList& L, int64_t i,
              double& rho, double& rh, double& rhh) {
    K2 self = m4_full(0.0, h[i]);
    rho = m[i] * self.w;
    rh = m[i] * self.wh;
    rhh = m[i] * self.whh;
    for (int64_t e = L.off[i]; e < L.off[i + 1]; ++e) {
        int32_t j = L.idx[e];
        double dx, dy, dz;
        double r2 = dist2(P.x, P.y, P.z, i, j, dx, dy, dz);
        if (!(r2 < h[i] * h[i])) continue;
        K2 k = m4_full(std::sqrt(r2), h[i]);
        rho += m[j] * k.w;
        rh += m[j] * k.wh;
        rhh += m[j] * k.whh;
    }
}

// Newton on G(h) = (4 pi/3) h^3 rho(h) - N m at a fixed neighbour list (the lists of
// the given state; W and W_h vanish at the support edge, so the solution is smooth in
// the pair distances).
double solve_h_exact(const Particles& P, const double* m, double* h, const PairList& L, int64_t i,
                     double nngb) {
    double hh = h[i];
    for (int it = 0; it < 60; ++it) {
        double rho, rh, rhh;
        double saved = h[i];
        h[i] = hh;
        density3(P, m, h, L, i, rho, rh, rhh);
        h[i] = saved;
        double g = 4.0 * kPi / 3.0 * hh * hh * hh * rho - nngb * m[i];
        double gp = 4.0 * kPi * hh * hh * rho + 4.0 * kPi / 3.0 * hh * hh * hh * rh;
        double step = g / gp;
        hh -= step;
        if (std::fabs(step) <= 1e-15 * hh) break;
    }
    return hh;
}

}  // namespace

extern "C" {

// Solves the exact constraint for every particle, starting from h (overwritten),
// with the hydro neighbour lists of the starting h held fixed.
int orc_h_exact(int64_t n, const double* x, const double* y, const double* z, const double* m,
                double* h, double nngb, int use_tree) {
    Particles P{n, x, y, z};
    std::vector<double> out(n);
    // a few rounds: lists at the current h, exact solve, repeat until the lists hold
    for (int round = 0; round < 4; ++round) {
        PairList L = hydro_lists(P, h, use_tree != 0);
        parallel_for(n, [&](int64_t i) { out[i] = solve_h_exact(P, m, h, L, i, nngb); });
        for (int64_t i = 0; i < n; ++i) h[i] = out[i];
    }
    return 0;
}

// Loss and its gradient.  h: smoothing lengths satisfying the exact constraint (see
// orc_h_exact); w: n x 3 weights of the accelerations, s: n weights of the densities.
// Outputs: loss (scalar), gx (n x 3), gv (n x 3), gm (n).
int orc_loss_grad(int64_t n, const double* x, const double* y, const double* z, const double* vel,
                  const double* m, const double* u, const double* h, const double* w, const double* s,
                  double nngb, double gamma, double alpha, double beta, double eps, int use_tree,
                  double* loss, double* gx, double* gv, double* gm) {
    Particles P{n, x, y, z};
    PairList L = hydro_lists(P, h, use_tree != 0);
    std::vector<double> rho(n), rh(n), rhh(n), f(n), A(n), c(n);
    parallel_for(n, [&](int64_t i) {
        density3(P, m, h, L, i, rho[i], rh[i], rhh[i]);
        f[i] = 1.0 / (1.0 + h[i] * rh[i] / (3.0 * rho[i]));
        A[i] = f[i] * (gamma - 1.0) * u[i] / rho[i];
        c[i] = std::sqrt(gamma * (gamma - 1.0) * u[i]);
    });
    // forward accelerations (for the loss value)
    std::vector<double> lossi(n, 0.0);
    // adjoints
    std::vector<double> hb(n, 0.0), rb(n, 0.0), Ab(n, 0.0);
    parallel_for(n, [&](int64_t k) {
        double acc[3] = {0, 0, 0}, xb[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
        double mb = 0.0, hbk = 0.0, rbk = 0.0, Abk = 0.0;
        const double* wk = w + 3 * k;
        for (int64_t e = L.off[k]; e < L.off[k + 1]; ++e) {
            int32_t j = L.idx[e];
            double dx, dy, dz;
            double r2 = dist2(x, y, z, k, j, dx, dy, dz);
            if (r2 == 0.0) continue;
            double r = std::sqrt(r2);
            double D[3] = {-dx, -dy, -dz};  // x_k - x_j
            double rhat[3] = {D[0] / r, D[1] / r, D[2] / r};
            K2 kk = m4_full(r, h[k]), kj = m4_full(r, h[j]);
            double v[3] = {vel[3 * k] - vel[3 * j], vel[3 * k + 1] - vel[3 * j + 1], vel[3 * k + 2] - vel[3 * j + 2]};
            double vr = v[0] * D[0] + v[1] * D[1] + v[2] * D[2];
            double hbar = 0.5 * (h[k] + h[j]);
            double Dn = r2 + eps * hbar * hbar;
            double cbar = 0.5 * (c[k] + c[j]), rbar = 0.5 * (rho[k] + rho[j]);
            double mu = 0.0, Pi = 0.0, Pmu = 0.0;
            if (vr < 0.0) {
                mu = hbar * vr / Dn;
                Pi = (-alpha * cbar * mu + beta * mu * mu) / rbar;
                Pmu = (-alpha * cbar + 2.0 * beta * mu) / rbar;
            }
            double sdw = kk.wr + kj.wr;
            double B = A[k] * kk.wr + A[j] * kj.wr + Pi * 0.5 * sdw;
            const double* wj = w + 3 * j;
            double U[3], Q = 0.0;
            for (int a = 0; a < 3; ++a) {
                U[a] = m[j] * wk[a] - m[k] * wj[a];
                Q += rhat[a] * U[a];
            }
            // forward: a_k += -m_j B rhat
            for (int a = 0; a < 3; ++a) acc[a] -= m[j] * B * rhat[a];
            // dE/d(.) with E = -B Q
            double rw = rhat[0] * wj[0] + rhat[1] * wj[1] + rhat[2] * wj[2];
            mb += B * rw;
            Abk += -Q * kk.wr;
            double dmu_dh = (vr < 0.0) ? 0.5 * vr * (r2 - eps * hbar * hbar) / (Dn * Dn) : 0.0;
            hbk += -Q * (A[k] * kk.wrh + Pi * 0.5 * kk.wrh + 0.5 * sdw * Pmu * dmu_dh);
            rbk += Q * Pi * sdw / (4.0 * rbar);
            if (vr < 0.0)
                for (int a = 0; a < 3; ++a) vb[a] += -Q * 0.5 * sdw * Pmu * hbar * D[a] / Dn;
            double dBr = A[k] * kk.wrr + A[j] * kj.wrr + Pi * 0.5 * (kk.wrr + kj.wrr);
            for (int a = 0; a < 3; ++a) {
                double dmu = (vr < 0.0) ? hbar * v[a] / Dn - 2.0 * hbar * vr * D[a] / (Dn * Dn) : 0.0;
                double dB = dBr * rhat[a] + 0.5 * sdw * Pmu * dmu;
                double dQ = (U[a] - Q * rhat[a]) / r;
                xb[a] += -Q * dB - B * dQ;
            }
        }
        lossi[k] = wk[0] * acc[0] + wk[1] * acc[1] + wk[2] * acc[2] + s[k] * rho[k];
        for (int a = 0; a < 3; ++a) {
            gx[3 * k + a] = xb[a];
            gv[3 * k + a] = vb[a];
        }
        gm[k] = mb;
        hb[k] = hbk;
        rb[k] = rbk;
        Ab[k] = Abk;
    });
    // per particle: A -> f, rho; f -> h, rho, rho'; rho(h), rho'(h) -> h; implicit h
    std::vector<double> al(n), be(n);
    for (int64_t k = 0; k < n; ++k) {
        double rbk = rb[k] + s[k];
        double fb = Ab[k] * (gamma - 1.0) * u[k] / rho[k];
        rbk += -Ab[k] * A[k] / rho[k];
        double Db = -f[k] * f[k] * fb;
        double hbk = hb[k] + Db * rh[k] / (3.0 * rho[k]);
        double rpb = Db * h[k] / (3.0 * rho[k]);
        rbk += -Db * h[k] * rh[k] / (3.0 * rho[k] * rho[k]);
        hbk += rbk * rh[k] + rpb * rhh[k];
        double lam = hbk * f[k] / (4.0 * kPi * h[k] * h[k] * rho[k]);
        al[k] = rbk - lam * 4.0 * kPi / 3.0 * h[k] * h[k] * h[k];
        be[k] = rpb;
        gm[k] += lam * nngb;
    }
    // density gather: rho_i and rho'_i at fixed h over (x, m)
    parallel_for(n, [&](int64_t k) {
        double xb[3] = {0, 0, 0};
        double mb = al[k] * m4_full(0.0, h[k]).w + be[k] * m4_full(0.0, h[k]).wh;
        for (int64_t e = L.off[k]; e < L.off[k + 1]; ++e) {
            int32_t j = L.idx[e];
            double dx, dy, dz;
            double r2 = dist2(x, y, z, k, j, dx, dy, dz);
            double r = std::sqrt(r2);
            K2 kk = m4_full(r, h[k]), kj = m4_full(r, h[j]);
            if (r2 < h[j] * h[j]) mb += al[j] * kj.w + be[j] * kj.wh;
            if (r2 == 0.0) continue;
            double coef = al[k] * m[j] * kk.wr + be[k] * m[j] * kk.wrh + al[j] * m[k] * kj.wr + be[j] * m[k] * kj.wrh;
            xb[0] += coef * (-dx) / r;
            xb[1] += coef * (-dy) / r;
            xb[2] += coef * (-dz) / r;
        }
        for (int a = 0; a < 3; ++a) gx[3 * k + a] += xb[a];
        gm[k] += mb;
    });
    double Ls = 0.0;
    for (int64_t k = 0; k < n; ++k) Ls += lossi[k];
    *loss = Ls;
    return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Forward-mode check of the adjoint on small sets: the loss with every quantity a
// dual number (value, derivative along one seeded input), the exact constraint
// solved by Newton in dual arithmetic (the derivative part converges to the implicit
// derivative), neighbour lists fixed.  One pass per seeded input.
// ---------------------------------------------------------------------------------
namespace {

struct Dual {
    double v, d;
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
inline Dual dsqrt(Dual a) {
    double s = std::sqrt(a.v);
    return {s, a.d / (2.0 * s)};
}
inline Dual C(double x) { return {x, 0.0}; }

Dual m4_w(Dual r, Dual h) {
    Dual q = r / h;
    if (q.v >= 1.0) return C(0.0);
    Dual sigma = C(8.0 / kPi) / (h * h * h);
    if (q.v <= 0.5) return sigma * (C(1.0) - C(6.0) * q * q + C(6.0) * q * q * q);
    Dual u = C(1.0) - q;
    return sigma * C(2.0) * u * u * u;
}

Dual m4_wr(Dual r, Dual h) {
    Dual q = r / h;
    if (q.v >= 1.0) return C(0.0);
    Dual sigma = C(8.0 / kPi) / (h * h * h);
    if (q.v <= 0.5) return sigma / h * (C(-12.0) * q + C(18.0) * q * q);
    Dual u = C(1.0) - q;
    return sigma / h * (C(-6.0) * u * u);
}

}  // namespace

extern "C" int orc_grad_dual(int64_t n, const double* x, const double* y, const double* z,
                             const double* vel, const double* m, const double* u, const double* h0,
                             const double* w, const double* s, double nngb, double gamma, double alpha,
                             double beta, double eps, double* gx, double* gv, double* gm) {
    Particles P{n, x, y, z};
    PairList L = hydro_lists(P, h0, false);
    // seeded input t in [0, 7n): 0..3n-1 positions, 3n..6n-1 velocities, 6n..7n-1 masses
    parallel_for(7 * n, [&](int64_t t) {
        auto pos = [&](int64_t i, int a) -> Dual {
            const double* c = a == 0 ? x : (a == 1 ? y : z);
            return {c[i], (t < 3 * n && t == 3 * i + a) ? 1.0 : 0.0};
        };
        auto velo = [&](int64_t i, int a) -> Dual {
            return {vel[3 * i + a], (t >= 3 * n && t < 6 * n && t - 3 * n == 3 * i + a) ? 1.0 : 0.0};
        };
        auto mass = [&](int64_t i) -> Dual { return {m[i], (t >= 6 * n && t - 6 * n == i) ? 1.0 : 0.0}; };
        auto dvec = [&](int64_t i, int64_t j, Dual* d) {  // x_i - x_j, nearest image (shift from the values)
            for (int a = 0; a < 3; ++a) {
                Dual dd = pos(i, a) - pos(j, a);
                dd.v -= std::nearbyint(dd.v);
                d[a] = dd;
            }
        };
        std::vector<Dual> h(n), rho(n), f(n), A(n);
        for (int64_t i = 0; i < n; ++i) {
            // density as a function of h_i over the fixed lists
            auto rho_of = [&](Dual hi, Dual& rh) {
                Dual r0 = mass(i) * m4_w(C(0.0), hi);
                Dual q0 = C(0.0);
                rh = C(0.0);
                // d/dh by a second dual: differentiate W in h numerically-exact via W_h formula
                auto wh = [&](Dual r, Dual hh) {
                    Dual q = r / hh;
                    Dual w = m4_w(r, hh), wr = m4_wr(r, hh);
                    return C(-3.0) * w / hh - q * wr;
                };
                rh = mass(i) * wh(C(0.0), hi);
                for (int64_t e = L.off[i]; e < L.off[i + 1]; ++e) {
                    int32_t j = L.idx[e];
                    Dual d[3];
                    dvec(i, j, d);
                    Dual r = dsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    if (!(r.v < hi.v)) continue;
                    r0 = r0 + mass(j) * m4_w(r, hi);
                    rh = rh + mass(j) * wh(r, hi);
                }
                (void)q0;
                return r0;
            };
            Dual hi = {h0[i], 0.0};
            Dual rh;
            for (int it = 0; it < 80; ++it) {
                Dual r = rho_of(hi, rh);
                Dual g = C(4.0 * kPi / 3.0) * hi * hi * hi * r - C(nngb) * mass(i);
                Dual gp = C(4.0 * kPi) * hi * hi * r + C(4.0 * kPi / 3.0) * hi * hi * hi * rh;
                hi = hi - g / gp;
            }
            h[i] = hi;
            rho[i] = rho_of(hi, rh);
            f[i] = C(1.0) / (C(1.0) + hi * rh / (C(3.0) * rho[i]));
            A[i] = f[i] * C((gamma - 1.0) * u[i]) / rho[i];
        }
        Dual loss = C(0.0);
        for (int64_t i = 0; i < n; ++i) {
            Dual acc[3] = {C(0.0), C(0.0), C(0.0)};
            double ci = std::sqrt(gamma * (gamma - 1.0) * u[i]);
            for (int64_t e = L.off[i]; e < L.off[i + 1]; ++e) {
                int32_t j = L.idx[e];
                Dual d[3];
                dvec(i, j, d);
                Dual r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2.v == 0.0) continue;
                Dual r = dsqrt(r2);
                Dual dwi = m4_wr(r, h[i]), dwj = m4_wr(r, h[j]);
                Dual vr = C(0.0);
                for (int a = 0; a < 3; ++a) vr = vr + (velo(i, a) - velo(j, a)) * d[a];
                Dual Pi = C(0.0);
                if (vr.v < 0.0) {
                    Dual hb = C(0.5) * (h[i] + h[j]);
                    Dual mu = hb * vr / (r2 + C(eps) * hb * hb);
                    double cj = std::sqrt(gamma * (gamma - 1.0) * u[j]);
                    Dual rb = C(0.5) * (rho[i] + rho[j]);
                    Pi = (C(-alpha * 0.5 * (ci + cj)) * mu + C(beta) * mu * mu) / rb;
                }
                Dual B = A[i] * dwi + A[j] * dwj + Pi * C(0.5) * (dwi + dwj);
                for (int a = 0; a < 3; ++a) acc[a] = acc[a] - mass(j) * B * d[a] / r;
            }
            for (int a = 0; a < 3; ++a) loss = loss + C(w[3 * i + a]) * acc[a];
            loss = loss + C(s[i]) * rho[i];
        }
        if (t < 3 * n) gx[t] = loss.d;
        else if (t < 6 * n) gv[t - 3 * n] = loss.d;
        else gm[t - 6 * n] = loss.d;
    });
    return 0;
}
