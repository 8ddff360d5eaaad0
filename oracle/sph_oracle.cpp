// FP64 CPU oracle for the SPH neighbour search and the density / hydro-force loops.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call, link or
// load this file: only the tests, the package's smoke check and the CPU-baseline arm
// of the benchmark use it.  It shares no code, header or table with the CUDA path.
//
// Everything here is the plain definition, in FP64, compiled with -ffp-contract=off so
// that every product and sum is rounded exactly as written:
//
//  * Peano-Hilbert keys (Sec. 2: Gadget3 orders particles along the Hilbert curve;
//    the curve variant is not stated, the reading taken is Skilling's transpose
//    construction, "Programming the Hilbert curve", AIP Conf. Proc. 707 (2004), on a
//    2^21 grid per axis, axis order x, y, z, interleaved most significant bit first).
//  * stable order by key (ties keep the input order).
//  * neighbour sets (Sec. 2.1): density  N_i = { j : |r_ij| < h_i },
//                               hydro    N_i = { j : |r_ij| < max(h_i, h_j) },
//    minimum-image distances in the periodic unit cube, r^2 = dx*dx + dy*dy + dz*dz.
//  * M4 cubic-spline kernel with compact support h (the paper fixes no kernel; this is
//    the Gadget convention), the SPH density with its h-derivative, the grad-h
//    correction f_i, and the smoothing-length iteration to a fixed effective
//    neighbour number N_ngb = 4 pi rho h^3 / (3 m) (Sec. 3.2, the relation above Eq. 1).
//  * SPH hydro accelerations and du/dt (grad-h pressure term plus Monaghan
//    artificial viscosity); the paper only cites its hydro scheme, the reading is the
//    standard energy-conserving form.
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
int orc_hydro(int64_t n, const double* x, const double* y, const double* z,
              const double* vx, const double* vy, const double* vz, const double* m,
              const double* h, const double* rho, const double* fgrad, const double* u,
              int64_t nt, const int32_t* targets, double gamma, double alpha, double beta,
              double eps, int use_tree, double* ax, double* ay, double* az, double* dudt,
              int32_t* nngb) {
    Particles P{n, x, y, z};
    Tree tree;
    if (use_tree) build_tree(tree, n, x, y, z, h);
    parallel_for(nt, [&](int64_t t) {
        std::vector<int32_t> cand, nb;
        int64_t i = targets[t];
        neighbours(P, h, use_tree ? &tree : nullptr, i, 1, cand, nb);
        double Pi = (gamma - 1.0) * rho[i] * u[i];
        double ci = std::sqrt(gamma * Pi / rho[i]);
        double Ai = fgrad[i] * Pi / (rho[i] * rho[i]);
        double acc[3] = {0.0, 0.0, 0.0};
        double du = 0.0;
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
        ax[t] = acc[0];
        ay[t] = acc[1];
        az[t] = acc[2];
        dudt[t] = du;
        nngb[t] = (int32_t)nb.size();
    });
    return 0;
}

int orc_threads(void) { return n_threads(); }

}  // extern "C"
