// Internal declarations of the CUDA path: the context, the key-ordered particle
// layout, the octree layout and the device helpers used by several kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sphgrp.h"

namespace sphgrp {

// ---------------------------------------------------------------------------------
// Layout in HBM (all arrays indexed by rank = position in key order unless noted)
//
//   keys      uint64   sorted Peano-Hilbert keys
//   perm      int32    rank -> original index
//   rank_of   int32    original index -> rank
//   xd,yd,zd  double   absolute positions (FP64; read only by the rare FP64 re-tests)
//   pfix      uint4    {X, Y, Z, h_f32 bits}: fixed-point position X = floor(x 2^32)
//   poff      float4   {x 2^32 - X, ..., m}: sub-unit offsets in [0,1) and the mass
//   h64       double   smoothing length (FP64 master)
//   hyd0      float4   {vx, vy, vz, c}                        (hydro candidates)
//   hyd1      float4   {A = f P / rho^2, rho, 1/h, Balsara limiter or 1} (hydro candidates)
//
// A coordinate relative to a fixed-point centre C is
//   float(int32(X - C)) + off, scaled by 2^-32:
// the integer difference is exact and wraps to the minimum image of the periodic
// unit cube for free (two's complement), the offset keeps the FP64 position's
// precision, so the only rounding is the final FP32 one.
// ---------------------------------------------------------------------------------

constexpr float kUnitToBox = 2.3283064365386962890625e-10f;  // 2^-32
constexpr double kBoxToUnit = 4294967296.0;                   // 2^32
constexpr int kKeyLevels = 21;

// Walk stack overflow area of the grouped kernels: entries per warp, and warps per SM
// it is sized for (the persistent grids never exceed it).
constexpr int kStackSpillPerWarp = 1024;
constexpr int kStackSharedMax = 256;   // walk-stack entries per warp in shared memory
constexpr int kSpillWarpsPerSM = 64;

// Walk start table: for every level l = 1 .. kStartLevels, the node of every octree
// cell of that level (indexed by the cell's Morton number; -1 where the tree has no
// node of that level), so that a walk can start at the deepest cell holding its
// search sphere instead of the root.  Level l occupies entries
// [start_table_offset(l), start_table_offset(l) + 8^l).
constexpr int kStartLevels = 6;
__host__ __device__ constexpr int start_table_offset(int l) { return ((1 << (3 * l)) - 8) / 7; }
constexpr int kStartTableSize = start_table_offset(kStartLevels + 1);

// Octree: nodes are stored level by level; the children of a node are contiguous.
//   ncen  uint4  {cx, cy, cz, hmax bits}   centre of the tight box in fixed point
//   next  float4 {ex, ey, ez, nchild bits} half extents in fixed-point units, padded
//                                          to cover the sub-unit offsets
//   nlink int4   {first, count, child_first (-1 = leaf), skip}
// skip = the node visited after this one's subtree in a depth-first walk (-1 = end).
struct Tree {
    uint4* ncen = nullptr;
    float4* next = nullptr;
    int4* nlink = nullptr;
    int32_t* nlevel = nullptr;     // level of every node
    int64_t cap = 0;               // allocated nodes
    int64_t count = 0;             // nodes in the current tree
    int level_begin[kKeyLevels + 3] = {0};  // node ranges per level (host copy)
    int nlevels = 0;
    // build scratch kept between builds (no allocation per call): fixed-point node
    // boxes of the bottom-up pass (box_cap nodes) and the top levels' cell table
    uint4* box_lo = nullptr;
    uint4* box_hi = nullptr;
    int64_t box_cap = 0;
    int32_t* top_cells = nullptr;
};

struct DevCounters {
    unsigned long long walks, nodes, cands, tests, pairs, retests, max_stack, pad;
};

enum ErrBits : unsigned {
    kErrRange = 1u,      // position outside [0,1) or NaN
    kErrStack = 2u,      // walk stack overflow
    kErrNodes = 4u,      // node capacity exceeded
    kErrCap = 8u,        // export capacity exceeded
    kErrH = 16u,         // smoothing length outside (0, 0.5)
    kErrTimeout = 64u,   // a bounded device-side wait gave up
    kErrRank = 128u,     // a domain box's rank outside [0, world)
};

struct Ctx {
    sphgrp_params p;
    int64_t n_max = 0;
    int64_t n = 0;
    bool sorted = false;
    bool built = false;
    int sm_count = 0;

    // key order
    uint64_t* keys = nullptr;
    int32_t* perm = nullptr;
    int32_t* rank_of = nullptr;
    // sort scratch
    uint64_t* keys_alt = nullptr;
    int32_t* perm_alt = nullptr;
    uint32_t* hist = nullptr;      // radix histograms
    int64_t hist_cap = 0;
    // particle copies
    double *xd = nullptr, *yd = nullptr, *zd = nullptr;
    uint4* pfix = nullptr;
    float4* poff = nullptr;
    double* h64 = nullptr;
    float4* hyd0 = nullptr;
    float4* hyd1 = nullptr;
    uint32_t* stack_spill = nullptr;   // walk stack overflow (kStackSpillPerWarp per warp)
    int32_t* start_tab = nullptr;      // walk start table of the current octree
    bool start_valid = false;          // start_tab matches the tree (single-box tree only)
    // active / iteration state (rank space)
    int32_t* act = nullptr;        // active ranks (key order)
    int32_t* act2 = nullptr;       // compaction target
    int32_t* flag = nullptr;       // per-rank flags / scan input
    int32_t* scan = nullptr;       // scan output
    int32_t* scan_aux = nullptr;   // scan block sums
    int64_t scan_aux_cap = 0;
    double* lo = nullptr;          // bracket of the iteration
    double* hi = nullptr;
    float4* res4 = nullptr;        // per-rank results (key order): hydro {a, du/dt}, velocity
                                   // {div, curl}, density {S0, S1, count, passes} of finished particles
    float* acc_rho = nullptr;      // per-rank density sums of the current pass
    float* acc_drho = nullptr;
    int32_t* acc_n = nullptr;
    int64_t* cnt64 = nullptr;      // per-target pair counts (export)
    int2* groups = nullptr;        // group list of the current search (first, count)
    int2* groups_tmp = nullptr;
    int32_t* grp_cnt = nullptr;
    int32_t* grp_off = nullptr;
    // backward (allocated by the first backward call)
    float* acc_s2 = nullptr;       // per-rank d2Rho/dh2 sums
    float4* wadj = nullptr;        // weights of the accelerations, rank order
    float4* dadj = nullptr;        // density-adjoint coefficients {alpha, beta, 1/h, s}
    float4* adj0 = nullptr;        // hydro adjoint {xb, mb}
    float4* adj1 = nullptr;        // hydro adjoint {vb, mb of the implicit h}
    float4* adj2 = nullptr;        // hydro adjoint {hb, rhob, Ab, n}
    float4* adj3 = nullptr;        // density adjoint {xb, mb}
    // recycled smoothing-length iteration (allocated by the first call that uses it; a
    // failed allocation falls back to walk passes)
    int32_t* lst = nullptr;        // candidate lists, kListCap entries per slot
    int4* lrec = nullptr;          // list records
    double* lhw = nullptr;         // widened h per slot
    int32_t* lslot = nullptr;      // rank -> slot
    int32_t* npass = nullptr;      // passes made per rank
    bool lst_failed = false;
    // tree
    Tree tree;
    // counters and error flags
    DevCounters* ctr = nullptr;
    unsigned* err = nullptr;
    int* work = nullptr;           // dynamic work counters for persistent kernels
    int* host_small = nullptr;     // pinned host scratch
    sphgrp_stats last{};
    // device timing of the search kernels of the current call
    static constexpr int kMaxTimed = 128;
    cudaEvent_t tev[2 * kMaxTimed] = {};
    int ntimed = 0;
    DevCounters* ctr_log = nullptr;       // counters after every timed launch (device)
    int64_t log_members[kMaxTimed] = {};  // particles processed by every timed launch
    DevCounters* ctr_log_host = nullptr;  // pinned copy
    float log_ms[kMaxTimed] = {};
};

// CUDA-event bracket around one search-kernel launch (api.cu)
void timer_begin(Ctx* c, cudaStream_t s);
void timer_end(Ctx* c, cudaStream_t s, int64_t members);

// process-wide count of the kernels this library has launched (api.cu)
void note_launch();

// error reporting (api.cu)
int set_error(int code, const std::string& msg);
int check_cuda(cudaError_t e, const char* what);

// ---------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------

__device__ __forceinline__ float rel_coord(uint32_t X, float off, uint32_t C) {
    return (__int2float_rn((int32_t)(X - C)) + off) * kUnitToBox;
}

// M4 cubic-spline shape w(q) (support q < 1) and its derivative dw/dq.
// W(r,h) = 8/(pi h^3) w(r/h).
__device__ __forceinline__ void m4_shape(float q, float& w, float& dw) {
    float u = 1.0f - q;
    float w_in = fmaf(q * q, 6.0f * q - 6.0f, 1.0f);
    float dw_in = q * (18.0f * q - 12.0f);
    float w_out = 2.0f * u * u * u;
    float dw_out = -6.0f * u * u;
    bool inner = q <= 0.5f;
    w = inner ? w_in : w_out;
    dw = inner ? dw_in : dw_out;
    if (q >= 1.0f) { w = 0.0f; dw = 0.0f; }
}

// compensated (Kahan) accumulation
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// exact FP64 minimum-image squared distance of the oracle's definition (no FMA)
__device__ __forceinline__ double exact_r2(const double* xd, const double* yd, const double* zd,
                                           int i, int j) {
    double dx = __dsub_rn(xd[j], xd[i]);
    double dy = __dsub_rn(yd[j], yd[i]);
    double dz = __dsub_rn(zd[j], zd[i]);
    dx = __dsub_rn(dx, rint(dx));
    dy = __dsub_rn(dy, rint(dy));
    dz = __dsub_rn(dz, rint(dz));
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Relative half-width of the FP32 decision band: a pair whose FP32 r^2 lies within
// 3 kBandRel H^2 + 8 kBandRel |m|^2 of the threshold H^2 (H = h, or max(h_i, h_j) for the
// symmetric criterion; m = the member's coordinate relative to the group centre) is
// re-decided from the FP64 positions.  Error bound, u = 2^-24 the FP32 unit roundoff,
// D the exact distance, P and M the exact centre-relative candidate and member
// coordinates, all in box units:
//  * coordinates: p = (float(int32(X - C)) + off) 2^-32 rounds at most twice (the int32
//    conversion above 2^24 units and the sum), the offset once at 2^-25 units: each
//    component is within 2u |P| + 2^-57 of the exact one (same for m);
//  * difference form (phase B, r^2 = fma(dx, dx, fma(dy, dy, dz dz)), d = p - m, also
//    after the wrap d - rint(d), which is exact): |d - D| <= u |D| + 2u (|P| + |M|) per
//    component, so |r^2 - D^2| <= 2 |D| |d - D| + 3u D^2 <= 9u D^2 + 4u D (|P| + |M|);
//    with |P| <= D + |M| near D = H this is <= 13u H^2 + 4u |M|^2 + 8u H |M|
//    <= 17u H^2 + 8u |M|^2, i.e. 0.27 kBandRel H^2 + 0.5 kBandRel |M|^2;
//  * dot form (phase A, t = |p|^2 - 2 p.m against H^2 - |m|^2 by three FMAs, |p|^2 and
//    |m|^2 rounded once per term): its own roundings add 6u |p|^2 + 6u |p||m| + 4u |m|^2
//    + u H^2 to the coordinate errors above, <= 26u H^2 + 29u |M|^2 in all, i.e.
//    0.41 kBandRel H^2 + 0.45 kBandRel |M|^2;
//  * H^2 in FP32 from the FP64 square (and h_j^2 from the FP32 h_j): within 3u H^2.
// The band (3 kBandRel H^2 + 8 kBandRel |m|^2) exceeds every bound at least 6-fold in
// the H^2 term and 16-fold in the |m|^2 term, for members at any distance from the
// centre and for wrapped groups.  Members farther than kPreciseReach h (8 h) from the
// centre take their pair physics (not their decisions) from exact fixed-point
// differences; nearer ones lose at most about 8 ulps of r in the FP32 difference.
constexpr float kBandRel = 3.814697265625e-06f;  // 2^-18

// Radix sort tile (sort.cu): 256 threads x 8 keys; the digit histograms take 256
// counters per tile.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

// launch helpers
// at least one block: kernels bound-check their index, and an empty grid is a launch error
inline int blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return b < 1 ? 1 : (int)b;
}

// kernels' host launchers (defined in the .cu files)
int sort_keys(Ctx* c, int64_t n, const double* pos, cudaStream_t s);              // sort.cu
int exclusive_scan_i32(Ctx* c, const int32_t* in, int32_t* out, int64_t n,
                       int32_t* total_dev, cudaStream_t s);                        // sort.cu
int build_tree(Ctx* c, cudaStream_t s);                                            // tree.cu
int refresh_hmax(Ctx* c, cudaStream_t s);                                          // tree.cu
int exclusive_scan_i32_dev(Ctx* c, const int32_t* in, int32_t* out, const int32_t* n_hi, const int32_t* n_lo,
                           int64_t n_bound, int32_t* total_dev, cudaStream_t s);            // sort.cu
int sort_keys_boxed(Ctx* c, int64_t n, const double* pos, const int64_t* box_off_dev, int nbox, uint64_t* tmp64a,
                    uint64_t* tmp64b, int32_t* tmp32a, int32_t* tmp32b, int32_t* box_of_rank,
                    cudaStream_t s);                                                        // sort.cu
int alloc_forest(Ctx* c, int64_t cap);                                                     // tree.cu
int build_forest(Ctx* c, int nbox, const int64_t* box_off_dev, int32_t* lvl, uint4* blo, uint4* bhi,
                 int32_t* tot, const int32_t* box_of_rank, int32_t* start_tabs, cudaStream_t s,
                 const int32_t* box_cfg = nullptr);                                         // tree.cu
int refresh_hmax_forest(Ctx* c, const int32_t* lvl, cudaStream_t s);                       // tree.cu
void note_launches(long long k);                                                           // api.cu

// results of a finished particle (caller's order; rho, dRho/dh and f are FP32 outputs)
__device__ __forceinline__ void hsml_write(int orig, double h, float s0, float s1, int n, int pass, double* h_out,
                                          float* rho, float* drhodh, float* fgrad, int32_t* nngb_out,
                                          int32_t* iters) {
    const float hf = (float)h;
    const float sigma = 2.54647908947032537f / (hf * hf * hf);   // 8 / (pi h^3)
    rho[orig] = sigma * s0;
    drhodh[orig] = -sigma / hf * s1;
    fgrad[orig] = 3.0f * s0 / (3.0f * s0 - s1);
    nngb_out[orig] = n;
    if (iters) iters[orig] = pass;
    h_out[orig] = h;
}

}  // namespace sphgrp
