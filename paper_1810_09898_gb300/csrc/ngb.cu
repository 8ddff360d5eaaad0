// Neighbour search and the SPH loops that consume it, forward and backward.
//
// Two forms (Sec. 1.1 standard search, Sec. 2.1 Neighbour Recycling):
//  * individual: one thread per active particle walks the octree depth-first with
//    skip pointers and radius h_i (hydro: max(h_i, node hmax)), testing the particles
//    of every opened leaf;
//  * grouped: one warp per group of consecutive active particles (key order).  The
//    warp walks the octree cooperatively once for the group (32 nodes tested per
//    step) with the radius that covers every member's sphere, streams the particles
//    of the opened leaves (the common superset) through shared memory in tiles (TMA
//    bulk copies), and every member filters the tile down to its own neighbours.
//
// The grouped kernel is shared by four kinds of pair loop: density (0), hydro (1),
// and the adjoints of the hydro accelerations (2) and of the density (3); the two
// adjoints recompute their pair terms over the same grouped candidate tiles instead
// of storing pair lists.
//
// Pair decisions are taken in FP32 on coordinates relative to a fixed-point centre;
// pairs whose FP32 r^2 falls inside the proven error band around the threshold are
// re-decided from the FP64 positions with the oracle's exact arithmetic, so the
// neighbour sets are those of the FP64 definition.  Sums are FP32 (forward sums
// compensated across tiles).
#include "search_args.cuh"

namespace sphgrp {

constexpr int kWarpsPerBlock = 4;
constexpr int kStackCap = kStackSharedMax;     // walk stack entries in shared memory
constexpr int kRangeCap = 64;                  // pending leaf ranges
constexpr int kSpillCap = kStackSpillPerWarp;  // overflow entries per warp (global memory)
constexpr int kTileD = 128;   // density tile (candidates)
constexpr int kTileH = 128;   // hydro tile
constexpr int kTileA = 128;   // adjoint tiles
constexpr int kTileV = 128;   // velocity-derivative tile



struct LocalCounters {
    unsigned long long nodes = 0, cands = 0, tests = 0, pairs = 0, retests = 0;
    int max_stack = 0;
};

__device__ __forceinline__ void flush_counters(const SearchArgs& a, LocalCounters& lc, int lane) {
    // warp-reduce then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        lc.nodes += __shfl_xor_sync(0xffffffffu, lc.nodes, o);
        lc.cands += __shfl_xor_sync(0xffffffffu, lc.cands, o);
        lc.tests += __shfl_xor_sync(0xffffffffu, lc.tests, o);
        lc.pairs += __shfl_xor_sync(0xffffffffu, lc.pairs, o);
        lc.retests += __shfl_xor_sync(0xffffffffu, lc.retests, o);
        lc.max_stack = max(lc.max_stack, __shfl_xor_sync(0xffffffffu, lc.max_stack, o));
    }
    if (lane == 0) {
        if (lc.nodes) atomicAdd(&a.ctr->nodes, lc.nodes);
        if (lc.cands) atomicAdd(&a.ctr->cands, lc.cands);
        if (lc.tests) atomicAdd(&a.ctr->tests, lc.tests);
        if (lc.pairs) atomicAdd(&a.ctr->pairs, lc.pairs);
        if (lc.retests) atomicAdd(&a.ctr->retests, lc.retests);
        atomicMax(&a.ctr->max_stack, (unsigned long long)lc.max_stack);
    }
}

// Squared distance, in fixed-point units^2 and rounded down, from the point C to a
// node's box (conservative: never larger than the true distance).
__device__ __forceinline__ float node_gap2(const uint4& cen, const float4& ext, uint32_t cx,
                                           uint32_t cy, uint32_t cz) {
    float dx = fabsf(__int2float_rz((int32_t)(cen.x - cx)));
    float dy = fabsf(__int2float_rz((int32_t)(cen.y - cy)));
    float dz = fabsf(__int2float_rz((int32_t)(cen.z - cz)));
    float gx = fmaxf(__fsub_rd(dx, ext.x), 0.0f);
    float gy = fmaxf(__fsub_rd(dy, ext.y), 0.0f);
    float gz = fmaxf(__fsub_rd(dz, ext.z), 0.0f);
    return __fadd_rd(__fadd_rd(__fmul_rd(gx, gx), __fmul_rd(gy, gy)), __fmul_rd(gz, gz));
}

// radius in box units -> squared radius in fixed-point units, rounded up, with a
// relative margin for the FP32 error of the radius itself
__device__ __forceinline__ float radius2_units(float r_box) {
    float r = __fmul_ru(__fmul_ru(r_box, 1.0000010f), 4294967296.0f);
    return __fmul_ru(r, r);
}

// Members farther than this many smoothing lengths from the group centre (per axis)
// evaluate the pair physics from exact fixed-point differences: the FP32 difference of
// two centre-relative coordinates loses up to |m| / h ulps of r, so below this reach the
// pair terms carry at most about 8 ulps (1e-6 relative) of error, far inside the density
// (1e-5) and acceleration (1e-4) bars; the decisions are exact at any reach (the band's
// |m|^2 term).  The exact path reloads both fixed-point records from global memory.
constexpr float kPreciseReach = 8.0f;

// x_j - x_k from the fixed-point layout: exact integer minimum image plus the offsets.
__device__ __forceinline__ float fix_diff(uint32_t Xj, float oj, uint32_t Xk, float ok) {
    return (__int2float_rn((int32_t)(Xj - Xk)) + (oj - ok)) * kUnitToBox;
}

// Difference of two coordinates relative to one centre.  Both lie in [-1/2, 1/2); when
// a group can reach half the box (WRAP) the difference is brought back to the nearest
// periodic image, otherwise it already is that image (|m| + h < 1/2 for every member).
template <bool WRAP>
__device__ __forceinline__ float rel_diff(float p, float m) {
    float d = p - m;
    if (WRAP) d -= rintf(d);
    return d;
}

// dW/dr = kSkernel h^-4 dw/dq for the M4 spline W = 8 / (pi h^3) w(r / h)
constexpr float kSkernel = 2.54647908947032537f;   // 8 / pi

// M4 shape w(q), w'(q), w''(q) (zero for q >= 1)
__device__ __forceinline__ void m4_shape2(float q, float& w, float& dw, float& d2w) {
    float u = 1.0f - q;
    bool inner = q <= 0.5f;
    w = inner ? fmaf(q * q, 6.0f * q - 6.0f, 1.0f) : 2.0f * u * u * u;
    dw = inner ? q * (18.0f * q - 12.0f) : -6.0f * u * u;
    d2w = inner ? fmaf(36.0f, q, -12.0f) : 12.0f * u;
    if (q >= 1.0f) { w = 0.0f; dw = 0.0f; d2w = 0.0f; }
}

// ---------------------------------------------------------------------------------
// TMA bulk copies (global -> shared) completing on an mbarrier
// ---------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// orders this thread's earlier generic accesses of shared memory before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Waits, with the whole warp, for the phase with the given parity; gives up after a
// bounded number of polls (the copies of a tile take microseconds), setting the timeout
// flag.  The result is the same on every lane: true only if every lane saw the phase
// complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity, unsigned* err) {
    bool ok = false;
    for (uint32_t k = 0; k < (1u << 24) && !ok; ++k) ok = mbar_try_wait(bar, parity);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(err, kErrTimeout);
    return ok;
}

// ---------------------------------------------------------------------------------
// Per-member state of the four pair loops
// ---------------------------------------------------------------------------------

// position part shared by all members: coordinates relative to the group centre (the
// exact fixed-point position is reloaded by the rare paths that need it)
struct MemberPos {
    float mx, my, mz;
    bool precise;       // far from the group centre: physics from exact differences
    int rank;           // -1: slot empty
    int n;              // neighbours found
    int64_t xpos;       // export write position
};

__device__ __forceinline__ bool pos_init(MemberPos& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                         uint32_t cz, float hf) {
    M.rank = rank;
    M.n = 0;
    M.xpos = 0;
    M.precise = false;
    if (rank < 0) {
        M.mx = M.my = M.mz = 0.0f;
        return false;
    }
    uint4 P = a.pfix[rank];
    float4 O = a.poff[rank];
    M.mx = rel_coord(P.x, O.x, cx);
    M.my = rel_coord(P.y, O.y, cy);
    M.mz = rel_coord(P.z, O.z, cz);
    M.precise = fmaxf(fabsf(M.mx), fmaxf(fabsf(M.my), fabsf(M.mz))) > kPreciseReach * hf;
    return true;
}

// density member
struct DMember : MemberPos {
    float hinv;
    float h2lo, h2hi;   // decided-inside below h2lo, candidate below h2hi
    float thr_dot;      // phase-A threshold of |p|^2 - 2 p.m (= h2hi - |m|^2)
    float s0, c0, s1, c1, s2, c2;   // compensated totals: sum m w, sum m (3w + q w'), sum of the W_hh shape
    float p0, p1, p2;               // plain partial sums of the current tile
};

// density member with the velocity derivatives over the same density set: the sums of
// -m v_ij . grad W (divergence) and m v_ij x grad W (curl) at h_i, before the 1/rho
struct DVMember : DMember {
    float vx, vy, vz, sk;
    float sd, cd, sx, cx_, sy, cy_, sz, cz_;   // compensated totals
    float pd, px_, py_, pz_;                   // plain partial sums of the current tile
};

// density member of the recycled smoothing-length iteration: besides the sums at h it
// keeps every candidate inside the widened radius h_w in its slice's sub-list
struct DLMember : DMember {
    float hwf;          // h_w (FP32): the walk radius covers it
    float h2whi;        // widened candidate threshold of the difference form
    float thr_dot_w;    // widened phase-A threshold of the dot form
    int lsub;           // capacity of this lane's sub-list
    int lcnt;           // candidates found (above lsub: the sub-list overflowed)
    int32_t* lptr;      // this lane's sub-list
};

// members of the symmetric criterion |r| < max(h_i, h_j) (hydro and both adjoints)
struct SymMember : MemberPos {
    float h, hinv, sk;  // sk = 8 / (pi h^4): dW/dr = sk * dw/dq
    float h2, bk;       // h^2 (FP32 of the FP64 square), band offset 8 b |m|^2
    float bk_dot;       // bk - |m|^2: phase-A offset of the dot form
};

struct HMember : SymMember {
    float vx, vy, vz, cs, A, rho, fb;   // fb: the viscosity limiter (1 without one)
    float sx, cx_, sy, cy_, sz, cz_, su, cu;   // compensated totals
    float px_, py_, pz_, pu;                   // plain partial sums of the current tile
};

// hydro-adjoint member: the forward hydro state, the weights w_k = dL/da_k, and the
// adjoint sums of x, v, m, h, rho and A = f P / rho^2
struct HAMember : SymMember {
    float vx, vy, vz, cs, A, rho, m;
    float wx, wy, wz;
    float xb[3], vb[3], mb, hb, rb, Ab;
};

// density-adjoint member: the coefficients alpha = adjoint of rho at fixed h (with the
// implicit-h term) and beta = adjoint of dRho/dh
struct DAMember : SymMember {
    float alpha, beta, m;
    float xb[3], mb;
};

// velocity-derivative member (density criterion): sums of -m v_ij . grad W (divergence)
// and m v_ij x grad W (curl), v_ij = v_i - v_j, grad W at h_i
struct VMember : MemberPos {
    float hinv;
    float h2lo, h2hi;
    float thr_dot;
    float sk;               // 8 / (pi h^4): dW/dr = sk * dw/dq
    float vx, vy, vz;
    float rrho;             // 1 / rho_i
    float sd, cd, sx, cx_, sy, cy_, sz, cz_;   // compensated totals
    float pd, px_, py_, pz_;                   // plain partial sums of the current tile
};

__device__ __forceinline__ void member_init(DMember& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                            uint32_t cz) {
    M.s0 = M.c0 = M.s1 = M.c1 = M.s2 = M.c2 = 0.0f;
    M.p0 = M.p1 = M.p2 = 0.0f;
    double h = rank >= 0 ? a.h64[rank] : 1.0;
    float hf = (float)h;
    if (!pos_init(M, a, rank, cx, cy, cz, hf)) {
        M.hinv = 0.0f;
        M.h2lo = M.h2hi = -1.0f;
        M.thr_dot = -3.0e38f;
        return;
    }
    M.hinv = 1.0f / hf;
    float h2 = (float)(h * h);
    float m2 = M.mx * M.mx + M.my * M.my + M.mz * M.mz;
    float bk = 8.0f * kBandRel * m2;
    M.h2hi = fmaf(h2, 1.0f + 3.0f * kBandRel, bk);
    M.h2lo = fmaf(h2, 1.0f - 3.0f * kBandRel, -bk);
    M.thr_dot = M.h2hi - m2;
}

__device__ __forceinline__ void member_init(DVMember& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                            uint32_t cz) {
    member_init(static_cast<DMember&>(M), a, rank, cx, cy, cz);
    M.sd = M.cd = M.sx = M.cx_ = M.sy = M.cy_ = M.sz = M.cz_ = 0.0f;
    M.pd = M.px_ = M.py_ = M.pz_ = 0.0f;
    M.vx = M.vy = M.vz = M.sk = 0.0f;
    if (rank < 0) return;
    const float4 V = a.hyd0[rank];
    M.vx = V.x;
    M.vy = V.y;
    M.vz = V.z;
    M.sk = kSkernel * (M.hinv * M.hinv) * (M.hinv * M.hinv);
}

__device__ __forceinline__ void member_init(DLMember& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                            uint32_t cz) {
    member_init(static_cast<DMember&>(M), a, rank, cx, cy, cz);
    M.lsub = 0;
    M.lcnt = 0;
    M.lptr = nullptr;
    if (rank < 0) {
        M.hwf = 0.0f;
        M.h2whi = -1.0f;
        M.thr_dot_w = -3.0e38f;
        return;
    }
    // the same band as the thresholds at h, at h_w: every candidate with an exact
    // distance below h_w passes it
    const double hw = a.h64[rank] * a.list_widen;
    M.hwf = (float)hw;
    const float m2 = M.mx * M.mx + M.my * M.my + M.mz * M.mz;
    M.h2whi = fmaf((float)(hw * hw), 1.0f + 3.0f * kBandRel, 8.0f * kBandRel * m2);
    M.thr_dot_w = M.h2whi - m2;
}

__device__ __forceinline__ bool sym_init(SymMember& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                         uint32_t cz) {
    double h = rank >= 0 ? a.h64[rank] : 1.0;
    M.h = (float)h;
    if (!pos_init(M, a, rank, cx, cy, cz, M.h)) {
        M.h = 0.0f; M.hinv = 0.0f; M.sk = 0.0f;
        M.h2 = -1.0f; M.bk = -1.0f;
        M.bk_dot = -3.0e38f;
        return false;
    }
    M.h2 = (float)(h * h);
    float m2 = M.mx * M.mx + M.my * M.my + M.mz * M.mz;
    M.bk = 8.0f * kBandRel * m2;
    M.bk_dot = M.bk - m2;
    return true;
}

__device__ __forceinline__ void member_init(HMember& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                            uint32_t cz) {
    M.sx = M.cx_ = M.sy = M.cy_ = M.sz = M.cz_ = M.su = M.cu = 0.0f;
    M.px_ = M.py_ = M.pz_ = M.pu = 0.0f;
    M.vx = M.vy = M.vz = M.cs = M.A = M.rho = 0.0f;
    M.fb = 1.0f;
    if (!sym_init(M, a, rank, cx, cy, cz)) return;
    float4 H0 = a.hyd0[rank];
    float4 H1 = a.hyd1[rank];   // {A, rho, 1/h, limiter}
    M.hinv = H1.z;
    M.sk = kSkernel * (H1.z * H1.z) * (H1.z * H1.z);
    M.fb = H1.w;
    M.vx = H0.x; M.vy = H0.y; M.vz = H0.z; M.cs = H0.w;
    M.A = H1.x;
    M.rho = H1.y;
}

__device__ __forceinline__ void member_init(HAMember& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                            uint32_t cz) {
    for (int k = 0; k < 3; ++k) M.xb[k] = M.vb[k] = 0.0f;
    M.mb = M.hb = M.rb = M.Ab = 0.0f;
    M.vx = M.vy = M.vz = M.cs = M.A = M.rho = M.m = 0.0f;
    M.wx = M.wy = M.wz = 0.0f;
    if (!sym_init(M, a, rank, cx, cy, cz)) return;
    float4 H0 = a.hyd0[rank];
    float4 H1 = a.hyd1[rank];
    float4 Wt = a.wadj[rank];
    M.hinv = H1.z;
    M.sk = H1.w;
    M.vx = H0.x; M.vy = H0.y; M.vz = H0.z; M.cs = H0.w;
    M.A = H1.x;
    M.rho = H1.y;
    M.m = a.poff[rank].w;
    M.wx = Wt.x; M.wy = Wt.y; M.wz = Wt.z;
}

__device__ __forceinline__ void member_init(DAMember& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                            uint32_t cz) {
    for (int k = 0; k < 3; ++k) M.xb[k] = 0.0f;
    M.mb = 0.0f;
    M.alpha = M.beta = M.m = 0.0f;
    if (!sym_init(M, a, rank, cx, cy, cz)) return;
    float4 D = a.dadj[rank];
    M.alpha = D.x;
    M.beta = D.y;
    M.hinv = D.z;
    M.sk = D.w;
    M.m = a.poff[rank].w;
}

__device__ __forceinline__ void member_init(VMember& M, const SearchArgs& a, int rank, uint32_t cx, uint32_t cy,
                                            uint32_t cz) {
    M.sd = M.cd = M.sx = M.cx_ = M.sy = M.cy_ = M.sz = M.cz_ = 0.0f;
    M.pd = M.px_ = M.py_ = M.pz_ = 0.0f;
    M.vx = M.vy = M.vz = 0.0f;
    M.sk = 0.0f;
    M.rrho = 0.0f;
    double h = rank >= 0 ? a.h64[rank] : 1.0;
    float hf = (float)h;
    if (!pos_init(M, a, rank, cx, cy, cz, hf)) {
        M.hinv = 0.0f;
        M.h2lo = M.h2hi = -1.0f;
        M.thr_dot = -3.0e38f;
        return;
    }
    M.hinv = 1.0f / hf;
    float h2 = (float)(h * h);
    float m2 = M.mx * M.mx + M.my * M.my + M.mz * M.mz;
    float bk = 8.0f * kBandRel * m2;
    M.h2hi = fmaf(h2, 1.0f + 3.0f * kBandRel, bk);
    M.h2lo = fmaf(h2, 1.0f - 3.0f * kBandRel, -bk);
    M.thr_dot = M.h2hi - m2;
    const float4 H0 = a.hyd0[rank];
    const float4 H1 = a.hyd1[rank];
    M.vx = H0.x; M.vy = H0.y; M.vz = H0.z;
    M.rrho = 1.0f / H1.y;
    M.sk = H1.w;
}

// walk radius ingredients: density R_s = max(|m| + h); symmetric R_g = max |m|, hmax_g
__device__ __forceinline__ void radius_terms(const VMember& M, float& rl, float& hl) {
    if (M.rank < 0) return;
    float mr = sqrt(M.mx * M.mx + M.my * M.my + M.mz * M.mz);
    rl = fmaxf(rl, mr + 1.0f / M.hinv);
}

__device__ __forceinline__ void radius_terms(const DLMember& M, float& rl, float& hl) {
    if (M.rank < 0) return;
    float mr = sqrtf(M.mx * M.mx + M.my * M.my + M.mz * M.mz);
    rl = fmaxf(rl, mr + M.hwf);
}

__device__ __forceinline__ void radius_terms(const DMember& M, float& rl, float& hl) {
    if (M.rank < 0) return;
    float mr = sqrtf(M.mx * M.mx + M.my * M.my + M.mz * M.mz);
    rl = fmaxf(rl, mr + 1.0f / M.hinv);
}

__device__ __forceinline__ void radius_terms(const SymMember& M, float& rl, float& hl) {
    if (M.rank < 0) return;
    float mr = sqrtf(M.mx * M.mx + M.my * M.my + M.mz * M.mz);
    rl = fmaxf(rl, mr);
    hl = fmaxf(hl, M.h);
}

// ---------------------------------------------------------------------------------
// Candidate tiles in shared memory.  The raw key-ordered records of a tile's leaf
// ranges land here by TMA bulk copies (cp.async.bulk, global -> shared, completion
// on an mbarrier); the fixed-point positions are then converted in place to FP32
// coordinates relative to the group centre, {px, py, pz, |p|^2}.  With S slices the
// lane of slice s filters positions s, s + S, s + 2S, ...; positions beyond the tile's
// candidates, up to whole chunks of 32 per slice, hold NaN dummies.
// ---------------------------------------------------------------------------------

struct DensTile {
    float4 p[kTileD];   // raw pfix -> {px, py, pz, |p|^2}
    float4 o[kTileD];   // raw poff {ox, oy, oz, m}
    int r[kTileD];      // ranks
    uint32_t masks[kTileD];   // phase-A bit masks [chunk][lane]
};

struct HydroTile {
    float4 p[kTileH];   // raw pfix -> {px, py, pz, |p|^2}
    float4 o[kTileH];   // raw poff {ox, oy, oz, m} -> {h^2, m, -, -}
    float4 v[kTileH];   // raw hyd0 {vx, vy, vz, c}
    float4 h[kTileH];   // raw hyd1 {A, rho, 1/h, 8/(pi h^4)}
    int r[kTileH];
    uint32_t masks[kTileH];
};

struct HAdjTile {
    float4 p[kTileA];
    float4 o[kTileA];   // -> {h^2, m, -, -}
    float4 v[kTileA];   // hyd0 {vx, vy, vz, c}
    float4 h[kTileA];   // hyd1 {A, rho, 1/h, 8/(pi h^4)}
    float4 w[kTileA];   // wadj {wx, wy, wz, -}
    int r[kTileA];
    uint32_t masks[kTileA];
};

struct DAdjTile {
    float4 p[kTileA];
    float4 o[kTileA];   // -> {h^2, m, -, -}
    float4 d[kTileA];   // dadj {alpha, beta, 1/h, 8/(pi h^4)}
    int r[kTileA];
    uint32_t masks[kTileA];
};

struct DensVTile {
    float4 p[kTileD];   // raw pfix -> {px, py, pz, |p|^2}
    float4 o[kTileD];   // raw poff {ox, oy, oz, m}
    float4 v[kTileD];   // raw hyd0 {vx, vy, vz, -}
    int r[kTileD];
    uint32_t masks[kTileD];
};

struct VelTile {
    float4 p[kTileV];   // raw pfix -> {px, py, pz, |p|^2}
    float4 o[kTileV];   // raw poff {ox, oy, oz, m}
    float4 v[kTileV];   // raw hyd0 {vx, vy, vz, -}
    int r[kTileV];
    uint32_t masks[kTileV];
};

// kind policies
struct KDens {
    static constexpr int min_blocks = 8;   // resident blocks per SM (register budget; 0: compiler's choice)
    static constexpr int id = 0;
    static constexpr bool sym = false;
    static constexpr int cap = kTileD;
    static constexpr uint32_t bytes = 32u;
    using Member = DMember;
    using Tile = DensTile;
};
struct KDensVel {
    static constexpr int min_blocks = 6;   // resident blocks per SM (register budget; 0: compiler's choice)
    static constexpr int id = kKindDensityVel;
    static constexpr bool sym = false;
    static constexpr int cap = kTileD;
    static constexpr uint32_t bytes = 48u;
    using Member = DVMember;
    using Tile = DensVTile;
};
struct KDensList {
    static constexpr int min_blocks = 7;   // resident blocks per SM (register budget; 0: compiler's choice)
    static constexpr int id = kKindDensityList;
    static constexpr bool sym = false;
    static constexpr int cap = kTileD;
    static constexpr uint32_t bytes = 32u;
    using Member = DLMember;
    using Tile = DensTile;
};
struct KHydro {
    static constexpr int min_blocks = 5;   // resident blocks per SM (register budget; 0: compiler's choice)
    static constexpr int id = 1;
    static constexpr bool sym = true;
    static constexpr int cap = kTileH;
    static constexpr uint32_t bytes = 64u;
    using Member = HMember;
    using Tile = HydroTile;
};
struct KHAdj {
    static constexpr int min_blocks = 0;   // resident blocks per SM (register budget; 0: compiler's choice)
    static constexpr int id = 2;
    static constexpr bool sym = true;
    static constexpr int cap = kTileA;
    static constexpr uint32_t bytes = 80u;
    using Member = HAMember;
    using Tile = HAdjTile;
};
struct KDAdj {
    static constexpr int min_blocks = 6;   // resident blocks per SM (register budget; 0: compiler's choice)
    static constexpr int id = 3;
    static constexpr bool sym = true;
    static constexpr int cap = kTileA;
    static constexpr uint32_t bytes = 48u;
    using Member = DAMember;
    using Tile = DAdjTile;
};

struct KVel {
    static constexpr int min_blocks = 0;   // resident blocks per SM (register budget; 0: compiler's choice)
    static constexpr int id = 4;
    static constexpr bool sym = false;
    static constexpr int cap = kTileV;
    static constexpr uint32_t bytes = 48u;
    using Member = VMember;
    using Tile = VelTile;
};

// bulk copies of one run of candidates into the tile
__device__ __forceinline__ void stage_run(DensTile& T, const SearchArgs& a, int dst, int src, uint32_t b,
                                          unsigned long long* bar) {
    bulk_to_smem(&T.p[dst], a.pfix + src, b, bar);
    bulk_to_smem(&T.o[dst], a.poff + src, b, bar);
}
__device__ __forceinline__ void stage_run(HydroTile& T, const SearchArgs& a, int dst, int src, uint32_t b,
                                          unsigned long long* bar) {
    bulk_to_smem(&T.p[dst], a.pfix + src, b, bar);
    bulk_to_smem(&T.o[dst], a.poff + src, b, bar);
    bulk_to_smem(&T.v[dst], a.hyd0 + src, b, bar);
    bulk_to_smem(&T.h[dst], a.hyd1 + src, b, bar);
}
__device__ __forceinline__ void stage_run(HAdjTile& T, const SearchArgs& a, int dst, int src, uint32_t b,
                                          unsigned long long* bar) {
    bulk_to_smem(&T.p[dst], a.pfix + src, b, bar);
    bulk_to_smem(&T.o[dst], a.poff + src, b, bar);
    bulk_to_smem(&T.v[dst], a.hyd0 + src, b, bar);
    bulk_to_smem(&T.h[dst], a.hyd1 + src, b, bar);
    bulk_to_smem(&T.w[dst], a.wadj + src, b, bar);
}
__device__ __forceinline__ void stage_run(DensVTile& T, const SearchArgs& a, int dst, int src, uint32_t b,
                                          unsigned long long* bar) {
    bulk_to_smem(&T.p[dst], a.pfix + src, b, bar);
    bulk_to_smem(&T.o[dst], a.poff + src, b, bar);
    bulk_to_smem(&T.v[dst], a.hyd0 + src, b, bar);
}
__device__ __forceinline__ void stage_run(VelTile& T, const SearchArgs& a, int dst, int src, uint32_t b,
                                          unsigned long long* bar) {
    bulk_to_smem(&T.p[dst], a.pfix + src, b, bar);
    bulk_to_smem(&T.o[dst], a.poff + src, b, bar);
    bulk_to_smem(&T.v[dst], a.hyd0 + src, b, bar);
}
__device__ __forceinline__ void stage_run(DAdjTile& T, const SearchArgs& a, int dst, int src, uint32_t b,
                                          unsigned long long* bar) {
    bulk_to_smem(&T.p[dst], a.pfix + src, b, bar);
    bulk_to_smem(&T.o[dst], a.poff + src, b, bar);
    bulk_to_smem(&T.d[dst], a.dadj + src, b, bar);
}

// ---------------------------------------------------------------------------------
// Pair physics
// ---------------------------------------------------------------------------------

// Plain per-tile partial sums are folded into the compensated totals after every
// tile (or leaf): a few tens of terms in plain FP32, Kahan across blocks.
__device__ __forceinline__ void flush(DMember& M) {
    kahan_add(M.s0, M.c0, M.p0);
    kahan_add(M.s1, M.c1, M.p1);
    kahan_add(M.s2, M.c2, M.p2);
    M.p0 = M.p1 = M.p2 = 0.0f;
}

__device__ __forceinline__ void flush(HMember& M) {
    kahan_add(M.sx, M.cx_, M.px_);
    kahan_add(M.sy, M.cy_, M.py_);
    kahan_add(M.sz, M.cz_, M.pz_);
    kahan_add(M.su, M.cu, M.pu);
    M.px_ = M.py_ = M.pz_ = M.pu = 0.0f;
}

__device__ __forceinline__ void flush(VMember& M) {
    kahan_add(M.sd, M.cd, M.pd);
    kahan_add(M.sx, M.cx_, M.px_);
    kahan_add(M.sy, M.cy_, M.py_);
    kahan_add(M.sz, M.cz_, M.pz_);
    M.pd = M.px_ = M.py_ = M.pz_ = 0.0f;
}

__device__ __forceinline__ void flush(DVMember& M) {
    flush(static_cast<DMember&>(M));
    kahan_add(M.sd, M.cd, M.pd);
    kahan_add(M.sx, M.cx_, M.px_);
    kahan_add(M.sy, M.cy_, M.py_);
    kahan_add(M.sz, M.cz_, M.pz_);
    M.pd = M.px_ = M.py_ = M.pz_ = 0.0f;
}

__device__ __forceinline__ void flush(HAMember&) {}
__device__ __forceinline__ void flush(DAMember&) {}

template <class Mem>
__device__ __forceinline__ void precise_diff(const Mem& M, const SearchArgs& a, int crank, float& dx, float& dy,
                                             float& dz, float& r2) {
    uint4 Q = a.pfix[crank];
    float4 O = a.poff[crank];
    // the member's own fixed-point position, reloaded (rare path: no registers held)
    const uint4 P = a.pfix[M.rank];
    const float4 Om = a.poff[M.rank];
    dx = fix_diff(Q.x, O.x, P.x, Om.x);
    dy = fix_diff(Q.y, O.y, P.y, Om.y);
    dz = fix_diff(Q.z, O.z, P.z, Om.z);
    r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// density pair: p = candidate's coordinates relative to the member's centre, m_j its mass
template <int MODE, bool WRAP = false>
__device__ __forceinline__ void density_pair(DMember& M, const SearchArgs& a, float4 p, float mj, int crank,
                                             LocalCounters& lc) {
    float dx = rel_diff<WRAP>(p.x, M.mx), dy = rel_diff<WRAP>(p.y, M.my), dz = rel_diff<WRAP>(p.z, M.mz);
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    bool in = r2 < M.h2lo;
    if (!in) {
        if (!(r2 < M.h2hi)) return;
        double e = exact_r2(a.xd, a.yd, a.zd, M.rank, crank);
        double h = a.h64[M.rank];
        in = e < __dmul_rn(h, h);
        lc.retests++;
    }
    if (!in) return;
    M.n++;
    if (MODE == kAcc) {
        if (M.precise) precise_diff(M, a, crank, dx, dy, dz, r2);
        float q = r2 * rsqrtf(fmaxf(r2, 1.0e-30f)) * M.hinv;
        if (a.o_s2) {
            float w, dw, d2w;
            m4_shape2(q, w, dw, d2w);
            M.p0 = fmaf(mj, w, M.p0);
            M.p1 = fmaf(mj, fmaf(q, dw, 3.0f * w), M.p1);
            M.p2 = fmaf(mj, fmaf(q * q, d2w, fmaf(8.0f * q, dw, 12.0f * w)), M.p2);
        } else {
            float w, dw;
            m4_shape(q, w, dw);
            M.p0 = fmaf(mj, w, M.p0);
            M.p1 = fmaf(mj, fmaf(q, dw, 3.0f * w), M.p1);
        }
    } else if (MODE == kFill) {
        int64_t q = M.xpos++;
        if (q < a.x_cap) a.x_idx[q] = a.perm[crank];
        else atomicOr(a.err, kErrCap);
    }
}

// density pair with the velocity derivatives: the density decision and sums of
// density_pair, then (for pairs at r > 0) the divergence and curl terms with
// grad_i W = W'(r, h_i) (x_i - x_j) / r and v_ij = v_i - v_j
template <int MODE, bool WRAP = false>
__device__ __forceinline__ void densvel_pair(DVMember& M, const SearchArgs& a, float4 p, float mj, float4 vj,
                                             int crank, LocalCounters& lc) {
    const int n0 = M.n;
    density_pair<MODE, WRAP>(M, a, p, mj, crank, lc);
    if (MODE != kAcc || M.n == n0) return;
    float dx, dy, dz, r2;
    if (M.precise) {
        precise_diff(M, a, crank, dx, dy, dz, r2);
    } else {
        dx = rel_diff<WRAP>(p.x, M.mx);
        dy = rel_diff<WRAP>(p.y, M.my);
        dz = rel_diff<WRAP>(p.z, M.mz);
        r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    }
    if (r2 == 0.0f) return;
    const float rinv = rsqrtf(r2);
    float w, dw;
    m4_shape(r2 * rinv * M.hinv, w, dw);
    const float c = -M.sk * dw * rinv;   // x_i - x_j = -d
    const float gx = c * dx, gy = c * dy, gz = c * dz;
    const float vx = M.vx - vj.x, vy = M.vy - vj.y, vz = M.vz - vj.z;
    M.pd = fmaf(-mj, fmaf(vx, gx, fmaf(vy, gy, vz * gz)), M.pd);
    M.px_ = fmaf(mj, fmaf(vy, gz, -vz * gy), M.px_);
    M.py_ = fmaf(mj, fmaf(vz, gx, -vx * gz), M.py_);
    M.pz_ = fmaf(mj, fmaf(vx, gy, -vy * gx), M.pz_);
}

// density pair of the recycled iteration: a candidate inside the widened threshold joins
// the member's sub-list, then the pair enters the sums at h as in density_pair
template <int MODE, bool WRAP = false>
__device__ __forceinline__ void density_list_pair(DLMember& M, const SearchArgs& a, float4 p, float mj, int crank,
                                                  LocalCounters& lc) {
    const float dx = rel_diff<WRAP>(p.x, M.mx), dy = rel_diff<WRAP>(p.y, M.my), dz = rel_diff<WRAP>(p.z, M.mz);
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (r2 < M.h2whi) {
        if (M.lcnt < M.lsub) M.lptr[M.lcnt] = crank;
        M.lcnt++;
    }
    density_pair<MODE, WRAP>(M, a, p, mj, crank, lc);
}

// velocity-derivative pair (density criterion): p = relative coordinates, mj the mass,
// vj = {vx, vy, vz, -}
template <int MODE, bool WRAP = false>
__device__ __forceinline__ void vel_pair(VMember& M, const SearchArgs& a, float4 p, float mj, float4 vj, int crank,
                                         LocalCounters& lc) {
    float dx = rel_diff<WRAP>(p.x, M.mx), dy = rel_diff<WRAP>(p.y, M.my), dz = rel_diff<WRAP>(p.z, M.mz);
    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    bool in = r2 < M.h2lo;
    if (!in) {
        if (!(r2 < M.h2hi)) return;
        double e = exact_r2(a.xd, a.yd, a.zd, M.rank, crank);
        double h = a.h64[M.rank];
        in = e < __dmul_rn(h, h);
        lc.retests++;
    }
    if (!in) return;
    M.n++;
    if (MODE != kAcc) return;
    if (M.precise) precise_diff(M, a, crank, dx, dy, dz, r2);
    if (r2 == 0.0f) return;   // the particle itself (and coincident ones): grad W = 0
    const float rinv = rsqrtf(r2);
    float w, dw;
    m4_shape(r2 * rinv * M.hinv, w, dw);
    const float c = -M.sk * dw * rinv;   // grad_i W = W' (x_i - x_j) / r, x_i - x_j = -d
    const float gx = c * dx, gy = c * dy, gz = c * dz;
    const float vx = M.vx - vj.x, vy = M.vy - vj.y, vz = M.vz - vj.z;
    M.pd = fmaf(-mj, fmaf(vx, gx, fmaf(vy, gy, vz * gz)), M.pd);
    M.px_ = fmaf(mj, fmaf(vy, gz, -vz * gy), M.px_);
    M.py_ = fmaf(mj, fmaf(vz, gx, -vx * gz), M.py_);
    M.pz_ = fmaf(mj, fmaf(vx, gy, -vy * gx), M.pz_);
}

// decision of the symmetric criterion |r| < max(h_i, h_j) with the FP64 band re-test
template <bool WRAP, class Mem>
__device__ __forceinline__ bool sym_decide(const Mem& M, const SearchArgs& a, float4 p, float hj2, int crank,
                                           LocalCounters& lc, float& dx, float& dy, float& dz, float& r2) {
    dx = rel_diff<WRAP>(p.x, M.mx);
    dy = rel_diff<WRAP>(p.y, M.my);
    dz = rel_diff<WRAP>(p.z, M.mz);
    r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float H2 = fmaxf(M.h2, hj2);
    bool in = r2 < fmaf(H2, 1.0f - 3.0f * kBandRel, -M.bk);
    if (!in) {
        if (!(r2 < fmaf(H2, 1.0f + 3.0f * kBandRel, M.bk))) return false;
        double e = exact_r2(a.xd, a.yd, a.zd, M.rank, crank);
        double hi = a.h64[M.rank], hj = a.h64[crank];
        in = e < fmax(__dmul_rn(hi, hi), __dmul_rn(hj, hj));
        lc.retests++;
    }
    return in;
}

// hydro pair: p = relative coordinates, q = {h_j^2, m_j, -, -}, v = {vx, vy, vz, c_j},
// hh = {A_j, rho_j, 1/h_j, limiter_j}
template <int MODE, bool WRAP = false>
__device__ __forceinline__ void hydro_pair(HMember& M, const SearchArgs& a, float4 p, float4 q,
                                           float4 v, float4 hh, int crank, LocalCounters& lc) {
    // The member itself is a candidate: the exports skip it by rank; the sums skip it
    // as a pair at r = 0 (counted, then taken off the neighbour count at the end).
    if (MODE != kAcc && crank == M.rank) return;
    float dx, dy, dz, r2;
    if (!sym_decide<WRAP>(M, a, p, q.x, crank, lc, dx, dy, dz, r2)) return;
    M.n++;
    if (MODE == kFill) {
        int64_t k = M.xpos++;
        if (k < a.x_cap) a.x_idx[k] = a.perm[crank];
        else atomicOr(a.err, kErrCap);
        return;
    }
    if (MODE != kAcc) return;
    if (M.precise) precise_diff(M, a, crank, dx, dy, dz, r2);
    if (r2 == 0.0f) return;  // coincident: the kernel gradient vanishes
    float rinv = rsqrtf(r2);
    float r = r2 * rinv;
    float wi, dwi, wj, dwj;
    m4_shape(r * M.hinv, wi, dwi);
    m4_shape(r * hh.z, wj, dwj);
    float dWi = M.sk * dwi;
    float dWj = kSkernel * (hh.z * hh.z) * (hh.z * hh.z) * dwj;
    float rx = -dx, ry = -dy, rz = -dz;  // r_ij = x_i - x_j
    float vx = M.vx - v.x, vy = M.vy - v.y, vz = M.vz - v.z;
    float vr = fmaf(vx, rx, fmaf(vy, ry, vz * rz));
    float visc = 0.0f;
    if (vr < 0.0f) {
        float hb = 0.5f * fmaf(q.x, hh.z, M.h);
        float mu = hb * vr * __frcp_rn(fmaf(a.eps * hb, hb, r2));
        float cb = 0.5f * (M.cs + v.w);
        // Pi = (-alpha cbar mu + beta mu^2) / rhobar, rhobar = (rho_i + rho_j) / 2, scaled by
        // the pair mean of the limiter (1 for the plain viscosity)
        visc = 2.0f * fmaf(-a.alpha * cb, mu, a.beta * mu * mu) * __frcp_rn(M.rho + hh.y);
        visc *= 0.5f * (M.fb + hh.w);
    }
    float gbar = 0.5f * (dWi + dWj);
    float coef = q.y * fmaf(M.A, dWi, fmaf(hh.x, dWj, visc * gbar)) * rinv;
    M.px_ = fmaf(coef, dx, M.px_);
    M.py_ = fmaf(coef, dy, M.py_);
    M.pz_ = fmaf(coef, dz, M.pz_);
    M.pu = fmaf(q.y * fmaf(M.A, dWi, 0.5f * visc * gbar) * rinv, vr, M.pu);
}

// Adjoint of sum_i w_i . a_i over one pair, gathered at member k.  The pair enters
// a_k and a_j through the symmetric factor B = A_k W'_k + A_j W'_j + Pi (W'_k + W'_j)/2
// (W' = dW/dr at h_k, h_j); their weighted sum is E = -B Q with
// Q = rhat . (m_j w_k - m_k w_j), rhat = (x_k - x_j) / r.  Accumulated: dE/d of x_k,
// v_k, m_k, h_k, rho_k (through the viscosity) and A_k.
template <int MODE, bool WRAP = false>
__device__ __forceinline__ void hydro_adj_pair(HAMember& M, const SearchArgs& a, float4 p, float4 q, float4 v,
                                               float4 hh, float4 wj, int crank, LocalCounters& lc) {
    // the member itself enters as a pair at r = 0, which contributes nothing
    float dx, dy, dz, r2;
    if (!sym_decide<WRAP>(M, a, p, q.x, crank, lc, dx, dy, dz, r2)) return;
    M.n++;
    if (MODE != kAcc) return;
    if (M.precise) precise_diff(M, a, crank, dx, dy, dz, r2);
    if (r2 == 0.0f) return;
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    const float D0 = -dx, D1 = -dy, D2 = -dz;   // x_k - x_j
    const float e0 = D0 * rinv, e1 = D1 * rinv, e2 = D2 * rinv;
    float wk_, dwk, d2wk, wj_, dwj, d2wj;
    const float qk = r * M.hinv, qj = r * hh.z;
    m4_shape2(qk, wk_, dwk, d2wk);
    m4_shape2(qj, wj_, dwj, d2wj);
    const float Wr_k = M.sk * dwk, Wr_j = hh.w * dwj;
    const float Wrr_k = M.sk * M.hinv * d2wk, Wrr_j = hh.w * hh.z * d2wj;
    const float Wrh_k = -M.sk * M.hinv * fmaf(qk, d2wk, 4.0f * dwk);
    const float v0 = M.vx - v.x, v1 = M.vy - v.y, v2 = M.vz - v.z;
    const float vr = fmaf(v0, D0, fmaf(v1, D1, v2 * D2));
    const float hbar = 0.5f * fmaf(q.x, hh.z, M.h);
    const float Dn = fmaf(a.eps * hbar, hbar, r2);
    const float iDn = __frcp_rn(Dn);
    const float irbar = 2.0f * __frcp_rn(M.rho + hh.y);   // 1 / rhobar
    float Pi = 0.0f, Pmu = 0.0f;
    if (vr < 0.0f) {
        const float cbar = 0.5f * (M.cs + v.w);
        const float mu = hbar * vr * iDn;
        Pi = fmaf(-a.alpha * cbar, mu, a.beta * mu * mu) * irbar;
        Pmu = fmaf(2.0f * a.beta, mu, -a.alpha * cbar) * irbar;
    }
    const float sdw = Wr_k + Wr_j;
    const float B = fmaf(M.A, Wr_k, fmaf(hh.x, Wr_j, 0.5f * Pi * sdw));
    const float mj = q.y;
    const float U0 = mj * M.wx - M.m * wj.x, U1 = mj * M.wy - M.m * wj.y, U2 = mj * M.wz - M.m * wj.z;
    const float Q = fmaf(e0, U0, fmaf(e1, U1, e2 * U2));
    M.mb = fmaf(B, fmaf(e0, wj.x, fmaf(e1, wj.y, e2 * wj.z)), M.mb);
    M.Ab = fmaf(-Q, Wr_k, M.Ab);
    float dmu_dh = 0.0f;
    if (vr < 0.0f) dmu_dh = 0.5f * vr * fmaf(-a.eps * hbar, hbar, r2) * iDn * iDn;
    M.hb = fmaf(-Q, fmaf(M.A, Wrh_k, fmaf(0.5f * Pi, Wrh_k, 0.5f * sdw * Pmu * dmu_dh)), M.hb);
    M.rb = fmaf(Q * Pi, 0.25f * sdw * irbar, M.rb);
    const float cm = 0.5f * sdw * Pmu;
    if (vr < 0.0f) {
        const float cv = -Q * cm * hbar * iDn;
        M.vb[0] = fmaf(cv, D0, M.vb[0]);
        M.vb[1] = fmaf(cv, D1, M.vb[1]);
        M.vb[2] = fmaf(cv, D2, M.vb[2]);
    }
    const float dBr = fmaf(M.A, Wrr_k, fmaf(hh.x, Wrr_j, 0.5f * Pi * (Wrr_k + Wrr_j)));
    const float ca = (vr < 0.0f) ? hbar * iDn : 0.0f;
    const float cb2 = (vr < 0.0f) ? -2.0f * hbar * vr * iDn * iDn : 0.0f;
    {
        const float dB = fmaf(dBr, e0, cm * fmaf(ca, v0, cb2 * D0));
        const float dQ = (U0 - Q * e0) * rinv;
        M.xb[0] = fmaf(-Q, dB, fmaf(-B, dQ, M.xb[0]));
    }
    {
        const float dB = fmaf(dBr, e1, cm * fmaf(ca, v1, cb2 * D1));
        const float dQ = (U1 - Q * e1) * rinv;
        M.xb[1] = fmaf(-Q, dB, fmaf(-B, dQ, M.xb[1]));
    }
    {
        const float dB = fmaf(dBr, e2, cm * fmaf(ca, v2, cb2 * D2));
        const float dQ = (U2 - Q * e2) * rinv;
        M.xb[2] = fmaf(-Q, dB, fmaf(-B, dQ, M.xb[2]));
    }
}

// Adjoint of sum_i (alpha_i rho_i + beta_i dRho_i/dh_i) at fixed h, gathered at member k:
// rho_k's own sum (x_k moves every pair) and the sums of every j with k in N_j (x_k and
// m_k enter as a neighbour).  q = {h_j^2, m_j, -, -}, d = {alpha_j, beta_j, 1/h_j, s_j}.
template <int MODE, bool WRAP = false>
__device__ __forceinline__ void dens_adj_pair(DAMember& M, const SearchArgs& a, float4 p, float4 q, float4 d,
                                              int crank, LocalCounters& lc) {
    // The member itself enters as a pair at r = 0 like any coincident neighbour:
    // alpha W(0, h) + beta W_h(0, h) = alpha s h - 3 beta s, and no position term.
    float dx, dy, dz, r2;
    if (!sym_decide<WRAP>(M, a, p, q.x, crank, lc, dx, dy, dz, r2)) return;
    M.n++;
    if (MODE != kAcc) return;
    if (M.precise) precise_diff(M, a, crank, dx, dy, dz, r2);
    const float rinv = r2 > 0.0f ? rsqrtf(r2) : 0.0f;
    const float r = r2 * rinv;
    float wk_, dwk, d2wk, wj_, dwj, d2wj;
    const float qk = r * M.hinv, qj = r * d.z;
    m4_shape2(qk, wk_, dwk, d2wk);
    m4_shape2(qj, wj_, dwj, d2wj);
    // k as a neighbour of j: rho_j gains m_k W(r, h_j), dRho_j/dh_j gains m_k W_h(r, h_j)
    const float hj = q.x * d.z;
    M.mb = fmaf(d.x * d.w, hj * wj_, fmaf(-d.y * d.w, fmaf(qj, dwj, 3.0f * wj_), M.mb));
    if (r2 == 0.0f) return;
    const float Wr_k = M.sk * dwk, Wr_j = d.w * dwj;
    const float Whr_k = -M.sk * M.hinv * fmaf(qk, d2wk, 4.0f * dwk);
    const float Whr_j = -d.w * d.z * fmaf(qj, d2wj, 4.0f * dwj);
    const float coef = fmaf(M.alpha * q.y, Wr_k, fmaf(M.beta * q.y, Whr_k, fmaf(d.x * M.m, Wr_j, d.y * M.m * Whr_j)));
    const float c = -coef * rinv;   // rhat = (x_k - x_j) / r = -d / r
    M.xb[0] = fmaf(c, dx, M.xb[0]);
    M.xb[1] = fmaf(c, dy, M.xb[1]);
    M.xb[2] = fmaf(c, dz, M.xb[2]);
}

// phase B dispatch
template <int MODE, bool WRAP>
__device__ __forceinline__ void tile_pair(DMember& M, const SearchArgs& a, const DensTile& T, int j,
                                          LocalCounters& lc) {
    density_pair<MODE, WRAP>(M, a, T.p[j], T.o[j].w, T.r[j], lc);
}
template <int MODE, bool WRAP>
__device__ __forceinline__ void tile_pair(DVMember& M, const SearchArgs& a, const DensVTile& T, int j,
                                          LocalCounters& lc) {
    densvel_pair<MODE, WRAP>(M, a, T.p[j], T.o[j].w, T.v[j], T.r[j], lc);
}
template <int MODE, bool WRAP>
__device__ __forceinline__ void tile_pair(DLMember& M, const SearchArgs& a, const DensTile& T, int j,
                                          LocalCounters& lc) {
    density_list_pair<MODE, WRAP>(M, a, T.p[j], T.o[j].w, T.r[j], lc);
}
template <int MODE, bool WRAP>
__device__ __forceinline__ void tile_pair(VMember& M, const SearchArgs& a, const VelTile& T, int j,
                                          LocalCounters& lc) {
    vel_pair<MODE, WRAP>(M, a, T.p[j], T.o[j].w, T.v[j], T.r[j], lc);
}
template <int MODE, bool WRAP>
__device__ __forceinline__ void tile_pair(HMember& M, const SearchArgs& a, const HydroTile& T, int j,
                                          LocalCounters& lc) {
    hydro_pair<MODE, WRAP>(M, a, T.p[j], T.o[j], T.v[j], T.h[j], T.r[j], lc);
}
template <int MODE, bool WRAP>
__device__ __forceinline__ void tile_pair(HAMember& M, const SearchArgs& a, const HAdjTile& T, int j,
                                          LocalCounters& lc) {
    hydro_adj_pair<MODE, WRAP>(M, a, T.p[j], T.o[j], T.v[j], T.h[j], T.w[j], T.r[j], lc);
}
template <int MODE, bool WRAP>
__device__ __forceinline__ void tile_pair(DAMember& M, const SearchArgs& a, const DAdjTile& T, int j,
                                          LocalCounters& lc) {
    dens_adj_pair<MODE, WRAP>(M, a, T.p[j], T.o[j], T.d[j], T.r[j], lc);
}

// phase A threshold of the dot form |p|^2 - 2 p.m (density) and of the difference
// form (WRAP); symmetric kinds read h_j^2 from the tile
__device__ __forceinline__ float thr_dot(const DMember& M, float) { return M.thr_dot; }
__device__ __forceinline__ float thr_dot(const SymMember& M, float hj2) {
    return fmaf(fmaxf(M.h2, hj2), 1.0f + 3.0f * kBandRel, M.bk_dot);
}
__device__ __forceinline__ float thr_diff(const DMember& M, float) { return M.h2hi; }
__device__ __forceinline__ float thr_dot(const DLMember& M, float) { return M.thr_dot_w; }
__device__ __forceinline__ float thr_diff(const DLMember& M, float) { return M.h2whi; }
__device__ __forceinline__ float thr_dot(const VMember& M, float) { return M.thr_dot; }
__device__ __forceinline__ float thr_diff(const VMember& M, float) { return M.h2hi; }
__device__ __forceinline__ float thr_diff(const SymMember& M, float hj2) {
    return fmaf(fmaxf(M.h2, hj2), 1.0f + 3.0f * kBandRel, M.bk);
}

// combine the slice copies of a member (lanes k, k+g, k+2g, ...)
__device__ __forceinline__ float xsum(float v, int o) { return v + __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ void slice_add(DMember& M, int o) {
    M.s0 = xsum(M.s0, o); M.c0 = xsum(M.c0, o); M.s1 = xsum(M.s1, o); M.c1 = xsum(M.c1, o);
    M.s2 = xsum(M.s2, o); M.c2 = xsum(M.c2, o);
    M.n += __shfl_xor_sync(0xffffffffu, M.n, o);
}
__device__ __forceinline__ void slice_add(DVMember& M, int o) {
    slice_add(static_cast<DMember&>(M), o);
    M.sd = xsum(M.sd, o); M.cd = xsum(M.cd, o); M.sx = xsum(M.sx, o); M.cx_ = xsum(M.cx_, o);
    M.sy = xsum(M.sy, o); M.cy_ = xsum(M.cy_, o); M.sz = xsum(M.sz, o); M.cz_ = xsum(M.cz_, o);
}
__device__ __forceinline__ void slice_add(HMember& M, int o) {
    M.sx = xsum(M.sx, o); M.cx_ = xsum(M.cx_, o); M.sy = xsum(M.sy, o); M.cy_ = xsum(M.cy_, o);
    M.sz = xsum(M.sz, o); M.cz_ = xsum(M.cz_, o); M.su = xsum(M.su, o); M.cu = xsum(M.cu, o);
    M.n += __shfl_xor_sync(0xffffffffu, M.n, o);
}
__device__ __forceinline__ void slice_add(VMember& M, int o) {
    M.sd = xsum(M.sd, o); M.cd = xsum(M.cd, o); M.sx = xsum(M.sx, o); M.cx_ = xsum(M.cx_, o);
    M.sy = xsum(M.sy, o); M.cy_ = xsum(M.cy_, o); M.sz = xsum(M.sz, o); M.cz_ = xsum(M.cz_, o);
    M.n += __shfl_xor_sync(0xffffffffu, M.n, o);
}
__device__ __forceinline__ void slice_add(HAMember& M, int o) {
    for (int k = 0; k < 3; ++k) { M.xb[k] = xsum(M.xb[k], o); M.vb[k] = xsum(M.vb[k], o); }
    M.mb = xsum(M.mb, o); M.hb = xsum(M.hb, o); M.rb = xsum(M.rb, o); M.Ab = xsum(M.Ab, o);
    M.n += __shfl_xor_sync(0xffffffffu, M.n, o);
}
__device__ __forceinline__ void slice_add(DAMember& M, int o) {
    for (int k = 0; k < 3; ++k) M.xb[k] = xsum(M.xb[k], o);
    M.mb = xsum(M.mb, o);
    M.n += __shfl_xor_sync(0xffffffffu, M.n, o);
}

// results of a member
template <int MODE>
__device__ __forceinline__ void write_result(const DMember& D, const SearchArgs& a) {
    if (MODE == kAcc) {
        a.o_s0[D.rank] = D.s0 - D.c0;
        a.o_s1[D.rank] = D.s1 - D.c1;
        if (a.o_s2) a.o_s2[D.rank] = D.s2 - D.c2;
        a.o_n[D.rank] = D.n;
    } else if (MODE == kCount) {
        a.x_cnt[a.perm[D.rank]] = D.n;
    }
}
template <int MODE>
__device__ __forceinline__ void write_result(const DVMember& D, const SearchArgs& a) {
    write_result<MODE>(static_cast<const DMember&>(D), a);
    if (MODE == kAcc)
        a.o_vsum[D.rank] = make_float4(D.sd - D.cd, D.sx - D.cx_, D.sy - D.cy_, D.sz - D.cz_);
}
template <int MODE>
__device__ __forceinline__ void write_result(const HMember& H, const SearchArgs& a) {
    if (MODE == kAcc && a.o_res4) {
        // key order: the members of a group are consecutive ranks, so these writes are
        // contiguous; a gather pass moves them to the caller's order
        a.o_res4[H.rank] = make_float4(H.sx - H.cx_, H.sy - H.cy_, H.sz - H.cz_, H.su - H.cu);
        a.o_rcnt[H.rank] = H.n - 1;   // the member itself was counted as a pair
        return;
    }
    int orig = a.perm[H.rank];
    if (MODE == kAcc) {
        a.o_acc[3 * (int64_t)orig] = H.sx - H.cx_;
        a.o_acc[3 * (int64_t)orig + 1] = H.sy - H.cy_;
        a.o_acc[3 * (int64_t)orig + 2] = H.sz - H.cz_;
        a.o_dudt[orig] = H.su - H.cu;
        if (a.o_nh) a.o_nh[orig] = H.n - 1;   // the member itself was counted as a pair
    } else if (MODE == kCount) {
        a.x_cnt[orig] = H.n;
    }
}
template <int MODE>
__device__ __forceinline__ void write_result(const HAMember& H, const SearchArgs& a) {
    if (MODE != kAcc) return;
    a.o_adj0[H.rank] = make_float4(H.xb[0], H.xb[1], H.xb[2], H.mb);
    a.o_adj1[H.rank] = make_float4(H.vb[0], H.vb[1], H.vb[2], 0.0f);
    a.o_adj2[H.rank] = make_float4(H.hb, H.rb, H.Ab, (float)H.n);
}
template <int MODE>
__device__ __forceinline__ void write_result(const VMember& V, const SearchArgs& a) {
    if (MODE != kAcc) return;
    if (a.o_res4) {
        a.o_res4[V.rank] = make_float4(V.rrho * (V.sd - V.cd), V.rrho * (V.sx - V.cx_), V.rrho * (V.sy - V.cy_),
                                       V.rrho * (V.sz - V.cz_));
        return;
    }
    const int orig = a.perm[V.rank];
    a.o_divv[orig] = V.rrho * (V.sd - V.cd);
    a.o_curl[3 * (int64_t)orig] = V.rrho * (V.sx - V.cx_);
    a.o_curl[3 * (int64_t)orig + 1] = V.rrho * (V.sy - V.cy_);
    a.o_curl[3 * (int64_t)orig + 2] = V.rrho * (V.sz - V.cz_);
}
template <int MODE>
__device__ __forceinline__ void write_result(const DAMember& D, const SearchArgs& a) {
    if (MODE != kAcc) return;
    a.o_adj3[D.rank] = make_float4(D.xb[0], D.xb[1], D.xb[2], D.mb);
}

// ---------------------------------------------------------------------------------
// Grouped form: one warp per group
// ---------------------------------------------------------------------------------

struct alignas(16) WalkSmem {
    unsigned long long bar;      // mbarrier of the tile copies
    uint32_t stack[kStackCap];   // node ranges: (first child << 3) | (count - 1)
    int2 ranges[kRangeCap];      // pending leaf ranges (first rank, count)
    int rpre[kRangeCap + 1];     // prefix of the pending counts
};

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Member slot layout of a lane: with group size g <= 32 a power of two, the warp
// holds S = 32 / g copies ("slices") of the g members and each slice filters a
// different subset of the candidates; otherwise the lane holds M members, one slice.
struct Layout {
    int S;       // slices
    int slice;   // this lane's slice
    int gw;      // members per slice row (min(g, 32))
};

__device__ __forceinline__ Layout make_layout(int g, int lane, bool allow_slices, int max_slices) {
    Layout L;
    L.gw = g < 32 ? g : 32;
    bool pow2 = (g & (g - 1)) == 0;
    L.S = (allow_slices && g < 32 && pow2) ? min(32 / g, max_slices) : 1;
    L.slice = L.S > 1 ? lane / g : 0;
    if (L.slice >= L.S) L.slice = L.S;   // lanes beyond the last slice hold no member
    return L;
}

// member index (within the group) held by slot mm of this lane; -1 if none
__device__ __forceinline__ int member_of(const Layout& L, int lane, int mm, int g) {
    int k;
    if (L.S > 1) {
        if (L.slice >= L.S) return -1;
        k = lane % g;
    } else {
        k = lane + 32 * mm;
    }
    return k < g ? k : -1;
}

// Member x candidate filter of one staged tile.  Phase A: for every chunk of 32 of
// the lane's slice, a bit mask of the candidates inside the member's FP32 threshold,
// tested in dot-product form |p|^2 - 2 p.m < h^2 - |m|^2 (three FMAs; its rounding
// stays inside the FP64 decision band).  Phase B: every lane walks its own set bits
// across all chunks (no per-chunk wait for the slowest lane) for the exact decision
// and the pair terms; forward partial sums are folded into the compensated totals
// after the tile.
template <class K, int MODE, int M, bool WRAP>
__device__ __forceinline__ void filter_tile(typename K::Tile& T, const Layout& L, typename K::Member* mem, int nt,
                                            const SearchArgs& a, LocalCounters& lc, int lane) {
    const int S = L.S;
    if (L.slice >= S) return;
    const int cnt_slice = (nt > L.slice) ? (nt - L.slice + S - 1) / S : 0;
    const int nch = ((nt + S - 1) / S + 31) >> 5;
#pragma unroll
    for (int mm = 0; mm < M; ++mm) {
        auto& Mb = mem[mm];
        const float mx = Mb.mx, my = Mb.my, mz = Mb.mz;
        const float ax = -2.0f * mx, ay = -2.0f * my, az = -2.0f * mz;
        for (int c = 0; c < nch; ++c) {
            uint32_t mask = 0u;
            const int j0 = L.slice + S * (c << 5);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int j = j0 + q * S;
                const float4 cp = T.p[j];
                float hj2 = 0.0f;
                if constexpr (K::sym) hj2 = T.o[j].x;
                bool pass;
                if constexpr (!WRAP) {
                    float t = fmaf(cp.x, ax, fmaf(cp.y, ay, fmaf(cp.z, az, cp.w)));
                    pass = t < thr_dot(Mb, hj2);
                } else {
                    float dx = rel_diff<true>(cp.x, mx), dy = rel_diff<true>(cp.y, my), dz = rel_diff<true>(cp.z, mz);
                    float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    pass = r2 < thr_diff(Mb, hj2);
                }
                mask |= (pass ? 1u : 0u) << q;
            }
            T.masks[(c << 5) + lane] = mask;
            if (Mb.rank >= 0) lc.tests += min(32, cnt_slice - (c << 5));
        }
        int c = 0;
        uint32_t cur = T.masks[lane];
        for (;;) {
            while (cur == 0u) {
                if (++c >= nch) break;
                cur = T.masks[(c << 5) + lane];
            }
            if (cur == 0u) break;
            const int q = __ffs(cur) - 1;
            cur &= cur - 1u;
            tile_pair<MODE, WRAP>(Mb, a, T, L.slice + S * ((c << 5) + q), lc);
        }
        if (MODE == kAcc) flush(Mb);
    }
}

// Filter of the nt converted candidates held in the tile: NaN dummies up to whole chunks of
// 32 in every slice, then the member x candidate filter (dot form unless the group wraps).
template <class K, int MODE, int M>
__device__ __forceinline__ void filter_staged(typename K::Tile& T, const Layout& L, typename K::Member* mem, int nt,
                                              const SearchArgs& a, LocalCounters& lc, int lane, bool wrap_safe) {
    const int padded = L.S * ((((nt + L.S - 1) / L.S) + 31) >> 5) * 32;
    const float nanv = __int_as_float(0x7fffffff);
    for (int t = nt + lane; t < padded; t += 32) T.p[t] = make_float4(nanv, nanv, nanv, nanv);
    __syncwarp();
    if (wrap_safe) filter_tile<K, MODE, M, false>(T, L, mem, nt, a, lc, lane);
    else filter_tile<K, MODE, M, true>(T, L, mem, nt, a, lc, lane);
    __syncwarp();
}

// Work item of the grouped kernels: members U[base, base + cnt), the walk's start node
// (a root of the forest), the group size of the member layout and the slice limit.
struct GroupDesc {
    int base, cnt, root, g, smax;
};

__device__ __forceinline__ GroupDesc group_desc(const SearchArgs& a, int gid) {
    GroupDesc d;
    d.root = 0;
    d.g = a.g;
    d.smax = 32;
    if (a.groups4) {
        const int4 G = a.groups4[gid];
        d.base = G.x;
        d.cnt = G.y;
        d.root = G.z;
        d.g = G.w & 0xff;
        d.smax = (G.w >> 8) & 0xff;   // bits 16.. carry the box's leaf size
    } else if (a.groups) {
        const int2 G = a.groups[gid];
        d.base = G.x;
        d.cnt = G.y;
    } else {
        d.base = gid * a.g;
        d.cnt = min(a.g, a.nu - d.base);
    }
    // member slots: the group's count rounded up to a power of two, so that a group cut
    // smaller by the split keeps every lane busy with more slices
    const int p2 = d.cnt <= 1 ? 1 : 1 << (32 - __clz(d.cnt - 1));
    d.g = min(d.g, p2);
    return d;
}

__device__ __forceinline__ int group_count(const SearchArgs& a) {
    return a.ngroups_dev ? *a.ngroups_dev : a.ngroups;
}

// Group centre: the fixed-point position of the first member (lowest slot of the
// lowest lane), or the centre of the members' bounding box (offsets from the first
// member are exact minimum-image integers).  Ranks < 0 are empty slots.  Returns
// false when the group has no member.
template <int M>
__device__ __forceinline__ bool group_centre(const SearchArgs& a, const int (&rk)[M], uint32_t& cx, uint32_t& cy,
                                             uint32_t& cz) {
    int ref = -1;
#pragma unroll
    for (int mm = 0; mm < M; ++mm) {
        const unsigned b = __ballot_sync(0xffffffffu, rk[mm] >= 0);
        const int cand = __shfl_sync(0xffffffffu, rk[mm], b ? __ffs(b) - 1 : 0);
        if (ref < 0 && b) ref = cand;
    }
    if (ref < 0) return false;
    const uint4 P0 = a.pfix[ref];
    cx = P0.x;
    cy = P0.y;
    cz = P0.z;
    if (a.centre_box) {
        int lox = 0, loy = 0, loz = 0, hix = 0, hiy = 0, hiz = 0;
#pragma unroll
        for (int mm = 0; mm < M; ++mm) {
            if (rk[mm] >= 0) {
                const uint4 P = a.pfix[rk[mm]];
                const int dx = (int32_t)(P.x - cx), dy = (int32_t)(P.y - cy), dz = (int32_t)(P.z - cz);
                lox = min(lox, dx); hix = max(hix, dx);
                loy = min(loy, dy); hiy = max(hiy, dy);
                loz = min(loz, dz); hiz = max(hiz, dz);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lox = min(lox, __shfl_xor_sync(0xffffffffu, lox, o));
            loy = min(loy, __shfl_xor_sync(0xffffffffu, loy, o));
            loz = min(loz, __shfl_xor_sync(0xffffffffu, loz, o));
            hix = max(hix, __shfl_xor_sync(0xffffffffu, hix, o));
            hiy = max(hiy, __shfl_xor_sync(0xffffffffu, hiy, o));
            hiz = max(hiz, __shfl_xor_sync(0xffffffffu, hiz, o));
        }
        cx += (uint32_t)(int32_t)(((int64_t)lox + hix) >> 1);
        cy += (uint32_t)(int32_t)(((int64_t)loy + hiy) >> 1);
        cz += (uint32_t)(int32_t)(((int64_t)loz + hiz) >> 1);
    }
    return true;
}

// Morton index of a cell of level l (l bits per axis, axis 0 most significant).
__device__ __forceinline__ uint32_t cell_morton(uint32_t x, uint32_t y, uint32_t z, int l) {
    uint32_t m = 0;
    for (int b = l - 1; b >= 0; --b) m = (m << 3) | (((x >> b) & 1u) << 2) | (((y >> b) & 1u) << 1) | ((z >> b) & 1u);
    return m;
}

// First node of the walk: the node of the deepest cell (level <= kStartLevels) of the
// tree rooted at `root` (tab: that tree's start table) that
// holds the whole search sphere (centre C, radius Rb in box units).  Every particle
// within the sphere lies in that cell and hence in that node's subtree (a node is the
// set of particles whose keys share its cell's prefix).  Cells the tree did not reach
// fall back to the nearest ancestor cell with a node.
__device__ __forceinline__ int walk_start(const int32_t* __restrict__ tab, int root, uint32_t cx, uint32_t cy,
                                          uint32_t cz, float Rb) {
    // radius in fixed-point units, rounded up, plus the sub-unit offsets of the positions
    const double Ru = ceil((double)Rb * 4294967296.0 * (1.0 + 1e-6)) + 2.0;
    if (!(Ru < 2147483648.0)) return root;
    const int64_t r = (int64_t)Ru;
    int lvl = kStartLevels;
    const uint32_t c3[3] = {cx, cy, cz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int64_t lo = (int64_t)c3[ax] - r, hi = (int64_t)c3[ax] + r;
        if (lo < 0 || hi > 0xffffffffll) lvl = 0;   // the sphere wraps around the box
        else lvl = min(lvl, __clz((uint32_t)lo ^ (uint32_t)hi));
    }
    for (; lvl >= 1; --lvl) {
        const int nd = tab[start_table_offset(lvl) +
                           cell_morton(cx >> (32 - lvl), cy >> (32 - lvl), cz >> (32 - lvl), lvl)];
        if (nd >= 0) return nd;
    }
    return root;
}

// One group's walk from node `root` and the member x candidate filter of every staged
// tile (the members are initialised relative to the centre C).  kSupFill writes the
// superset at sup_pos + sup_n; sup_n accumulates the candidates.
// Returns false if a tile copy timed out: the warp must then stop taking work.
template <class K, int MODE, int M>
__device__ __forceinline__ bool group_search(const SearchArgs& a, WalkSmem& W, typename K::Tile& T, const Layout& L,
                                             typename K::Member (&mem)[M], uint32_t cx, uint32_t cy, uint32_t cz,
                                             int root, LocalCounters& lc, uint32_t& tma_phase, int lane,
                                             int64_t sup_pos, int64_t& sup_n) {
    constexpr int TCAP = K::cap;
    constexpr bool kSup = (MODE == kSupCount || MODE == kSupFill);
    const uint32_t lt = (1u << lane) - 1u;
    float rlane = 0.0f, hlane = 0.0f;   // walk radius ingredients of this lane
#pragma unroll
    for (int mm = 0; mm < M; ++mm) radius_terms(mem[mm], rlane, hlane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rlane = fmaxf(rlane, __shfl_xor_sync(0xffffffffu, rlane, o));
        hlane = fmaxf(hlane, __shfl_xor_sync(0xffffffffu, hlane, o));
    }
    // density: R_s = max_k (|m_k| + h_k); symmetric: R_g = max_k |m_k|, hmax_g
    const float Rd2 = radius2_units(rlane);
    const float Rg = rlane, hmax_g = hlane;
    // every relevant pair difference is already the nearest image when the group's
    // reach stays below half the box (symmetric: with the largest h of the tree)
    const float reach = K::sym ? Rg + fmaxf(hmax_g, __uint_as_float(a.ncen[root].w)) : rlane;
    const bool wrap_safe = reach < 0.49f;
    // the start table of the walk's tree (one per box of a forest, whose roots are the
    // first nodes)
    const int start = a.start_tab ? walk_start(a.start_tab + (size_t)root * kStartTableSize, root, cx, cy, cz, reach)
                                  : root;

    // The stack lives in shared memory (at most a.stack_cap entries); when it fills up,
    // its oldest entries move to this warp's overflow area in global memory, which holds
    // the bottom of the stack and refills the shared part when that runs empty.
    uint32_t* spill = a.stack_spill + (size_t)(blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) * kSpillCap;
    int sp = 1, gsp = 0;
    if (lane == 0) W.stack[0] = (uint32_t)start << 3;   // one node
    int nr = 0, pending = 0;
    int nf = 0;   // converted candidates held in the tile, waiting for the filter
    __syncwarp();
    for (;;) {
        while ((sp > 0 || gsp > 0) && sp <= a.stack_cap - 32 && pending < TCAP - nf && nr <= kRangeCap - 32) {
            if (sp == 0) {
                const int m = min(gsp, 32);
                if (lane < m) W.stack[lane] = spill[gsp - m + lane];
                gsp -= m;
                sp = m;
                __syncwarp();
            }
            // take range entries from the top of the stack, up to 32 nodes
            uint32_t ent = 0;
            int ecnt = 0;
            if (lane < sp) {
                ent = W.stack[sp - 1 - lane];
                ecnt = (int)(ent & 7u) + 1;
            }
            int incl = warp_incl_scan(ecnt, lane);
            bool take = (lane < sp) && (incl <= 32);
            unsigned tm = __ballot_sync(0xffffffffu, take);
            int nent = __popc(tm);
            int nnodes = __shfl_sync(0xffffffffu, incl, nent - 1);
            // node slot l belongs to the taken entry whose first slot is the highest entry
            // start <= l (the starts as a bit mask; entries sit on lanes 0 .. nent-1)
            const unsigned starts = __reduce_or_sync(0xffffffffu, take ? 1u << (incl - ecnt) : 0u);
            const unsigned below = (lane == 31) ? starts : (starts & ((2u << lane) - 1u));
            const int e_of = max(__popc(below) - 1, 0);
            const uint32_t my_ent = __shfl_sync(0xffffffffu, ent, e_of);
            sp -= nent;
            int node = lane < nnodes ? (int)(my_ent >> 3) + (lane - (31 - __clz(below))) : -1;
            bool open = false, leaf = false;
            int4 lk = make_int4(0, 0, -1, 0);
            int nch = 0;
            if (node >= 0) {
                uint4 cen = a.ncen[node];
                float4 ext = a.next[node];
                lk = a.nlink[node];
                nch = __float_as_int(ext.w);
                float gap2 = node_gap2(cen, ext, cx, cy, cz);
                float R2;
                if constexpr (!K::sym) R2 = Rd2;
                else R2 = radius2_units(Rg + fmaxf(hmax_g, __uint_as_float(cen.w)));
                open = gap2 <= R2;
                leaf = lk.z < 0;
            }
            lc.nodes += (lane == 0) ? nnodes : 0;
            bool emit = open && leaf && lk.y > 0;
            unsigned em = __ballot_sync(0xffffffffu, emit);
            if (emit) {
                int pos = nr + __popc(em & lt);
                W.ranges[pos] = make_int2(lk.x, lk.y);
            }
            nr += __popc(em);
            int add = emit ? lk.y : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
            pending += add;
            bool push = open && !leaf;
            unsigned pm = __ballot_sync(0xffffffffu, push);
            const int npush = __popc(pm);
            if (push) W.stack[sp + __popc(pm & lt)] = ((uint32_t)lk.z << 3) | (uint32_t)(nch - 1);
            sp += npush;
            lc.max_stack = max(lc.max_stack, sp + gsp);
            __syncwarp();
        }
        const bool walk_done = (sp == 0 && gsp == 0);
        if (kSup) {
            if (nr > 0) {
                // superset export: every pending range's particles, in walk order
                int run = 0;
                for (int e0 = 0; e0 < nr; e0 += 32) {
                    const int e = e0 + lane;
                    const int c = e < nr ? W.ranges[e].y : 0;
                    const int inc = warp_incl_scan(c, lane);
                    if (e < nr) W.rpre[e] = run + inc - c;
                    run += __shfl_sync(0xffffffffu, inc, 31);
                }
                __syncwarp();
                lc.cands += (lane == 0) ? run : 0;
                if (MODE == kSupFill) {
                    for (int e = lane >> 4; e < nr; e += 2) {
                        const int rb = W.rpre[e];
                        const int2 R = W.ranges[e];
                        for (int gt = rb + (lane & 15); gt < rb + R.y; gt += 16) {
                            const int64_t q = sup_pos + sup_n + gt;
                            if (q < a.x_cap) a.x_idx[q] = a.perm[R.x + (gt - rb)];
                            else atomicOr(a.err, kErrCap);
                        }
                    }
                }
                sup_n += run;
                nr = 0;
                pending = 0;
                __syncwarp();
            }
        } else {
            // Stage the pending ranges from their front into the tile's free part [nf, TCAP)
            // (what does not fit stays pending for the next tile) and filter whenever the tile
            // is full, so that every tile but a group's last holds TCAP candidates.
            for (;;) {
                const int room = TCAP - nf;
                if (!(nr > 0 && (walk_done || pending >= room || nr > kRangeCap - 32))) break;
                const int nt = min(pending, room);
                int run = 0;
                for (int e0 = 0; e0 < nr; e0 += 32) {
                    const int e = e0 + lane;
                    const int c = e < nr ? W.ranges[e].y : 0;
                    const int inc = warp_incl_scan(c, lane);
                    if (e < nr) W.rpre[e] = run + inc - c;
                    run += __shfl_sync(0xffffffffu, inc, 31);
                }
                __syncwarp();
                lc.cands += (lane == 0) ? nt : 0;
                // bulk copies of every SoA array; ranges adjacent in memory (consecutive
                // leaves of the walk usually are) are merged into one copy, issued by the
                // first range of the run (or of a 32-range block)
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_expect_tx(&W.bar, (uint32_t)nt * K::bytes);
                __syncwarp();
                int nfull = 0;   // ranges consumed entirely by this chunk
                for (int eb = 0; eb < nr; eb += 32) {
                    const int e = eb + lane;
                    int rb = 0, src = 0, dst = 0, cnt = 0;
                    bool valid = false, cont = false;
                    if (e < nr) {
                        rb = W.rpre[e];
                        valid = rb < nt;
                    }
                    if (valid) {
                        const int2 R = W.ranges[e];
                        src = R.x;
                        dst = nf + rb;
                        cnt = min(R.y, nt - rb);
                        if (lane > 0) {
                            const int2 Q = W.ranges[e - 1];
                            cont = Q.x + Q.y == R.x;
                        }
                        for (int k = 0; k < cnt; ++k) T.r[dst + k] = src + k;
                    }
                    nfull += __popc(__ballot_sync(0xffffffffu, valid && cnt == W.ranges[e < nr ? e : 0].y));
                    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
                    if (vmask == 0u) break;
                    const bool head = valid && !cont;
                    const unsigned hmask = __ballot_sync(0xffffffffu, head);
                    const int last = 31 - __clz(vmask);
                    const int chunk_end = __shfl_sync(0xffffffffu, dst + cnt, last);
                    const unsigned above = (lane == 31) ? 0u : (hmask >> (lane + 1)) << (lane + 1);
                    const int nxt = above ? __ffs(above) - 1 : 0;
                    const int nxt_dst = __shfl_sync(0xffffffffu, dst, nxt);
                    if (head) {
                        const int runlen = (above ? nxt_dst : chunk_end) - dst;
                        stage_run(T, a, dst, src, (uint32_t)runlen * 16u, &W.bar);
                    }
                    if (vmask != 0xffffffffu) break;
                }
                // the chunk leaves the pending list: drop the consumed ranges, shorten a
                // partly consumed one, move the rest to the front
                {
                    const int keep_n = nr - nfull;
                    int2 r0 = make_int2(0, 0), r1 = make_int2(0, 0);
                    if (lane < keep_n) r0 = W.ranges[nfull + lane];
                    if (lane + 32 < keep_n) r1 = W.ranges[nfull + lane + 32];
                    if (lane == 0 && keep_n > 0) {
                        const int used = nt - W.rpre[nfull];   // > 0 only for a partly consumed range
                        if (used > 0) { r0.x += used; r0.y -= used; }
                    }
                    __syncwarp();
                    if (lane < keep_n) W.ranges[lane] = r0;
                    if (lane + 32 < keep_n) W.ranges[lane + 32] = r1;
                    __syncwarp();
                    nr = keep_n;
                    pending -= nt;
                }
                if (!mbar_wait_bounded(&W.bar, tma_phase, a.err)) {
                    // The chunk never completed: nothing of it may be used, and the barrier's
                    // phase no longer matches tma_phase.  Give the copies in flight one more
                    // bounded wait to land in shared memory, then the warp abandons its work
                    // (the timeout flag is set; the call reports ETIMEOUT).
                    mbar_wait_bounded(&W.bar, tma_phase, a.err);
                    return false;
                }
                tma_phase ^= 1u;
                // in place: fixed point -> coordinates relative to the centre
                for (int t = nf + lane; t < nf + nt; t += 32) {
                    const uint4 P = *reinterpret_cast<const uint4*>(&T.p[t]);
                    const float4 O = T.o[t];
                    const float px = rel_coord(P.x, O.x, cx), py = rel_coord(P.y, O.y, cy),
                                pz = rel_coord(P.z, O.z, cz);
                    T.p[t] = make_float4(px, py, pz, fmaf(px, px, fmaf(py, py, pz * pz)));
                    if constexpr (K::sym) {
                        const float hj = __uint_as_float(P.w);
                        T.o[t] = make_float4(hj * hj, O.w, 0.0f, 0.0f);
                    }
                }
                __syncwarp();
                nf += nt;
                if (nf >= TCAP) {
                    filter_staged<K, MODE, M>(T, L, mem, nf, a, lc, lane, wrap_safe);
                    nf = 0;
                }
            }
            if (walk_done && nf > 0) {
                filter_staged<K, MODE, M>(T, L, mem, nf, a, lc, lane, wrap_safe);
                nf = 0;
            }
        }
        if (sp > a.stack_cap - 32) {
            // the next step could push 32 entries: the oldest (up to 32, the bottom of the
            // shared part) move to the top of the overflow area, which stays below the
            // shared part, so the whole stack remains last in, first out
            const int ev = min(32, sp);
            if (gsp + ev > kSpillCap) atomicOr(a.err, kErrStack);
            else if (lane < ev) spill[gsp + lane] = W.stack[lane];
            __syncwarp();
            for (int b = 0; b < sp - ev; b += 32) {
                const uint32_t v = (b + lane < sp - ev) ? W.stack[ev + b + lane] : 0u;
                __syncwarp();
                if (b + lane < sp - ev) W.stack[b + lane] = v;
                __syncwarp();
            }
            gsp = min(gsp + ev, kSpillCap);
            sp -= ev;
        }
        if (sp == 0 && gsp == 0) break;
    }
    return true;
}

// One work item of the grouped kernels: set-up, search, results.  Returns false if the
// warp must stop taking work (a tile copy timed out).
template <class K, int MODE, int M>
__device__ __forceinline__ bool process_group(const SearchArgs& a, WalkSmem& W, typename K::Tile& T, int gid,
                                              LocalCounters& lc, uint32_t& tma_phase, int lane) {
    using Member = typename K::Member;
    constexpr bool kSup = (MODE == kSupCount || MODE == kSupFill);
    const GroupDesc d = group_desc(a, gid);
    const Layout L = make_layout(d.g, lane, MODE == kAcc, min(K::cap / 32, d.smax));
    int rk[M];
#pragma unroll
    for (int mm = 0; mm < M; ++mm) {
        const int k = member_of(L, lane, mm, d.g);
        rk[mm] = (k >= 0 && k < d.cnt) ? a.U[d.base + k] : -1;
    }
    uint32_t cx = 0, cy = 0, cz = 0;
    if (!group_centre<M>(a, rk, cx, cy, cz)) return true;
    Member mem[M];
#pragma unroll
    for (int mm = 0; mm < M; ++mm) member_init(mem[mm], a, rk[mm], cx, cy, cz);
    if constexpr (K::id == kKindDensityList) {
        // list slot = the member's index in the work list; sub-list of this lane's slice
        static_assert(M == 1, "the recycled iteration keeps lists for one member per lane");
        const int k = member_of(L, lane, 0, d.g);
        if (mem[0].rank >= 0) {
            mem[0].lsub = kListCap / L.S;
            mem[0].lptr = a.o_list + (int64_t)(d.base + k) * kListCap + L.slice * mem[0].lsub;
        }
    }
    // export: write positions of every slot
    if (MODE == kFill) {
#pragma unroll
        for (int mm = 0; mm < M; ++mm)
            if (mem[mm].rank >= 0) mem[mm].xpos = a.x_off[a.perm[mem[mm].rank]];
    }
    int64_t sup_pos = 0, sup_n = 0;
    if (MODE == kSupFill) sup_pos = a.x_off[gid];
    if (!group_search<K, MODE, M>(a, W, T, L, mem, cx, cy, cz, d.root, lc, tma_phase, lane, sup_pos, sup_n))
        return false;
    // the symmetric sums count the member itself as a pair at r = 0 (once, in slice 0)
    constexpr bool kSelfPair = MODE == kAcc && (K::id == kKindHydro || K::id == kKindHydroAdj);
#pragma unroll
    for (int mm = 0; mm < M; ++mm)
        lc.pairs += mem[mm].n - ((kSelfPair && L.slice == 0 && mem[mm].rank >= 0) ? 1 : 0);
    if (kSup) {
        if (MODE == kSupCount && lane == 0) a.x_cnt[gid] = sup_n;
        return true;
    }
    if constexpr (K::id == kKindDensityList) {
        // the member's slice-0 lane records its sub-list lengths, S and whether all fit
        int cnt[4];
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) {
            const int src = L.S > 1 ? sl * d.g + (lane & (d.g - 1)) : lane;
            const int v = __shfl_sync(0xffffffffu, mem[0].lcnt, (sl < L.S && src < 32) ? src : lane);
            cnt[sl] = sl < L.S ? v : 0;
        }
        if (L.slice == 0 && mem[0].rank >= 0) {
            const int lsub = kListCap / L.S;
            const bool ok = cnt[0] <= lsub && cnt[1] <= lsub && cnt[2] <= lsub && cnt[3] <= lsub;
            const int slot = d.base + member_of(L, lane, 0, d.g);
            a.o_lrec[slot] = make_int4(ok ? cnt[0] | (cnt[1] << 16) : 0, ok ? cnt[2] | (cnt[3] << 16) : 0, L.S,
                                       ok ? 1 : 0);
            a.o_lhw[slot] = a.h64[mem[0].rank] * a.list_widen;
            a.o_lslot[mem[0].rank] = slot;
        }
    }
    if (L.S > 1) {
#pragma unroll
        for (int mm = 0; mm < M; ++mm)
            for (int o = d.g; o < 32; o <<= 1) slice_add(mem[mm], o);
    }
    if (L.slice == 0) {
#pragma unroll
        for (int mm = 0; mm < M; ++mm) {
            if (mem[mm].rank >= 0) write_result<MODE>(mem[mm], a);
        }
    }
    return true;
}

__device__ __forceinline__ int next_item(const SearchArgs& a, int lane) {
    int gid = 0;
    if (lane == 0) gid = atomicAdd(a.work, 1);
    return __shfl_sync(0xffffffffu, gid, 0);
}

template <class K, int MODE, int M>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, M == 1 ? K::min_blocks : 0)
k_group(SearchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WalkSmem& W = reinterpret_cast<WalkSmem*>(smem_raw)[wib];
    auto& T = reinterpret_cast<typename K::Tile*>(smem_raw + kWarpsPerBlock * sizeof(WalkSmem))[wib];
    LocalCounters lc;
    uint32_t tma_phase = 0u;
    if (lane == 0) mbar_init(&W.bar, 1u);
    __syncwarp();
    const int ng = group_count(a);
    for (;;) {
        const int gid = next_item(a, lane);
        if (gid >= ng) break;
        if (!process_group<K, MODE, M>(a, W, T, gid, lc, tma_phase, lane)) break;
    }
    flush_counters(a, lc, lane);
}

// Two kinds of work item in one persistent queue: the groups of a0 (kind K0) first,
// then those of a1 (kind K1).  Both share the work counter of a0.
template <class K0, class K1, int M>
__global__ void __launch_bounds__(kWarpsPerBlock * 32,
                                  M > 1 ? 0 : (K0::min_blocks < K1::min_blocks ? K0::min_blocks : K1::min_blocks))
k_group_pair(SearchArgs a0, SearchArgs a1) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr size_t kTileBytes = sizeof(typename K0::Tile) > sizeof(typename K1::Tile) ? sizeof(typename K0::Tile)
                                                                                        : sizeof(typename K1::Tile);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WalkSmem& W = reinterpret_cast<WalkSmem*>(smem_raw)[wib];
    unsigned char* tile = smem_raw + kWarpsPerBlock * sizeof(WalkSmem) + wib * kTileBytes;
    LocalCounters lc;
    uint32_t tma_phase = 0u;
    if (lane == 0) mbar_init(&W.bar, 1u);
    __syncwarp();
    const int n0 = group_count(a0), n1 = group_count(a1);
    for (;;) {
        const int gid = next_item(a0, lane);
        if (gid >= n0 + n1) break;
        const bool ok =
            gid < n0 ? process_group<K0, kAcc, M>(a0, W, *reinterpret_cast<typename K0::Tile*>(tile), gid, lc,
                                                  tma_phase, lane)
                     : process_group<K1, kAcc, M>(a1, W, *reinterpret_cast<typename K1::Tile*>(tile), gid - n0, lc,
                                                  tma_phase, lane);
        if (!ok) break;
    }
    flush_counters(a0, lc, lane);
}

// Density with the smoothing-length iteration inside the group (no host loop, no
// regrouping): after every walk + filter the members update h in FP64 (the same
// Newton / bisection step as k_hsml_update); converged members leave the group, the
// centre and radius are recomputed over the remaining ones and the group walks again,
// until every member has converged or reached max_iter passes.  A particle's density
// at h depends only on the positions and its own h, so the iterates equal those of the
// pass-by-pass iteration (up to the order of the FP32 sums).
__device__ __forceinline__ bool hsml_step(const SearchArgs& a, const IterArgs& it, int r, double& h, double& lo,
                                          double& hi, float s0, float s1, int nngb, int pass, bool writer) {
    const double kPi = 3.14159265358979323846;
    const double m = (double)a.poff[r].w;
    const double sigma = 8.0 / (kPi * h * h * h);
    const double rho = sigma * (double)s0;
    const double drho = -sigma / h * (double)s1;
    const double neff = 4.0 * kPi / 3.0 * h * h * h * rho / m;
    const bool done = fabs(neff - it.nngb) <= it.tol;
    if (done || pass >= it.max_iter) {
        if (writer) {
            const int orig = a.perm[r];
            it.rho[orig] = (float)rho;
            it.drhodh[orig] = (float)drho;
            it.fgrad[orig] = (float)(1.0 / (1.0 + h / (3.0 * rho) * drho));
            it.nngb_out[orig] = nngb;
            if (it.iters) it.iters[orig] = pass;
            it.h_out[orig] = h;
            if (!done) atomicAdd(it.nfail, 1);
            if (it.max_pass) atomicMax(it.max_pass, pass);
        }
        return true;
    }
    if (neff < it.nngb) lo = h; else hi = h;
    const double g = 4.0 * kPi / 3.0 * h * h * h * rho - it.nngb * m;
    const double gp = 4.0 * kPi * h * h * rho + 4.0 * kPi / 3.0 * h * h * h * drho;
    double hn = h - g / gp;
    const double cbrt2 = 1.2599210498948731647672106;
    if (!(hn > lo && hn < hi) || !isfinite(hn)) {
        if (isinf(hi)) hn = h * cbrt2;
        else if (lo == 0.0) hn = h / cbrt2;
        else hn = cbrt(0.5 * (lo * lo * lo + hi * hi * hi));
    }
    hn = fmin(hn, 0.49);   // the minimum image needs h < 1/2 (such a particle cannot converge)
    h = hn;
    if (writer) {
        it.h64[r] = hn;
        it.pfix[r].w = __float_as_uint((float)hn);
    }
    return false;
}

template <int M>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, M == 1 ? 6 : 0)
k_group_dens_iter(SearchArgs a, IterArgs it) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WalkSmem& W = reinterpret_cast<WalkSmem*>(smem_raw)[wib];
    DensTile& T = reinterpret_cast<DensTile*>(smem_raw + kWarpsPerBlock * sizeof(WalkSmem))[wib];
    LocalCounters lc;
    uint32_t tma_phase = 0u;
    if (lane == 0) mbar_init(&W.bar, 1u);
    __syncwarp();
    const int ng = group_count(a);
    bool alive = true;
    while (alive) {
        const int gid = next_item(a, lane);
        if (gid >= ng) break;
        const GroupDesc d = group_desc(a, gid);
        const Layout L = make_layout(d.g, lane, true, min(kTileD / 32, d.smax));
        int rk[M];
        double hc[M], lo[M], hi[M];
#pragma unroll
        for (int mm = 0; mm < M; ++mm) {
            const int k = member_of(L, lane, mm, d.g);
            rk[mm] = (k >= 0 && k < d.cnt) ? a.U[d.base + k] : -1;
            hc[mm] = rk[mm] >= 0 ? a.h64[rk[mm]] : 1.0;
            lo[mm] = 0.0;
            hi[mm] = __longlong_as_double(0x7ff0000000000000ll);
        }
        for (int pass = 1;; ++pass) {
            uint32_t cx = 0, cy = 0, cz = 0;
            if (!group_centre<M>(a, rk, cx, cy, cz)) break;
            DMember mem[M];
#pragma unroll
            for (int mm = 0; mm < M; ++mm) member_init(mem[mm], a, rk[mm], cx, cy, cz);
            int64_t sup_n = 0;
            if (!group_search<KDens, kAcc, M>(a, W, T, L, mem, cx, cy, cz, d.root, lc, tma_phase, lane, 0, sup_n)) {
                alive = false;
                break;
            }
#pragma unroll
            for (int mm = 0; mm < M; ++mm) lc.pairs += mem[mm].n;
            if (L.S > 1) {
#pragma unroll
                for (int mm = 0; mm < M; ++mm)
                    for (int o = d.g; o < 32; o <<= 1) slice_add(mem[mm], o);
            }
#pragma unroll
            for (int mm = 0; mm < M; ++mm) {
                if (rk[mm] >= 0 &&
                    hsml_step(a, it, rk[mm], hc[mm], lo[mm], hi[mm], mem[mm].s0 - mem[mm].c0, mem[mm].s1 - mem[mm].c1,
                              mem[mm].n, pass, L.slice == 0))
                    rk[mm] = -1;
            }
            // the new h (global memory) is read by the next pass's FP64 re-tests
            __syncwarp();
        }
    }
    flush_counters(a, lc, lane);
}

// ---------------------------------------------------------------------------------
// Individual form: one thread per particle, depth-first walk with skip pointers
// ---------------------------------------------------------------------------------

template <int KIND, int MODE>
__global__ void __launch_bounds__(128) k_indiv(SearchArgs a) {
    const int lane = threadIdx.x & 31;
    LocalCounters lc;
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < a.nu) {
        const int rank = a.U[u];
        uint4 P = a.pfix[rank];
        const uint32_t cx = P.x, cy = P.y, cz = P.z;
        DMember dm;
        HMember hm;
        float Rbox;
        if (KIND == 0) {
            member_init(dm, a, rank, cx, cy, cz);
            Rbox = (float)a.h64[rank];
            if (MODE == kFill) dm.xpos = a.x_off[a.perm[rank]];
        } else {
            member_init(hm, a, rank, cx, cy, cz);
            Rbox = hm.h;
            if (MODE == kFill) hm.xpos = a.x_off[a.perm[rank]];
        }
        const float R2d = radius2_units(Rbox);
        int node = 0;
        while (node >= 0) {
            uint4 cen = a.ncen[node];
            float4 ext = a.next[node];
            int4 lk = a.nlink[node];
            lc.nodes++;
            float gap2 = node_gap2(cen, ext, cx, cy, cz);
            float R2 = KIND == 0 ? R2d : radius2_units(fmaxf(Rbox, __uint_as_float(cen.w)));
            if (gap2 <= R2) {
                if (lk.z < 0) {
                    lc.cands += lk.y;
                    lc.tests += lk.y;
                    for (int q = lk.x; q < lk.x + lk.y; ++q) {
                        uint4 Q = a.pfix[q];
                        float4 O = a.poff[q];
                        float4 rel = make_float4(rel_coord(Q.x, O.x, cx), rel_coord(Q.y, O.y, cy),
                                                 rel_coord(Q.z, O.z, cz), O.w);
                        if (KIND == 0) {
                            density_pair<MODE>(dm, a, rel, O.w, q, lc);
                        } else {
                            float hj = __uint_as_float(Q.w);
                            float dx = rel.x - hm.mx, dy = rel.y - hm.my, dz = rel.z - hm.mz;
                            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            float thr = fmaf(fmaxf(hm.h2, hj * hj), 1.0f + 3.0f * kBandRel, hm.bk);
                            if (r2 < thr) {
                                float4 H0 = a.hyd0[q], H1 = a.hyd1[q];
                                hydro_pair<MODE>(hm, a, rel, make_float4(hj * hj, O.w, 0.0f, 0.0f), H0, H1, q, lc);
                            }
                        }
                    }
                    if (MODE == kAcc) {
                        if (KIND == 0) flush(dm);
                        else flush(hm);
                    }
                    node = lk.w;
                } else {
                    node = lk.z;
                }
            } else {
                node = lk.w;
            }
        }
        lc.pairs += (KIND == 0) ? dm.n : hm.n - (MODE == kAcc ? 1 : 0);
        if (KIND == 0) write_result<MODE>(dm, a);
        else write_result<MODE>(hm, a);
    }
    flush_counters(a, lc, lane);
}

// ---------------------------------------------------------------------------------
// Grouping: chunks of g consecutive entries of the work list, each split (recursively)
// while the group's search sphere, ((sqrt(3)/2) box width + h_min)^3, exceeds split *
// (members) member spheres h_min^3.  The cut is at the largest gap in key order (see
// below).  A criterion on the walk's exact radius, max_k (|x_k - c| + h_k), against the
// smallest h split the same groups of the full workload but kept fewer members per walk
// on sparse active sets made of runs, 1.2-2x slower there at g >= 16.
// ---------------------------------------------------------------------------------

__global__ void k_split_groups(const int32_t* __restrict__ U, int nu, int g, float split,
                               const uint4* __restrict__ pfix, const double* __restrict__ h64,
                               int2* __restrict__ tmp, int32_t* __restrict__ cnt) {
    int ch = blockIdx.x * blockDim.x + threadIdx.x;
    int nch = (nu + g - 1) / g;
    if (ch >= nch) return;
    const int s0 = ch * g, e0 = min(s0 + g, nu);
    int2 st[16];
    int sp = 0, ng = 0;
    st[sp++] = make_int2(s0, e0);
    while (sp > 0) {
        int2 r = st[--sp];
        int s = r.x, e = r.y;
        bool keep = (e - s == 1) || split <= 0.0f;
        if (!keep) {
            uint4 P0 = pfix[U[s]];
            int lox = 0, loy = 0, loz = 0, hix = 0, hiy = 0, hiz = 0;
            float hmin = (float)h64[U[s]];
            for (int k = s + 1; k < e; ++k) {
                int rk = U[k];
                uint4 P = pfix[rk];
                int dx = (int32_t)(P.x - P0.x), dy = (int32_t)(P.y - P0.y), dz = (int32_t)(P.z - P0.z);
                lox = min(lox, dx); hix = max(hix, dx);
                loy = min(loy, dy); hiy = max(hiy, dy);
                loz = min(loz, dz); hiz = max(hiz, dz);
                hmin = fminf(hmin, (float)h64[rk]);
            }
            // search sphere of the group (box centre) relative to one member's sphere,
            // in volume: the candidates every member filters, per member's own
            const float ext = fmaxf(fmaxf((float)((int64_t)hix - lox), (float)((int64_t)hiy - loy)),
                                    (float)((int64_t)hiz - loz)) * kUnitToBox;
            const float rel = fmaf(0.8660254f, ext / hmin, 1.0f);
            keep = rel * rel * rel <= split * (float)(e - s);
        }
        if (keep) {
            tmp[s0 + ng++] = make_int2(s, e - s);
        } else {
            // Cut at the largest gap in key order (ties: the one nearest the middle): an
            // active set made of runs along the curve splits where one run ends and the
            // next begins; contiguous members split in the middle.  The stack holds one
            // pending range per level of the current path; gap cuts, which may peel one
            // member at a time, are taken while it holds fewer than 8, so that the
            // halving below them (at most log2(128) = 7 more levels) stays within 16.
            int mid = s + (e - s + 1) / 2;
            if (sp < 8) {
                int best = 1, bk = mid;
                for (int k = s + 1; k < e; ++k) {
                    const int gap = U[k] - U[k - 1];
                    if (gap > best || (gap == best && abs(k - mid) < abs(bk - mid))) {
                        best = gap;
                        bk = k;
                    }
                }
                mid = bk;
            }
            st[sp++] = make_int2(mid, e);
            st[sp++] = make_int2(s, mid);
        }
    }
    cnt[ch] = ng;
}

// Radius grouping (Sec. 2.1): a group starts at a work-list entry and takes the entries
// that follow while they lie closer than R = f h to its first particle (periodic
// minimum image), at most cap of them; the first entry farther away starts the next
// group.  One thread scans each run of kRadiusRun entries; groups go to tmp at the
// run's first entry.
__global__ void k_radius_groups(const int32_t* __restrict__ U, int nu, int cap, float f,
                                const uint4* __restrict__ pfix, const float4* __restrict__ poff,
                                const double* __restrict__ h64, int2* __restrict__ tmp, int32_t* __restrict__ cnt) {
    const int run = blockIdx.x * blockDim.x + threadIdx.x;
    const int s0 = run * kRadiusRun;
    if (s0 >= nu) return;
    const int e0 = min(s0 + kRadiusRun, nu);
    int ng = 0;
    int i = s0;
    while (i < e0) {
        const int r0 = U[i];
        const uint4 P0 = pfix[r0];
        const float4 O0 = poff[r0];
        const float R = f * (float)h64[r0];
        const float R2 = R * R;
        int j = i + 1;
        while (j < e0 && j - i < cap) {
            const int rj = U[j];
            const uint4 P = pfix[rj];
            const float4 O = poff[rj];
            const float dx = fix_diff(P.x, O.x, P0.x, O0.x);
            const float dy = fix_diff(P.y, O.y, P0.y, O0.y);
            const float dz = fix_diff(P.z, O.z, P0.z, O0.z);
            if (!(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < R2)) break;
            ++j;
        }
        tmp[s0 + ng++] = make_int2(i, j - i);
        i = j;
    }
    cnt[run] = ng;
}

int launch_radius_groups(const int32_t* U, int nu, int cap, double f, const uint4* pfix, const float4* poff,
                         const double* h64, int2* tmp, int32_t* cnt, cudaStream_t s) {
    const int runs = (nu + kRadiusRun - 1) / kRadiusRun;
    k_radius_groups<<<blocks_for(runs, 64), 64, 0, s>>>(U, nu, cap, (float)f, pfix, poff, h64, tmp, cnt);
    note_launch();
    return check_cuda(cudaGetLastError(), "radius grouping");
}

__global__ void k_gather_groups(int nch, int g, const int2* __restrict__ tmp, const int32_t* __restrict__ cnt,
                                const int32_t* __restrict__ off, int2* __restrict__ groups) {
    int ch = blockIdx.x * blockDim.x + threadIdx.x;
    if (ch >= nch) return;
    int o = off[ch];
    for (int k = 0; k < cnt[ch]; ++k) groups[o + k] = tmp[ch * g + k];
}

int launch_split_groups(const int32_t* U, int nu, int g, float split, const uint4* pfix, const double* h64,
                        int2* tmp, int32_t* cnt, cudaStream_t s) {
    int nch = (nu + g - 1) / g;
    k_split_groups<<<blocks_for(nch, 128), 128, 0, s>>>(U, nu, g, split, pfix, h64, tmp, cnt);
    note_launch();
    return check_cuda(cudaGetLastError(), "group split");
}

int launch_gather_groups(int nch, int g, const int2* tmp, const int32_t* cnt, const int32_t* off, int2* groups,
                         cudaStream_t s) {
    k_gather_groups<<<blocks_for(nch, 256), 256, 0, s>>>(nch, g, tmp, cnt, off, groups);
    note_launch();
    return check_cuda(cudaGetLastError(), "group gather");
}

// ---------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------

template <class K>
static size_t group_smem() {
    return kWarpsPerBlock * (sizeof(WalkSmem) + sizeof(typename K::Tile));
}

// Persistent grid: every resident block slot of the GPU (at most one block per four
// groups when the group count is known on the host).
template <typename Kern, typename... Args>
static int launch_persistent(Kern kern, bool& configured, size_t sh, int64_t ngroups_host, int sm_count,
                             cudaStream_t s, const char* what, Args... args) {
    if (!configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
        configured = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarpsPerBlock * 32, sh);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)std::min(per_sm, kSpillWarpsPerSM / kWarpsPerBlock) * sm_count;
    if (ngroups_host >= 0) grid = std::min<int64_t>(grid, (ngroups_host + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kWarpsPerBlock * 32, sh, s>>>(args...);
    note_launch();
    return check_cuda(cudaGetLastError(), what);
}

template <class K, int MODE, int M>
static int launch_group_t(const SearchArgs& a, int sm_count, cudaStream_t s) {
    static bool configured = false;
    return launch_persistent(k_group<K, MODE, M>, configured, group_smem<K>(), a.ngroups_dev ? -1 : a.ngroups,
                             sm_count, s, "grouped search kernel", a);
}

template <class K, int MODE>
static int launch_group_m(const SearchArgs& a, int sm_count, cudaStream_t s) {
    int M = (a.g + 31) / 32;
    if (M <= 1) return launch_group_t<K, MODE, 1>(a, sm_count, s);
    if (M <= 2) return launch_group_t<K, MODE, 2>(a, sm_count, s);
    if (M <= 4) return launch_group_t<K, MODE, 4>(a, sm_count, s);
    return set_error(SPHGRP_EINVAL, "group_size must be <= 128");
}

template <class K>
static int launch_group_k(const SearchArgs& a, int mode, int sm_count, cudaStream_t s) {
    switch (mode) {
        case kAcc: return launch_group_m<K, kAcc>(a, sm_count, s);
        case kCount: return launch_group_m<K, kCount>(a, sm_count, s);
        case kFill: return launch_group_m<K, kFill>(a, sm_count, s);
        case kSupCount: return launch_group_m<K, kSupCount>(a, sm_count, s);
        case kSupFill: return launch_group_m<K, kSupFill>(a, sm_count, s);
    }
    return set_error(SPHGRP_EINVAL, "bad search mode");
}

static int members_per_lane(int max_g) { return max_g <= 32 ? 1 : (max_g <= 64 ? 2 : 4); }

int launch_search_dev(const SearchArgs& a, int kind, int max_g, int sm_count, cudaStream_t s) {
    if (max_g < 1 || max_g > 128) return set_error(SPHGRP_EINVAL, "group size outside [1, 128]");
    cudaMemsetAsync(a.work, 0, sizeof(int), s);
    SearchArgs b = a;
    b.g = max_g;   // selects the member slots per lane; groups4 carries every group's size
    switch (kind) {
        case kKindDensity: return launch_group_m<KDens, kAcc>(b, sm_count, s);
        case kKindHydro: return launch_group_m<KHydro, kAcc>(b, sm_count, s);
        case kKindHydroAdj: return launch_group_m<KHAdj, kAcc>(b, sm_count, s);
        case kKindDensityAdj: return launch_group_m<KDAdj, kAcc>(b, sm_count, s);
    }
    return set_error(SPHGRP_EINVAL, "bad kind");
}

template <int M>
static int launch_iter_t(const SearchArgs& a, const IterArgs& it, int sm_count, cudaStream_t s) {
    static bool configured = false;
    return launch_persistent(k_group_dens_iter<M>, configured, group_smem<KDens>(), a.ngroups_dev ? -1 : a.ngroups,
                             sm_count, s, "grouped density iteration kernel", a, it);
}

int launch_density_iter(const SearchArgs& a, const IterArgs& it, int max_g, int sm_count, cudaStream_t s) {
    if (max_g < 1 || max_g > 128) return set_error(SPHGRP_EINVAL, "group size outside [1, 128]");
    cudaMemsetAsync(a.work, 0, sizeof(int), s);
    switch (members_per_lane(max_g)) {
        case 1: return launch_iter_t<1>(a, it, sm_count, s);
        case 2: return launch_iter_t<2>(a, it, sm_count, s);
        default: return launch_iter_t<4>(a, it, sm_count, s);
    }
}

template <class K0, class K1, int M>
static int launch_pair_t(const SearchArgs& a0, const SearchArgs& a1, int sm_count, cudaStream_t s) {
    static bool configured = false;
    constexpr size_t tile = sizeof(typename K0::Tile) > sizeof(typename K1::Tile) ? sizeof(typename K0::Tile)
                                                                                  : sizeof(typename K1::Tile);
    const size_t sh = kWarpsPerBlock * (sizeof(WalkSmem) + tile);
    return launch_persistent(k_group_pair<K0, K1, M>, configured, sh, -1, sm_count, s, "paired search kernel", a0,
                             a1);
}

template <class K0, class K1>
static int launch_pair_m(const SearchArgs& a0, const SearchArgs& a1, int max_g, int sm_count, cudaStream_t s) {
    switch (members_per_lane(max_g)) {
        case 1: return launch_pair_t<K0, K1, 1>(a0, a1, sm_count, s);
        case 2: return launch_pair_t<K0, K1, 2>(a0, a1, sm_count, s);
        default: return launch_pair_t<K0, K1, 4>(a0, a1, sm_count, s);
    }
}

int launch_search_pair(const SearchArgs& a0, int kind0, const SearchArgs& a1, int kind1, int max_g, int sm_count,
                       cudaStream_t s) {
    if (max_g < 1 || max_g > 128) return set_error(SPHGRP_EINVAL, "group size outside [1, 128]");
    cudaMemsetAsync(a0.work, 0, sizeof(int), s);
    if (kind0 == kKindHydro && kind1 == kKindHydroAdj) return launch_pair_m<KHydro, KHAdj>(a0, a1, max_g, sm_count, s);
    return set_error(SPHGRP_EINVAL, "unsupported kind pair");
}

int launch_search(const SearchArgs& a, int kind, int mode, bool grouped, int sm_count, cudaStream_t s) {
    if (a.nu <= 0) return SPHGRP_OK;
    if (grouped) {
        cudaMemsetAsync(a.work, 0, sizeof(int), s);
        switch (kind) {
            case 0: return launch_group_k<KDens>(a, mode, sm_count, s);
            case 1: return launch_group_k<KHydro>(a, mode, sm_count, s);
            case 2:
                if (mode != kAcc) return set_error(SPHGRP_EINVAL, "adjoint kernels accumulate only");
                return launch_group_m<KHAdj, kAcc>(a, sm_count, s);
            case 3:
                if (mode != kAcc) return set_error(SPHGRP_EINVAL, "adjoint kernels accumulate only");
                return launch_group_m<KDAdj, kAcc>(a, sm_count, s);
            case kKindVelocity:
                if (mode != kAcc) return set_error(SPHGRP_EINVAL, "the velocity derivatives accumulate only");
                return launch_group_m<KVel, kAcc>(a, sm_count, s);
            case kKindDensityVel:
                if (mode != kAcc) return set_error(SPHGRP_EINVAL, "velocity derivatives accumulate only");
                return launch_group_m<KDensVel, kAcc>(a, sm_count, s);
            case kKindDensityList:
                if (mode != kAcc || a.g > 32)
                    return set_error(SPHGRP_EINVAL, "candidate lists: accumulation, group size <= 32");
                return launch_group_t<KDensList, kAcc, 1>(a, sm_count, s);
        }
        return set_error(SPHGRP_EINVAL, "bad kind");
    }
    int blocks = blocks_for(a.nu, 128);
    if (kind == 0) {
        if (mode == kAcc) k_indiv<0, kAcc><<<blocks, 128, 0, s>>>(a);
        else if (mode == kCount) k_indiv<0, kCount><<<blocks, 128, 0, s>>>(a);
        else if (mode == kFill) k_indiv<0, kFill><<<blocks, 128, 0, s>>>(a);
        else return set_error(SPHGRP_EINVAL, "bad search mode");
    } else if (kind == 1) {
        if (mode == kAcc) k_indiv<1, kAcc><<<blocks, 128, 0, s>>>(a);
        else if (mode == kCount) k_indiv<1, kCount><<<blocks, 128, 0, s>>>(a);
        else if (mode == kFill) k_indiv<1, kFill><<<blocks, 128, 0, s>>>(a);
        else return set_error(SPHGRP_EINVAL, "bad search mode");
    } else {
        return set_error(SPHGRP_EINVAL, "the adjoint kernels exist in the grouped form only");
    }
    note_launch();
    return check_cuda(cudaGetLastError(), "individual search kernel");
}

// ---------------------------------------------------------------------------------
// Smoothing-length iteration: per unconverged particle, FP64
// ---------------------------------------------------------------------------------

// One particle's step of the smoothing-length iteration from its density sums at h
// (S0 = sum m w, S1 = sum m (q w' + 3 w)) after `pass` passes.  With rho = sigma S0,
// dRho/dh = -(sigma / h) S1 and sigma = 8 / (pi h^3), the quantities of the iteration
// reduce to the sums themselves:
//   N_eff = (4 pi / 3) h^3 rho / m = (32 / 3) S0 / m,
//   f = 1 / (1 + h / (3 rho) dRho/dh) = 3 S0 / (3 S0 - S1),
//   g / g' = h (32 S0 - 3 N_ngb m) / (32 (3 S0 - S1))  (the Newton step).
// The convergence test |N_eff - N_ngb| <= tol is taken in FP64, as
// |(32/3) S0 - N_ngb m| <= tol m (no division); the sums themselves are FP32, so the
// Newton step and the bisection of the bracket carry no more than FP32 accuracy either
// and are taken in FP32 (FP64 division is slow on this part and would buy nothing).
// finish: converged (or no iteration asked), or the last pass; else hn is the next h and
// [lo, hi) the updated bracket (opened at pass 1).
struct HsmlStep {
    bool finish, converged;
    double hn;
};

__device__ __forceinline__ HsmlStep hsml_next(double h, float m, float s0, float s1, double nngb, double tol,
                                              bool iterate, int pass, int max_iter, double& lo, double& hi) {
    HsmlStep o;
    const double t = (32.0 / 3.0) * (double)s0, nm = nngb * (double)m;
    o.converged = !iterate || fabs(t - nm) <= tol * (double)m;
    o.finish = o.converged || pass >= max_iter;
    o.hn = h;
    if (o.finish) return o;
    if (pass == 1) {
        lo = 0.0;
        hi = __longlong_as_double(0x7ff0000000000000ll);
    }
    if (t < nm) lo = h; else hi = h;
    const float hf = (float)h;
    const float num = fmaf(-3.0f * (float)nngb, m, 32.0f * s0);
    const float den = 32.0f * (3.0f * s0 - s1);
    double hn = (double)(hf - hf * (num / den));
    if (!(hn > lo && hn < hi) || !isfinite(hn)) {
        // volume bisection of the bracket
        if (isinf(hi)) hn = (double)(hf * 1.25992104989487316f);
        else if (lo == 0.0) hn = (double)(hf * 0.79370052598409974f);
        else {
            const float l = (float)lo, u = (float)hi;
            hn = (double)cbrtf(0.5f * (l * l * l + u * u * u));
        }
    }
    o.hn = hn;
    return o;
}


// One particle's pass of the smoothing-length iteration: u = its work-list entry, r its
// rank, s0 / s1 / n its density sums at the current h.  Runs as its own kernel with one
// particle per thread: in the search kernel's epilogue only one slice of each warp would
// hold the members, which doubles the FP64 issue.
__device__ __forceinline__ void hsml_update(const UpdateArgs& a, int u, int r, float s0f, float s1f, int n) {
    const double h = a.h64[r];
    const float m = a.poff[r].w;
    const int pass = a.npass ? a.npass[r] + 1 : a.it;
    if (a.npass) a.npass[r] = pass;
    double lo = pass == 1 ? 0.0 : a.lo[r];
    double hi = pass == 1 ? __longlong_as_double(0x7ff0000000000000ll) : a.hi[r];
    const HsmlStep st = hsml_next(h, m, s0f, s1f, a.nngb, a.tol, a.iterate != 0, pass, a.max_iter, lo, hi);
    if (st.finish) {
        if (a.res_k) {
            a.res_k[r] = make_float4(s0f, s1f, __int_as_float(n), __int_as_float(pass));
        } else {
            hsml_write(a.perm[r], h, s0f, s1f, n, pass, a.h_out, a.rho, a.drhodh, a.fgrad, a.nngb_out, a.iters);
        }
        if (a.vsum && !a.res_k) {
            // div v = -(1/rho) sum m v_ij . grad W, curl v = (1/rho) sum m v_ij x grad W
            const int orig = a.perm[r];
            const float hf = (float)h;
            const float rinv = hf * hf * hf / (2.54647908947032537f * s0f);   // 1 / rho
            const float4 V = a.vsum[r];
            a.divv[orig] = V.x * rinv;
            a.curlv[3 * (int64_t)orig] = V.y * rinv;
            a.curlv[3 * (int64_t)orig + 1] = V.z * rinv;
            a.curlv[3 * (int64_t)orig + 2] = V.w * rinv;
        }
        a.keep[u] = 0;
        if (!st.converged) atomicAdd(a.nfail, 1);
        return;
    }
    a.lo[r] = lo;
    a.hi[r] = hi;
    a.h64[r] = st.hn;
    a.pfix[r].w = __float_as_uint((float)st.hn);
    a.keep[u] = 1;
}

__global__ void k_hsml_update(UpdateArgs a) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= a.nu) return;
    const int r = a.U[u];
    hsml_update(a, u, r, a.s0[r], a.s1[r], a.n[r]);
}

// Passes 2, 3, ... of the recycled iteration, one thread per unconverged particle: while
// its h stays within the widened radius h_w of its pass-1 candidate list, the density
// sums at h are those of the list's members inside h (the list holds every particle
// within h_w), so the particle iterates on its own list without a tree walk.  The
// decisions are the exact ones of the grouped kernel (FP32 on exact fixed-point
// differences, FP64 re-test in the band).  A particle whose h leaves h_w, or whose list
// overflowed, is flagged for a walk pass (keep = 1) with its iterate and bracket stored.
__global__ void __launch_bounds__(128) k_list_iterate(ListIterArgs a) {
    const int lane = threadIdx.x & 31;
    LocalCounters lc;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < a.nu) {
        const int r = a.U[u];
        const int slot = a.lslot[r];
        const int4 rec = a.lrec[slot];
        const double hw = a.lhw[slot];
        int pass = a.npass[r];
        double h = a.h64[r], lo = a.lo[r], hi = a.hi[r];
        const uint4 P = a.pfix_in[r];
        const float4 O = a.poff[r];
        const float m = O.w;
        bool walk = rec.w == 0;
        while (!walk) {
            if (!(h <= hw)) {
                walk = true;
                break;
            }
            ++pass;
            const float hf = (float)h;
            const float h2 = (float)(h * h);
            const float h2lo = h2 * (1.0f - 3.0f * kBandRel), h2hi = h2 * (1.0f + 3.0f * kBandRel);
            const float hinv = 1.0f / hf;
            const double hh = __dmul_rn(h, h);
            const int lsub = kListCap / rec.z;
            float S0 = 0.0f, C0 = 0.0f, S1 = 0.0f, C1 = 0.0f, p0 = 0.0f, p1 = 0.0f;
            int n = 0;
            for (int sl = 0; sl < rec.z; ++sl) {
                const int cnt = sl == 0 ? (rec.x & 0xffff) : sl == 1 ? (rec.x >> 16) : sl == 2 ? (rec.y & 0xffff)
                                                                                               : (rec.y >> 16);
                // sub-lists start at multiples of 4 entries (kListCap / S, S in {1, 2, 4}):
                // four entries per step, read as one int4 and gathered together, so that a
                // thread keeps eight candidate loads in flight
                const int4* L4 = reinterpret_cast<const int4*>(a.list + (int64_t)slot * kListCap + sl * lsub);
                for (int k0 = 0; k0 < cnt; k0 += 4) {
                    const int4 J4 = L4[k0 >> 2];
                    const int jj[4] = {J4.x, J4.y, J4.z, J4.w};
                    uint4 Q[4];
                    float4 Oj[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (k0 + e < cnt) {
                            Q[e] = __ldg(a.pfix_in + jj[e]);
                            Oj[e] = __ldg(a.poff + jj[e]);
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if (k0 + e >= cnt) break;
                        const float dx = fix_diff(Q[e].x, Oj[e].x, P.x, O.x);
                        const float dy = fix_diff(Q[e].y, Oj[e].y, P.y, O.y);
                        const float dz = fix_diff(Q[e].z, Oj[e].z, P.z, O.z);
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        bool in = r2 < h2lo;
                        if (!in && r2 < h2hi) {
                            in = exact_r2(a.xd, a.yd, a.zd, r, jj[e]) < hh;
                            lc.retests++;
                        }
                        if (!in) continue;
                        ++n;
                        const float q = r2 * rsqrtf(fmaxf(r2, 1.0e-30f)) * hinv;
                        float w, dw;
                        m4_shape(q, w, dw);
                        p0 = fmaf(Oj[e].w, w, p0);
                        p1 = fmaf(Oj[e].w, fmaf(q, dw, 3.0f * w), p1);
                    }
                    if ((k0 & 15) == 12) {
                        kahan_add(S0, C0, p0);
                        kahan_add(S1, C1, p1);
                        p0 = p1 = 0.0f;
                    }
                }
            }
            kahan_add(S0, C0, p0);
            kahan_add(S1, C1, p1);
            lc.pairs += n;
            const float s0 = S0 - C0, s1 = S1 - C1;
            const HsmlStep st = hsml_next(h, m, s0, s1, a.nngb, a.tol, true, pass, a.max_iter, lo, hi);
            if (st.finish) {
                hsml_write(a.perm[r], h, s0, s1, n, pass, a.h_out, a.rho, a.drhodh, a.fgrad, a.nngb_out, a.iters);
                if (!st.converged) atomicAdd(a.nfail, 1);
                break;
            }
            h = st.hn;
        }
        // (positions are read through the read-only path: pfix is not written here; its
        // FP32 copy of h is not read during the density call, and the hydro and velocity
        // entry points rewrite it from the caller's h)
        a.keep[u] = walk ? 1 : 0;
        a.npass[r] = pass;
        a.h64[r] = h;
        a.lo[r] = lo;
        a.hi[r] = hi;
    }
    // only pairs and re-tests are counted: the lists are not tree-search candidates
    int mp = u < a.nu ? a.npass[a.U[u]] : 0;
    for (int o = 16; o > 0; o >>= 1) {
        lc.pairs += __shfl_xor_sync(0xffffffffu, lc.pairs, o);
        lc.retests += __shfl_xor_sync(0xffffffffu, lc.retests, o);
        mp = max(mp, __shfl_xor_sync(0xffffffffu, mp, o));
    }
    if (lane == 0) {
        if (lc.pairs) atomicAdd(&a.ctr->pairs, lc.pairs);
        if (lc.retests) atomicAdd(&a.ctr->retests, lc.retests);
        if (a.max_pass) atomicMax(a.max_pass, mp);
    }
}

int launch_list_iterate(const ListIterArgs& a, cudaStream_t s) {
    if (a.nu <= 0) return SPHGRP_OK;
    static bool configured = false;
    if (!configured) {
        // no shared memory: all of it as L1, which holds the candidates that neighbouring
        // particles gather
        cudaFuncSetAttribute(k_list_iterate, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        configured = true;
    }
    k_list_iterate<<<blocks_for(a.nu, 128), 128, 0, s>>>(a);
    note_launch();
    return check_cuda(cudaGetLastError(), "list iteration");
}

int launch_hsml_update(const UpdateArgs& a, cudaStream_t s) {
    if (a.nu <= 0) return SPHGRP_OK;
    k_hsml_update<<<blocks_for(a.nu, 256), 256, 0, s>>>(a);
    note_launch();
    return check_cuda(cudaGetLastError(), "hsml update");
}

}  // namespace sphgrp
