// Gather into key order and the linear octree over the key-ordered particles
// (Sec. 1.2: an octree divides the volume; particles follow the Hilbert curve, so
// every octree cell is one contiguous range of the sorted order).
#include <algorithm>

#include "sph_internal.cuh"

namespace sphgrp {

// x * 2^32 is exact; its floor is the fixed-point coordinate, the remainder (exact in
// FP64, < 1) keeps the rest of the position and is rounded once to FP32.  For
// 2^-32 <= x < 1 both come from the bits of x with integer operations (FP64 arithmetic
// is a slow pipe on this part): x 2^32 = M 2^-s with M = 2^52 + f and s = 1043 - e in
// [21, 52], so the floor is M >> s and the remainder (M mod 2^s) 2^-s, whose integer
// part converts to FP32 with one rounding and scales by 2^-s exactly.  Other x take
// the FP64 form.
__device__ __forceinline__ uint32_t fix_split(double x, float& rem) {
    const uint64_t b = __double_as_longlong(x);
    const int e = (int)(b >> 52);   // biased exponent; the sign bit makes it >= 2048
    const int s = 1043 - e;
    if (s >= 21 && s <= 52) {
        const uint64_t M = (b & 0xfffffffffffffull) | (1ull << 52);
        rem = __ull2float_rn(M & ((1ull << s) - 1ull)) * __int_as_float((127 - s) << 23);
        return (uint32_t)(M >> s);
    }
    const double sx = x * kBoxToUnit, fx = floor(sx);
    rem = (float)(sx - fx);
    return (uint32_t)fx;
}

// pos/m (original order) -> key-ordered FP64 copies and the fixed-point layout.
__global__ void k_gather(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ pos,
                         const float* __restrict__ m, double* __restrict__ xd, double* __restrict__ yd,
                         double* __restrict__ zd, uint4* __restrict__ pfix, float4* __restrict__ poff) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    int i = perm[r];
    double x = pos[3 * (int64_t)i], y = pos[3 * (int64_t)i + 1], z = pos[3 * (int64_t)i + 2];
    float ox, oy, oz;
    uint4 P;
    P.x = fix_split(x, ox);
    P.y = fix_split(y, oy);
    P.z = fix_split(z, oz);
    P.w = 0u;
    pfix[r] = P;
    poff[r] = make_float4(ox, oy, oz, m[i]);
    xd[r] = x;
    yd[r] = y;
    zd[r] = z;
}

__device__ __forceinline__ int key_digit(uint64_t key, int shift) { return (int)((key >> shift) & 7u); }

// Octant boundaries of the key range [lo, hi) (hi > lo) at the digit of `shift`: b[d] is
// the first index whose digit is >= d, b[0] = lo, b[8] = hi (digits are non-decreasing
// in the range).  The seven lower bounds run in lockstep: each step halves a range of
// the same length for all of them, so their loads are independent and a node's search
// costs the latency of one binary search, not of seven in a row.
__device__ __forceinline__ void octant_bounds(const uint64_t* __restrict__ keys, int lo, int hi, int shift,
                                              int (&b)[9]) {
    int base[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) base[d] = lo;
    // invariant: indices below base[d] have digit < d + 1, and the bound lies in
    // [base[d], base[d] + n]
    int n = hi - lo;
    while (n > 1) {
        const int half = n >> 1;
        int dg[7];
#pragma unroll
        for (int d = 0; d < 7; ++d) dg[d] = key_digit(keys[base[d] + half], shift);
#pragma unroll
        for (int d = 0; d < 7; ++d)
            if (dg[d] < d + 1) base[d] += half;
        n -= half;
    }
    b[0] = lo;
    b[8] = hi;
#pragma unroll
    for (int d = 0; d < 7; ++d) b[d + 1] = base[d] + (key_digit(keys[base[d]], shift) < d + 1 ? 1 : 0);
}

// Cells of the top levels 1 .. kTopLevels: the first index of every non-empty cell, in a
// direct-indexed table per level (8^l entries at offset top_offset(l); -1 = empty).  A
// level-l node (l < kTopLevels) then reads its octant bounds from the 8 entries of its
// children instead of searching a key range of up to n keys, which at these levels is
// one long chain of dependent loads for a handful of threads.
constexpr int kTopLevels = 6;
constexpr int kTopTableSize = 299592;   // 8 + 8^2 + ... + 8^6
__host__ __device__ constexpr int top_offset(int l) { return ((1 << (3 * l)) - 8) / 7; }   // 8 + ... + 8^(l-1)
static_assert(top_offset(kTopLevels + 1) == kTopTableSize, "top-level cell table size");

// i starts a cell at every level deeper than the number of leading digits its key shares
// with key i - 1 (digit j of a 63-bit key is bits 62 - 3j .. 60 - 3j, so the first
// differing digit of x = k_i ^ k_{i-1} is (clz(x) - 1) / 3)
__global__ void k_top_cells(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ tab) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = keys[i];
    int d = 0;
    if (i > 0) {
        const uint64_t x = k ^ keys[i - 1];
        d = x == 0 ? kKeyLevels : (__clzll((long long)x) - 1) / 3;
    }
    for (int l = d + 1; l <= kTopLevels; ++l) tab[top_offset(l) + (int)(k >> (3 * (kKeyLevels - l)))] = (int32_t)i;
}

// octant bounds of a node of level `level` over the keys [lo, hi): from the top-cell
// table above the top levels (tab non-null), else by the lockstep search
__device__ __forceinline__ void node_bounds(const uint64_t* __restrict__ keys, const int32_t* __restrict__ tab,
                                            int level, int lo, int hi, int (&b)[9]) {
    if (tab && level < kTopLevels) {
        const int P = level == 0 ? 0 : (int)(keys[lo] >> (3 * (kKeyLevels - level)));
        const int32_t* ch = tab + top_offset(level + 1) + 8 * P;
        int st[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) st[d] = ch[d];
        b[8] = hi;
#pragma unroll
        for (int d = 7; d >= 0; --d) b[d] = st[d] >= 0 ? st[d] : b[d + 1];
        return;
    }
    octant_bounds(keys, lo, hi, 3 * (kKeyLevels - 1 - level), b);
}

// Number of non-empty octants of every node of one level that must split.
__global__ void k_split_count(const uint64_t* __restrict__ keys, const int4* __restrict__ nlink,
                              int a, int nf, int level, int leaf_size, int32_t* __restrict__ nchild,
                              const int32_t* __restrict__ tab) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    int4 L = nlink[a + k];
    int cnt = 0;
    if (L.y > leaf_size && level < kKeyLevels) {
        int b[9];
        node_bounds(keys, tab, level, L.x, L.x + L.y, b);
#pragma unroll
        for (int d = 0; d < 8; ++d) cnt += b[d + 1] > b[d] ? 1 : 0;
    }
    nchild[k] = cnt;
}

// Writes the children of every splitting node of one level.
__global__ void k_split_write(const uint64_t* __restrict__ keys, int4* __restrict__ nlink,
                              float4* __restrict__ next, int32_t* __restrict__ nlevel, int a,
                              int nf, int level, const int32_t* __restrict__ nchild,
                              const int32_t* __restrict__ coff, int b, const int32_t* __restrict__ tab) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    int nc = nchild[k];
    int4 L = nlink[a + k];
    next[a + k].w = __int_as_float(nc);
    if (nc == 0) return;
    int child0 = b + coff[k];
    int bd[9];
    node_bounds(keys, tab, level, L.x, L.x + L.y, bd);
    int c = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        if (bd[d + 1] > bd[d]) {
            int id = child0 + c;
            int skip = (c + 1 < nc) ? id + 1 : L.w;
            nlink[id] = make_int4(bd[d], bd[d + 1] - bd[d], -1, skip);
            nlevel[id] = level + 1;
            ++c;
        }
    }
    L.z = child0;
    nlink[a + k] = L;
}

// Tight boxes (fixed point) and hmax of one level, leaves from their particles,
// internal nodes from their children.
__global__ void k_box_level(int a, int nf, const int4* __restrict__ nlink, const float4* __restrict__ next,
                            const uint4* __restrict__ pfix, uint4* __restrict__ blo, uint4* __restrict__ bhi,
                            uint4* __restrict__ ncen) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    int id = a + k;
    int4 L = nlink[id];
    uint32_t lx = 0xffffffffu, ly = 0xffffffffu, lz = 0xffffffffu, hx = 0, hy = 0, hz = 0;
    float hm = 0.0f;
    if (L.z < 0) {
        for (int q = L.x; q < L.x + L.y; ++q) {
            uint4 P = pfix[q];
            lx = min(lx, P.x); ly = min(ly, P.y); lz = min(lz, P.z);
            hx = max(hx, P.x); hy = max(hy, P.y); hz = max(hz, P.z);
            hm = fmaxf(hm, __uint_as_float(P.w));
        }
    } else {
        int nc = __float_as_int(next[id].w);
        for (int c = L.z; c < L.z + nc; ++c) {
            uint4 l = blo[c], h = bhi[c];
            lx = min(lx, l.x); ly = min(ly, l.y); lz = min(lz, l.z);
            hx = max(hx, h.x); hy = max(hy, h.y); hz = max(hz, h.z);
            hm = fmaxf(hm, __uint_as_float(ncen[c].w));
        }
    }
    blo[id] = make_uint4(lx, ly, lz, 0u);
    bhi[id] = make_uint4(hx, hy, hz, 0u);
    ncen[id].w = __float_as_uint(hm);
}

// Box -> centre (fixed point) and padded half extents.  Particles of the node lie in
// [lo, hi + 1) units; with the centre rounded down to a whole unit the half extent
// (hi - lo + 2) / 2 covers that interval.  Extents are rounded up.
__global__ void k_box_final(int64_t nn, const uint4* __restrict__ blo, const uint4* __restrict__ bhi,
                            uint4* __restrict__ ncen, float4* __restrict__ next) {
    int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nn) return;
    uint4 l = blo[id], h = bhi[id];
    uint4 C = ncen[id];
    uint64_t wx = (uint64_t)h.x - l.x + 1, wy = (uint64_t)h.y - l.y + 1, wz = (uint64_t)h.z - l.z + 1;
    C.x = l.x + (uint32_t)(wx >> 1);
    C.y = l.y + (uint32_t)(wy >> 1);
    C.z = l.z + (uint32_t)(wz >> 1);
    ncen[id] = C;
    float4 E = next[id];
    E.x = __fmul_ru(__ull2float_ru(wx + 1), 0.5f);
    E.y = __fmul_ru(__ull2float_ru(wy + 1), 0.5f);
    E.z = __fmul_ru(__ull2float_ru(wz + 1), 0.5f);
    next[id] = E;
}

// hmax only (after the smoothing lengths changed)
__global__ void k_hmax_level(int a, int nf, const int4* __restrict__ nlink, const float4* __restrict__ next,
                             const uint4* __restrict__ pfix, uint4* __restrict__ ncen) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    int id = a + k;
    int4 L = nlink[id];
    float hm = 0.0f;
    if (L.z < 0) {
        for (int q = L.x; q < L.x + L.y; ++q) hm = fmaxf(hm, __uint_as_float(pfix[q].w));
    } else {
        int nc = __float_as_int(next[id].w);
        for (int c = L.z; c < L.z + nc; ++c) hm = fmaxf(hm, __uint_as_float(ncen[c].w));
    }
    ncen[id].w = __float_as_uint(hm);
}

// Walk start table (see kStartLevels): every node of levels 1 .. kStartLevels enters
// under its cell, found from any of its particles (the cell of level l is the top l
// bits of the fixed-point coordinates).
__global__ void k_start_table(int first, int count, const int4* __restrict__ nlink,
                              const int32_t* __restrict__ nlevel, const uint4* __restrict__ pfix,
                              int32_t* __restrict__ tab) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int id = first + k;
    const int l = nlevel[id];
    const int4 L = nlink[id];
    if (l < 1 || l > kStartLevels || L.y <= 0) return;
    const uint4 P = pfix[L.x];
    const uint32_t x = P.x >> (32 - l), y = P.y >> (32 - l), z = P.z >> (32 - l);
    uint32_t m = 0;
    for (int b = l - 1; b >= 0; --b) m = (m << 3) | (((x >> b) & 1u) << 2) | (((y >> b) & 1u) << 1) | ((z >> b) & 1u);
    tab[start_table_offset(l) + m] = id;
}

static int grow_tree(Ctx* c, int64_t need, cudaStream_t s) {
    Tree& t = c->tree;
    if (need <= t.cap) return SPHGRP_OK;
    int64_t cap = std::max<int64_t>(need + need / 2, 1024);
    uint4* ncen;
    float4* next;
    int4* nlink;
    int32_t* nlevel;
    if (cudaMallocAsync(&ncen, cap * sizeof(uint4), s) != cudaSuccess ||
        cudaMallocAsync(&next, cap * sizeof(float4), s) != cudaSuccess ||
        cudaMallocAsync(&nlink, cap * sizeof(int4), s) != cudaSuccess ||
        cudaMallocAsync(&nlevel, cap * sizeof(int32_t), s) != cudaSuccess)
        return set_error(SPHGRP_ENOMEM, "octree allocation failed");
    if (t.count > 0) {
        cudaMemcpyAsync(ncen, t.ncen, t.count * sizeof(uint4), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(next, t.next, t.count * sizeof(float4), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(nlink, t.nlink, t.count * sizeof(int4), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(nlevel, t.nlevel, t.count * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    }
    if (t.ncen) {
        cudaFreeAsync(t.ncen, s);
        cudaFreeAsync(t.next, s);
        cudaFreeAsync(t.nlink, s);
        cudaFreeAsync(t.nlevel, s);
    }
    t.ncen = ncen;
    t.next = next;
    t.nlink = nlink;
    t.nlevel = nlevel;
    t.cap = cap;
    return check_cuda(cudaGetLastError(), "octree allocation");
}

int build_tree(Ctx* c, cudaStream_t s) {
    Tree& t = c->tree;
    const int64_t n = c->n;
    int rc = grow_tree(c, std::max<int64_t>(1024, 2 * n / std::max(1, c->p.leaf_size) + 64), s);
    if (rc) return rc;
    int4 root = make_int4(0, (int)n, -1, -1);
    cudaMemcpyAsync(t.nlink, &root, sizeof(int4), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(t.nlevel, 0, sizeof(int32_t), s);
    cudaMemsetAsync(t.next, 0, sizeof(float4), s);
    t.level_begin[0] = 0;
    t.level_begin[1] = 1;
    t.count = 1;
    int level = 0;
    int32_t* total_dev = reinterpret_cast<int32_t*>(c->work) + 12;
    if (!t.top_cells && cudaMalloc(&t.top_cells, kTopTableSize * sizeof(int32_t)) != cudaSuccess) {
        t.top_cells = nullptr;
        return set_error(SPHGRP_ENOMEM, "octree top-cell table");
    }
    int32_t* top = t.top_cells;
    cudaMemsetAsync(top, 0xff, kTopTableSize * sizeof(int32_t), s);
    if (n > 0) {
        k_top_cells<<<blocks_for(n, 256), 256, 0, s>>>(c->keys, n, top);
        note_launch();
    }
    for (level = 0; level <= kKeyLevels; ++level) {
        int a = t.level_begin[level], b = t.level_begin[level + 1];
        int nf = b - a;
        if (nf == 0) break;
        k_split_count<<<blocks_for(nf, 256), 256, 0, s>>>(c->keys, t.nlink, a, nf, level,
                                                          c->p.leaf_size, c->flag, top);
        note_launch();
        rc = exclusive_scan_i32(c, c->flag, c->scan, nf, total_dev, s);
        if (rc) return rc;
        cudaMemcpyAsync(c->host_small, total_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if ((rc = check_cuda(cudaStreamSynchronize(s), "octree level"))) return rc;
        int total = c->host_small[0];
        if (b + (int64_t)total > t.cap) {
            if ((rc = grow_tree(c, b + (int64_t)total, s))) return rc;
        }
        k_split_write<<<blocks_for(nf, 256), 256, 0, s>>>(c->keys, t.nlink, t.next, t.nlevel, a, nf,
                                                          level, c->flag, c->scan, b, top);
        note_launch();
        t.level_begin[level + 2] = b + total;
        t.count = b + total;
        if (total == 0) { ++level; break; }
    }
    t.nlevels = level;
    // boxes bottom-up, in scratch kept by the tree (grown to the node count when needed)
    if (t.box_cap < t.count) {
        if (t.box_lo) cudaFree(t.box_lo);
        if (t.box_hi) cudaFree(t.box_hi);
        t.box_lo = t.box_hi = nullptr;
        t.box_cap = 0;
        const int64_t cap = t.count + t.count / 4 + 1024;
        if (cudaMalloc(&t.box_lo, cap * sizeof(uint4)) != cudaSuccess ||
            cudaMalloc(&t.box_hi, cap * sizeof(uint4)) != cudaSuccess) {
            cudaGetLastError();
            return set_error(SPHGRP_ENOMEM, "octree box scratch");
        }
        t.box_cap = cap;
    }
    uint4* blo = t.box_lo;
    uint4* bhi = t.box_hi;
    for (int lv = t.nlevels - 1; lv >= 0; --lv) {
        int a = t.level_begin[lv], nf = t.level_begin[lv + 1] - a;
        if (nf > 0) {
            k_box_level<<<blocks_for(nf, 128), 128, 0, s>>>(a, nf, t.nlink, t.next, c->pfix, blo, bhi, t.ncen);
            note_launch();
        }
    }
    k_box_final<<<blocks_for(t.count, 256), 256, 0, s>>>(t.count, blo, bhi, t.ncen, t.next);
    note_launch();
    {
        const int first = t.level_begin[1];
        const int last = t.level_begin[std::min(t.nlevels, kStartLevels) + 1];
        cudaMemsetAsync(c->start_tab, 0xff, kStartTableSize * sizeof(int32_t), s);
        if (last > first) {
            k_start_table<<<blocks_for(last - first, 256), 256, 0, s>>>(first, last - first, t.nlink, t.nlevel,
                                                                        c->pfix, c->start_tab);
            note_launch();
        }
        c->start_valid = true;
    }
    return check_cuda(cudaGetLastError(), "octree build");
}

int refresh_hmax(Ctx* c, cudaStream_t s) {
    Tree& t = c->tree;
    for (int lv = t.nlevels - 1; lv >= 0; --lv) {
        int a = t.level_begin[lv], nf = t.level_begin[lv + 1] - a;
        if (nf > 0) {
            k_hmax_level<<<blocks_for(nf, 128), 128, 0, s>>>(a, nf, t.nlink, t.next, c->pfix, t.ncen);
            note_launch();
        }
    }
    return check_cuda(cudaGetLastError(), "hmax refresh");
}

// ---------------------------------------------------------------------------------
// Forest of one octree per box (batch path).  Box k's particles are the ranks
// [box_off[k], box_off[k+1]) (sorted by box, then key); node k < nbox is box k's
// root.  Levels are built as above, but every count stays on the device (the level
// table lvl, lvl[L] = first node of level L), so that the whole build can be captured
// in a CUDA graph: the kernels of a level run over a grid-stride range read from lvl.
// ---------------------------------------------------------------------------------

constexpr int kForestGrid = 1024;   // blocks of the grid-stride kernels

__global__ void k_forest_roots(int nbox, const int64_t* __restrict__ box_off, int4* __restrict__ nlink,
                               float4* __restrict__ next, int32_t* __restrict__ nlevel, int32_t* __restrict__ lvl) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nbox) {
        nlink[k] = make_int4((int)box_off[k], (int)(box_off[k + 1] - box_off[k]), -1, -1);
        next[k] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(0));
        nlevel[k] = 0;
    }
    if (k <= kKeyLevels + 2) lvl[k] = (k == 0) ? 0 : nbox;
}

// box_cfg (optional): per box, bits 16..23 = that box's leaf size (0: leaf_size); the
// node's box is the box of its first particle
__global__ void k_split_count_dev(const uint64_t* __restrict__ keys, const int4* __restrict__ nlink,
                                  const int32_t* __restrict__ lvl, int level, int leaf_size,
                                  int32_t* __restrict__ nchild, const int32_t* __restrict__ box_cfg,
                                  const int32_t* __restrict__ box_of_rank) {
    const int a = lvl[level], nf = lvl[level + 1] - a;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
        int4 L = nlink[a + k];
        int cnt = 0;
        int leaf = leaf_size;
        if (box_cfg && L.y > 0) {
            const int lb = (box_cfg[box_of_rank[L.x]] >> 16) & 0xff;
            if (lb > 0) leaf = lb;
        }
        if (L.y > leaf && level < kKeyLevels) {
            int b[9];
            octant_bounds(keys, L.x, L.x + L.y, 3 * (kKeyLevels - 1 - level), b);
#pragma unroll
            for (int d = 0; d < 8; ++d) cnt += b[d + 1] > b[d] ? 1 : 0;
        }
        nchild[k] = cnt;
    }
}

// children of one level; nodes beyond the capacity are not created (their parent stays
// a leaf, the error flag is set and the results of the call are invalid)
__global__ void k_split_write_dev(const uint64_t* __restrict__ keys, int4* __restrict__ nlink,
                                  float4* __restrict__ next, int32_t* __restrict__ nlevel, int32_t* lvl, int level,
                                  const int32_t* __restrict__ nchild, const int32_t* __restrict__ coff,
                                  const int32_t* __restrict__ total, int64_t cap, unsigned* err) {
    const int a = lvl[level], b = lvl[level + 1], nf = b - a;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
        const int nc = nchild[k];
        int4 L = nlink[a + k];
        const int child0 = b + coff[k];
        if (nc == 0 || (int64_t)child0 + nc > cap) {
            if (nc > 0) atomicOr(err, kErrNodes);
            next[a + k].w = __int_as_float(0);
            continue;
        }
        next[a + k].w = __int_as_float(nc);
        int bd[9];
        octant_bounds(keys, L.x, L.x + L.y, 3 * (kKeyLevels - 1 - level), bd);
        int c = 0;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            if (bd[d + 1] > bd[d]) {
                const int id = child0 + c;
                const int skip = (c + 1 < nc) ? id + 1 : L.w;
                nlink[id] = make_int4(bd[d], bd[d + 1] - bd[d], -1, skip);
                next[id] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(0));
                nlevel[id] = level + 1;
                ++c;
            }
        }
        L.z = child0;
        nlink[a + k] = L;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) lvl[level + 2] = (int)min((int64_t)b + *total, cap);
}

__global__ void k_box_level_dev(const int32_t* __restrict__ lvl, int level, const int4* __restrict__ nlink,
                                const float4* __restrict__ next, const uint4* __restrict__ pfix,
                                uint4* __restrict__ blo, uint4* __restrict__ bhi, uint4* __restrict__ ncen) {
    const int a = lvl[level], nf = lvl[level + 1] - a;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
        const int id = a + k;
        const int4 L = nlink[id];
        uint32_t lx = 0xffffffffu, ly = 0xffffffffu, lz = 0xffffffffu, hx = 0, hy = 0, hz = 0;
        float hm = 0.0f;
        const int nc = __float_as_int(next[id].w);
        if (nc == 0) {
            for (int q = L.x; q < L.x + L.y; ++q) {
                const uint4 P = pfix[q];
                lx = min(lx, P.x); ly = min(ly, P.y); lz = min(lz, P.z);
                hx = max(hx, P.x); hy = max(hy, P.y); hz = max(hz, P.z);
                hm = fmaxf(hm, __uint_as_float(P.w));
            }
        } else {
            for (int c = L.z; c < L.z + nc; ++c) {
                const uint4 l = blo[c], h = bhi[c];
                lx = min(lx, l.x); ly = min(ly, l.y); lz = min(lz, l.z);
                hx = max(hx, h.x); hy = max(hy, h.y); hz = max(hz, h.z);
                hm = fmaxf(hm, __uint_as_float(ncen[c].w));
            }
        }
        if (L.y == 0) lx = ly = lz = hx = hy = hz = 0u;   // an empty box
        blo[id] = make_uint4(lx, ly, lz, 0u);
        bhi[id] = make_uint4(hx, hy, hz, 0u);
        ncen[id].w = __float_as_uint(hm);
    }
}

__global__ void k_box_final_dev(const int32_t* __restrict__ lvl, const uint4* __restrict__ blo,
                                const uint4* __restrict__ bhi, uint4* __restrict__ ncen, float4* __restrict__ next) {
    const int64_t nn = lvl[kKeyLevels + 1];
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < nn; id += (int64_t)gridDim.x * blockDim.x) {
        const uint4 l = blo[id], h = bhi[id];
        uint4 C = ncen[id];
        const uint64_t wx = (uint64_t)h.x - l.x + 1, wy = (uint64_t)h.y - l.y + 1, wz = (uint64_t)h.z - l.z + 1;
        C.x = l.x + (uint32_t)(wx >> 1);
        C.y = l.y + (uint32_t)(wy >> 1);
        C.z = l.z + (uint32_t)(wz >> 1);
        ncen[id] = C;
        float4 E = next[id];
        E.x = __fmul_ru(__ull2float_ru(wx + 1), 0.5f);
        E.y = __fmul_ru(__ull2float_ru(wy + 1), 0.5f);
        E.z = __fmul_ru(__ull2float_ru(wz + 1), 0.5f);
        next[id] = E;
    }
}

__global__ void k_hmax_level_dev(const int32_t* __restrict__ lvl, int level, const int4* __restrict__ nlink,
                                 const float4* __restrict__ next, const uint4* __restrict__ pfix,
                                 uint4* __restrict__ ncen) {
    const int a = lvl[level], nf = lvl[level + 1] - a;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
        const int id = a + k;
        const int4 L = nlink[id];
        const int nc = __float_as_int(next[id].w);
        float hm = 0.0f;
        if (nc == 0) {
            for (int q = L.x; q < L.x + L.y; ++q) hm = fmaxf(hm, __uint_as_float(pfix[q].w));
        } else {
            for (int c = L.z; c < L.z + nc; ++c) hm = fmaxf(hm, __uint_as_float(ncen[c].w));
        }
        ncen[id].w = __float_as_uint(hm);
    }
}

// Start tables of a forest (one per box, see k_start_table): every node of levels
// 1 .. kStartLevels enters its box's table under its cell.
__global__ void k_start_table_forest(const int32_t* __restrict__ lvl, const int4* __restrict__ nlink,
                                     const int32_t* __restrict__ nlevel, const uint4* __restrict__ pfix,
                                     const int32_t* __restrict__ box_of_rank, int32_t* __restrict__ tab) {
    const int first = lvl[1], count = lvl[kStartLevels + 1] - first;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const int id = first + k;
        const int l = nlevel[id];
        const int4 L = nlink[id];
        if (l < 1 || l > kStartLevels || L.y <= 0) continue;
        const uint4 P = pfix[L.x];
        const uint32_t x = P.x >> (32 - l), y = P.y >> (32 - l), z = P.z >> (32 - l);
        uint32_t m = 0;
        for (int b = l - 1; b >= 0; --b) m = (m << 3) | (((x >> b) & 1u) << 2) | (((y >> b) & 1u) << 1) | ((z >> b) & 1u);
        tab[(size_t)box_of_rank[L.x] * kStartTableSize + start_table_offset(l) + m] = id;
    }
}

int alloc_forest(Ctx* c, int64_t cap) {
    Tree& t = c->tree;
    if (t.cap >= cap) return SPHGRP_OK;
    if (t.ncen) {
        cudaFree(t.ncen);
        cudaFree(t.next);
        cudaFree(t.nlink);
        cudaFree(t.nlevel);
        t.ncen = nullptr;
        t.next = nullptr;
        t.nlink = nullptr;
        t.nlevel = nullptr;
        t.cap = 0;
    }
    if (cudaMalloc(&t.ncen, cap * sizeof(uint4)) != cudaSuccess ||
        cudaMalloc(&t.next, cap * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&t.nlink, cap * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(&t.nlevel, cap * sizeof(int32_t)) != cudaSuccess)
        return set_error(SPHGRP_ENOMEM, "forest allocation failed");
    t.cap = cap;
    return SPHGRP_OK;
}

// lvl: device, kKeyLevels + 3 entries; blo/bhi: device scratch of t.cap entries;
// tot: one device int.  Uses c->flag and c->scan as per-level scratch.
int build_forest(Ctx* c, int nbox, const int64_t* box_off_dev, int32_t* lvl, uint4* blo, uint4* bhi, int32_t* tot,
                 const int32_t* box_of_rank, int32_t* start_tabs, cudaStream_t s, const int32_t* box_cfg) {
    Tree& t = c->tree;
    c->start_valid = false;   // the single-box table does not describe a forest
    const int64_t n = c->n;
    k_forest_roots<<<blocks_for(std::max(nbox, kKeyLevels + 3), 256), 256, 0, s>>>(nbox, box_off_dev, t.nlink,
                                                                                 t.next, t.nlevel, lvl);
    note_launch();
    int rc = SPHGRP_OK;
    for (int level = 0; level < kKeyLevels; ++level) {
        k_split_count_dev<<<kForestGrid, 256, 0, s>>>(c->keys, t.nlink, lvl, level, c->p.leaf_size, c->flag,
                                                      box_cfg, box_of_rank);
        note_launch();
        if ((rc = exclusive_scan_i32_dev(c, c->flag, c->scan, lvl + level + 1, lvl + level, n, tot, s))) return rc;
        k_split_write_dev<<<kForestGrid, 256, 0, s>>>(c->keys, t.nlink, t.next, t.nlevel, lvl, level, c->flag,
                                                      c->scan, tot, t.cap, c->err);
        note_launch();
    }
    // lvl[kKeyLevels + 1] = node count
    for (int level = kKeyLevels; level >= 0; --level) {
        k_box_level_dev<<<kForestGrid, 128, 0, s>>>(lvl, level, t.nlink, t.next, c->pfix, blo, bhi, t.ncen);
        note_launch();
    }
    k_box_final_dev<<<kForestGrid, 256, 0, s>>>(lvl, blo, bhi, t.ncen, t.next);
    note_launch();
    if (start_tabs) {
        cudaMemsetAsync(start_tabs, 0xff, (size_t)nbox * kStartTableSize * sizeof(int32_t), s);
        k_start_table_forest<<<kForestGrid, 256, 0, s>>>(lvl, t.nlink, t.nlevel, c->pfix, box_of_rank, start_tabs);
        note_launch();
    }
    return check_cuda(cudaGetLastError(), "forest build");
}

int refresh_hmax_forest(Ctx* c, const int32_t* lvl, cudaStream_t s) {
    Tree& t = c->tree;
    for (int level = kKeyLevels; level >= 0; --level) {
        k_hmax_level_dev<<<kForestGrid, 128, 0, s>>>(lvl, level, t.nlink, t.next, c->pfix, t.ncen);
        note_launch();
    }
    return check_cuda(cudaGetLastError(), "forest hmax refresh");
}

int gather_particles(Ctx* c, const double* pos, const float* m, cudaStream_t s) {
    k_gather<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, pos, m, c->xd, c->yd, c->zd,
                                                  c->pfix, c->poff);
    note_launch();
    return check_cuda(cudaGetLastError(), "gather");
}

}  // namespace sphgrp
