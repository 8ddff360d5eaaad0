// Peano-Hilbert keys, the stable device radix sort of (key, index) and a device
// exclusive scan (Sec. 1.2: Gadget3 orders its particles along the Hilbert curve).
#include <cooperative_groups.h>

#include <utility>

#include "sph_internal.cuh"

namespace sphgrp {

// ---------------------------------------------------------------------------------
// Keys
// ---------------------------------------------------------------------------------

// Spreads the low 21 bits of v so that bit b lands on bit 3b.
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Hilbert index of a cell of the 2^21 grid by Skilling's transpose construction:
// from the coarsest level down, every axis either reflects (bit set) or swaps its
// lower bits with axis 0 (bit clear); then a Gray code across the axes and a common
// correction; the index interleaves the transposed words, axis 0 most significant.
__device__ __forceinline__ uint64_t hilbert_key(uint32_t a0, uint32_t a1, uint32_t a2) {
#pragma unroll
    for (uint32_t q = 1u << (kKeyLevels - 1); q > 1u; q >>= 1) {
        const uint32_t lowmask = q - 1u;
        if (a0 & q) a0 ^= lowmask;
        if (a1 & q) {
            a0 ^= lowmask;
        } else {
            uint32_t t = (a0 ^ a1) & lowmask;
            a0 ^= t;
            a1 ^= t;
        }
        if (a2 & q) {
            a0 ^= lowmask;
        } else {
            uint32_t t = (a0 ^ a2) & lowmask;
            a0 ^= t;
            a2 ^= t;
        }
    }
    a1 ^= a0;
    a2 ^= a1;
    uint32_t corr = 0;
#pragma unroll
    for (uint32_t q = 1u << (kKeyLevels - 1); q > 1u; q >>= 1)
        if (a2 & q) corr ^= q - 1u;
    a0 ^= corr;
    a1 ^= corr;
    a2 ^= corr;
    return (spread3(a0) << 2) | (spread3(a1) << 1) | spread3(a2);
}

// The cell of the 2^21 grid, floor(x 2^21) clamped to [0, 2^21 - 1] (a NaN to 0), taken
// from the bits of x with integer operations: x = (2^52 + f) 2^(e - 1075), so
// floor(x 2^21) = (2^52 + f) >> (1054 - e) for 0 < x < 1; FP64 arithmetic is a slow
// pipe on this part, and this form is exact.
__device__ __forceinline__ uint32_t grid21(uint64_t b) {
    if (b >> 63) return 0u;                                     // x <= -0 (or a negative NaN)
    const int e = (int)(b >> 52);                               // biased exponent
    if (e >= 1023) return (e == 2047 && (b << 12)) ? 0u : 2097151u;   // x >= 1, inf; NaN
    const int sh = 1054 - e;                                    // >= 32
    if (sh > 52) return 0u;                                     // x 2^21 < 1 (zero, subnormal)
    return (uint32_t)(((b & 0xfffffffffffffull) | (1ull << 52)) >> sh);
}

// 0 <= x < 1 from the bits (-0 included, NaN excluded)
__device__ __forceinline__ bool unit_bits(uint64_t b) {
    return b < 0x3ff0000000000000ull || b == 0x8000000000000000ull;
}

__global__ void k_keys(int64_t n, const double* __restrict__ pos, uint64_t* __restrict__ keys,
                       unsigned* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t* pb = reinterpret_cast<const uint64_t*>(pos);
    const uint64_t x = pb[3 * i], y = pb[3 * i + 1], z = pb[3 * i + 2];
    if (!(unit_bits(x) && unit_bits(y) && unit_bits(z))) atomicOr(err, kErrRange);
    keys[i] = hilbert_key(grid21(x), grid21(y), grid21(z));
}

// ---------------------------------------------------------------------------------
// Exclusive scan (int32 / int64), three phases: tile sums, scan of the sums
// (recursive), tile scan with carry.  Tiles of 4096 = 1024 threads x 4 items.
// ---------------------------------------------------------------------------------

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive(T v, T* warp_tot, T& block_total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : T(0);
        T si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        warp_tot[lane] = si - s;  // exclusive prefix of warp totals
        if (lane == 31) warp_tot[32] = si;
    }
    __syncthreads();
    block_total = warp_tot[32];
    T r = warp_tot[w] + inc - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, T* __restrict__ sums) {
    __shared__ T wt[33];
    int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    T tot;
    block_exclusive<T>(s, wt, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_down(const T* in, T* out, int64_t n, const T* __restrict__ carry,
                            T* total) {
    __shared__ T wt[33];
    int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : T(0);
        s += v[k];
    }
    T tot;
    T ex = block_exclusive<T>(s, wt, tot);
    T c = carry ? carry[blockIdx.x] : T(0);
    T run = c + ex;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *total = c + tot;
}

template <typename T>
static void scan_rec(const T* in, T* out, int64_t n, T* aux, T* total, cudaStream_t s) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= 1) {
        k_scan_down<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total);
        note_launch();
        return;
    }
    k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, aux);
    note_launch();
    scan_rec<T>(aux, aux, nb, aux + nb, nullptr, s);
    k_scan_down<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, aux, total);
    note_launch();
}

static int64_t scan_aux_need(int64_t n) {
    int64_t need = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        need += n;
    }
    return need + 8;
}

int exclusive_scan_i32(Ctx* c, const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev,
                       cudaStream_t s) {
    if (n <= 0) return SPHGRP_OK;
    if (scan_aux_need(n) > c->scan_aux_cap) return set_error(SPHGRP_EOVERFLOW, "scan scratch too small");
    scan_rec<int32_t>(in, out, n, c->scan_aux, total_dev, s);
    return check_cuda(cudaGetLastError(), "scan");
}

int exclusive_scan_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                       cudaStream_t s) {
    if (n <= 0) return SPHGRP_OK;
    if (2 * scan_aux_need(n) > c->scan_aux_cap) return set_error(SPHGRP_EOVERFLOW, "scan scratch too small");
    scan_rec<int64_t>(in, out, n, reinterpret_cast<int64_t*>(c->scan_aux), total_dev, s);
    return check_cuda(cudaGetLastError(), "scan");
}

// ---------------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, stable.  Per pass: tile histograms (digit-major),
// exclusive scan, and a scatter that ranks keys inside the tile with warp matching.
// A tile is 256 threads x 8 keys; warp w owns the contiguous 256 keys
// [w*256, w*256+256) of the tile, processed 32 at a time in order, so ranks follow
// the input order (stability).  The scatter first sorts the tile by digit in shared
// memory, then writes every digit's run with consecutive threads on consecutive
// addresses (about 8 keys per run and tile), instead of one scattered store per key.
// ---------------------------------------------------------------------------------

constexpr int kSortWarps = kSortThreads / 32;

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                             uint32_t* __restrict__ hist, int nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = blockIdx.x * (int64_t)kSortTile;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        int64_t i = base + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t* __restrict__ kin,
                                                                const int32_t* __restrict__ vin,
                                                                uint64_t* __restrict__ kout,
                                                                int32_t* __restrict__ vout, int64_t n, int shift,
                                                                const uint32_t* __restrict__ offs, int nblocks) {
    __shared__ uint32_t wh[kSortWarps][256];
    __shared__ uint32_t gbase[256];    // global position of the tile's run of every digit
    __shared__ uint32_t lbase[256];    // tile-local position of the same run
    __shared__ uint32_t wsum[kSortWarps];
    __shared__ uint64_t sk[kSortTile];  // the tile, sorted by digit (stable)
    __shared__ int32_t sv[kSortTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortThreads) (&wh[0][0])[d] = 0;
    gbase[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
    const int64_t tile0 = blockIdx.x * (int64_t)kSortTile;
    const int64_t base = tile0 + w * 256;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t kk[kSortItems];
    int32_t vv[kSortItems];
    uint32_t rk[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * 32 + lane;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0ull;
        kk[r] = key;
        vv[r] = valid ? (vin ? vin[i] : (int32_t)i) : 0;
        uint32_t d = valid ? (uint32_t)((key >> shift) & 0xffu) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t prev = (d < 256u) ? wh[w][d] : 0u;
        __syncwarp();
        if (d < 256u && lane == __ffs(peers) - 1) wh[w][d] = prev + __popc(peers);
        __syncwarp();
        rk[r] = prev + __popc(peers & lt);
    }
    __syncthreads();
    // per digit (thread t owns digit t): exclusive prefix over the warps, then the
    // tile-local start of the digit's run (exclusive scan of the digit totals)
    {
        uint32_t run = 0;
        const int d = threadIdx.x;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ++ww) {
            uint32_t c = wh[ww][d];
            wh[ww][d] = run;
            run += c;
        }
        uint32_t v = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        uint32_t off = 0;
        for (int ww = 0; ww < w; ++ww) off += wsum[ww];
        lbase[d] = off + v - run;
    }
    __syncthreads();
    // the tile in digit order in shared memory
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * 32 + lane;
        if (i < n) {
            const uint32_t d = (uint32_t)((kk[r] >> shift) & 0xffu);
            const uint32_t p = lbase[d] + wh[w][d] + rk[r];
            sk[p] = kk[r];
            sv[p] = vv[r];
        }
    }
    __syncthreads();
    // runs of equal digits go out with consecutive threads on consecutive addresses
    const int cnt = (int)min((int64_t)kSortTile, n - tile0);
    for (int e = threadIdx.x; e < cnt; e += kSortThreads) {
        const uint64_t key = sk[e];
        const uint32_t d = (uint32_t)((key >> shift) & 0xffu);
        const uint32_t p = gbase[d] + ((uint32_t)e - lbase[d]);
        kout[p] = key;
        vout[p] = sv[e];
    }
}

__global__ void k_invert_perm(int64_t n, const int32_t* __restrict__ perm, int32_t* __restrict__ rank_of) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) rank_of[perm[r]] = (int32_t)r;
}

int sort_keys(Ctx* c, int64_t n, const double* pos, cudaStream_t s) {
    // keys in input order go to keys_alt; the passes ping-pong keys_alt <-> keys
    k_keys<<<blocks_for(n, 256), 256, 0, s>>>(n, pos, c->keys_alt, c->err);
    note_launch();
    int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    int64_t nh = (int64_t)256 * nblocks;
    if (nh > c->hist_cap) return set_error(SPHGRP_EOVERFLOW, "radix histogram scratch too small");
    uint64_t* kin = c->keys_alt;
    uint64_t* kout = c->keys;
    int32_t* vin = nullptr;
    int32_t* vout = c->perm;
    for (int pass = 0; pass < 8; ++pass) {
        int shift = 8 * pass;
        k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(kin, n, shift, c->hist, nblocks);
        note_launch();
        int rc = exclusive_scan_i32(c, reinterpret_cast<const int32_t*>(c->hist),
                                    reinterpret_cast<int32_t*>(c->hist), nh, nullptr, s);
        if (rc) return rc;
        k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, c->hist, nblocks);
        note_launch();
        // swap
        uint64_t* tk = kin; kin = kout; kout = tk;
        if (pass == 0) { vin = c->perm; vout = c->perm_alt; }
        else { int32_t* tv = vin; vin = vout; vout = tv; }
    }
    // the last pass wrote into the alternate buffers: swap the context's pointers
    if (kin != c->keys) { uint64_t* t = c->keys; c->keys = c->keys_alt; c->keys_alt = t; }
    if (vin != c->perm) { int32_t* t = c->perm; c->perm = c->perm_alt; c->perm_alt = t; }
    k_invert_perm<<<blocks_for(n, 256), 256, 0, s>>>(n, c->perm, c->rank_of);
    note_launch();
    return check_cuda(cudaGetLastError(), "sort");
}

// ---------------------------------------------------------------------------------
// Scan over a count held in device memory (n = *n_hi - *n_lo, at most n_bound), for
// graph-captured sequences: the grids cover n_bound; tiles beyond n contribute zero.
// ---------------------------------------------------------------------------------

__device__ __forceinline__ int64_t dev_count(const int32_t* n_hi, const int32_t* n_lo, int64_t n_bound) {
    int64_t n = (int64_t)*n_hi - (n_lo ? (int64_t)*n_lo : 0);
    return n < 0 ? 0 : (n > n_bound ? n_bound : n);
}

template <typename T>
__global__ void k_scan_reduce_dev(const T* __restrict__ in, const int32_t* n_hi, const int32_t* n_lo,
                                  int64_t n_bound, T* __restrict__ sums) {
    __shared__ T wt[33];
    const int64_t n = dev_count(n_hi, n_lo, n_bound);
    const int64_t tile0 = blockIdx.x * (int64_t)kScanTile;
    if (tile0 >= n) {   // block-uniform
        if (threadIdx.x == 0) sums[blockIdx.x] = T(0);
        return;
    }
    int64_t base = tile0 + threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    T tot;
    block_exclusive<T>(s, wt, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_down_dev(const T* in, T* out, const int32_t* n_hi, const int32_t* n_lo, int64_t n_bound,
                                const T* __restrict__ carry, T* total) {
    __shared__ T wt[33];
    const int64_t n = dev_count(n_hi, n_lo, n_bound);
    const int64_t tile0 = blockIdx.x * (int64_t)kScanTile;
    const bool last_block = blockIdx.x == gridDim.x - 1;
    if (tile0 >= n && !last_block) return;   // block-uniform
    int64_t base = tile0 + threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : T(0);
        s += v[k];
    }
    T tot;
    T ex = block_exclusive<T>(s, wt, tot);
    T c = carry ? carry[blockIdx.x] : T(0);
    T run = c + ex;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (total && last_block && threadIdx.x == blockDim.x - 1) *total = c + tot;
}

int exclusive_scan_i32_dev(Ctx* c, const int32_t* in, int32_t* out, const int32_t* n_hi, const int32_t* n_lo,
                           int64_t n_bound, int32_t* total_dev, cudaStream_t s) {
    if (n_bound <= 0) n_bound = 1;
    const int64_t nb = (n_bound + kScanTile - 1) / kScanTile;
    if (nb <= 1) {
        k_scan_down_dev<int32_t><<<1, kScanThreads, 0, s>>>(in, out, n_hi, n_lo, n_bound, nullptr, total_dev);
        note_launch();
        return check_cuda(cudaGetLastError(), "scan (device count)");
    }
    if (scan_aux_need(nb) + nb > c->scan_aux_cap) return set_error(SPHGRP_EOVERFLOW, "scan scratch too small");
    k_scan_reduce_dev<int32_t><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n_hi, n_lo, n_bound, c->scan_aux);
    note_launch();
    scan_rec<int32_t>(c->scan_aux, c->scan_aux, nb, c->scan_aux + nb, nullptr, s);
    k_scan_down_dev<int32_t><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n_hi, n_lo, n_bound, c->scan_aux,
                                                                    total_dev);
    note_launch();
    return check_cuda(cudaGetLastError(), "scan (device count)");
}

// ---------------------------------------------------------------------------------
// Sort of several boxes at once: keys as above, then one stable pass per byte of the
// box index, so that the order is (box, key); the context's keys and perm end in
// that order and box_of_rank holds every rank's box.
// ---------------------------------------------------------------------------------

__global__ void k_box_digit(int64_t n, const int32_t* __restrict__ perm, const int64_t* __restrict__ box_off,
                            int nbox, uint64_t* __restrict__ dkey) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t i = perm[r];
    int lo = 0, hi = nbox;   // box_off[lo] <= i < box_off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (box_off[mid] <= i) lo = mid; else hi = mid;
    }
    dkey[r] = (uint64_t)lo;
}

__global__ void k_box_gather(int64_t n, const int32_t* __restrict__ src, const uint64_t* __restrict__ keys,
                             const int32_t* __restrict__ perm, const uint64_t* __restrict__ dkey,
                             uint64_t* __restrict__ keys_out, int32_t* __restrict__ perm_out,
                             int32_t* __restrict__ box_of_rank) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t r = src[p];
    keys_out[p] = keys[r];
    perm_out[p] = perm[r];
    box_of_rank[p] = (int32_t)dkey[p];
}

int sort_keys_boxed(Ctx* c, int64_t n, const double* pos, const int64_t* box_off_dev, int nbox, uint64_t* tmp64a,
                    uint64_t* tmp64b, int32_t* tmp32a, int32_t* tmp32b, int32_t* box_of_rank, cudaStream_t s) {
    int rc = sort_keys(c, n, pos, s);
    if (rc) return rc;
    if (nbox <= 1) {
        cudaMemsetAsync(box_of_rank, 0, n * sizeof(int32_t), s);
        return check_cuda(cudaGetLastError(), "box sort");
    }
    k_box_digit<<<blocks_for(n, 256), 256, 0, s>>>(n, c->perm, box_off_dev, nbox, tmp64a);
    note_launch();
    const int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    const int64_t nh = (int64_t)256 * nblocks;
    if (nh > c->hist_cap) return set_error(SPHGRP_EOVERFLOW, "radix histogram scratch too small");
    const int passes = nbox > 256 ? 2 : 1;
    uint64_t* kin = tmp64a;
    uint64_t* kout = tmp64b;
    const int32_t* vin = nullptr;
    int32_t* vout = tmp32a;
    for (int pass = 0; pass < passes; ++pass) {
        k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(kin, n, 8 * pass, c->hist, nblocks);
        note_launch();
        if ((rc = exclusive_scan_i32(c, reinterpret_cast<const int32_t*>(c->hist), reinterpret_cast<int32_t*>(c->hist),
                                     nh, nullptr, s)))
            return rc;
        k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, 8 * pass, c->hist, nblocks);
        note_launch();
        std::swap(kin, kout);
        vin = vout;
        vout = (vout == tmp32a) ? tmp32b : tmp32a;
    }
    // kin: box digits in (box, key) order; vin: the rank in key order of every position
    k_box_gather<<<blocks_for(n, 256), 256, 0, s>>>(n, vin, c->keys, c->perm, kin, c->keys_alt, c->perm_alt,
                                                     box_of_rank);
    note_launch();
    std::swap(c->keys, c->keys_alt);
    std::swap(c->perm, c->perm_alt);
    k_invert_perm<<<blocks_for(n, 256), 256, 0, s>>>(n, c->perm, c->rank_of);
    note_launch();
    return check_cuda(cudaGetLastError(), "box sort");
}

// The same keys + stable radix sort on caller-provided buffers: the sorted keys and
// the permutation end in keys_out / perm_out (which also serve as one ping-pong pair;
// eight passes return to them), keys_alt / perm_alt are the other pair, hist holds
// hist_words >= 256 * ceil(n / kSortTile) counters and scan_aux the scan's block sums
// (scan_aux_words entries).  err receives the range-check flag.  No allocation.
int sort_keys_scratch(int64_t n, const double* pos, uint64_t* keys_out, int32_t* perm_out,
                      uint64_t* keys_alt, int32_t* perm_alt, uint32_t* hist, int64_t hist_words,
                      int32_t* scan_aux, int64_t scan_aux_words, unsigned* err, cudaStream_t s) {
    const int nblocks = (int)((n + kSortTile - 1) / kSortTile);
    const int64_t nh = (int64_t)256 * nblocks;
    if (nh > hist_words) return set_error(SPHGRP_EOVERFLOW, "histogram scratch too small");
    if (scan_aux_need(nh) > scan_aux_words) return set_error(SPHGRP_EOVERFLOW, "scan scratch too small");
    k_keys<<<blocks_for(n, 256), 256, 0, s>>>(n, pos, keys_out, err);
    note_launch();
    uint64_t* kbuf[2] = {keys_out, keys_alt};
    int32_t* vbuf[2] = {perm_out, perm_alt};
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 8 * pass;
        uint64_t* kin = kbuf[pass & 1];
        uint64_t* kout = kbuf[(pass + 1) & 1];
        const int32_t* vin = pass == 0 ? nullptr : vbuf[pass & 1];
        int32_t* vout = vbuf[(pass + 1) & 1];
        k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(kin, n, shift, hist, nblocks);
        note_launch();
        scan_rec<int32_t>(reinterpret_cast<const int32_t*>(hist), reinterpret_cast<int32_t*>(hist), nh,
                          scan_aux, nullptr, s);
        k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, hist, nblocks);
        note_launch();
    }
    return check_cuda(cudaGetLastError(), "sort (caller buffers)");
}

}  // namespace sphgrp
