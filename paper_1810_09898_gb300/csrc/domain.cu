// Domain decomposition with halo import, for one particle set split over several GPUs.
//
// The paper's code splits the particles along the Hilbert curve into one contiguous key
// range per MPI process (Sec. 1.2) and finds neighbours across the ranges by exporting
// particles to the processes whose nodes their walks open, in a second search phase
// (Sec. 1.1).  Here every rank instead imports, before its search, the particles of the
// other ranks that any of its own particles can reach (the halo); the walk is then local
// to the rank.  These kernels are the per-rank steps of that scheme; the exchanges run
// on the host (torch.distributed, paper_1810_09898_gb300/domain.py):
//   * sphgrp_key_split: the owner rank of every particle (as a one-bit mask) from the
//     splitters of the key order (the rank's range is [splitter_{r-1}, splitter_r));
//   * sphgrp_domain_boxes: the rank's domain as the tight boxes of its particles in every
//     octree cell of a given level they occupy (cells are key-prefix blocks, so the key
//     order holds each cell's particles contiguously), with the largest h in each box;
//   * sphgrp_halo_select: the ranks every own particle must be sent to.  For density a
//     particle j is a neighbour of i iff |x_j - x_i| < h_i, so j is needed by a remote
//     box B (holding i) iff dist(x_j, B) < hmax(B); for hydro iff dist(x_j, B) <
//     max(hmax(B), h_j).  Distances are periodic (minimum image per axis);
//   * sphgrp_mask_compact: the own particles flagged for one rank, ascending.
#include "sph_internal.cuh"

namespace sphgrp {

int exclusive_scan_i32(Ctx* c, const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev, cudaStream_t s);

namespace {

__global__ void k_key_split(int64_t n, const uint64_t* __restrict__ keys, const int32_t* __restrict__ perm,
                            int nsplit, const uint64_t* __restrict__ split, uint64_t* __restrict__ dest) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint64_t k = keys[r];
    int lo = 0, hi = nsplit;   // number of splitters <= k
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (split[mid] <= k) lo = mid + 1; else hi = mid;
    }
    dest[perm[r]] = (uint64_t)1 << lo;
}

// cell heads of the key order at a given level (3 * level key bits)
__global__ void k_cell_heads(int64_t n, const uint64_t* __restrict__ keys, int shift, int32_t* __restrict__ head) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    head[r] = (r == 0 || (keys[r] >> shift) != (keys[r - 1] >> shift)) ? 1 : 0;
}

// box {lo[3], hi[3]} in fixed point (inclusive), hmax bits, count, per cell
struct FixBox {
    uint32_t lo[3], hi[3];
    uint32_t hmax;   // FP32 bits of the largest h (non-negative: integer order = float order)
    uint32_t count;
};

__global__ void k_box_init(int nb, FixBox* __restrict__ b) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    for (int a = 0; a < 3; ++a) {
        b[k].lo[a] = 0xffffffffu;
        b[k].hi[a] = 0u;
    }
    b[k].hmax = 0u;
    b[k].count = 0u;
}

__global__ void k_box_reduce(int64_t n, const int32_t* __restrict__ head, const int32_t* __restrict__ seg,
                             const uint4* __restrict__ pfix, const int32_t* __restrict__ perm,
                             const double* __restrict__ h, FixBox* __restrict__ b) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int k = seg[r] + head[r] - 1;   // inclusive segment index
    const uint4 P = pfix[r];
    atomicMin(&b[k].lo[0], P.x);
    atomicMin(&b[k].lo[1], P.y);
    atomicMin(&b[k].lo[2], P.z);
    atomicMax(&b[k].hi[0], P.x);
    atomicMax(&b[k].hi[1], P.y);
    atomicMax(&b[k].hi[2], P.z);
    // the FP32 copy of h rounded up, so that hmax covers the FP64 h
    const float hf = __double2float_ru(h[perm[r]]);
    atomicMax(&b[k].hmax, __float_as_uint(hf));
    atomicAdd(&b[k].count, 1u);
}

// fixed point -> box coordinates: a particle at X (with its sub-unit offset in [0, 1))
// lies in [X, X + 1) units, so the box is [lo, hi + 1) * 2^-32
__global__ void k_box_out(int nb, const FixBox* __restrict__ b, double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const double u = 1.0 / 4294967296.0;
    for (int a = 0; a < 3; ++a) {
        out[8 * (int64_t)k + a] = (double)b[k].lo[a] * u;
        out[8 * (int64_t)k + 3 + a] = ((double)b[k].hi[a] + 1.0) * u;
    }
    out[8 * (int64_t)k + 6] = (double)__uint_as_float(b[k].hmax);
    out[8 * (int64_t)k + 7] = (double)b[k].count;
}

// squared periodic distance from a point in [0,1)^3 to a box inside the unit cube
__device__ __forceinline__ double box_gap2(double x, double y, double z, const double* b) {
    const double p[3] = {x, y, z};
    double s = 0.0;
    for (int a = 0; a < 3; ++a) {
        double best = 1.0;
        for (int sh = -1; sh <= 1; ++sh) {
            const double q = p[a] + (double)sh;
            best = fmin(best, fmax(0.0, fmax(b[a] - q, q - b[3 + a])));
        }
        s += best * best;
    }
    return s;
}

__global__ void k_halo_select(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ xd,
                              const double* __restrict__ yd, const double* __restrict__ zd,
                              const double* __restrict__ h, int kind, double widen, int nbox,
                              const double* __restrict__ boxes,
                              const int32_t* __restrict__ box_rank, int self_rank, int world,
                              uint64_t* __restrict__ mask, unsigned long long* __restrict__ counts,
                              unsigned* err) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t i = perm[r];
    const double x = xd[r], y = yd[r], z = zd[r], hj = h[i];
    uint64_t m = 0;
    for (int b = 0; b < nbox; ++b) {
        const int rk = box_rank[b];
        if (rk < 0 || rk >= world) {   // the caller's rank array: skipped, reported
            if (r == 0) atomicOr(err, kErrRank);
            continue;
        }
        if (rk == self_rank || ((m >> rk) & 1u)) continue;
        const double* B = boxes + 8 * (int64_t)b;
        const double reach = kind == SPHGRP_HYDRO ? fmax(widen * B[6], hj) : widen * B[6];
        // a relative margin over the rounding of the gap (the neighbour tests are strict)
        if (box_gap2(x, y, z, B) < reach * reach * (1.0 + 1e-12)) m |= (uint64_t)1 << rk;
    }
    mask[i] = m;
    while (m) {
        const int rk = __ffsll((long long)m) - 1;
        m &= m - 1;
        atomicAdd(&counts[rk], 1ull);
    }
}

__global__ void k_mask_bit(int64_t n, const uint64_t* __restrict__ mask, int bit, int32_t* __restrict__ flag) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (int32_t)((mask[i] >> bit) & 1u);
}

__global__ void k_flag_compact(int64_t n, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                               int32_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = (int32_t)i;
}

}  // namespace
}  // namespace sphgrp

using namespace sphgrp;

extern "C" {

int sphgrp_key_split(sphgrp_ctx* ctx, int nsplit, const uint64_t* splitters, uint64_t* dest, cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c) return set_error(SPHGRP_EINVAL, "null context");
    if (!c->sorted) return set_error(SPHGRP_ESTATE, "key_split needs a preceding sfc_keys_sort");
    if (nsplit < 0 || nsplit > 63 || (nsplit > 0 && !splitters) || !dest)
        return set_error(SPHGRP_EINVAL, "nsplit outside [0, 63] or null array");
    k_key_split<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->keys, c->perm, nsplit, splitters, dest);
    note_launch();
    return check_cuda(cudaGetLastError(), "key split");
}

int sphgrp_domain_boxes(sphgrp_ctx* ctx, const double* h, int level, int cap, double* boxes, int* nbox,
                        cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c) return set_error(SPHGRP_EINVAL, "null context");
    if (!c->built) return set_error(SPHGRP_ESTATE, "domain_boxes needs a preceding tree_build");
    if (!h || !boxes || !nbox || cap < 1 || level < 0 || level > kKeyLevels)
        return set_error(SPHGRP_EINVAL, "null array, cap < 1 or level outside [0, 21]");
    const int64_t n = c->n;
    // heads and segment numbers (c->flag, c->scan), the boxes in c->hyd0 (48 B <= 2 x 16 B
    // per box, at most n boxes)
    k_cell_heads<<<blocks_for(n, 256), 256, 0, s>>>(n, c->keys, 3 * (kKeyLevels - level), c->flag);
    note_launch();
    int32_t* total = reinterpret_cast<int32_t*>(c->work) + 24;
    int rc = exclusive_scan_i32(c, c->flag, c->scan, n, total, s);
    if (rc) return rc;
    cudaMemcpyAsync(c->host_small + 44, total, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "box count"))) return rc;
    const int nb = c->host_small[44];
    *nbox = nb;
    if (nb > cap) return set_error(SPHGRP_EOVERFLOW, "more domain boxes than cap");
    if ((int64_t)nb * (int64_t)sizeof(FixBox) > c->n_max * (int64_t)sizeof(float4))
        return set_error(SPHGRP_EOVERFLOW, "level too deep: more domain boxes than half the particles");
    FixBox* fb = reinterpret_cast<FixBox*>(c->hyd0);
    static_assert(sizeof(FixBox) <= 2 * sizeof(float4), "a box takes at most two hyd0 entries");
    k_box_init<<<blocks_for(nb, 256), 256, 0, s>>>(nb, fb);
    note_launch();
    k_box_reduce<<<blocks_for(n, 256), 256, 0, s>>>(n, c->flag, c->scan, c->pfix, c->perm, h, fb);
    note_launch();
    k_box_out<<<blocks_for(nb, 256), 256, 0, s>>>(nb, fb, boxes);
    note_launch();
    return check_cuda(cudaGetLastError(), "domain boxes");
}

int sphgrp_halo_select(sphgrp_ctx* ctx, const double* h, int kind, double widen, int nbox, const double* boxes,
                       const int32_t* box_rank, int self_rank, int world, uint64_t* mask, int64_t* counts,
                       cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c) return set_error(SPHGRP_EINVAL, "null context");
    if (!c->built) return set_error(SPHGRP_ESTATE, "halo_select needs a preceding tree_build");
    if (kind != SPHGRP_DENSITY && kind != SPHGRP_HYDRO) return set_error(SPHGRP_EINVAL, "bad kind");
    if (!(widen >= 1.0 && widen <= 4.0)) return set_error(SPHGRP_EINVAL, "widen outside [1, 4]");
    if (world < 1 || world > 64 || self_rank < 0 || self_rank >= world || nbox < 0 || !h || !mask || !counts ||
        (nbox > 0 && (!boxes || !box_rank)))
        return set_error(SPHGRP_EINVAL, "world outside [1, 64], bad rank or null array");
    cudaMemsetAsync(counts, 0, world * sizeof(int64_t), s);
    cudaMemsetAsync(c->err, 0, sizeof(unsigned), s);
    k_halo_select<<<blocks_for(c->n, 128), 128, 0, s>>>(c->n, c->perm, c->xd, c->yd, c->zd, h, kind, widen, nbox, boxes,
                                                        box_rank, self_rank, world, mask,
                                                        reinterpret_cast<unsigned long long*>(counts), c->err);
    note_launch();
    // the box ranks are device data: their check is read back (one stream synchronisation)
    int rc = check_cuda(cudaMemcpyAsync(c->host_small, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s),
                        "halo select status");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "halo select");
    if (rc) return rc;
    if ((unsigned)c->host_small[0] & kErrRank) return set_error(SPHGRP_EINVAL, "a box rank is outside [0, world)");
    return SPHGRP_OK;
}

int sphgrp_mask_compact(sphgrp_ctx* ctx, int64_t n, const uint64_t* mask, int bit, int32_t* idx, int64_t* count,
                        cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c) return set_error(SPHGRP_EINVAL, "null context");
    if (n < 1 || n > c->n_max) return set_error(SPHGRP_EINVAL, "n outside [1, n_max]");
    if (!mask || !idx || !count || bit < 0 || bit > 63) return set_error(SPHGRP_EINVAL, "bad bit or null array");
    k_mask_bit<<<blocks_for(n, 256), 256, 0, s>>>(n, mask, bit, c->flag);
    note_launch();
    int32_t* total = reinterpret_cast<int32_t*>(c->work) + 25;
    int rc = exclusive_scan_i32(c, c->flag, c->scan, n, total, s);
    if (rc) return rc;
    k_flag_compact<<<blocks_for(n, 256), 256, 0, s>>>(n, c->flag, c->scan, idx);
    note_launch();
    cudaMemcpyAsync(c->host_small + 45, total, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "compact count"))) return rc;
    *count = c->host_small[45];
    return SPHGRP_OK;
}

}  // extern "C"
