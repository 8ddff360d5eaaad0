// Batched solve of many independent periodic boxes (C ABI sphgrp_batch_*).
//
// All boxes live in one context: their particles are sorted by (box, key), one octree
// per box forms a forest whose roots are nodes 0 .. nbox-1, and every box's active
// particles are cut into groups that never cross a box (each group walks from its
// box's root).  Every phase is one persistent work-queue kernel over the groups of all
// boxes, so boxes of very different sizes share the GPU without per-box launches:
//   density with the smoothing-length iteration inside the group (k_group_dens_iter),
//   hydro forces, and with the backward the hydro-adjoint items in the same queue as
//   the hydro items (k_group_pair), then the density adjoint.
// Counts (active particles, chunks, groups, tree levels) never leave the device, so
// the call has no host synchronisation until its final status read and can be
// captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "search_args.cuh"

namespace sphgrp {

namespace {

constexpr int kGrid = 1024;   // blocks of the grid-stride kernels
constexpr int kLevels = kKeyLevels + 3;
constexpr int kMaxTableBoxes = 256;   // boxes that get a walk start table
constexpr int kMinBatchLeaf = 8;      // smallest per-class leaf size: the forest's node
                                      // capacity (n/2 + 64 per box) holds trees of leaves >= 8

// device scalars of a batch call
enum Scalar {
    kNu = 0,         // active particles
    kNChunk = 1,     // chunks of the active list
    kNGroups = 2,    // groups of the active list
    kNChunkAll = 3,  // chunks of the all-particle list (backward)
    kNGroupsAll = 4, // groups of the all-particle list
    kNFail = 5,      // particles that did not converge
    kTot = 6,        // scan total scratch
    kNScalars = 16
};

struct ClassCfg {
    int g = 16;
    int smax = 4;
    float split = 2.0f;
    float tuned_ms = 0.0f;        // the tuner's best density + hydro pass over the class
    int64_t tuned_members = 0;    // active particles of that pass
    int leaf = 0;                 // octree leaf size of the class's boxes (0: the context's)
};

struct Batch {
    Ctx* c = nullptr;
    int nbox = 0;
    int64_t n = 0;
    std::vector<int64_t> box_off_h;
    std::vector<int32_t> cls_h;
    ClassCfg cfg[SPHGRP_BATCH_CLASSES];
    int max_g = 16;
    // device
    int64_t* box_off = nullptr;     // nbox + 1
    int32_t* box_g = nullptr;       // nbox: g | smax << 8 | leaf size << 16
    float* box_split = nullptr;     // nbox
    int32_t* box_cls = nullptr;     // nbox
    int32_t* box_of_rank = nullptr; // n
    uint64_t* tmp64a = nullptr;     // sort scratch
    uint64_t* tmp64b = nullptr;
    int32_t* tmp32a = nullptr;
    int32_t* tmp32b = nullptr;
    int32_t* lvl = nullptr;         // forest level table
    uint4* blo = nullptr;
    uint4* bhi = nullptr;
    int32_t* U_all = nullptr;       // identity work list
    int32_t* dsc = nullptr;         // device scalars
    int32_t* box_act = nullptr;     // nbox + 1: first entry of the box in the work list
    int32_t* box_chunk = nullptr;   // nbox + 1: first chunk of the box
    int4* chunks = nullptr;         // (first entry, count, box, -)
    int32_t* ccnt = nullptr;        // groups per chunk
    int32_t* coff = nullptr;
    int2* gtmp = nullptr;           // split output
    int4* groups = nullptr;         // active groups
    int4* groups_all = nullptr;     // all-particle groups (backward)
    float4* hyd0b = nullptr;        // hydro inputs of the backward (all particles at h)
    float4* hyd1b = nullptr;
    int32_t* start_tabs = nullptr;  // walk start tables, one per box
    // graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long exec_kernels = 0;
    sphgrp_batch_io cap_io{};
    int cap_flags = -1;
    // pinned host status: [0] err, [1] nfail, [2..] scalars; counters after
    int32_t* host = nullptr;
    DevCounters* host_ctr = nullptr;
    bool replayed = false;
    int64_t walks = 0, members = 0;
    long long step_kernels = 0;
};

__device__ __forceinline__ int warp_scan_incl(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__global__ void k_iota(int64_t n, int32_t* __restrict__ out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        out[r] = (int32_t)r;
}

// flag[r] = 1 for active ranks (optionally only those of one class)
__global__ void k_batch_flags(int64_t n, const int32_t* __restrict__ perm, const uint8_t* __restrict__ active,
                              const int32_t* __restrict__ box_of_rank, const int32_t* __restrict__ box_cls,
                              int only_cls, int32_t* __restrict__ flag) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        int f = active ? (active[perm[r]] != 0) : 1;
        if (only_cls >= 0 && box_cls[box_of_rank[r]] != only_cls) f = 0;
        flag[r] = f;
    }
}

__global__ void k_batch_compact(int64_t n, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                int32_t* __restrict__ U) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        if (flag[r]) U[pos[r]] = (int32_t)r;
}

// One warp: per box, the first entry of the work list (from the flag scan, or the box
// offsets for the all-particle list) and the chunk offsets (chunks of g entries).
__global__ void k_box_chunks(int nbox, const int64_t* __restrict__ box_off, const int32_t* __restrict__ scan,
                             const int32_t* __restrict__ nu_dev, int all, int64_t n,
                             const int32_t* __restrict__ box_g, int32_t* __restrict__ box_act,
                             int32_t* __restrict__ box_chunk, int32_t* __restrict__ nchunk) {
    const int lane = threadIdx.x;
    const int nu = all ? (int)n : *nu_dev;
    int run = 0;
    for (int b0 = 0; b0 < nbox; b0 += 32) {
        const int b = b0 + lane;
        int ch = 0;
        if (b < nbox) {
            const int a0 = all ? (int)box_off[b] : scan[box_off[b]];
            const int a1 = (b + 1 < nbox) ? (all ? (int)box_off[b + 1] : scan[box_off[b + 1]]) : nu;
            const int g = box_g[b] & 0xff;
            ch = (a1 - a0 + g - 1) / g;
            box_act[b] = a0;
        }
        const int inc = warp_scan_incl(ch, lane);
        if (b < nbox) box_chunk[b] = run + inc - ch;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) {
        box_chunk[nbox] = run;
        box_act[nbox] = nu;
        *nchunk = run;
    }
}

__global__ void k_chunk_desc(int nbox, const int32_t* __restrict__ box_act, const int32_t* __restrict__ box_chunk,
                             const int32_t* __restrict__ box_g, const int32_t* __restrict__ nchunk,
                             int4* __restrict__ chunks) {
    const int nc = *nchunk;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        int lo = 0, hi = nbox;   // box_chunk[lo] <= c < box_chunk[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (box_chunk[mid] <= c) lo = mid; else hi = mid;
        }
        const int g = box_g[lo] & 0xff;
        const int start = box_act[lo] + (c - box_chunk[lo]) * g;
        chunks[c] = make_int4(start, min(g, box_act[lo + 1] - start), lo, 0);
    }
}

// The chunk cut in halves (recursively) while the group's search sphere exceeds split
// times its members' spheres in volume (as k_split_groups); output at the chunk's
// first entry (a chunk of c entries gives at most c groups).
__global__ void k_split_chunks(const int32_t* __restrict__ U, const int4* __restrict__ chunks,
                               const int32_t* __restrict__ nchunk, const uint4* __restrict__ pfix,
                               const double* __restrict__ h64, const float* __restrict__ box_split,
                               int2* __restrict__ tmp, int32_t* __restrict__ cnt) {
    const int nc = *nchunk;
    for (int ch = blockIdx.x * blockDim.x + threadIdx.x; ch < nc; ch += gridDim.x * blockDim.x) {
        const int4 C = chunks[ch];
        const float split = box_split[C.z];
        int2 st[16];
        int sp = 0, ng = 0;
        st[sp++] = make_int2(C.x, C.x + C.y);
        while (sp > 0) {
            const int2 r = st[--sp];
            const int s = r.x, e = r.y;
            bool keep = (e - s == 1) || split <= 0.0f;
            if (!keep) {
                const uint4 P0 = pfix[U[s]];
                int lox = 0, loy = 0, loz = 0, hix = 0, hiy = 0, hiz = 0;
                float hmin = (float)h64[U[s]];
                for (int k = s + 1; k < e; ++k) {
                    const int rk = U[k];
                    const uint4 P = pfix[rk];
                    const int dx = (int32_t)(P.x - P0.x), dy = (int32_t)(P.y - P0.y), dz = (int32_t)(P.z - P0.z);
                    lox = min(lox, dx); hix = max(hix, dx);
                    loy = min(loy, dy); hiy = max(hiy, dy);
                    loz = min(loz, dz); hiz = max(hiz, dz);
                    hmin = fminf(hmin, (float)h64[rk]);
                }
                const float ext = fmaxf(fmaxf((float)((int64_t)hix - lox), (float)((int64_t)hiy - loy)),
                                        (float)((int64_t)hiz - loz)) * kUnitToBox;
                const float rel = fmaf(0.8660254f, ext / hmin, 1.0f);
                keep = rel * rel * rel <= split * (float)(e - s);
            }
            if (keep) {
                tmp[C.x + ng++] = make_int2(s, e - s);
            } else if (sp + 2 <= 16) {
                const int mid = s + (e - s + 1) / 2;
                st[sp++] = make_int2(mid, e);
                st[sp++] = make_int2(s, mid);
            } else {
                tmp[C.x + ng++] = make_int2(s, e - s);
            }
        }
        cnt[ch] = ng;
    }
}

__global__ void k_gather_chunk_groups(const int4* __restrict__ chunks, const int32_t* __restrict__ nchunk,
                                      const int32_t* __restrict__ cnt, const int32_t* __restrict__ off,
                                      const int2* __restrict__ tmp, const int32_t* __restrict__ box_g,
                                      int4* __restrict__ groups) {
    const int nc = *nchunk;
    for (int ch = blockIdx.x * blockDim.x + threadIdx.x; ch < nc; ch += gridDim.x * blockDim.x) {
        const int4 C = chunks[ch];
        const int o = off[ch];
        const int gw = box_g[C.z];
        for (int k = 0; k < cnt[ch]; ++k) {
            const int2 t = tmp[C.x + k];
            groups[o + k] = make_int4(t.x, t.y, C.z, gw);
        }
    }
}

template <typename T>
int dalloc(T** p, int64_t count) {
    if (count < 1) count = 1;
    return check_cuda(cudaMalloc(reinterpret_cast<void**>(p), (size_t)count * sizeof(T)), "cudaMalloc (batch)");
}

int upload_box_cfg(Batch* b, cudaStream_t s) {
    std::vector<int32_t> g(b->nbox);
    std::vector<float> sp(b->nbox);
    b->max_g = 1;
    for (int k = 0; k < b->nbox; ++k) {
        const ClassCfg& cc = b->cfg[b->cls_h[k]];
        g[k] = cc.g | (cc.smax << 8) | (cc.leaf << 16);
        sp[k] = cc.split;
        b->max_g = std::max(b->max_g, cc.g);
    }
    int rc = check_cuda(cudaMemcpyAsync(b->box_g, g.data(), b->nbox * sizeof(int32_t), cudaMemcpyHostToDevice, s),
                        "box configuration");
    if (!rc) rc = check_cuda(cudaMemcpyAsync(b->box_split, sp.data(), b->nbox * sizeof(float),
                                             cudaMemcpyHostToDevice, s), "box configuration");
    if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "box configuration");
    return rc;
}

void drop_graph(Batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->cap_flags = -1;
}

// Work list U (active ranks, or all ranks), its chunks, split groups and the group
// count on the device.
int make_batch_groups(Batch* b, bool all, int only_cls, const uint8_t* active, cudaStream_t s) {
    Ctx* c = b->c;
    const int64_t n = b->n;
    int rc = SPHGRP_OK;
    const int32_t* U = b->U_all;
    int32_t* nchunk = b->dsc + (all ? kNChunkAll : kNChunk);
    int32_t* ngroups = b->dsc + (all ? kNGroupsAll : kNGroups);
    int4* groups = all ? b->groups_all : b->groups;
    if (!all) {
        k_batch_flags<<<kGrid, 256, 0, s>>>(n, c->perm, active, b->box_of_rank, b->box_cls, only_cls, c->flag);
        note_launch();
        if ((rc = exclusive_scan_i32(c, c->flag, c->scan, n, b->dsc + kNu, s))) return rc;
        k_batch_compact<<<kGrid, 256, 0, s>>>(n, c->flag, c->scan, c->act);
        note_launch();
        U = c->act;
    }
    k_box_chunks<<<1, 32, 0, s>>>(b->nbox, b->box_off, c->scan, b->dsc + kNu, all ? 1 : 0, n, b->box_g, b->box_act,
                                  b->box_chunk, nchunk);
    note_launch();
    k_chunk_desc<<<kGrid, 256, 0, s>>>(b->nbox, b->box_act, b->box_chunk, b->box_g, nchunk, b->chunks);
    note_launch();
    k_split_chunks<<<kGrid, 128, 0, s>>>(U, b->chunks, nchunk, c->pfix, c->h64, b->box_split, b->gtmp, b->ccnt);
    note_launch();
    if ((rc = exclusive_scan_i32_dev(c, b->ccnt, b->coff, nchunk, nullptr, n, ngroups, s))) return rc;
    k_gather_chunk_groups<<<kGrid, 256, 0, s>>>(b->chunks, nchunk, b->ccnt, b->coff, b->gtmp, b->box_g, groups);
    note_launch();
    return check_cuda(cudaGetLastError(), "batch groups");
}

SearchArgs batch_args(Batch* b, bool all) {
    SearchArgs a = base_args(b->c);
    a.U = all ? b->U_all : b->c->act;
    a.nu = (int)b->n;   // bound only; groups4 carries the ranges
    a.g = b->max_g;
    a.groups4 = all ? b->groups_all : b->groups;
    a.start_tab = b->start_tabs;   // one start table per box, indexed by the box's root
    a.ngroups_dev = b->dsc + (all ? kNGroupsAll : kNGroups);
    return a;
}

// The whole step as stream work (no host synchronisation): graph-capturable.
int issue_step(Batch* b, const sphgrp_batch_io* io, int flags, cudaStream_t s) {
    Ctx* c = b->c;
    const int64_t n = b->n;
    const bool bwd = (flags & SPHGRP_BATCH_BACKWARD) != 0;
    int rc = SPHGRP_OK;
    cudaMemsetAsync(c->err, 0, sizeof(unsigned), s);
    cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), s);
    cudaMemsetAsync(b->dsc, 0, kNScalars * sizeof(int32_t), s);
    // order, particles, forest
    if ((rc = sort_keys_boxed(c, n, io->pos, b->box_off, b->nbox, b->tmp64a, b->tmp64b, b->tmp32a, b->tmp32b,
                              b->box_of_rank, s)))
        return rc;
    if ((rc = gather_particles(c, io->pos, io->m, s))) return rc;
    if ((rc = launch_gather_h(c, io->h, s))) return rc;
    if ((rc = build_forest(c, b->nbox, b->box_off, b->lvl, b->blo, b->bhi, b->dsc + kTot, b->box_of_rank,
                           b->start_tabs, s, b->box_g)))
        return rc;
    // density with the smoothing-length iteration over the active groups
    if ((rc = make_batch_groups(b, false, -1, io->active, s))) return rc;
    {
        SearchArgs a = batch_args(b, false);
        IterArgs it;
        std::memset(&it, 0, sizeof(it));
        it.nngb = c->p.nngb;
        it.tol = c->p.nngb_tol;
        it.max_iter = c->p.max_iter;
        it.h64 = c->h64;
        it.pfix = c->pfix;
        it.h_out = io->h;
        it.rho = io->rho;
        it.drhodh = io->drhodh;
        it.fgrad = io->fgrad;
        it.nngb_out = io->nngb;
        it.nfail = b->dsc + kNFail;
        if ((rc = launch_density_iter(a, it, b->max_g, c->sm_count, s))) return rc;
    }
    // hydro inputs of every particle, node hmax at the new h
    if ((rc = launch_hydro_prep(c, io->h, io->rho, io->fgrad, io->vel, io->u, s))) return rc;
    if ((rc = refresh_hmax_forest(c, b->lvl, s))) return rc;
    SearchArgs ah = batch_args(b, false);
    ah.o_acc = io->acc;
    ah.o_dudt = io->dudt;
    if (!bwd) return launch_search_dev(ah, kKindHydro, b->max_g, c->sm_count, s);
    // backward: density sums of every particle at its h, adjoint inputs
    if ((rc = make_batch_groups(b, true, -1, nullptr, s))) return rc;
    SearchArgs ad = batch_args(b, true);
    ad.o_s0 = c->acc_rho;
    ad.o_s1 = c->acc_drho;
    ad.o_s2 = c->acc_s2;
    ad.o_n = c->acc_n;
    if ((rc = launch_search_dev(ad, kKindDensity, b->max_g, c->sm_count, s))) return rc;
    if ((rc = launch_bwd_prep(c, io->vel, io->u, io->g_acc, b->hyd0b, b->hyd1b, s))) return rc;
    // hydro items and hydro-adjoint items in one work queue
    SearchArgs ab = batch_args(b, true);
    ab.hyd0 = b->hyd0b;
    ab.hyd1 = b->hyd1b;
    ab.o_adj0 = c->adj0;
    ab.o_adj1 = c->adj1;
    ab.o_adj2 = c->adj2;
    if ((rc = launch_search_pair(ah, kKindHydro, ab, kKindHydroAdj, b->max_g, c->sm_count, s))) return rc;
    if ((rc = launch_bwd_chain(c, io->u, io->g_rho, s))) return rc;
    SearchArgs aa = batch_args(b, true);
    aa.o_adj3 = c->adj3;
    if ((rc = launch_search_dev(aa, kKindDensityAdj, b->max_g, c->sm_count, s))) return rc;
    return launch_bwd_combine(c, io->g_pos, io->g_vel, io->g_m, s);
}

// status copies at the end of the step (part of the captured graph)
void issue_status(Batch* b, cudaStream_t s) {
    cudaMemcpyAsync(b->host, b->c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(b->host + 2, b->dsc, kNScalars * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(b->host_ctr, b->c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
}

int read_status(Batch* b, int flags) {
    const unsigned err = (unsigned)b->host[0];
    const int32_t* sc = b->host + 2;
    Ctx* c = b->c;
    std::memset(&c->last, 0, sizeof(c->last));
    const DevCounters& dc = *b->host_ctr;
    c->last.nodes_tested = (int64_t)dc.nodes;
    c->last.candidates = (int64_t)dc.cands;
    c->last.pair_tests = (int64_t)dc.tests;
    c->last.pairs = (int64_t)dc.pairs;
    c->last.fp64_retests = (int64_t)dc.retests;
    c->last.max_stack = (int64_t)dc.max_stack;
    const bool bwd = (flags & SPHGRP_BATCH_BACKWARD) != 0;
    c->last.walks = 2 * (int64_t)sc[kNGroups] + (bwd ? 3 * (int64_t)sc[kNGroupsAll] : 0);
    c->last.members = 2 * (int64_t)sc[kNu] + (bwd ? 3 * b->n : 0);
    c->last.iterations = b->replayed ? 1 : 0;
    c->last.search_launches = b->step_kernels;
    if (err & kErrRange) return set_error(SPHGRP_EINVAL, "a position is outside [0,1) or not finite");
    if (err & kErrH) return set_error(SPHGRP_EINVAL, "a smoothing length is outside (0, 0.5)");
    if (err & kErrStack) return set_error(SPHGRP_EOVERFLOW, "walk stack overflow");
    if (err & kErrNodes) return set_error(SPHGRP_EOVERFLOW, "forest capacity exceeded");
    if (err & kErrTimeout) return set_error(SPHGRP_ETIMEOUT, "a bounded device wait (tile copy) gave up");
    if (sc[kNFail] > 0) return set_error(SPHGRP_ENOCONV, std::to_string(sc[kNFail]) + " particles did not converge");
    return SPHGRP_OK;
}

int check_io(const sphgrp_batch_io* io, int flags) {
    if (!io) return set_error(SPHGRP_EINVAL, "null io");
    if (!io->pos || !io->m || !io->vel || !io->u || !io->h || !io->rho || !io->drhodh || !io->fgrad || !io->nngb ||
        !io->acc || !io->dudt)
        return set_error(SPHGRP_EINVAL, "null forward array in io");
    if (flags & SPHGRP_BATCH_BACKWARD) {
        if (!io->g_acc) return set_error(SPHGRP_EINVAL, "backward needs g_acc");
        if (!io->g_pos && !io->g_vel && !io->g_m) return set_error(SPHGRP_EINVAL, "backward with no output");
    }
    if (flags & ~(SPHGRP_BATCH_BACKWARD | SPHGRP_BATCH_GRAPH)) return set_error(SPHGRP_EINVAL, "unknown flags");
    return SPHGRP_OK;
}

long long graph_kernel_nodes(cudaGraph_t g) {
    size_t num = 0;
    if (cudaGraphGetNodes(g, nullptr, &num) != cudaSuccess || num == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(num);
    if (cudaGraphGetNodes(g, nodes.data(), &num) != cudaSuccess) return 0;
    long long k = 0;
    for (size_t i = 0; i < num; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

}  // namespace
}  // namespace sphgrp

using namespace sphgrp;

struct sphgrp_batch {
    Batch b;
};

extern "C" {

int sphgrp_batch_create(sphgrp_batch** out, const sphgrp_params* params, int nbox, const int64_t* box_off,
                        const int32_t* box_class) {
    if (!out) return set_error(SPHGRP_EINVAL, "null output pointer");
    *out = nullptr;
    if (nbox < 1 || !box_off) return set_error(SPHGRP_EINVAL, "need nbox >= 1 and box offsets");
    if (box_off[0] != 0) return set_error(SPHGRP_EINVAL, "box_off[0] must be 0");
    for (int k = 0; k < nbox; ++k)
        if (box_off[k + 1] <= box_off[k]) return set_error(SPHGRP_EINVAL, "every box needs at least one particle");
    const int64_t n = box_off[nbox];
    if (n > ((int64_t)1 << 30)) return set_error(SPHGRP_EINVAL, "more than 2^30 particles");
    if (box_class)
        for (int k = 0; k < nbox; ++k)
            if (box_class[k] < 0 || box_class[k] >= SPHGRP_BATCH_CLASSES)
                return set_error(SPHGRP_EINVAL, "box class outside [0, SPHGRP_BATCH_CLASSES)");
    sphgrp_ctx* ch = nullptr;
    int rc = sphgrp_ctx_create(&ch, params, n);
    if (rc) return rc;
    sphgrp_batch* w = new sphgrp_batch();
    Batch* b = &w->b;
    b->c = reinterpret_cast<Ctx*>(ch);
    b->c->n = n;
    b->nbox = nbox;
    b->n = n;
    b->box_off_h.assign(box_off, box_off + nbox + 1);
    b->cls_h.assign(nbox, 0);
    if (box_class) std::copy(box_class, box_class + nbox, b->cls_h.begin());
    for (auto& cc : b->cfg) {
        cc.g = 16;
        cc.smax = 4;
        cc.split = (float)b->c->p.group_split;
    }
    const int64_t node_cap = n / 2 + 64 * (int64_t)nbox + 1024;
    rc = 0;
    rc = rc ? rc : dalloc(&b->box_off, nbox + 1);
    rc = rc ? rc : dalloc(&b->box_g, nbox);
    rc = rc ? rc : dalloc(&b->box_split, nbox);
    rc = rc ? rc : dalloc(&b->box_cls, nbox);
    rc = rc ? rc : dalloc(&b->box_of_rank, n);
    rc = rc ? rc : dalloc(&b->tmp64a, n);
    rc = rc ? rc : dalloc(&b->tmp64b, n);
    rc = rc ? rc : dalloc(&b->tmp32a, n);
    rc = rc ? rc : dalloc(&b->tmp32b, n);
    rc = rc ? rc : dalloc(&b->lvl, kLevels);
    rc = rc ? rc : dalloc(&b->blo, node_cap);
    rc = rc ? rc : dalloc(&b->bhi, node_cap);
    rc = rc ? rc : dalloc(&b->U_all, n);
    rc = rc ? rc : dalloc(&b->dsc, kNScalars);
    rc = rc ? rc : dalloc(&b->box_act, nbox + 1);
    rc = rc ? rc : dalloc(&b->box_chunk, nbox + 1);
    rc = rc ? rc : dalloc(&b->chunks, n);
    rc = rc ? rc : dalloc(&b->ccnt, n + 1);
    rc = rc ? rc : dalloc(&b->coff, n + 1);
    rc = rc ? rc : dalloc(&b->gtmp, n);
    rc = rc ? rc : dalloc(&b->groups, n);
    rc = rc ? rc : dalloc(&b->groups_all, n);
    rc = rc ? rc : dalloc(&b->hyd0b, n);
    rc = rc ? rc : dalloc(&b->hyd1b, n);
    // walk start tables: 1.2 MB per box, so only for batches of up to kMaxTableBoxes
    // boxes (larger batches walk from their boxes' roots)
    if (nbox <= kMaxTableBoxes) rc = rc ? rc : dalloc(&b->start_tabs, (int64_t)nbox * kStartTableSize);
    rc = rc ? rc : alloc_forest(b->c, node_cap);
    rc = rc ? rc : backward_buffers(b->c);
    if (!rc && cudaMallocHost(&b->host, (2 + kNScalars) * sizeof(int32_t)) != cudaSuccess) rc = SPHGRP_ENOMEM;
    if (!rc && cudaMallocHost(&b->host_ctr, sizeof(DevCounters)) != cudaSuccess) rc = SPHGRP_ENOMEM;
    if (!rc) rc = check_cuda(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "capture stream");
    if (!rc) {
        cudaStream_t s = b->cap_stream;
        rc = check_cuda(cudaMemcpyAsync(b->box_off, box_off, (nbox + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s),
                        "box offsets");
        if (!rc)
            rc = check_cuda(cudaMemcpyAsync(b->box_cls, b->cls_h.data(), nbox * sizeof(int32_t),
                                            cudaMemcpyHostToDevice, s), "box classes");
        if (!rc) {
            k_iota<<<kGrid, 256, 0, s>>>(n, b->U_all);
            note_launch();
        }
        if (!rc) rc = upload_box_cfg(b, s);
    }
    if (rc) {
        sphgrp_batch_destroy(w);
        return rc == SPHGRP_ENOMEM ? set_error(SPHGRP_ENOMEM, "batch allocation failed") : rc;
    }
    *out = w;
    return SPHGRP_OK;
}

int sphgrp_batch_destroy(sphgrp_batch* w) {
    if (!w) return SPHGRP_OK;
    Batch* b = &w->b;
    drop_graph(b);
    void* ptrs[] = {b->box_off, b->box_g, b->box_split, b->box_cls, b->box_of_rank, b->tmp64a, b->tmp64b,
                    b->tmp32a, b->tmp32b, b->lvl, b->blo, b->bhi, b->U_all, b->dsc, b->box_act, b->box_chunk,
                    b->chunks, b->ccnt, b->coff, b->gtmp, b->groups, b->groups_all, b->hyd0b, b->hyd1b,
                    b->start_tabs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (b->host) cudaFreeHost(b->host);
    if (b->host_ctr) cudaFreeHost(b->host_ctr);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->c) sphgrp_ctx_destroy(reinterpret_cast<sphgrp_ctx*>(b->c));
    delete w;
    return SPHGRP_OK;
}

int sphgrp_batch_run(sphgrp_batch* w, const sphgrp_batch_io* io, int flags, cudaStream_t s) {
    if (!w) return set_error(SPHGRP_EINVAL, "null batch");
    Batch* b = &w->b;
    int rc = check_io(io, flags);
    if (rc) return rc;
    b->replayed = false;
    if (flags & SPHGRP_BATCH_GRAPH) {
        const bool same = b->exec && b->cap_flags == flags && std::memcmp(&b->cap_io, io, sizeof(*io)) == 0;
        if (!same) {
            drop_graph(b);
            cudaGraph_t graph = nullptr;
            rc = check_cuda(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
            if (rc) return rc;
            int irc = issue_step(b, io, flags, b->cap_stream);
            if (!irc) issue_status(b, b->cap_stream);
            rc = check_cuda(cudaStreamEndCapture(b->cap_stream, &graph), "end capture");
            if (irc) {
                if (graph) cudaGraphDestroy(graph);
                return irc;
            }
            if (rc) return rc;
            rc = check_cuda(cudaGraphInstantiate(&b->exec, graph, 0), "graph instantiate");
            b->exec_kernels = graph_kernel_nodes(graph);
            cudaGraphDestroy(graph);
            if (rc) return rc;
            b->cap_io = *io;
            b->cap_flags = flags;
        } else {
            b->replayed = true;
        }
        rc = check_cuda(cudaGraphLaunch(b->exec, s), "graph launch");
        if (rc) return rc;
        note_launches(b->exec_kernels);
        b->step_kernels = b->exec_kernels;
    } else {
        int64_t l0 = 0, l1 = 0;
        sphgrp_kernel_launches(&l0);
        if ((rc = issue_step(b, io, flags, s))) return rc;
        issue_status(b, s);
        sphgrp_kernel_launches(&l1);
        b->step_kernels = l1 - l0;
    }
    if ((rc = check_cuda(cudaStreamSynchronize(s), "batch step"))) return rc;
    return read_status(b, flags);
}

int sphgrp_batch_get_config(sphgrp_batch* w, int cls, int* group_size, int* max_slices, double* group_split,
                            int* leaf_size, double* pass_ms, int64_t* pass_members) {
    if (!w || cls < 0 || cls >= SPHGRP_BATCH_CLASSES) return set_error(SPHGRP_EINVAL, "bad batch or class");
    const ClassCfg& cc = w->b.cfg[cls];
    if (pass_ms) *pass_ms = cc.tuned_ms;
    if (pass_members) *pass_members = cc.tuned_members;
    if (group_size) *group_size = cc.g;
    if (max_slices) *max_slices = cc.smax;
    if (group_split) *group_split = cc.split;
    if (leaf_size) *leaf_size = cc.leaf;
    return SPHGRP_OK;
}

int sphgrp_batch_set_config(sphgrp_batch* w, int cls, int group_size, int max_slices, double group_split,
                            int leaf_size) {
    if (!w || cls < 0 || cls >= SPHGRP_BATCH_CLASSES) return set_error(SPHGRP_EINVAL, "bad batch or class");
    if (group_size < 1 || group_size > 128) return set_error(SPHGRP_EINVAL, "group_size outside [1, 128]");
    if (max_slices != 1 && max_slices != 2 && max_slices != 4) return set_error(SPHGRP_EINVAL, "max_slices not 1, 2, 4");
    if (!(group_split >= 0.0)) return set_error(SPHGRP_EINVAL, "group_split < 0");
    if (leaf_size != 0 && (leaf_size < kMinBatchLeaf || leaf_size > 255))
        return set_error(SPHGRP_EINVAL, "leaf_size not 0 or in [8, 255]");
    Batch* b = &w->b;
    b->cfg[cls] = ClassCfg{group_size, max_slices, (float)group_split, 0.0f, 0, leaf_size};
    drop_graph(b);
    return upload_box_cfg(b, b->cap_stream);
}

int sphgrp_batch_tune(sphgrp_batch* w, const sphgrp_batch_io* io, cudaStream_t s) {
    if (!w) return set_error(SPHGRP_EINVAL, "null batch");
    Batch* b = &w->b;
    Ctx* c = b->c;
    drop_graph(b);
    // a full step at the current configuration: converged h, hydro inputs, node hmax
    int rc = sphgrp_batch_run(w, io, 0, s);
    if (rc && rc != SPHGRP_ENOCONV) return rc;
    struct Cand {
        int g, smax;
        float split;
    };
    std::vector<Cand> cands;
    const float splits[] = {1.5f, 2.0f, 4.0f};
    for (float sp : splits) {
        for (int smax : {1, 2, 4}) cands.push_back({4, smax, sp});
        for (int smax : {1, 2, 4}) cands.push_back({8, smax, sp});
        for (int smax : {1, 2}) cands.push_back({16, smax, sp});
        cands.push_back({32, 1, sp});
        cands.push_back({64, 1, sp});
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float* acc_scratch = reinterpret_cast<float*>(c->adj0);   // n x 4 floats
    float* dudt_scratch = reinterpret_cast<float*>(c->adj3);
    // best of two density + hydro passes over the class's active particles
    auto time_class = [&](int cls, float* out) -> int {
        float t_best = 3.0e38f;
        int r = SPHGRP_OK;
        for (int rep = 0; rep < 2 && !r; ++rep) {
            cudaEventRecord(e0, s);
            if ((r = make_batch_groups(b, false, cls, io->active, s))) break;
            SearchArgs ad = batch_args(b, false);
            ad.o_s0 = c->acc_rho;
            ad.o_s1 = c->acc_drho;
            ad.o_n = c->acc_n;
            if ((r = launch_search_dev(ad, kKindDensity, b->max_g, c->sm_count, s))) break;
            SearchArgs ah = batch_args(b, false);
            ah.o_acc = acc_scratch;
            ah.o_dudt = dudt_scratch;
            if ((r = launch_search_dev(ah, kKindHydro, b->max_g, c->sm_count, s))) break;
            cudaEventRecord(e1, s);
            if ((r = check_cuda(cudaEventSynchronize(e1), "tuning step"))) break;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            t_best = std::min(t_best, ms);
        }
        *out = t_best;
        return r;
    };
    // the forest again (the order is unchanged) with the classes' current leaf sizes,
    // and its node hmax at the converged h; reports whether it fit the node capacity
    auto rebuild = [&](bool* fits) -> int {
        int r = build_forest(c, b->nbox, b->box_off, b->lvl, b->blo, b->bhi, b->dsc + kTot, b->box_of_rank,
                             b->start_tabs, s, b->box_g);
        if (!r) r = refresh_hmax_forest(c, b->lvl, s);
        unsigned err = 0;
        if (!r) r = check_cuda(cudaMemcpyAsync(b->host, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s),
                               "forest status");
        if (!r) r = check_cuda(cudaStreamSynchronize(s), "forest status");
        if (!r) std::memcpy(&err, b->host, sizeof(unsigned));
        *fits = (err & kErrNodes) == 0u;
        if (!r && !*fits) cudaMemsetAsync(c->err, 0, sizeof(unsigned), s);
        return r;
    };
    for (int cls = 0; cls < SPHGRP_BATCH_CLASSES && !rc; ++cls) {
        if (std::find(b->cls_h.begin(), b->cls_h.end(), cls) == b->cls_h.end()) continue;
        const ClassCfg keep = b->cfg[cls];
        float best = 3.0e38f;
        ClassCfg best_cfg = keep;
        for (const Cand& cd : cands) {
            b->cfg[cls] = ClassCfg{cd.g, cd.smax, cd.split, 0.0f, 0, keep.leaf};
            if ((rc = upload_box_cfg(b, s))) break;
            float t = 0.0f;
            if ((rc = time_class(cls, &t))) break;
            if (t < best) {
                best = t;
                best_cfg = b->cfg[cls];
            }
        }
        // then the octree leaf size of the class's boxes, at its best grouping: each
        // candidate rebuilds the forest before its timed passes; one that overflows the
        // node capacity is skipped
        for (int leaf : {0, 8, 12, 24, 32}) {
            if (rc || leaf == keep.leaf) continue;
            ClassCfg cd = best_cfg;
            cd.leaf = leaf;
            b->cfg[cls] = cd;
            bool fits = true;
            if ((rc = upload_box_cfg(b, s)) || (rc = rebuild(&fits))) break;
            if (!fits) continue;
            float t = 0.0f;
            if ((rc = time_class(cls, &t))) break;
            if (t < best) {
                best = t;
                best_cfg = cd;
            }
        }
        if (!rc) {
            // the class's chosen forest for the passes that follow
            bool fits = true;
            b->cfg[cls] = best_cfg;
            if (!(rc = upload_box_cfg(b, s))) rc = rebuild(&fits);
        }
        b->cfg[cls] = rc ? keep : best_cfg;
        if (!rc) {
            int32_t members = 0;
            rc = check_cuda(cudaMemcpyAsync(b->host + 2 + kNu, b->dsc + kNu, sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                            "tuned class size");
            if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "tuned class size");
            members = b->host[2 + kNu];
            b->cfg[cls].tuned_ms = best;
            b->cfg[cls].tuned_members = members;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc2 = upload_box_cfg(b, s);
    return rc ? rc : rc2;
}

int sphgrp_batch_stats(sphgrp_batch* w, sphgrp_stats* out) {
    if (!w || !out) return set_error(SPHGRP_EINVAL, "null argument");
    *out = w->b.c->last;
    return SPHGRP_OK;
}

}  // extern "C"
