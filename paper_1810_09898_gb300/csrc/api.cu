// C ABI of the library (declared in include/sphgrp.h): context, argument checks and
// the orchestration of the kernels of sort.cu, tree.cu and ngb.cu.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>

#include "search_args.cuh"

namespace sphgrp {


static thread_local std::string g_last_error = "no error";
static std::atomic<long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void timer_begin(Ctx* c, cudaStream_t s) {
    if (c->ntimed < Ctx::kMaxTimed) cudaEventRecord(c->tev[2 * c->ntimed], s);
}

void timer_end(Ctx* c, cudaStream_t s, int64_t members) {
    if (c->ntimed < Ctx::kMaxTimed) {
        cudaEventRecord(c->tev[2 * c->ntimed + 1], s);
        cudaMemcpyAsync(c->ctr_log + c->ntimed, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToDevice, s);
        c->log_members[c->ntimed] = members;
        c->ntimed++;
    }
}

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int check_cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SPHGRP_OK;
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SPHGRP_ENOMEM : SPHGRP_ECUDA;
}

}  // namespace sphgrp


using namespace sphgrp;

namespace {

template <typename T>
int dalloc(T** p, int64_t count) {
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (size_t)count * sizeof(T));
    if (e != cudaSuccess) return check_cuda(e, "cudaMalloc");
    return SPHGRP_OK;
}

__global__ void k_mark_active(int64_t n_act, const int32_t* __restrict__ active, int64_t n,
                              const int32_t* __restrict__ rank_of, int32_t* __restrict__ flag,
                              unsigned* err) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act) return;
    int i = active[k];
    if (i < 0 || i >= n) {
        atomicOr(err, 32u);
        return;
    }
    flag[rank_of[i]] = 1;
}

__global__ void k_compact_ranks(int64_t n, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                int32_t* __restrict__ out) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n && flag[r]) out[pos[r]] = (int32_t)r;
}

__global__ void k_compact_list(int nu, const int32_t* __restrict__ keep, const int32_t* __restrict__ pos,
                               const int32_t* __restrict__ in, int32_t* __restrict__ out) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < nu && keep[u]) out[pos[u]] = in[u];
}

__global__ void k_gather_h(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ h,
                           double* __restrict__ h64, uint4* __restrict__ pfix, unsigned* err) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    double v = h[perm[r]];
    if (!(v > 0.0 && v < 0.5)) atomicOr(err, kErrH);
    h64[r] = v;
    pfix[r].w = __float_as_uint((float)v);
}

// Hydro inputs in key order: hyd0 = {v, c}, hyd1 = {A = f P / rho^2, rho, 1/h, fbal}.
// fbal is Balsara's viscosity limiter |div v| / (|div v| + |curl v| + 1e-4 c / h) when the
// caller gives div v and curl v, else 1 (the plain Monaghan viscosity).
// One thread per rank: the caller-order inputs are gathered through the permutation and
// the key-ordered records written coalesced (the scattered-store form, one thread per
// caller index, measured 1.6x slower: its partial-sector writes cost more than these loads).
__global__ void k_hydro_prep(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ h,
                             const float* __restrict__ rho, const float* __restrict__ fgrad,
                             const float* __restrict__ vel, const float* __restrict__ u, float gamma,
                             double* __restrict__ h64, uint4* __restrict__ pfix, float4* __restrict__ hyd0,
                             float4* __restrict__ hyd1, unsigned* err, const float* __restrict__ divv,
                             const float* __restrict__ curlv) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int i = perm[r];
    double hv = h[i];
    if (!(hv > 0.0 && hv < 0.5)) atomicOr(err, kErrH);
    h64[r] = hv;
    float hf = (float)hv;
    pfix[r].w = __float_as_uint(hf);
    float rh = rho[i];
    float P = (gamma - 1.0f) * rh * u[i];
    float cs = sqrtf(gamma * P / rh);
    float A = fgrad[i] * P / (rh * rh);
    hyd0[r] = make_float4(vel[3 * (int64_t)i], vel[3 * (int64_t)i + 1], vel[3 * (int64_t)i + 2], cs);
    float fb = 1.0f;
    if (divv) {
        const float ad = fabsf(divv[i]);
        const float cx = curlv[3 * (int64_t)i], cy = curlv[3 * (int64_t)i + 1], cz = curlv[3 * (int64_t)i + 2];
        fb = ad / (ad + sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz))) + 1.0e-4f * cs / hf);
    }
    hyd1[r] = make_float4(A, rh, 1.0f / hf, fb);
}

// velocities in key order for the density loop with velocity derivatives: hyd0 = {v, 0}
__global__ void k_vel_gather(int64_t n, const int32_t* __restrict__ perm, const float* __restrict__ vel,
                             float4* __restrict__ hyd0) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t i = perm[r];
    hyd0[r] = make_float4(vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], 0.0f);
}

// velocity-derivative inputs in key order: hyd0 = {v, 0}, hyd1 = {0, rho, 1/h, 8/(pi h^4)}
__global__ void k_velocity_prep(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ h,
                                const float* __restrict__ rho, const float* __restrict__ vel,
                                double* __restrict__ h64, uint4* __restrict__ pfix, float4* __restrict__ hyd0,
                                float4* __restrict__ hyd1, unsigned* err) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    int i = perm[r];
    double hv = h[i];
    if (!(hv > 0.0 && hv < 0.5)) atomicOr(err, kErrH);
    h64[r] = hv;
    float hf = (float)hv;
    pfix[r].w = __float_as_uint(hf);
    hyd0[r] = make_float4(vel[3 * (int64_t)i], vel[3 * (int64_t)i + 1], vel[3 * (int64_t)i + 2], 0.0f);
    const double kPi = 3.14159265358979323846;
    float s = (float)(8.0 / (kPi * hv * hv * hv * hv));
    hyd1[r] = make_float4(0.0f, rho[i], 1.0f / hf, s);
}

// Results of the density loop and its smoothing-length iteration from key order to the
// caller's order, over the caller's active list: the final h stays in h64 and the sums at
// that h, the neighbour count and the pass count in one float4 (rank space) when a
// particle finishes, so that the outputs are written here in one coalesced pass
// instead of by scattered stores from the update kernel.  Indices outside [0, n) were
// flagged by k_mark_active and are skipped.
__global__ void k_out_density(int64_t n_act, const int32_t* __restrict__ active, int64_t n,
                              const int32_t* __restrict__ rank_of, const double* __restrict__ h64,
                              const float4* __restrict__ res_k, const float4* __restrict__ vsum,
                              double* __restrict__ h_out, float* __restrict__ rho, float* __restrict__ drhodh,
                              float* __restrict__ fgrad, int32_t* __restrict__ nngb, int32_t* __restrict__ iters,
                              float* __restrict__ divv, float* __restrict__ curlv) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act) return;
    const int64_t i = active[k];
    if (i < 0 || i >= n) return;
    const int r = rank_of[i];
    const double h = h64[r];
    const float4 R = res_k[r];   // {s0, s1, count, pass count}
    const float a0 = R.x, a1 = R.y;
    hsml_write((int)i, h, a0, a1, __float_as_int(R.z), __float_as_int(R.w), h_out, rho, drhodh, fgrad, nngb, iters);
    if (vsum) {
        // div v = -(1/rho) sum m v_ij . grad W, curl v = (1/rho) sum m v_ij x grad W
        const float hf = (float)h;
        const float rinv = hf * hf * hf / (2.54647908947032537f * a0);   // 1 / rho
        const float4 V = vsum[r];
        divv[i] = V.x * rinv;
        curlv[3 * i] = V.y * rinv;
        curlv[3 * i + 1] = V.z * rinv;
        curlv[3 * i + 2] = V.w * rinv;
    }
}

// Results of the hydro loop from key order to the caller's order, over the caller's
// active list (ascending active lists give sequential writes).
__global__ void k_out_hydro(int64_t n_act, const int32_t* __restrict__ active, int64_t n,
                            const int32_t* __restrict__ rank_of, const float4* __restrict__ res4,
                            const int32_t* __restrict__ rcnt, float* __restrict__ acc, float* __restrict__ dudt,
                            int32_t* __restrict__ nngb) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act) return;
    const int64_t i = active[k];
    if (i < 0 || i >= n) return;
    const int r = rank_of[i];
    const float4 v = res4[r];
    acc[3 * i] = v.x;
    acc[3 * i + 1] = v.y;
    acc[3 * i + 2] = v.z;
    dudt[i] = v.w;
    if (nngb) nngb[i] = rcnt[r];
}

// div v and curl v from key order to the caller's order
__global__ void k_out_vel(int64_t n_act, const int32_t* __restrict__ active, int64_t n,
                          const int32_t* __restrict__ rank_of, const float4* __restrict__ res4,
                          float* __restrict__ divv, float* __restrict__ curlv) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act) return;
    const int64_t i = active[k];
    if (i < 0 || i >= n) return;
    const float4 v = res4[rank_of[i]];
    divv[i] = v.x;
    curlv[3 * i] = v.y;
    curlv[3 * i + 1] = v.z;
    curlv[3 * i + 2] = v.w;
}

// (active indices outside [0, n) were flagged by k_mark_active; the call reports EINVAL
// and these kernels skip them: a count of 0, no write)
__global__ void k_counts_by_caller(int64_t n_act, const int32_t* __restrict__ active, int64_t n,
                                   const int64_t* __restrict__ cnt, int64_t* __restrict__ out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act) return;
    const int64_t i = active[k];
    out[k] = (i >= 0 && i < n) ? cnt[i] : 0;
}

__global__ void k_offsets_by_orig(int64_t n_act, const int32_t* __restrict__ active, int64_t n,
                                  const int64_t* __restrict__ off, int64_t* __restrict__ out) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n_act) return;
    const int64_t i = active[k];
    if (i >= 0 && i < n) out[i] = off[k];
}

__global__ void k_group_first(int ng, int nu, int g, const int2* __restrict__ groups, int32_t* __restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ng) out[k] = groups ? groups[k].x : k * g;
    else if (k == ng) out[k] = nu;
}

__global__ void k_members(int nu, const int32_t* __restrict__ U, const int32_t* __restrict__ perm,
                          int32_t* __restrict__ out) {
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < nu) out[u] = perm[U[u]];
}

}  // namespace

namespace sphgrp {

// smoothing lengths (original order) -> h64 and the FP32 copy in pfix.w
int launch_gather_h(Ctx* c, const double* h, cudaStream_t s) {
    k_gather_h<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, h, c->h64, c->pfix, c->err);
    note_launch();
    return check_cuda(cudaGetLastError(), "gather h");
}

// hydro inputs of every particle in key order (hyd0, hyd1, h64, pfix.w)
int launch_hydro_prep(Ctx* c, const double* h, const float* rho, const float* fgrad, const float* vel,
                      const float* u, cudaStream_t s, const float* divv, const float* curlv) {
    k_hydro_prep<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, h, rho, fgrad, vel, u, (float)c->p.gamma,
                                                      c->h64, c->pfix, c->hyd0, c->hyd1, c->err, divv, curlv);
    note_launch();
    return check_cuda(cudaGetLastError(), "hydro prep");
}

int finish(Ctx* c, cudaStream_t s, int rc) {
    if (rc) return rc;
    unsigned err = 0;
    rc = check_cuda(cudaMemcpyAsync(&c->host_small[1], c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s),
                    "error flag copy");
    if (rc) return rc;
    DevCounters dc;
    rc = check_cuda(cudaMemcpyAsync(reinterpret_cast<DevCounters*>(c->host_small + 8), c->ctr,
                                    sizeof(DevCounters), cudaMemcpyDeviceToHost, s),
                    "counter copy");
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(s), "stream");
    if (rc) return rc;
    err = (unsigned)c->host_small[1];
    std::memcpy(&dc, c->host_small + 8, sizeof(dc));
    c->last.nodes_tested = (int64_t)dc.nodes;
    c->last.candidates = (int64_t)dc.cands;
    c->last.pair_tests = (int64_t)dc.tests;
    c->last.pairs = (int64_t)dc.pairs;
    c->last.fp64_retests = (int64_t)dc.retests;
    c->last.max_stack = (int64_t)dc.max_stack;
    double ms = 0.0;
    for (int k = 0; k < c->ntimed; ++k) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, c->tev[2 * k], c->tev[2 * k + 1]) == cudaSuccess) ms += t;
        c->log_ms[k] = t;
    }
    if (c->ntimed > 0)
        cudaMemcpy(c->ctr_log_host, c->ctr_log, c->ntimed * sizeof(DevCounters), cudaMemcpyDeviceToHost);
    c->last.search_ms = ms;
    c->last.search_launches = c->ntimed;
    if (err & kErrRange) return set_error(SPHGRP_EINVAL, "a position is outside [0,1) or not finite");
    if (err & kErrH) return set_error(SPHGRP_EINVAL, "a smoothing length is outside (0, 0.5)");
    if (err & 32u) return set_error(SPHGRP_EINVAL, "an active index is outside [0, n)");
    if (err & kErrStack) return set_error(SPHGRP_EOVERFLOW, "walk stack overflow");
    if (err & kErrNodes) return set_error(SPHGRP_EOVERFLOW, "octree capacity exceeded");
    if (err & kErrCap) return set_error(SPHGRP_EOVERFLOW, "export capacity exceeded");
    if (err & kErrTimeout) return set_error(SPHGRP_ETIMEOUT, "a bounded device wait (tile copy) gave up");
    return SPHGRP_OK;
}

void reset_flags(Ctx* c, cudaStream_t s) {
    cudaMemsetAsync(c->err, 0, sizeof(unsigned), s);
    cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), s);
    std::memset(&c->last, 0, sizeof(c->last));
    c->ntimed = 0;
}

// active original indices -> key-ordered ranks in c->act; returns the count
int prepare_active(Ctx* c, int64_t n_act, const int32_t* active, cudaStream_t s, int* nu) {
    const int64_t n = c->n;
    cudaMemsetAsync(c->flag, 0, n * sizeof(int32_t), s);
    k_mark_active<<<blocks_for(n_act, 256), 256, 0, s>>>(n_act, active, n, c->rank_of, c->flag, c->err);
    note_launch();
    int32_t* total = reinterpret_cast<int32_t*>(c->work) + 4;
    int rc = exclusive_scan_i32(c, c->flag, c->scan, n, total, s);
    if (rc) return rc;
    k_compact_ranks<<<blocks_for(n, 256), 256, 0, s>>>(n, c->flag, c->scan, c->act);
    note_launch();
    cudaMemcpyAsync(c->host_small, total, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    rc = check_cuda(cudaStreamSynchronize(s), "active list");
    if (rc) return rc;
    *nu = c->host_small[0];
    return SPHGRP_OK;
}

// The work-list entries flagged in c->flag move to *U2 (order kept), which becomes the
// work list; reads the new count back (stream sync).
int compact_unconverged(Ctx* c, int32_t** U, int32_t** U2, int* nu, cudaStream_t s) {
    int32_t* total = reinterpret_cast<int32_t*>(c->work) + 4;
    int rc = exclusive_scan_i32(c, c->flag, c->scan, *nu, total, s);
    if (rc) return rc;
    k_compact_list<<<blocks_for(*nu, 256), 256, 0, s>>>(*nu, c->flag, c->scan, *U, *U2);
    note_launch();
    cudaMemcpyAsync(c->host_small, total, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "iteration count"))) return rc;
    *nu = c->host_small[0];
    std::swap(*U, *U2);
    return SPHGRP_OK;
}

// Candidate-list buffers of the recycled iteration for n_max particles (kListCap ranks
// per particle); ENOMEM if the device cannot hold them (the caller then walks every pass).
int list_buffers(Ctx* c) {
    if (c->lst) return SPHGRP_OK;
    if (c->lst_failed) return SPHGRP_ENOMEM;
    const int64_t n = c->n_max;
    int rc = 0;
    rc |= dalloc(&c->lst, n * kListCap);
    rc |= dalloc(&c->lrec, n);
    rc |= dalloc(&c->lhw, n);
    rc |= dalloc(&c->lslot, n);
    rc |= dalloc(&c->npass, n);
    if (rc) {
        void* ptrs[] = {c->lst, c->lrec, c->lhw, c->lslot, c->npass};
        for (void* p : ptrs)
            if (p) cudaFree(p);
        c->lst = nullptr;
        c->lrec = nullptr;
        c->lhw = nullptr;
        c->lslot = nullptr;
        c->npass = nullptr;
        c->lst_failed = true;
        cudaGetLastError();   // the failed allocation is not a sticky error
        return set_error(SPHGRP_ENOMEM, "no device memory for the candidate lists");
    }
    return SPHGRP_OK;
}

// Groups of the grouped form over the work list U (see k_split_groups); fills
// a->groups and a->ngroups.  Reads the group count back (stream sync).
// Tree grouping (Sec. 2): the actives under one node of depth L share the key's first
// 3 L bits, and every node is a contiguous range of the key order, so a group is a run
// of consecutive actives with one prefix, cut into pieces of at most g.
__global__ void k_prefix_runs(int nu, const int32_t* __restrict__ U, const uint64_t* __restrict__ keys, int shift,
                              int32_t* __restrict__ flag) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nu) return;
    flag[u] = (u == 0 || (keys[U[u]] >> shift) != (keys[U[u - 1]] >> shift)) ? 1 : 0;
}

// run k starts at the entry u whose flag begins it: run_start[pos[u]] = u
__global__ void k_run_starts(int nu, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                             int32_t* __restrict__ run_start) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < nu && flag[u]) run_start[pos[u]] = u;
}

__global__ void k_run_pieces(int nruns, int nu, int g, const int32_t* __restrict__ run_start,
                             int32_t* __restrict__ pieces) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nruns) return;
    const int len = (k + 1 < nruns ? run_start[k + 1] : nu) - run_start[k];
    pieces[k] = (len + g - 1) / g;
}

__global__ void k_run_groups(int nruns, int nu, int g, const int32_t* __restrict__ run_start,
                             const int32_t* __restrict__ piece_off, int2* __restrict__ groups) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nruns) return;
    const int s0 = run_start[k], e0 = k + 1 < nruns ? run_start[k + 1] : nu;
    int o = piece_off[k];
    for (int s1 = s0; s1 < e0; s1 += g) groups[o++] = make_int2(s1, min(g, e0 - s1));
}

int make_tree_groups(Ctx* c, SearchArgs* a, const int32_t* U, int nu, int g, cudaStream_t s) {
    a->groups = nullptr;
    a->ngroups = 0;
    if (nu <= 0) return SPHGRP_OK;
    const int shift = 3 * (kKeyLevels - c->p.group_level);
    int32_t* nruns_dev = reinterpret_cast<int32_t*>(c->work) + 20;
    int32_t* ngroups_dev = reinterpret_cast<int32_t*>(c->work) + 21;
    k_prefix_runs<<<blocks_for(nu, 256), 256, 0, s>>>(nu, U, c->keys, shift, c->grp_cnt);
    note_launch();
    int rc = exclusive_scan_i32(c, c->grp_cnt, c->grp_off, nu, nruns_dev, s);
    if (rc) return rc;
    // run starts go to scan (free here), piece counts to grp_cnt, their offsets to grp_off
    k_run_starts<<<blocks_for(nu, 256), 256, 0, s>>>(nu, c->grp_cnt, c->grp_off, c->scan);
    note_launch();
    cudaMemcpyAsync(c->host_small + 41, nruns_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "tree groups"))) return rc;
    const int nruns = c->host_small[41];
    k_run_pieces<<<blocks_for(nruns, 256), 256, 0, s>>>(nruns, nu, g, c->scan, c->grp_cnt);
    note_launch();
    if ((rc = exclusive_scan_i32(c, c->grp_cnt, c->grp_off, nruns, ngroups_dev, s))) return rc;
    k_run_groups<<<blocks_for(nruns, 256), 256, 0, s>>>(nruns, nu, g, c->scan, c->grp_off, c->groups);
    note_launch();
    cudaMemcpyAsync(c->host_small + 40, ngroups_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "tree group count"))) return rc;
    a->groups = c->groups;
    a->ngroups = c->host_small[40];
    return SPHGRP_OK;
}

int make_groups(Ctx* c, SearchArgs* a, const int32_t* U, int nu, int g, cudaStream_t s) {
    a->groups = nullptr;
    a->ngroups = (nu + g - 1) / g;
    const bool radius = c->p.group_mode == SPHGRP_GROUP_RADIUS;
    if (c->p.group_mode == SPHGRP_GROUP_TREE) return make_tree_groups(c, a, U, nu, g, s);
    if (nu <= 0 || g <= 1 || (!radius && !(c->p.group_split > 0.0))) return SPHGRP_OK;
    int nch = radius ? (nu + kRadiusRun - 1) / kRadiusRun : (nu + g - 1) / g;
    int rc = radius ? launch_radius_groups(U, nu, g, c->p.group_f, c->pfix, c->poff, c->h64, c->groups_tmp,
                                           c->grp_cnt, s)
                    : launch_split_groups(U, nu, g, (float)c->p.group_split, c->pfix, c->h64, c->groups_tmp,
                                          c->grp_cnt, s);
    if (rc) return rc;
    int32_t* total = reinterpret_cast<int32_t*>(c->work) + 16;
    if ((rc = exclusive_scan_i32(c, c->grp_cnt, c->grp_off, nch, total, s))) return rc;
    if ((rc = launch_gather_groups(nch, radius ? kRadiusRun : g, c->groups_tmp, c->grp_cnt, c->grp_off, c->groups,
                                   s)))
        return rc;
    cudaMemcpyAsync(c->host_small + 40, total, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "group count"))) return rc;
    a->groups = c->groups;
    a->ngroups = c->host_small[40];
    return SPHGRP_OK;
}

SearchArgs base_args(Ctx* c) {
    SearchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.ncen = c->tree.ncen;
    a.next = c->tree.next;
    a.nlink = c->tree.nlink;
    a.pfix = c->pfix;
    a.poff = c->poff;
    a.xd = c->xd;
    a.yd = c->yd;
    a.zd = c->zd;
    a.h64 = c->h64;
    a.hyd0 = c->hyd0;
    a.hyd1 = c->hyd1;
    a.wadj = c->wadj;
    a.dadj = c->dadj;
    a.perm = c->perm;
    a.alpha = (float)c->p.alpha;
    a.beta = (float)c->p.beta;
    a.eps = (float)c->p.eps;
    a.ctr = c->ctr;
    a.err = c->err;
    a.work = c->work;
    a.stack_spill = c->stack_spill;
    a.start_tab = c->start_valid ? c->start_tab : nullptr;
    a.stack_cap = c->p.stack_shared;
    a.centre_box = c->p.group_centre == SPHGRP_CENTRE_BOX;
    return a;
}

int check_common(Ctx* c, int64_t n_act, const int32_t* active, int mode, int group_size) {
    if (!c) return set_error(SPHGRP_EINVAL, "null context");
    if (!c->built) return set_error(SPHGRP_ESTATE, "no octree: call sphgrp_tree_build first");
    if (n_act < 0 || n_act > c->n) return set_error(SPHGRP_EINVAL, "n_act outside [0, n]");
    if (n_act > 0 && !active) return set_error(SPHGRP_EINVAL, "null active list");
    if (mode != SPHGRP_INDIVIDUAL && mode != SPHGRP_GROUPED) return set_error(SPHGRP_EINVAL, "bad mode");
    if (mode == SPHGRP_GROUPED && (group_size < 1 || group_size > 128))
        return set_error(SPHGRP_EINVAL, "group_size must be in [1, 128]");
    return SPHGRP_OK;
}

}  // namespace sphgrp

extern "C" {

void sphgrp_default_params(sphgrp_params* p) {
    if (!p) return;
    p->nngb = 64.0;
    p->nngb_tol = 2.0;
    p->max_iter = 100;
    p->leaf_size = 16;
    p->gamma = 5.0 / 3.0;
    p->alpha = 1.0;
    p->beta = 2.0;
    p->eps = 0.01;
    p->group_centre = SPHGRP_CENTRE_BOX;
    p->group_split = 2.0;
    p->iteration = SPHGRP_ITER_PASSES;
    p->group_mode = SPHGRP_GROUP_COUNT;
    p->group_f = 0.5;
    p->group_level = 7;
    p->stack_shared = 256;
    p->iter_widen = 1.1;
}

const char* sphgrp_last_error(void) { return g_last_error.c_str(); }

int sphgrp_kernel_launches(int64_t* count) {
    if (!count) return set_error(SPHGRP_EINVAL, "null count");
    *count = (int64_t)g_launches.load();
    return SPHGRP_OK;
}

int sphgrp_ctx_create(sphgrp_ctx** out, const sphgrp_params* p, int64_t n_max) {
    if (!out) return set_error(SPHGRP_EINVAL, "null output pointer");
    *out = nullptr;
    if (n_max < 1 || n_max > (int64_t)1 << 30) return set_error(SPHGRP_EINVAL, "n_max outside [1, 2^30]");
    Ctx* c = new Ctx();
    if (p) c->p = *p;
    else sphgrp_default_params(&c->p);
    if (c->p.leaf_size < 1 || c->p.leaf_size > 1024 || !(c->p.nngb > 0) || !(c->p.nngb_tol >= 0) ||
        c->p.max_iter < 1 || (c->p.group_centre != SPHGRP_CENTRE_FIRST && c->p.group_centre != SPHGRP_CENTRE_BOX) ||
        (c->p.iteration != SPHGRP_ITER_PASSES && c->p.iteration != SPHGRP_ITER_IN_GROUP &&
         c->p.iteration != SPHGRP_ITER_RECYCLE) ||
        !(c->p.iter_widen >= 1.0 && c->p.iter_widen <= 2.0) ||
        (c->p.group_mode != SPHGRP_GROUP_COUNT && c->p.group_mode != SPHGRP_GROUP_RADIUS &&
         c->p.group_mode != SPHGRP_GROUP_TREE) ||
        (c->p.group_mode == SPHGRP_GROUP_TREE && (c->p.group_level < 1 || c->p.group_level > kKeyLevels)) ||
        (c->p.group_mode == SPHGRP_GROUP_RADIUS && !(c->p.group_f > 0.0 && c->p.group_f < 1e3)) ||
        c->p.stack_shared < 32 || c->p.stack_shared > kStackSharedMax) {
        delete c;
        return set_error(SPHGRP_EINVAL, "bad parameters");
    }
    c->n_max = n_max;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n = n_max;
    int rc = 0;
    rc |= dalloc(&c->keys, n);
    rc |= dalloc(&c->keys_alt, n);
    rc |= dalloc(&c->perm, n);
    rc |= dalloc(&c->perm_alt, n);
    rc |= dalloc(&c->rank_of, n);
    c->hist_cap = 256 * ((n + 2047) / 2048) + 256;
    rc |= dalloc(&c->hist, c->hist_cap);
    rc |= dalloc(&c->xd, n);
    rc |= dalloc(&c->yd, n);
    rc |= dalloc(&c->zd, n);
    rc |= dalloc(&c->pfix, n);
    rc |= dalloc(&c->poff, n);
    rc |= dalloc(&c->h64, n);
    rc |= dalloc(&c->hyd0, n);
    rc |= dalloc(&c->hyd1, n);
    rc |= dalloc(&c->act, n);
    rc |= dalloc(&c->act2, n);
    rc |= dalloc(&c->flag, n);
    rc |= dalloc(&c->scan, n);
    c->scan_aux_cap = 2 * (n / 1024 + 4096);
    rc |= dalloc(&c->scan_aux, c->scan_aux_cap);
    rc |= dalloc(&c->lo, n);
    rc |= dalloc(&c->hi, n);
    rc |= dalloc(&c->res4, n);
    rc |= dalloc(&c->acc_rho, n);
    rc |= dalloc(&c->acc_drho, n);
    rc |= dalloc(&c->acc_n, n);
    rc |= dalloc(&c->cnt64, n + 1);
    rc |= dalloc(&c->groups, n + 1);
    rc |= dalloc(&c->groups_tmp, n + 1);
    rc |= dalloc(&c->grp_cnt, n + 1);
    rc |= dalloc(&c->grp_off, n + 1);
    rc |= dalloc(&c->stack_spill, (int64_t)c->sm_count * kSpillWarpsPerSM * kStackSpillPerWarp);
    rc |= dalloc(&c->start_tab, kStartTableSize);
    rc |= dalloc(&c->ctr, 1);
    rc |= dalloc(&c->err, 1);
    rc |= dalloc(&c->work, 64);
    rc |= dalloc(&c->ctr_log, Ctx::kMaxTimed);
    if (rc == 0 && cudaMallocHost(&c->ctr_log_host, Ctx::kMaxTimed * sizeof(DevCounters)) != cudaSuccess)
        rc = SPHGRP_ENOMEM;
    if (rc == 0 && cudaMallocHost(&c->host_small, 64 * sizeof(int)) != cudaSuccess) rc = SPHGRP_ENOMEM;
    for (int k = 0; rc == 0 && k < 2 * Ctx::kMaxTimed; ++k)
        if (cudaEventCreate(&c->tev[k]) != cudaSuccess) rc = SPHGRP_ECUDA;
    if (rc) {
        sphgrp_ctx_destroy(reinterpret_cast<sphgrp_ctx*>(c));
        return set_error(SPHGRP_ENOMEM, "device allocation failed for n_max = " + std::to_string(n_max));
    }
    *out = reinterpret_cast<sphgrp_ctx*>(c);
    return SPHGRP_OK;
}

int sphgrp_ctx_destroy(sphgrp_ctx* ctx) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c) return SPHGRP_OK;
    void* ptrs[] = {c->keys, c->keys_alt, c->perm, c->perm_alt, c->rank_of, c->hist, c->xd, c->yd,
                    c->zd, c->pfix, c->poff, c->h64, c->hyd0, c->hyd1, c->act, c->act2, c->flag,
                    c->scan, c->scan_aux, c->lo, c->hi, c->res4, c->acc_rho, c->acc_drho, c->acc_n,
                    c->cnt64, c->groups, c->groups_tmp, c->grp_cnt, c->grp_off,
                    c->acc_s2, c->wadj, c->dadj, c->adj0, c->adj1, c->adj2, c->adj3,
                    c->stack_spill, c->start_tab, c->ctr, c->err, c->work, c->ctr_log, c->tree.ncen, c->tree.next, c->tree.nlink,
                    c->tree.nlevel, c->tree.box_lo, c->tree.box_hi, c->tree.top_cells, c->lst, c->lrec, c->lhw,
                    c->lslot, c->npass};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->host_small) cudaFreeHost(c->host_small);
    if (c->ctr_log_host) cudaFreeHost(c->ctr_log_host);
    for (int k = 0; k < 2 * Ctx::kMaxTimed; ++k)
        if (c->tev[k]) cudaEventDestroy(c->tev[k]);
    delete c;
    return SPHGRP_OK;
}

int sphgrp_sfc_keys_sort(sphgrp_ctx* ctx, int64_t n, const double* pos, uint64_t* keys_out,
                         int32_t* perm_out, cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c) return set_error(SPHGRP_EINVAL, "null context");
    if (n < 1 || n > c->n_max) return set_error(SPHGRP_EINVAL, "n outside [1, n_max]");
    if (!pos) return set_error(SPHGRP_EINVAL, "null positions");
    c->sorted = false;
    c->built = false;
    c->n = n;
    reset_flags(c, s);
    int rc = sort_keys(c, n, pos, s);
    if (!rc && keys_out) rc = check_cuda(cudaMemcpyAsync(keys_out, c->keys, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s), "keys copy");
    if (!rc && perm_out) rc = check_cuda(cudaMemcpyAsync(perm_out, c->perm, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s), "perm copy");
    rc = finish(c, s, rc);
    if (!rc) c->sorted = true;
    return rc;
}

int sphgrp_tree_build(sphgrp_ctx* ctx, int64_t n, const double* pos, const float* m, cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c) return set_error(SPHGRP_EINVAL, "null context");
    if (!c->sorted || n != c->n) return set_error(SPHGRP_ESTATE, "tree_build needs a preceding sfc_keys_sort of the same n");
    if (!pos || !m) return set_error(SPHGRP_EINVAL, "null positions or masses");
    c->built = false;
    reset_flags(c, s);
    int rc = gather_particles(c, pos, m, s);
    if (!rc) rc = build_tree(c, s);
    rc = finish(c, s, rc);
    if (!rc) c->built = true;
    return rc;
}

int sphgrp_ngb_search(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, const double* h,
                      int kind, int mode, int group_size, int64_t cap, int64_t* offsets,
                      int32_t* idx, int64_t* n_pairs, cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    int rc = check_common(c, n_act, active, mode, group_size);
    if (rc) return rc;
    if (kind != SPHGRP_DENSITY && kind != SPHGRP_HYDRO) return set_error(SPHGRP_EINVAL, "bad kind");
    if (!h || !offsets || !n_pairs) return set_error(SPHGRP_EINVAL, "null h, offsets or n_pairs");
    reset_flags(c, s);
    k_gather_h<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, h, c->h64, c->pfix, c->err);
    note_launch();
    if (kind == SPHGRP_HYDRO) {
        cudaMemsetAsync(c->hyd0, 0, c->n * sizeof(float4), s);
        cudaMemsetAsync(c->hyd1, 0, c->n * sizeof(float4), s);
        if ((rc = refresh_hmax(c, s))) return rc;
    }
    int nu = 0;
    if ((rc = prepare_active(c, n_act, active, s, &nu))) return rc;
    const bool grouped = mode == SPHGRP_GROUPED;
    SearchArgs a = base_args(c);
    a.U = c->act;
    a.nu = nu;
    a.g = grouped ? group_size : 1;
    a.ngroups = grouped ? (nu + group_size - 1) / group_size : nu;
    if (grouped && (rc = make_groups(c, &a, c->act, nu, group_size, s))) return rc;
    a.x_cnt = c->cnt64;
    a.x_off = c->cnt64;
    a.x_cap = cap;
    cudaMemsetAsync(c->cnt64, 0, c->n * sizeof(int64_t), s);
    timer_begin(c, s);
    rc = launch_search(a, kind, kCount, grouped, c->sm_count, s);
    timer_end(c, s, a.nu);
    if (rc) return rc;
    k_counts_by_caller<<<blocks_for(n_act, 256), 256, 0, s>>>(n_act, active, c->n, c->cnt64, offsets);
    note_launch();
    if ((rc = exclusive_scan_i64(c, offsets, offsets, n_act, offsets + n_act, s))) return rc;
    if (n_act == 0) cudaMemsetAsync(offsets, 0, sizeof(int64_t), s);
    int64_t total = 0;
    cudaMemcpyAsync(c->host_small + 32, offsets + n_act, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "pair count"))) return rc;
    std::memcpy(&total, c->host_small + 32, sizeof(int64_t));
    *n_pairs = total;
    if (idx) {
        k_offsets_by_orig<<<blocks_for(n_act, 256), 256, 0, s>>>(n_act, active, c->n, offsets, c->cnt64);
        note_launch();
        a.x_idx = idx;
        timer_begin(c, s);
        rc = launch_search(a, kind, kFill, grouped, c->sm_count, s);
        timer_end(c, s, a.nu);
        if (rc) return rc;
        if (total > cap) {
            finish(c, s, 0);
            return set_error(SPHGRP_EOVERFLOW, "more pairs than cap");
        }
    }
    c->last.walks = a.ngroups;
    c->last.members = nu;
    return finish(c, s, 0);
}

int sphgrp_group_supersets(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, const double* h,
                           int kind, int group_size, int64_t cap, int64_t* group_offsets,
                           int32_t* group_first, int32_t* members, int32_t* cand, int64_t* n_groups,
                           int64_t* n_cand, cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    int rc = check_common(c, n_act, active, SPHGRP_GROUPED, group_size);
    if (rc) return rc;
    if (kind != SPHGRP_DENSITY && kind != SPHGRP_HYDRO) return set_error(SPHGRP_EINVAL, "bad kind");
    if (!h || !group_offsets || !n_cand || !n_groups)
        return set_error(SPHGRP_EINVAL, "null h, group_offsets, n_groups or n_cand");
    reset_flags(c, s);
    k_gather_h<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, h, c->h64, c->pfix, c->err);
    note_launch();
    if (kind == SPHGRP_HYDRO) {
        cudaMemsetAsync(c->hyd0, 0, c->n * sizeof(float4), s);
        cudaMemsetAsync(c->hyd1, 0, c->n * sizeof(float4), s);
        if ((rc = refresh_hmax(c, s))) return rc;
    }
    int nu = 0;
    if ((rc = prepare_active(c, n_act, active, s, &nu))) return rc;
    SearchArgs a = base_args(c);
    a.U = c->act;
    a.nu = nu;
    a.g = group_size;
    if ((rc = make_groups(c, &a, c->act, nu, group_size, s))) return rc;
    a.x_cnt = c->cnt64;
    a.x_cap = cap;
    timer_begin(c, s);
    rc = launch_search(a, kind, kSupCount, true, c->sm_count, s);
    timer_end(c, s, a.nu);
    if (rc) return rc;
    int ng = a.ngroups;
    if ((rc = exclusive_scan_i64(c, c->cnt64, group_offsets, ng, group_offsets + ng, s))) return rc;
    if (ng == 0) cudaMemsetAsync(group_offsets, 0, sizeof(int64_t), s);
    if (members) {
        k_members<<<blocks_for(nu, 256), 256, 0, s>>>(nu, c->act, c->perm, members);
        note_launch();
    }
    if (group_first) {
        k_group_first<<<blocks_for(ng + 1, 256), 256, 0, s>>>(ng, nu, group_size, a.groups, group_first);
        note_launch();
    }
    cudaMemcpyAsync(c->host_small + 32, group_offsets + ng, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "superset count"))) return rc;
    int64_t total = 0;
    std::memcpy(&total, c->host_small + 32, sizeof(int64_t));
    *n_cand = total;
    *n_groups = ng;
    if (cand) {
        a.x_off = group_offsets;
        a.x_idx = cand;
        timer_begin(c, s);
        rc = launch_search(a, kind, kSupFill, true, c->sm_count, s);
        timer_end(c, s, a.nu);
        if (rc) return rc;
        if (total > cap) {
            finish(c, s, 0);
            return set_error(SPHGRP_EOVERFLOW, "more candidates than cap");
        }
    }
    c->last.walks = ng;
    c->last.members = nu;
    return finish(c, s, 0);
}

}  // extern "C"

namespace sphgrp {

// The density with the smoothing-length iteration; with vel (not NULL) the same density
// loop also sums the velocity divergence and curl (grouped form, walk passes), written to
// divv / curlv at each particle's final h.
int density_call(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, double* h, int iterate, int mode,
                 int group_size, float* rho, float* drhodh, float* fgrad, int32_t* nngb, int32_t* iters,
                 const float* vel, float* divv, float* curlv, cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    int rc = check_common(c, n_act, active, mode, group_size);
    if (rc) return rc;
    if (!h || !rho || !drhodh || !fgrad || !nngb) return set_error(SPHGRP_EINVAL, "null output array");
    const bool with_vel = vel != nullptr;
    if (with_vel && (!divv || !curlv)) return set_error(SPHGRP_EINVAL, "null divv or curlv");
    reset_flags(c, s);
    k_gather_h<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, h, c->h64, c->pfix, c->err);
    note_launch();
    if (with_vel) {
        k_vel_gather<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, vel, c->hyd0);
        note_launch();
    }
    int nu = 0;
    if ((rc = prepare_active(c, n_act, active, s, &nu))) return rc;
    const bool grouped = mode == SPHGRP_GROUPED;
    int32_t* U = c->act;
    int32_t* U2 = c->act2;
    int* nfail = c->work + 8;
    cudaMemsetAsync(nfail, 0, sizeof(int), s);
    const int iteration = with_vel ? SPHGRP_ITER_PASSES : c->p.iteration;
    if (grouped && iterate && iteration == SPHGRP_ITER_IN_GROUP) {
        // one launch: every group iterates its members to convergence
        SearchArgs a = base_args(c);
        a.U = U;
        a.nu = nu;
        a.g = group_size;
        a.ngroups = (nu + group_size - 1) / group_size;
        if (nu > 0 && (rc = make_groups(c, &a, U, nu, group_size, s))) return rc;
        int* max_pass = c->work + 10;
        cudaMemsetAsync(max_pass, 0, sizeof(int), s);
        IterArgs it;
        std::memset(&it, 0, sizeof(it));
        it.nngb = c->p.nngb;
        it.tol = c->p.nngb_tol;
        it.max_iter = c->p.max_iter;
        it.h64 = c->h64;
        it.pfix = c->pfix;
        it.h_out = h;
        it.rho = rho;
        it.drhodh = drhodh;
        it.fgrad = fgrad;
        it.nngb_out = nngb;
        it.iters = iters;
        it.nfail = nfail;
        it.max_pass = max_pass;
        if (nu > 0) {
            timer_begin(c, s);
            rc = launch_density_iter(a, it, group_size, c->sm_count, s);
            timer_end(c, s, nu);
            if (rc) return rc;
        }
        cudaMemcpyAsync(c->host_small + 2, nfail, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(c->host_small + 3, max_pass, sizeof(int), cudaMemcpyDeviceToHost, s);
        rc = finish(c, s, 0);
        c->last.walks = a.ngroups;
        c->last.members = nu;
        c->last.iterations = c->host_small[3];
        if (rc) return rc;
        if (c->host_small[2] > 0)
            return set_error(SPHGRP_ENOCONV, std::to_string(c->host_small[2]) + " particles did not converge");
        return SPHGRP_OK;
    }
    int64_t walks = 0, members = 0;
    int it = 1;
    const int max_iter = iterate ? c->p.max_iter : 1;
    // Recycled iteration (Sec. 2.2 iteration with the Sec. 2.1 supersets reused): the
    // first pass keeps every member's candidates within h_w = iter_widen * h, and the
    // later passes of the members whose h stays within h_w iterate on those lists in one
    // kernel; the rest continue with walk passes as below.
    bool recycle = grouped && iterate && iteration == SPHGRP_ITER_RECYCLE && group_size <= 32 && nu > 0;
    if (recycle && (rc = list_buffers(c)) != SPHGRP_OK) {
        if (rc != SPHGRP_ENOMEM) return rc;
        recycle = false;   // not enough device memory for the lists: walk passes only
    }
    int32_t* npass = recycle ? c->npass : nullptr;
    int* max_pass = c->work + 10;
    int list_passes = 0;
    if (recycle) {
        cudaMemsetAsync(c->npass, 0, c->n * sizeof(int32_t), s);
        cudaMemsetAsync(max_pass, 0, sizeof(int), s);
    }
    for (it = 1; it <= max_iter && nu > 0; ++it) {
        SearchArgs a = base_args(c);
        a.U = U;
        a.nu = nu;
        a.g = grouped ? group_size : 1;
        a.ngroups = grouped ? (nu + group_size - 1) / group_size : nu;
        if (grouped && (rc = make_groups(c, &a, U, nu, group_size, s))) return rc;
        walks += a.ngroups;
        members += nu;
        UpdateArgs ua;
        std::memset(&ua, 0, sizeof(ua));
        ua.U = U;
        ua.nu = nu;
        ua.it = it;
        ua.max_iter = max_iter;
        ua.nngb = c->p.nngb;
        ua.tol = c->p.nngb_tol;
        ua.poff = c->poff;
        ua.h64 = c->h64;
        ua.pfix = c->pfix;
        ua.lo = c->lo;
        ua.hi = c->hi;
        ua.keep = c->flag;
        ua.perm = c->perm;
        ua.h_out = h;
        ua.rho = rho;
        ua.drhodh = drhodh;
        ua.fgrad = fgrad;
        ua.nngb_out = nngb;
        ua.iters = iters;
        ua.iterate = iterate;
        ua.nfail = nfail;
        a.o_s0 = c->acc_rho;
        a.o_s1 = c->acc_drho;
        a.o_n = c->acc_n;
        ua.s0 = c->acc_rho;
        ua.s1 = c->acc_drho;
        ua.n = c->acc_n;
        ua.npass = npass;
        // the recycled iteration's list passes write their finished particles directly;
        // the walk passes leave theirs in rank space for one gather after the loop
        ua.res_k = recycle ? nullptr : c->res4;
        if (with_vel) {
            // the raw div / curl sums of the pass in hyd1 (not used by the density loop)
            a.o_vsum = c->hyd1;
            ua.vsum = c->hyd1;
            ua.divv = divv;
            ua.curlv = curlv;
        }
        const bool lists = recycle && it == 1;
        if (lists) {
            a.o_list = c->lst;
            a.o_lrec = c->lrec;
            a.o_lhw = c->lhw;
            a.o_lslot = c->lslot;
            a.list_widen = c->p.iter_widen;
        }
        timer_begin(c, s);
        rc = launch_search(a, lists ? kKindDensityList : with_vel ? kKindDensityVel : SPHGRP_DENSITY, kAcc, grouped,
                           c->sm_count, s);
        timer_end(c, s, a.nu);
        if (rc) return rc;
        if ((rc = launch_hsml_update(ua, s))) return rc;
        if (!iterate) break;
        if ((rc = compact_unconverged(c, &U, &U2, &nu, s))) return rc;
        if (lists && nu > 0) {
            // passes 2, 3, ... of the particles whose h stays within their list's h_w
            ListIterArgs la;
            std::memset(&la, 0, sizeof(la));
            la.U = U;
            la.nu = nu;
            la.max_iter = max_iter;
            la.nngb = c->p.nngb;
            la.tol = c->p.nngb_tol;
            la.pfix_in = c->pfix;
            la.pfix = c->pfix;
            la.poff = c->poff;
            la.xd = c->xd;
            la.yd = c->yd;
            la.zd = c->zd;
            la.h64 = c->h64;
            la.lo = c->lo;
            la.hi = c->hi;
            la.lslot = c->lslot;
            la.lrec = c->lrec;
            la.lhw = c->lhw;
            la.list = c->lst;
            la.npass = c->npass;
            la.max_pass = max_pass;
            la.keep = c->flag;
            la.perm = c->perm;
            la.h_out = h;
            la.rho = rho;
            la.drhodh = drhodh;
            la.fgrad = fgrad;
            la.nngb_out = nngb;
            la.iters = iters;
            la.nfail = nfail;
            la.ctr = c->ctr;
            if ((rc = launch_list_iterate(la, s))) return rc;
            if ((rc = compact_unconverged(c, &U, &U2, &nu, s))) return rc;
            cudaMemcpyAsync(c->host_small + 3, max_pass, sizeof(int), cudaMemcpyDeviceToHost, s);
            if ((rc = check_cuda(cudaStreamSynchronize(s), "list passes"))) return rc;
            list_passes = c->host_small[3];
            it = std::max(it, list_passes);   // the walk passes continue the count
        }
    }
    if (!recycle && n_act > 0) {
        k_out_density<<<blocks_for(n_act, 256), 256, 0, s>>>(n_act, active, c->n, c->rank_of, c->h64, c->res4,
                                                            with_vel ? c->hyd1 : nullptr, h, rho, drhodh, fgrad,
                                                            nngb, iters, divv, curlv);
        note_launch();
    }
    cudaMemcpyAsync(c->host_small + 2, nfail, sizeof(int), cudaMemcpyDeviceToHost, s);
    rc = finish(c, s, 0);
    c->last.walks = walks;
    c->last.members = members;
    c->last.iterations = std::min(std::max(it, list_passes), max_iter);
    if (rc) return rc;
    if (c->host_small[2] > 0)
        return set_error(SPHGRP_ENOCONV, std::to_string(c->host_small[2]) + " particles did not converge");
    return SPHGRP_OK;
}

// hydro forces, with Balsara's limiter when divv / curlv are given
int hydro_force(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, const double* h, const float* rho,
                const float* fgrad, const float* vel, const float* u, const float* divv, const float* curlv,
                int mode, int group_size, float* acc, float* dudt, int32_t* nngb, cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    int rc = check_common(c, n_act, active, mode, group_size);
    if (rc) return rc;
    if (!h || !rho || !fgrad || !vel || !u || !acc || !dudt) return set_error(SPHGRP_EINVAL, "null array");
    reset_flags(c, s);
    if ((rc = launch_hydro_prep(c, h, rho, fgrad, vel, u, s, divv, curlv))) return rc;
    if ((rc = refresh_hmax(c, s))) return rc;
    int nu = 0;
    if ((rc = prepare_active(c, n_act, active, s, &nu))) return rc;
    const bool grouped = mode == SPHGRP_GROUPED;
    SearchArgs a = base_args(c);
    a.U = c->act;
    a.nu = nu;
    a.g = grouped ? group_size : 1;
    a.ngroups = grouped ? (nu + group_size - 1) / group_size : nu;
    if (grouped && (rc = make_groups(c, &a, c->act, nu, group_size, s))) return rc;
    a.o_res4 = c->res4;
    a.o_rcnt = c->acc_n;
    timer_begin(c, s);
    rc = launch_search(a, SPHGRP_HYDRO, kAcc, grouped, c->sm_count, s);
    timer_end(c, s, a.nu);
    if (rc) return rc;
    if (n_act > 0) {
        k_out_hydro<<<blocks_for(n_act, 256), 256, 0, s>>>(n_act, active, c->n, c->rank_of, c->res4, c->acc_n, acc, dudt,
                                                          nngb);
        note_launch();
    }
    c->last.walks = a.ngroups;
    c->last.members = nu;
    return finish(c, s, 0);
}

}  // namespace sphgrp

extern "C" {

int sphgrp_density(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, double* h, int iterate,
                   int mode, int group_size, float* rho, float* drhodh, float* fgrad, int32_t* nngb,
                   int32_t* iters, cudaStream_t s) {
    return density_call(ctx, n_act, active, h, iterate, mode, group_size, rho, drhodh, fgrad, nngb, iters,
                        nullptr, nullptr, nullptr, s);
}

int sphgrp_density_derivs(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, double* h, int iterate,
                          int group_size, const float* vel, float* rho, float* drhodh, float* fgrad,
                          int32_t* nngb, int32_t* iters, float* divv, float* curlv, cudaStream_t s) {
    if (!vel) return set_error(SPHGRP_EINVAL, "null vel");
    return density_call(ctx, n_act, active, h, iterate, SPHGRP_GROUPED, group_size, rho, drhodh, fgrad, nngb,
                        iters, vel, divv, curlv, s);
}

int sphgrp_hydro_force(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, const double* h,
                       const float* rho, const float* fgrad, const float* vel, const float* u,
                       int mode, int group_size, float* acc, float* dudt, int32_t* nngb,
                       cudaStream_t s) {
    return hydro_force(ctx, n_act, active, h, rho, fgrad, vel, u, nullptr, nullptr, mode, group_size, acc, dudt,
                       nngb, s);
}

int sphgrp_hydro_force_balsara(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, const double* h,
                               const float* rho, const float* fgrad, const float* vel, const float* u,
                               const float* divv, const float* curlv, int mode, int group_size, float* acc,
                               float* dudt, int32_t* nngb, cudaStream_t s) {
    if (!divv || !curlv) return set_error(SPHGRP_EINVAL, "null divv or curlv");
    return hydro_force(ctx, n_act, active, h, rho, fgrad, vel, u, divv, curlv, mode, group_size, acc, dudt,
                       nngb, s);
}

int sphgrp_velocity_derivs(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, const double* h,
                           const float* rho, const float* vel, int group_size, float* divv, float* curlv,
                           cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    int rc = check_common(c, n_act, active, SPHGRP_GROUPED, group_size);
    if (rc) return rc;
    if (!h || !rho || !vel || !divv || !curlv) return set_error(SPHGRP_EINVAL, "null array");
    reset_flags(c, s);
    k_velocity_prep<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, h, rho, vel, c->h64, c->pfix, c->hyd0,
                                                         c->hyd1, c->err);
    note_launch();
    if ((rc = refresh_hmax(c, s))) return rc;
    int nu = 0;
    if ((rc = prepare_active(c, n_act, active, s, &nu))) return rc;
    SearchArgs a = base_args(c);
    a.U = c->act;
    a.nu = nu;
    a.g = group_size;
    a.ngroups = (nu + group_size - 1) / group_size;
    if ((rc = make_groups(c, &a, c->act, nu, group_size, s))) return rc;
    a.o_res4 = c->res4;
    timer_begin(c, s);
    rc = launch_search(a, kKindVelocity, kAcc, true, c->sm_count, s);
    timer_end(c, s, a.nu);
    if (rc) return rc;
    if (n_act > 0) {
        k_out_vel<<<blocks_for(n_act, 256), 256, 0, s>>>(n_act, active, c->n, c->rank_of, c->res4, divv, curlv);
        note_launch();
    }
    c->last.walks = a.ngroups;
    c->last.members = nu;
    return finish(c, s, 0);
}

int sphgrp_get_launch_log(sphgrp_ctx* ctx, int cap, int64_t* members, int64_t* candidates,
                          int64_t* pair_tests, int64_t* nodes, double* ms, int* count) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c || !count || cap < 0) return set_error(SPHGRP_EINVAL, "null argument");
    int n = std::min(cap, c->ntimed);
    for (int k = 0; k < n; ++k) {
        const DevCounters& cur = c->ctr_log_host[k];
        DevCounters prev{};
        if (k > 0) prev = c->ctr_log_host[k - 1];
        if (members) members[k] = c->log_members[k];
        if (candidates) candidates[k] = (int64_t)(cur.cands - prev.cands);
        if (pair_tests) pair_tests[k] = (int64_t)(cur.tests - prev.tests);
        if (nodes) nodes[k] = (int64_t)(cur.nodes - prev.nodes);
        if (ms) ms[k] = c->log_ms[k];
    }
    *count = n;
    return SPHGRP_OK;
}

int sphgrp_get_stats(sphgrp_ctx* ctx, sphgrp_stats* out) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c || !out) return set_error(SPHGRP_EINVAL, "null argument");
    *out = c->last;
    return SPHGRP_OK;
}

}  // extern "C"
