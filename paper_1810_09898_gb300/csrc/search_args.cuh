// Argument blocks of the search and smoothing-length kernels (ngb.cu), filled by
// the C ABI layer (api.cu).
#pragma once

#include "sph_internal.cuh"

namespace sphgrp {

enum Mode { kAcc = 0, kCount = 1, kFill = 2, kSupCount = 3, kSupFill = 4 };

// pair loops of the search kernels: SPHGRP_DENSITY (0), SPHGRP_HYDRO (1) and the adjoints
enum Kind { kKindDensity = 0, kKindHydro = 1, kKindHydroAdj = 2, kKindDensityAdj = 3, kKindVelocity = 4,
            kKindDensityList = 5, kKindDensityVel = 6 };

// Candidate lists of the recycled smoothing-length iteration: every member of a pass-1
// group keeps the candidates of the group's superset that lie within its widened radius
// h_w = widen * h, in up to four sub-lists (one per slice of the member layout) of
// kListCap / S entries.  A record per list slot {c0 | c1 << 16, c2 | c3 << 16, S, valid}.
constexpr int kListCap = 192;

// smoothing-length update of the density passes (per unconverged particle, FP64)
struct UpdateArgs {
    const int32_t* U;
    int nu;
    int it;
    int max_iter;
    double nngb, tol;
    const float* s0;
    const float* s1;
    const int32_t* n;
    const float4* poff;
    double* h64;
    uint4* pfix;
    double* lo;
    double* hi;
    int32_t* keep;        // 1 = still unconverged
    const int32_t* perm;
    // caller outputs (original order)
    double* h_out;
    float* rho;
    float* drhodh;
    float* fgrad;
    int32_t* nngb_out;
    int32_t* iters;
    int iterate;
    int* nfail;
    int32_t* npass;       // optional: passes made so far per rank (null: every particle is at pass it)
    // optional: velocity divergence / curl sums of the density pass (rank space, {div, curl}
    // before the 1/rho); a finished particle writes div v and curl v to the caller's order
    const float4* vsum;
    float* divv;
    float* curlv;
    // optional: a finished particle only records {s0, s1, count, pass count} here (rank
    // space, one float4; its h stays in h64) and the caller's outputs are written after
    // the iteration by one gather over the active list (k_out_density)
    float4* res_k;
};

// passes 2, 3, ... of the recycled iteration over the members' candidate lists
struct ListIterArgs {
    const int32_t* U;     // unconverged work list (ranks)
    int nu;
    int max_iter;
    double nngb, tol;
    const uint4* pfix_in;   // positions (read); pfix.w is written through pfix
    uint4* pfix;
    const float4* poff;
    const double *xd, *yd, *zd;
    double* h64;
    double* lo;
    double* hi;
    const int32_t* lslot;   // rank -> list slot
    const int4* lrec;       // list records
    const double* lhw;      // widened h of every slot
    const int32_t* list;    // kListCap entries per slot
    int32_t* npass;
    int* max_pass;          // largest pass count reached on a list
    int32_t* keep;          // 1: the member needs a walk pass (h beyond h_w or a list overflowed)
    const int32_t* perm;
    double* h_out;
    float* rho;
    float* drhodh;
    float* fgrad;
    int32_t* nngb_out;
    int32_t* iters;
    int* nfail;
    DevCounters* ctr;
};

struct SearchArgs {
    // octree
    const uint4* ncen;
    const float4* next;
    const int4* nlink;
    // key-ordered particles
    const uint4* pfix;
    const float4* poff;
    const double *xd, *yd, *zd;
    const double* h64;
    const float4* hyd0;   // {vx, vy, vz, c}
    const float4* hyd1;   // {A, rho, hinv, s}
    const float4* wadj;   // {wx, wy, wz, -}: weights dL/da of the hydro adjoint
    const float4* dadj;   // {alpha, beta, hinv, s}: coefficients of the density adjoint
    const int32_t* perm;
    // work list: ranks of the particles to process, in key order
    const int32_t* U;
    int nu;
    int g;          // group size (grouped form)
    int ngroups;
    bool centre_box; // group sphere centred on the members' box (else on the first member)
    const int2* groups; // (first entry of U, count) per group; null: chunks of g
    const int4* groups4; // batch groups: (first entry of U, count, root node, g | max_slices << 8)
    const int* ngroups_dev; // device group count (graph-capturable launches); null: ngroups
    // density pass results (rank space)
    float* o_s0;
    float* o_s1;
    float* o_s2;          // optional: d2Rho/dh2 sum (backward)
    int32_t* o_n;
    float4* o_vsum;       // density with velocity derivatives: {div, curl} sums (rank space)
    // adjoint results (rank space)
    float4* o_adj0;       // hydro adjoint {xb, mb}
    float4* o_adj1;       // hydro adjoint {vb, -}
    float4* o_adj2;       // hydro adjoint {hb, rhob, Ab, n}
    float4* o_adj3;       // density adjoint {xb, mb}
    // velocity derivatives (original order)
    float* o_divv;
    float* o_curl;        // n x 3
    // hydro / velocity-derivative results in key order (rank space, one float4 per
    // member: {a, du/dt} or {div v, curl v}) and the hydro neighbour counts; null: the
    // results go straight to the caller's order below
    float4* o_res4;
    int32_t* o_rcnt;
    // hydro results (original order)
    float* o_acc;
    float* o_dudt;
    int32_t* o_nh;
    // export (indexed by original particle index)
    const int64_t* x_off;
    int64_t* x_cnt;
    int32_t* x_idx;
    int64_t x_cap;
    // candidate lists of the recycled iteration (kind kKindDensityList)
    int32_t* o_list;      // kListCap entries per slot; slot = pass-1 work-list index
    int4* o_lrec;
    double* o_lhw;
    int32_t* o_lslot;     // rank -> slot
    double list_widen;    // h_w / h
    // hydro constants
    float alpha, beta, eps;
    // bookkeeping
    DevCounters* ctr;
    unsigned* err;
    int* work;
    uint32_t* stack_spill;   // walk stack overflow, kStackSpillPerWarp entries per warp
    const int32_t* start_tab; // walk start table (null: walks start at their root)
    int stack_cap;            // walk-stack entries kept in shared memory (<= kStackSharedMax)
};


// smoothing-length iteration inside the grouped density kernel (batch path)
struct IterArgs {
    double nngb, tol;
    int max_iter;
    double* h64;          // rank order, updated in place
    uint4* pfix;          // .w = FP32 copy of h
    // results (original order)
    double* h_out;
    float* rho;
    float* drhodh;
    float* fgrad;
    int32_t* nngb_out;
    int32_t* iters;
    int* nfail;
    int* max_pass;        // optional: largest pass count of any particle
};

int launch_search(const SearchArgs& a, int kind, int mode, bool grouped, int sm_count, cudaStream_t s);
int launch_hsml_update(const UpdateArgs& a, cudaStream_t s);
int launch_list_iterate(const ListIterArgs& a, cudaStream_t s);
// persistent launches over a device-side group count (a.ngroups_dev), graph-capturable
int launch_search_dev(const SearchArgs& a, int kind, int max_g, int sm_count, cudaStream_t s);
int launch_density_iter(const SearchArgs& a, const IterArgs& it, int max_g, int sm_count, cudaStream_t s);
int launch_search_pair(const SearchArgs& a0, int kind0, const SearchArgs& a1, int kind1, int max_g, int sm_count,
                       cudaStream_t s);
int launch_split_groups(const int32_t* U, int nu, int g, float split, const uint4* pfix, const double* h64,
                        int2* tmp, int32_t* cnt, cudaStream_t s);
// radius grouping: the greedy scan restarts at the start of every run of this many
// work-list entries (one thread per run)
constexpr int kRadiusRun = 1024;
int launch_radius_groups(const int32_t* U, int nu, int cap, double f, const uint4* pfix, const float4* poff,
                         const double* h64, int2* tmp, int32_t* cnt, cudaStream_t s);
int launch_gather_groups(int nch, int g, const int2* tmp, const int32_t* cnt, const int32_t* off, int2* groups,
                         cudaStream_t s);
int gather_particles(Ctx* c, const double* pos, const float* m, cudaStream_t s);
int exclusive_scan_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_dev,
                       cudaStream_t s);

// per-particle kernels shared by the entry points (api.cu, backward.cu)
int launch_gather_h(Ctx* c, const double* h, cudaStream_t s);
int launch_hydro_prep(Ctx* c, const double* h, const float* rho, const float* fgrad, const float* vel,
                      const float* u, cudaStream_t s, const float* divv = nullptr, const float* curlv = nullptr);
int backward_buffers(Ctx* c);
int launch_bwd_prep(Ctx* c, const float* vel, const float* u, const float* g_acc, float4* hyd0, float4* hyd1,
                    cudaStream_t s);
int launch_bwd_chain(Ctx* c, const float* u, const float* g_rho, cudaStream_t s);
int launch_bwd_combine(Ctx* c, float* g_pos, float* g_vel, float* g_m, cudaStream_t s);

// call orchestration shared by the entry points (api.cu)
int finish(Ctx* c, cudaStream_t s, int rc);
void reset_flags(Ctx* c, cudaStream_t s);
int prepare_active(Ctx* c, int64_t n_act, const int32_t* active, cudaStream_t s, int* nu);
int make_groups(Ctx* c, SearchArgs* a, const int32_t* U, int nu, int g, cudaStream_t s);
SearchArgs base_args(Ctx* c);
int check_common(Ctx* c, int64_t n_act, const int32_t* active, int mode, int group_size);

}  // namespace sphgrp
