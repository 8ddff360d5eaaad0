// Backward (adjoint) of the density and hydro loops: the gradient of
//   L = sum_k w_k . a_k + sum_k s_k rho_k
// with respect to positions, velocities and masses.  The paper has no backward pass;
// this differentiates the density (Sec. 2.2 relation between h, rho and the
// neighbour number) and the hydro accelerations of the forward loops, with the
// neighbour sets of the given state held fixed and h defined by the exact constraint
// (4 pi / 3) h_k^3 rho_k = N_ngb m_k (implicit function theorem).
//
// Three grouped pair loops over the same groups and walks as the forward path
// (ngb.cu kinds 0, 2, 3) recompute every pair term from the staged candidate tiles; no
// pair list is stored.  Between them, per-particle FP64 kernels turn the density sums
// into rho, dRho/dh, d2Rho/dh2, f, A and c, and chain the adjoints of A, f, rho and h
// into the coefficients the density-adjoint loop gathers.
#include "search_args.cuh"

namespace sphgrp {

namespace {

constexpr double kPi = 3.14159265358979323846;

__global__ void k_iota_ranks(int64_t n, int32_t* __restrict__ out) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r < n) out[r] = (int32_t)r;
}

// rho, dRho/dh and f from the density sums s0 = sum m w, s1 = sum m (3w + q w')
struct DensityState {
    double h, rho, rh, f;
};

__device__ __forceinline__ DensityState density_state(double h, float s0, float s1) {
    DensityState d;
    d.h = h;
    const double sigma = 8.0 / (kPi * h * h * h);
    d.rho = sigma * (double)s0;
    d.rh = -sigma / h * (double)s1;
    d.f = 1.0 / (1.0 + h * d.rh / (3.0 * d.rho));
    return d;
}

// Inputs of the hydro-adjoint loop in key order: hyd0 = {v, c}, hyd1 = {A, rho, 1/h,
// 8/(pi h^4)}, wadj = {w, 0}, with A = f (gamma - 1) u / rho, c = sqrt(gamma (gamma - 1) u).
__global__ void k_bwd_prep(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ h64,
                           const float* __restrict__ s0, const float* __restrict__ s1,
                           const float* __restrict__ vel, const float* __restrict__ u,
                           const float* __restrict__ w, double gamma, float4* __restrict__ hyd0,
                           float4* __restrict__ hyd1, float4* __restrict__ wadj) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t i = perm[r];
    const DensityState d = density_state(h64[r], s0[r], s1[r]);
    const double ui = (double)u[i];
    const double A = d.f * (gamma - 1.0) * ui / d.rho;
    const double c = sqrt(gamma * (gamma - 1.0) * ui);
    hyd0[r] = make_float4(vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], (float)c);
    hyd1[r] = make_float4((float)A, (float)d.rho, (float)(1.0 / d.h), (float)(8.0 / (kPi * d.h * d.h * d.h * d.h)));
    wadj[r] = make_float4(w[3 * i], w[3 * i + 1], w[3 * i + 2], 0.0f);
}

// Per particle, FP64: the adjoints gathered by the hydro loop (h, rho, A) plus the
// density weight s flow through A = f (gamma-1) u / rho, f = 1 / (1 + h rho' / (3 rho)),
// rho(h), rho'(h) and the implicit h(x, m):
//   lambda = hbar f / (4 pi h^2 rho)  (adjoint of the constraint),
//   alpha = rhobar - lambda (4 pi / 3) h^3, beta = rho'bar,  mbar += lambda N_ngb.
// alpha and beta weight rho and rho' at fixed h in the density-adjoint loop.
__global__ void k_bwd_chain(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ h64,
                            const float* __restrict__ s0, const float* __restrict__ s1,
                            const float* __restrict__ s2, const float* __restrict__ u,
                            const float* __restrict__ g_rho, const float4* __restrict__ adj2, double gamma,
                            double nngb, float4* __restrict__ dadj, float4* __restrict__ adj1) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t i = perm[r];
    const DensityState d = density_state(h64[r], s0[r], s1[r]);
    const double h = d.h, rho = d.rho, rh = d.rh, f = d.f;
    const double sigma = 8.0 / (kPi * h * h * h);
    const double rhh = sigma / (h * h) * (double)s2[r];
    const double ui = u ? (double)u[i] : 0.0;   // no u: no acceleration term (Abar = 0)
    const double A = f * (gamma - 1.0) * ui / rho;
    const float4 G = adj2[r];   // {hbar, rhobar, Abar, -} of the hydro loop
    double rbar = (double)G.y + (g_rho ? (double)g_rho[i] : 0.0);
    const double fbar = (double)G.z * (gamma - 1.0) * ui / rho;
    rbar -= (double)G.z * A / rho;
    const double Dbar = -f * f * fbar;   // adjoint of 1 + h rho' / (3 rho)
    double hbar = (double)G.x + Dbar * rh / (3.0 * rho);
    const double rpbar = Dbar * h / (3.0 * rho);
    rbar -= Dbar * h * rh / (3.0 * rho * rho);
    hbar += rbar * rh + rpbar * rhh;
    const double lam = hbar * f / (4.0 * kPi * h * h * rho);
    const double alpha = rbar - lam * (4.0 * kPi / 3.0) * h * h * h;
    dadj[r] = make_float4((float)alpha, (float)rpbar, (float)(1.0 / h), (float)(8.0 / (kPi * h * h * h * h)));
    reinterpret_cast<float*>(adj1)[4 * r + 3] = (float)(lam * nngb);
}

// gradients in the caller's order
__global__ void k_bwd_combine(int64_t n, const int32_t* __restrict__ perm, const float4* __restrict__ adj0,
                              const float4* __restrict__ adj1, const float4* __restrict__ adj3,
                              float* __restrict__ g_pos, float* __restrict__ g_vel, float* __restrict__ g_m) {
    int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t i = perm[r];
    const float4 a = adj0[r], b = adj1[r], c = adj3[r];
    if (g_pos) {
        g_pos[3 * i] = a.x + c.x;
        g_pos[3 * i + 1] = a.y + c.y;
        g_pos[3 * i + 2] = a.z + c.z;
    }
    if (g_vel) {
        g_vel[3 * i] = b.x;
        g_vel[3 * i + 1] = b.y;
        g_vel[3 * i + 2] = b.z;
    }
    if (g_m) g_m[i] = a.w + b.w + c.w;
}

}  // namespace

template <typename T>
static int lazy_alloc(T** p, int64_t count) {
    if (*p) return SPHGRP_OK;
    return check_cuda(cudaMalloc(reinterpret_cast<void**>(p), (size_t)(count < 1 ? 1 : count) * sizeof(T)),
                      "cudaMalloc (backward buffers)");
}

int backward_buffers(Ctx* c) {
    const int64_t n = c->n_max;
    int rc = 0;
    if ((rc = lazy_alloc(&c->acc_s2, n))) return rc;
    float4** bufs[] = {&c->wadj, &c->dadj, &c->adj0, &c->adj1, &c->adj2, &c->adj3};
    for (float4** b : bufs)
        if ((rc = lazy_alloc(b, n))) return rc;
    return SPHGRP_OK;
}

int launch_bwd_prep(Ctx* c, const float* vel, const float* u, const float* g_acc, float4* hyd0, float4* hyd1,
                    cudaStream_t s) {
    k_bwd_prep<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, c->h64, c->acc_rho, c->acc_drho, vel, u, g_acc,
                                                     c->p.gamma, hyd0, hyd1, c->wadj);
    note_launch();
    return check_cuda(cudaGetLastError(), "backward prep");
}

int launch_bwd_chain(Ctx* c, const float* u, const float* g_rho, cudaStream_t s) {
    k_bwd_chain<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, c->h64, c->acc_rho, c->acc_drho, c->acc_s2, u,
                                                      g_rho, c->adj2, c->p.gamma, c->p.nngb, c->dadj, c->adj1);
    note_launch();
    return check_cuda(cudaGetLastError(), "backward chain");
}

int launch_bwd_combine(Ctx* c, float* g_pos, float* g_vel, float* g_m, cudaStream_t s) {
    k_bwd_combine<<<blocks_for(c->n, 256), 256, 0, s>>>(c->n, c->perm, c->adj0, c->adj1, c->adj3, g_pos, g_vel, g_m);
    note_launch();
    return check_cuda(cudaGetLastError(), "backward combine");
}

}  // namespace sphgrp

using namespace sphgrp;

extern "C" int sphgrp_backward(sphgrp_ctx* ctx, const double* h, const float* vel, const float* u,
                               const float* g_acc, const float* g_rho, int group_size, float* g_pos,
                               float* g_vel, float* g_m, cudaStream_t s) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    if (!c) return set_error(SPHGRP_EINVAL, "null context");
    if (!c->built) return set_error(SPHGRP_ESTATE, "no octree: call sphgrp_tree_build first");
    if (group_size < 1 || group_size > 128) return set_error(SPHGRP_EINVAL, "group_size must be in [1, 128]");
    const int64_t n = c->n;
    int rc = SPHGRP_OK;
    // g_acc NULL: L = sum g_rho . rho alone; the hydro adjoint is not run, vel and u are
    // not read
    const bool with_acc = g_acc != nullptr;
    if (!h || (with_acc && (!vel || !u))) return set_error(SPHGRP_EINVAL, "null h, or null vel or u with g_acc");
    if (!with_acc && !g_rho) return set_error(SPHGRP_EINVAL, "neither g_acc nor g_rho: nothing to differentiate");
    if (!g_pos && !g_vel && !g_m) return set_error(SPHGRP_EINVAL, "no gradient requested");
    if ((rc = backward_buffers(c))) return rc;
    reset_flags(c, s);
    if ((rc = launch_gather_h(c, h, s))) return rc;
    // the smoothing lengths are checked before any walk uses them
    cudaMemcpyAsync(c->host_small + 1, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "smoothing-length check"))) return rc;
    if ((unsigned)c->host_small[1] & kErrH) return finish(c, s, 0);
    if ((rc = refresh_hmax(c, s))) return rc;
    k_iota_ranks<<<blocks_for(n, 256), 256, 0, s>>>(n, c->act);
    note_launch();
    const int nu = (int)n;
    SearchArgs a = base_args(c);
    a.U = c->act;
    a.nu = nu;
    a.g = group_size;
    a.ngroups = (nu + group_size - 1) / group_size;
    if ((rc = make_groups(c, &a, c->act, nu, group_size, s))) return rc;

    // 1. density sums at the given h: rho, rho', rho''
    SearchArgs ad = a;
    ad.o_s0 = c->acc_rho;
    ad.o_s1 = c->acc_drho;
    ad.o_s2 = c->acc_s2;
    ad.o_n = c->acc_n;
    timer_begin(c, s);
    rc = launch_search(ad, kKindDensity, kAcc, true, c->sm_count, s);
    timer_end(c, s, nu);
    if (rc) return rc;
    if (with_acc) {
        if ((rc = launch_bwd_prep(c, vel, u, g_acc, c->hyd0, c->hyd1, s))) return rc;
        // 2. adjoint of sum w . a over every hydro pair
        SearchArgs ah = a;
        ah.o_adj0 = c->adj0;
        ah.o_adj1 = c->adj1;
        ah.o_adj2 = c->adj2;
        timer_begin(c, s);
        rc = launch_search(ah, kKindHydroAdj, kAcc, true, c->sm_count, s);
        timer_end(c, s, nu);
        if (rc) return rc;
    } else {
        // no acceleration term: its adjoints are zero
        cudaMemsetAsync(c->adj0, 0, n * sizeof(float4), s);
        cudaMemsetAsync(c->adj1, 0, n * sizeof(float4), s);
        cudaMemsetAsync(c->adj2, 0, n * sizeof(float4), s);
    }
    // 3. per particle: A, f, rho, h and the implicit h
    if ((rc = launch_bwd_chain(c, with_acc ? u : nullptr, g_rho, s))) return rc;
    // 4. adjoint of rho and rho' at fixed h over every density pair
    SearchArgs aa = a;
    aa.o_adj3 = c->adj3;
    timer_begin(c, s);
    rc = launch_search(aa, kKindDensityAdj, kAcc, true, c->sm_count, s);
    timer_end(c, s, nu);
    if (rc) return rc;
    if ((rc = launch_bwd_combine(c, g_pos, g_vel, g_m, s))) return rc;
    rc = check_cuda(cudaGetLastError(), "backward kernels");
    c->last.walks = (with_acc ? 3 : 2) * (int64_t)a.ngroups;
    c->last.members = (with_acc ? 3 : 2) * (int64_t)nu;
    return finish(c, s, rc);
}
