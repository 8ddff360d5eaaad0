/*
 * sphgrp.h -- C ABI of the GB300 SPH neighbour-search library.
 *
 * The library computes the hot path of "Exploiting the Space Filling Curve Ordering of
 * Particles in the Neighbour Search of Gadget3" (Ragagnin et al., arXiv:1810.09898):
 * Peano-Hilbert ordering of the particles, an octree over that order, the neighbour
 * search in its two forms -- one tree walk per active particle (Sec. 1.1, "standard
 * method", Fig. 1 left) and Neighbour Recycling (Sec. 2 and 2.1, Fig. 1 right: active
 * particles consecutive along the curve form a group, the group makes one walk for a
 * common superset of candidates, and each member filters the superset down to its own
 * neighbours) -- and the SPH density (with the smoothing-length iteration to a fixed
 * effective neighbour number, Sec. 2.2) and hydro-force loops that consume it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an int status: SPHGRP_OK (0) or a negative SPHGRP_E* code.
 *    sphgrp_last_error() returns a text describing the most recent failure of the
 *    calling thread (never NULL).
 *  - Positions are in units of the box side; the box is the periodic unit cube
 *    [0,1)^3 and every coordinate must lie in [0,1).  Distances use the minimum image.
 *    Smoothing lengths must satisfy 0 < h < 0.5 so that the minimum image is unique.
 *  - Arrays named "device" are device pointers in the caller's memory; the caller
 *    owns them, keeps them alive until the stream has passed the call, and the
 *    library never frees them.  Particle arrays are indexed by the caller's particle
 *    index ("original order"); the library keeps its own copies in key order.
 *  - pos and vel are row-major n x 3 arrays (x0 y0 z0 x1 ...).
 *  - Work is issued on the given stream.  Calls that report a count or a device-side
 *    error (every call that returns a status derived from device work) synchronise
 *    that stream before returning.
 *  - The context owns its device workspace (key-ordered particle copies, the octree,
 *    group and iteration state).  A context is used by one host thread at a time.
 */
#ifndef SPHGRP_H
#define SPHGRP_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SPHGRP_OK = 0,
    SPHGRP_EINVAL = -1,    /* bad argument: NaN or out-of-box position, h outside (0, 0.5), n = 0 ... */
    SPHGRP_ENOMEM = -2,    /* device allocation failed */
    SPHGRP_ENOCONV = -3,   /* smoothing-length iteration did not converge within max_iter */
    SPHGRP_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
    SPHGRP_EOVERFLOW = -5, /* an internal capacity was exceeded (results invalid) */
    SPHGRP_ECUDA = -6,     /* a CUDA runtime call failed */
    SPHGRP_ESTATE = -7     /* calls made out of order (e.g. a search before a tree) */
};

/* Neighbour-search forms. */
enum {
    SPHGRP_INDIVIDUAL = 0, /* one walk per active particle with radius h_i (Sec. 1.1) */
    SPHGRP_GROUPED = 1     /* Neighbour Recycling: one walk per group of group_size
                              consecutive active particles in key order (Sec. 2.1) */
};

/* Neighbour definitions (Sec. 1.1, last paragraph). */
enum {
    SPHGRP_DENSITY = 0, /* j is a neighbour of i iff |r_ij| < h_i (i itself included) */
    SPHGRP_HYDRO = 1    /* j != i is a neighbour of i iff |r_ij| < max(h_i, h_j) */
};

typedef struct sphgrp_params {
    double nngb;      /* target effective neighbour number 4 pi rho h^3 / (3 m), e.g. 64 */
    double nngb_tol;  /* iteration stops when |N_eff - nngb| <= nngb_tol, e.g. 2 */
    int max_iter;     /* smoothing-length passes before SPHGRP_ENOCONV, e.g. 100 */
    int leaf_size;    /* octree leaf bucket size B (nodes with more particles split), e.g. 16 */
    double gamma;     /* adiabatic index, P = (gamma - 1) rho u, e.g. 5/3 */
    double alpha;     /* Monaghan viscosity alpha, e.g. 1 */
    double beta;      /* Monaghan viscosity beta, e.g. 2 */
    double eps;       /* viscosity softening (mu denominator r^2 + eps hbar^2), e.g. 0.01 */
    int group_centre; /* centre of a group's search sphere: SPHGRP_CENTRE_FIRST (the group's
                         first particle, Sec. 2.1) or SPHGRP_CENTRE_BOX (the centre of the
                         members' bounding box; same superset guarantee, smaller radius) */
    double group_split; /* a group is cut (recursively) while its search sphere,
                           ((sqrt(3)/2) * largest extent of the members' box + smallest h)^3,
                           exceeds group_split * members * (smallest h)^3 in volume, i.e.
                           while a member would filter more than group_split * members times
                           its own sphere; the cut is at the largest gap in key order between
                           consecutive members (the middle when they are contiguous); <= 0
                           keeps plain chunks of group_size.  e.g. 2 */
    int iteration;      /* smoothing-length iteration of the grouped density:
                           SPHGRP_ITER_PASSES (default: one search launch per pass over the
                           still unconverged particles, regrouped), SPHGRP_ITER_IN_GROUP (one
                           launch; every group repeats walk, filter and update until its
                           members converge) or SPHGRP_ITER_RECYCLE (the first pass
                           also keeps, for every member, the candidates of its group's
                           superset within iter_widen * h; later passes of the particles
                           whose h stays within that radius iterate on those candidates in
                           one launch, the others take walk passes as in SPHGRP_ITER_PASSES;
                           group_size <= 32; device memory for 192 candidate ranks per
                           particle is allocated by the first such call, and without it the
                           call walks every pass).  The iterates are those of the pass-by-pass
                           iteration in every mode.  The individual form always iterates in
                           passes. */
    int group_mode;     /* how the grouped form cuts the active list (in key order) into groups:
                           SPHGRP_GROUP_COUNT: chunks of group_size, split as group_split says;
                           SPHGRP_GROUP_RADIUS (Sec. 2.1, the paper's rule): a group starts at an
                           active particle and takes the following ones while they lie within
                           R = group_f * h of its first particle, at most group_size of them
                           (the scan restarts at the start of every run of 1024 actives);
                           SPHGRP_GROUP_TREE: see group_level */
    double group_f;     /* R / h of the radius mode, e.g. 0.5 */
    int group_level;    /* depth of the tree mode (SPHGRP_GROUP_TREE, the octree grouping of
                           Sec. 2): a group is the active particles under one node of this
                           depth (the actives sharing the key's first 3 * group_level bits),
                           cut into pieces of at most group_size; 1 .. 21, e.g. 7 */
    int stack_shared;   /* walk-stack entries per warp kept in shared memory (32 .. 256); deeper
                           walks continue in a global overflow area.  e.g. 256 */
    double iter_widen;  /* SPHGRP_ITER_RECYCLE: radius of the kept candidates over h, in
                           [1, 2]; a particle whose h grows beyond it walks again.  e.g. 1.1 */
} sphgrp_params;

enum { SPHGRP_ITER_PASSES = 0, SPHGRP_ITER_IN_GROUP = 1, SPHGRP_ITER_RECYCLE = 2 };
enum { SPHGRP_GROUP_COUNT = 0, SPHGRP_GROUP_RADIUS = 1, SPHGRP_GROUP_TREE = 2 };

enum { SPHGRP_CENTRE_FIRST = 0, SPHGRP_CENTRE_BOX = 1 };

/* Fills p with the defaults quoted above. */
void sphgrp_default_params(sphgrp_params* p);

typedef struct sphgrp_stats {
    int64_t walks;          /* tree walks started (groups, or particles in the individual form) */
    int64_t nodes_tested;   /* node-overlap tests */
    int64_t candidates;     /* candidate particles taken from opened leaves (summed over walks) */
    int64_t pair_tests;     /* member x candidate distance tests */
    int64_t pairs;          /* neighbour pairs found */
    int64_t fp64_retests;   /* pairs re-decided from FP64 positions (within the FP32 error band) */
    int64_t iterations;     /* smoothing-length passes made by the last density call */
    int64_t max_stack;      /* deepest walk stack seen */
    int64_t members;        /* particles processed by the search kernels (summed over passes) */
    int64_t search_launches; /* search-kernel launches timed in the last call */
    double search_ms;       /* their summed device time (CUDA events on the call's stream) */
} sphgrp_stats;

typedef struct sphgrp_ctx sphgrp_ctx;

/* Creates a context for up to n_max particles, 1 <= n_max <= 2^30 (ranks and indices
 * are int32 on the device).  p may be NULL (defaults).  Device memory for n_max
 * particles is allocated here; the octree grows on demand.  Errors: EINVAL for n_max
 * outside that range or bad parameters, ENOMEM if an allocation fails (nothing is
 * left allocated). */
int sphgrp_ctx_create(sphgrp_ctx** ctx, const sphgrp_params* p, int64_t n_max);
int sphgrp_ctx_destroy(sphgrp_ctx* ctx);
const char* sphgrp_last_error(void);

/* a1 + a2 (Sec. 1.2: particles ordered along the Hilbert curve).
 * keys: 63-bit Peano-Hilbert key of every particle -- coordinates mapped to a 2^21
 * grid per axis, i = floor(x * 2^21), and the cell's Hilbert index by Skilling's
 * construction (axis order x, y, z, most significant level first) -- sorted
 * ascending by a stable device radix sort.
 * pos:      device, n x 3 FP64, in [0,1).
 * keys_out: device, n uint64, the sorted keys (may be NULL).
 * perm_out: device, n int32, perm_out[r] = original index of the particle of rank r
 *           (may be NULL).
 * The context keeps the order for the following calls.  Errors: EINVAL for n < 1,
 * n > n_max or a coordinate outside [0,1) (including NaN). */
int sphgrp_sfc_keys_sort(sphgrp_ctx* ctx, int64_t n, const double* pos, uint64_t* keys_out,
                         int32_t* perm_out, cudaStream_t stream);

/* a3 (Sec. 1.2: octree over the curve-ordered particles).  Gathers pos and m into key
 * order and builds the linear octree: a node with more than leaf_size particles is
 * split into its non-empty octants (the next 3 key bits), down to the 2^21 grid.
 * Each node keeps its tight bounding box, its particle range and the largest h of
 * its particles (set by the density and hydro calls).
 * pos: device n x 3 FP64 (the same positions as the last sfc_keys_sort);
 * m:   device n FP32 masses.  Errors: ESTATE without a preceding sort of n particles. */
int sphgrp_tree_build(sphgrp_ctx* ctx, int64_t n, const double* pos, const float* m,
                      cudaStream_t stream);

/* a4 + a5 (Sec. 1.1 and 2.1): neighbour sets of the active particles, exported as
 * CSR for inspection.  The hot path never materialises pair lists; this call exists
 * so that sets can be compared.
 * active:  device, n_act distinct original indices (any order).
 * h:       device, n FP64 smoothing lengths (all particles; hydro reads h_j too).
 * kind:    SPHGRP_DENSITY or SPHGRP_HYDRO.   mode: SPHGRP_INDIVIDUAL or SPHGRP_GROUPED.
 * group_size: members per group for the grouped form (1..256).
 * offsets: device, n_act + 1 int64; offsets[k]..offsets[k+1] index the neighbours of
 *          active[k] in idx (original indices, in no particular order).
 * idx:     device, cap int32, or NULL to count only.
 * n_pairs: host, receives the total number of pairs.
 * Errors: EOVERFLOW if the total exceeds cap (offsets still valid). */
int sphgrp_ngb_search(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, const double* h,
                      int kind, int mode, int group_size, int64_t cap, int64_t* offsets,
                      int32_t* idx, int64_t* n_pairs, cudaStream_t stream);

/* The candidate superset of every group of the grouped form (Sec. 2.1), for
 * inspection.  Groups are runs of consecutive active particles in key order: chunks
 * of group_size, each cut in halves while its members are spread wider than
 * params.group_split times their smallest h.
 * group_offsets: device, n_act + 1 int64 offsets of every group's candidates in cand;
 * group_first:   device, n_act + 1 int32 (may be NULL): group k's members are
 *                members[group_first[k] .. group_first[k+1]);
 * members:       device, n_act int32 (may be NULL): the active original indices in
 *                key order;
 * cand:          device, cap int32 original indices, or NULL to count only;
 * n_groups, n_cand: host, number of groups (walks) and total candidates.
 * kind selects the density or hydro radius. */
int sphgrp_group_supersets(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active,
                           const double* h, int kind, int group_size, int64_t cap,
                           int64_t* group_offsets, int32_t* group_first, int32_t* members,
                           int32_t* cand, int64_t* n_groups, int64_t* n_cand, cudaStream_t stream);

/* a6 + a7: SPH density of the active particles,
 *   rho_i = sum_{j in N_i} m_j W(r_ij, h_i),   dRho_i/dh_i,
 *   f_i = 1 / (1 + h_i / (3 rho_i) dRho_i/dh_i),  n_i = |N_i|,
 * with W the M4 cubic spline of support h.  With iterate != 0, h_i is iterated per
 * particle until |4 pi rho_i h_i^3 / (3 m_i) - nngb| <= nngb_tol (Sec. 2.2 relation
 * N_ngb = 4 pi rho h^3 / 3): Newton steps on that function inside a bracket, with a
 * volume bisection when a step leaves the bracket; each pass re-walks only the
 * unconverged particles, regrouped.
 * h:      device, n FP64; read for every particle, overwritten for active ones.
 * rho, drhodh, fgrad: device n FP32; nngb, iters: device n int32 (iters may be NULL).
 * Only entries of active particles are written.  Errors: ENOCONV if a particle did
 * not converge within max_iter passes (its last values are still written). */
int sphgrp_density(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, double* h,
                   int iterate, int mode, int group_size, float* rho, float* drhodh,
                   float* fgrad, int32_t* nngb, int32_t* iters, cudaStream_t stream);

/* a8: SPH hydro accelerations and du/dt of the active particles (Sec. 1.1 hydro
 * neighbour definition).  For j in the hydro set of i:
 *   a_i  -= m_j [ A_i dW(h_i) + A_j dW(h_j) + Pi_ij (dW(h_i) + dW(h_j))/2 ] r_ij / r
 *   du_i += m_j [ A_i dW(h_i) + Pi_ij (dW(h_i) + dW(h_j))/4 ] v_ij . r_ij / r
 * A_k = f_k P_k / rho_k^2, P = (gamma - 1) rho u, dW = dW/dr, Pi_ij the Monaghan
 * viscosity (alpha, beta, eps; zero for receding pairs).
 * h: device n FP64; rho, fgrad, u: device n FP32; vel: device n x 3 FP32 -- all
 * particles (neighbours may be inactive).  acc: device n x 3 FP32, dudt: device n FP32,
 * nngb: device n int32 (may be NULL); only active entries are written. */
int sphgrp_hydro_force(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active,
                       const double* h, const float* rho, const float* fgrad,
                       const float* vel, const float* u, int mode, int group_size,
                       float* acc, float* dudt, int32_t* nngb, cudaStream_t stream);

/* Velocity divergence and curl of the active particles over their density sets (the
 * a6 neighbour definition, support h_i), the inputs of the viscosity limiters used with
 * the Sec. 1.1 hydro loop.  The paper prints no formula for them; the standard SPH
 * estimates are taken:
 *   div v_i  = -(1/rho_i) sum_j m_j (v_i - v_j) . grad_i W(r_ij, h_i),
 *   curl v_i =  (1/rho_i) sum_j m_j (v_i - v_j) x grad_i W(r_ij, h_i),
 * grad_i W = dW/dr (x_i - x_j) / r, W the M4 spline of a6; pairs at r = 0 add nothing.
 * h: device n FP64 (0 < h < 0.5); rho: device n FP32 (> 0 for active particles);
 * vel: device n x 3 FP32 -- all particles.  divv: device n FP32, curlv: device n x 3
 * FP32; only active entries are written.  Grouped form only (mode is implied), group_size
 * in [1, 128].  Errors as sphgrp_hydro_force. */
int sphgrp_velocity_derivs(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active,
                           const double* h, const float* rho, const float* vel,
                           int group_size, float* divv, float* curlv, cudaStream_t stream);

/* a6 + a7 with the velocity derivatives of the call above accumulated in the same
 * density loop (the same staged candidates and the same neighbour decisions), instead
 * of a separate walk: as sphgrp_density (grouped form, walk passes in any iteration
 * mode), plus
 * vel:   device n x 3 FP32 velocities of all particles (read);
 * divv:  device n FP32, curlv: device n x 3 FP32 -- div v and curl v of the active
 *        particles at their final h, with the final rho (as sphgrp_velocity_derivs
 *        computes them from that h and rho).
 * Errors as sphgrp_density. */
int sphgrp_density_derivs(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active, double* h,
                          int iterate, int group_size, const float* vel, float* rho,
                          float* drhodh, float* fgrad, int32_t* nngb, int32_t* iters,
                          float* divv, float* curlv, cudaStream_t stream);

/* a8 with Balsara's limiter on the viscosity (Balsara 1995, as used with Gadget's SPH;
 * the paper names no limiter): every pair's Pi_ij is scaled by (fb_i + fb_j) / 2 with
 *   fb_i = |div v_i| / (|div v_i| + |curl v_i| + 1e-4 c_i / h_i),
 * c_i = sqrt(gamma (gamma - 1) u_i), formed on the device from
 * divv:  device n FP32, curlv: device n x 3 FP32 of all particles (e.g. from
 *        sphgrp_density_derivs or sphgrp_velocity_derivs).
 * Everything else as sphgrp_hydro_force (fb = 1 there).  EINVAL for NULL divv or curlv. */
int sphgrp_hydro_force_balsara(sphgrp_ctx* ctx, int64_t n_act, const int32_t* active,
                               const double* h, const float* rho, const float* fgrad,
                               const float* vel, const float* u, const float* divv,
                               const float* curlv, int mode, int group_size, float* acc,
                               float* dudt, int32_t* nngb, cudaStream_t stream);

/* a9: backward (adjoint) of the density and the hydro accelerations.  The paper has
 * no backward pass; this differentiates the a6 and a8 loops above.  For the positions
 * x and masses m of the last sphgrp_tree_build, and the given h, vel and u, it returns
 * the gradients with respect to x, v and m of
 *   L = sum_k g_acc_k . a_k + sum_k g_rho_k rho_k,
 * where rho_k is the density (a6) at h_k and a_k the hydro acceleration (a8) with
 * rho, f = 1 / (1 + h dRho/dh / (3 rho)), A = f (gamma - 1) u / rho and
 * c = sqrt(gamma (gamma - 1) u) taken from that density, and h_k(x, m) is the function
 * defined by (4 pi / 3) h_k^3 rho_k = nngb m_k (the Sec. 2.2 relation between h, rho
 * and the neighbour number, imposed exactly) through the given h: its dependence
 * enters by the implicit function theorem, including that of f through d2Rho/dh2.
 * The caller passes h satisfying the relation (e.g. sphgrp_density with a small
 * nngb_tol); for other h the result is the gradient of the relation's solution near h.
 * Neighbour sets are those of the given state, held fixed.  Every particle takes part
 * (there is no active list).  Grouped form only: the three pair loops (density sums,
 * hydro adjoint, density adjoint) walk the tree once per group each and recompute
 * every pair term from the staged candidates; no pair list is stored.
 * h:     device, n FP64, 0 < h < 0.5;
 * vel:   device, n x 3 FP32;  u: device, n FP32 (u >= 0);
 * g_acc: device, n x 3 FP32 (dL/da), or NULL for 0: then only the density term is
 *        differentiated, the hydro-adjoint loop is skipped and vel and u may be NULL;
 * g_rho: device, n FP32 (dL/drho), or NULL for 0 (not both NULL);
 * g_pos, g_vel: device, n x 3 FP32;  g_m: device, n FP32 -- outputs in original
 *        order, each may be NULL (not all three).
 * group_size in [1, 128].  The first call allocates 100 bytes per particle of n_max of
 * device workspace, kept by the context.  Errors as sphgrp_hydro_force; ESTATE
 * without a tree. */
int sphgrp_backward(sphgrp_ctx* ctx, const double* h, const float* vel, const float* u,
                    const float* g_acc, const float* g_rho, int group_size, float* g_pos,
                    float* g_vel, float* g_m, cudaStream_t stream);

/* a10: batched solve of many independent periodic boxes.  The paper treats one
 * simulation box; serving many small and large boxes at once is a deployment pattern
 * of the same method.  The boxes' particles are concatenated: box k holds the rows
 * [box_off[k], box_off[k+1]) of every per-particle array, positions in its own unit
 * cube.  One call runs, for all boxes together:
 *   keys + a stable sort by (box, key); a forest of one octree per box; grouping of
 *   every box's active particles (groups never cross a box); the density with the
 *   smoothing-length iteration (Sec. 2.2) inside one persistent work-queue kernel
 *   over every box's groups (each group iterates its members until they converge;
 *   no host loop); the hydro forces in a second persistent kernel; and, with
 *   SPHGRP_BATCH_BACKWARD, the adjoint of sphgrp_backward over every particle of every
 *   box (its hydro-adjoint items share the hydro kernel's work queue).
 * Every count stays on the device, so the whole call can be captured in one CUDA graph
 * (SPHGRP_BATCH_GRAPH: captured on a private stream by the first call, replayed by the
 * following calls with the same io pointers and flags, re-captured otherwise).
 * Per box, the group size, the slice limit (member copies per warp that split a
 * candidate tile) and the group split factor come from the box's class (box_class,
 * e.g. 0 = uniform, 1 = clustered); sphgrp_batch_tune picks them per class by timing. */
#define SPHGRP_BATCH_CLASSES 8
enum {
    SPHGRP_BATCH_BACKWARD = 1, /* also compute g_pos, g_vel, g_m */
    SPHGRP_BATCH_GRAPH = 2     /* capture / replay the call as a CUDA graph */
};

typedef struct sphgrp_batch sphgrp_batch;

/* Per-particle arrays of a batch call: device pointers, n_total rows (the sum of the
 * box sizes), original (concatenated) order. */
typedef struct sphgrp_batch_io {
    const double* pos;      /* n x 3 FP64 in [0,1) of the particle's box */
    const float* m;         /* masses */
    const float* vel;       /* n x 3 */
    const float* u;         /* specific internal energy, >= 0 */
    double* h;              /* in: smoothing lengths (first guess for active particles);
                               out: converged h of the active particles */
    const uint8_t* active;  /* nonzero = active, or NULL: every particle active */
    float* rho;             /* in/out: density (inactive entries are inputs to the hydro) */
    float* drhodh;          /* out (active) */
    float* fgrad;           /* in/out, as rho */
    int32_t* nngb;          /* out (active): neighbour count */
    float* acc;             /* out (active): n x 3 hydro accelerations */
    float* dudt;            /* out (active) */
    const float* g_acc;     /* backward: n x 3 dL/da (every particle) */
    const float* g_rho;     /* backward: n dL/drho, or NULL */
    float* g_pos;           /* backward outputs (each may be NULL, not all three) */
    float* g_vel;
    float* g_m;
} sphgrp_batch_io;

/* box_off: host, nbox + 1 ascending offsets, box_off[0] = 0, every box non-empty,
 * box_off[nbox] <= 2^30; box_class: host, nbox classes in [0, SPHGRP_BATCH_CLASSES),
 * or NULL (all class 0).  Allocates the device workspace for box_off[nbox] particles
 * (about 0.5 KB per particle with the backward buffers). */
int sphgrp_batch_create(sphgrp_batch** out, const sphgrp_params* params, int nbox,
                        const int64_t* box_off, const int32_t* box_class);
int sphgrp_batch_destroy(sphgrp_batch* b);

/* One batched step (see above).  flags: SPHGRP_BATCH_BACKWARD | SPHGRP_BATCH_GRAPH.
 * Synchronises the stream to read the device-side status.  Errors: EINVAL (a position
 * or h out of range), ENOCONV (a particle did not converge within max_iter passes;
 * its last values are written), EOVERFLOW (forest capacity or walk stack; results
 * invalid), ETIMEOUT, ECUDA. */
int sphgrp_batch_run(sphgrp_batch* b, const sphgrp_batch_io* io, int flags, cudaStream_t stream);

/* Autotuner: runs one step (updating io like sphgrp_batch_run), then for every class
 * present times a density + hydro pass over that class's boxes for every candidate
 * (group size 4..64, slice limit, split factor) and keeps the fastest; then, at that
 * grouping, the octree leaf size of the class's boxes (the context's, 8, 12, 24, 32;
 * each candidate rebuilds the forest before its timed pass).  Drops the captured
 * graph. */
int sphgrp_batch_tune(sphgrp_batch* b, const sphgrp_batch_io* io, cudaStream_t stream);

/* Read / set the configuration of one class (group_size in [1, 128], max_slices in
 * {1, 2, 4}, group_split >= 0; 0 = no splitting; leaf_size: octree leaf bucket of the
 * class's boxes, 0 = the context's params.leaf_size, else in [8, 255]).  Setting drops
 * the captured graph.  pass_ms / pass_members (host, may be NULL) receive the
 * autotuner's best time of one density + hydro pass over the class's active particles
 * and their count (0 when the class was not tuned): the class's own throughput. */
int sphgrp_batch_get_config(sphgrp_batch* b, int cls, int* group_size, int* max_slices,
                            double* group_split, int* leaf_size, double* pass_ms, int64_t* pass_members);
int sphgrp_batch_set_config(sphgrp_batch* b, int cls, int group_size, int max_slices,
                            double group_split, int leaf_size);

/* Counters of the last sphgrp_batch_run (no device work): walks and members summed
 * over its grouped launches (density, hydro, and the backward's three), candidates,
 * pair tests, pairs, FP64 re-tests and nodes tested over all of them, the deepest walk
 * stack, search_launches = kernels the call launched (graph nodes when replayed), and
 * iterations = 1 when the call replayed a captured graph, else 0. */
int sphgrp_batch_stats(sphgrp_batch* b, sphgrp_stats* out);

/* Counters of the most recent search, density or hydro call. */
int sphgrp_get_stats(sphgrp_ctx* ctx, sphgrp_stats* out);

/* Per-launch record of the search kernels of the most recent call, in launch order
 * (one entry per smoothing-length pass for sphgrp_density): particles processed,
 * candidates staged, member x candidate tests, node tests and device time in ms
 * (CUDA events).  All arrays are host arrays of cap entries and may be NULL;
 * count receives the number of entries written.  No device work. */
int sphgrp_get_launch_log(sphgrp_ctx* ctx, int cap, int64_t* members, int64_t* candidates,
                          int64_t* pair_tests, int64_t* nodes, double* ms, int* count);

/* f3: domain decomposition with halo import.  The paper splits the particles along
 * the Hilbert curve into one contiguous key range per process (Sec. 1.2) and finds
 * neighbours across ranges by exporting particles in a second search phase (Sec. 1.1).
 * Here each rank (one GPU) imports, before its search, the particles of the other ranks
 * its own particles can reach (the halo), and then searches locally.  These are the
 * per-rank device steps; paper_1810_09898_gb300.domain runs the exchanges.
 *
 * sphgrp_key_split: after sphgrp_sfc_keys_sort of the rank's particles, dest[i] (device,
 * n uint64, caller order) = 1 << (the rank owning particle i's key), that rank being the
 * number of splitters <= key (device, nsplit uint64 ascending, nsplit <= 63).  ESTATE
 * without the sort. */
int sphgrp_key_split(sphgrp_ctx* ctx, int nsplit, const uint64_t* splitters, uint64_t* dest,
                     cudaStream_t stream);

/* sphgrp_domain_boxes: after sphgrp_tree_build of the rank's particles, the tight boxes
 * of its particles in every octree cell of depth `level` (0 .. 21) they occupy, in key
 * order: boxes (device, cap x 8 FP64) = {lo x, y, z, hi x, y, z, hmax, count} with
 * lo <= x < hi (box units) and hmax >= the largest h (device n FP64, caller order) in the
 * box; *nbox (host) receives the number of boxes.  EOVERFLOW if more than cap boxes (or
 * more than n_max / 2); ESTATE without a tree.  Synchronises the stream. */
int sphgrp_domain_boxes(sphgrp_ctx* ctx, const double* h, int level, int cap, double* boxes,
                        int* nbox, cudaStream_t stream);

/* sphgrp_halo_select: for every particle j of the rank (device n FP64 h, caller order),
 * the ranks that must import it: bit r of mask[j] (device n uint64) is set iff r !=
 * self_rank and j lies within reach of one of rank r's boxes (box_rank, device nbox
 * int32, gives each box's rank; boxes as sphgrp_domain_boxes wrote them, all ranks'
 * concatenated): periodic distance to the box below widen * hmax (density: j is a
 * neighbour of i iff |x_j - x_i| < h_i) or below max(widen * hmax, h_j) (hydro: iff
 * below max(h_i, h_j)).  widen in [1, 4] covers the growth of h in a later
 * smoothing-length iteration.  counts (device, world int64) = particles per rank.
 * world <= 64.  The call synchronises the stream to read back the check of box_rank:
 * a rank outside [0, world) is skipped and reported as EINVAL (the mask then leaves
 * that box out).  Errors: EINVAL, ESTATE without a tree. */
int sphgrp_halo_select(sphgrp_ctx* ctx, const double* h, int kind, double widen, int nbox,
                       const double* boxes, const int32_t* box_rank, int self_rank, int world,
                       uint64_t* mask, int64_t* counts, cudaStream_t stream);

/* sphgrp_mask_compact: the entries (ascending) with bit `bit` of mask (device n uint64,
 * 1 <= n <= n_max; the context only lends its scan workspace) set, to idx (device, n
 * int32); *count (host) receives how many.  Synchronises the stream. */
int sphgrp_mask_compact(sphgrp_ctx* ctx, int64_t n, const uint64_t* mask, int bit, int32_t* idx,
                        int64_t* count, cudaStream_t stream);

/* Keys + stable sort (as sphgrp_sfc_keys_sort) without any device allocation, for
 * callers that may not call cudaMalloc / cudaFree: plug-ins whose host application
 * owns all device memory through its own pool, and latency-critical paths that cannot
 * take the implicit device synchronisation of an allocation.  The paper has no
 * counterpart; this is a deployment variant of the a1 + a2 step.
 * The sort's scratch lives in one fixed-size __device__ array inside the library
 * (about 6.3 MB, held on every GPU that loads the library until the process exits),
 * so n may not exceed SPHGRP_STATIC_SORT_MAX_N (EINVAL otherwise).
 * pos:      device, n x 3 FP64 in [0,1).
 * keys_out: device, n uint64, receives the sorted keys (also used as sort scratch).
 * perm_out: device, n int32, receives rank -> original index (also used as scratch).
 * No context is involved and nothing is kept for later calls.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for the life of the process: this assumes one primary context
 * per device for that time (do not call it after a cudaDeviceReset of the device).
 * All calls share the one array: calls whose work overlaps on the GPU (different
 * streams, or different host threads without ordering) race and give wrong results;
 * serialise them.  Every call synchronises the stream to read back the range check, so
 * it must never be called while its stream is being captured into a graph. */
#define SPHGRP_STATIC_SORT_MAX_N (1 << 19)
int sphgrp_sfc_keys_sort_static(int64_t n, const double* pos, uint64_t* keys_out,
                                int32_t* perm_out, cudaStream_t stream);

/* Number of CUDA kernels the library has launched in this process so far (all
 * contexts, all threads).  Diagnostics only; no device work. */
int sphgrp_kernel_launches(int64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* SPHGRP_H */
