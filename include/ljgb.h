/*
 * ljgb.h -- C ABI of the GB300 (sm_103a) Lennard-Jones short-range force library.
 *
 * The library computes the hot path of "Tuning of Vectorization Parameters
 * for Molecular Dynamics Simulations in AutoPas" (arXiv 2512.03565):
 *   - the pairwise force sum F_i = sum_j F_ij (Sec. 2.1, Eq. 1) over pairs
 *     within the cutoff (Sec. 2.1), Lennard-Jones 12-6 (named in Sec. 4.1;
 *     textbook form U = 4 eps [(sigma/r)^12 - (sigma/r)^6], truncated);
 *   - neighbour identification by Linked Cells (cells of edge >= r_c, or
 *     sub-cells of edge >= r_c/2), by Verlet lists with a skin and by Verlet
 *     cluster lists (Sec. 2.1.1);
 *   - the interaction order, i.e. which particles of the two lists a functor
 *     holds against which (Sec. 4.1, Fig. 4: 1/V, V/1, 2/V2, V2/2), as GPU
 *     orders chosen at run time; Newton's third law on or off (Sec. 4.1.3);
 *   - the full-search auto-tuner over the Cartesian product of configurations
 *     (Sec. 2.3.2), by run time or by energy (Sec. 2.3.3), and a learned tuner
 *     (the data-driven tuning of Sec. 6) trained by the library's own kernels;
 *   - velocity-Verlet time integration (Sec. 2.1), for one box or for a batch
 *     of independent boxes in one persistent launch (lj_ensemble_*).
 *
 * Conventions for every entry point:
 *   - Status codes only: nothing throws, exits or aborts across the ABI.
 *     LJ_ERR_* codes are listed below; lj_last_error() gives a message.
 *   - Geometry: a cubic periodic box of edge L.  Positions are stored as 32-bit
 *     fixed point per axis, x = x_fp * u with u = L / 2^32; the minimum image of
 *     a difference is the wrapping 32-bit difference read as signed.  A pair
 *     interacts iff 0 < R^2 <= floor((r_c/u)^2), R^2 the exact integer sum of
 *     squared fixed-point differences (pairs at zero separation are excluded).
 *   - Arrays are SoA with 3*n entries: x[0..n), y[0..n), z[0..n).  Arrays
 *     passed in are borrowed for the duration of the call only.
 *     on_device = 1 means a CUDA device pointer (e.g. a torch tensor's
 *     data_ptr()), 0 a host pointer (pinned or pageable).
 *   - Ownership: the library owns all of its device state; lj_destroy frees it.
 *   - Streams: all work is issued on the stream given at lj_init_domain (NULL =
 *     the legacy default stream).  Calls that return host values synchronise
 *     that stream.
 *   - Ordering: forces, positions and velocities are returned in the caller's
 *     original particle order.
 *   - Units: reduced LJ units (eps, sigma, mass as given).
 *   - Threading: one context must not be used from two host threads at once.
 */
#ifndef LJGB_H
#define LJGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lj_ctx lj_ctx;

typedef enum {
  LJ_OK = 0,
  LJ_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, bad config) */
  LJ_ERR_CUDA = 2,       /* a CUDA runtime call failed; in the index-check build (LJGB_CHECKS=1)
                            also a kernel that met an index outside its array (lj_last_error:
                            "device index check failed"); it skipped that access */
  LJ_ERR_CAPACITY = 3,   /* a Verlet list overflowed its capacity (the library regrows and rebuilds) */
  LJ_ERR_SKIN = 4,       /* a particle moved more than skin/2 since the last list build */
  LJ_ERR_NONFINITE = 5,  /* a force, energy or virial was NaN or infinite */
  LJ_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up */
  LJ_ERR_STATE = 7,      /* call out of order (e.g. forces before particles) */
  LJ_ERR_OOM = 8         /* device allocation failed */
} lj_status;

typedef enum { LJ_PREC_FP64 = 0, LJ_PREC_FP32_ACC64 = 1 } lj_precision;

/* Neighbour identification (Sec. 2.1.1): linked cells of edge >= r_c, rebinned
 * at every force evaluation; Verlet lists built on cells of edge >= r_c + skin;
 * Verlet cluster lists: clusters of M particles (M = 4, 6 or 8, the cluster
 * sizes of Sec. 5.1) with lists of whole neighbour clusters within r_c + skin
 * (see lj_build_clusters).  Both list containers are rebuilt every few steps
 * and whenever a particle has moved more than skin/2 since the build.
 * LJ_LCS is linked cells of edge >= r_c / 2 (sub-cells; the paper's cells of
 * edge = cutoff are its special case of edge r_c): a particle visits the
 * 5 x 5 x 5 cells around its own, which hold a quarter of the 27-cell
 * candidates' volume, so about twice the fraction of candidates lies inside
 * r_c.  It needs at least 5 cells per axis and runs the JSPLIT order only. */
typedef enum { LJ_LC = 0, LJ_VL = 1, LJ_VCL = 2, LJ_LCS = 3 } lj_container;

/* Interaction orders: the GPU analogues of the paper's register-filling
 * patterns (Sec. 4.1.1, Fig. 4).
 *   LJ_ORD_IPT_SMEM  one i per lane, the j tile staged in shared memory and
 *                    broadcast to the warp (V/1: V i's against one j).
 *   LJ_ORD_IPT_TMA   as IPT_SMEM, the j tile brought in by bulk asynchronous
 *                    copies (cp.async.bulk) on an mbarrier double buffer.
 *   LJ_ORD_KI        k i's per lane (param = k in {2,4}): one j load serves k pairs.
 *   LJ_ORD_JSPLIT    w lanes per i striding over the j list, shuffle reduction
 *                    of the i force (param = w in {32,16,8,4,2}): 1/V for
 *                    w=32, 2/V2 for w=16, V2/2 for w=2.
 *   LJ_ORD_ROT32     one i and one j per lane, j rotated through the warp by
 *                    shuffles: a full 32 x 32 tile (the "full/rotated" order).
 *   LJ_ORD_VL_IPT    Verlet lists only: one i per lane, gathering its list.
 *   LJ_ORD_CL_TILE   cluster lists only (param = cluster size M): lane =
 *                    (i of the base cluster, j-slot), 32/M j's per pass from
 *                    one or more neighbour clusters.
 *   LJ_ORD_CL_JLANE  cluster lists only (param = M): one j per lane (32 per
 *                    pass), the M base-cluster i's held in every lane. */
typedef enum {
  LJ_ORD_IPT_SMEM = 0,
  LJ_ORD_IPT_TMA = 1,
  LJ_ORD_KI = 2,
  LJ_ORD_JSPLIT = 3,
  LJ_ORD_ROT32 = 4,
  LJ_ORD_VL_IPT = 5,
  LJ_ORD_CL_TILE = 6,
  LJ_ORD_CL_JLANE = 7
} lj_order;

/* Newton's third law (Sec. 2.1, Sec. 4.1.3): off (every pair evaluated from
 * both sides), on with the j contribution scattered by atomics, or on with a
 * deterministic two-pass reduction (j partials written to a buffer, then
 * gathered per particle in a fixed order; Verlet lists, VL_IPT only).  With
 * FP32 pair arithmetic the atomic scatter is one 16-byte FP32 vector
 * reduction per contribution into the particle's FP32 partial sum (performed
 * in L2; its order of summation, and so the last bits of the result, vary
 * between runs), folded once per particle into the FP64 force; with FP64 pair
 * arithmetic it is FP64 atomics on the force itself.
 * LJ_N3_ATOMIC_BWD (linked cells only) is LJ_N3_ATOMIC with the roles of the
 * two cells of every cell pair swapped: each i visits the backward half shell
 * (the neighbour cells before its own in cell order) instead of the forward
 * one.  The pair set is the same; which particles are loaded as i's and which
 * receive the scattered j forces differs (the domain-traversal dimension of
 * Sec. 5.1, where the two orders of a cell pair run at different speeds). */
typedef enum { LJ_N3_OFF = 0, LJ_N3_ATOMIC = 1, LJ_N3_TWOPASS = 2, LJ_N3_ATOMIC_BWD = 3 } lj_newton3;

typedef struct {
  int32_t container; /* lj_container */
  int32_t order;     /* lj_order */
  int32_t param;     /* k for LJ_ORD_KI, w for LJ_ORD_JSPLIT, else 0 */
  int32_t newton3;   /* lj_newton3 */
} lj_config;

/* Create a context for a cubic periodic box.  box[0..2] must be equal (cubic);
 * cutoff > 0, skin >= 0, cutoff + skin < L/2, eps > 0, sigma > 0.
 * cuda_stream: a cudaStream_t (may be NULL).  *out receives the context.
 * Errors: LJ_ERR_ARG, LJ_ERR_CUDA. */
lj_status lj_init_domain(lj_ctx** out, const double box[3], double cutoff, double skin,
                         double eps, double sigma, lj_precision prec, void* cuda_stream);

/* Load n particles.  pos: 3*n doubles (SoA), quantised to fixed point as
 * x_fp = floor(x/L * 2^32) mod 2^32.  vel: 3*n doubles or NULL (zero).
 * Copies in on the context's stream (host arrays through a device staging
 * buffer; a pinned host array must not change until the stream has passed the
 * copy); previous particles are replaced.  Errors: LJ_ERR_ARG (n < 1, null
 * pos), LJ_ERR_OOM, LJ_ERR_CUDA. */
lj_status lj_set_particles(lj_ctx* ctx, int64_t n, const double* pos, const double* vel,
                           double mass, int on_device);

/* As lj_set_particles with positions already in fixed point (3*n uint32). */
lj_status lj_set_particles_fp(lj_ctx* ctx, int64_t n, const uint32_t* pos_fp, const double* vel,
                              double mass, int on_device);

/* New positions for the loaded particles (caller's order, n as loaded,
 * float64 [3][n], host or device), velocities kept.  Unlike lj_set_particles
 * the cell (or cluster) order and the Verlet (or cluster) lists are kept: the next force evaluation
 * reuses the lists while every particle stays within skin/2 of its position
 * at the last build and rebuilds them otherwise (Sec. 2.1.1: lists are kept
 * over several steps thanks to the skin); linked cells are rebinned.  This
 * is the call of a host-driven time loop.  A pending closing kick (see
 * lj_integrate_step) is applied first.  Errors: LJ_ERR_ARG, LJ_ERR_STATE (no
 * particles loaded), LJ_ERR_CUDA. */
lj_status lj_update_positions(lj_ctx* ctx, const double* pos, int32_t on_device);

/* Bin the particles into the cells of one container by a stable counting sort
 * on the cell id (Sec. 2.1.1, Linked Cells): cells of edge >= r_c (LJ_LC),
 * >= r_c / 2 (LJ_LCS) or >= r_c + skin (LJ_VL), n_c = floor(L / edge) per
 * axis, at least 3 (5 for LJ_LCS).  The
 * library's particle storage is reordered to cell order (ties keep ascending
 * original index).  Errors: LJ_ERR_STATE, LJ_ERR_ARG (too few cells), LJ_ERR_CUDA. */
lj_status lj_bin_cells(lj_ctx* ctx, int32_t container);

/* Build Verlet lists (Sec. 2.1.1) on the r_c + skin cells: every j != i within
 * r_c + skin (half_list = 1: only j after i in cell order, for Newton3).
 * Bins first.  Grows the list capacity and rebuilds on overflow. */
lj_status lj_build_verlet(lj_ctx* ctx, int32_t half_list);

/* Build Verlet cluster lists (Sec. 2.1.1, the cluster container; cluster size
 * M in {4, 6, 8}, Sec. 5.1).  The particle storage is reordered into cluster
 * order: n_t x n_t towers over (x, y), n_t the largest k >= 1 with
 * k^3 M <= n; tower of a particle (floor(x_fp n_t / 2^32), floor(y_fp n_t /
 * 2^32)); storage by tower id cx n_t + cy, then z_fp, then original index.
 * Each tower's run is cut into clusters of M consecutive particles (the last
 * one shorter).  Clusters I and J are neighbours iff some member pair (two
 * different particles, one of each) lies within r_c + skin by the exact
 * integer rule; the search prunes by the clusters' boxes (min/max of their
 * fixed-point coordinates) and records each listed pair's member mask
 * (lj_get_cluster_masks).  Full lists hold every neighbour J (I itself when
 * two of its members are within range); half lists (half_list = 1, for
 * Newton-3) only J >= I, with the pairs of I itself counted once.  Grows the
 * list capacity and rebuilds on overflow.
 * Errors: LJ_ERR_ARG (M not 4, 6 or 8; n >= 2^29), LJ_ERR_STATE,
 * LJ_ERR_CAPACITY, LJ_ERR_OOM, LJ_ERR_CUDA. */
lj_status lj_build_clusters(lj_ctx* ctx, int32_t M, int32_t half_list);

/* The current cluster order (after lj_build_clusters or a force evaluation on
 * LJ_VCL): *ncl receives the number of clusters, cl_start (ncl + 1 entries,
 * host, may be NULL) the first storage slot of each cluster and n at the end
 * (lj_get_cells gives perm), *ntower (may be NULL) n_t.  Errors: LJ_ERR_STATE
 * if no cluster order is current. */
lj_status lj_get_clusters(lj_ctx* ctx, int64_t* ncl, uint32_t* cl_start, int32_t* ntower);

/* The cluster-pair lists: nn[ncl] their lengths and nbr[ncl][cap] (row-major,
 * host) the neighbour cluster indices in the library's search order (the set
 * is defined; the order is not); *cap_out the capacity.  Either array may be
 * NULL.  Errors: LJ_ERR_STATE if no cluster list is current. */
lj_status lj_get_cluster_lists(lj_ctx* ctx, int32_t* nbr, int32_t* nn, int32_t* cap_out);

/* The member masks of the cluster-pair lists (Sec. 2.1.1, Verlet cluster
 * lists; the paper gives no bit layout, this one is the library's): masks
 * (host, [ncl][cap] uint64, row-major, in the order of lj_get_cluster_lists'
 * entries, 0 beyond a list's length).  Bit a * M + b of an entry (I, J) is set
 * iff the a-th particle of cluster I and the b-th of J (in cluster order, M
 * the cluster size) are two different particles within r_c + skin, for a
 * half list's entry J = I only with b > a.  A cluster pair is listed iff its
 * mask is not empty; the force kernels take exactly the pairs of set bits.
 * Errors: LJ_ERR_ARG (null), LJ_ERR_STATE if no cluster list is current. */
lj_status lj_get_cluster_masks(lj_ctx* ctx, uint64_t* masks);

/* One force evaluation F_i = sum_j F_ij (Eq. 1) with the given configuration.
 * LC rebins; VL and VCL build their lists when they are stale (never built,
 * other half mode or cluster size, or a particle moved more than skin/2).  energy_out / virial_out (host,
 * may be NULL) receive U = sum_pairs U(r) and W = sum_pairs r . F_ij.
 * Forces stay on the device (lj_get_forces).  Errors: LJ_ERR_ARG (invalid
 * configuration; see lj_config_valid), LJ_ERR_STATE, LJ_ERR_NONFINITE, LJ_ERR_CUDA. */
lj_status lj_compute_forces(lj_ctx* ctx, lj_config cfg, double* energy_out, double* virial_out);

/* 1 if cfg is a valid configuration, else 0. */
int32_t lj_config_valid(lj_config cfg);

/* The valid configurations in a fixed order.  Writes up to cap entries to out
 * (may be NULL) and returns the total count. */
int32_t lj_config_list(lj_config* out, int32_t cap);

/* nsteps of velocity Verlet (Sec. 2.1): v += dt/(2m) F; x += v dt (fixed
 * point, rounded to nearest, periodic wrap); F = F(x) with cfg; v += dt/(2m) F.
 * Verlet and cluster lists are rebuilt every rebuild_every steps (and early
 * when a particle moved more than skin/2).  Computes the initial forces if none are current.
 * The last step's closing half kick is kept pending on the device and applied
 * by the next call's first kick (as a separate FMA, so the arithmetic is that
 * of unfused kicks), or first thing by lj_get_state, lj_kinetic_energy and any
 * force evaluation; lj_set_particles drops it.  Errors: as lj_compute_forces. */
lj_status lj_integrate_step(lj_ctx* ctx, double dt, int32_t nsteps, int32_t rebuild_every,
                            lj_config cfg);

/* Tuning (Sec. 2.3.2).  kind 0 = full search: every valid configuration is
 * timed over `samples` force evaluations (CUDA events) and reduced by the
 * mean; the fastest is returned in *chosen.  kind 1 = learned: the tuner
 * network (loaded by lj_tuner_set_model) ranks the configurations from the
 * features (lj_features) and the best predicted one is returned, confirmed by
 * timing the top `samples` candidates (0 = no timing).  Without a model, kind 1
 * falls back to the full search.  times_ms (host, may be NULL) receives the
 * measured mean time of each configuration in lj_config_list order (NaN when
 * not timed).  Errors: LJ_ERR_STATE, LJ_ERR_ARG, LJ_ERR_CUDA. */
lj_status lj_tune(lj_ctx* ctx, int32_t kind, int32_t samples, lj_config* chosen, double* times_ms);

/* Energy as the tuning metric (Sec. 2.3.3; Sec. 5.2 reports that the energy-
 * and runtime-optimal orders can differ).  The source is the GPU's total-energy
 * counter, read through NVML (loaded at run time; read-only calls).
 *
 * lj_energy_read: *mj = the counter of CUDA device `device` (-1 = current) in
 * millijoules since the driver loaded.
 *
 * lj_energy_period: polls the counter until it has updated 5 times or probe_ms
 * has passed, and returns in *period_ms the median interval between
 * consecutive updates (the one interval seen when only 2 updates came; NaN when
 * fewer than 2 did).  A probe_ms of at least 10 counter periods (about 1 s on
 * GB300) makes the NaN case mean a counter that is not updating.
 *
 * lj_tune_energy: full search by energy.  Every valid configuration runs a
 * warm-up evaluation, then a batch of force evaluations lasting at least
 * min_ms (Verlet lists rebuilt every rebuild period, linked cells rebinned per
 * evaluation, as in lj_tune's cost).  The energy per evaluation is the average
 * power between two counter updates inside the batch (a host thread records
 * them) times the time per evaluation.  time_ms and energy_mj (host, may be
 * NULL, lj_config_list order, NaN when not measured) receive both, and *chosen
 * the configuration of least energy.  min_ms should span at least 3 counter
 * periods; with fewer, energies are NaN and LJ_ERR_STATE is returned if none
 * was measured.
 *
 * Errors: LJ_ERR_STATE when NVML or the counter is not available, LJ_ERR_CUDA,
 * LJ_ERR_ARG; lj_tune_energy also those of lj_compute_forces. */
lj_status lj_energy_read(int32_t device, double* mj);
lj_status lj_energy_period(int32_t device, double probe_ms, double* period_ms);
lj_status lj_tune_energy(lj_ctx* ctx, double min_ms, lj_config* chosen, double* time_ms, double* energy_mj);

/* Full-search selection rule alone (host, no GPU): given `samples` timings per
 * configuration (row-major [n_cfg][samples], NaN = missing) and a validity
 * mask, reduce each row (reduce 0 = mean, 1 = minimum) and return the index
 * of the smallest, or -1 if none is valid. */
int32_t lj_tune_select(const double* timings, int32_t n_cfg, int32_t samples, const int32_t* valid,
                       int32_t reduce);

/* The 16 tuner features of the current particles (host out[16]): log density,
 * log N, mean/std occupancy of the r_c cells, fraction of empty cells, an
 * 8-bin occupancy histogram (0, 1-2, 3-4, 5-8, 9-16, 17-32, 33-64, >64),
 * homogeneity (std/mean over 4x4x4 coarse blocks), r_c / cell edge and the
 * expected Verlet-list length.  Integer statistics are gathered on the device. */
lj_status lj_features(lj_ctx* ctx, double* out16);

/* Load the learned tuner: an MLP 16-64-64-C (tanh, tanh, linear) with
 * parameters in the layout W1[64][16] b1[64] W2[64][64] b2[64] W3[C][64]
 * b3[C] (host, FP32), feature standardisation mean[16] and std[16], and the
 * C configurations its outputs stand for.  The network predicts log time. */
lj_status lj_tuner_set_model(lj_ctx* ctx, const float* params, int32_t C, const float* feat_mean,
                             const float* feat_std, const lj_config* cfgs);

/* The tuner network on the GPU (hand-written FP32 kernels; no counterpart
 * code in the paper, which proposes data-driven tuning in Sec. 6).  All arrays
 * are host pointers; each call copies in, runs on the GPU and copies out.
 * params: the MLP 16-64-64-C parameters (layout as in lj_tuner_set_model).
 * X: M rows of 16 standardised features; T: M x C target log times;
 * mask: M x C weights (1 = measured, 0 = missing).  Loss: sum mask (y - T)^2
 * / sum mask.  stream: a cudaStream_t or NULL (lj_mlp_train uses a stream of
 * its own and replays one captured epoch as a CUDA graph).
 * Errors: LJ_ERR_ARG, LJ_ERR_OOM, LJ_ERR_CUDA. */
lj_status lj_mlp_forward(const float* params, int32_t C, const float* X, int64_t M, float* Y, void* stream);
lj_status lj_mlp_loss_grad(const float* params, int32_t C, const float* X, const float* T, const float* mask,
                           int64_t M, float* grad, float* loss, void* stream);
/* Full-batch Adam (lr, betas 0.9/0.999, eps 1e-8) for `epochs` steps; params
 * updated in place; losses (may be NULL) receives epochs + 1 values: the loss
 * before each step and after the last. */
lj_status lj_mlp_train(const float* X, const float* T, const float* mask, int64_t M, int32_t C, float* params,
                       int32_t epochs, float lr, float* losses, void* stream);

/* The training inputs of the learned tuner, computed on the GPU from the
 * full-search timings and the features (data-driven tuning, Sec. 6; no
 * counterpart code in the paper).  T: M x C timings (host, row-major,
 * double; NaN or a non-positive value = not timed); X: M x 16 features
 * (host, double).  Outputs (host, float): Y[M][C] = log(t / t_best) of each
 * row's valid entries (0 elsewhere), mask[M][C] = 1 where valid, and the
 * standardised features Xs[M][16] = (X - mean) / std with the columns' mean[16]
 * and population standard deviation std[16] (a deviation below 1e-12 becomes
 * 1).  Synchronises stream (a cudaStream_t or NULL).  Errors: LJ_ERR_ARG,
 * LJ_ERR_OOM, LJ_ERR_CUDA. */
lj_status lj_tuner_prepare(const double* T, int64_t M, int32_t C, const double* X, float* Y, float* mask, float* Xs,
                           float* mean, float* std, void* stream);

/* Copy out forces (3*n doubles, original order).  Synchronises if on_device = 0. */
lj_status lj_get_forces(lj_ctx* ctx, double* dst, int32_t on_device);

/* Copy out positions (fixed point, 3*n uint32) and velocities (3*n doubles),
 * original order; either pointer may be NULL. */
lj_status lj_get_state(lj_ctx* ctx, uint32_t* pos_fp, double* vel, int32_t on_device);

/* The pair set of a container, as original-index pairs (i < j) sorted
 * lexicographically: LJ_LC = pairs within r_c found by the linked-cell scan;
 * LJ_VL = the entries of the Verlet lists (pairs within r_c + skin);
 * LJ_VCL = the member pairs of the listed cluster pairs that lie within
 * r_c + skin (exact integer test), so equal to the LJ_VL set.  With
 * ij == NULL only *n_pairs is set (size query); otherwise ij must hold
 * 2 * (*n_pairs) int32 on the host. */
lj_status lj_get_pairs(lj_ctx* ctx, int32_t container, int64_t* n_pairs, int32_t* ij);

/* The current cell order: perm[k] = original index of the k-th particle
 * (n entries) and cell_start (n_c^3 + 1 entries, n_c of the last binning;
 * after a cluster build the cells are the towers' z-slabs, id (cx n_t + cy)
 * n_t + cz, and n_c = n_t).
 * Host pointers; either may be NULL.  *nc_out (may be NULL) gets n_c. */
lj_status lj_get_cells(lj_ctx* ctx, uint32_t* perm, uint32_t* cell_start, int32_t* nc_out);

/* Verlet lists in cell order: nnbr[n] and the entries nbr[n][cap] (row-major,
 * sorted j indices in the Sec. 2.1.1 scan order), host pointers; *cap_out
 * receives the capacity.  Errors: LJ_ERR_STATE if no list was built. */
lj_status lj_get_verlet(lj_ctx* ctx, int32_t* nbr, int32_t* nnbr, int32_t* cap_out);

/* Counters since the context was created: cnt[0] = force evaluations,
 * cnt[1] = unique in-cutoff pairs of the last evaluation, cnt[2] = list builds,
 * cnt[3] = early (skin) rebuilds, cnt[4] = capacity regrowths.  In
 * lj_integrate_step the force of a step without a scheduled rebuild starts
 * before the skin check is read back; a step that then needs an early rebuild
 * evaluates the forces twice and cnt[0] counts both. */
lj_status lj_get_counters(lj_ctx* ctx, int64_t* cnt5);

/* Force-kernel timing with CUDA events recorded on the context's stream
 * around every force-kernel launch (the pair kernel and, for the two-pass
 * Newton-3 variant, its gather; not the binning or list build).  enable = 1
 * clears and starts recording, 0 stops.  force_ms / launches (may be NULL)
 * receive the summed event time and the number of timed evaluations since the
 * last enable; total_launches (may be NULL) receives the number of kernels this
 * context has launched.  Synchronises the stream. */
lj_status lj_timing(lj_ctx* ctx, int32_t enable, double* force_ms, int64_t* launches,
                    int64_t* total_launches);

/* Kinetic energy 1/2 m sum v^2 of the current state (host out). */
lj_status lj_kinetic_energy(lj_ctx* ctx, double* ke);

/* ------------------------------------------------------------------------
 * Ensembles: many independent periodic boxes of uneven sizes advanced together
 * by one persistent kernel launch (cooperative, all blocks resident), captured
 * as a CUDA graph and replayed.  Each box runs velocity Verlet (Sec. 2.1) with
 * linked-cell forces (Sec. 2.1.1; cells of edge >= cutoff rebinned every
 * step, boxes with fewer than 3 cells per axis use all pairs) in the JSPLIT<w>
 * order (Sec. 4.1), FP32 pair math and FP64 accumulation.  The phases of a
 * step are separated by a grid barrier whose waits are bounded: a wait that
 * gives up ends the launch and the run returns LJ_ERR_TIMEOUT.
 * ------------------------------------------------------------------------ */
typedef struct lj_ens lj_ens;

/* nboxes boxes; box b has edge box_L[b] (> 2 cutoff) and counts[b] particles.
 * pos_fp / vel (host): per box 3*n_b entries (SoA) at offset 3*off_b, off_b =
 * sum of the counts before b; vel may be NULL.  cuda_stream may be NULL (the
 * ensemble then uses a stream of its own).  Errors: LJ_ERR_ARG, LJ_ERR_OOM,
 * LJ_ERR_CUDA. */
lj_status lj_ensemble_create(lj_ens** out, int32_t nboxes, const double* box_L, const int64_t* counts,
                             const uint32_t* pos_fp, const double* vel, double cutoff, double eps, double sigma,
                             double mass, void* cuda_stream);
/* Verlet-list mode (Sec. 2.1.1) for the whole batch: with skin > 0 every box
 * bins on cells of edge >= cutoff + skin and keeps Verlet lists (the builder
 * of lj_build_verlet, one warp per cell, whole-box lists for boxes of fewer
 * than 3 such cells per axis), rebuilt inside the launch every rebuild_every
 * steps or when a particle moved beyond skin/2 since the last build; forces
 * use the JSPLIT<w> list order.  skin = 0 returns to linked cells rebinned
 * every step.  cap = list capacity per particle (0 = from the densest box).
 * A list longer than cap stops the run mid-step with LJ_ERR_CAPACITY.
 * Errors: LJ_ERR_ARG, LJ_ERR_OOM, LJ_ERR_CUDA. */
lj_status lj_ensemble_set_lists(lj_ens* ens, double skin, int32_t rebuild_every, int32_t cap);
/* nsteps steps of every box in one launch (initial forces first if none are
 * current); use_graph = 1 captures the launch as a CUDA graph and replays it.
 * Synchronises.  Errors: LJ_ERR_ARG, LJ_ERR_TIMEOUT, LJ_ERR_NONFINITE,
 * LJ_ERR_CAPACITY (list mode), LJ_ERR_CUDA. */
lj_status lj_ensemble_run(lj_ens* ens, double dt, int32_t nsteps, int32_t use_graph);
/* Autotunes the launch shape (JSPLIT width w in {2,4,8,16}, block size in
 * {128,256,512}) by timing `steps` steps of each on a copy of the state. */
lj_status lj_ensemble_tune(lj_ens* ens, double dt, int32_t steps, int32_t* w_out, int32_t* block_out);
/* Copies the state out in the caller's layout and order (any pointer may be NULL). */
lj_status lj_ensemble_get(lj_ens* ens, uint32_t* pos_fp, double* vel, double* frc);
/* Failure-path test hook: barrier spin bound (0 = default, about seconds) and
 * a block that leaves before its first barrier (-1 = none). */
lj_status lj_ensemble_debug(lj_ens* ens, uint32_t spin_limit, int32_t skip_block);
int64_t lj_ensemble_size(const lj_ens* ens);
/* Unique in-cutoff pairs summed over the force evaluations since the last
 * call (resets the count; synchronises); -1 on error. */
int64_t lj_ensemble_pairs(lj_ens* ens);
/* Message of the last ensemble error or fallback (never NULL). */
const char* lj_ensemble_last_error(const lj_ens* ens);
/* 1 if the last run replayed a captured CUDA graph. */
int32_t lj_ensemble_uses_graph(const lj_ens* ens);
void lj_ensemble_destroy(lj_ens* ens);

/* Allocation-free stable counting sort by cell id, for callers that cannot
 * allocate device memory when they need cell lists: code running while
 * another allocator owns the device's memory pool, real-time loops where the
 * implicit synchronisation of cudaMalloc is not allowed, or programs that must
 * not fail on allocation after start-up.  The paper has no counterpart; this
 * is the binning of lj_bin_cells without a context and without allocation.
 *
 * pos_fp: device array of 3*n uint32 fixed-point coordinates (SoA), in the
 * caller's order.  nc: cells per axis (cell of a coordinate = (x * nc) >> 32).
 * Outputs (device, caller-owned): perm[n] = original index of the k-th
 * particle in cell order (ties keep ascending original index) and
 * cell_start[nc^3 + 1].  Work is queued on cuda_stream (NULL = legacy default
 * stream); the call does not synchronise.
 *
 * Scratch lives in one fixed device array inside the library, sized for
 * n <= LJ_STATIC_MAX_N particles and nc^3 <= LJ_STATIC_MAX_CELLS cells (about
 * 1.7 MB, held by every GPU that loads the library until the process exits);
 * larger inputs return LJ_ERR_ARG.  No cudaMalloc, cudaFree or other
 * allocating call is made.  The first call on each device looks up the
 * array's device address (with that device current); make that first call
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU (other streams or threads) race and must be serialised by the
 * caller.  Errors: LJ_ERR_ARG (null pointer, n < 1, nc < 1, sizes above the
 * maxima), LJ_ERR_CUDA. */
#define LJ_STATIC_MAX_N 65536
#define LJ_STATIC_MAX_CELLS 32768
lj_status lj_bin_cells_static(const uint32_t* pos_fp, int64_t n, int32_t nc, uint32_t* perm,
                              uint32_t* cell_start, void* cuda_stream);

/* Message of the last error on this context (never NULL). */
const char* lj_last_error(const lj_ctx* ctx);

void lj_destroy(lj_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LJGB_H */
