/*
 * bte.h — C ABI of libbte, the GB300 (sm_103a) implementation of the
 * conservative spectral collision operator of Haack & Gamba,
 * "High Performance Computing with a Conservative Spectral Boltzmann Solver"
 * (arXiv:1211.0540).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Velocity grid (Sec. 3.1, Eq. meshpoints): N points per dimension on [-L, L)^3,
 *   v_j = dv (j - N/2), dv = 2L/N; Fourier grid zeta_k = dz (k - N/2), dz = pi/L.
 *   N must be even; the library supports N in {8, 12, 16, 24, 32, 48}. At N = 48
 *   the stored FP32 weight table (10 GB) is built on first use by a variant that
 *   streams it (option conv_impl 5 builds the weights on the fly instead, with
 *   no table), and the plain FP64 operator and the transport step take N <= 32.
 * - A "cell" is one distribution f on that grid: M = N^3 doubles, index
 *   (j1*N + j2)*N + j3 (j3 fastest). Arrays of cells are cell-major.
 * - f and Q pointers are DEVICE pointers (cudaMalloc / torch tensors) owned by
 *   the caller, unless a call says otherwise. The context owns everything it
 *   allocates (weight tables, scratch) and frees it in bte_destroy.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Calls enqueue work on the stream and return without synchronising, unless
 *   stated. Errors detected inside kernels (non-finite input, a bounded wait
 *   that ran out) are recorded in a device status word, read by
 *   bte_sync_status.
 * - Every call returns a bte_status; on failure bte_last_error() describes it.
 *   No call traps the GPU on bad input: shapes are checked on the host.
 * - A context is not thread-safe; use one context per host thread. Contexts
 *   on different host threads are independent (the library's process-wide
 *   caches of kernel configurations are locked).
 *
 * Instances (uneven batches)
 * --------------------------
 * `inst == NULL` means `ninst` uniform cells of table 0 stored back to back
 * (cell c at f + c*M). Otherwise inst[i] names the weight table of instance i
 * (its grid, hence its M) and the element offset of its data inside f and Q.
 */
#ifndef BTE_H
#define BTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bte_ctx bte_ctx;

typedef enum {
    BTE_OK = 0,
    BTE_EINVAL = -1,      /* bad argument, shape or state of the arguments      */
    BTE_ENOMEM = -2,      /* device or host allocation failed                  */
    BTE_ECUDA = -3,       /* a CUDA runtime call failed                         */
    BTE_ETIMEOUT = -4,    /* a bounded in-kernel wait ran out (device status)   */
    BTE_ENONFINITE = -5,  /* NaN/Inf found in an input (device status)          */
    BTE_ESTATE = -6       /* call made in the wrong state (e.g. no tables yet)  */
} bte_status;

typedef enum {
    BTE_FP64_PLAIN = 0,   /* plain FP64 operator: direct sums, FP64 weights     */
    BTE_FP32 = 1,         /* FP32 compensated convolution, FP64 projection      */
    BTE_LEARNED = 2       /* MLP surrogate + FP64 projection + exact fallback   */
} bte_mode;

/* Boundary of the 1-D slab: diffuse wall (Sec. 2.1, Eq. BC), specular wall,
 * or no flux for the incoming characteristics (Sec. 3.4: for boundaries
 * without wall interaction; incoming components enter as 0, outgoing ones
 * leave freely). */
typedef enum { BTE_BC_DIFFUSE = 0, BTE_BC_SPECULAR = 1, BTE_BC_NOFLUX = 2 } bte_bc;

/* bte_collide_ex flags */
#define BTE_FLAG_RAW 1u          /* return Qt (skip the conservation projection)  */
#define BTE_FLAG_NO_FALLBACK 2u  /* BTE_LEARNED: projected surrogate output only  */

/* Velocity grid and collision kernel of one weight table: B = |u|^lambda / (4 pi)
 * (isotropic, Sec. 2.2). lambda = 0: Maxwell molecules, 1: hard spheres,
 * 0 < lambda < 1 variable hard and -3 < lambda < 0 variable soft potentials
 * (Sec. 2.1). */
typedef struct {
    int N;
    double L;
    double lambda;
} bte_grid;

/* A weight table's grid and collision model, with the restitution parameter
 * beta of the collision rule v' = v + (beta/2)(|u| sigma - u) (Sec. 2.2,
 * Eq. G_eqn / GHat_calc): beta = 1 elastic; 0 < beta < 1 inelastic (beta =
 * (1 + e)/2 for a restitution coefficient e), whose projection conserves mass
 * and momentum only (Sec. 3.3). */
typedef struct {
    int N;
    double L;
    double lambda;
    double beta;
} bte_grid_ex;

typedef struct {
    int32_t table;   /* id returned by bte_init_weights                        */
    int32_t pad_;
    int64_t offset;  /* element offset of the instance inside f and Q           */
} bte_instance;

/* 1-D slab [x0, x1] of nx uniform cells with a wall at each end (Sec. 2.1,
 * Eq. BC; Sec. 3.4). bc_*: BTE_BC_DIFFUSE (wall temperature Tw_*, zero wall
 * velocity), BTE_BC_SPECULAR or BTE_BC_NOFLUX. */
typedef struct {
    int nx;
    double x0, x1;
    int bc_left, bc_right;
    double Tw_left, Tw_right;
} bte_transport;

/* The slab with cells of unequal width (Sec. 3.4: cells of size dx_j, "not
 * necessarily uniform"; the paper refines the grid near a wall, Sec. 5).
 * dx: HOST array of nx positive widths, or NULL for nx uniform cells of
 * [x0, x1] (x0, x1 are ignored when dx is given). */
typedef struct {
    int nx;
    const double *dx;
    double x0, x1;
    int bc_left, bc_right;
    double Tw_left, Tw_right;
} bte_transport_ex;

/* Create a context on CUDA device `device`. *ctx receives the handle.
 * Errors: BTE_EINVAL (ctx NULL, bad device), BTE_ECUDA. */
bte_status bte_create(bte_ctx **ctx, int device);

/* Release everything the context owns. Safe on NULL. Synchronises the device. */
void bte_destroy(bte_ctx *ctx);

/* Message for the last failing call of this context ("" if none). The string
 * belongs to the context. */
const char *bte_last_error(const bte_ctx *ctx);

/* Tabulate the convolution weights Ghat(xi_m, zeta_k) of Sec. 2.2,
 * Eq. GHat_calc (isotropic b, radial integral cut off at r0 = L, Sec. 3.1) in
 * FP64 on the host for each grid, and store them on the device: the FP32
 * pair-symmetrised table of the fast path and the moment/projection constants
 * of Sec. 3.3. lambda = 0, 1: closed forms of the radial integrals; other
 * lambda in (-3, 1), as Sec. 2.2 prescribes, by quadrature: the power series of
 * the integrand integrated term by term on [0, 1/omega] (exact for the factor
 * r^(lambda+2), singular at 0 for lambda < -2) and composite Clenshaw-Curtis
 * panels beyond (omega: the table's largest radial frequency).
 * The FP64 table of the plain operator is built on the first BTE_FP64_PLAIN
 * call that needs it. table_ids[i] (host array of ngrids ints) receives the id
 * of grid i. Synchronous. bte_init_weights: elastic grids (beta = 1).
 * bte_init_weights_ex: any beta in (0, 1]; beta < 1 needs lambda = 0 or 1.
 * Errors: BTE_EINVAL (N unsupported, L <= 0, lambda outside (-3, 1], beta
 * outside (0, 1]), BTE_ENOMEM. */
bte_status bte_init_weights(bte_ctx *ctx, const bte_grid *grids, int ngrids, int *table_ids);
bte_status bte_init_weights_ex(bte_ctx *ctx, const bte_grid_ex *grids, int ngrids, int *table_ids);

/* Collision operator Q = P_N Qt(f) of Sec. 3.2-3.3 for a batch of cells:
 * forward transform of f, weighted convolution
 * Qhat(zeta_k) = dz^3 sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m)
 * with zero extension, inverse transform (real part), conservation projection.
 * f, Q: device FP64 arrays (see Instances); inst: HOST array or NULL.
 * f and Q must not overlap. mode: bte_mode. Asynchronous on `stream`.
 * Errors: BTE_EINVAL, BTE_ESTATE (no tables / no trained surrogate), BTE_ECUDA,
 * BTE_ENOMEM (scratch). */
bte_status bte_collide(bte_ctx *ctx, const double *f, double *Q, const bte_instance *inst,
                       int64_t ninst, int mode, void *stream);

/* bte_collide with flags (BTE_FLAG_RAW returns the unprojected Qt).
 * Mode BTE_LEARNED (uniform cells of table 0, surrogate built with
 * bte_mlp_init): Q = P_N(Q_nn) from the surrogate, then a residual indicator
 * per cell: the exact operator is evaluated at about 64 sampled Fourier modes
 * (bte_learned_sample: whole pencils with |k1'|, |k2'| <= N/4) and
 *   ind = ||F[Q](zeta_s) - Qhat(zeta_s)|| / ||Qhat_loss(zeta_s)||
 * (Qhat_loss: the same sum with the loss term of Ghat only). Cells with ind
 * above the option "learned_tol_ppm" * 1e-6 (default 1e-2) are recomputed with
 * the FP32 operator (conv_impl 5 if chosen, else 4, unsplit work list). The
 * list of those cells and the recompute's work list are built on the device,
 * so the call does not synchronise (it is asynchronous like the FP32 mode).
 * BTE_FLAG_NO_FALLBACK skips the indicator. Counts: bte_learned_stats. */
bte_status bte_collide_ex(bte_ctx *ctx, const double *f, double *Q, const bte_instance *inst,
                          int64_t ninst, int mode, unsigned flags, void *stream);

/* Conservation projection of Sec. 3.3 in place on device array Q:
 * Q <- Q - C^T (C C^T)^{-1} C Q, C = dv^3 (1, v1, v2, v3, |v|^2) per grid
 * point, FP64 (for inelastic tables, beta < 1, C keeps the mass and momentum
 * rows only). (The paper prints "+ C"; the Lagrange solution of the stated
 * minimisation has "- C^T".) Asynchronous. Errors: BTE_EINVAL, BTE_ESTATE. */
bte_status bte_project(bte_ctx *ctx, double *Q, const bte_instance *inst, int64_t ninst,
                       void *stream);

/* One time step on device array f, in place.
 * tr == NULL: space-homogeneous Heun (RK2) step of df/dt = Q(f,f)/eps with the
 *   projection at each stage (Sec. 3.1): Q1 = P Qt(f); f* = f + dt/eps Q1;
 *   Q2 = P Qt(f*); f <- f + dt/(2 eps) (Q1 + Q2).
 * tr != NULL: Strang step T(dt/2) C(dt) T(dt/2) (Sec. 3.1) of the 1-D slab,
 *   T = Heun step of the second-order upwind / minmod finite-volume transport
 *   (Sec. 3.4, Eq. upwind) with diffuse (Eq. BC, sigma_w balancing the
 *   discrete outgoing flux) or specular walls, C = the homogeneous step above
 *   over all tr->nx cells (inst must be NULL and ninst == tr->nx).
 * The homogeneous and Strang steps are replayed from a CUDA graph captured on
 * the first call with a given shape. Asynchronous. Errors as bte_collide.
 * mode BTE_LEARNED (uniform cells of table 0): both stages take Q from the
 *   learned mode of bte_collide_ex (surrogate, projection, indicator, FP32
 *   recompute of the flagged cells, all on the device), so a replayed graph
 *   recomputes whichever cells each stage flags. The graph is captured anew
 *   when the surrogate's buffers or scales change.
 * bte_step_ex: the same with a bte_transport_ex slab. On cells of unequal
 * width the upwind reconstruction of Eq. upwind uses the upwind cell's width
 * dx_j, and the minmod slope divided differences over the distances between
 * cell centres, (dx_j + dx_{j+1}) / 2; the two ghost cells at each end mirror
 * the widths of the adjacent cells; the update divides by dx_j. */
bte_status bte_step(bte_ctx *ctx, double *f, const bte_instance *inst, int64_t ninst, double dt,
                    double eps, const bte_transport *tr, int mode, void *stream);
bte_status bte_step_ex(bte_ctx *ctx, double *f, const bte_instance *inst, int64_t ninst, double dt,
                       double eps, const bte_transport_ex *tr, int mode, void *stream);

/* Synchronise `stream`, read and clear the device status word.
 * Returns BTE_OK, BTE_ETIMEOUT, BTE_ENONFINITE or BTE_ECUDA. */
bte_status bte_sync_status(bte_ctx *ctx, void *stream);

/* Copy `bytes` between a HOST buffer and DEVICE memory, ordered on `stream`
 * (the state in and out of a step, e.g.). kind BTE_HOST_TO_DEVICE: src host,
 * dst device; BTE_DEVICE_TO_HOST: src device, dst host. Where the host buffer
 * is reachable from the device (page-locked memory on a system with unified
 * addressing; on GB300 over the chip-to-chip link) a kernel of the library
 * moves it from every SM; otherwise cudaMemcpyAsync (synchronous for pageable
 * memory). Both buffers must hold `bytes`; they stay the caller's. No
 * counterpart in the paper. Errors: BTE_EINVAL (null buffer, unknown kind),
 * BTE_ECUDA. */
#define BTE_HOST_TO_DEVICE 0
#define BTE_DEVICE_TO_HOST 1
bte_status bte_transfer(bte_ctx *ctx, void *dst, const void *src, size_t bytes, int kind, void *stream);

/* Moments (C f)_i, i = mass, momentum 1..3, energy, per cell: out is a DEVICE
 * array of 5*ninst doubles. FP64. Asynchronous. */
bte_status bte_moments(bte_ctx *ctx, const double *f, double *out, const bte_instance *inst,
                       int64_t ninst, void *stream);

/* Kernel timing for benchmarks. When enabled, CUDA events are recorded on the
 * launching stream around every launch of the kernels named below (also inside
 * the graphs bte_step captures; switching profiling on or off drops the
 * captured step graphs, so that the next steps capture again with or without
 * the events). bte_profile_read synchronises
 * `stream`, returns the number of launches of `kernel` completed since they
 * were last read and their summed device time in milliseconds, and forgets
 * them (entries of other kernels stay pending).
 * kernel: "conv32" (FP32 convolution), "conv64" (plain FP64 convolution),
 * "forward" (all forward transforms of a collide), "inverse" (all inverse
 * transforms of a collide with the projection and time update fused into
 * them; with dft_fuse_stages, the first Heun stage's inverse also runs the
 * second stage's forward transform, so a Heun step records one "forward"
 * and two "inverse" launches), "transport" (one transport sub-step, two launches), "collide" (a
 * whole collide call), or "*" (all of them, summed).
 * bte_launch_count returns the number of libbte kernels enqueued by this context
 * so far (a graph replay counts its kernels). */
bte_status bte_profile_enable(bte_ctx *ctx, int enable);
bte_status bte_profile_read(bte_ctx *ctx, const char *kernel, int64_t *launches, double *total_ms,
                            void *stream);
bte_status bte_launch_count(const bte_ctx *ctx, int64_t *count);

/* Number of instance layouts (batches) the context keeps: each distinct
 * (inst, ninst) given to bte_collide / bte_step / bte_autotune builds a batch
 * (slot map, work items; device memory) that later calls reuse. The cache
 * holds at most the "batch_cache" option (default 64); a new layout beyond it
 * evicts the least recently used one, which waits for the kernels this context
 * has enqueued and drops captured step graphs. count (HOST) receives the number. */
bte_status bte_batch_count(const bte_ctx *ctx, int64_t *count);

/* Number of captured step graphs the context keeps (bte_step on a non-default
 * stream captures one per (instance list, mode, transport, dt, eps, f,
 * stream)). The cache holds at most the "graph_cache" option (default 32); a
 * new graph beyond it destroys the least recently replayed one (a replay
 * still in flight completes first). count (HOST) receives the number. */
bte_status bte_graph_count(const bte_ctx *ctx, int64_t *count);

/* Tuning options of the FP32 convolution (read by the autotuner and tests).
 * name: "conv_impl"   0 = one warp per work item, 1 = all warps of a CTA share
 *                      an item (reduced in shared memory), 2 = as 1 with packed
 *                      f32x2 arithmetic, 3 = as 2 with up to 255 registers per
 *                      thread (2 CTAs per SM), 4 (default) = as 2 with each
 *                      warp's compensated sums in shared memory instead of
 *                      registers (the b-row stays in registers as packed
 *                      operands for the whole block), 5 = as 4 with the weights
 *                      built on the fly: each warp computes its block's
 *                      pair-symmetrised weights from the radial integrals
 *                      I(|k'|^2, |2m' - k'|^2) and J(|m'|^2) (FP32 tables of
 *                      0.5 MB at N = 16, 9 MB at N = 32) instead of streaming
 *                      the stored weight table (elastic tables only). Kinds of
 *                      N = 48 run on 4 and 5, and on 3 when they are the
 *                      batch's only kinds (its four warps per CTA fit there);
 *       "conv_warps"  warps per CTA (1..8 for impl 0, 1..4 otherwise);
 *       "conv_stages" blocks in flight per warp (1..4; 0 = automatic, the
 *                      default: the deepest ring up to 2 that keeps the
 *                      resident CTAs per SM of a one-block ring);
 *       "conv_merge"  blocks accumulated in plain FP32 between compensated
 *                      (TwoSum) merges (>= 1, default 16);
 *       "batch_cache" instance layouts kept (2..2^20, default 64; see
 *                      bte_batch_count);
 *       "graph_cache" captured step graphs kept (1..2^20, default 32; see
 *                      bte_graph_count);
 *       "conv_split"  variant 4: 1 (default) runs the batch's plan in which
 *                      the costliest pencil items are cut into two block
 *                      ranges (chosen when the batch is built, by simulating
 *                      the work queue on 3 CTAs per SM); the half that
 *                      finishes second adds both halves' sums in a fixed
 *                      order (deterministic); 0 runs every pencil whole;
 *       "learned_tol_ppm" fallback threshold of the learned mode in 1e-6 units;
 *       "dft_fuse_stages" 1 (default): in an FP32 Heun step the first stage's
 *                      inverse transform also forms the second stage's forward
 *                      transform (the intermediate state is not stored), bit
 *                      for bit the result of separate launches (0);
 *       "dft_split"   CTAs (one thread-block cluster) per cell in the fused
 *                      transforms of N <= 16: 1, 2 or 4 (default 4);
 *       "debug_conv_stall" testing only: 1 makes every warp of the
 *                      cooperative convolution (conv_impl 1..4) skip the
 *                      copies of its first block, so that its bounded wait runs
 *                      out: the call completes after about two seconds, the
 *                      next bte_sync_status returns BTE_ETIMEOUT and the
 *                      context stays usable (the test of the timeout path);
 *       "profile_mask" which kernels bte_profile_enable times, bit k for
 *                      conv32 (0), conv64 (1), collide (2), forward (3),
 *                      inverse (4), transport (5); default 63 (all).
 * Changing an option drops the captured step graphs. Errors: BTE_EINVAL. */
bte_status bte_set_option(bte_ctx *ctx, const char *name, int value);
bte_status bte_get_option(const bte_ctx *ctx, const char *name, int *value);

/* Checkpoint of a solver state (no counterpart in the paper: long runs stop
 * and resume). bte_state_save writes the n FP64 values of the DEVICE array f
 * (e.g. the cells of a slab, instance-ordered as the caller keeps them), the
 * time t and the step counter to `path`: a header (magic "BTESTATE", format
 * version, n, t, step, the FNV-1a hash of this context's weight grids (N, L,
 * lambda of every table, in order)), the values, and the FNV-1a checksum of
 * header and values. bte_state_load reads it into the DEVICE array f (n values,
 * which must equal the stored count) and returns t and step (HOST, optional).
 * Both synchronise `stream`. The kernels reduce in a fixed order, so steps
 * taken after a load reproduce the uninterrupted run bit for bit.
 * Errors: BTE_EINVAL (unreadable/unwritable file, bad magic or version,
 * checksum mismatch, n differs), BTE_ESTATE (the file was written under other
 * weight grids), BTE_ECUDA. */
bte_status bte_state_save(bte_ctx *ctx, const char *path, const double *f, int64_t n, double t, int64_t step,
                          void *stream);
bte_status bte_state_load(bte_ctx *ctx, const char *path, double *f, int64_t n, double *t, int64_t *step,
                          void *stream);

/* Autotuner of the FP32 path. For the batch described by (inst, ninst) (as in
 * bte_collide) it runs one projected FP32 collide of f per candidate
 * configuration -- convolution variant 1, 2, 3 or 4, 3 or 4 warps per CTA, 1 or 2
 * blocks in flight per warp, compensated merge every 16 or 32 blocks, for
 * variant 4 with and without split pencil items, and for N <= 16 one, two or
 * four CTAs per cell in the fused transforms -- times reps
 * repetitions with CUDA events on `stream`, and keeps the fastest as this
 * context's configuration for batches of the same shape (the same set of
 * grid sizes and number of 32-cell slots); it takes precedence over the
 * options until any conv_* or dft_split option is set. f (DEVICE, read only) is
 * the input the timing runs on; results go to internal scratch. out_cfg (HOST,
 * 6 ints, optional) receives (conv_impl, conv_warps, conv_stages, conv_merge,
 * dft_split, conv_split), out_ms (optional) the time of one collide. Synchronous; drops
 * captured step graphs. Errors: as bte_collide, BTE_ETIMEOUT / BTE_ENONFINITE
 * from the trial runs. */
bte_status bte_autotune(bte_ctx *ctx, const double *f, const bte_instance *inst, int64_t ninst, int reps,
                        int *out_cfg, double *out_ms, void *stream);

/* The tuning cache as a small JSON file: the GPU name and one entry per batch
 * shape. bte_tune_load applies the entries only if they were tuned on a GPU
 * of the same name (else it loads nothing and returns BTE_OK); *loaded (HOST,
 * optional) receives the number of entries applied. Errors: BTE_EINVAL
 * (unreadable, malformed or out-of-range file; nothing is applied). */
bte_status bte_tune_save(const bte_ctx *ctx, const char *path);
bte_status bte_tune_load(bte_ctx *ctx, const char *path, int *loaded);

/* BF16 GEMM on the tensor cores (tcgen05 + TMA), the building block of the
 * learned surrogate's training and inference:
 *   D[M, N] = A[M, K] . B[N, K]^T (+ bias[N]),  A, B: device bf16, row-major with K
 *   contiguous; FP32 accumulation. Outputs (each optional, device): D (FP32,
 *   [M][N], before the activation), D_bf16 ([M][N]) and D_bf16_t (transposed,
 *   [N][ld_t], ld_t >= M), both after GELU when gelu != 0 (tanh form).
 * Requirements: K % 64 == 0, N % 64 == 0 (M is free). Asynchronous.
 * Errors: BTE_EINVAL (shapes), BTE_ECUDA. */
bte_status bte_tc_gemm(bte_ctx *ctx, const void *A, const void *B, float *D, int M, int N, int K,
                       const float *bias, int gelu, void *D_bf16, void *D_bf16_t, int ld_t, void *stream);

/* Learned surrogate of the collision operator (no counterpart in the paper: a
 * residual MLP trained on (f, Q(f)) pairs that the operator itself produces):
 *   x = s_in f / rho, h1 = GELU(W1 x + b1), h2 = h1 + GELU(W2 h1 + b2),
 *   y = W3 h2 + b3, Q_nn = rho^2 y / s_out   (rho = sum f dv^3; Q is bilinear),
 * GELU in tanh form; BF16 weights/activations on the tensor cores, FP32
 * accumulation, FP32 master weights and AdamW. Parameters are one flat FP32
 * vector: W1 [H][M], b1 [H], W2 [H][H], b2 [H], W3 [M][H], b3 [M] (M = N^3).
 * bte_mlp_init: create it for weight table `table` (N^3 % 64 == 0, N <= 16),
 *   width H (multiple of 128), seeded initialisation. Synchronous.
 * bte_mlp_train: `epochs` passes over nsamples device pairs (f[i], Q[i]) (FP64,
 *   M values each, back to back), mini-batches of `batch`, AdamW (lr with cosine
 *   decay to lr/20, weight decay). *final_loss: mean square error of the last batch.
 * bte_mlp_grads: one forward/backward on the first n pairs without an update;
 *   copies the gradient (nparams floats) to host_grads and the loss to *loss.
 * bte_mlp_infer: Q_nn for n cells (device FP64; no projection).
 * bte_mlp_get/set_params: host FP32 vector of nparams values.
 * The surrogate is used by bte_collide and bte_step with mode BTE_LEARNED
 * (projection and fallback there). Errors: BTE_EINVAL, BTE_ESTATE (no surrogate), BTE_ENOMEM, BTE_ECUDA. */
bte_status bte_mlp_init(bte_ctx *ctx, int table, int width, uint64_t seed);
bte_status bte_mlp_info(const bte_ctx *ctx, int64_t *nparams, int *width, int *ndim, double *s_in, double *s_out);
bte_status bte_mlp_set_scales(bte_ctx *ctx, double s_in, double s_out);
/* bte_mlp_fit_scales: s_in as given, and s_out making the training targets
 *   s_out Q / rho^2 of the n pairs (f[i], Q[i]) (DEVICE, FP64, back to back)
 *   unit-RMS: s_out = 1 / sqrt(mean_i,j (Q_ij / rho_i^2)^2), rho_i = sum f_i dv^3.
 *   FP64, summed in a fixed order. *s_out (HOST, optional) receives it. Synchronous. */
bte_status bte_mlp_fit_scales(bte_ctx *ctx, const double *f, const double *Q, int64_t n, double s_in, double *s_out,
                              void *stream);
bte_status bte_mlp_get_params(bte_ctx *ctx, float *host, int64_t n);
bte_status bte_mlp_set_params(bte_ctx *ctx, const float *host, int64_t n);
bte_status bte_mlp_train(bte_ctx *ctx, const double *f, const double *Q, int64_t nsamples, int epochs, int batch,
                         double lr, double weight_decay, uint64_t seed, double *final_loss, void *stream);
bte_status bte_mlp_grads(bte_ctx *ctx, const double *f, const double *Q, int64_t n, double *loss, float *host_grads,
                         void *stream);
bte_status bte_mlp_infer(bte_ctx *ctx, const double *f, double *Q, int64_t n, void *stream);

/* Cells evaluated and recomputed by the learned mode since the last reset, and
 * the largest indicator seen (counted on the device by every learned collide
 * and every stage of a learned step; BTE_FLAG_NO_FALLBACK calls are not
 * counted). Waits for the work this context has enqueued; reset != 0 clears
 * the counts. Outputs (HOST) are optional. */
bte_status bte_learned_stats(bte_ctx *ctx, int64_t *cells, int64_t *fallbacks, double *max_indicator, int reset);

/* The fallback indicator of the learned mode (no counterpart in the paper).
 * Sampled modes: S = max(1, 64 / N) distinct zeta pencils (k1, k2) of table 0,
 * each with all N values of k3; the offsets k1' = k1 - N/2 and k2' lie in
 * [-N/4, N/4] and are drawn from SplitMix64 (Steele, Lea and Flood, OOPSLA
 * 2014) seeded with 12345: offset = (next mod (N/2 + 1)) - N/4, k1' first,
 * repeated pencils skipped (integer arithmetic, the same on every platform).
 * bte_learned_sample: *S (HOST) receives the pencil count and kk (HOST,
 *   optional, cap ints) the pencils as k1 N + k2 in drawing order.
 * bte_learned_indicator: for ncells uniform cells of table 0 (N <= 16) with
 *   distributions f and candidate operator values Q (DEVICE, FP64, ncells N^3
 *   each), writes per cell (DEVICE, ncells doubles)
 *     ind = ||F[Q](zeta_s) - Qhat(zeta_s)|| / ||Qhat_loss(zeta_s)||
 *   over the sampled modes: F is the forward transform of Sec. 3.2 in FP32,
 *   Qhat the weighted convolution of Sec. 3.2 at those modes (FP32, the fast
 *   path's pair-symmetrised weights) and Qhat_loss the same sum with the loss
 *   term of Ghat only. This is the quantity BTE_LEARNED compares with the
 *   threshold. Asynchronous. Errors: BTE_EINVAL, BTE_ESTATE, BTE_ENOMEM, BTE_ECUDA. */
bte_status bte_learned_sample(bte_ctx *ctx, int *kk, int cap, int *S);
bte_status bte_learned_indicator(bte_ctx *ctx, const double *f, const double *Q, int64_t ncells, double *ind,
                                 void *stream);

/* Size of the static device work area used by bte_collide_noalloc (16 MiB). */
#define BTE_NOALLOC_SCRATCH_BYTES (16u << 20)

/* bte_collide_noalloc -- the FP32 collision operator (as bte_collide with
 * mode BTE_FP32, inst == NULL: ncells uniform cells of table 0, projected Q)
 * for callers that cannot allocate GPU memory while they run: code that works
 * inside a fixed memory budget handed out up front (an embedding application's
 * own arena, or a device whose memory is already reserved by another
 * allocator), or a time-critical loop that must not pay for, or be
 * synchronised by, cudaMalloc/cudaFree. The paper has no counterpart; this is
 * a service of the library.
 * The call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine, and on success no host heap either. Its work area (queue
 * counter, per-cell offsets, work list, fhat and Qhat) is one file-scope
 * device array of BTE_NOALLOC_SCRATCH_BYTES, which every GPU that loads the
 * library holds until the process exits. A small kernel fills the work list
 * from a template built with the weight tables, so the call copies nothing
 * from the host and does not wait for `stream`. The caller passes f and Q
 * (device, ncells * N^3 doubles); the weight tables must have been built
 * before (bte_init_weights, at set-up), which also prepares the kernel
 * configurations the call looks up (as do bte_set_option and bte_autotune).
 * It runs the configuration autotuned for this batch shape if there is one
 * (without split work items), else the context's options.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. The caller's current device is left as it was.
 * Every call shares the array and leaves its contents behind; each call resets
 * what must start at zero. Calls that overlap on the GPU (two streams, or two
 * threads) race on the array: serialise them.
 * Limits: table 0 must have N = 8, 12 or 16; the cells must fit the array
 * (2 * ceil(ncells/32) * 32 * N^3 * 8 bytes of work arrays plus the work list):
 * up to 224 cells at N = 16, 576 at N = 12, 2016 at N = 8. Larger requests fail
 * with BTE_EINVAL and a message naming the bytes needed. Errors: BTE_EINVAL,
 * BTE_ESTATE, BTE_ECUDA. */
bte_status bte_collide_noalloc(bte_ctx *ctx, const double *f, double *Q, int64_t ncells, void *stream);

/* Arithmetic-rate probe of this GPU (no counterpart in the paper; the
 * denominators of the kernels' rooflines). kind 0: FP32 FMA (fma.rn.f32),
 * 1: packed FP32 FMA (fma.rn.f32x2), 2: FP64 FMA. Every SM runs 2048 threads of
 * independent FMA chains; *tflops (HOST) receives 2 flops per FMA over the
 * CUDA-event time of 5 launches after one warm-up, *ms (HOST, optional) the
 * time of one launch. Synchronous (on `stream`). Errors: BTE_EINVAL, BTE_ENOMEM,
 * BTE_ECUDA. */
bte_status bte_alu_peak(bte_ctx *ctx, int kind, double *tflops, double *ms, void *stream);

/* Library build identification (static string). */
const char *bte_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BTE_H */
