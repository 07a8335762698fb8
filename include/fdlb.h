/*
 * fdlb.h -- C ABI of the GB300 FDLB solver for the simplified Enskog equation
 * (Busuioc & Sofonea, "Bounded flows of dense gases", arXiv 2308.15407).
 *
 * What one call computes: the per-time-step update of the discrete reduced
 * (or unreduced) distribution f(x_i, p_kappa) of Eqs. (evolution_1D) and
 * (evolution_2D) -- moments (Eq. macro_LB), the Carnahan-Starling contact
 * value (Eq. chi), the Shakhov relaxation (Eq. j0), the first-order Enskog
 * correction J1 (Eq. j1), WENO-5 advection (Sec. III B 2) with diffuse-
 * reflection walls (Sec. III B) and the force term (App. A, Eq. kernel_H),
 * all inside the TVD Runge-Kutta scheme (Eq. rk3) -- for a batch of
 * independent wall-bounded 1D channel problems (Fourier, Couette, Poiseuille
 * flow, Sec. IV).
 *
 * Conventions
 *  - Units: m = k_B = T_ref = 1, channel width D = 1 (walls at x = -1/2 and
 *    x = +1/2), mean number density 1.  Kn refers to the channel width:
 *    mu0(T) = (5/16) sqrt(2 pi) chi(eta0) Kn sqrt(T).
 *  - Every call returns an int: FDLB_OK (0) or a negative FDLB_E* code; no
 *    C++ exception crosses the ABI.  fdlb_last_error() gives a message.
 *  - Ownership: the caller owns the device workspace (any device allocation,
 *    e.g. a torch uint8 tensor of fdlb_workspace_bytes() bytes, 256-byte
 *    aligned) and every host buffer.  The context owns only a small host-side
 *    record; fdlb_destroy() frees it and never touches the workspace.
 *  - Streams: all device work is enqueued on the cudaStream_t passed to
 *    fdlb_create (as void*; NULL = legacy default stream).  fdlb_step is
 *    asynchronous; every call that returns host data synchronises that stream.
 *  - Layout of f in the workspace: per instance, f[kappa][node] (node index
 *    contiguous, row stride rounded up to 32), kappa = kx * T_c + t with
 *    kx = 0..Q-1 for +p_k and Q..2Q-1 for -p_k (half-range nodes, Eq. hh_pk, or the
 *    positive nodes of the full-range rule of order 2Q with FDLB_XQ_FULL),
 *    t the transverse index: t = ky*Q_z + kz (unreduced), t = 2 ky + slot
 *    (2D reduced, slot 0 = phi, 1 = theta), t = slot (1D reduced).
 */
#ifndef FDLB_H
#define FDLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FDLB_ABI_VERSION 6

/* Return codes. */
#define FDLB_OK            0
#define FDLB_EINVAL       -1   /* invalid argument or parameter set */
#define FDLB_ENOMEM       -2   /* workspace too small or misaligned */
#define FDLB_ECUDA        -3   /* a CUDA runtime call failed (message in fdlb_last_error) */
#define FDLB_ENONFINITE   -4   /* an instance produced a non-finite moment */
#define FDLB_EUNPHYSICAL  -5   /* an instance produced n <= 0 or T <= 0 */
#define FDLB_ETIMEOUT     -6   /* fdlb_run hit its wall-clock limit */
#define FDLB_ESTATE       -7   /* state buffer does not match this context */

/* Flow types (Sec. IV): informational; the physics is set by the walls and the force. */
#define FDLB_FOURIER      0
#define FDLB_COUETTE      1
#define FDLB_POISEUILLE   2

/* Grid mapping x(s), s in (-1, 1), cell-centred nodes s_i = -1 + (i + 1/2) 2/nx. */
#define FDLB_GRID_UNIFORM 0    /* x = s/2 */
#define FDLB_GRID_TANH    1    /* x = tanh(A s)/(2 tanh A), A = stretch (nodes crowd at the walls) */

/* Storage precision of f. */
#define FDLB_FP64          0   /* everything in FP64 */
#define FDLB_FP32_STORAGE  1   /* f stored, advected and combined in FP32; moments, gradients,
                                  projections and the residual in FP64 */
#define FDLB_FP32_THEN_FP64 2  /* two phases: FDLB_FP32_STORAGE until the per-step residual
                                  stagnates, then FDLB_FP64 for the rest of the solve.  f is
                                  up-cast exactly on the device at the end of the step that
                                  detects the stagnation.  Stagnated: the residual is exactly 0,
                                  or at the end of a window of FDLB_STAGNATION_WINDOW steps it
                                  is not below FDLB_STAGNATION_FACTOR times its value at the
                                  window start (windows restart after each check).  An instance
                                  whose residual falls below freeze_tol first stays FP32.  The
                                  workspace holds f at FP64 size from the start.  FP32 storage
                                  cannot resolve per-step changes below half an FP32 ulp of f,
                                  so its residual floor can lie above the requested tolerance. */
#define FDLB_STAGNATION_WINDOW 2000
#define FDLB_STAGNATION_FACTOR 0.9

/* Contact value of the pair correlation function (Sec. II A).
 *   FDLB_CHI_SET:    chi_SET of the local density, Eq. (chi) (Carnahan-Starling).
 *   FDLB_CHI_RET_FM: the Fischer-Methfessel prescription, Eq. (chi_ret): chi_SET of the density
 *                    averaged over a ball of radius sigma, sigma = 6 sqrt(2) eta0 chi(eta0) Kn
 *                    in units of the channel width (the Kn definition of Sec. II A with n0 = 1).
 *                    The density depends on x only, is taken constant on each grid cell and zero
 *                    beyond the walls; the ball average is then a 1D average with weight
 *                    3 (sigma^2 - t^2)/(4 sigma^3), integrated exactly over each cell.  b rho in
 *                    the closure stays local.  Needs eta0 > 0.  It is what produces the density
 *                    layering next to the walls; with the channel-width units above sigma exceeds
 *                    the channel for large eta0 Kn, so it is meant for small sigma. */
#define FDLB_CHI_SET     0
#define FDLB_CHI_RET_FM  1

/* Quadrature on the wall-normal axis x (fdlb_params.x_quadrature).
 *   FDLB_XQ_HALF: half-range Gauss-Hermite rules of order qx_half on each half-axis
 *                 (Sec. III A 2); the discrete equilibrium is truncated at order qx_half - 1
 *                 on each half-axis.
 *   FDLB_XQ_FULL: one full-range Gauss-Hermite rule of even order 2 qx_half (App. A), the
 *                 variant the paper compares against; its nodes are +-p_k (no zero node), so
 *                 the 2 qx_half x-velocities keep their layout.  The discrete equilibrium is
 *                 the expansion over the whole axis truncated at order 2 qx_half - 1.  Needs
 *                 qx_half <= 100.  Walls, fluxes and moments are the same as with FDLB_XQ_HALF. */
#define FDLB_XQ_HALF     0
#define FDLB_XQ_FULL     1

/* Per-instance status (fdlb_status). */
#define FDLB_ACTIVE        0
#define FDLB_CONVERGED     1
#define FDLB_FAILED_NONFINITE  2
#define FDLB_FAILED_UNPHYSICAL 3
#define FDLB_STAGNATED     4   /* FDLB_FP32_STORAGE stepped with freeze_tol > 0: f stopped changing
                                  (residual exactly 0) before the residual reached freeze_tol */
#define FDLB_FAILED_COPY   5   /* an asynchronous copy into shared memory did not complete within the
                                  kernel's wait limit (~2 s); the instance is no longer advanced and
                                  fdlb_run reports FDLB_ETIMEOUT */

/* Parameters of one channel problem.  Set struct_size = sizeof(fdlb_params). */
typedef struct fdlb_params {
    uint32_t struct_size;
    int32_t  flow;        /* FDLB_FOURIER | FDLB_COUETTE | FDLB_POISEUILLE */
    int32_t  nx;          /* grid nodes, 8 <= nx <= 4096 */
    int32_t  grid;        /* FDLB_GRID_UNIFORM | FDLB_GRID_TANH */
    int32_t  qx_half;     /* half-range Gauss-Hermite order per side, 1..100 (2*qx_half x-velocities);
                             with FDLB_XQ_FULL half the full-range order, 1..100 (order <= 200) */
    int32_t  qy;          /* full-range order on y, 0 or 2..8; 0 = 1D reduced (p_y integrated out) */
    int32_t  qz;          /* full-range order on z, 0 or 3..8; 0 = (phi, theta) reduced slots */
    int32_t  precision;   /* FDLB_FP64 | FDLB_FP32_STORAGE | FDLB_FP32_THEN_FP64 */
    int32_t  j1_shear;    /* 0: J1 as printed for 2D flows; 1: add the 2 zeta_x zeta_y d_x u_y term of Eq. (j1) */
    int32_t  chi_model;   /* FDLB_CHI_SET | FDLB_CHI_RET_FM */
    int32_t  x_quadrature;  /* FDLB_XQ_HALF | FDLB_XQ_FULL */
    double   stretch;     /* A of FDLB_GRID_TANH (> 0) */
    double   kn;          /* Knudsen number referred to the channel width (> 0) */
    double   eta0;        /* mean reduced density eta0 = b n0/4, 0 <= eta0 < 0.5 */
    double   T_left, T_right;   /* wall temperatures (> 0) */
    double   U_left, U_right;   /* wall velocities along y */
    double   accel_y;     /* body-force acceleration along y (Poiseuille) */
    double   cfl;         /* dt = cfl * min_i dx_i / max_k p_k when dt == 0 */
    double   dt;          /* explicit time step, or 0 */
    double   T_init;      /* initial uniform temperature, or 0 for the mean wall temperature */
} fdlb_params;

typedef struct fdlb_ctx fdlb_ctx;

/* ABI version of the loaded library (FDLB_ABI_VERSION). */
int32_t fdlb_abi_version(void);

/* Message for the last error on ctx (or the last context-free error when ctx == NULL).
 * The string is owned by the library and valid until the next call on ctx. */
const char* fdlb_last_error(const fdlb_ctx* ctx);

/* Device workspace needed by a batch of `count` instances described by params[0..count-1].
 * Returns 0 for an invalid parameter set (fdlb_last_error(NULL) says why). */
size_t fdlb_workspace_bytes(const fdlb_params* params, int32_t count);

/* Build the quadratures, grids and tables of every instance, place them and the state in
 * dev_workspace (ws_bytes >= fdlb_workspace_bytes, 256-byte aligned device memory), and
 * enqueue the initial uniform projected equilibrium (n = 1, u = 0, T = T_init) on `stream`.
 * *out receives the context.  Errors: FDLB_EINVAL, FDLB_ENOMEM, FDLB_ECUDA. */
int fdlb_create(fdlb_ctx** out, const fdlb_params* params, int32_t count,
                void* dev_workspace, size_t ws_bytes, void* stream);

/* Release the host record.  The workspace stays owned by the caller. */
void fdlb_destroy(fdlb_ctx* ctx);

/* Number of instances, nodes of instance i, velocities of instance i. */
int fdlb_info(const fdlb_ctx* ctx, int32_t inst, int32_t* nx, int32_t* nvel, double* dt);

/* How the tiled schedule splits instance `inst` (Sec. III B's per-node / per-velocity
 * structure; the split is a property of the batch, not of the method): *chunk = velocities
 * per update block, *chunks_per_tile = update blocks per 32-node tile (> 1: the blocks'
 * partial moment sums are added in chunk order by the last block of the tile), *tiles =
 * 32-node tiles.  The chunk is 16 velocities for batches of fewer than 38 tiles, 32 up to
 * 1215 tiles, and the whole velocity set (at most 256 per block) from 1216 tiles on.  Any
 * output pointer may be NULL.  Errors: FDLB_EINVAL (null context, instance out of range). */
int fdlb_layout(const fdlb_ctx* ctx, int32_t inst, int32_t* chunk, int32_t* chunks_per_tile, int32_t* tiles);

/* Advance every ACTIVE instance by nsteps RK3 steps (asynchronous).  Each step computes the
 * per-step residual of every instance (change of n, T, u_x, u_y in the cell-width-weighted
 * L2 norm; relative for n and T) and marks non-finite or unphysical instances FAILED.
 * With freeze_tol > 0 an instance whose residual falls below freeze_tol is marked CONVERGED
 * and is not advanced further.  Errors: FDLB_EINVAL, FDLB_ECUDA. */
int fdlb_step(fdlb_ctx* ctx, int64_t nsteps, double freeze_tol);

/* Steady-state solve: step in chunks of check_every steps until every instance is CONVERGED
 * (residual < tol) or FAILED, or max_steps steps were taken, or timeout_s seconds of wall
 * time passed (FDLB_ETIMEOUT).  On stopping it returns FDLB_ENONFINITE or FDLB_EUNPHYSICAL
 * when some instance failed (the others are still advanced until they stop), else FDLB_OK
 * when all converged, 2 when all stopped but some STAGNATED, or 1 when max_steps was
 * reached with instances still active. */
int fdlb_run(fdlb_ctx* ctx, double tol, int64_t max_steps, int64_t check_every, double timeout_s);

/* Host copy of the moments of instance `inst` (synchronises the stream):
 * host_out[8 * nx] = rows n, u_x, u_y, T, q_x, q_y, Pi_xx, Pi_xy (kinetic, Eq. macro_LB). */
int fdlb_moments(fdlb_ctx* ctx, int32_t inst, double* host_out);

/* Per-instance last residual, status and step count (synchronises).  Any pointer may be NULL. */
int fdlb_status(fdlb_ctx* ctx, double* residual, int32_t* status, int64_t* steps);

/* Per-instance residual of the last step (synchronises): host_out[count] receives the
 * residual that fdlb_status reports, the largest of the step's changes of n and T (relative)
 * and of u_x and u_y, each in the cell-width-weighted L2 norm over the channel (the
 * steady-state measure; the paper gives none).  Errors: FDLB_EINVAL (null ctx or host_out),
 * FDLB_ECUDA. */
int fdlb_residual(fdlb_ctx* ctx, double* host_out);

/* Reset instance `inst` to the projected local equilibrium with the given profiles
 * (u_x = 0; host arrays of nx values; n > 0, T > 0) and mark it ACTIVE with 0 steps
 * (an FDLB_FP32_THEN_FP64 instance restarts in its FP32 phase). */
int fdlb_set_profiles(fdlb_ctx* ctx, int32_t inst, const double* n, const double* uy, const double* T);

/* Per-instance storage precision in use now (FDLB_FP64 or FDLB_FP32_STORAGE) and, for
 * FDLB_FP32_THEN_FP64 instances, the step count at which f was up-cast (-1: not yet, and for
 * the other precision forms).  Synchronises.  Either pointer may be NULL. */
int fdlb_precision(fdlb_ctx* ctx, int32_t* storage, int64_t* switch_step);

/* Checkpoint of instance `inst`: f, step count and a parameter hash (FDLB_FP32_THEN_FP64:
 * also the storage phase and switch step; f always takes its FP64 size there, the first
 * half holding the floats in the FP32 phase).  fdlb_state_bytes gives the size; get copies
 * device -> host (synchronises), set copies host -> device (FDLB_ESTATE when the buffer
 * belongs to other parameters). */
size_t fdlb_state_bytes(const fdlb_ctx* ctx, int32_t inst);
int fdlb_get_state(fdlb_ctx* ctx, int32_t inst, void* host, size_t bytes);
int fdlb_set_state(fdlb_ctx* ctx, int32_t inst, const void* host, size_t bytes);

/* Schedules of fdlb_step.  Both compute the same arithmetic in the same order (results are
 * bitwise identical); they differ in how the work reaches the GPU.
 *   TILED:    one kernel per phase of an RK stage over every instance of the batch (work
 *             lists of 32-node tiles), replayed from a CUDA graph of 16 steps.  Fills the GPU
 *             with large batches.
 *   RESIDENT: one thread-block cluster per instance (up to 16 CTAs) runs whole steps in one
 *             launch, the phases separated by cluster barriers; instances advance
 *             independently and a converged instance's cluster exits.  It has no launches
 *             inside a step; on the GB300 the tiled schedule still measured faster on every
 *             workload tried (one instance: 113 against 244 us per RK3 step), because it
 *             spreads an instance's latency-bound items over more SMs than a cluster has.
 *   MIXED:    the instances whose three RK buffers fit in one block's shared memory together
 *             with the items' scratch (fdlb_get_schedule_mix; not FDLB_FP32_THEN_FP64) are
 *             stepped by one CTA each that keeps f in shared memory across all stages and steps
 *             of the call (f crosses HBM once at the start and once at the end of the call);
 *             the other instances take the tiled steps at the same time, on a second stream
 *             that the call forks from and joins back into the context's stream.
 *   AUTO:     (default) the first fdlb_step call with at least FDLB_AUTOTUNE_STEPS steps
 *             times every available schedule (its own steps, an equal share each) and keeps the
 *             fastest; shorter calls use TILED until then.
 * fdlb_profile's per-kernel timing always uses the tiled schedule. */
#define FDLB_SCHED_AUTO      0
#define FDLB_SCHED_TILED     1
#define FDLB_SCHED_RESIDENT  2
#define FDLB_SCHED_MIXED     3
#define FDLB_AUTOTUNE_STEPS  96

/* Request a schedule (FDLB_EINVAL for RESIDENT when the device cannot launch the cluster
 * kernel for this batch, and for MIXED when no instance fits in shared memory). */
int fdlb_set_schedule(fdlb_ctx* ctx, int32_t schedule);

/* Schedule in use (FDLB_SCHED_AUTO while not chosen yet) and the CTAs per cluster of the
 * resident schedule (0 when it is unavailable).  Either pointer may be NULL. */
int fdlb_get_schedule(const fdlb_ctx* ctx, int32_t* schedule, int32_t* cluster_ctas);

/* Which instances FDLB_SCHED_MIXED keeps in shared memory (chosen by size at creation):
 * smem_resident[count] (may be NULL) receives 1 for those, 0 for the others; *n (may be NULL)
 * their number (0: FDLB_SCHED_MIXED is unavailable for this batch). */
int fdlb_get_schedule_mix(const fdlb_ctx* ctx, int32_t* smem_resident, int32_t* n);

/* Optional per-kernel timing with CUDA events recorded on the context's stream around every
 * launch (off by default).  fdlb_profile(ctx, 1) clears the records and starts recording,
 * fdlb_profile(ctx, 0) stops.  fdlb_profile_read synchronises and returns, for kernel class
 * kind (0 moments, 1 per-node closure, 2 update, 3 residual), the summed duration in ms and
 * the number of launches recorded.  A launch of a class may run one kernel per storage
 * precision present in the batch.  During steps the moments are computed in the epilogue of
 * the update kernel (class 2); class 0 only records moments computed from scratch. */
int fdlb_profile(fdlb_ctx* ctx, int32_t on);
int fdlb_profile_read(fdlb_ctx* ctx, int32_t kind, double* total_ms, int64_t* launches);

/* Largest scratch fdlb_step_noalloc can use (8 MiB = 8,388,608 B): enough for one instance
 * of nx = 400 with 16 x-velocities (qx_half = 8) x 6 x 6 in FP64 (8,218,880 B, the
 * Poiseuille set-up of Sec. IV), or the 200-node Couette instance with 12 x 6 x 4 velocities
 * (1.7 MB in FP32 storage).  fdlb_workspace_bytes(params, 1) is the amount an instance needs;
 * nx = 400 with qx_half = 16 x 6 x 6 (15.9 MB in FP64) is rejected. */
#define FDLB_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)

/* Stepping without any device allocation, for callers that cannot call cudaMalloc (or any
 * allocator): code running where allocation is forbidden or unsafe, e.g. inside a
 * host-side callback of a framework that owns all device memory, a plug-in sandboxed
 * from the allocator, or a real-time loop that must not trigger allocator
 * synchronisation.  The paper has no counterpart; this is a library service.
 *
 * Advances ONE instance (params) by nsteps RK3 steps in place: dev_f (f_bytes bytes of
 * device memory) holds its f in the layout described at the top of this file, i.e.
 * K * ceil(nx/32)*32 values of double (FDLB_FP64) or float (FDLB_FP32_STORAGE) with
 * K = 2 qx_half * T_c (FDLB_FP32_THEN_FP64 is rejected with FDLB_EINVAL).  If dev_moments
 * is not NULL it receives the 8 x nx moment rows of the result (as fdlb_moments, device
 * memory, 8 nx doubles).  All scratch lives in one static device array of
 * FDLB_NOALLOC_SCRATCH_BYTES that every device loading the library holds until the process
 * exits; instances that need more are rejected with FDLB_ENOMEM.  The array is shared by
 * every call and keeps the last call's contents (each call rebuilds what it reads), so calls
 * that overlap on the GPU race: serialise them.  Each call launches its kernels one by one
 * (it builds no CUDA graph), uploads its tables from the host and synchronises `stream`
 * twice, so it must never be called while its stream, or the process, is being captured into
 * a CUDA graph.  The first call on a device also looks up the array's device address
 * (cudaGetSymbolAddress).
 * Errors: FDLB_EINVAL (bad params or f_bytes), FDLB_ENOMEM, FDLB_ECUDA. */
int fdlb_step_noalloc(const fdlb_params* params, void* dev_f, size_t f_bytes, int64_t nsteps,
                      double* dev_moments, void* stream);

/* ---- Learned warm start (no counterpart in the paper): a multilayer perceptron that
 * predicts steady profiles from channel parameters, run on the tcgen05 tensor cores (BF16
 * operands, FP32 accumulation; FP32 master weights, Adam).  16 inputs (features, zero
 * padded), 4 hidden layers of 128 GELU units, 3 outputs.  Parameters are one flat FP32
 * vector (fdlb_mlp_param_count values) in the order W1 [16 x 128], b1, W2 [128 x 128], b2,
 * W3, b3, W4, b4, W5 [128 x 16] (columns 3..15 unused, kept zero), b5 [16]; W_l is stored
 * [inputs][outputs].  Inputs: device FP32 [points][16]; targets and predictions: device
 * FP32 [points][3].  The caller owns the workspace (fdlb_mlp_workspace_bytes(max_points)
 * bytes, 256-byte aligned); all work is enqueued on `stream`; calls returning host data
 * synchronise it.  FDLB_ETIMEOUT reports a tensor-core completion wait that gave up. */
typedef struct fdlb_mlp fdlb_mlp;
int32_t fdlb_mlp_param_count(void);
size_t fdlb_mlp_workspace_bytes(int32_t max_points);
const char* fdlb_mlp_last_error(const fdlb_mlp* h);
/* Glorot-uniform weights from a counter-based hash of `seed`, zero biases, zero Adam state. */
int fdlb_mlp_create(fdlb_mlp** out, void* dev_workspace, size_t bytes, int32_t max_points, uint64_t seed, void* stream);
void fdlb_mlp_destroy(fdlb_mlp* h);
int fdlb_mlp_get_params(fdlb_mlp* h, float* host_params);
int fdlb_mlp_set_params(fdlb_mlp* h, const float* host_params);      /* also resets Adam state */
/* Forward pass: dev_y[points][3] = network(dev_x[points][16]). */
int fdlb_mlp_predict(fdlb_mlp* h, const float* dev_x, int32_t points, float* dev_y);
/* One training step on points <= max_points samples: loss = mean over points and the 3
 * outputs of (prediction - target)^2; gradient by backpropagation; Adam (beta1 0.9, beta2
 * 0.999, eps 1e-8) with learning rate lr (lr = 0: gradient only, no update).  dev_grad
 * (device FP32 [param_count], may be NULL) receives the gradient; host_loss (may be NULL) the
 * loss before the update. */
int fdlb_mlp_train_step(fdlb_mlp* h, const float* dev_x, const float* dev_y, int32_t points, float lr,
                        float* dev_grad, double* host_loss);

/* Host-only: the library's own Gauss rules (for checking the tables; no GPU needed).
 * kind 0 = half-range Gauss-Hermite on [0, inf) (Sec. III A 2), kind 1 = full-range (App. A);
 * weights are normalised to the weight omega(p) = exp(-p^2/2)/sqrt(2 pi).  nodes/weights
 * receive q values; q in 1..100 (half-range) or 1..200 (full-range).  Errors: FDLB_EINVAL. */
int fdlb_quadrature(int32_t kind, int32_t q, double* nodes, double* weights);

#ifdef __cplusplus
}
#endif

#endif /* FDLB_H */
