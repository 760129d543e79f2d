/*
 * lbm.h -- C ABI of a GB300 (sm_103a) solver for the three-dimensional MRT lattice
 * Boltzmann model for multiphase flow of Liang, Shi and Chai (arXiv:1507.07294).
 *
 * One time step couples two lattices on a regular grid of nx * ny * nz cells:
 *   - a D3Q7 lattice f_i for the Cahn-Hilliard equation of the order parameter phi
 *     (Sec. II A, Eqs. 4-19), and
 *   - a D3Q15 lattice g_i for the incompressible Navier-Stokes equations with pressure
 *     p and velocity u (Sec. II B, Eqs. 20-33),
 * with the isotropic difference schemes of Eqs. 34-36 for grad(phi), lap(phi) and
 * lap(mu).  Lattice units: c = dx = dt = 1.
 *
 * Conventions shared by every call:
 *   - Every call returns an lbm_status; nothing throws across the ABI.  After a
 *     failure lbm_last_error(ctx) holds a one-line message.
 *   - Host arrays hold one value per cell, x fastest: index (z * ny + y) * nx + x.
 *     Vector fields are planar: component a of cell c at a * N + c, N = nx * ny * nz.
 *     The caller owns every host buffer; the library copies in or out before it
 *     returns.
 *   - Device state is owned by the context.  It is allocated through the caller's
 *     lbm_allocator (or cudaMalloc when none is given) and released by lbm_destroy.
 *   - All device work runs on the CUDA stream given to lbm_create (0 = the legacy
 *     default stream).  lbm_step only enqueues work; calls that return data to the
 *     host synchronise that stream.
 *   - A context is used by one host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,     /* bad argument: null pointer, size, parameter out of range  */
  LBM_ENOMEM = 2,     /* the allocator returned NULL                               */
  LBM_ECUDA = 3,      /* a CUDA runtime call failed (message in lbm_last_error)    */
  LBM_EUNSTABLE = 4,  /* a non-finite value was found by lbm_reduce                */
  LBM_ETIMEOUT = 5,   /* a bounded device-side wait ran out (reported by the next  */
                      /* lbm_reduce, lbm_step_reduce or lbm_read_fields)          */
  LBM_EBUSY = 6       /* reserved                                                  */
} lbm_status;

/* Grid.  x and y are periodic.  walls_z = 0: z periodic too; walls_z = 1: no-slip
 * walls at z = 0 and z = nz (node k at z = k + 1/2), closed by halfway bounce-back of
 * both f and g.  The paper names the no-slip condition (Sec. III C) but not the scheme;
 * the difference stencils see a ghost layer equal to the adjacent fluid node. */
typedef struct {
  int nx, ny, nz;
  int walls_z;
} lbm_grid;

/* Flags for lbm_params.flags. */
#define LBM_FLAG_BUOYANCY 1u     /* G = (rho - (rho_l + rho_g)/2) g instead of G = rho g  */
#define LBM_FLAG_SRT_FLOW 2u     /* single-relaxation-time flow lattice: every lambda_k
                                    is the viscous rate 1/(nu(phi)/c_s^2 + 1/2), the SRT
                                    special case named after Eq. 10                     */
#define LBM_FLAG_D3Q7_STENCIL 4u /* Eqs. 35-36 with the D3Q7 lattice's weights: 7-point
                                    central differences instead of the 15-point D3Q15
                                    stencil                                             */

/* Storage types of the populations for lbm_params.storage.  Arithmetic is FP32 in
 * every case; phi u, phi and mu stay FP32.  With FP16/BF16 the population f_0 is kept as
 * f_0 - phi (phi of the step that wrote it), since f_0 ~ phi ~ +-1 would lose ~3 decimal
 * digits in 16 bits.  Every storage type works with both patterns. */
#define LBM_STORAGE_FP32 0
#define LBM_STORAGE_FP16 1
#define LBM_STORAGE_BF16 2

/* Population storage patterns for lbm_params.pattern.
 * LBM_PATTERN_AB: two arrays; each step pulls from one and writes the other (176
 *   bytes of FP32 populations per cell).  The batched calls (lbm_batch_*) take these
 *   runs only.
 * LBM_PATTERN_AA: one array updated in place (88 bytes of FP32 populations per cell);
 *   alternate steps read and write neighbouring cells' slots.  On GB300 it runs as
 *   fast as LBM_PATTERN_AB.  Same results either way, bit for bit. */
#define LBM_PATTERN_AB 0
#define LBM_PATTERN_AA 1

/* Physical and lattice parameters (the problem statement of Sec. II). */
typedef struct {
  double rho_l, rho_g; /* phase densities; rho(phi) by Eq. 14, phi = +1 is rho_l      */
  double nu_l, nu_g;   /* kinematic viscosities; nu(phi) = (1+phi)/2 nu_l +
                          (1-phi)/2 nu_g, and lambda_9..13 = 1/(nu(phi)/c_s^2 + 1/2)
                          per cell (Eq. 33, c_s^2 = 1/3)                            */
  double mobility;     /* Mob of Eq. 1; eta = Mob / (A (1/s_1 - 1/2)) by Eq. 19      */
  double D, sigma;     /* interface width and surface tension: kappa = 3 D sigma / 8,
                          beta = 3 sigma / (4 D) (text after Eq. 2)                  */
  double g[3];         /* body acceleration; the external force is G = rho g         */
  double A;            /* free parameter of the D3Q7 weights, 0 < A < 1/3 (Eq. 8)   */
  double sf[7];        /* S^f = diag(s_0..s_6), 0 < s_i < 2, s_1 = s_2 = s_3 (Eq. 10)*/
  double sg[15];       /* S^g = diag(lambda_0..lambda_14), 0 < lambda < 2 (Eq. 26);
                          lambda_9..13 are ignored: they follow nu(phi)              */
  unsigned flags;      /* LBM_FLAG_*; any other bit is LBM_EINVAL                     */
  int storage;         /* LBM_STORAGE_FP32 (default), LBM_STORAGE_FP16, LBM_STORAGE_BF16 */
  int pattern;         /* LBM_PATTERN_AB (default, 0) or LBM_PATTERN_AA               */
} lbm_params;

/* Device allocator.  alloc returns device memory of at least `bytes` bytes (aligned
 * to 256 bytes) or NULL; free releases it.  Calls happen inside lbm_create,
 * lbm_init_phi and lbm_read_fields (one transient staging buffer each, for pageable
 * host buffers only), lbm_read_state_at (the listed cells' buffer) and lbm_destroy
 * only. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} lbm_allocator;

/* Field selection for lbm_read_fields. */
#define LBM_FIELD_PHI 1u
#define LBM_FIELD_RHO 2u
#define LBM_FIELD_P 4u
#define LBM_FIELD_U 8u
#define LBM_FIELD_MU 16u

/* Create a solver for `grid` and `params`.  `alloc` may be NULL (cudaMalloc is then
 * used); `cuda_stream` is a cudaStream_t or NULL.  Fails with LBM_EINVAL when a size
 * is < 1, N = nx ny nz >= 2^31 - 64, a rate is outside (0, 2), s_1..3 differ, A is
 * outside (0, 1/3), a density or viscosity is not positive, or the storage type or
 * pattern is unknown.
 * Device memory per cell: the cell state (22 populations + phi u of the previous
 * step: 100 bytes in FP32, 56 bytes with 16-bit populations; twice for LBM_PATTERN_AB)
 * + phi + mu + 7 staging floats + the fused-sum partials, i.e. about 237 bytes (FP32,
 * AB), 137 bytes (FP32, AA), 149 bytes (16-bit, AB) or 93 bytes (16-bit, AA: the
 * largest admitted grids, 200 GB at 2^31 - 128 cells); lbm_memory_bytes gives the
 * exact figure. */
lbm_status lbm_create(const lbm_grid* grid, const lbm_params* params,
                      const lbm_allocator* alloc, void* cuda_stream, lbm_ctx** out);

/* Initial condition (Sec. III): phi (N values, host) and optionally u (3N, planar)
 * and p (N); NULL means zero.  mu follows from phi by Eq. 2 with the stencil of
 * Eq. 36; f and g are set to their equilibria f^eq (Eq. 5) and g^eq (Eq. 21).  Resets
 * the step count to 0; the first step after it takes d_t(phi u) = 0 (Eq. 34 has no
 * earlier value).  Page-locked inputs are read by the narrowing kernel directly;
 * pageable ones are first copied through a temporary device buffer of N doubles from
 * the context's allocator.  Synchronises the stream. */
lbm_status lbm_init_phi(lbm_ctx* ctx, const double* phi, const double* u, const double* p);

/* Prescribed velocity fields for lbm_set_velocity. */
#define LBM_VELOCITY_NONE 0        /* coupled: u from the flow lattice (default)        */
#define LBM_VELOCITY_UNIFORM 1     /* u = (U, 0, 0)                                      */
#define LBM_VELOCITY_ROTATION 2    /* Eq. 37: rigid rotation about the x axis through the
                                      box centre, Omega = U pi / ny (one turn in 2 ny / U
                                      steps)                                             */
#define LBM_VELOCITY_DEFORMATION 3 /* Eq. 41 with L = nx, times cos(pi t / period), t the
                                      step count                                         */

/* Interface-tracking mode (Sec. III A, B): with kind != LBM_VELOCITY_NONE only the D3Q7
 * lattice evolves (Eq. 4) and u is the prescribed field, evaluated at the integer node
 * coordinates of the (periodic) box; the flow lattice is not used (lbm_reduce reports
 * zero momentum, lbm_read_fields a zero pressure and the prescribed u).  Call before
 * lbm_init_phi, which then starts f from f^eq with the field's u at t = 0 (the u
 * argument is ignored).  LBM_EINVAL for an unknown kind or, for the deformation field, a
 * period <= 0. */
lbm_status lbm_set_velocity(lbm_ctx* ctx, int kind, double U, double period);

/* Advance n >= 0 time steps (Eqs. 4 and 20: stream, then collide in moment space with
 * Eqs. 17-18 and 31-32).  Asynchronous on the context's stream.  Pairs of steps are
 * replayed from CUDA graphs captured on first use (see LBM_TUNE_GRAPHS). */
lbm_status lbm_step(lbm_ctx* ctx, int n);

/* Macroscopic fields at the current time, computed on the device from the current
 * populations: phi (Eq. 13), rho (Eq. 14), p (Eq. 30), u (Eq. 29, planar 3N) and mu
 * (Eq. 2).  Only the fields selected in `mask` are written; the others may be NULL.
 * Values are computed in FP32 and widened to double on the device.  Page-locked
 * buffers (cudaHostAlloc, cudaHostRegister) receive them straight from the widening
 * kernel, which stores into host memory; when any selected buffer is pageable, the
 * values go through n doubles of temporary device memory from the context's allocator
 * (LBM_ENOMEM if refused) and a copy.  Synchronises the stream. */
lbm_status lbm_read_fields(lbm_ctx* ctx, unsigned mask, double* phi, double* rho,
                           double* p, double* u, double* mu);

/* Global sums in FP64 on the device: sum_x phi and sum_x sum_i c_i g_i (the lattice
 * momentum of the current populations).  Summation order is fixed, so results are
 * reproducible run to run.  Returns LBM_EUNSTABLE (sums still written) if any phi or
 * momentum value is not finite.  Synchronises the stream. */
lbm_status lbm_reduce(lbm_ctx* ctx, double* sum_phi, double mom[3]);

/* Advance n >= 1 steps and return the sums of lbm_reduce for the resulting state.  In
 * the coupled model's default variant the last step's stream-collide pass computes them
 * from the values it stores (streaming with bounce-back only permutes post-collision
 * populations, a bounced one re-entering its cell with the opposite velocity), so no
 * extra pass over the state is made; otherwise it runs lbm_step then lbm_reduce.  The
 * 32 cells of a warp are summed in FP32, everything above in FP64 in a fixed order:
 * results are reproducible run to run, and agree with lbm_reduce to the FP32 rounding of
 * those warp sums (about 1e-6 of a warp sum).  Returns LBM_EUNSTABLE (sums still
 * written) if any contribution is not finite.  Synchronises the stream. */
lbm_status lbm_step_reduce(lbm_ctx* ctx, int n, double* sum_phi, double mom[3]);

/* lbm_step_reduce without waiting: the 5 doubles of lbm_reduce_async land in out_dev
 * (same contract) once the stream has passed the n steps. */
lbm_status lbm_step_reduce_async(lbm_ctx* ctx, int n, double* out_dev);

/* The same sums without waiting: enqueued on the context's stream, they land in
 * out_dev[0..4] = {sum phi, momentum x, y, z, number of cells with a non-finite phi or
 * momentum}.  out_dev: 5 doubles, 8-byte aligned, device memory (or host memory the
 * device can write), owned by the caller; valid once the stream has passed this
 * point.  Lets a scheduler watch many runs for divergence without a synchronisation
 * per run.  LBM_EINVAL for NULL or misaligned out_dev or an uninitialised context. */
lbm_status lbm_reduce_async(lbm_ctx* ctx, double* out_dev);

/* Full state in the paper's velocity order (Eqs. 6 and 23): the populations at the
 * current time just after propagation, f (7N) and g (15N), planar by population, and
 * the phi u of the previous step (3N, planar; all zero while no step has been taken
 * since lbm_init_phi).  FP32 exactly as stored.  Any output may be NULL.  `step`
 * receives the step count.  Page-locked outputs are written by the gathering kernel
 * directly, pageable ones through the context's staging plane and a copy.
 * Synchronises the stream. */
lbm_status lbm_read_state(lbm_ctx* ctx, float* f, float* g, float* phiu_prev,
                          long long* step);

/* The same state at `count` listed cells only: cells[k] is the linear index
 * x + nx (y + ny z) of a cell (host array, caller-owned, each in [0, nx ny nz), else
 * LBM_EINVAL and nothing is read); f (7 count), g (15 count) and phiu_prev (3 count)
 * receive the values lbm_read_state gives for those cells, planar by population
 * (f[i count + k] is f_i of cells[k]).  Any output may be NULL; count may be 0.  For
 * probes and for checks on grids whose whole state would not fit in host memory.
 * Uses a device buffer of 108 bytes per listed cell for the call's duration
 * (LBM_ENOMEM if the allocator refuses it).  Synchronises the stream. */
lbm_status lbm_read_state_at(lbm_ctx* ctx, const long long* cells, long long count, float* f,
                             float* g, float* phiu_prev, long long* step);

/* Replace the state (same layout as lbm_read_state).  When phiu_prev is NULL or step
 * is 0, the next step takes d_t(phi u) = 0, as after lbm_init_phi.  Resuming from a
 * state read by lbm_read_state reproduces the original run bit for bit.  Synchronises
 * the stream. */
lbm_status lbm_write_state(lbm_ctx* ctx, const float* f, const float* g,
                           const float* phiu_prev, long long step);

/* Tuning parameters (no effect on results, only on speed).
 * LBM_TUNE_PREFETCH_COLLIDE / LBM_TUNE_PREFETCH_PHI: how many thread blocks ahead the
 * fused stream-collide kernel / the order-parameter kernel prefetch cell data into L2
 * (0 disables).  Default: one wave, the number of SMs times the kernel's resident
 * blocks per SM, set by lbm_create.  LBM_TUNE_PREFETCH_COLLIDE_SUMS: the same distance
 * for the stream-collide kernel of the last step of lbm_step_reduce and
 * lbm_step_reduce_async, which also sums the state it writes and has its own best
 * distance (default: that of LBM_TUNE_PREFETCH_COLLIDE at creation).
 * LBM_TUNE_MU_TMA: 1 (default) lets the chemical-potential pass fetch its halo bricks
 * with TMA tensor copies, 0 uses plain loads; the TMA path exists when nx is a multiple
 * of 32 (and >= 40), ny a multiple of 8 (10 to 524280) and nz is 18 to 1048560, and
 * lbm_get_tuning reports 1 only while it is in use.  Both give identical results.
 * LBM_TUNE_GRAPHS: 1 (default) lets lbm_step replay pairs of steps as CUDA graphs
 * (coupled model, after the first step, while not profiling), 0 launches every kernel;
 * identical results.  LBM_TUNE_TMA_WAIT_POLLS: how many times a block of the TMA
 * chemical-potential pass polls for its copy before giving up (default 2^22, far more
 * than a copy takes); a block that gives up waits once more (2^22 polls) for its copy
 * to land and returns, setting the error word that the next lbm_reduce,
 * lbm_step_reduce or lbm_read_fields reports as LBM_ETIMEOUT, and that step's results
 * are not valid.  If the copy had not landed even then, the call reports LBM_ECUDA
 * instead and retires the context: every later call that launches work on it fails
 * with LBM_ECUDA, and it can only be destroyed.  0 makes every first wait give up at
 * once, which exercises the recoverable path.
 * LBM_TUNE_ROWS: 1 (default) lets the order-parameter and stream-collide passes address
 * the populations they exchange with neighbouring cells a whole row of tiles at a time
 * (the pulls of LBM_PATTERN_AB, the reads and writes of the odd LBM_PATTERN_AA steps),
 * which needs nx a multiple of 32 (lbm_get_tuning reports 1 only while it is in use);
 * 0 keeps the per-cell addressing everywhere.  Identical results.
 * LBM_TUNE_FUSED: 1 runs each step as ONE kernel instead of three (default 0) where it
 * applies -- LBM_PATTERN_AB, the coupled model without LBM_FLAG_SRT_FLOW or
 * LBM_FLAG_D3Q7_STENCIL, nx a multiple of 32 and ny a multiple of 8: every block
 * marches up z through a 32 x 8 column of cells, forming phi (with a 2-cell halo) and
 * mu (1-cell halo) in shared memory a plane or two ahead of the collision, so neither
 * goes through global memory and the 7 f slots are read once (200 B per cell instead
 * of 248 in FP32).  lbm_get_tuning reports 1 only while it applies.  Identical results
 * to the three-kernel step.  LBM_TUNE_FUSED_SEGMENT: planes of z per block (0, the
 * default, chooses by grid size; each segment also forms phi on 2 planes and mu on 1
 * plane beyond each of its ends).  LBM_TUNE_FUSED_PREFETCH: how many planes ahead each
 * block prefetches its tiles into L2 (default 0, off; at most 64).
 * LBM_TUNE_CELL_PAIRS: 1 (default) lets the three-kernel step's stream-collide pass
 * (either pattern) take two cells per thread (cells x and x + 32 of a row, nx a multiple
 * of 64), doing the arithmetic of both in paired FP32 instructions; lbm_get_tuning
 * reports 1 only while it applies.  Identical results.
 * LBM_TUNE_STENCIL_STAGE: 1 (default with FP32 populations; 0 with 16-bit ones, where it
 * is slower) lets that two-cell pass (either pattern), on grids whose rows are 64, 128
 * or 256 cells, fetch the rows of phi and mu its block's stencils need into shared
 * memory with TMA bulk copies (one per row and field) instead of loading each stencil
 * value per cell; its wait for the copies is bounded like the chemical-potential pass's
 * (LBM_TUNE_TMA_WAIT_POLLS, same error reporting).  lbm_get_tuning reports 1 only while
 * it applies.  Identical results.
 * Setting any parameter drops the captured graphs (and waits for the context's
 * stream).
 * lbm_set_tuning returns LBM_EINVAL for an unknown parameter or a value out of range. */
#define LBM_TUNE_PREFETCH_COLLIDE 0
#define LBM_TUNE_PREFETCH_PHI 1
#define LBM_TUNE_MU_TMA 2
#define LBM_TUNE_GRAPHS 3
#define LBM_TUNE_TMA_WAIT_POLLS 4
#define LBM_TUNE_ROWS 5
#define LBM_TUNE_FUSED 6
#define LBM_TUNE_FUSED_SEGMENT 7
#define LBM_TUNE_FUSED_PREFETCH 8
#define LBM_TUNE_CELL_PAIRS 9
#define LBM_TUNE_STENCIL_STAGE 10
#define LBM_TUNE_PREFETCH_COLLIDE_SUMS 11
lbm_status lbm_set_tuning(lbm_ctx* ctx, int param, int value);
lbm_status lbm_get_tuning(const lbm_ctx* ctx, int param, int* value);

/* Number of steps taken since lbm_init_phi / lbm_write_state. */
lbm_status lbm_get_step(const lbm_ctx* ctx, long long* step);

/* Per-kernel timing with CUDA events on the context's stream.  While enabled,
 * lbm_step brackets each kernel launch with events.  lbm_profile_read synchronises,
 * then returns for kernel k (0: order parameter, 1: chemical potential, 2: fused
 * stream-collide, or the single-pass step kernel where LBM_TUNE_FUSED applies) the
 * summed duration in ms and the number of launches since the last lbm_profile(ctx, 1). */
lbm_status lbm_profile(lbm_ctx* ctx, int enable);
lbm_status lbm_profile_read(lbm_ctx* ctx, int kernel, double* total_ms,
                            long long* launches);

/* FP64 sum of an FP32 device array with no memory allocation: out[0] = sum of
 * field[0..n-1], out[1] = number of non-finite values, both written to `out`, a device
 * pointer to 2 doubles.  The paper has no counterpart; this exists for callers that
 * may not allocate device memory when they need the sum -- code running under a fixed,
 * pre-planned memory budget, or inside a framework that forbids cudaMalloc/cudaFree
 * and allocating library calls on its hot path.  It calls none of them: its scratch is
 * a 16 KiB array compiled into the library (held on every GPU that loads it until the
 * process exits).  n must lie in [0, 2^31 - 1], else LBM_EINVAL with a message in
 * lbm_last_error(NULL).  Asynchronous on `cuda_stream`.  The first call on each device
 * looks up the scratch address on that device; make that first call before any stream
 * capture.  The address is kept for the life of the process, so do not call this
 * function again after cudaDeviceReset (or any other teardown of the device's primary
 * context) in the same process.  All calls on a device share the scratch, so calls that
 * overlap on the GPU (other streams, other host threads) race and give wrong sums;
 * serialise them. */
lbm_status lbm_field_sum_noalloc(const float* field, long long n, double* out,
                                 void* cuda_stream);

/* Device bytes lbm_create would allocate for `grid` and `params` (same checks as
 * lbm_create); lets a scheduler admit runs against a memory budget.  Transient
 * staging (lbm_init_phi: n doubles; lbm_read_fields: n doubles) is not included. */
lbm_status lbm_memory_bytes(const lbm_grid* grid, const lbm_params* params, size_t* bytes);

/* Release all device memory of the context and the context itself. */
lbm_status lbm_destroy(lbm_ctx* ctx);

/* ---------------------------------------------------------------------------------
 * Batches: many runs advanced together.  The paper has no counterpart; this serves
 * many simulations on one GPU.  lbm_batch_step(b, runs, n, steps) advances every run
 * by `steps` time steps with one launch per pass per time step for all of them: each
 * launch takes (run, block) work items listed in a device table, and the launches of
 * a batch step are a CUDA graph instantiated once per launch shape (steps, storage
 * type, grid sizes, prefetch distances) and replayed for any run set with that shape.
 * Each run's state comes out bit for bit as lbm_step alone would leave it (same
 * per-cell device code), whatever shares the launch.  Runs need LBM_PATTERN_AB, the coupled model
 * (no prescribed velocity), no LBM_FLAG_SRT_FLOW / LBM_FLAG_D3Q7_STENCIL, one storage
 * type per batch, at most 256 per call, and at least one step taken since lbm_init_phi
 * (the first step, with d_t(phi u) = 0, goes through lbm_step); LBM_EINVAL otherwise.
 * Every run advances by exactly `steps`.  The batch's stream waits for each run's stream
 * and each run's stream then waits for the batch, so batched and single steps mix
 * safely; with cuda_stream NULL the batch uses a stream of its own (graph capture needs
 * one).  A run must not be destroyed before its stream has passed the batch step.
 * Schedule: each pass's work items (blocks of 256 cells; bricks for pass 1) are taken
 * by a persistent grid that strides over them, or by one block per item.
 * lbm_batch_set_grid sets the blocks of pass 0 (order parameter), 1 (chemical
 * potential) or 2 (stream-collide): 1..2^24 persistent blocks, 0 one block per item;
 * defaults 8 and 6 persistent blocks per SM for passes 0 and 1, one block per item for
 * pass 2.  lbm_batch_set_prefetch sets how many items ahead passes 0
 * and 2 prefetch into L2: -1 (default) one wave (the persistent grid, else SMs x
 * resident blocks), 0 off.  lbm_batch_set_split(b, cells): runs of at least `cells`
 * cells are stepped by lbm_step on their own streams instead (they fill the GPU alone,
 * and the single-run kernels take their parameters from the constant bank); the other
 * runs share the batched launches on the batch's stream, and the two overlap.  0
 * (default) sends every run through the shared launches.  Errors:
 * LBM_EINVAL for a refused call (nothing is launched and no run changes), LBM_ECUDA
 * for a failed capture or launch; lbm_batch_last_error says why.
 * --------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(const lbm_allocator* alloc, void* cuda_stream, lbm_batch** out);
lbm_status lbm_batch_step(lbm_batch* b, lbm_ctx* const* runs, int nruns, int steps);
lbm_status lbm_batch_set_grid(lbm_batch* b, int pass, int blocks);
lbm_status lbm_batch_get_grid(const lbm_batch* b, int pass, int* blocks);
lbm_status lbm_batch_set_split(lbm_batch* b, long long cells);
lbm_status lbm_batch_get_split(const lbm_batch* b, long long* cells);
lbm_status lbm_batch_set_prefetch(lbm_batch* b, int pass, int items);
lbm_status lbm_batch_get_prefetch(const lbm_batch* b, int pass, int* items);
lbm_status lbm_batch_destroy(lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* Message of the last failure on ctx ("" if none); for ctx == NULL, the message of the
 * last lbm_create failure in this process. */
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
