/*
 * dbasmppi.h -- C ABI of the GB300 (sm_103a) DBaS-Log-MPPI step.
 *
 * One call of mppi_step() runs one outer-loop body of Algorithm 1 of
 * "Safe Navigation ... DBaS-Log-MPPI" (arXiv 2504.06437) on the GPU for one
 * controller: K perturbed control sequences drawn from the normal-log-normal
 * mixture (Eq. 11) scaled by the exploration rate S_e, rolled out through
 * the dynamics f (Eq. 1, 8) with the discrete barrier state (Eq. 5-7), scored
 * with the DBaS cost-to-go (Eq. 9), combined by min-shifted exponentiated
 * weights (Eq. 4), then the nominal rollout of U* gives C_B and the next S_e
 * (Eq. 10), and the sequence is shifted for the next call.
 *
 * Conventions (all entry points):
 *   - Return 0 (MPPI_OK) on success, a negative MPPI_E* code on failure;
 *     mppi_last_error() then describes the failure (thread-local text).
 *   - The library copies every array it is given; the caller keeps
 *     ownership of its buffers.  A context is owned by the library from
 *     mppi_create() until mppi_destroy(); mppi_destroy(NULL) is a no-op.
 *   - A context is used from one host thread at a time.
 *   - "stream" is a cudaStream_t passed as void*; NULL selects the
 *     context's own stream.  mppi_step*() only enqueue work; the mppi_get_*()
 *     calls synchronise with the stream of the last step.
 *   - Device work that times out on a bounded wait reports MPPI_ETIMEOUT at
 *     the next mppi_get_*() call.
 */
#ifndef DBASMPPI_H
#define DBASMPPI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define MPPI_OK 0
#define MPPI_EINVAL (-1)   /* bad argument: shape, NaN, range */
#define MPPI_ENOMEM (-2)   /* device or pinned allocation failed / admission */
#define MPPI_ECUDA (-3)    /* a CUDA runtime call failed */
#define MPPI_ETIMEOUT (-4) /* a bounded device-side wait expired */
#define MPPI_ESTATE (-5)   /* call out of order (e.g. no step yet) */

/* Dynamics (Eq. 1), explicit Euler with the right-hand side at step k as
 * in Eq. 12 and Eq. 14.  MPPI_UNICYCLE: state (x, y, theta), control
 * (v, omega), x' = x + v cos(theta) dt, y' = y + v sin(theta) dt,
 * theta' = theta + omega dt.  MPPI_QUAD2D: planar quadrotor with the
 * constants of Sec. V-A, state (y, z, phi, ydot, zdot, phidot), control
 * (u1, u2) = thrust deviations with F_i = m g / 2 + u_i.  MPPI_ACKERMANN: the
 * ground vehicle of Eq. 14, state (x, y, theta, v), control (steering phi,
 * acceleration a), theta' = theta + v tan(phi) / wheelbase dt, v' = v + a dt.
 * MPPI_QUAD5: the planar quadrotor of Eq. 12, state (x, z, theta, vx, vz),
 * control (pitch rate omega, thrust deviation u_t), thrust m g + u_t.  The
 * shape points of every model sit at (state[0], state[1]) + R(state[2]) s. */
#define MPPI_UNICYCLE 0
#define MPPI_QUAD2D 1
#define MPPI_ACKERMANN 2
#define MPPI_QUAD5 3
#define MPPI_NUM_MODELS 4
#define MPPI_SGF_MAX_WINDOW 63
#define MPPI_SGF_MAX_ORDER 6

/* Size limits. */
#define MPPI_MAX_T 256        /* horizon */
#define MPPI_MAX_K (1 << 22)  /* samples */
#define MPPI_MAX_OBSTACLES 4096
#define MPPI_MAX_GRID_SIDE 65535
#define MPPI_MAX_GRID_SAMPLES (1 << 26)
#define MPPI_MAX_SHAPE 8      /* shape points per body */
#define MPPI_MAX_COORD 1.0e6  /* |cx|, |cy| and r of an obstacle, metres */
#define MPPI_MIN_H_EPS 1.0e-18 /* smallest accepted h_eps */

/* Problem parameters.  Names follow the paper: K = M samples, T = N horizon,
 * dt (Sec. V), lambda the temperature of Eq. 4 (the cost is divided by it),
 * Sigma_u the 2x2 sampling covariance, (ln_mu, ln_sigma) the log-normal factor
 * of Eq. 11, mu_coarse the coarseness factor mu of Eq. 10 (<= 0 keeps
 * S_e = 1), gamma_ctrl the control-cost gamma of Eq. 9, gamma_bas the gamma
 * in (0,1) of Eq. 7, R_B the barrier-state weight of Eq. 9.  The barrier is
 * B(h) = 1 / max(h, h_eps) with h = |p_i - c_j|^2 - r_j^2 over all shape
 * points i and obstacles j (Eq. 13/15), fused by summation; a step with some
 * h <= 0 is a collision and adds C_coll to the cost.  Q, Qf are the diagonal
 * stage and terminal weights over the n state entries; the control box
 * [u_min, u_max] is G(u) <= 0 of Eq. 2 and is applied by clamping.  x_goal is
 * x_d of Eq. 7.  shape holds n_shape body-frame points (sx, sy), placed at
 * position + R(heading) (sx, sy).  seed keys the Philox4x32-10 generator.
 * mass, inertia, arm, gravity are the quadrotor constants (mass and gravity
 * also for MPPI_QUAD5); wheelbase is L of Eq. 14 (MPPI_ACKERMANN, > 0, whose
 * steering limits must lie inside (-pi/2, pi/2)).
 * sgf_window, sgf_order: Savitzky-Golay smoothing of the weighted
 * perturbation before it is added to U (Algorithm 1 smooths the update this
 * way; the paper gives no window or order).  0 leaves the update unsmoothed.  Otherwise
 * each control channel of the T x 2 update is replaced, at every t, by the
 * value at t of the degree-sgf_order least-squares polynomial through the
 * sgf_window steps centred on t, or through the first or last sgf_window
 * steps within sgf_window / 2 of an end.  sgf_window odd, 3..MPPI_SGF_MAX_WINDOW
 * and <= T; 0 <= sgf_order < sgf_window, sgf_order <= MPPI_SGF_MAX_ORDER. */
typedef struct mppi_params {
  int32_t model;
  int32_t K, T;
  double dt, lambda;
  double sigma[4];
  double ln_mu, ln_sigma;
  double mu_coarse;
  double gamma_ctrl, gamma_bas;
  double R_B, C_coll, h_eps;
  double Q[6], Qf[6];
  double u_min[2], u_max[2];
  double x_goal[6];
  int32_t n_shape;
  double shape[2 * MPPI_MAX_SHAPE];
  uint64_t seed;
  double mass, inertia, arm, gravity;
  double wheelbase;
  int32_t sgf_window, sgf_order;
} mppi_params;

/* Kernel launch shape.  Zero fields are chosen by the library. */
typedef struct mppi_tiling {
  int32_t samples_per_cta;  /* S, 1..32 */
  int32_t threads;          /* 64, 128, 256 or 512 */
  int32_t positions_per_thread; /* 8 or 14 world points per barrier
                                   thread, >= n_shape (whole units) */
  int32_t chunk_steps;      /* reserved: ignored on input, 0 on output */
} mppi_tiling;

typedef struct mppi_ctx mppi_ctx;

/* Create a controller.  u_init: T x 2 initial control sequence (row t =
 * u_t), or NULL for zeros.  S_e starts at mu ln(e) = mu (Eq. 10 with
 * C_B = 0).  Errors: MPPI_EINVAL (sizes beyond the limits, Sigma_u not
 * symmetric positive semi-definite, Sigma_u singular while gamma_ctrl != 0,
 * lambda <= 0, gamma_bas outside (0,1), h_eps < MPPI_MIN_H_EPS, u_min > u_max, non-finite
 * values), MPPI_ENOMEM, MPPI_ECUDA. */
int mppi_create(const mppi_params* p, const double* u_init, mppi_ctx** out);

/* Same, with an explicit launch shape (NULL = automatic). */
int mppi_create_tiled(const mppi_params* p, const double* u_init,
                      const mppi_tiling* tiling, mppi_ctx** out);

/* Replace the obstacle set: the circles {c_j, r_j} of the constraint
 * functions h_j(x) = |p - c_j|^2 - r_j^2 of Eq. 13 (quadrotor) and Eq. 15
 * (vehicle), evaluated at every shape point p of the body, whose barrier
 * terms B(h) = 1/h enter the barrier state of Eq. 7.  cxcyr: J x 3 (centre
 * x, centre y, radius) in the world frame; copied.  J may be 0 (empty set,
 * barrier sum 0).  Errors:
 * MPPI_EINVAL (J < 0, J > MPPI_MAX_OBSTACLES, non-finite value, radius < 0,
 * |cx|, |cy| or r above MPPI_MAX_COORD).
 * Synchronises with the context's last stream before replacing the set. */
int mppi_set_obstacles(mppi_ctx* c, const double* cxcyr, int32_t J);

/* Set or remove the grid map (Sec. V-C: the vehicle plans on a 2D grid map
 * built from its point cloud; the paper does not say how h is read from it).
 * sdf: ny x nx row-major FP32 signed distances (m) to the nearest obstacle,
 * negative inside one; sample (i, j) = sdf[j nx + i] lies at
 * (ox + i res, oy + j res) in the world frame.  The library copies it to
 * device memory.  Every shape point then adds B(h) = 1 / max(h, h_eps) to
 * the circle obstacles' terms (Eq. 13), where h is the bilinear
 * interpolation of the four samples around the point, whose grid coordinates
 * are first clamped to [0, nx - 1] x [0, ny - 1]; h <= 0 counts as a
 * collision.  The same holds for the barrier at the goal (beta_d of Eq. 7),
 * at the measured state and along the nominal rollout.  nx = ny = 0 removes
 * the map (sdf may then be NULL).  The step launches the grid form of the
 * kernel while a map is set.  The controller's own API only: batches and
 * the allocation-free step take circle obstacles.  Errors: MPPI_EINVAL
 * (a side outside [2, MPPI_MAX_GRID_SIDE], more than MPPI_MAX_GRID_SAMPLES
 * samples, a non-finite value, origin or cell size, cell size <= 0, NULL
 * sdf), MPPI_ENOMEM.  Synchronises with the context's last stream before
 * replacing the map. */
int mppi_set_grid(mppi_ctx* c, const float* sdf, int32_t nx, int32_t ny, double ox, double oy,
                  double res);

/* One iteration from host data.  x0: measured state (n doubles).  xref:
 * (T+1) x n reference, row t compared with x_t (row 0 unused), or NULL for
 * x_goal repeated.  Copies the inputs into one of two mapped pinned staging
 * buffers, used in turn, and enqueues the step, whose kernel reads them from
 * host memory over the host link (no separate copy precedes the launch);
 * returns without waiting, and the caller's arrays may be reused at once.
 * A staging buffer is rewritten only after the step that read it has
 * finished: a third call in a row without a synchronisation waits for the
 * first step. */
int mppi_step(mppi_ctx* c, const double* x0, const double* xref, void* stream);

/* One iteration from device data (x0, xref in device memory, same layout;
 * xref must not be NULL).  Enqueues only the step kernel, which writes no
 * host mirror: a following mppi_get_control copies u0 from device memory
 * and synchronises. */
int mppi_step_device(mppi_ctx* c, const double* d_x0, const double* d_xref,
                     void* stream);

/* After a step: u0 = u*_0 (2 doubles), the control Algorithm 1 actuates on
 * the plant after the update (first element of U* of Eq. 4), and, if U is
 * not NULL, the shifted nominal sequence for the next step (T x 2;
 * Algorithm 1's receding-horizon shift, the last element repeated).
 * After mppi_step, u0 and the status word are written by the step itself
 * into mapped pinned host memory, followed (after a system-scope fence) by
 * the step's iteration number.  With U NULL the call then returns as soon
 * as that number shows the last enqueued step, which can be before its
 * kernel has retired; the stream keeps the order of later work.  If the
 * stream ends without it (an error), when U is asked for, or after
 * mppi_step_device, it synchronises with the context's last stream and
 * copies what the mirror does not hold.  Errors: MPPI_ESTATE (no step has run),
 * MPPI_ETIMEOUT (a bounded device wait of the step expired), MPPI_ECUDA. */
int mppi_get_control(mppi_ctx* c, double* u0, double* U);

/* Diagnostics of the last step (any pointer may be NULL):
 * costs[K] (cost-to-go of Eq. 9 per sample), collided[K] (1 if any step of
 * the sample collided), weights[K] (Eq. 4), Ustar[T x 2] (U* before the
 * shift), scalars[8] = {rho, Z, CB_star, S_e_next, beta_used, beta_d,
 * S_e_used, iteration}.  Synchronises. */
int mppi_get_debug(mppi_ctx* c, double* costs, uint8_t* collided,
                   double* weights, double* Ustar, double* scalars);

/* Bytes one mppi_step() moves host -> device (x0 and xref, read by the
 * kernel from the mapped staging) and device -> host for one
 * mppi_get_control(c, u0, NULL) (u0 and the status word, written by the
 * step into the mapped mirror). */
int mppi_io_bytes(mppi_ctx* c, uint64_t* h2d, uint64_t* d2h);

/* Autotuner: runs the step of this problem (params, obstacle set) under
 * each candidate launch shape -- samples per CTA, threads per CTA, world
 * points per barrier thread -- on scratch controllers, at least `iters` timed
 * steps each and enough to cover about 2 ms of device time (CUDA events),
 * and returns the fastest in *best and its time per step
 * in microseconds in *best_us (may be NULL).  Allocates and frees its own
 * scratch controllers; synchronises.  Errors: MPPI_EINVAL, MPPI_ECUDA (no
 * candidate ran). */
int mppi_autotune(const mppi_params* p, const double* cxcyr, int32_t J,
                  int32_t iters, mppi_tiling* best, float* best_us);

/* The same for a controller with a grid map (arguments as mppi_set_grid;
 * sdf NULL = no map, as mppi_autotune): the candidates run the grid form of
 * the step kernel.  Errors: as mppi_autotune, and mppi_set_grid's for the
 * map. */
int mppi_autotune_grid(const mppi_params* p, const double* cxcyr, int32_t J, const float* sdf,
                       int32_t nx, int32_t ny, double ox, double oy, double res, int32_t iters,
                       mppi_tiling* best, float* best_us);

/* The same, timing each candidate's steps the way a caller that steps once
 * per control period sees them: with flush_bytes > 0 every timed step runs
 * alone, after a device-memory write of flush_bytes (an L2 flush when it
 * exceeds the 129 MB L2), between its own pair of events; at least `iters`
 * such steps, at most 40.  flush_bytes = 0 is mppi_autotune_grid (steps back
 * to back).  The small one-wave problems rank their launch shapes
 * differently the two ways.  Errors: as mppi_autotune_grid; MPPI_EINVAL for
 * flush_bytes above 4 GiB, MPPI_ENOMEM if the flush buffer cannot be
 * allocated. */
int mppi_autotune_flush(const mppi_params* p, const double* cxcyr, int32_t J, const float* sdf,
                        int32_t nx, int32_t ny, double ox, double oy, double res, int32_t iters,
                        uint64_t flush_bytes, mppi_tiling* best, float* best_us);

/* The launch shape in use and the number of CTAs of one step. */
int mppi_get_tiling(mppi_ctx* c, mppi_tiling* t, int32_t* n_ctas);

/* Register cap of the step kernel the context launches: 96, or 80 when the
 * grid spans more than one wave of the 96-register form and the lower cap
 * adds resident CTAs per SM (re-chosen on create and on a new obstacle
 * set).  Both forms compute the same results bit for bit.  A library
 * choice with no counterpart in the paper.  Errors: MPPI_ESTATE (NULL
 * context), MPPI_EINVAL (NULL output). */
int mppi_get_kernel_regs(mppi_ctx* c, int32_t* regs_cap);

/* Checkpoint / resume of the per-controller state: U (T x 2), S_e, beta,
 * first-call flag, iteration counter.  Restoring a state reproduces the
 * following steps exactly, since the generator is counter-based. */
int mppi_get_state(mppi_ctx* c, double* U, double* S_e, double* beta,
                   int32_t* first, uint64_t* iter);
int mppi_set_state(mppi_ctx* c, const double* U, double S_e, double beta,
                   int32_t first, uint64_t iter);

/* Diagnostic: the device generator's draws for iteration `iter`, samples
 * k < K and steps t < T, without a context.  raw (K x T x 4, may be NULL)
 * receives the Philox4x32-10 words of counter (k, t, iter_lo, iter_hi) under
 * key (seed_lo, seed_hi); du (K x T x 2, may be NULL) the NLN perturbations
 * of Eq. 11 for exploration rate S_e, before clamping.  Allocates its own
 * device scratch; synchronises.  Errors: MPPI_EINVAL (K*T > 2^26, S_e <= 0,
 * bad params), MPPI_ENOMEM, MPPI_ECUDA. */
int mppi_debug_draws(const mppi_params* p, double S_e, uint64_t iter, int32_t K,
                     int32_t T, uint32_t* raw, float* du);

/* Diagnostic of the bounded device wait that guards the obstacle staging
 * (a bulk copy completing on an mbarrier): one CTA waits on a fresh
 * mbarrier for at most max_cycles SM clock cycles (1 .. 4e9).  With
 * arrive = 1 one thread arrives first, so the wait completes; with
 * arrive = 0 nothing arrives and the bound runs out.  Returns MPPI_OK when
 * the wait completed, MPPI_ETIMEOUT when the bound expired (the device stays
 * usable), MPPI_EINVAL for a bound out of range, MPPI_ECUDA.  Synchronises.
 * The paper has no counterpart; this is test support for the failure path. */
int mppi_debug_wait_probe(int64_t max_cycles, int32_t arrive);

/* One step without any device allocation and without a context, for callers
 * that may not allocate once they run: real-time control loops that keep
 * every step's latency bounded (cudaMalloc can block and synchronise the
 * device) and programs whose device memory belongs to another allocator.
 * The paper has no counterpart; it is the step of mppi_step_device() with its
 * scratch in a fixed 8 MiB array inside the library (each GPU that loads the
 * library keeps it until the process exits).
 *   d_obst   device, J x 3 (cx, cy, r); copied into the scratch.
 *   d_x0     device, n doubles;  d_xref device, (T+1) x n.
 *   d_U      device, T x 2, in/out: the nominal sequence; shifted on return.
 *   d_ctl    device, 5 doubles, in/out: {S_e, beta, first (1 before the
 *            first step, else 0), iteration count, status}; start a
 *            controller with {mu (or 1 if mu <= 0), 0, 1, 0, 0}.  status
 *            becomes 1 if a bounded device wait expired.
 *   d_u0     device out, 2 doubles: u*_0.
 *   d_costs  device out, K doubles, or NULL.
 * All work is enqueued on `stream` (NULL = the legacy default stream); the
 * call returns without waiting.  Set-up happens on first use, not at load:
 * the first call on each device looks up the array's device address (once,
 * under a lock, so host threads may race to it), and the first call for each
 * (device, model, smoothing on or off) sets that step kernel's shared-memory
 * limit and queries its occupancy; a new launch shape queries occupancy
 * again.  Make one such call for every (device, model, smoothing) you will
 * use before any stream capture.  Every call shares the one array: calls
 * whose GPU work overlaps (other streams, other host threads) race; order
 * them.  Errors:
 * MPPI_EINVAL (bad params, NULL pointer, or a problem whose scratch exceeds
 * the 8 MiB limit -- the message gives the bytes needed), MPPI_ECUDA. */
int mppi_step_static(const mppi_params* p, const double* d_obst, int32_t J,
                     const double* d_x0, const double* d_xref, double* d_U,
                     double* d_ctl, double* d_u0, double* d_costs, void* stream);

/* ---- Batched execution.  Many controllers -- mixed model, K, T and
 * obstacle count -- stepped together by one persistent launch: CTAs pull
 * (controller, tile) work items, longest first, from a device work table;
 * the copy-in, the launch and the copy-out are captured in a CUDA graph and
 * replayed while the set of stepped controllers is unchanged.  Each
 * controller's results are identical, bit for bit, to those of a context
 * created with the same launch shape (256 threads per CTA).  Not part of the
 * paper, which steps one controller. */
typedef struct mppi_batch mppi_batch;

/* A batch of at most max_ctrl controllers whose device state comes from one
 * pool of pool_bytes (allocated here).  Errors: MPPI_EINVAL, MPPI_ENOMEM. */
int mppi_batch_create(int32_t max_ctrl, size_t pool_bytes, mppi_batch** out);

/* Admit a controller: parameters as for mppi_create, launch shape (NULL or
 * zero fields = automatic; threads is always 256), obstacle set (J x 3,
 * copied; J may be 0).  *slot receives its id.  MPPI_ENOMEM when no slot is
 * free or the pool cannot hold its state and obstacles (admission refusal;
 * nothing changes). */
int mppi_batch_add(mppi_batch* b, const mppi_params* p, const double* u_init,
                   const mppi_tiling* tiling, const double* cxcyr, int32_t J,
                   int32_t* slot);

/* Replace the obstacle set of one controller, as mppi_set_obstacles; a
 * larger set than the slot holds moves it within the pool (MPPI_ENOMEM if
 * the pool has no room for the larger copy). */
int mppi_batch_set_obstacles(mppi_batch* b, int32_t slot, const double* cxcyr,
                             int32_t J);

/* Release a controller's slot and its pool memory. */
int mppi_batch_remove(mppi_batch* b, int32_t slot);

/* One iteration of the n listed controllers (each at most once).  x0s:
 * n x 6 doubles (the first n_state of each row are used); xrefs: NULL, or n
 * pointers each to a (T+1) x n_state reference or NULL (goal repeated).
 * Copies the inputs; enqueues the step and returns. */
int mppi_batch_step(mppi_batch* b, const int32_t* slots, int32_t n,
                    const double* x0s, const double* const* xrefs, void* stream);

/* u*_0 of the controllers of the last step, in the order listed (n x 2).
 * Synchronises. */
int mppi_batch_get_controls(mppi_batch* b, double* u0s, int32_t n);

/* One controller's shifted sequence (T x 2), costs of its last step (K) and
 * scalars[8] as in mppi_get_debug (any pointer may be NULL).  Synchronises. */
int mppi_batch_get_state(mppi_batch* b, int32_t slot, double* U, double* costs,
                         double* scalars);

/* Launch shape and pool bytes of a slot (slot < 0: none) and the pool's free
 * bytes. */
int mppi_batch_info(mppi_batch* b, int32_t slot, mppi_tiling* t, uint64_t* bytes,
                    uint64_t* pool_free_bytes);

/* Enable (default) or disable CUDA-graph capture and replay of the step. */
int mppi_batch_set_graph(mppi_batch* b, int32_t enable);

/* Tiling policy of a batch: the launch shape given to controllers that
 * mppi_batch_add receives without an explicit tiling, per model (index
 * MPPI_UNICYCLE .. MPPI_QUAD5).  samples_per_cta in 1..32 (capped at K);
 * positions_per_thread 8 or 14, or 0 to choose from n_shape.  The batch
 * kernel's CTAs have 256 threads.  Default: {32, 32}, {0, 0}. */
typedef struct {
  int32_t samples_per_cta[MPPI_NUM_MODELS];
  int32_t positions_per_thread[MPPI_NUM_MODELS];
} mppi_batch_policy;

/* Set or read the policy used by later mppi_batch_add calls (controllers
 * already added keep their shape).  Errors: MPPI_EINVAL (out of range). */
int mppi_batch_set_policy(mppi_batch* b, const mppi_batch_policy* pol);
int mppi_batch_get_policy(const mppi_batch* b, mppi_batch_policy* pol);

/* Autotuner of the batched step.  For n representative controllers
 * (parameters ps[i], obstacles cxcyrs[i] with Js[i] rows), each model's
 * policy in turn is chosen from samples_per_cta {8, 16, 32} x
 * positions_per_thread {8, 14} (the other models' held at their best so far;
 * models absent from the set are skipped):
 * for each candidate a temporary batch of pool_bytes holds all n
 * controllers, and `iters` graph-replayed steps of all of them (each from
 * its x_goal) are timed with CUDA events after two untimed ones.  best
 * receives the fastest policy and best_ms (may be NULL) its time per step.
 * Candidates that do not fit the pool or the kernel are skipped.  Errors:
 * MPPI_EINVAL, MPPI_ENOMEM (not even the default fits), MPPI_ECUDA. */
int mppi_batch_autotune(const mppi_params* ps, const double* const* cxcyrs,
                        const int32_t* Js, int32_t n, int32_t iters, size_t pool_bytes,
                        mppi_batch_policy* best, float* best_ms);

/* Release the batch and its pool.  NULL is a no-op. */
int mppi_batch_destroy(mppi_batch* b);

/* ---- Serving runtime: continuous batching of control-step requests from
 * many robots.  Robots join by taking a slot of a device pool (admission by
 * memory) and keep their warm-start sequence, generator counter, exploration
 * rate and barrier state on the device.  A scheduler thread keeps up to
 * `lanes` batched steps in flight, each on its own stream; when a lane is
 * free it launches one persistent batch of queued requests, so requests that
 * arrive while others run are served by the next batch and the batches
 * overlap on the device.  Under a size-class policy (mppi_server_set_policy)
 * small and large requests have their own queues and lanes, batches are
 * bounded by work, and the large-request kernels leave part of the GPU to
 * the small ones.  Each result equals, bit for bit, the robot's result alone
 * through a context with the same launch shape.  Not part of the paper. */
typedef struct mppi_server mppi_server;

/* Scheduling policy of a server.  The work of a request is
 * K T (7 P J + 135) FP32 operations (its samples, steps, shape points and
 * obstacles).
 *   small_ops_max    requests of at most this work are small, the rest
 *                    large; 0 = one class (every lane serves one queue).
 *   small_lanes      lanes that serve the small class (the others serve the
 *                    large class), at least 1 and at most lanes - 1; used
 *                    when small_ops_max > 0 and lanes >= 2.
 *   large_share      in (0, 1]: the large-class kernels use at most this
 *                    fraction of the CTAs the GPU holds at once, so that the
 *                    rest of the SMs stay free for small requests.
 *   batch_ops_small, batch_ops_large
 *                    work cap of one batch of each class (requests are taken
 *                    in queue order up to the cap; a request above it goes
 *                    alone); 0 = no cap.
 *   shortest_first   0: each class's queue is served oldest first; 1: least
 *                    work first, except that requests queued longer than
 *                    max_wait_s go first, oldest first (0 = no such limit).
 *   max_wait_s       see shortest_first.
 *   device_queue     0: the lanes above.  1: one resident persistent kernel
 *                    serves every request: the scheduler publishes each
 *                    request's tiles into a ring in mapped host memory that
 *                    the running kernel claims from, small requests' tiles
 *                    first, so a request that arrives mid-flight joins the
 *                    running kernel at the next tile boundary; the
 *                    scheduler closes the kernel after 0.3 ms with nothing
 *                    queued or in flight and launches it again when work
 *                    arrives.  small_ops_max sets the classes;
 *                    small_lanes and large_share do not apply; the batch
 *                    caps bound each class's published, unfinished work
 *                    (requests beyond it wait on the host), and
 *                    shortest_first / max_wait_s order the requests so
 *                    held.  The poll's queue time is then submission to
 *                    publication and its device time publication to
 *                    completion (host clock). */
typedef struct {
  double small_ops_max;
  int32_t small_lanes;
  int32_t shortest_first;
  double large_share;
  double batch_ops_small, batch_ops_large;
  double max_wait_s;
  int32_t device_queue;
  int32_t reserved;
} mppi_server_policy;

/* A server of at most max_robots robots whose state lives in a pool of
 * pool_bytes, with `lanes` (1..8) launch lanes, one class of requests and
 * no work caps until a policy is set.  Errors: MPPI_EINVAL, MPPI_ENOMEM,
 * MPPI_ECUDA. */
int mppi_server_create(int32_t max_robots, size_t pool_bytes, int32_t lanes,
                       mppi_server** out);

/* Set the scheduling policy (copied).  Only while no request is queued or
 * in flight (MPPI_ESTATE otherwise).  Errors: MPPI_EINVAL (negative or
 * non-finite work values, large_share outside (0, 1], small_lanes < 1,
 * shortest_first or device_queue not 0 or 1, max_wait_s negative or
 * non-finite), MPPI_ENOMEM (the device queue's mapped rings). */
int mppi_server_set_policy(mppi_server* s, const mppi_server_policy* pol);

/* The policy in force and, if lane_classes is not NULL, the class each lane
 * serves (lanes entries: 0 small or the only class, 1 large). */
int mppi_server_get_policy(mppi_server* s, mppi_server_policy* pol,
                           int32_t* lane_classes);

/* Admit a robot (parameters, initial sequence or NULL, obstacle set).
 * MPPI_ENOMEM: no free slot or no room in the pool now (retry after others
 * leave). */
int mppi_server_join(mppi_server* s, const mppi_params* p, const double* u_init,
                     const double* cxcyr, int32_t J, int32_t* robot);

/* Release a robot's slot (MPPI_ESTATE if it has a request in flight). */
int mppi_server_leave(mppi_server* s, int32_t robot);

/* Queue one step request: measured state x0 (n doubles), reference
 * ((T+1) x n) or NULL (goal repeated); copied.  One request per robot at a
 * time (MPPI_ESTATE otherwise).  Thread-safe; returns at once. */
int mppi_server_submit(mppi_server* s, int32_t robot, const double* x0,
                       const double* xref);

/* Up to max completed requests, oldest first: robot ids, u0 (2 each), the
 * model-predicted next state (6 each), latency from submission in seconds,
 * status (MPPI_OK or the error of the launch).  *n receives the count.
 * Any output pointer but n may be NULL. */
int mppi_server_poll(mppi_server* s, int32_t max, int32_t* robots, double* u0s,
                     double* x1s, double* latency_s, int32_t* status, int32_t* n);

/* The same, with the latency split: queue_s = submission to the launch of
 * the request's batch (host clock), device_s = that batch's time on the GPU
 * from its copy-in to its copy-out (CUDA events), size_class = 0 small (or
 * the only class), 1 large. */
int mppi_server_poll_timed(mppi_server* s, int32_t max, int32_t* robots, double* u0s,
                           double* x1s, double* latency_s, double* queue_s,
                           double* device_s, int32_t* size_class, int32_t* status,
                           int32_t* n);

/* Counters: batches launched, requests completed, requests queued or in
 * flight, free pool bytes. */
int mppi_server_stats(mppi_server* s, uint64_t* batches, uint64_t* requests,
                      int32_t* pending, uint64_t* pool_free_bytes);

/* Stop the scheduler, wait for work in flight, release everything. */
int mppi_server_destroy(mppi_server* s);

/* Release everything owned by the context.  NULL is a no-op. */
int mppi_destroy(mppi_ctx* c);

/* Text of the last error on this host thread ("" if none). */
const char* mppi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DBASMPPI_H */
