/*
 * at.h -- C ABI of the GB300 weakly-synchronous AT Burgers solver.
 *
 * The library advances the viscous Burgers' equation u_t + u u_x = nu u_xx
 * (+ A sin x) on a periodic 1D grid with forward Euler (arXiv 1911.05769,
 * Eq. BS and Sec. 3.2).  The grid of N points is split into P subdomains of
 * M = N/P points, the paper's processing elements.  Interior points use the
 * standard central stencil of order 2 or 4; points next to a subdomain
 * boundary use asynchrony-tolerant (AT) stencils (Eq. AT1 / Eq. AT2): each
 * halo value at level n is approximated from the neighbour's delayed levels
 * n-k, n-k-1 (order 2) or n-k, n-k-1, n-k-2 (order 4), with 0 <= k <= L.
 *
 * On the GPU the subdomains are processed by the CTAs of one persistent,
 * cooperatively launched kernel.  Halo values travel through a ring buffer of
 * past boundary values in device memory with one progress flag per
 * subdomain face (the device counterpart of the notified puts and circular
 * receive buffers of Algorithm 2), so CTAs run ahead of one another by up to
 * L steps without a grid-wide barrier.  AT_SYNC instead puts a grid barrier
 * after every step (Algorithm 1).
 *
 * Memory and ownership.  The library never allocates device memory.  The
 * caller allocates one workspace of at_workspace_bytes() bytes (device
 * memory, 256-byte aligned) and passes it, with a CUDA stream, in at_grid.
 * The workspace holds the state u, the ring buffers, the progress flags and
 * the device status; it is borrowed until at_destroy().  Every call that
 * launches work is asynchronous and ordered on that stream unless it says it
 * synchronises.
 *
 * Errors.  Every int-returning call returns AT_OK (0) or a negative AT_ERR_*
 * code and leaves a message for at_last_error() (per thread).  A device wait
 * that exceeds timeout_ns latches AT_ERR_TIMEOUT in the workspace; every
 * kernel then stops early and the next synchronising call (at_state,
 * at_status, at_delay_stats) returns it.  The CUDA context stays usable.
 */
#ifndef AT_H
#define AT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define AT_OK             0
#define AT_ERR_ARG       (-1)  /* invalid argument (message says which)          */
#define AT_ERR_UNSTABLE  (-2)  /* nu dt / dx^2 above the stability limit         */
#define AT_ERR_RESIDENCY (-3)  /* the CTAs cannot all be resident at once        */
#define AT_ERR_CUDA      (-4)  /* a CUDA runtime call failed                     */
#define AT_ERR_TIMEOUT   (-5)  /* a device wait ran out of time (latched)        */
#define AT_ERR_STATE     (-6)  /* call out of order (e.g. at_step before state)  */

/* state and ring storage type (the arithmetic type of the stencil) */
#define AT_F64 0
#define AT_F32 1

/* boundary condition */
#define AT_BC_PERIODIC   0  /* periodic domain (the paper's setting, Sec. 3.2)     */
#define AT_BC_EXACT_TANH 1  /* ensembles only: points outside the domain take the
                               exact travelling-wave values at the current level,
                               undelayed (see at_instance)                        */

/* delay modes of at_step (Sec. 2 delay model; Algorithms 1 and 2) */
#define AT_SYNC   0  /* k = 0 everywhere, grid barrier every step (Alg. 1);    */
                     /* with steps_per_pass > 1: every pass (ghost cells)     */
#define AT_SEEDED 1  /* k prescribed by SplitMix64(seed) per (n, p, face)      */
#define AT_FREE   2  /* k = how far the neighbour lags, waiting only if > L    */
#define AT_REPLAY 3  /* k read from a caller array                             */

/* at_grid.flags */
#define AT_FLAG_PER_SUBDOMAIN_DELAY 1  /* SEEDED: one draw for both faces       */
#define AT_FLAG_ALLOW_UNSTABLE      2  /* skip the stability check of at_create */
#define AT_FLAG_TEST_SKIP_PUBLISH   4  /* test only: CTA 0 stops publishing its
                                          progress flags after level test_skip_step,
                                          so that its neighbours' waits time out
                                          (1D: its first warp; 3D: its subdomains) */
#define AT_FLAG_VISCOUS_FP64        8  /* FP32 state: form the viscous term nu dt D2 u
                                          and add it to u in FP64 (one rounding per
                                          update).  Chosen automatically when
                                          nu dt / dx^2 >= 0.8 x the stability limit */
#define AT_FLAG_VISCOUS_FP32       16  /* FP32 state: never use FP64 for it */
#define AT_FLAG_COMPENSATED        32  /* FP32 state (1D: single domain and
                                          ensembles): every value is a pair hi + lo
                                          of FP32 words (lo: the rounding error of
                                          hi); stencil differences and halo values
                                          are formed word by word, ring entries carry
                                          both words, and each update is added with
                                          an error-free two-sum, so that neither
                                          increments far below an ulp nor the
                                          quantisation of the stored field are lost;
                                          doubles the state memory and traffic;
                                          at_state returns hi; not with the adjoint,
                                          at_set_history or at_step_noalloc */

typedef struct at_solver at_solver;   /* opaque handle */

/* Problem and execution description (the "grid" argument of at_create).
 * Zero-initialise it and set the fields that apply. */
typedef struct at_grid {
  int32_t  dim;             /* 1, or 3 (scalar 3D Burgers, order 2; see below)     */
  int32_t  bc;              /* AT_BC_PERIODIC                                      */
  int32_t  dtype;           /* AT_F64 or AT_F32                                    */
  int32_t  flags;           /* AT_FLAG_*                                           */
  int64_t  n[3];            /* grid points per dimension; n[0] = N                 */
  double   length[3];       /* domain length; x_i = origin + i * length / N        */
  double   origin[3];       /* domain origin                                       */
  double   forcing_amp;     /* A of the forcing A sin(x); 0 = unforced (Eq. BS)    */
  uint64_t seed;            /* seed of AT_SEEDED delays                            */
  void    *workspace;       /* device memory, >= at_workspace_bytes(), 256-aligned */
  size_t   workspace_bytes;
  void    *stream;          /* cudaStream_t (NULL = legacy default stream)         */
  int64_t  timeout_ns;      /* bound of every device wait; 0 = 1 s                 */
  int32_t  max_ctas;        /* CTAs: 0 = all that can be resident at once (capped */
                            /* at P); else this many (AT_ERR_RESIDENCY if they    */
                            /* cannot all be resident)                            */
  int32_t  stages;          /* tile buffers per warp: 0 = 3; at least 2; fewer if */
                            /* shared memory cannot hold them                     */
  int64_t  test_skip_step;  /* level after which AT_FLAG_TEST_SKIP_PUBLISH acts    */
  int32_t  steps_per_pass;  /* levels advanced per pass over a tile (temporal      */
                            /* blocking), 0 or 1 = none, at most L+1.  AT_FREE:   */
                            /* halos of inner levels extrapolated with delay     */
                            /* k0 + i.  AT_SYNC: a grid barrier per pass, every  */
                            /* delay 0, the halos of inner levels recomputed     */
                            /* from the neighbours' edge strips of R x levels     */
                            /* points (ghost cells), bit for bit the result of    */
                            /* a barrier every step; the count is reduced until  */
                            /* a strip fits 16 words, 64 bytes and one subdomain */
                            /* (one level per pass with AT_FLAG_COMPENSATED).  3D:*/
                            /* AT_FREE only, see the 3D section below             */
  int32_t  tile_subdomains;  /* ensembles: subdomains per tile (0 or 1: one; 2 or  */
                            /* 4 with M of 128, 256 or 512 and K M <= 1024): in   */
                            /* AT_FREE and AT_SYNC a tile advances K consecutive  */
                            /* subdomains of an instance together, the faces      */
                            /* between them at delay 0 (recorded as such);        */
                            /* AT_SEEDED and AT_REPLAY take one subdomain per     */
                            /* tile.  Single domain: must be 0                    */
  int64_t  sub[3];          /* dim 3: points per subdomain along x, y, z; n[a] a  */
                            /* multiple of sub[a]; P = product of n[a] / sub[a]   */
} at_grid;

/* Launch facts of a solver, for tests and benchmarks. */
typedef struct at_info {
  int64_t N, P, M;          /* points, subdomains, points per subdomain            */
  int32_t order, L;         /* stencil order, maximal delay                        */
  int32_t R, s;             /* stencil radius, levels per halo approximation       */
  int32_t T;                /* ring slots (levels kept per boundary)               */
  int32_t ctas;             /* CTAs of the persistent kernel (3D with              */
                            /* steps_per_pass > 1: those of the blocked AT_FREE   */
                            /* kernel, as threads, stages and smem_bytes)         */
  int32_t threads;          /* threads per CTA                                     */
  int32_t stages;           /* tile buffers per warp (3D: plane buffers per CTA)   */
  int64_t smem_bytes;       /* dynamic shared memory per CTA                       */
  int64_t step;             /* time level of the state (steps taken)               */
  int32_t sm_count;         /* SMs of the device                                   */
  int32_t dtype;            /* AT_F64 or AT_F32                                    */
  int32_t steps_per_pass;   /* levels per pass (AT_FREE; AT_SYNC as reduced above) */
  int32_t viscous_fp64;     /* 1 if the viscous term is accumulated in FP64        */
  int32_t tile_subdomains;  /* ensembles: subdomains per tile in AT_FREE / AT_SYNC  */
} at_info;

/* Bytes of workspace needed for this problem, or 0 if the arguments are
 * invalid (see at_last_error()).  Host only; no CUDA call. */
size_t at_workspace_bytes(const at_grid *grid, int64_t P, int scheme_order, int L);

/* Creates a solver for N = grid->n[0] points split into P subdomains, central
 * stencils of order scheme_order (2 or 4, Sec. 3.2) with AT boundary stencils
 * (Eq. AT1/AT2; order 4 extrapolates quadratically in time), maximal delay L
 * (0..16, Sec. 2 and Algorithm 2), viscosity nu >= 0 and time step dt > 0.
 * Requires N % P == 0, M = N/P a multiple of 4 with 4 <= M <= 1024,
 * and nu dt / dx^2 <= 1/2 (order 2) or 3/8 (order 4) unless
 * AT_FLAG_ALLOW_UNSTABLE.  Checks that the kernel's CTAs can be co-resident.
 * The state is undefined until at_set_state().  *out receives the handle. */
int at_create(const at_grid *grid, int64_t P, int scheme_order, int L,
              double nu, double dt, at_solver **out);

/* Sets the state (time level 0) from u: N contiguous words of the grid's
 * dtype, in host or device memory.  Resets the step counter, the ring
 * buffers, the progress flags, the delay statistics and the device status.
 * Stream-ordered; a host source is copied before the call returns. */
int at_set_state(at_solver *h, const void *u);

/* Advances the state by n_steps >= 0 forward-Euler steps in one persistent
 * kernel launch on the grid's stream (asynchronous, no host synchronisation:
 * it may be captured into a CUDA graph).  The time level of the state is kept
 * in the workspace and advanced by the kernel itself, so every replay of a
 * captured graph continues from the level the previous replay reached.
 *   delay_mode: AT_SYNC, AT_SEEDED, AT_FREE or AT_REPLAY.
 *   delays:     device array int8 [n_steps][P][2] (face 0 = left neighbour
 *               p-1, face 1 = right neighbour p+1).  AT_REPLAY reads the delays
 *               from it (values 0..L; they are clamped to n-s+1 during start-up,
 *               as the oracle does).  In the other modes, if not NULL, it
 *               receives the delays actually used.  NULL is an error for
 *               AT_REPLAY.
 * Device waits are bounded by timeout_ns; see at_status(). */
int at_step(at_solver *h, int64_t n_steps, int delay_mode, int8_t *delays);

/* Copies the state (N words) to dst (host or device memory), waits for the
 * stream and returns the device status: AT_OK or AT_ERR_TIMEOUT. */
int at_state(at_solver *h, void *dst);

/* Compensated state (AT_FLAG_COMPENSATED) only: copies the N lo words -- the
 * rounding errors of the words at_state() returns, so that hi + lo is the
 * value the solver carries -- to dst (host or device memory), waits for the
 * stream and returns the device status.  AT_ERR_ARG without a compensated
 * state.  (An extension of at_state for the precision variant; the paper
 * has no counterpart.) */
int at_state_error(at_solver *h, void *dst);

/* Waits for the stream and returns the device status. */
int at_status(at_solver *h);

/* Delay statistics since at_set_state(): hist[0..L] counts the delays used
 * per (level, subdomain, face); mean_k and mean_k2 are <k> and <k^2>, the
 * moments of Eq. err_scaling.  Any pointer may be NULL.  Synchronises. */
int at_delay_stats(at_solver *h, int64_t *hist, double *mean_k, double *mean_k2);

/* Fills *info with the launch facts of the solver.  info->step is read from
 * the device (waiting for the stream) unless the stream is being captured;
 * then it counts the steps of the at_step calls made so far. */
int at_get_info(const at_solver *h, at_info *info);

/* Releases the handle (host memory only; the workspace stays the caller's). */
int at_destroy(at_solver *h);

/* Message of the last failed call on this thread ("" if none). */
const char *at_last_error(void);

/* ---------------------------------------------------------------------------
 * Three dimensions (grid->dim = 3): u_t + u (u_x + u_y + u_z) = nu lap u on a
 * periodic box of n[0] x n[1] x n[2] points (x fastest in memory), split into
 * subdomains of sub[0] x sub[1] x sub[2] points (sub[0] a multiple of 4,
 * sub[0] * sub[1] <= 1024, sub[2] >= 3), numbered (p2 P1 + p1) P0 + p0.
 * Order-2 central differences along each axis; a neighbour across any of the
 * six faces (0: -x, 1: +x, 2: -y, 3: +y, 4: -z, 5: +z) is extrapolated from the
 * levels n-k, n-k-1 of the neighbouring subdomain (Eq. AT1/AT2) with a delay
 * per (level, subdomain, face); AT_SEEDED draws it at counter (n P + p) 6 +
 * face.  at_create's P must equal the number of subdomains; scheme_order must
 * be 2.  The delay arrays of at_step are [n_steps][P][6].  Stability limit
 * for at_create: nu dt (1/dx^2 + 1/dy^2 + 1/dz^2) <= 1/2.
 * Temporal blocking (scalar equation, AT_FREE): grid->steps_per_pass b in
 * 2 .. min(L+1, 4) with sub[0] a power of two in 4..128 advances each
 * subdomain b levels per pass (the pass from level 0: one level) in a
 * wavefront along z; the halo of level n + j of a pass is extrapolated from
 * the neighbour's newest published level s <= n and s - 1 with delay
 * n + j - s, so a pass waits only until that delay stays within L.  Delays
 * are recorded per level as for one level per pass; AT_SEEDED, AT_REPLAY and
 * AT_SYNC calls of the same solver take one level per pass.  Its shared
 * memory (6 b halo faces, 2 (b - 1) planes, the plane stages) must fit one
 * CTA, else at_create fails with AT_ERR_RESIDENCY.  No forcing, ensembles,
 * adjoint or autotuner in 3D; the system below takes one level per pass.
 * --------------------------------------------------------------------------- */

/* The full system of Eq. BS in 3D: velocity components u, v, w and 0..2
 * passive scalars phi_k, nfields = 3..5 fields stored one after another
 * (field-major, each n[0] x n[1] x n[2] with x fastest):
 *     d_t q_f + u d_x q_f + v d_y q_f + w d_z q_f = kappa[f] lap q_f
 * with kappa[0..2] the viscosity nu and kappa[3..] the scalars'
 * diffusivities alpha_k (Eq. BS).  Same grid, subdomains (sub[0] * sub[1] <=
 * 512, or exactly 1024 with FP32 state and sub[0] a multiple of 4), order-2 stencils, AT halos and delays as the scalar 3D solver; one
 * delay per (level, subdomain, face) serves every field (one message per face
 * carries all fields).  The state and at_set_state / at_state buffers hold
 * nfields x n[0] n[1] n[2] words; at_info reports that as N. */
size_t at_system_workspace_bytes(const at_grid *grid, int64_t P, int L, int nfields);
int at_create_system(const at_grid *grid, int64_t P, int L, int nfields, const double *kappa, double dt,
                     at_solver **out);

/* Mean and mean square of every field of a 3D solver's state (the one-point
 * moments whose statistics the paper follows): out[2 f] = <q_f>,
 * out[2 f + 1] = <q_f^2>, summed in FP64.  Synchronises; returns the device
 * status. */
int at_moments(at_solver *h, double *out);

/* ---------------------------------------------------------------------------
 * Ensembles: many independent 1D problems advanced by one persistent launch.
 *
 * Instance j has n_j points (a multiple of the common subdomain size M, so
 * n_j / M subdomains of M points), its own viscosity, time step, delay bound
 * L_j and seed, and either a periodic domain or exact travelling-wave
 * boundary values: with AT_BC_EXACT_TANH the points just outside
 * [origin, origin + length) take u = c - a tanh(a (x - xc - c t) / (2 nu)),
 * the viscous Burgers travelling wave, at t = n dt (undelayed).  Inside an
 * instance the method is that of at_create: central stencils, AT stencils
 * at subdomain faces, delays per (level, subdomain, face).  With AT_SEEDED
 * the delays of instance j are those of a single-domain solver with
 * P = n_j / M, L = L_j and seed = seed_j.  The instances' subdomains are laid
 * end to end: the state is the concatenation of the instances' fields
 * (instance 0 first), N = sum n_j words, P = N / M subdomains in all.  A
 * processing element (warp) may hold subdomains of several instances; its
 * passes in AT_FREE are then no longer than the smallest L_j among them + 1.
 * The paper treats one domain; ensembles are an extension.
 * --------------------------------------------------------------------------- */
typedef struct at_instance {
  int64_t  n;               /* points of the instance (multiple of M)              */
  int32_t  L;               /* maximal delay of the instance, 0..16                */
  int32_t  bc;              /* AT_BC_PERIODIC or AT_BC_EXACT_TANH                  */
  double   length, origin;  /* domain [origin, origin + length); dx = length / n  */
  double   nu, dt;          /* viscosity (> 0 for AT_BC_EXACT_TANH), time step    */
  double   tanh_a, tanh_c, tanh_xc;  /* a, c, xc of the exact boundary values     */
  uint64_t seed;            /* AT_SEEDED seed of the instance                      */
} at_instance;

/* Workspace bytes for an ensemble, or 0 if the arguments are invalid. */
size_t at_batch_workspace_bytes(const at_grid *grid, int64_t n_inst, const at_instance *inst, int64_t M,
                                int scheme_order);

/* Creates a solver for the ensemble inst[0 .. n_inst-1] (host array, read
 * during the call) with subdomains of M points (a multiple of 4, 4..1024)
 * and stencil order scheme_order.  From grid it uses dtype, flags,
 * workspace, stream, timeout_ns, max_ctas, stages and steps_per_pass (at
 * most max L_j + 1); forcing_amp must be 0.  Copies the instance tables into
 * the workspace and waits for the stream.  The returned handle takes the
 * calls of a single-domain solver (at_set_state with N words, at_step with a
 * [n_steps][P][2] delay array over all subdomains, at_state, ...); at_info
 * reports the total N and P and L = max L_j. */
int at_create_batch(const at_grid *grid, int64_t n_inst, const at_instance *inst, int64_t M, int scheme_order,
                    at_solver **out);

/* ---------------------------------------------------------------------------
 * Autotuner.  Launch shapes of the persistent kernel: CTAs (1 up to the
 * resident limit per SM, times the SM count: so the processing elements per
 * subdomain), tile buffers per warp (2..4) and levels per pass: for AT_FREE
 * 1 .. L + 1 (in an ensemble each processing element then takes at most its
 * own smallest delay bound + 1); for AT_SYNC 1 .. L + 1 only if the solver
 * was created with steps_per_pass > 1 (the blocked synchronous mode), else 1.
 * --------------------------------------------------------------------------- */
typedef struct at_tune_result {
  int32_t ctas, stages, steps_per_pass;   /* the fastest shape                     */
  int32_t n_tried;                        /* shapes timed                          */
  double  best_ms;                        /* its time for at_step(n_steps)          */
  double  first_ms;                       /* time of the shape the solver had      */
  int32_t tile_subdomains;                /* ensembles: subdomains per tile        */
  int32_t pad_;
} at_tune_result;

/* Times at_step(h, n_steps, delay_mode, NULL) for every launch shape above
 * (one untimed launch, then the best of two timed ones, CUDA events on the
 * solver's stream) and keeps the fastest on the handle.  This runs the
 * solver: the state advances by 3 n_steps per shape, so set the state again
 * before a production run.  Synchronises; not for use under stream capture.
 * Returns AT_OK, or the first error (then the handle keeps its shape). */
int at_tune(at_solver *h, int64_t n_steps, int delay_mode, at_tune_result *res);

/* ---------------------------------------------------------------------------
 * Levels, restarts and the discrete adjoint (single-domain solvers).
 *
 * The paper's method maps (u^0, nu) to u^n; these calls give the gradient of
 * a scalar J(u^{n_steps}) with respect to u^0 and nu by reverse-mode
 * differentiation of exactly that discrete map (forward Euler, Sec. 3.2;
 * central stencils; AT halos of Eq. AT1/AT2 with the run's delays): checkpoints
 * every `interval` levels on the forward run, each interval recomputed from its
 * checkpoint on the way back.  The paper has no adjoint; this is an extension.
 * --------------------------------------------------------------------------- */

/* as at_step, and also writes every level l it computes (n0+1 .. n0+n_steps)
 * into levels + (l mod depth) * N words (device memory).  Passes are one level
 * long in every mode. */
int at_step_levels(at_solver *h, int64_t n_steps, int delay_mode, int8_t *delays, void *levels, int64_t depth);

/* Restarts the solver at time level `level` from stored full fields: levels
 * + (l mod depth) * N words must hold level l for l = max(0, level-L-s+1) ..
 * level (s = 2 for order 2, 3 for order 4: the oldest level the next step's
 * halos read).  Sets the state, the ring buffers and every progress flag;
 * clears the device status.  Stream-ordered. */
int at_set_history(at_solver *h, const void *levels, int64_t depth, int64_t level);

/* Bytes of checkpoint storage for n_steps in intervals of `interval`:
 * ceil(n_steps / interval) checkpoints of L + s levels, N words each. */
size_t at_checkpoint_bytes(const at_solver *h, int64_t n_steps, int64_t interval);

/* Forward run from level 0 (right after at_set_state) by n_steps, keeping in
 * ckpt (device memory, at_checkpoint_bytes) the levels c-L-s+1 .. c of every
 * c = 0, interval, 2 interval, ...  delays as in at_step (AT_FREE: pass an
 * array to record the delays, which the adjoint then replays); passes are one
 * level long except in the last interval. */
int at_step_checkpointed(at_solver *h, int64_t n_steps, int delay_mode, int8_t *delays, int64_t interval,
                         void *ckpt);

/* Bytes of the adjoint's scratch workspace (device memory, 256-byte aligned):
 * interval + L + s levels, one adjoint field, the pending adjoint of delayed
 * boundary reads and per-block FP64 sums. */
size_t at_adjoint_workspace_bytes(const at_solver *h, int64_t interval);

/* Discrete adjoint of the run made by at_step_checkpointed(h, n_steps, ...):
 *   lam (device, N words of the state's dtype): dJ/du^{n_steps} on entry,
 *       dJ/du^0 on return;
 *   *dnu: dJ/dnu, accumulated in FP64;
 *   delay_mode AT_SYNC, AT_SEEDED or AT_REPLAY with the forward run's delays
 *       (AT_FREE runs: the recorded array and AT_REPLAY).
 * Each interval is recomputed from its checkpoint with at_step_levels, then
 * one adjoint kernel launch per level takes lambda^{n+1} to lambda^n.
 * Leaves the solver's state at an intermediate level: set it again before
 * stepping.  Synchronises and returns the device status. */
int at_adjoint(at_solver *h, int64_t n_steps, int delay_mode, const int8_t *delays, int64_t interval,
               const void *ckpt, void *adj_ws, size_t adj_ws_bytes, void *lam, double *dnu);

/* Measured FMA throughput of the current device for dtype AT_F64 or AT_F32:
 * fused multiply-adds per second (2 flops each) over the whole GPU, from one
 * timed launch (after one warm-up launch) of a kernel whose threads run
 * independent FMA chains, `trips` x 64 FMAs per thread (8 CTAs of 256 threads
 * per SM).  The roofline of the arithmetic-bound variants (FP64 state) is
 * taken against it.  Synchronises the legacy default stream.  A measurement
 * utility; the paper has no counterpart. */
int at_fma_peak(int dtype, int64_t trips, double *fma_per_s);

/* Size in bytes of the fixed scratch array used by at_step_noalloc(). */
#define AT_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)

/* at_step_noalloc -- the same run as at_create + at_set_state + at_step +
 * at_status, for callers that cannot allocate device memory (for example a
 * plug-in whose host application owns all device memory and hands it only
 * the state buffer, or code that must never call cudaMalloc).  The paper has
 * no counterpart; this entry point exists only for such callers.
 *
 *   u        device memory, N words of grid->dtype, 16-byte aligned: level 0
 *            on entry, level n_steps on return (updated in place).
 *   delays   as in at_step (input for AT_REPLAY, optional record otherwise).
 *   The other arguments are those of at_create; grid->workspace and
 *   grid->workspace_bytes are ignored.
 *
 * Memory.  Nothing is allocated, on the device or on the host: the ring
 * buffers, progress flags, status word and counters live in one array of
 * AT_NOALLOC_SCRATCH_BYTES (8 MiB) that this library places in the device
 * memory of every GPU that loads it and keeps until the process exits.  A
 * problem whose scratch would not fit -- roughly 32 T + 16 bytes per
 * subdomain with T = 8 or 16 ring slots, i.e. up to about 15,000 subdomains at
 * order 4 and L = 3 -- is rejected with AT_ERR_ARG and a message giving both
 * sizes.
 *
 * Sharing.  All calls on a device share that one array, and it keeps what the
 * last call left in it; each call clears the parts that must start at zero
 * before it launches.  Calls whose work overlaps on the same GPU (other
 * streams, other host threads) race on the array and corrupt each other's
 * results: issue them one after another.
 *
 * Levels per pass.  One level per pass (no temporal blocking):
 * grid->steps_per_pass must be 0 or 1, else AT_ERR_ARG.  No compensated
 * state (AT_FLAG_COMPENSATED gives AT_ERR_ARG).
 *
 * Returns.  The call synchronises its stream (it reads the device status
 * after the run) and returns
 *   AT_OK;
 *   AT_ERR_ARG       bad arguments, as at_create and at_step, or a problem too
 *                    large for the array, or steps_per_pass > 1;
 *   AT_ERR_UNSTABLE  nu dt / dx^2 above the order's limit (as at_create);
 *   AT_ERR_RESIDENCY the CTAs cannot be co-resident, or no cooperative launch;
 *   AT_ERR_CUDA      a CUDA call failed (message from at_last_error());
 *   AT_ERR_TIMEOUT   a device wait expired.
 *
 * Set-up.  Every call looks up the device address of the array
 * (cudaGetSymbolAddress) with the calling thread's current device; the first
 * call on a device also loads this library's device code there. */
int at_step_noalloc(const at_grid *grid, int64_t P, int scheme_order, int L,
                    double nu, double dt, void *u, int64_t n_steps,
                    int delay_mode, int8_t *delays);

#ifdef __cplusplus
}
#endif

#endif /* AT_H */
