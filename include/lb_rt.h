/*
 * lb_rt.h -- C ABI of the GB300 grey radiative Lattice-Boltzmann library.
 *
 * The library advances the discrete specific intensities I_i(r, t) of the
 * radiative LB equation (Weih et al. 2020, Sec. 3.2, Eqs. rte_discrete and
 * source-and-equil) on a uniform 2D or 3D grid: every step pull-streams each
 * direction with the trilinear (bilinear) rule of Eq. (interp), solves the
 * implicit collision of Eq. (rte_implicit) exactly (or the explicit
 * Eq. collision-step, or a fixed number of Lambda-iteration cycles), and can
 * reduce the moments E, F^a, P^ab of Eqs. (moments_discrete, higher_moments).
 * A moving background fluid uses the mixed-frame equation of App. B.
 *
 * Conventions shared by every call
 *   - c = 1; dt = cfl * dx; opacities in 1/length, emissivities in E/length.
 *   - The populations carry their quadrature weight: E = sum_i I_i.
 *   - Site fields are float32, layout [nz][ny][nx] (x fastest), "sites" =
 *     nx*ny*nz.  Vector fields are [3][nz][ny][nx]; populations are
 *     direction-major [N][nz][ny][nx].
 *   - ptr_kind = LB_RT_HOST or LB_RT_DEVICE says where a caller pointer
 *     lives.  Device pointers must be valid on the handle's device.  Inputs
 *     are copied into library-owned memory before the call returns (host) or
 *     stream-ordered on the handle's stream (device): the caller may reuse
 *     host buffers at once and device buffers after the stream reaches the
 *     call.
 *   - Every call returns lb_rt_status; negative values are errors and
 *     lb_rt_last_error() gives a message.  No call throws.  A handle is
 *     bound to one CUDA stream and is not thread-safe.
 *   - lb_rt_step() only enqueues work; errors raised on the device surface
 *     on the next lb_rt_sync(), lb_rt_moments() or lb_rt_get_*() call.
 */
#ifndef LB_RT_H
#define LB_RT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_rt lb_rt;

typedef enum {
  LB_RT_OK = 0,
  LB_RT_EINVAL = -1,    /* bad argument or configuration */
  LB_RT_ENOMEM = -2,    /* device or host allocation failed */
  LB_RT_ECUDA = -3,     /* a CUDA runtime call failed */
  LB_RT_ETIMEDOUT = -4, /* a bounded device wait gave up */
  LB_RT_ESTATE = -5,    /* call not valid in the handle's current state */
  LB_RT_EBUSY = -6      /* batch: the problem does not fit the free memory or slots now */
} lb_rt_status;

/* built-in direction sets (used when lb_rt_config.dirs == NULL) */
enum {
  LB_RT_RING2D = 1,          /* N equally spaced on the circle, phi_k = ring_offset + 2 pi k/N,
                                w = 1/N (Sec. 3.2.1, 2D quadrature of order N-1) */
  LB_RT_ICOSPHERE = 2,       /* icosahedral geodesic set, level = dirset_param[0]:
                                10*4^level + 2 points, w = 1/N */
  LB_RT_GAUSS_LEGENDRE = 3   /* Gauss-Legendre (dirset_param[0] nodes in cos theta) x
                                trapezoid (dirset_param[1] points in phi) product rule
                                (Sec. 3.2.1) */
};

enum { LB_RT_PERIODIC = 0, LB_RT_VACUUM = 1 };               /* per-axis boundary */
/* Population storage.  LB_RT_F32: float32 populations.  The 16-bit modes
 * keep, per site, E in float32 and per direction the relative deviation
 * q_i = I_i / (w_i E) - 1 in 16 bits; all arithmetic is float32.
 * LB_RT_F16_DEV (11 significant bits) holds E and F within 2e-3 relative L2
 * of the FP64 oracle on every tested regime, free-streaming beams included.
 * LB_RT_BF16_DEV (8 significant bits) is validated to 2e-3 only where the
 * field stays near isotropy, as in scattering-dominated (optically thick)
 * problems such as the diffusion configuration; in free-streaming, strongly
 * beamed regions its flux error exceeds that bound (about 5e-3 after 150
 * steps of the radiating sphere), so use LB_RT_F16_DEV there. */
enum { LB_RT_F32 = 0, LB_RT_F16_DEV = 1, LB_RT_BF16_DEV = 2 };
enum {
  LB_RT_IMPLICIT_EXACT = 0,  /* exact solution of Eq. (rte_implicit) */
  LB_RT_EXPLICIT = 1,        /* Eq. (collision-step) */
  LB_RT_LAMBDA_K = 2         /* lambda_iters cycles of the Lambda iteration (Sec. 3.3) */
};
enum {
  LB_RT_HOST = 0,
  LB_RT_DEVICE = 1,
  /* lb_rt_set_fluid only: page-locked host memory the device can address
   * (cudaHostAlloc, cudaHostRegister with cudaHostRegisterMapped).  The step
   * kernels read the fields in place across the host link instead of a copy,
   * so the caller keeps the memory valid and unchanged until every step that
   * uses it has completed (a later synchronising call) or a later
   * lb_rt_set_fluid replaces it.  Memory the device cannot address: EINVAL
   * (where the device translates host page tables, as on coherent CPU-GPU
   * systems, ordinary pageable memory qualifies too). */
  LB_RT_HOST_MAPPED = 2
};
enum {
  LB_RT_STATE_POPULATIONS = 0, /* N*sites floats, direction-major */
  LB_RT_STATE_ISOTROPIC = 1,   /* sites floats E0: I_i = w_i E0 */
  LB_RT_STATE_P1 = 2           /* 4*sites floats (E0, F0x, F0y, F0z): I_i = w_i (E0 + d n_i.F0) */
};

/* Maximum number of directions a handle accepts. */
#define LB_RT_MAX_DIRS 192

typedef struct {
  int dims;                /* 2 or 3 */
  int nx, ny, nz;          /* grid; nz must be 1 when dims == 2 */
  int ndir;                /* N when dirs != NULL (or for LB_RT_RING2D); else derived */
  const double* dirs;      /* N*3 unit vectors, caller-owned, copied at create; or NULL */
  const double* weights;   /* N weights (NULL => 1/N); used only with dirs */
  int dirset;              /* built-in set when dirs == NULL */
  int dirset_param[2];     /* see the LB_RT_ICOSPHERE / LB_RT_GAUSS_LEGENDRE comments */
  double ring_offset;      /* phi_0 of LB_RT_RING2D, radians */
  double cfl;              /* c dt / dx, 0 < cfl <= 1 (keeps the weights of Eq. interp in [0,1]) */
  double dx;               /* cell size */
  int bc[3];               /* per axis x, y, z: LB_RT_PERIODIC or LB_RT_VACUUM (reads 0 outside) */
  int storage;             /* LB_RT_F32 | LB_RT_F16_DEV | LB_RT_BF16_DEV */
  int collision;           /* LB_RT_IMPLICIT_EXACT | LB_RT_EXPLICIT | LB_RT_LAMBDA_K */
  int lambda_iters;        /* cycles for LB_RT_LAMBDA_K (the paper's timing runs use 5) */
  int moving;              /* 0: static fluid; 1: mixed-frame moving fluid (App. B) */
  int budget;              /* 1: accumulate the FP64 energy budget every step */
  void* stream;            /* cudaStream_t to run on; NULL => the library creates one */
} lb_rt_config;

/* Fluid coefficients.  For each site field, a NULL pointer means "uniform,
 * use the scalar next to it".
 * Static fluid (Eq. rte_gray_bgkform): absorption kappa_a, scattering
 * kappa_0, lambda = 3 kappa_1 / kappa_0, emissivity eta.
 * Moving fluid (App. B, kappa_1 = 0): three-velocity v ([3][sites], |v| < 1;
 * NULL => at rest), fluid-frame kt_a, kt_0 and eta_t. */
typedef struct {
  const float* kappa_a; float kappa_a_s;
  const float* kappa_0; float kappa_0_s;
  const float* lambda;  float lambda_s;
  const float* eta;     float eta_s;
  const float* v;
  const float* kt_a;    float kt_a_s;
  const float* kt_0;    float kt_0_s;
  const float* eta_t;   float eta_t_s;
} lb_rt_fluid;

/* Energy budget in FP64, summed since the last lb_rt_set_state()
 * (all quantities are sums over sites of E = sum_i I_i):
 *   total     current sum E
 *   initial   sum E right after lb_rt_set_state()
 *   outflow   sum over steps of (sum E^n - sum E*): what streaming moved out of
 *             the domain through vacuum faces
 *   source    sum over steps of (sum E_collided - sum E*): net emission minus
 *             absorption of the collision, dt sum (eta - kappa_a E^{n+1}) for a
 *             static fluid
 *   injection sum over steps of what frozen cells added over the collided values
 * so that total - initial = source - outflow + injection up to rounding. */
typedef struct {
  double total, initial, outflow, source, injection;
  long long steps;
} lb_rt_budget;

/* Create a handle: validates the configuration, builds the direction table
 * (Sec. 3.2.1), allocates device state (two population buffers, fields) and
 * sets I = 0, kappa = eta = 0.  Errors: EINVAL (bad config), ENOMEM, ECUDA. */
lb_rt_status lb_rt_create(const lb_rt_config* cfg, lb_rt** out);

/* Copy fluid coefficients (static or moving, per the handle's config) into
 * library storage, or with ptr_kind = LB_RT_HOST_MAPPED reference them in
 * page-locked host memory (read in place by the kernels; a coupled fluid
 * code hands over new fields every step without a copy).  Takes effect for
 * the next lb_rt_step().  Errors: EINVAL (NULL handle/fields, moving fields
 * on a static handle or the reverse, LB_RT_HOST_MAPPED memory the device
 * cannot address). */
lb_rt_status lb_rt_set_fluid(lb_rt* h, const lb_rt_fluid* f, int ptr_kind);

/* Set the populations (kind = LB_RT_STATE_*), reset the step counter and the
 * energy budget.  In the reduced-precision storage modes the populations are
 * encoded on the device (equilibrium-deviation form). */
lb_rt_status lb_rt_set_state(lb_rt* h, const float* data, int kind, int ptr_kind);

/* Frozen (prescribed) cells: after every collision the populations of
 * cells[k] (linear site index z*ny*nx + y*nx + x) are overwritten by
 * values[k*N + i] (Sec. 4.1.1, injected and frozen beam regions).
 * ncells == 0 clears the list.  Arrays are host arrays, copied. */
lb_rt_status lb_rt_set_frozen(lb_rt* h, const int64_t* cells, int ncells, const float* values);

/* Enqueue nsteps timesteps on the handle's stream.  One step is the fused
 * pull-stream and collision of Sec. 3.3: the populations are streamed along
 * their directions with the trilinear (bilinear in 2D) interpolation of
 * Eq. interp, then relaxed by the collision chosen at create -- the exact
 * implicit step of Eq. rte_implicit (closed form of its fixed point), the
 * explicit step of Eq. collision-step, or a fixed number of Lambda
 * iterations -- or, for a moving fluid, the mixed-frame implicit step of
 * App. B.  Then frozen cells are overwritten (Sec. 4.1.1) and, with
 * config.budget = 1, the FP64 energy budget is updated.  nsteps >= 0.
 * Asynchronous: returns launch errors only; device-side errors (a bounded
 * wait that gave up) surface at the next lb_rt_sync(). */
lb_rt_status lb_rt_step(lb_rt* h, int nsteps);

/* Moments of the current populations (Eqs. moments_discrete, higher_moments):
 * E [sites], F [3][sites] (z component 0 in 2D), P [6][sites] in the order
 * xx, xy, xz, yy, yz, zz.  Any output pointer may be NULL.  budget (host
 * pointer or NULL) receives the FP64 energy budget (zeros unless
 * config.budget = 1).  With host pointers the call synchronises the stream. */
lb_rt_status lb_rt_moments(lb_rt* h, float* E, float* F, float* P,
                           lb_rt_budget* budget, int ptr_kind);

/* lb_rt_step followed by the moments E [sites] and F [3][sites] of the new
 * state (the coupling loop of Sec. 5: step 3 then step 4), with E and F taken
 * from the last step's collision instead of a second pass over the
 * populations.  The collision writes I' = alpha I* + w_i (c0 + n_i . c1)
 * (Sec. 3.3, Eq. rte_implicit); for an isotropic table (Eq. iso-tensors:
 * sum w = 1, sum w n = 0, sum w n n = Id/d) its moments are E' = alpha E* + c0
 * and F' = alpha F* + c1/d, which the step kernel stores per site.
 * Host memory that the device can address (page-locked memory from
 * cudaHostAlloc or cudaHostRegister, and on coherent CPU-GPU systems any host
 * memory) is written by the step kernel itself across the host link; other
 * host memory goes through a device buffer.
 * With host pointers the call synchronises the stream.  For 16-bit storage,
 * a moving fluid, frozen cells, a table that is not isotropic, or nsteps = 0,
 * it runs lb_rt_step and then lb_rt_moments.  E or F may be NULL.
 * Agrees with lb_rt_step + lb_rt_moments to float32 rounding (the two sum in
 * different orders).  Errors: EINVAL, ECUDA, ETIMEDOUT as lb_rt_step and
 * lb_rt_sync. */
lb_rt_status lb_rt_step_moments(lb_rt* h, int nsteps, float* E, float* F, int ptr_kind);

/* Coupling outputs of the current state for a fluid code (Sec. 5, step 4 of
 * the coupling): the comoving radiation energy density J [sites] and
 * momentum density H [3][sites] (Eq. J), and the radiative four-force
 * S [4][sites] = (S_0, S_x, S_y, S_z) with S_0 = W (kt_a J - eta_t) + kt H^0,
 * S_j = W (kt_a J - eta_t) v_j + kt H_j, kt = kt_a + kt_0: the lab components
 * of the four-vector (kt_a J - eta_t) u^mu + kt H^mu, u^mu = W (1, v), whose
 * comoving flux H^mu has the time component H^0 = v.H fixed by
 * H^mu u_mu = 0 (signature -+++).  A static handle uses v = 0 and its static
 * opacities.  Any output may be NULL.  With host pointers the call
 * synchronises the stream.  Errors: EINVAL, ECUDA. */
lb_rt_status lb_rt_coupling(lb_rt* h, float* J, float* H, float* S, int ptr_kind);

/* Decoded float32 populations, direction-major [N][sites]. */
lb_rt_status lb_rt_get_populations(lb_rt* h, float* out, int ptr_kind);

/* Checkpoint: raw device state (populations in their storage format, the
 * per-site moment field of the reduced-precision modes, step counter and
 * budget).  lb_rt_state_bytes() gives the size; buf is a host buffer.
 * lb_rt_restore_state() puts it back bit for bit. */
size_t lb_rt_state_bytes(const lb_rt* h);
lb_rt_status lb_rt_save_state(lb_rt* h, void* buf, size_t bytes);
lb_rt_status lb_rt_restore_state(lb_rt* h, const void* buf, size_t bytes);

/* Wait for the handle's stream; returns the first device-side or CUDA error.
 * LB_RT_ETIMEDOUT means a bounded wait inside a step kernel gave up: the
 * populations written since the previous successful lb_rt_sync() are not
 * trusted.  The device error word is cleared when it is reported, so the
 * handle stays usable after lb_rt_restore_state() or lb_rt_set_state();
 * stepping on without either continues from an undefined state. */
lb_rt_status lb_rt_sync(lb_rt* h);

/* Direction table in the canonical order the library uses: dirs [N*3],
 * weights [N], signs [N*3] (sgn(n) with sgn(0) = +1, the upwind side of
 * Eq. interp).  Any pointer may be NULL.  Host pointers. */
lb_rt_status lb_rt_directions(const lb_rt* h, int* ndir, double* dirs, double* weights,
                              int8_t* signs);

/* Time of the last lb_rt_step() batch's step kernels, measured with CUDA
 * events on the handle's stream (ms per step kernel, summed over the batch)
 * -- valid after lb_rt_sync(). Returns EINVAL if timing was not enabled. */
lb_rt_status lb_rt_enable_timing(lb_rt* h, int on);
lb_rt_status lb_rt_last_step_ms(lb_rt* h, float* ms, int* nlaunch);

/* ---- Batched problems (many independent solves in one launch) ----------
 *
 * Not a construct of the paper, which solves one problem at a time: a batch
 * keeps many independent static-fluid problems resident on the device and
 * advances them together.  Problems whose direction table, tile plan and
 * storage agree form one group; each step of a group is ONE persistent
 * kernel launch over the concatenated tiles of all its problems (Sec. 3.3
 * stream and collision per problem, exactly as lb_rt_step), and a tick (the
 * steps_per_tick steps of every group) is captured into a CUDA graph and
 * replayed while its launch plan is unchanged.  Two groups whose direction
 * counts differ (for instance 42 and 162 directions) can share ONE launch
 * per step (pair_groups): the persistent grid is split between the two
 * groups' tiles in proportion to their work, each CTA running its group's
 * tile plan.  An autotuner picks, per group, the tile shape: the z-chunk
 * length of the tiles, timed over the candidates on the first ticks of a
 * new set of problems, then the planes per batch, where an alternative
 * batched kernel of the same memory layout exists (the 42-direction plans);
 * and (pair_groups = 2) whether the paired launch beats the two separate
 * ones.  Every choice gives the same bits.  Admission is by device memory: a
 * problem is admitted when its buffers fit the batch's budget and a slot is
 * free; otherwise lb_rt_batch_admit returns LB_RT_EBUSY and the caller
 * retries after completed problems are released.  Batched problems have no
 * energy budget, no frozen cells and a static fluid.  The result of a
 * problem is the same alone and in any mix: its tiles depend only on its
 * own data. */
typedef struct lb_rt_batch lb_rt_batch;

#define LB_RT_BATCH_MAX 256

typedef struct {
  size_t mem_budget;   /* device bytes for admitted problems; 0 => 80 % of free memory at create */
  int max_problems;    /* slots, 1 .. LB_RT_BATCH_MAX */
  int storage;         /* LB_RT_F32 | LB_RT_F16_DEV | LB_RT_BF16_DEV, every problem */
  int steps_per_tick;  /* steps per lb_rt_batch_tick, >= 1 */
  int use_graph;       /* 1: capture ticks into a CUDA graph */
  int autotune;        /* 1: time the tile shapes (z chunk, planes per batch) on new sets of problems */
  void* stream;        /* cudaStream_t; NULL => the batch creates one */
  int pair_groups;     /* two groups of different direction counts in one launch per step:
                          0 never, 1 whenever their tile plans have a paired kernel (the 42-
                          and 162-direction icosahedral sets, every storage), 2 when the
                          autotuner measures it faster than separate launches */
} lb_rt_batch_config;

lb_rt_status lb_rt_batch_create(const lb_rt_batch_config* cfg, lb_rt_batch** out);
void lb_rt_batch_destroy(lb_rt_batch* b);

/* Device bytes a problem with this configuration would hold (populations,
 * moment field, coefficient fields, staging); 0 with an invalid cfg. */
size_t lb_rt_batch_problem_bytes(const lb_rt_batch* b, const lb_rt_config* cfg);

/* Admit a problem: cfg as for lb_rt_create (storage and stream are taken
 * from the batch; moving and budget must be 0), its fluid fields and
 * initial state as for lb_rt_set_fluid / lb_rt_set_state, and the number of
 * steps to run.  *slot receives its slot.  Errors: EINVAL, EBUSY (does not
 * fit now), ENOMEM, ECUDA.  The problem's initial state and fields are set
 * on a stream of its own, so an admission overlaps the ticks in flight. */
lb_rt_status lb_rt_batch_admit(lb_rt_batch* b, const lb_rt_config* cfg, const lb_rt_fluid* fluid,
                               int fluid_ptr_kind, const float* state, int state_kind,
                               int state_ptr_kind, long long nsteps, int* slot);

/* Enqueue one tick: every active problem advances by min(steps_per_tick,
 * remaining steps).  *n_active (may be NULL) receives the number of
 * problems that took part (0: nothing was enqueued).  Asynchronous on the
 * batch stream: two ticks may be in flight; the call waits only for the
 * tick before the previous one, whose descriptor tables it reuses.  A
 * problem's first tick waits (on the device) for its admission work. */
lb_rt_status lb_rt_batch_tick(lb_rt_batch* b, int* n_active);

/* Wait for the enqueued ticks and surface device errors.  LB_RT_ETIMEDOUT
 * (a bounded wait in a batched step gave up) leaves every active problem's
 * state untrusted and the batch's error word set: destroy the batch. */
lb_rt_status lb_rt_batch_sync(lb_rt_batch* b);

/* Slots whose problems have run all their steps on the device (the tick
 * with the last step has completed) and are not yet released; does not
 * wait.  Writes at most max slots; *n the count. */
lb_rt_status lb_rt_batch_poll(lb_rt_batch* b, int* slots, int max, int* n);

/* Moments of a problem's current state, as lb_rt_moments (budget NULL);
 * waits for the ticks enqueued so far. */
lb_rt_status lb_rt_batch_moments(lb_rt_batch* b, int slot, float* E, float* F, float* P,
                                 int ptr_kind);

/* Steps enqueued for the problem in `slot` (done once poll reports it). */
lb_rt_status lb_rt_batch_steps(const lb_rt_batch* b, int slot, long long* steps);

/* Free a problem's slot.  Its device memory goes back to the batch at the
 * next lb_rt_batch_sync(), or at an admission that needs the room (its last
 * tick may still be in flight when the slot is released). */
lb_rt_status lb_rt_batch_release(lb_rt_batch* b, int slot);

/* The autotuner's current choice for the group of `slot`: z-chunk length
 * (planes per tile) and CTAs of its last persistent launch. */
lb_rt_status lb_rt_batch_tuning(const lb_rt_batch* b, int slot, int* zchunk, int* ctas);

/* Tile plan of the group of `slot`: directions per warp, planes per batch
 * of the batched kernel its last launch ran (the autotuner's choice, or its
 * trial while tuning), and whether its last tick shared a launch with
 * another group (1) or not (0).  Any output pointer may be NULL. */
lb_rt_status lb_rt_batch_plan(const lb_rt_batch* b, int slot, int* dirs_per_warp,
                              int* planes_per_batch, int* paired);

/* Message of the batch's last error. */
const char* lb_rt_batch_last_error(const lb_rt_batch* b);

/* FP64 total energy sum_sites sum_i I_i of a dense float32 population array
 * pop [ndir][sites] in device memory (for example the output of
 * lb_rt_get_populations with a device pointer), computed without allocating
 * anything.  The paper has no counterpart: this is a service for callers that
 * cannot call cudaMalloc where they need the number -- code running while
 * another framework owns the device memory pool, a real-time loop that may not
 * pay allocation latency, or a process whose device memory budget is fixed in
 * advance.  The per-block partial sums live in a fixed 32 KB array that every
 * GPU loading the library holds until exit, which limits sites to
 * 16,777,216 (larger inputs return LB_RT_EINVAL).  out is a device pointer
 * (ptr_kind = LB_RT_DEVICE: the result is written stream-ordered on `stream`)
 * or a host pointer (LB_RT_HOST: the call synchronises `stream`).  The first
 * call on a device looks up the array's device address; make that first call
 * before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU (for example on two streams) race.  The device address
 * is cached per device ordinal for the life of the process: do not use this
 * entry point across cudaDeviceReset() or from a context other than the
 * device's primary context.  pop (and out with LB_RT_DEVICE) must be device
 * or managed memory; anything else returns LB_RT_EINVAL before a launch.
 * Errors: EINVAL (bad argument, host memory where device memory is required,
 * or too many sites), ECUDA; lb_rt_last_error(NULL) says which. */
lb_rt_status lb_rt_total_energy_noalloc(const float* pop, int ndir, long long sites, double* out,
                                        int ptr_kind, void* stream);

/* Message of the last error on h; with h == NULL, why the calling thread's
 * last failed call without a handle (lb_rt_create(),
 * lb_rt_total_energy_noalloc()) failed. */
const char* lb_rt_last_error(const lb_rt* h);
const char* lb_rt_version(void);

/* NULL-safe; frees every device and host resource of the handle. */
void lb_rt_destroy(lb_rt* h);

#ifdef __cplusplus
}
#endif
#endif /* LB_RT_H */
