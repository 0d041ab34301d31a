/*
 * hrm.h -- C ABI of the GB300 library for the positivity-preserving fractional
 * algorithm of Wong, Angel & Kiris (arXiv 2208.04488): the five-equation model of
 * Allaire et al. advanced by PP-WCNS-IS with SSP-RK time stepping, followed after
 * every Runge-Kutta stage by the algebraic thermal relaxation at infinite rate,
 * which yields the four-equation homogeneous relaxation model (HRM).
 *
 * Plain C types only. Every call is ordered on the CUDA stream given at creation
 * (NULL = the legacy default stream). Device pointers are CUDA device addresses of
 * the current device; host pointers are ordinary host memory.
 *
 * Conservative state layout (Sec. 2, vector W): structure of arrays
 *   W[m][z][y][x], m = 0..M-1, x fastest, M = 2N + D, interior cells only:
 *   m = 0..N-1      alpha_k rho_k      (partial densities)
 *   m = N..N+D-1    rho u_d            (momentum)
 *   m = N+D         E                  (total energy per unit volume)
 *   m = N+D+1..M-1  alpha_k, k < N     (alpha_N = 1 - sum of the others)
 * Species may be given in any order; at most one may have p_inf > 0 (the
 * stiffened gas of Sec. 4.2), the others are ideal gases.
 *
 * Errors: every call returns an hrm_status; nothing aborts. hrm_last_error()
 * gives a one-line description of the last failure on a context.
 */
#ifndef HRM_H
#define HRM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hrm_ctx hrm_ctx; /* opaque, owned by the library */

typedef enum {
  HRM_OK = 0,
  HRM_E_INVAL = -1,         /* invalid argument (message in hrm_last_error) */
  HRM_E_CUDA = -2,          /* a CUDA call failed */
  HRM_E_ADMISSIBILITY = -3, /* a step produced cells outside the admissible set */
  HRM_E_TIMEOUT = -4,       /* a bounded device wait ran out */
  HRM_E_NOMEM = -5          /* device allocation failed */
} hrm_status;

/* Boundary conditions of a grid side. Transmissive: the three ghost layers copy
 * the adjacent interior cell (zeroth-order extrapolation). Periodic: pairs with
 * the opposite side. Dirichlet: every ghost layer holds a prescribed state, one
 * value per boundary cell (hrm_set_boundary), e.g. the jet inflow of Sec. 5.9. */
enum { HRM_BC_TRANSMISSIVE = 0, HRM_BC_PERIODIC = 1, HRM_BC_DIRICHLET = 2 };

enum {
  HRM_SCHEME_WCNS = 0,      /* PP-WCNS-IS (Sec. 4.3) */
  HRM_SCHEME_HLLC1 = 1      /* first-order HLLC (Sec. 4.1.1) */
};

enum {
  HRM_RELAX_OFF = 0,        /* five-equation model without relaxation */
  HRM_RELAX_STAGE = 1,      /* after every RK stage (Sec. 4.4, the paper's choice) */
  HRM_RELAX_STEP = 2        /* after the full step only */
};

enum { HRM_RK3 = 0, HRM_EULER = 1, HRM_RK2 = 2 }; /* SSP integrators (Sec. 4.4, 5.1) */

enum {
  HRM_FP64 = 0,             /* everything in FP64 */
  HRM_FP32 = 1              /* WENO, HLLC, HCS in FP32; state, limiter theta and
                               relaxation in FP64 */
};

/* Uniform Cartesian grid: n[d] cells on [lo[d], hi[d]] (Sec. 4.1, grid midpoints
 * x_{i+1/2} = x_a + i dx); bc[2d], bc[2d+1] = low / high side of direction d. */
typedef struct {
  int32_t ndim;
  int32_t pad;
  int64_t n[3];
  double lo[3], hi[3];
  int32_t bc[6];
} hrm_grid;

/* Scheme options and the paper's constants; hrm_params_default() fills the
 * values of Sec. 4.3 and App. C. */
typedef struct {
  double cfl;          /* CFL number for the automatic time step (<= 0.5, Sec. 4.1.2) */
  int32_t limiters;    /* interpolation + flux limiters on (Sec. 4.3.2) */
  int32_t blend;       /* shock-sensor flux/velocity blending (Eq. flux_blending) */
  int32_t relax_mode;  /* HRM_RELAX_* */
  int32_t scheme;      /* HRM_SCHEME_* */
  int32_t integrator;  /* HRM_RK3 / HRM_EULER / HRM_RK2 */
  int32_t precision;   /* HRM_FP64 / HRM_FP32 */
  int32_t learned;     /* 0 off; 1 learned gate (needs hrm_set_detector); 2 fixed gate
                          (needs hrm_set_gate for every direction) -- see below */
  int32_t check;       /* 1: hrm_step synchronises and reports admissibility */
  double eps_ar, eps_a, eps_rhoe;      /* limiter thresholds 1e-10, 1e-10, 1e-8 */
  double hs_ar, hs_a, hs_rc2, hs_rhoe; /* hard switches 1e-11, 1e-11, 1e-9, 1e-9 */
  double weno_eps;                     /* 1e-15 (App. C); (0, 1e50] */
  double Cs, q_sensor;                 /* shock sensor 1e12 and 2 (Sec. 4.3.1) */
  double learned_threshold;            /* gate probability in (0, 1) above which d_k are used */
  int32_t screen;      /* precision form: 1 (default) first certifies in FP32, with rounding
                          margins, that the limiters would leave a midpoint unchanged (every
                          checked quantity above its threshold) and evaluates them in FP64
                          only where it cannot; results are the same as with 0 (always FP64) */
  int32_t cfl_sound;   /* sound speed of the CFL maxima tau_d (Sec. 4.1.2): 0 (default) the
                          five-equation c of the hyperbolic step, which the positivity bound of
                          the HLLC fluxes rests on; 1 the four-equation HRM c of Eq. 4_eqn_sos
                          (smaller, so a larger step without that guarantee). hrm_dt follows it;
                          hrm_dt_noalloc and the batched form use the five-equation c. */
} hrm_params;

/* Field selectors of hrm_get. */
enum {
  HRM_FIELD_W = 0,     /* M planes, layout above */
  HRM_FIELD_V = 1,     /* M planes: alpha_k rho_k, u_d, p (five-equation EOS), alpha_k */
  HRM_FIELD_C5 = 2,    /* 1 plane: five-equation sound speed, rho c^2 = gbar (p + pbar_inf) (Sec. 2) */
  HRM_FIELD_PT = 3,    /* 2 planes: equilibrium p and T of the four-equation HRM (Sec. 4.2) */
  HRM_FIELD_C4 = 4,    /* 1 plane: four-equation HRM sound speed (Eq. 4_eqn_sos) */
  HRM_FIELD_PSI_GAMMA = 5, /* N + 1 planes: Psi_1..Psi_N, Gamma of the four-equation HRM at the
                              equilibrium pressure (Sec. 3: derivatives of the relaxed pressure
                              with respect to alpha_k rho_k and to rho e) */
  HRM_FIELD_ALPHA = 6,    /* N planes: alpha_1..alpha_N (alpha_N = 1 - the others, Sec. 2) */
  HRM_FIELD_Y = 7,        /* N planes: mass fractions Y_k = alpha_k rho_k / rho */
  HRM_FIELD_SCHLIEREN = 8 /* 1 plane: numerical schlieren |grad rho| / rho of the paper's figures,
                             central differences with neighbours through the boundary conditions */
};

/* Device memory of contexts. By default a context takes its state and scratch
 * from cudaMalloc at hrm_create (plus the gate buffers it adds later) and
 * returns them at hrm_destroy. A caller that manages device memory itself (a
 * framework's caching allocator, a memory pool) installs alloc / free_fn here:
 * contexts created afterwards take every buffer from alloc(bytes, stream,
 * user) -- stream being the context's CUDA stream -- and return it through
 * free_fn(ptr, stream, user); a NULL result of alloc makes hrm_create fail with
 * HRM_E_NOMEM. Both NULL restore cudaMalloc. Process-wide, read at hrm_create;
 * not thread-safe against concurrent hrm_create. Batches and detectors keep
 * cudaMalloc. (The paper has no counterpart: this is the library's boundary.)
 * Errors: HRM_E_INVAL when exactly one of the two is NULL. */
typedef void* (*hrm_alloc_fn)(size_t bytes, void* cuda_stream, void* user);
typedef void (*hrm_free_fn)(void* ptr, void* cuda_stream, void* user);
hrm_status hrm_set_allocator(hrm_alloc_fn alloc, hrm_free_fn free_fn, void* user);

/* Fill p with the paper's constants (Sec. 4.3.2, App. C, Sec. 4.3.1), PP-WCNS-IS,
 * SSP-RK3, relaxation after every stage, FP64, CFL 0.5, check on. */
void hrm_params_default(hrm_params* p);

/* Create a context for one problem (Sec. 4: grid, N species, D dimensions).
 * gamma[N] > 1, p_inf[N] >= 0 with at most one positive, c_v[N] > 0 (c_p = gamma c_v,
 * Sec. 2), q[N] (NULL: all 0). params NULL: defaults. cuda_stream: a cudaStream_t
 * (NULL: default stream). Allocates the state and the scratch on the device.
 * Errors: HRM_E_INVAL (bad species table, N outside 2..3, ndim outside 1..3,
 * periodic direction with fewer than 3 cells, CFL > 0.5 with limiters on),
 * HRM_E_NOMEM, HRM_E_CUDA. On failure *out is NULL. */
hrm_status hrm_create(hrm_ctx** out, const hrm_grid* grid, int32_t nspecies,
                      const double* gamma, const double* p_inf, const double* c_v,
                      const double* q, const hrm_params* params, void* cuda_stream);

/* Release every resource of ctx (NULL is accepted). Synchronises its stream. */
void hrm_destroy(hrm_ctx* ctx);

/* One-line description of the last error on ctx (never NULL); with ctx NULL,
 * the reason the last hrm_create on this thread failed. */
const char* hrm_last_error(const hrm_ctx* ctx);

/* Replace the scheme options (same checks as hrm_create). */
hrm_status hrm_set_params(hrm_ctx* ctx, const hrm_params* params);

/* Set the state from W (layout above, M x ncells doubles), host (on_device = 0)
 * or device memory; resets the time to 0. With params.check the state is then
 * tested for admissibility (Sec. 2) and HRM_E_INVAL returned, with the four
 * counts of hrm_admissibility in hrm_last_error, if a cell lies outside the
 * admissible set (the state stays set). */
hrm_status hrm_set(hrm_ctx* ctx, const double* W, int32_t on_device);

/* Set the state from primitive planes prim[(N + D + 1) x ncells] =
 * (alpha_1..alpha_{N-1}, u_1..u_D, p, T) in pressure and temperature
 * equilibrium (Sec. 5): rho_k = (p + p_inf_k) / ((gamma_k - 1) c_v,k T)
 * (Eq. rho_k_thermally_relaxed), E from the mixture EOS (Sec. 2). The same
 * admissibility test as hrm_set with params.check. */
hrm_status hrm_set_primitive(hrm_ctx* ctx, const double* prim, int32_t on_device);

/* Time step of the current state (Sec. 4.1.2): tau_d = max(|u_d| + c) / dx_d,
 * dt = cfl / sum_d tau_d. Synchronises. tau_out (optional) receives D values. */
hrm_status hrm_dt(hrm_ctx* ctx, double cfl, double* dt_out, double* tau_out);

/* Advance nsteps full time steps (Sec. 4.4). dt > 0: that step size; dt <= 0:
 * the CFL step of params.cfl from the state at the start of each step
 * (footnote of Sec. 5). The directional split sigma_d and lambda_d of the flux
 * limiter come from the step-start state. Launches one captured CUDA graph per
 * step. With params.check it synchronises and returns HRM_E_ADMISSIBILITY when
 * a cell left the admissible set (the state is kept for inspection), or
 * HRM_E_TIMEOUT when a bounded wait of the learned gate's tensor-core kernel
 * ran out (its gate bytes are then unreliable). */
hrm_status hrm_step(hrm_ctx* ctx, double dt, int32_t nsteps);

/* How hrm_step runs a step. path 0 (the default): the captured graph of
 * per-phase kernels. path 1: where the context is in the precision form in 2D
 * with PP-WCNS-IS, SSP-RK3, the five-equation CFL speed, no Dirichlet side and
 * no learned gate, as three persistent cooperative launches of the batched
 * form's stage kernel over this one context (one per RK stage, every phase in
 * it; work items from device queues, phases separated by a bounded grid
 * barrier; with params.check a barrier wait that ran out is returned as
 * HRM_E_TIMEOUT); otherwise as path 0. Both give the same state bit for bit
 * (path 1 is the slower one on a single large grid: its FP64-bound update runs
 * under the midpoint body's register budget). With profiling on,
 * hrm_profile_read reports the persistent step's phases (primitives, step
 * scalars, midpoints of both directions, update) from %globaltimer stamps.
 * hrm_step_launches: kernel launches per step of the current step graph (0
 * before the first step). */
hrm_status hrm_set_step_path(hrm_ctx* ctx, int32_t path);
int32_t hrm_step_launches(const hrm_ctx* ctx);

/* The same step taken one RK stage at a time, so that a caller can exchange
 * halo layers between stages and reduce the CFL maxima over several contexts
 * (domain decomposition: one context per subdomain, each holding its layers
 * plus 3 ghost layers per inner side; the stencil of a midpoint spans nodes
 * i-2..i+3 and the HCS flux difference nodes i-3..i+3, Sec. 4.3.1). A step is
 * hrm_begin_step, then hrm_stage(0) .. hrm_stage(hrm_stages() - 1); with the
 * step state given, the results equal hrm_step's bit for bit.
 *
 * hrm_step_tau: the maxima tau_d = max(|u_d| + c) / dx_d of the step state as a
 * step computes them (Sec. 4.1.2; the form's sound speed and precision), over
 * every cell the context holds; D values. Synchronises.
 * hrm_begin_step: start a step from maxima tau_d (e.g. the maxima over all
 * subdomains): dt = cfl / sum_d tau_d unless dt > 0 is given, sigma_d =
 * tau_d / sum tau, lambda_d = dt / (sigma_d dx_d); advances the time and step
 * counters. HRM_E_INVAL for a negative or NaN tau_d, or when dt <= 0 and every
 * tau_d is 0. Synchronises.
 * hrm_stage: RK stage `stage` (0-based; 3 stages for SSP-RK3, 2 for SSP-RK2,
 * 1 for forward Euler): primitives of the stage's input state, the sweeps, the
 * update with the relaxation of params.relax_mode; the last stage writes the
 * step state. Launches without a graph and without the admissibility count
 * (use hrm_admissibility). Does not synchronise.
 * hrm_layers: copy `count` whole layers of cells along the slowest direction
 * (z in 3D, y in 2D, x in 1D), starting at layer `first`, between `buf`
 * (M planes of count x layer cells, layer = cells of one layer; caller-owned,
 * device memory when on_device) and the state stage `stage` reads (stage 0:
 * the step state; later stages: the RK stage state): set = 0 copies out, set =
 * 1 copies in. HRM_E_INVAL for layers outside the grid. Synchronises for host
 * buffers. */
hrm_status hrm_step_tau(hrm_ctx* ctx, double* tau);
hrm_status hrm_begin_step(hrm_ctx* ctx, const double* tau, double dt);
int32_t hrm_stages(const hrm_ctx* ctx);
hrm_status hrm_stage(hrm_ctx* ctx, int32_t stage);
hrm_status hrm_layers(hrm_ctx* ctx, int32_t stage, int32_t set, int64_t first, int64_t count, double* buf,
                      int32_t on_device);

/* Apply the thermal relaxation (Sec. 4.2) to the current state in place. */
hrm_status hrm_relax(hrm_ctx* ctx);

/* Prescribed state of Dirichlet side `side` (= 2 d + 0 for the low side of
 * direction d, 2 d + 1 for the high side). `values` holds one value per cell of
 * the boundary slice (the other directions' cell indices, lowest fastest):
 * with primitive = 0 the M conservative planes of W (layout above), with
 * primitive = 1 the N + D + 1 primitive planes of hrm_set_primitive, converted
 * in p-T equilibrium. Host or device memory; copied, not retained. The state
 * stays until the next call (hrm_set does not clear it); it enters the
 * reconstruction stencils of the side's first three midpoints and the CFL
 * maximum (Sec. 4.1.2). Every Dirichlet side needs a state before hrm_step,
 * hrm_dt or hrm_rhs, which otherwise return HRM_E_INVAL.
 * Errors: HRM_E_INVAL (NULL, or `side` not a Dirichlet side), HRM_E_CUDA. */
hrm_status hrm_set_boundary(hrm_ctx* ctx, int32_t side, const double* values, int32_t primitive,
                            int32_t on_device);

/* Semi-discrete right-hand side L(W) of the current state (Eq. semi_W_G_pm_eqn)
 * with flux-limiter lambda_d = lam[d], into rhs (M x ncells, device memory). */
hrm_status hrm_rhs(hrm_ctx* ctx, const double* lam, double* rhs_device);

/* Copy a field (HRM_FIELD_*) of the current state to dst (host: on_device = 0,
 * synchronises; device otherwise). Planes x ncells doubles. */
hrm_status hrm_get(hrm_ctx* ctx, int32_t field, double* dst, int32_t on_device);

/* Simulated time and number of steps taken since the last hrm_set. */
hrm_status hrm_time(hrm_ctx* ctx, double* t, int64_t* steps);

/* Out-of-range indices met by the kernels of ctx so far, in a library built
 * with -DHRM_BOUNDS_CHECK (HRM_BOUNDS_CHECK=1 in the environment of the build),
 * where every midpoint's node index and every cell's midpoint index is checked
 * against its array and, when outside, counted and replaced by 0; -1 in a
 * release build or on error. A debugging aid in place of a memory checker (the
 * paper has no counterpart). Synchronises. */
int64_t hrm_bounds_violations(hrm_ctx* ctx);

/* Restore the simulated time and step count (checkpoint / restart: W from
 * hrm_get, then hrm_set and hrm_set_time; the steps that follow are those of an
 * uninterrupted run bit for bit, the step size depending only on the state).
 * Synchronises. Errors: HRM_E_INVAL (steps < 0), HRM_E_CUDA. */
hrm_status hrm_set_time(hrm_ctx* ctx, double t, int64_t steps);

/* Admissibility counters of the current state (Sec. 2, sets G and script-G):
 * counts[0] cells with a negative partial density, [1] a volume fraction outside
 * [0, 1], [2] rho c^2 <= 0 or NaN, [3] rho (e - qbar) <= 0 or NaN. Synchronises. */
hrm_status hrm_admissibility(hrm_ctx* ctx, int64_t counts[4]);

/* Number of kernels the library has launched on ctx since creation
 * (graph launches count their kernel nodes). */
int64_t hrm_kernel_launches(const hrm_ctx* ctx);

/* Kernel kinds reported by hrm_profile_read. */
enum {
  HRM_KERNEL_PRIM = 0,      /* per-cell primitives (+ CFL reduction at the first stage) */
  HRM_KERNEL_FINALIZE = 1,  /* dt, sigma_d, lambda_d */
  HRM_KERNEL_FACE_X = 2,    /* per-midpoint sweep in x (HRM_KERNEL_FACE_X + d for direction d) */
  HRM_KERNEL_UPDATE = 5,    /* flux difference, RK combination, relaxation */
  HRM_KERNEL_GATE = 6,      /* learned smoothness gate of one direction */
  HRM_KERNEL_SWEEPS = 7     /* all sweeps of one stage, fork to join: in 2D and 3D the directions run
                               concurrently (direction d > 0 on its own stream of the step graph), so
                               their own brackets overlap and this one times them together */
};

/* Tracing: with on != 0 the step graph is (re)captured with a CUDA event pair
 * around every kernel and one around the sweeps of each stage
 * (HRM_KERNEL_SWEEPS). Costs one event-record node per bracket boundary. */
hrm_status hrm_set_profiling(hrm_ctx* ctx, int32_t on);

/* After a step with tracing on: synchronises the stream and writes, for the
 * brackets of the last step in the order they open, their device time in ms
 * and their kind (HRM_KERNEL_*). Returns how many were written (at most max). */
int32_t hrm_profile_read(hrm_ctx* ctx, int32_t max, float* ms, int32_t* kind);

/* ------------------------------------------------------------------------
 * Learned smoothness gate (not a part of the paper's method: an optional
 * acceleration of its WENO-IS interpolation, App. C).
 *
 * Per midpoint x_{i+1/2} and direction, a multilayer perceptron reads the
 * six-node stencil i-2 .. i+3 -- for q in (alpha_1, alpha_2, rho, u_n, p) the
 * normalised shape (q_j - mean q) / (max q - min q + 1e-30), formed on the
 * differences q_j - q_i, zero for an absent alpha_2: 30 inputs -- through
 * 32 and 32 ReLU units to one logit. Where sigmoid(logit) > learned_threshold
 * the midpoint is gated: both biased interpolations of every characteristic
 * field use the linear weights d_k instead of the WENO-IS weights; the
 * characteristic projection (App. D), both positivity limiters (Sec. 4.3.2),
 * the Riemann solves, HCS and blending are unchanged. Inference: bfloat16
 * inputs and weights, FP32 accumulation, on the tensor cores: in the FP64
 * form (and the precision form with params.screen = 0) a gate kernel runs
 * before each sweep (tcgen05: one 128-row tile of midpoints per CTA,
 * accumulators in tensor memory); in the precision form's screened sweep the
 * sweep runs the network itself with warp-level MMA, only in warps that hold a
 * stencil that is not uniform (a uniform stencil -- every FP32 plane equal at
 * the six nodes -- takes the exact node flux, which the interpolation weights
 * do not affect).
 *
 * Training data come from states the method produces: the label of a midpoint
 * is 1 when every WENO-IS weight of every characteristic field and both biases
 * lies within delta of its linear weight d_k (FP64), else 0.
 *
 * Parameter vector (2081 floats): W1[30][32], b1[32], W2[32][32], b2[32],
 * w3[32], b3 with h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2),
 * logit = h2 . w3 + b3. Loss: binary cross-entropy, batch mean; Adam
 * (beta 0.9, 0.999, eps 1e-8).
 * ------------------------------------------------------------------------ */
typedef struct hrm_detector hrm_detector; /* opaque: weights, Adam state, samples */

#define HRM_DETECTOR_PARAMS 2081
#define HRM_DETECTOR_INPUTS 30

/* capacity: samples the detector can hold (each 136 B of device memory);
 * seed: initial weights (He-uniform) and the sample draws. stream: nullable.
 * Errors: HRM_E_INVAL (capacity outside 0..2^31), HRM_E_NOMEM, HRM_E_CUDA. */
hrm_status hrm_detector_create(hrm_detector** out, int64_t capacity, uint64_t seed, void* stream);
void hrm_detector_destroy(hrm_detector* det);
const char* hrm_detector_last_error(const hrm_detector* det);
/* Host arrays of HRM_DETECTOR_PARAMS floats; set_weights also resets Adam. */
hrm_status hrm_detector_set_weights(hrm_detector* det, const float* theta);
hrm_status hrm_detector_get_weights(hrm_detector* det, float* theta);
int64_t hrm_detector_size(const hrm_detector* det);
hrm_status hrm_detector_clear(hrm_detector* det);
/* Append samples: X host [n][30], y host [n] (labels 0/1). INVAL beyond capacity. */
hrm_status hrm_detector_add_samples(hrm_detector* det, const float* X, const float* y, int64_t n);
/* Read samples [first, first+n) into host arrays (each nullable): X [n][30],
 * y [n], dev [n] (the weight deviation of collected samples, 0 for added ones). */
hrm_status hrm_detector_samples(hrm_detector* det, int64_t first, int64_t n, float* X, float* y, float* dev);
/* Append samples from every midpoint of every direction of ctx's current
 * state (runs its primitive kernel): label 1 when the deviation is below
 * delta. Each midpoint is kept with probability keep_rough (label 0),
 * keep_flat (label 1, all features zero) or keep_smooth (other label 1),
 * drawn from a hash of (seed, call, direction, midpoint); kept midpoints are
 * stored in index order; beyond the capacity they are dropped. *added: count. */
hrm_status hrm_detector_collect(hrm_detector* det, hrm_ctx* ctx, double delta, double keep_rough,
                                double keep_smooth, double keep_flat, int64_t* added);
/* Summed loss and its gradient (host [2081]) at the current weights over
 * samples [first, first+n), FP32 training arithmetic. */
hrm_status hrm_detector_gradient(hrm_detector* det, int64_t first, int64_t n, float* grad, double* loss);
/* steps Adam steps with learning rate lr on batches of `batch` samples drawn
 * with replacement (batch <= 0 or >= size: the whole set, in order, every
 * step); loss_per_step (host, nullable): the batch-mean loss before each step. */
hrm_status hrm_detector_train(hrm_detector* det, int32_t steps, int32_t batch, double lr, float* loss_per_step);
/* Logits of samples [first, first+n) into host z: bf16 = 1 the inference
 * (tensor-core) arithmetic, 0 the FP32 training arithmetic. HRM_E_TIMEOUT (also
 * from hrm_detector_evaluate): a bounded tensor-core wait ran out. */
hrm_status hrm_detector_logits(hrm_detector* det, int64_t first, int64_t n, int32_t bf16, float* z);
/* Over all samples at probability threshold: counts = {gated & smooth,
 * gated & not smooth, not gated & not smooth, not gated & smooth}; *loss = mean
 * cross-entropy. */
hrm_status hrm_detector_evaluate(hrm_detector* det, double threshold, int32_t bf16, int64_t counts[4],
                                 double* loss);

/* Copy det's current inference weights into ctx (a snapshot; det may be
 * destroyed afterwards) and allocate its gate buffers; then params.learned = 1
 * is accepted. The network runs once per direction and stage (in a gate kernel
 * before the sweep, or inside the precision form's screened sweep) on the FP32
 * planes (and their rounding residues) that the primitive kernel writes. */
hrm_status hrm_set_detector(hrm_ctx* ctx, const hrm_detector* det);
/* Fixed gate of direction dir (host, one byte per midpoint over the midpoint
 * grid of dir: n_d + 1 along d, x fastest; nonzero = gated), used at every
 * stage while params.learned = 2. */
hrm_status hrm_set_gate(hrm_ctx* ctx, int32_t dir, const uint8_t* gate);
/* The gate bytes last used in direction dir (host, same layout): 1 gated, 0
 * not gated; after a precision-form sweep that evaluated the network itself,
 * 2 marks a uniform stencil (exact node flux, no gate needed). */
hrm_status hrm_get_gate(hrm_ctx* ctx, int32_t dir, uint8_t* gate);

/* Diagnostic, not a step of the method: measured FMA-pipe throughput of the
 * current device in flop/s (2 flops per FMA) for HRM_FP64 or HRM_FP32, from
 * independent FMA chains on every SM (`iters` FMAs per chain); the denominator
 * of the ALU roofline of the per-midpoint kernels. Synchronises `stream`. */
hrm_status hrm_probe_fma_peak(int32_t precision, int32_t iters, void* stream, double* flops_per_s);

/* Diagnostic, not a step of the method: one CTA of 128 threads waits, with the
 * bounded wait of the tensor-core kernels (2^22 polls or 200 ms), on an
 * mbarrier phase that nothing completes. Returns HRM_E_TIMEOUT with *expired =
 * the number of waits that ran out (128); the device stays usable. Synchronises
 * `stream`. */
hrm_status hrm_probe_wait_timeout(void* stream, int64_t* expired);
/* Diagnostic (not a step of the method): the precision form converts between
 * FP32 and FP64 with integer operations on the IEEE-754 encodings (FP64
 * instructions, conversions included, are scarce on this GPU). For n elements of
 * device arrays: narrowed[i] = in_d[i] rounded to the nearest float (ties to
 * even), widened[i] = in_f[i] as a double -- which must equal the hardware
 * conversions bit for bit. Enqueued on `stream`; no synchronisation;
 * HRM_E_INVAL for n < 0 or a NULL array with n > 0. */
hrm_status hrm_probe_convert(const double* in_d, const float* in_f, int64_t n, float* narrowed, double* widened,
                             void* stream);

/* Diagnostic, not a step of the method: the bounded grid barrier of the
 * batched form's persistent kernel, made to run out: 4 blocks wait at a barrier
 * that counts 5 (nothing completes it), each wait limited to limit_ms. Returns
 * HRM_E_TIMEOUT with *expired = the waits that ran out (4); the device stays
 * usable. Synchronises `stream`. */
hrm_status hrm_probe_barrier_timeout(void* stream, double limit_ms, int64_t* expired);

/* ---------------------------------------------------------------------------
 * Batched form: many independent 2D problems of uneven size (each its own grid
 * and species table, N = 2 or 3) advanced together. Each RK stage is ONE
 * persistent cooperative launch for every instance: its blocks take work items
 * (instance, range of cells; instance, direction, 128-midpoint tile) from
 * device queues through the primitive phase (at the first stage with the CFL
 * maxima, then every instance's step scalars), the midpoint phase (both
 * directions) and the update with relaxation, separated by a grid barrier
 * whose waits are bounded (2^26 polls or 2 s). One step is one captured CUDA
 * graph of three such launches. Every instance keeps its own CFL time step
 * (params.cfl, Sec. 4.1.2) and simulated time. The per-element arithmetic is
 * that of the single-problem path: every instance reproduces an hrm_ctx of the
 * same problem bit for bit, in both forms. Only PP-WCNS-IS with SSP-RK3 is
 * offered.
 * ------------------------------------------------------------------------- */
typedef struct hrm_batch hrm_batch; /* opaque, owned by the library */

typedef struct {
  hrm_grid grid;       /* ndim must be 2; transmissive or periodic sides only */
  int32_t nspecies;    /* 2 or 3 */
  int32_t pad;
  double gamma[4], p_inf[4], c_v[4], q[4];
} hrm_instance;

/* Create a batch of ninst instances (device memory for every state and scratch).
 * Errors as hrm_create; on failure *out is NULL and hrm_batch_last_error(NULL)
 * explains. */
hrm_status hrm_batch_create(hrm_batch** out, int32_t ninst, const hrm_instance* inst,
                            const hrm_params* params, void* cuda_stream);
void hrm_batch_destroy(hrm_batch* b);
const char* hrm_batch_last_error(const hrm_batch* b);
/* Initial state of instance i from primitive planes (as hrm_set_primitive). */
hrm_status hrm_batch_set_primitive(hrm_batch* b, int32_t i, const double* prim, int32_t on_device);
/* State of instance i from W (as hrm_set). */
hrm_status hrm_batch_set(hrm_batch* b, int32_t i, const double* W, int32_t on_device);
/* Copy the state W of instance i (host: synchronises). */
hrm_status hrm_batch_get(hrm_batch* b, int32_t i, double* dst, int32_t on_device);
/* nsteps CFL steps of every instance: one graph launch per step. With
 * params.check, synchronises and returns HRM_E_TIMEOUT if a grid-barrier wait
 * ran out since the last check (the launch then left its blocks early: the
 * states are unreliable), else HRM_E_ADMISSIBILITY if any cell of any instance
 * left the admissible set. */
hrm_status hrm_batch_step(hrm_batch* b, int32_t nsteps);
hrm_status hrm_batch_time(hrm_batch* b, int32_t i, double* t, int64_t* steps);
/* Admissibility counters summed over the instances (as hrm_admissibility). */
hrm_status hrm_batch_admissibility(hrm_batch* b, int64_t counts[4]);
/* Launch shape of the persistent stage kernel: cells per work item of its
 * per-cell phases (>= 256) and blocks per SM (1 .. the most that can be
 * resident; 0 or larger values: all that fit). face_threads and face_tile are
 * accepted and ignored (midpoints go in tiles of 128, one thread each). */
hrm_status hrm_batch_set_launch(hrm_batch* b, int32_t face_threads, int32_t face_tile, int32_t cell_tile,
                                int32_t blocks_per_sm);
/* Autotuner: times steps_per_trial steps of the batch itself for each candidate
 * launch shape (cells per item {1024, 4096, 16384} x blocks per SM 1 .. the most
 * resident), restores the states after every trial, keeps the fastest and
 * writes it to best[4] (128, 128, cell_tile, blocks_per_sm). */
hrm_status hrm_batch_tune(hrm_batch* b, int32_t steps_per_trial, int32_t* best);
int64_t hrm_batch_kernel_launches(const hrm_batch* b);
int64_t hrm_batch_total_cells(const hrm_batch* b);

/* Allocation-free time step. The paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory -- an application
 * whose device memory is already owned by its own pool (for example a caching
 * allocator holding the free memory, or a fixed memory budget per solver), or a
 * time-critical loop that must not call cudaMalloc or cudaFree (both can
 * synchronise the device). It computes what hrm_dt computes (the per-direction
 * maxima tau_d = max(|u_d| + c)/dx_d and dt = cfl / sum tau_d) for a state the
 * caller owns, without a context and without calling cudaMalloc, cudaFree or
 * any allocating library routine.
 *   W_device: the state, layout above, nspecies (2..3), ndim (1..3), n[ndim],
 *             dx[ndim], species table as for hrm_create (q may be NULL);
 *   out_device: 1 + ndim doubles of device memory, receives dt then tau_d.
 * Work is enqueued on `stream` (NULL: default stream); the call does not
 * synchronise. Its only scratch is a file-scope device array of 1.5 MiB (one
 * partial maximum per 2048 cells and direction) that every GPU which loads the
 * library holds until the process exits; grids above 65536 x 2048 =
 * 134,217,728 cells are rejected with HRM_E_INVAL (hrm_last_error(NULL) says
 * why). Every call overwrites the part of the array it reads, so nothing has to
 * be cleared, but calls that overlap on the GPU (other streams, other threads)
 * share the array and race. The first call on a device looks up the array's
 * device address for that device (cudaGetSymbolAddress, once per device); make
 * that first call before any stream capture. A CUDA error left pending by
 * earlier work in the process is not taken over: the call then launches
 * nothing, returns HRM_E_CUDA and leaves that error pending for its owner. */
/* (The state's interior cells only: the prescribed states of a context's
 * Dirichlet sides, which hrm_dt includes, are not part of W.) */
hrm_status hrm_dt_noalloc(int32_t nspecies, int32_t ndim, const int64_t* n, const double* dx,
                          const double* gamma, const double* p_inf, const double* c_v,
                          const double* q, const double* W_device, double cfl,
                          double* out_device, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HRM_H */
