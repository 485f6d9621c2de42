/*
 * vlbm.h -- C ABI of the GB300 vielbein lattice Boltzmann library (libvlbm.so).
 *
 * The library advances the discrete Boltzmann equation on the unit sphere of
 * Ambrus, Busuioc, Gabbana et al., arXiv 2504.15574, Sec. 3 (Eq. Lf):
 *
 *   d f_k/dt = L[f]_k = - flux-form advection in theta and phi  (Sec. 3.5, Eq. discrete_advection_sphere)
 *                       - geometric force via K^H, Ktilde^H       (Sec. 3.3, Eqs. df, kernels)
 *                       - (f_k - f^eq_k) / tau                    (Sec. 3.2, App. A.2 Eq. feq_Q=4)
 *
 * with the D2Q16 Gauss-Hermite velocity set (App. A.2, Tab. velocity_set_Q=4),
 * WENO-5 fluxes (Eqs. fluxes_W5, WENO5_delta, WENO5_sigma), periodic phi and
 * pole boundary conditions (Sec. 3.6, Eqs. bcs_phi, bcs_theta) and SSP-RK3
 * time stepping (Sec. 3.7).  Every step runs in CUDA kernels for sm_103a; there
 * is no CPU fallback: without a usable GPU every call that needs one returns
 * VLBM_ERR_CUDA.
 *
 * Conventions shared by every entry point:
 *   - Grid: n_theta rows x n_phi columns, cell-centred (Eq. discrete_coord_sphere):
 *     theta_s = pi (s - 1/2) / n_theta, phi_q = 2 pi (q - 1/2) / n_phi.
 *   - Host moment arrays are row-major [n_theta][n_phi] doubles; element
 *     (s-1)*n_phi + (q-1) is cell (s, q).  Velocities are vielbein (orthonormal
 *     frame) components u^theta-hat, u^phi-hat; rho = n (particle mass 1), T0 = 1.
 *   - Population arrays are [16][n_theta][n_phi] doubles, population
 *     k = 4 a + b with v_theta = v[a], v_phi = v[b] and v ascending
 *     (v[0] = -sqrt(3+sqrt6) < v[1] < v[2] < v[3] = sqrt(3+sqrt6)).
 *   - Ownership: the caller owns every host buffer and may reuse it as soon as
 *     the call returns (the library copies, it keeps no host pointer).  The
 *     library owns its device memory and the handle.
 *   - Threading: a handle is used by one host thread at a time.  Its kernels
 *     run on the stream given in vlbm_options (NULL: a stream the handle owns);
 *     an FP32 step with the polar filter also forks onto a second stream the
 *     handle owns (highest priority) and joins back before the step ends, so all
 *     work is ordered on the handle's stream as seen by the caller.
 *   - Errors: every int-returning call returns VLBM_OK or a negative code;
 *     vlbm_last_error() gives a message.  A NULL handle or buffer is VLBM_ERR_ARG.
 */
#ifndef VLBM_H
#define VLBM_H

#include <stddef.h>

#if defined(__GNUC__)
#define VLBM_API __attribute__((visibility("default")))
#else
#define VLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define VLBM_OK               0
#define VLBM_ERR_ARG         -1  /* invalid argument (size, pointer, parameter) */
#define VLBM_ERR_UNSUPPORTED -2  /* valid request the library does not implement */
#define VLBM_ERR_CUDA        -3  /* CUDA error, including no device and out of memory */
#define VLBM_ERR_NONFINITE   -4  /* the non-finite guard found a NaN/Inf population */
#define VLBM_ERR_TIMEOUT     -5  /* a bounded device-side wait gave up */

/* Velocity sets (App. A): the enum value is the quadrature order Q. */
#define VLBM_D2Q9  3             /* Q = 3 (App. A.1): 9 populations, second-order equilibrium */
#define VLBM_D2Q16 4

/* Advection schemes (Sec. 3.5): WENO-5, Eqs. (fluxes_W5)-(WENO5_sigma), or the
 * first/second/third-order upwind fluxes of Eq. (fluxes_U1-3). */
#define VLBM_WENO5 0
#define VLBM_U1    1
#define VLBM_U2    2
#define VLBM_U3    3

/* Storage / arithmetic precision of the populations. */
#define VLBM_FP64 0              /* f in FP64, same operation order as the FP64 oracle */
#define VLBM_FP32 1              /* delta f = f - w_k rho_ref in FP32, FP64 tables */

typedef struct vlbm vlbm_t;

typedef struct vlbm_options {
    int precision;      /* VLBM_FP64 (default) or VLBM_FP32 */
    double weno_eps;    /* regulariser of the WENO weights, wt_i = delta_i/(sigma_i+eps)^2; default 1e-6 */
    double radius;      /* sphere radius R; default 1 */
    int polar_filter;   /* 1: block-average rings near the poles after every stage (not in the
                           paper; lets dt follow the theta spacing); default 0 */
    int guard;          /* 1: vlbm_step checks every population for NaN/Inf once per call; default 1 */
    void *stream;       /* cudaStream_t to run on, or NULL for a stream the handle creates */
    double rho_ref;     /* VLBM_FP32 only: reference density of the deviation storage;
                           <= 0 means the area-weighted mean of the initial rho; default 0 */
    int tile_rows;      /* VLBM_FP32 only: rows per stage tile, 4 or 8 (0: 8; other values: VLBM_ERR_ARG);
                           tiles are 32 columns wide */
    int scheme;         /* VLBM_WENO5 (default), VLBM_U1, VLBM_U2 or VLBM_U3, in theta and phi */
    int komissarov;     /* 1: theta flux in the Komissarov form of Eqs. (Komissarov_scheme),
                           (Komissarov_sin_cos): -d/dcos(theta) of v_theta sin(theta_{s+-1/2}) times
                           the reconstruction of f at the interfaces theta_{s+-1/2} = (s - 1/2 +- 1/2)
                           dtheta; no flux crosses a pole; default 0 */
    int velocity_set;   /* vlbm_batch_create only: the members' velocity set, VLBM_D2Q16 (default; 0
                           also means D2Q16) or VLBM_D2Q9; vlbm_create takes it as an argument and
                           ignores this field */
} vlbm_options;

/* Diagnostics in FP64 (not in the paper).  Area element R^2 sin(theta) dtheta dphi. */
typedef struct vlbm_diag {
    double time;        /* simulated time t = steps * dt */
    long long steps;    /* RK3 steps taken since the last init/set */
    double mass;        /* sum rho dA */
    double momentum[3]; /* Cartesian sum rho (u^theta e_theta + u^phi e_phi) dA */
    double energy;      /* sum_k f_k |v_k|^2 / 2 dA (reported; the isothermal BGK does not conserve it) */
    double pole_flux;   /* sum over steps of dt * RK-weighted mass flux through both poles;
                           mass - mass0 - pole_flux vanishes to round-off on the FP64 path and to
                           the rounding of the FP32 state's updates on the FP32 path (0 with the
                           Komissarov theta flux: no flux crosses a pole) */
    double mass0;       /* mass at the last init/set */
    int nonfinite;      /* 1 if any population is NaN/Inf */
} vlbm_diag;

/* Fills *opt with the defaults listed above.  NULL-safe. */
VLBM_API void vlbm_default_options(vlbm_options *opt);

/* Creates a solver on an n_theta x n_phi grid.
 *   velocity_set: VLBM_D2Q16 (16 populations, Eq. feq_Q=4), or VLBM_D2Q9 (9 populations,
 *   Eq. feq_Q=3, kernels of Eq. Q3_kernels; both precisions, FP32 stored in five population
 *   pairs, the fifth with one empty member).
 *   n_theta >= 6 (three WENO ghost rows per pole), n_phi even or 1,
 *   n_theta <= 65536, n_phi <= 65536; tau > 0 (BGK relaxation time, Sec. 3.2);
 *   dt > 0 (the caller chooses it; see vlbm_max_stable_dt); opt may be NULL.
 * Allocates the device state (three population arrays with ghost rows and
 * columns); the handle owns it.  *out is set to NULL on failure. */
VLBM_API int vlbm_create(int n_theta, int n_phi, int velocity_set, double tau, double dt,
                const vlbm_options *opt, vlbm_t **out);

/* Sets f to the equilibrium of the given moments (Eq. feq_Q=4, or feq_Q=3 for D2Q9); with T != NULL
 * the Hermite projection (third order; second for D2Q9) of a Maxwellian at temperature T is used
 * instead (the BGK target stays at T0 = 1).  Resets t, steps and the pole-flux
 * budget.  Host arrays, layout [n_theta][n_phi]; T may be NULL. */
VLBM_API int vlbm_init_moments(vlbm_t *h, const double *rho, const double *u_theta, const double *u_phi,
                      const double *T);

/* Advances n >= 0 SSP-RK3 steps (Sec. 3.7) and waits for them.  Returns
 * VLBM_ERR_NONFINITE if the guard finds a NaN/Inf (the state is then left as
 * computed, readable for debugging) and VLBM_ERR_TIMEOUT if a device wait gave up. */
VLBM_API int vlbm_step(vlbm_t *h, int n);

/* Enqueues n steps on the handle's stream and returns without waiting or
 * checking (for timing and overlap); errors surface at the next vlbm_step,
 * vlbm_sync or read-back. */
VLBM_API int vlbm_step_async(vlbm_t *h, int n);

/* Waits for the handle's stream and reports deferred device errors. */
VLBM_API int vlbm_sync(vlbm_t *h);

/* Moments of the current state (Eq. f_moments_sum): rho, u^theta-hat, u^phi-hat and,
 * if T != NULL, T = sum_k f_k |v_k - u|^2 / (2 n).  Host outputs [n_theta][n_phi]. */
VLBM_API int vlbm_moments(vlbm_t *h, double *rho, double *u_theta, double *u_phi, double *T);

/* Copies the populations out / in as FP64 host arrays [Q^2][n_theta][n_phi] (k = Q k_theta + k_phi)
 * (checkpoint / resume; the FP32 path converts to and from f = w_k rho_ref + delta f).
 * vlbm_set_populations resets t, steps and the pole-flux budget. */
VLBM_API int vlbm_get_populations(vlbm_t *h, double *f);
VLBM_API int vlbm_set_populations(vlbm_t *h, const double *f);

/* FP64 diagnostics of the current state (see vlbm_diag). */
VLBM_API int vlbm_diagnostics(vlbm_t *h, vlbm_diag *out);

/* Largest dt this library considers stable: 0.25 min(dtheta, sin(dtheta/2) dphi) / v_max
 * without the polar filter, 0.25 dtheta / v_max with it (v_max = sqrt(3+sqrt6),
 * R = 1), capped at tau (the paper keeps dt below tau, Sec. 5).  Needs no GPU. */
VLBM_API int vlbm_max_stable_dt(int n_theta, int n_phi, int velocity_set, double tau, int polar_filter,
                       double *out);

/* Per-kernel time of the stages, and the number of kernels one step launches.
 * vlbm_profile_step runs n steps launching each stage kernel (over the whole grid)
 * and each polar filter individually between CUDA events on the handle's stream and
 * stores, in ms_per_stage[0..2], the mean device time of stage kernel 1, 2, 3 and in
 * ms_per_stage[3..5] that of the polar filter after stage 1, 2, 3 (0 when the
 * filter is off); ms_per_stage (6 doubles) may be NULL.  The steps give the same
 * state as vlbm_step's.  Returns in *launches (may be NULL) the launch count of one
 * vlbm_step step: 3 stage launches, plus 3 filters with the filter on, plus (FP32
 * with the filter, when some tile rows are clear of every filtered row) 3 more
 * stage launches, the stage then being split into polar and interior tile rows
 * that run on two streams. */
VLBM_API int vlbm_profile_step(vlbm_t *h, int n, double *ms_per_stage, int *launches);

/* Limit, in seconds (0 <= limit <= 10, default 1), of the FP32 stage kernels' first wait for a
 * tile's asynchronous copies.  A copy that has not arrived by then makes the kernel flag a
 * timeout, wait (at most one more second) for its copies in flight and leave the tile, and the
 * next vlbm_step / vlbm_sync returns VLBM_ERR_TIMEOUT; the state is then undefined (finite) and
 * the handle keeps the flag until the next vlbm_init_moments / vlbm_set_populations.  A limit
 * of 0 gives up whenever the copies have not landed at the first test, which exercises that path
 * on purpose.  The step graphs are rebuilt on the next step.  FP64 handles:
 * VLBM_ERR_UNSUPPORTED (no such waits). */
VLBM_API int vlbm_set_wait_limit(vlbm_t *h, double seconds);
/* Bytes of device memory the handle holds. */
VLBM_API size_t vlbm_device_bytes(const vlbm_t *h);

/* Last error message of a handle (or of the last failed vlbm_create when h is NULL).
 * The string stays valid until the next call on that handle. */
VLBM_API const char *vlbm_last_error(const vlbm_t *h);

/* Frees the handle and its device memory.  NULL-safe. */
VLBM_API void vlbm_destroy(vlbm_t *h);

/* ---- Batched ensembles (not in the paper) ----------------------------------------
 * Many independent FP32 runs of uneven grid sizes, advanced together: one
 * persistent kernel launch per RK3 stage walks the (run, tile) work items of all
 * runs, and vlbm_batch_step captures its step loop as a CUDA graph.  Every run
 * follows the same method and numerics as a VLBM_FP32 solver (the batch is a
 * scheduling of the same stage, not a different method). */
typedef struct vlbm_batch vlbm_batch_t;

/* Creates nruns FP32 solvers; arrays of length nruns give each run's grid, tau
 * and dt (same constraints as vlbm_create).  opt->precision must be VLBM_FP32
 * (VLBM_ERR_UNSUPPORTED otherwise); opt->stream is the batch's stream;
 * opt->velocity_set the members' velocity set (D2Q16 or D2Q9).  WENO-5 with the
 * Komissarov theta flux is not offered for batches (VLBM_ERR_UNSUPPORTED). */
VLBM_API int vlbm_batch_create(int nruns, const int *n_theta, const int *n_phi, const double *tau,
                               const double *dt, const vlbm_options *opt, vlbm_batch_t **out);
/* Initial moments of run `run` (as vlbm_init_moments).  Every run must be
 * initialised before the first step. */
VLBM_API int vlbm_batch_init_moments(vlbm_batch_t *b, int run, const double *rho, const double *u_theta,
                                     const double *u_phi, const double *T);
/* Advances every run n steps (graph-launched) and waits; the guard (if enabled)
 * checks all runs once per call.  _async enqueues without waiting. */
VLBM_API int vlbm_batch_step(vlbm_batch_t *b, int n);
VLBM_API int vlbm_batch_step_async(vlbm_batch_t *b, int n);
VLBM_API int vlbm_batch_sync(vlbm_batch_t *b);
/* Moments of run `run` (as vlbm_moments). */
VLBM_API int vlbm_batch_moments(vlbm_batch_t *b, int run, double *rho, double *u_theta, double *u_phi, double *T);
/* Populations of run `run` as FP64 host array [16][n_theta][n_phi] (as vlbm_get_populations). */
VLBM_API int vlbm_batch_get_populations(vlbm_batch_t *b, int run, double *f);
/* Launch schedule: tile rows (4 or 8; tiles are 32 columns wide) and persistent CTAs
 * per SM (0: the occupancy limit; -1: one CTA per (run, tile) work item, a grid over all
 * tiles instead of a persistent one). */
VLBM_API int vlbm_batch_set_schedule(vlbm_batch_t *b, int tile_rows, int ctas_per_sm);
/* Autotuner: times every schedule (tile rows x CTAs per SM) on the batch's own
 * state, restores the state, and applies the fastest.  With cache_path != NULL the
 * result is looked up in / stored to that JSON file, keyed by GPU and grid mix.
 * Outputs (each may be NULL): chosen tile rows, CTAs per SM, ms per step. */
VLBM_API int vlbm_batch_tune(vlbm_batch_t *b, const char *cache_path, int *tile_rows, int *ctas_per_sm,
                             double *ms_per_step);
/* Times n graph-launched steps with CUDA events on the batch stream. */
VLBM_API int vlbm_batch_profile(vlbm_batch_t *b, int n, double *ms_per_step, int *launches_per_step);
/* Total cells over all runs. */
VLBM_API size_t vlbm_batch_cells(const vlbm_batch_t *b);
VLBM_API const char *vlbm_batch_last_error(const vlbm_batch_t *b);
VLBM_API void vlbm_batch_destroy(vlbm_batch_t *b);

/* ---- Learned correction (not in the paper) -------------------------------------
 * A 4-layer 3x3 convolutional network (16 -> 32 -> 32 -> 32 -> 3 channels, ReLU
 * between) on a coarse grid, mapping the moments (rho, u^theta, u^phi, T) of a
 * coarse FP32 solver, cos(theta) and sin(theta) of each row, and undivided 6th
 * differences of rho, u^theta, u^phi and 4th differences of u^theta, u^phi along
 * theta and along phi (formed in FP32 on the deviations rho - 1, u, T - 1), to a
 * correction (drho, du^theta, du^phi)
 * toward a finer run.  Padding and the differences follow the sphere: periodic in
 * phi; beyond a pole, the row on the opposite meridian with the velocity
 * components (and their differences, and sin(theta)) negated (Sec. 3.6, Eq.
 * bcs_theta, applied to moments).  BF16 activations and
 * weights, FP32 accumulation on the tensor cores, FP32 master weights and Adam.
 * Host arrays: inputs [4][n_theta][n_phi] (rho, u^theta, u^phi, T), targets and
 * outputs [3][n_theta][n_phi] (drho, du^theta, du^phi), physical units; the
 * network sees inputs / in_scale and predicts targets / out_scale.  Loss: the
 * sin(theta)-area-weighted mean square of the scaled residual. */
typedef struct vlbm_lc vlbm_lc_t;

/* Creates a network for an n_theta x n_phi grid (n_theta >= 4, n_phi even) with
 * weights drawn from splitmix64(seed). */
VLBM_API int vlbm_lc_create(int n_theta, int n_phi, unsigned long long seed, vlbm_lc_t **out);
/* Number of FP32 parameters; layout per layer l = 0..3: W[co][ci][3][3] then b[co]
 * (input channels of layer 0: rho-1, u^theta, u^phi, T-1, cos theta, sin theta,
 * d6_theta rho, d6_phi rho, d6_theta u^theta, d6_phi u^theta, d6_theta u^phi,
 * d6_phi u^phi, d4_theta u^theta, d4_phi u^theta, d4_theta u^phi, d4_phi u^phi). */
VLBM_API int vlbm_lc_num_params(const vlbm_lc_t *lc);
VLBM_API int vlbm_lc_get_weights(vlbm_lc_t *lc, float *w);
/* Sets the weights and resets the Adam state. */
VLBM_API int vlbm_lc_set_weights(vlbm_lc_t *lc, const float *w);
/* in_scale[14] (> 0) divides the 14 data channels (rho-1, u^theta, u^phi, T-1 and the ten
 * differences in the order above; each scaled input is then clamped to [-8, 8]);
 * out_scale[3] (>= 0) multiplies the outputs.  An output scale of 0 drops that output from
 * predictions and corrections (e.g. 0 for drho: a velocity-only correction); training with
 * it returns VLBM_ERR_ARG. */
VLBM_API int vlbm_lc_set_scales(vlbm_lc_t *lc, const double *in_scale, const double *out_scale);
/* Output forms of vlbm_lc_set_output_form. */
#define VLBM_LC_DIRECT 0
#define VLBM_LC_STREAM 1
#define VLBM_LC_VORTICITY 2
/* The form of the correction (not in the paper).  VLBM_LC_DIRECT (the default): the three
 * outputs times out_scale are (drho, du^theta, du^phi).  VLBM_LC_STREAM: output 0 times
 * out_scale[0] is a stream function psi on the cell grid of a sphere of the given radius, and
 * the correction is its curl, drho = 0, du^theta = d_phi psi / (R sin theta), du^phi =
 * -d_theta psi / R, in centred differences with psi continued across a pole by the row on the
 * opposite meridian (column + n_phi/2).  That correction has zero centred divergence: it moves
 * the vorticity without launching sound waves.  Training then fits the velocity targets
 * (residuals scaled by out_scale[1], out_scale[2]; the mean over cells and the two channels)
 * and ignores the drho target; outputs 1 and 2 of the network are unused.
 * VLBM_LC_VORTICITY: output 0 times out_scale[0] is a vorticity correction w, psi solves the
 * cell-centred finite-volume Poisson equation on the sphere, L psi = w - (sin theta-area mean
 * of w) (no flux through the pole faces; a DFT along phi and a tridiagonal solve per Fourier
 * mode), and the correction is the curl of psi as in VLBM_LC_STREAM (same training): the
 * network's output stays local while psi, an integral of the correction, spans the grid.
 * vlbm_lc_apply and vlbm_lc_rollout require radius = the solver's for both (VLBM_ERR_ARG
 * otherwise).  VLBM_ERR_ARG for an unknown form or radius <= 0; VLBM_ERR_UNSUPPORTED for the
 * vorticity form on grids whose mode solve (one CTA per four modes staging 16 n_theta bytes per
 * mode in shared memory) does not fit, n_theta above ~3,500.  Rebuilds the rollout graph. */
VLBM_API int vlbm_lc_set_output_form(vlbm_lc_t *lc, int form, double radius);
/* Forward pass: the correction in physical units (drho not mean-corrected). */
VLBM_API int vlbm_lc_predict(vlbm_lc_t *lc, const double *inputs, double *outputs);
/* Loss and its gradient with respect to every parameter (grad: num_params floats; either may be NULL). */
VLBM_API int vlbm_lc_gradients(vlbm_lc_t *lc, const double *inputs, const double *targets, double *loss,
                               float *grad);
/* One Adam step (beta 0.9 / 0.999) on one (inputs, targets) sample; returns the loss before the step. */
VLBM_API int vlbm_lc_train_step(vlbm_lc_t *lc, const double *inputs, const double *targets, float lr,
                                double *loss);
/* Corrects an FP32 solver on the network's grid in place: moments of its state,
 * forward pass, drho with its area mean removed (mass is kept), then
 * f += f^eq(rho + drho, u + du) - f^eq(rho, u) (Eq. feq_Q=4).  Device-resident. */
VLBM_API int vlbm_lc_apply(vlbm_lc_t *lc, vlbm_t *h);
/* Learned-coarse rollout: `steps` times (one RK3 step of h, then the correction of
 * vlbm_lc_apply), enqueued on the solver's stream as a captured CUDA graph (built on
 * the first call for this solver; rebuilt after vlbm_lc_set_scales,
 * vlbm_lc_set_output_form, for another solver, and once the solver's step has new launch
 * parameters: a vlbm_init_moments / vlbm_set_populations whose state changes the FP32 reference
 * density, vlbm_set_wait_limit) with no host synchronisation between steps; returns after the
 * last step with the solver's status (vlbm_sync).  h must be FP32 D2Q16 on the network's grid. */
VLBM_API int vlbm_lc_rollout(vlbm_lc_t *lc, vlbm_t *h, int steps);
VLBM_API const char *vlbm_lc_last_error(const vlbm_lc_t *lc);
VLBM_API void vlbm_lc_destroy(vlbm_lc_t *lc);

/* ---- Diagnostics without device allocation --------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that cannot
 * call cudaMalloc where they need the numbers: hosts whose device memory comes from
 * their own pool or is held to a fixed budget (a library must not grow or fragment
 * it), and latency-bound loops that cannot afford the device synchronisation an
 * allocation can cause.  It reduces a population array the caller owns and writes
 * to a device buffer the caller owns; the library allocates nothing.
 *
 *   f_dev:   device pointer, FP64 populations of the D2Q16 set, dense layout
 *            [16][n_theta][n_phi] (the layout of vlbm_get_populations for D2Q16), read
 *            only.  Arrays of another velocity set (D2Q9: 9 planes) are not supported
 *            and the call cannot tell them apart: it would read 16 planes.
 *   out_dev: device pointer to 6 doubles: mass, Cartesian momentum x, y, z, energy
 *            sum_k f_k |v_k|^2 / 2 (area element R^2 sin(theta) dtheta dphi, as in
 *            vlbm_diagnostics) and the number of cells holding a NaN or Inf population;
 *   stream:  cudaStream_t to run on (NULL: the legacy default stream).  The call
 *            only enqueues; the caller synchronises before reading out_dev.
 * Scratch: a fixed array inside the library sized for n_theta <= VLBM_NOALLOC_MAX_ROWS
 * (768 KiB per GPU that loads the library, held until exit); larger grids return
 * VLBM_ERR_ARG.  The first call on each device looks up that array's address (with
 * the device current) and caches it: make that first call before any stream capture;
 * the cached address does not survive a cudaDeviceReset of the device.  All calls
 * share the one array, so calls whose kernels overlap on the GPU race with each
 * other.  Errors: VLBM_ERR_ARG / VLBM_ERR_CUDA, message in vlbm_noalloc_last_error(). */
#define VLBM_NOALLOC_MAX_ROWS 16384
VLBM_API int vlbm_diagnostics_noalloc(const double *f_dev, int n_theta, int n_phi, double radius, double *out_dev,
                                      void *stream);
VLBM_API const char *vlbm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VLBM_H */
