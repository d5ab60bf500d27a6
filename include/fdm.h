/*
 * fdm.h -- C ABI of the GB300 (sm_103a) library for the field-dislocation-mechanics
 * layer-case time step of Morin, Brenner & Suquet (arXiv 1911.03225).
 *
 * Problem (Sec. 2.1 and Sec. 3.2.1): for a periodic plastic distortion
 * U^p = U13(x1,x2) e1 (x) e3 confined to a thin layer, find the layer-averaged shear
 * stress tau13 (static problem, Sec. 3.1.2) and advance U13 by the transport equation
 * dU13/dt + v0 |grad U13| = 0 (Sec. 3.2.3), with v0 = M (tau_y cos(U13/beta) - tau13)
 * (stress driven) or a prescribed uniform v0 (Sec. 4.1).  The Nye tensor of the layer is
 * alpha = alpha11 e1(x)e1 + alpha12 e1(x)e2 with alpha11 = -dU13/dx2, alpha12 = dU13/dx1.
 * Each step (Sec. 3.1.1): static solve with U13^n, then the Kurganov-Noelle-Petrova
 * central-upwind update (Sec. 3.2.2-3.2.3) with a CFL-bounded time step.
 *
 * Units are the dimensionless ones of Sec. 3.2.1 (lengths / b, stresses / mu, ...).
 *
 * Conventions for every call:
 *   - Host arrays are caller-owned, row-major [n2][n1] float64 (x1 fastest); they are
 *     copied in or out before the call returns.  The handle owns all device memory.
 *   - Every call returns an fdm_status and never aborts the process.  A NULL handle or
 *     pointer where one is required gives FDM_ERR_INVALID_ARG.
 *   - Calls on one handle are not thread-safe; distinct handles are independent.
 *   - Work is enqueued on the stream given to fdm_create (NULL = the legacy default
 *     stream); calls that return host data synchronise that stream.
 */
#ifndef FDM_GB300_H
#define FDM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdm_handle fdm_handle;

typedef enum {
    FDM_OK = 0,
    FDM_ERR_INVALID_ARG = 1,    /* bad parameter, size or pointer                           */
    FDM_ERR_OOM = 2,            /* device allocation failed                                  */
    FDM_ERR_NET_BURGERS = 3,    /* alpha has a non-zero mean (net Burgers vector, Sec. 4.2);
                                   a periodic U13 cannot represent it; state unchanged       */
    FDM_WARN_NOT_DIV_FREE = 4,  /* div alpha != 0 beyond tolerance (Sec. 2.1); the state was
                                   set from the divergence-free part (warning only)           */
    FDM_ERR_NONFINITE = 5,      /* a non-finite time step or field appeared                  */
    FDM_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up                         */
    FDM_ERR_DEVICE = 7,         /* a CUDA call failed                                        */
    FDM_ERR_STATE = 8,          /* call out of order (e.g. fdm_step before any fdm_set_*)    */
    FDM_ERR_TOO_LARGE = 9       /* grid exceeds the fixed scratch of fdm_static_solve_noalloc */
} fdm_status;

enum { FDM_V_PRESCRIBED = 0, FDM_V_STRESS = 1 };
enum { FDM_LOAD_STRESS = 0, FDM_LOAD_STRAIN_RAMP = 1, FDM_LOAD_ZERO_MEAN_STRESS = 2, FDM_LOAD_STRAIN_RATE = 3 };
enum { FDM_FP64 = 0, FDM_MIXED = 1, FDM_DF64 = 2 };
enum { FDM_T_MIDPOINT = 0, FDM_T_LITERAL = 1 };

/* Problem parameters (dimensionless, Sec. 3.2.1). */
typedef struct {
    int32_t n1, n2;          /* in-plane grid, each a power of two in [16, 4096]             */
    int32_t nz, nh;          /* depth of the 3-D periodic cell and of the layer in voxels;
                                nz = 0 means nz = n1 (cubic cell); 1 <= nh <= nz (Sec. 5.1)   */
    double dx;               /* cell size (> 0)                                              */
    double E, nu;            /* isotropic elasticity, mu = E / (2 (1 + nu)), -1 < nu < 0.5    */
    int32_t velocity_mode;   /* FDM_V_PRESCRIBED (Sec. 4.1) or FDM_V_STRESS (Sec. 3.2.3)      */
    double v0;               /* prescribed celerity                                          */
    double mobility;         /* M = 1 / eta~ (Sec. 3.2.1)                                    */
    double tau_y, beta;      /* lattice-friction amplitude and period of G (Sec. 3.2.1);
                                tau_y = 0 disables the term.  Meaningful in FDM_FP64 only.   */
    double theta;            /* minmod limiter parameter in [1, 2] (Sec. 3.2.2)               */
    double cfl;              /* |v0|max dt / dx (Sec. 4.3, Sec. 5.2), in (0, 1]               */
    double dt_max;           /* upper bound on dt (<= 0: none); dt when every v0 is 0         */
    int32_t loading_mode;    /* FDM_LOAD_* (Sec. 3.1.2 sigma-hat(0); Sec. 5.1)                 */
    double sigma_bar13;      /* FDM_LOAD_STRESS: macroscopic stress                          */
    double eps_bar13_0;      /* FDM_LOAD_STRAIN_RAMP: eps_bar13 = eps_bar13_0 + rate * step;
                                FDM_LOAD_STRAIN_RATE: eps_bar13 = eps_bar13_0 + rate * t
                                (Sec. 5.1); FDM_LOAD_ZERO_MEAN_STRESS: eps_bar13 = <U13>/2,
                                so that sigma_bar13 = 0 (the equilibration stage, Sec. 5.1) */
    double eps_bar13_rate;
    int32_t time_level;      /* FDM_T_MIDPOINT (default) or FDM_T_LITERAL (Sec. 3.2.2 Step 3) */
    int32_t precision;       /* FDM_FP64: native FP64 throughout.
                                FDM_MIXED: FP32 arithmetic in the FFT and stencil; U13 held
                                as a pair of FP32 words (the stencil adds each step's
                                increment exactly), tau13 and spectra in FP32; the mean
                                plastic slip, loading, dt and conserved sums in FP64.
                                FDM_DF64: fields/FFT/stencil in double-word arithmetic (two
                                FP32 words, ~48-bit significand, on the FP32 pipes), scalars
                                in FP64; FP64 accuracy class at FP32-pipe speed             */
    int32_t autotune;        /* 1: at creation, time the candidate launch shapes of the step
                                kernels on this GPU and keep the fastest (cached per device,
                                precision, grid and instance count for the process, and across
                                processes in the JSON-lines file named by the environment
                                variable FDM_TUNE_CACHE, if set); 0: fixed heuristic shapes.
                                Every shape computes bit-identical values.                    */
} fdm_params;

/* Launch shapes of the step kernels of a handle (or of a batch instance's group). */
typedef struct {
    int32_t rows_per_block;      /* rows of U13 per block of the row FFT kernels               */
    int32_t cols_per_block;      /* spectral columns per block of the column kernel            */
    int32_t stencil_block_rows;  /* stencil block: 32 x stencil_block_rows threads             */
    int32_t stencil_nodes;       /* nodes per stencil thread, stacked along x2                 */
    int32_t stencil_min_blocks;  /* blocks per SM the stencil's register budget keeps resident */
    int32_t tuned;               /* 1: chosen by timing on this GPU, 0: heuristic              */
    double kernel_us[4];         /* tuned: best measured time of each step kernel (row forward,
                                    column pass, row inverse, stencil) in microseconds; else 0 */
} fdm_launch_config;

/* Scalars after the last step of a call.  The sums are over all nodes of the staggered
 * Nye components a12 = (U_{j+1,k} - U_{jk})/dx, a11 = -(U_{j,k+1} - U_{jk})/dx; the total
 * Burgers vector per unit length is dx^2 (sum_pos + sum_neg) of each (Sec. 4.2). */
typedef struct {
    int64_t step;            /* steps taken since the last fdm_set_*                           */
    double t;                /* dimensionless time                                             */
    double dt;               /* last time step                                                 */
    double max_abs_v0;       /* max |v0| of the last step                                      */
    double mean_up13;        /* <U13> over the layer after the last step                      */
    double eps_bar13;        /* macroscopic strain for the next step                          */
    double sigma_bar13;      /* macroscopic stress for the next step                          */
    double sum_a12_pos, sum_a12_neg, sum_a11_pos, sum_a11_neg, sum_abs_alpha;
    int32_t status;          /* fdm_status of the device-side checks                           */
} fdm_step_info;

enum {
    FDM_FIELD_UP13 = 1,      /* U13                                                          */
    FDM_FIELD_ALPHA11 = 2,   /* alpha11 = -dU13/dx2, spectral derivative                     */
    FDM_FIELD_ALPHA12 = 4,   /* alpha12 =  dU13/dx1, spectral derivative                     */
    FDM_FIELD_TAU13 = 8,     /* layer-averaged stress of the last static solve                */
    FDM_FIELD_V1 = 16,       /* V = v0 (alpha12, -alpha11) / |alpha| (Sec. 4.1), 0 where     */
    FDM_FIELD_V2 = 32        /*   |alpha| = 0                                                */
};

/* Fills p with the defaults: nz = 0, nh = 4, dx = 1, E = 1, nu = 0.3, prescribed v0 = 1,
 * M = 1, tau_y = 0, beta = 1, theta = 1, cfl = 0.5, dt_max = 0, stress loading 0,
 * midpoint time level, FP64, autotune = 1.  n1 = n2 = 0 (must be set). */
void fdm_default_params(fdm_params *p);

/* Bytes of device memory a handle with these parameters holds (0 if invalid). */
size_t fdm_device_bytes(const fdm_params *p);

/* Validates p, allocates device memory, builds the twiddle tables and the layer Green
 * kernel K(xi1,xi2) of Sec. 3.1.2/3.2.1.  stream: a cudaStream_t or NULL.  On success
 * *out is a new handle; on failure *out is NULL and nothing is leaked. */
fdm_status fdm_create(const fdm_params *p, void *stream, fdm_handle **out);

/* Sets the state from a Nye field (Sec. 2.2, Poisson problem for U^p_0; Sec. 3.1.2,
 * U^p-hat = i (alpha-hat x xi)/|xi|^2): U13-hat = i (a11-hat xi2 - a12-hat xi1)/|xi|^2,
 * <U13> = mean_up13.  alpha11, alpha12: host [n2][n1].  Returns FDM_ERR_NET_BURGERS if
 * |<alpha>| > 1e-9 max|alpha| (state unchanged), FDM_WARN_NOT_DIV_FREE if the relative
 * divergence residual exceeds 1e-6 (state set from the divergence-free part).  If
 * div_residual is not NULL it receives the residual
 * |xi1 a11-hat + xi2 a12-hat| / (|xi| |alpha-hat|) (l2 over the spectrum). Resets step/t. */
fdm_status fdm_set_density(fdm_handle *h, const double *alpha11, const double *alpha12,
                           double mean_up13, double *div_residual);

/* Sets U13 directly (host [n2][n1]); resets step and t to 0.  Used for restarts. */
fdm_status fdm_set_plastic_distortion(fdm_handle *h, const double *up13);

/* Overrides the step counter and time (restart of a run written out earlier). */
fdm_status fdm_set_clock(fdm_handle *h, int64_t step, double t);

/* Static problem only (Sec. 3.1.2): tau13 for the current U13 and loading; readable with
 * FDM_FIELD_TAU13 afterwards. */
fdm_status fdm_static_solve(fdm_handle *h);

/* Advances nsteps >= 0 steps (Sec. 3.1.1).  If info is not NULL it receives the scalars of
 * the last step (this adds one small reduction and a device-to-host copy).  Returns the
 * first device-side error seen (FDM_ERR_NONFINITE) or FDM_OK. */
fdm_status fdm_step(fdm_handle *h, int32_t nsteps, fdm_step_info *info);

/* Enqueues nsteps >= 0 steps on the handle's stream and returns without waiting.
 * Device-side errors surface at the next synchronising call (fdm_sync, fdm_step,
 * fdm_get_info).  Requires that no partial step is pending (see fdm_enqueue_phase). */
fdm_status fdm_enqueue_steps(fdm_handle *h, int32_t nsteps);

/* Enqueues one kernel ("phase") of a step without waiting, so that a caller can bracket
 * each kernel with its own stream events.  Phases of a step are 0 .. k-1 with
 * k = fdm_kernels_per_step(h) and must be issued in that order: 0 row transforms of U13,
 * 1 spectral column pass with the Green kernel, 2 inverse row transforms giving tau13 and
 * max |v0|, 3 transport update (which completes the step).  FDM_ERR_STATE on a phase out
 * of order. */
fdm_status fdm_enqueue_phase(fdm_handle *h, int32_t phase);

/* Waits for the handle's stream; returns the first device-side error (or FDM_OK). */
fdm_status fdm_sync(fdm_handle *h);

/* Copies the requested fields (mask of FDM_FIELD_*) to host arrays [n2][n1]; pointers of
 * fields not in the mask may be NULL.  Synchronises the handle's stream. */
fdm_status fdm_read_fields(fdm_handle *h, uint32_t mask, double *up13, double *alpha11,
                           double *alpha12, double *tau13, double *v1, double *v2);

/* Scalars of the current state (same content as fdm_step's info). */
fdm_status fdm_get_info(fdm_handle *h, fdm_step_info *info);

/* Host-side fault injection for tests of the error paths: the n-th device or pinned-host
 * allocation from now on (0 = the next one) fails as if the device were out of memory, once;
 * n < 0 switches it off.  Process-wide; not thread-safe.  The call that hits the failure
 * returns FDM_ERR_OOM and releases everything it had allocated. */
void fdm_debug_fail_allocation(int32_t n);

/* Number of kernel launches one step issues (for launch accounting). */
int32_t fdm_kernels_per_step(const fdm_handle *h);

/* sigma13 of the current state on planes of the 3-D periodic cell (Sec. 3.1.2 static problem
 * on the cell of nz voxels; the layer occupies planes 0 .. nh-1, Sec. 3.2.1): planes[k] in
 * [0, nz), out [nplanes][n2][n1] (host, float64).  The layer average of these planes is
 * tau13.  For each plane the 3-D transform's sum over xi3 is folded into a 2-D symbol,
 * (1/nz) sum_k3 m(xi) D(k3) cos(2 pi k3 (x3 - (nh - 1)/2) / nz) with D(k3) the layer's
 * transform sin(pi k3 nh / nz) / sin(pi k3 / nz), built on the GPU in O(n1 n2 nz), then
 * applied by the static-solve kernels.  Leaves the state and its scalars unchanged. */
fdm_status fdm_read_stress13_planes(fdm_handle *h, int32_t nplanes, const int32_t *planes, double *out);

/* Heterogeneous elasticity (Sec. 3.1.2, heterogeneous medium) for a plastic layer filling
 * the cell (p.nh == p.nz, else FDM_ERR_INVALID_ARG): U^p = U13(x1, x2) e1 (x) e3 is then
 * uniform along x3 and the static problem is antiplane shear in a medium of shear modulus
 * mu(x) = mu * mu_factor[x] (mu = E / (2 (1 + nu)); mu_factor host [n2][n1], every entry
 * finite and > 0).  Unknown g = grad u3; sigma13 = mu(x) (g1 - U13), sigma23 = mu(x) g2.
 * With the reference medium mu0 = (min mu + max mu) / 2 the polarisation is
 * tau = (mu - mu0) g - mu (U13, 0), and the paper's series expansion is summed by the
 * fixed-point iteration g <- G - Gamma0 * tau(g), Gamma0-hat(xi) = xi (x) xi / (mu0 |xi|^2)
 * (odd products xi1 xi2 zeroed at Nyquist indices), g-hat(0) = G, starting from g = 0.
 * Loading of the current step: FDM_LOAD_STRESS and FDM_LOAD_ZERO_MEAN_STRESS prescribe
 * <sigma13> (G follows from each iterate's <tau>); the strain modes prescribe
 * <g1> = 2 eps_bar13, <g2> = 0.  Stops when rms(g_new - g) <= tol max(rms(g_new),
 * rms(U13 - <U13>)) or after max_iter (>= 1) iterations; tol = 0 runs exactly max_iter.
 * Writes sigma13 to the handle's tau13 (fdm_read_fields) and, when not NULL, to the host
 * arrays sigma13 and sigma23 ([n2][n1] float64); iterations and residual (nullable) receive
 * the count and the last ratio.  The state is unchanged; FDM_ERR_STATE without a state or
 * during a step, FDM_ERR_NONFINITE if the iteration diverges. */
fdm_status fdm_static_solve_heterogeneous(fdm_handle *h, const double *mu_factor, double tol, int32_t max_iter,
                                          double *sigma13, double *sigma23, int32_t *iterations,
                                          double *residual);

/* Heterogeneous elasticity for a plastic layer thinner than the cell (Sec. 3.1.2,
 * heterogeneous medium; the layer of nh planes in the cell of nz, Sec. 3.2.1), FDM_FP64
 * handles with nz even.  The medium is isotropic with both Lame moduli scaled by
 * mu_factor(x1, x2) (host [n2][n1], finite, > 0), uniform through the cell's depth; the
 * eigenstrain is eps^p_13 = eps^p_31 = U13(x1, x2) chi(x3) / 2 of the current state.  The
 * paper's series expansion is summed by the fixed-point iteration on the strain,
 *   eps <- E - Gamma0 * ((C - C0) : eps - C : eps^p),
 * from eps = 0, with the isotropic reference C0 = f0 C, f0 = (min + max of mu_factor) / 2, and
 * the Green operator's terms odd in an axis at its Nyquist frequency removed (the operator
 * averaged over that axis's sign).  Because the medium does not vary along x3 the Fourier
 * modes in x3 are independent: the GPU iterates the nz/2 + 1 modes' complex 2-D fields
 * together.  Loading of the current step as fdm_static_solve_heterogeneous: stress control
 * prescribes the cell average <sigma> = sigma_bar13 (e1 (x) e3 + e3 (x) e1) (E from each
 * iterate), strain control E = eps_bar13 (e1 (x) e3 + e3 (x) e1).  Stops when
 * rms(eps_new - eps) <= tol max(rms(eps_new), rms(eps^p - <eps^p>)) over the cell (Frobenius)
 * or after max_iter iterations (tol = 0: exactly max_iter).  Writes the layer average of
 * sigma13 = 2 mu_factor mu (eps13 - eps^p13) to tau13 (host [n2][n1]) and, for nplanes > 0,
 * sigma13 on planes[k] in [0, nz) to sigma13_planes ([nplanes][n2][n1]).  Device memory of
 * the solve, allocated and freed by the call: 3 x 12 (nz/2 + 1) n1 n2 doubles plus the
 * outputs (FDM_ERR_OOM when it does not fit).  The state is unchanged.  Errors:
 * FDM_ERR_INVALID_ARG (not FP64, nz odd, bad field or planes), FDM_ERR_STATE (no state, or a
 * step in progress), FDM_ERR_NONFINITE (the iteration diverged). */
fdm_status fdm_static_solve_heterogeneous_layer(fdm_handle *h, const double *mu_factor, double tol, int32_t max_iter,
                                                double *tau13, int32_t nplanes, const int32_t *planes,
                                                double *sigma13_planes, int32_t *iterations, double *residual);

/* Time steps with heterogeneous elasticity: mu_factor (host [n2][n1], as for
 * fdm_static_solve_heterogeneous; requires nh == nz) becomes the shear-modulus field of every
 * later fdm_static_solve and step of the handle, whose static problem is then the
 * fixed-point iteration above with tol and max_iter; the step's dt follows the resulting
 * max |v0| (Sec. 5.2) and the transport is unchanged.  The iteration's stopping test runs on
 * the host, so fdm_step and fdm_enqueue_steps return when their steps are done and
 * fdm_enqueue_phase is refused (FDM_ERR_STATE).  mu_factor NULL returns to the layer solve.
 * A later fdm_static_solve_heterogeneous replaces the field.  Errors as
 * fdm_static_solve_heterogeneous; FDM_ERR_STATE during a step. */
fdm_status fdm_set_shear_modulus_field(fdm_handle *h, const double *mu_factor, double tol, int32_t max_iter);

/* Stress components, Voigt order. */
enum { FDM_S11 = 0, FDM_S22 = 1, FDM_S33 = 2, FDM_S23 = 3, FDM_S13 = 4, FDM_S12 = 5 };

/* Any component of the stress of the current state on planes of the 3-D periodic cell (Sec.
 * 3.1.2 static problem for U^p = U13(x1, x2) chi(x3) e1 (x) e3, chi = 1 on planes 0 .. nh-1).
 * comp: FDM_S11 .. FDM_S12; FDM_S13 is fdm_read_stress13_planes.  planes[k] in [0, nz),
 * out [nplanes][n2][n1] (host, float64, caller-owned).  Per unit U13-hat and n = xi/|xi|
 * the isotropic Green-operator symbols are
 *   11: 2 mu n1 n3 (1 - n1^2)/(1 - nu)      22: 2 mu n1 n3 (nu - n2^2)/(1 - nu)
 *   33: 2 mu n1 n3 (1 - n3^2)/(1 - nu)      23: mu n1 n2 (1 - 2 n3^2/(1 - nu))
 *   13: -mu (n2^2 + 2 n1^2 n3^2/(1 - nu))   12: mu n2 n3 (1 - 2 n1^2/(1 - nu));
 * the sum over xi3 at plane x3 folds into a 2-D symbol (cos weights for symbols even in n3,
 * i times sin weights for odd ones), applied by the static-solve kernels.  A symbol odd in
 * one direction is zero at that axis's Nyquist index.  The plane means are sigma_bar13 for
 * 13 and zero for the others.  Leaves the state unchanged.  Errors: FDM_ERR_INVALID_ARG
 * (null handle, comp or plane out of range, null arrays with nplanes > 0), FDM_ERR_STATE
 * (no state, or a step in progress). */
fdm_status fdm_read_stress_planes(fdm_handle *h, int32_t comp, int32_t nplanes, const int32_t *planes,
                                  double *out);

/* Switches the macroscopic loading between stages of a run (Sec. 5.1: equilibration at
 * zero mean stress, then a strain rate): the next step uses the new mode and values; step
 * and time carry on.  Same validation as fdm_create; waits for the stream. */
fdm_status fdm_set_loading(fdm_handle *h, int32_t mode, double sigma_bar13, double eps_bar13_0,
                           double eps_bar13_rate);

/* The equilibration stage of Sec. 5.1: switches the loading to FDM_LOAD_ZERO_MEAN_STRESS and
 * steps in chunks of `chunk` steps until a chunk changes U13 by less than tol in relative L2
 * (||U_after - U_before|| / ||U_before||, reduced on the device in FP64; only two numbers per
 * chunk leave the device) or max_steps steps are taken.  *taken (nullable) receives the steps
 * taken, *change (nullable) the last relative change.  The loading stays at zero mean stress.
 * Errors: FDM_ERR_INVALID_ARG (tol <= 0, chunk < 1, max_steps < 0), FDM_ERR_STATE (no state),
 * the first device-side error of a chunk. */
fdm_status fdm_equilibrate(fdm_handle *h, double tol, int32_t chunk, int64_t max_steps, int64_t *taken,
                           double *change);

/* Heterogeneous drag (Sec. 5.3, Orowan mechanism: precipitates with infinite drag):
 * factor[n2][n1] (host, float64, finite, >= 0) multiplies the celerity of every node,
 * v0(x) = m(x) v0_law(x), i.e. eta(x) = eta~ / m(x); m = 0 inside impenetrable particles,
 * whose nodes then never change.  NULL restores m = 1.  The time step follows the
 * resulting max |v0|.  Copied to the device; waits for the stream. */
fdm_status fdm_set_mobility_field(fdm_handle *h, const double *factor);

/* Launch shapes the handle's step kernels use (see fdm_params.autotune). */
fdm_status fdm_get_launch_config(const fdm_handle *h, fdm_launch_config *cfg);

/* Pins the launch shapes (e.g. a configuration stored from an earlier run): rows and
 * columns per block and the stencil's (block rows, nodes, min blocks) must be one of the
 * candidates of this grid and precision (FDM_ERR_INVALID_ARG otherwise; tuned and
 * kernel_us are ignored).  Waits for the stream; FDM_ERR_STATE while a step is partially
 * enqueued.  Results are the same for every shape. */
fdm_status fdm_set_launch_config(fdm_handle *h, const fdm_launch_config *cfg);

/* The configurations the autotuner times for these parameters (no GPU needed): entry i
 * pairs the i-th candidate of each kernel, cycling through the shorter lists, so that every
 * candidate of every kernel appears.  Writes min(count, max) entries to out (may be NULL
 * when max is 0) and returns count, or 0 for invalid parameters. */
int32_t fdm_launch_candidates(const fdm_params *p, fdm_launch_config *out, int32_t max);

/* Measured arithmetic rate of the current GPU, for the roofline fractions of kernels bound
 * by arithmetic rather than by memory (not part of the paper's method).  A kernel of
 * independent multiply-add chains occupies every SM for about 50 ms (after calibration
 * launches) and is timed with CUDA events on `stream` (NULL = legacy default stream); the
 * best of three launches is returned in *gflops as 1e9 flops per second, a multiply-add
 * counting two flops.  precision: FDM_FP64 (FP64 fused multiply-add), FDM_MIXED (FP32 fused
 * multiply-add) or FDM_DF64 (a double-word multiply then a double-word add, the library's
 * FP32-pair arithmetic, counted as two FP64-equivalent flops).  The rate depends on the SM
 * clock at the time of the call.  Allocates and frees a small device buffer and waits for
 * the stream.  Errors: FDM_ERR_INVALID_ARG (bad precision, NULL gflops), FDM_ERR_OOM,
 * FDM_ERR_DEVICE. */
fdm_status fdm_measure_arith_rate(int32_t precision, void *stream, double *gflops);

/* Test hook (not part of the paper's method): y[i] = 1/sqrt(x[i]) (op 0) or 1/x[i] (op 1)
 * as the FP64 stencil computes them (Sec. 3.2.3: the one-sided speeds, the midpoint
 * predictor and |grad| use the first, the Step 4 weights the second), for checking those
 * routines' accuracy.  x, y: n doubles in host memory (caller-owned).  op 0 is defined for
 * x[i] > 0 (+inf gives 0, NaN gives NaN), op 1 for any x[i] (IEEE division outside the
 * normal range).  Allocates and frees 16 n bytes of device memory and waits for the legacy
 * default stream.  Errors: FDM_ERR_INVALID_ARG (op not 0 or 1, n < 0, NULL array with
 * n > 0), FDM_ERR_OOM, FDM_ERR_DEVICE. */
fdm_status fdm_debug_fp64_math(int32_t op, const double *x, double *y, int64_t n);

/* Static solve that allocates no device memory (the paper has no counterpart: this entry
 * point exists for callers that cannot allocate -- e.g. a process whose HBM is already
 * fully handed out to other buffers, or an embedding that forbids allocations outside its
 * own pool).  Computes tau13 = IFFT(K FFT(U13)) + sigma_bar13 exactly like fdm_static_solve
 * with FDM_LOAD_STRESS, in FP64, for caller-owned DEVICE arrays d_up13 (input) and
 * d_tau13 (output), both [n2][n1] float64 and 16-byte aligned; the two ranges may not
 * overlap (FDM_ERR_INVALID_ARG otherwise).  Only the grid, nz, nh, dx, E and nu fields of p are used;
 * p->precision must be FDM_FP64.
 * Limits: n1, n2 <= 256 and nz <= 4096; larger grids return FDM_ERR_TOO_LARGE.
 * All intermediates live in one fixed device array of 692,992 bytes that every GPU which
 * loads this library holds until the process exits.  The first call on a device sets that
 * device up (resolves the array's address, sets kernel attributes).  With CUDA's default
 * lazy module loading that first call is also when the driver brings the library's device
 * code and this array onto the device, which needs device memory: make one call (or set
 * CUDA_MODULE_LOADING=EAGER) before committing the rest of the device memory, and before
 * any stream capture.  If the driver cannot get that memory the call returns FDM_ERR_OOM.
 * Every call uses the same array: calls that overlap on the GPU (different streams or
 * threads at once) race and give wrong results; serialise them.
 * Work is enqueued on `stream` (NULL = legacy default stream) and the call returns without
 * waiting; no cudaMalloc, cudaFree or other allocating routine is called. */
fdm_status fdm_static_solve_noalloc(const fdm_params *p, double sigma_bar13, const double *d_up13,
                                    double *d_tau13, void *stream);

/* Frees everything; NULL-safe. */
void fdm_destroy(fdm_handle *h);

/* ---------------------------------------------------------------------------------
 * Batches: many independent instances stepped together.  Instances with identical
 * parameters form a group; each step runs every kernel once per group over all of the
 * group's instances (the instance is a grid dimension), and steps are replayed from CUDA
 * graphs.  Every instance has a step budget: a step advances only instances whose budget
 * is non-zero and decrements it, so instances of different lengths share launches and
 * finished or empty slots cost almost nothing.  Same conventions as the single-instance
 * calls (host arrays [n2][n1] float64, status codes, the stream given at creation).
 * --------------------------------------------------------------------------------- */
typedef struct fdm_batch fdm_batch;

/* count >= 1 instances, params[i] for instance i (each valid as for fdm_create). */
fdm_status fdm_batch_create(int32_t count, const fdm_params *params, void *stream, fdm_batch **out);

/* Bytes of device memory fdm_batch_create would hold for these instances (0 if invalid). */
size_t fdm_batch_device_bytes(int32_t count, const fdm_params *params);

/* Sets instance i's U13 (host [n2][n1]), resets its step and time to 0 and its budget to 0
 * (idle until fdm_batch_set_budget). */
fdm_status fdm_batch_set_plastic_distortion(fdm_batch *b, int32_t i, const double *up13);

/* Sets the number of further steps instance i takes (>= 0).  Enqueued on the stream. */
fdm_status fdm_batch_set_budget(fdm_batch *b, int32_t i, int64_t steps);

/* Enqueues nsteps batched steps (instances with budget 0 are skipped); no wait. */
fdm_status fdm_batch_enqueue_steps(fdm_batch *b, int32_t nsteps);

/* Waits for the stream; copies every instance's remaining budget to steps_left[count]
 * (may be NULL) and returns the first device-side error of any instance. */
fdm_status fdm_batch_sync(fdm_batch *b, int64_t *steps_left);

/* As fdm_batch_sync, but instance errors do not fail the call: status[count] (may be NULL)
 * receives each instance's device-side status (FDM_OK, or FDM_ERR_NONFINITE once a time
 * step or max |v0| stopped being finite), so that a server can retire a failed instance and
 * keep the others running.  Returns only errors of the call itself. */
fdm_status fdm_batch_sync_status(fdm_batch *b, int64_t *steps_left, int32_t *status);

/* Scalars of instance i (as fdm_get_info). */
fdm_status fdm_batch_get_info(fdm_batch *b, int32_t i, fdm_step_info *info);

/* Copies U13 and/or tau13 of instance i (mask of FDM_FIELD_UP13 | FDM_FIELD_TAU13). */
fdm_status fdm_batch_read_fields(fdm_batch *b, int32_t i, uint32_t mask, double *up13, double *tau13);

/* Enqueues nsteps batched steps (as fdm_batch_enqueue_steps) as ONE persistent launch: a
 * cooperative grid of resident blocks runs, step after step, the four phases of the step
 * (row transforms, column pass with the Green kernel, inverse rows with max |v0| and dt,
 * transport; Sec. 3.1.1) for every group, the blocks taking the phase's tiles of every
 * instance in turn, with a grid-wide barrier between phases.  Results equal those of
 * fdm_batch_enqueue_steps bit for bit.  Every barrier wait is bounded (1 s by default): a
 * block that gives up records FDM_ERR_TIMEOUT, all blocks leave, the next fdm_batch_sync*
 * returns FDM_ERR_TIMEOUT, and the batch's states are then undefined until set again.
 * Requires every instance to be FDM_MIXED with n1 >= 32 (FDM_ERR_INVALID_ARG otherwise);
 * the first call allocates the launch's descriptors.  Returns without waiting. */
fdm_status fdm_batch_enqueue_steps_persistent(fdm_batch *b, int32_t nsteps);

/* Test hook of the persistent step's barrier: from the next launch on, each barrier waits for
 * extra_arrivals more blocks than the grid holds (so with extra_arrivals > 0 no wait ever
 * completes) and a wait gives up after limit_seconds (<= 0: the default 1 s).  Process-wide;
 * fdm_debug_barrier(0, 0) restores the defaults. */
void fdm_debug_barrier(int32_t extra_arrivals, double limit_seconds);

/* Kernel launches one batched step issues (kernels per step x groups). */
int32_t fdm_batch_launches_per_step(const fdm_batch *b);

/* Launch shapes of the group holding instance i. */
fdm_status fdm_batch_get_launch_config(const fdm_batch *b, int32_t i, fdm_launch_config *cfg);

/* Frees everything; NULL-safe. */
void fdm_batch_destroy(fdm_batch *b);

/* Static description of a status code. */
const char *fdm_status_str(fdm_status s);

#ifdef __cplusplus
}
#endif
#endif /* FDM_GB300_H */
