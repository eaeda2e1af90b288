/*
 * pat.h -- C ABI of the GB300 (sm_103a) photoacoustic forward/adjoint library.
 *
 * Method: Javaherian & Holman, "A Multi-Grid Iterative Method for Photoacoustic Tomography",
 * arXiv:1603.02329.  The library evaluates the discrete forward operator H = M w P of Sec. III
 * (k-space pseudospectral time stepping of the first-order acoustic system of Sec. II.A,
 * Eqs. (mom), (mass), (state), (Twelve), with a split-field PML, Sec. VI.A) and its exact
 * transpose H^T (the discrete counterpart of the analytic adjoint of Sec. III, Eqs. (moma),
 * (massa), (statea), (adjj)).  Every step of both solves runs in this library's own CUDA
 * kernels; there is no CPU fallback.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Fields are dense, row-major, x fastest: index (z * Ny + y) * Nx + x.  n[0] = Nx, n[1] = Ny,
 *    n[2] = Nz (Nz = 1 and n[2] ignored for ndim = 2).  Physical coordinates are grid-centred:
 *    x_i = (i - n/2) * dx.
 *  - Data (sensor time series) are [Nt][Ns], one row per time sample t = 0, dt, ..., (Nt-1) dt.
 *  - The element type of every field/data pointer is the plan's precision: float for PAT_F32,
 *    double for PAT_F64.  Medium arrays passed to pat_plan_create are always double.
 *  - Field/data pointers may be host (pageable or pinned) or device pointers; the library copies
 *    them into its own device workspaces with cudaMemcpyAsync(cudaMemcpyDefault) on `stream`.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls enqueue work and
 *    return without synchronising, except where a host pointer forces the copy to complete.
 *  - Ownership: the caller owns every pointer it passes; the library never frees them.  A plan
 *    owns its device workspaces, its CUDA graphs and its tables until pat_plan_destroy.
 *  - Two calls on the same plan must not run concurrently (they share the plan's workspaces).
 *  - Errors: every call returns a pat_status; nothing aborts, traps or exits.  pat_last_error()
 *    returns a message for the calling thread's last failure.
 */
#ifndef PAT_H
#define PAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PAT_OK = 0,
    PAT_EINVAL = 1,        /* bad argument: null pointer, bad size, sensor outside the grid, ... */
    PAT_ECUDA = 2,         /* a CUDA runtime call failed (message has the CUDA error string)      */
    PAT_ENOMEM = 3,        /* device allocation failed                                           */
    PAT_ENONFINITE = 4,    /* a result contains NaN or Inf                                        */
    PAT_ETIMEOUT = 5,      /* reserved for bounded device-side waits                              */
    PAT_EUNSUPPORTED = 6   /* valid but unsupported request (e.g. an FFT length with a prime > 7) */
} pat_status;

typedef enum { PAT_F32 = 0, PAT_F64 = 1 } pat_precision;

/* Computational grid.  Every n[i] must be even and factor into 2, 3, 5, 7 (the FFT radices).
 * The PML occupies the outer pml[i] points of each axis (inside the grid); its absorption
 * rises as (depth / pml)^4 to pml_alpha nepers per grid point at the edge (Sec. VI.A uses
 * 20 points and 2 Np per point). */
typedef struct {
    int ndim;          /* 2 or 3 */
    int n[3];          /* points per axis: x, y, z */
    double dx[3];      /* spacing per axis [m] */
    int pml[3];        /* PML thickness per axis [points]; 0 = no PML on that axis */
    double pml_alpha;  /* maximum PML absorption [Np per grid point] */
} pat_grid;

/* Point sensors (Sec. III: M w restricts p to the sensors; Sec. VI.A: linear interpolation).
 * Exactly one of pos / index is non-NULL.
 *   pos   [count][ndim] physical positions (x, y[, z]) [m], grid-centred; multilinear weights.
 *   index [count] flat field indices of on-grid sensors (weight 1). */
typedef struct {
    int count;
    const double* pos;
    const int64_t* index;
} pat_sensors;

typedef struct pat_plan pat_plan;

/* Sizes of a plan, for callers that allocate inputs and outputs. */
typedef struct {
    int ndim;
    int n[3];
    int64_t N;          /* grid points */
    int Ns;             /* sensors */
    int Nt;             /* time samples */
    int lossy;          /* 1 if any alpha0 != 0 (absorption/dispersion terms active) */
    pat_precision precision;
    double dt;
    double c_ref;       /* max sound speed (kappa correction, PML scaling) */
    int path;           /* 0: CUDA graph of per-phase kernels; 1: one persistent kernel per solve;
                           2: the same, register-fused transforms (power-of-two 2-D grids) */
    int layout[2];      /* launch layout: path 0 -> columns per spectral CTA, x-lines per row CTA;
                           paths 1, 2 -> columns per CTA, x-line pairs per CTA */
    int tuned;          /* 1 when the layout was chosen by timing the feasible candidates */
    int schedule;       /* radix schedule of the 3-D spectral passes over 128- or 256-point lines, timed
                           with the layouts on path 0 (PAT_SPEC16 pins it): 0 = stages (r0, 8, ..., 8)
                           everywhere, 1 = two stages (n/16, 16) for the plain y transforms, 2 = two
                           stages for every pass, 3 = two stages for the plain transforms and for the
                           multiply passes whose fields are independent (D-, its transpose, the
                           absorption pass); 0 where no axis has such lines */
    int spec_chunks;    /* 3-D path 0: each spectral operation runs its y / z / y passes over this many
                           chunks of the half-spectrum column tiles, one chunk after the other, so
                           that a chunk's intermediate spectra can stay in L2 (timed with the layouts;
                           PAT_SPEC_CHUNKS pins it); 1 elsewhere */
    int tma;            /* 1 when the 3-D spectral passes stage their 8-column tiles with tensor-memory-access
                           copies (cp.async.bulk.tensor, FP32 plans with lines of at most 256 points) */
    int zreg;           /* 1 when the D- z passes (and with PAT_ZREG=2 every z pass with a multiply) hold
                           each 256-point line in registers: 16 x 16 transform, half a warp per line
                           (FP32 plans with tensor-copy staging and 256-point z-lines; PAT_ZREG=0 off) */
    int ywide;          /* 1 when the plain y transforms of 128- or 256-point y-lines run on 16-column tiles,
                           one field per CTA, in place in the tile staged by one tensor copy (FP32 plans
                           with tensor-copy staging; radix schedules 1-3, whose two-stage y transforms
                           they compute with the same operations; one chunk; PAT_YWIDE=0 off) */
    int zwide;          /* 1 when the z passes with the multiply (D+, D-, their transposes, the absorption
                           pass) of 128- or 256-point z-lines run on 16-column tiles transformed in place
                           in shared memory after one tensor copy per input field, with the multipliers
                           from tables the plan fills once (FP32 plans with tensor-copy staging; one
                           chunk; PAT_ZWIDE=0 off) */
    int rowu1;          /* 1 when the u update and its transpose run one velocity component per CTA (FP32
                           3-D plans with x-lines of 128 or 256 points; PAT_ROWU1=0 off) */
} pat_plan_info_t;

/* pat_plan_create -- build a plan: medium, geometry and time axis (Sec. II.A, Sec. III).
 *   c, rho   [N] host doubles: sound speed [m/s] and ambient density [kg/m^3].
 *   alpha0   [N] host doubles (or one value if alpha0_is_scalar): power-law absorption
 *            coefficient in dB MHz^-y cm^-1 (Sec. II.A); all zeros = lossless.
 *   y        power-law exponent (Sec. II.A), y != 1.
 *   sensors  sensor geometry (see pat_sensors).
 *   dt, Nt   time step [s] and number of recorded samples (t = 0 .. (Nt-1) dt), Nt >= 1.
 *   prec     arithmetic precision of the fields (PAT_F32: FP32 stepping; PAT_F64: FP64).
 * Derived per-point quantities (c0^2, 1/rho0 on the staggered grids, tau and eta of
 * Eq. (Twelve), PML factors, k-space tables, interpolation weights) are computed here in FP64
 * on the host and stored on the current device in the plan's precision.
 * Errors: PAT_EINVAL (bad sizes, NULLs, y = 1, sensor outside grid), PAT_EUNSUPPORTED (FFT
 * length not 2^a 3^b 5^c 7^d, or odd, or above 1024; more than 2^27 grid points; Nt * Ns above
 * 2^31 - 1), PAT_ENOMEM, PAT_ECUDA. */
pat_status pat_plan_create(const pat_grid* grid, const double* c, const double* rho,
                           const double* alpha0, int alpha0_is_scalar, double y,
                           const pat_sensors* sensors, double dt, int Nt, pat_precision prec,
                           pat_plan** out);

/* pat_plan_destroy -- free a plan and everything it owns (NULL is a no-op).  Synchronises the
 * device work the plan enqueued. */
pat_status pat_plan_destroy(pat_plan* plan);

/* pat_plan_get_info -- sizes of a plan. */
pat_status pat_plan_get_info(const pat_plan* plan, pat_plan_info_t* info);

/* pat_forward_plan -- data = H p0 (Sec. III: H[p0] = M w p; forward model of Sec. II.A).
 *   p0    [N]      initial pressure (host or device, plan precision).
 *   data  [Nt][Ns] output, overwritten (host or device, plan precision).
 * Runs the whole Nt-step solve on `stream` as one launch: a persistent kernel for 2-D plans whose
 * state fits in the GPU's shared memory (pat_plan_info_t.path 1 or 2), otherwise one CUDA-graph
 * launch of the per-phase kernels (path 0).  The inputs and outputs move by cudaMemcpyAsync on
 * `stream`: an output in device or page-locked host memory is ready once `stream` is synchronised,
 * one in pageable host memory when the call returns (that copy waits for the solve). */
pat_status pat_forward_plan(pat_plan* plan, const void* p0, void* data, void* stream);

/* pat_adjoint -- grad = H^T residual (Sec. III, Eq. (adjj); Sec. IV, Eq. (Six) uses it as
 * grad f = H^T (H x - p_hat)).  The transpose is exact: <H x, h> = <x, H^T h> to rounding.
 *   residual [Nt][Ns] input (host or device, plan precision).
 *   grad     [N]      output, overwritten (host or device, plan precision; ready as in
 *                     pat_forward_plan). */
pat_status pat_adjoint(pat_plan* plan, const void* residual, void* grad, void* stream);

/* pat_plan_set_smoothing -- the optional smoothing of the initial pressure (Sec. VI.A: the high
 * frequencies of p0 are filtered by a self-adjoint operator S before each forward solve, and S is
 * included in the adjoint).  enable = 1: pat_forward_plan computes H S p0, pat_adjoint returns
 * S H^T h, pat_gradient_c2 starts from S p0 and returns S H^T h, batches and pat_mg_fista follow
 * (a coarse level made by pat_plan_create_coarse inherits the switch).  enable = 0 (the default
 * after pat_plan_create) turns it off.  The paper names no filter; S = F^-1 diag(W) F with the
 * radial Blackman window W(k) = 0.42 + 0.5 cos(pi q) + 0.08 cos(2 pi q), q = |k| / k_c < 1, and
 * W = 0 for q >= 1, k_c = min over axes of pi / dx.  enable = 1 allocates a workspace of N
 * complex values (plan-owned, kept until the plan is destroyed), so the solves never allocate.
 * Errors: PAT_EINVAL (NULL plan, enable not 0 or 1), PAT_EUNSUPPORTED (static-arena plan),
 * PAT_ENOMEM. */
pat_status pat_plan_set_smoothing(pat_plan* plan, int enable);

/* pat_plan_smooth -- y = S x with the plan's window (whatever the switch), x and y [N] device
 * fields of the plan's precision (y may equal x, otherwise the two must not overlap;
 * caller-owned).  Enqueued on `stream`.
 * Errors: PAT_EINVAL (NULL argument), PAT_ENOMEM / PAT_ECUDA (workspace, launch). */
pat_status pat_plan_smooth(pat_plan* plan, const void* x, void* y, void* stream);

/* pat_gradient_c2 -- medium sensitivity: grad_c2 = d<H p0, h>/d(c0^2) at every grid point, and
 * grad_p0 = H^T h from the same reverse sweep.  The paper has no medium gradient; it follows from
 * Sec. III's adjoint-state construction applied to the discrete forward map, for the joint
 * sound-speed reconstruction that Sec. VII motivates.  Held fixed: alpha0, y, rho0 and the plan's
 * reference speed, dt, kappa and PML; tau and eta follow c0 through Eq. (Twelve).  With q^n =
 * d p^n/d c0^2 = r + (y+1)/2 tau L_{y-2} dd - (y+2)/2 eta L_{y-1} r (q = r without absorption) and
 * p_bar^n the adjoint of p^n:
 *     grad_c2 = sum_{n>=1} p_bar^n q^n - p0 / (d c0^4) sum_xi rho_bar_xi   (rho_xi^0 = p0/(d c0^2)).
 * Memory is bounded by checkpoints: the forward state (u_xi, rho_xi, spectrum of p) is stored every
 * `checkpoint_every` = K >= 1 time levels, and each segment of K levels is recomputed from its
 * checkpoint (storing its K fields q^n) just before the adjoint steps that consume it: one extra
 * forward solve in total, ceil((Nt-1)/K) checkpoints of (2d + 1) N values and K N values of q.
 * The result does not depend on K (the recomputation repeats the same operations).
 *   p0       [N]      initial pressure (host or device, plan precision).
 *   residual [Nt][Ns] h (host or device, plan precision).
 *   grad_c2  [N]      output, overwritten (host or device, plan precision).
 *   grad_p0  [N]      output or NULL.
 * Works in device memory it allocates for the call and frees before returning (the stream is
 * synchronised); PAT_ENOMEM if it cannot.  Runs the per-phase kernels (also for plans whose
 * forward/adjoint take the persistent kernel); the plan's data buffer holds `residual` afterwards. */
pat_status pat_gradient_c2(pat_plan* plan, const void* p0, const void* residual, void* grad_c2, void* grad_p0,
                           int checkpoint_every, void* stream);

/* pat_gradient_rho -- density sensitivity: grad_rho = d<H p0, h>/d(rho0) at every grid point, and
 * grad_p0 = H^T h from the same reverse sweep.  Like pat_gradient_c2, this follows from Sec. III's
 * adjoint-state construction applied to the discrete forward map, for the joint reconstruction of
 * the medium that Sec. VII motivates; the paper states no medium gradient.  Held fixed: c0, alpha0,
 * y, p0 and the plan's reference speed, dt, kappa and PML; tau and eta depend on c0 only
 * (Eq. (Twelve)).  rho0 enters the step in three places: b_xi = 2 / (rho0 + rho0 shifted by one point
 * along xi) in the momentum update and in u^{-1/2} = (dt/2) b D+ p0, -dt rho0 e_xi in the mass
 * update (e_xi = D-_xi u_xi), and dd = rho0 sum e_xi in the absorption term (Sec. II.A).  With
 * g_xi^n = D+_xi p^n, e_xi^n = D-_xi u_xi^{n+1/2} of the forward solve and the adjoint variables
 * u_bar, rho_bar, dd_bar of the exact transpose:
 *     dJ/db_xi  = sum_n u_bar_xi^{n+1/2} (-dt au_xi g_xi^n) + u_bar_xi^{-1/2} (dt/2) g_xi^0,
 *     dJ/drho0  = sum_n sum_xi e_xi^n (dd_bar^n - dt a_xi rho_bar_xi^{n+1}) + (the dJ/db part, through
 *                 db_xi[j]/drho0[j] = db_xi[j]/drho0[j + e_xi] = -b_xi[j]^2 / 2).
 * Checkpoints as in pat_gradient_c2 (the same K, the same extra forward solve); each recomputed
 * segment stores g_xi and e_xi of its K steps: (K + 1) 2d N values, plus d N accumulators.  The
 * result does not depend on K.  Arguments, memory and errors as in pat_gradient_c2 (grad_rho in
 * place of grad_c2). */
pat_status pat_gradient_rho(pat_plan* plan, const void* p0, const void* residual, void* grad_rho, void* grad_p0,
                            int checkpoint_every, void* stream);

/* pat_gradient_medium -- pat_gradient_c2 and pat_gradient_rho in one sweep (one extra forward solve in
 * all): any of grad_c2, grad_rho, grad_p0 may be NULL, not all three.  Memory is the sum of the two. */
pat_status pat_gradient_medium(pat_plan* plan, const void* p0, const void* residual, void* grad_c2, void* grad_rho,
                               void* grad_p0, int checkpoint_every, void* stream);

/* pat_time_reversal -- time-reversal image (Sec. II.B.1), the paper's comparison baseline and a warm
 * start for the iterative methods.  The measured pressure is enforced at the sensors in reversed
 * time, p(r_s, t) = data(r_s, T - t), on the plan's grid, medium, PML, time step and reference speed,
 * and the image is the pressure at the end (original time 0).  Readings:
 *   - the scheme is the forward one with tau replaced by -tau, eta kept (Sec. II.B.1 reverses the
 *     sign of the absorption term and keeps the dispersion term);
 *   - sensors must be on grid nodes, one per node (on-grid sensors; PAT_EINVAL otherwise);
 *   - start: p^0 = 0 except the last datum at the sensors, rho_xi^0 = p^0 / (d c0^2), u^{-1/2} = 0;
 *     after every step the pressure at the sensor nodes is set to the next reversed datum and the
 *     split densities to datum / (d c0^2);
 *   - compensate = 1: with the sign reversed the absorption term amplifies each mode at the rate the
 *     forward model damped it, which grows like |k|^y, and high-|k| rounding noise grows without
 *     bound.  The reversed term is therefore band-limited by the radial Blackman window
 *     W(q) = 0.42 + 0.5 cos(pi q) + 0.08 cos(2 pi q), q = |k| / k_c < 1 (0 beyond), with
 *     k_c = k_cut * min over axes of pi / dx (0 < k_cut <= 1; 0.5 recommended).  compensate = 0 keeps
 *     the forward sign (no window, k_cut ignored).
 *   data  [Nt][Ns] measured data (host or device, plan precision); image [N] output.
 * The plan's smoothing switch is not applied.  Runs the per-phase kernels on the plan's own state
 * (the first call allocates a node map of N ints and (Nt + 1) Ns values, kept by the plan). */
pat_status pat_time_reversal(pat_plan* plan, const void* data, void* image, int compensate, double k_cut,
                             void* stream);

/* pat_adjoint_atd -- the paper's own adjoint, "adjoint-then-discretize" (Sec. VI): the continuous
 * adjoint system of Sec. III (Eqs. (moma), (massa), (statea), (adjj)) discretised with the same
 * k-space staggered scheme, for comparison with the exact transpose pat_adjoint.  Readings:
 *   - the system runs forward in adjoint time on the reversed residual h~^n = h^{Nt-1-n}, from a
 *     zero state; the source M^T (h~^n + h~^{n+1}) / 2 enters the mass update at the half step,
 *     shared equally by the d split densities: rho*_xi <- a (a rho*_xi - dt rho0 e*_xi + dt rho0 s / d);
 *   - in the state equation tau and eta act before the fractional Laplacians:
 *     p* = c0^2 sum rho* - rho0 L_{y-2}(c0^2 tau (s - sum e*)) - rho0 L_{y-1}(c0^2 eta sum rho* / rho0);
 *   - the same split-field PML factors as the forward solve;
 *   - initial_paper = 1: the image is rho*(T) / rho0 (Eq. (adjj)), the gradient for the paper's
 *     initial condition c0^2 {1 - eta (-lap)^((y-1)/2)} rho(0) = p0; initial_paper = 0: the gradient
 *     for the forward map's rho^0 = p0 / (d c0^2), g - L_{y-1}(c0^2 eta g) / c0^2 with g = rho*(T)/rho0
 *     (identical when lossless).
 * The data term is a plain sum over samples (no dt weight), so dt * pat_adjoint converges to this
 * image as dt -> 0; it is not the transpose and fails the dot test by O(dt) and inside the PML.
 *   residual [Nt][Ns] (host or device, plan precision); image [N] output.  The smoothing switch
 * applies (S at the end).  The first call allocates (Nt + 1) Ns values kept by the plan. */
pat_status pat_adjoint_atd(pat_plan* plan, const void* residual, void* image, int initial_paper, void* stream);

/* ===========================================================================================
 * Batches: several independent instances in one launch
 * ===========================================================================================
 * The paper solves one problem at a time; batching independent instances (uneven grids, each with
 * its own medium, sensors and time axis) has no counterpart there.  A batch runs every instance's
 * per-phase solve (the CUDA-graph path, whatever path the plan's own calls take) as one graph
 * launch whose instances have no dependencies on one another, so the GPU overlaps them.  The
 * batch borrows the plans: destroy it before them; a plan may sit in one batch at a time and runs
 * no other call while a batch launch that holds it is in flight. */
typedef struct pat_batch pat_batch;

/* pat_batch_create -- a batch over `count` >= 1 distinct plans of one device (not static-arena
 * plans).  Graphs are captured on first use of each direction. */
pat_status pat_batch_create(pat_plan* const* plans, int count, pat_batch** out);

/* pat_batch_destroy -- waits for the device and frees the batch (not its plans). */
pat_status pat_batch_destroy(pat_batch* batch);

/* pat_batch_forward -- data[i] = H_i p0[i] for every instance i (arrays of `count` pointers,
 * host or device, each plan's precision and sizes as in pat_forward_plan). */
pat_status pat_batch_forward(pat_batch* batch, const void* const* p0, void* const* data, void* stream);

/* pat_batch_adjoint -- grad[i] = H_i^T residual[i] for every instance i (as pat_adjoint). */
pat_status pat_batch_adjoint(pat_batch* batch, const void* const* residual, void* const* grad, void* stream);

/* pat_forward -- one-shot form of the forward operator following the paper's statement of the
 * problem (Sec. II.B, Sec. III): builds a plan from (c, rho, alpha0, y, grid, sensor_mask, dt,
 * Nt), runs pat_forward_plan, synchronises `stream` and frees the plan.  For repeated solves
 * create a plan once instead. */
pat_status pat_forward(const void* p0, const double* c, const double* rho, const double* alpha0,
                       int alpha0_is_scalar, double y, const pat_grid* grid,
                       const pat_sensors* sensor_mask, double dt, int Nt, pat_precision prec,
                       void* data, void* stream);

/* ===========================================================================================
 * Optimisation shell (Sec. IV, Sec. V): image-space operators on a grid (only ndim and n[] of
 * pat_grid are used; images are [Nz][Ny][Nx], device pointers, plan-independent precision).
 * D = forward differences per axis with a zero difference at the last index (Neumann),
 * TV(x) = sum_i sqrt(sum_xi (D_xi x)_i^2) (isotropic).  Calls that return a host scalar
 * synchronise `stream`; the others only enqueue.
 * =========================================================================================== */

/* pat_tv_prox -- x = argmin_u weight * TV(u) + indicator(u >= 0 if nonneg) + 1/2 ||u - z||^2, the
 * proximal map of Sec. IV Eq. (proxmal) with weight = alpha * lambda, by n_inner iterations of the
 * dual fast gradient projection cited there (zero warm start; step 1/(4 d weight)).
 * weight <= 0 or n_inner = 0 returns the projection of z.  z and x must not alias. */
pat_status pat_tv_prox(const pat_grid* grid, const void* z, void* x, double weight, int n_inner, int nonneg,
                       pat_precision prec, void* stream);

/* pat_tv -- *value = TV(x) (rho = 0) or the smoothed J_rho(x) = sum_i (sqrt(|D x|_i^2 + rho^2) - rho)
 * of Sec. V.B Eq. (Thirty-two) (rho > 0), accumulated in FP64. */
pat_status pat_tv(const pat_grid* grid, const void* x, double rho, double* value, pat_precision prec, void* stream);

/* pat_tv_smooth_grad -- grad = D^T (D y / sqrt(|D y|^2 + rho^2)), the gradient of J_rho
 * (Sec. V.B Eq. (Twentyone) without the data term), rho > 0. */
pat_status pat_tv_smooth_grad(const pat_grid* grid, const void* y, double rho, void* grad, pat_precision prec,
                              void* stream);

/* pat_restrict / pat_prolong -- the grid transfer of Sec. V.A between the fine grid `fine` (even
 * sizes) and the coarse grid of half the points per axis: prolongation P is tensor-product linear
 * interpolation (fine 2i <- coarse i, fine 2i+1 <- mean of coarse i and min(i+1, n_c-1)),
 * restriction R = 2^-d P^T (full weighting). */
pat_status pat_restrict(const pat_grid* fine, const void* xf, void* xc, pat_precision prec, void* stream);
pat_status pat_prolong(const pat_grid* fine, const void* xc, void* xf, pat_precision prec, void* stream);

/* pat_coarse_bound -- the restricted lower bound of Sec. V.C Eq. (constraint), taken at y:
 * phi_i = (R y)_i - min_{j in {2i-1, 2i, 2i+1}^d, clamped} y_j.  x = y + P(x_c - R y) is >= 0
 * whenever x_c >= phi. */
pat_status pat_coarse_bound(const pat_grid* fine, const void* y, void* phi, pat_precision prec, void* stream);

/* pat_dot -- *out = sum_i a_i b_i over n elements, accumulated in FP64 (deterministic order). */
pat_status pat_dot(const void* a, const void* b, int64_t n, pat_precision prec, double* out, void* stream);

/* pat_power_iteration -- L_f = sigma_max(H^T H) by the power method (Sec. IV): v = v0 / ||v0||,
 * then n_iter times w = H^T H v, L = ||w||, v = w / L.  v0 [N] device, plan precision. */
pat_status pat_power_iteration(pat_plan* plan, const void* v0, int n_iter, double* L, void* stream);

/* pat_plan_create_coarse -- the next coarser level of a plan (Sec. V): half the points per axis
 * (fine sizes divisible by 4), twice the spacing, half the PML points (Sec. VI.A keeps its
 * thickness), twice the time step and ceil(Nt / 2) samples, the medium sampled at the even fine
 * points, the sensors at the same physical positions (on-grid sensors become point positions;
 * a position beyond the first or last coarse node is clamped onto that node). */
pat_status pat_plan_create_coarse(const pat_plan* fine, pat_plan** coarse);

/* Options of pat_mg_fista; the defaults of Sec. VI.A are noted. */
typedef struct {
    int variant;          /* 0: ISTA (theta = 0), 1: FISTA t-sequence (Alg. 2) */
    double lambda;        /* TV weight (1e-2) */
    double step_scale;    /* alpha = step_scale / L (2 for ISTA, 1 for FISTA) */
    double kappa;         /* recursion test, Eq. (conditions) (1/4 in 2-D, 1/8 in 3-D) */
    double vartheta;      /* recursion test (0.1) */
    int q_d;              /* recursion test (3) */
    int q_c;              /* maximum coarse iterations (8) */
    double eps_d;         /* fine stopping tolerance on the relative decrease of F (1e-3) */
    double eps_c;         /* coarse stopping tolerance on the relative decrease of phi (1e-2) */
    double tv_rho;        /* smoothing of Eq. (Thirty-two) (1e-2 in 2-D, 3e-2 in 3-D) */
    int n_tv;             /* inner iterations of the TV prox (20) */
    int max_iter;         /* fine iterations at most */
    int recursion;        /* 0: never take the coarse branch (plain ISTA / FISTA) */
    double L;             /* sigma_max(H^T H) of the fine level (pat_power_iteration) */
    double L_coarse;      /* the same for the coarse level; the coarse step is 1/(w L_coarse + 4 d lambda / tv_rho) */
    double target_re;     /* > 0: also stop when ||x - p_exact|| / ||p_exact|| <= target_re */
    const void* p_exact;  /* optional [N] device image for RE reporting (plan precision) */
    double coarse_weight; /* w of the coarse data term w/2 ||H_c x - p_c||^2; <= 0: 2^(1-d).  The paper
                             does not weight it; with R = 2^-d P^T and data decimated 2:1 in time the
                             unweighted coarse Hessian is 2^(d-1) times R (grad^2 f) P, so its minimiser
                             under-shoots by that factor (reading O11 of the optimisation oracle) */
} pat_fista_opts;

typedef struct {
    int iters, recursive_iters, fwd_solves, adj_solves;
    double F;      /* 1/2 ||H x - p_hat||^2 + lambda TV(x) at the returned x */
    double RES;    /* ||H x - p_hat|| */
    double RE;     /* ||x - p_exact|| / ||p_exact|| (NaN without p_exact) */
} pat_fista_report;

/* called after every fine iteration k >= 1 (recursive = 1 if the coarse branch was taken) */
typedef void (*pat_iter_callback)(void* ctx, int k, int recursive, double F, double RES, double RE, int fwd_solves,
                                  int adj_solves);

/* pat_mg_fista -- line-search multi-grid FISTA / ISTA with TV (Alg. 3, Sec. V.E) on two levels,
 * or plain FISTA (Alg. 2) / ISTA (Alg. 1) when coarse is NULL or opts->recursion = 0.
 *   fine, coarse   plans of the two levels (coarse from pat_plan_create_coarse, or NULL)
 *   data [Nt][Ns]  measured data p_hat (device); x0 [N] start (device); x_out [N] result (device)
 * Each fine iteration costs one forward and one adjoint solve (the cost-saving identity
 * H y_{k+1} = (1 + theta) H x_k - theta H x_{k-1}); objective values, norms and the recursion test
 * are FP64 scalars on the host (one synchronisation per reduction).  Stops when the relative
 * decrease of F falls below eps_d, after max_iter iterations, or at target_re. */
pat_status pat_mg_fista(pat_plan* fine, pat_plan* coarse, const void* data, const void* x0,
                        const pat_fista_opts* opts, void* x_out, pat_fista_report* report, pat_iter_callback cb,
                        void* cb_ctx, void* stream);

/* pat_mg_fista_levels -- the same method on nlevels >= 1 levels (at most 8): levels[0] is the fine
 * plan and levels[l] the coarse plan of levels[l - 1] (pat_plan_create_coarse); L_levels[l] is
 * sigma_max(H_l^T H_l) (pat_power_iteration; L_levels[0] takes the place of opts->L and
 * L_levels[1] of opts->L_coarse, which are not read here).  The paper states Alg. 3 for two
 * grids (Sec. V.E).  With more, the projected FISTA of a coarse level l may itself take recursive
 * directions to level l + 1 under the same test, applied to its model phi_l (reading O12 of the
 * optimisation oracle):
 *   - the coherence term is formed from grad phi_l;
 *   - the bound is restricted from level l's own bound, R y - min over the fine neighbourhood of
 *     (y - b_l);
 *   - the data term's weight compounds per level step (w_l = w^l, w as in opts->coarse_weight).
 * With two levels it is pat_mg_fista exactly.  Errors: PAT_EINVAL for NULL arguments, nlevels
 * outside 1 .. 8, a level that is not the coarse level of the one above, or L_levels <= 0 on a
 * level the recursion uses.  report->recursive_iters counts the fine level's recursive
 * iterations; fwd_solves / adj_solves count the solves of every level. */
pat_status pat_mg_fista_levels(pat_plan* const* levels, int nlevels, const double* L_levels, const void* data,
                               const void* x0, const pat_fista_opts* opts, void* x_out, pat_fista_report* report,
                               pat_iter_callback cb, void* cb_ctx, void* stream);

/* pat_plan_status -- synchronise the device and return the status of the plan's last solve
 * through pat_forward_plan or pat_adjoint:
 *   PAT_OK;
 *   PAT_ETIMEOUT if a bounded device-side wait (the grid barrier of the persistent kernel) ran out,
 *     so the kernel stopped early and its outputs are not valid;
 *   PAT_ENONFINITE if the solve's output (the data record after H, the image after H^T) holds a
 *     NaN or an infinity.  A device-side scan of the output sets it after every solve. It is cleared
 *     before the next one.
 * pat_forward_static returns PAT_ENONFINITE directly. */
pat_status pat_plan_status(pat_plan* plan);

/* Kernel-timing probe (tracing).  With stride S > 0, the next captured graphs bracket every kernel
 * launch of every S-th time step (starting at step S/2) with CUDA events; after a solve has
 * completed, pat_plan_probe_read returns, for launch slot `slot` of the step (0 <= slot <
 * pat_plan_probe_slots), its kernel name and its mean duration over the sampled steps of the last
 * solve.  stride = 0 turns the probe off.  Changing the stride drops the captured graphs (they are
 * re-captured on the next call).  `adjoint` selects the H (0) or H^T (1) graph. */
pat_status pat_plan_set_probe(pat_plan* plan, int stride);
int pat_plan_probe_slots(const pat_plan* plan, int adjoint);
pat_status pat_plan_probe_read(pat_plan* plan, int adjoint, int slot, const char** name, double* mean_ms,
                               int* samples);

/* Size of the fixed device scratch array that pat_forward_static works in: 32 MiB in the memory of
 * every GPU where the library's device code is loaded, held until the process exits.  With lazy
 * module loading (CUDA's default) that happens at the first pat_forward_static call on the GPU. */
#define PAT_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* pat_forward_static -- pat_forward for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is a deployment variant of the same forward operator H.
 *
 * Some callers cannot call cudaMalloc: an application that hands the whole device to its own pool
 * allocator and forbids any other device allocation, or a long-running service that must not
 * allocate (and so risk fragmentation or an out-of-memory failure) once it is running.  This call
 * computes exactly what pat_forward computes, with the same arguments, but allocates nothing:
 * every device buffer it needs (medium tables, state fields, spectrum workspaces, sensor lists,
 * the data record) is carved from one fixed array of PAT_STATIC_SCRATCH_BYTES that the library
 * embeds as a device global.  It calls no cudaMalloc, cudaFree or allocating library routine and
 * launches its kernels directly on `stream`; it returns after synchronising `stream`.
 *   - The caller still passes p0 and data (host or device pointers, plan precision).
 *   - A problem whose buffers do not fit in PAT_STATIC_SCRATCH_BYTES is rejected with PAT_EINVAL
 *     before any device work (for scale: a 2-D 512^2 FP32 absorbing problem with Nt = 2000 and
 *     512 sensors needs about 21 MB).
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current.  That lookup loads the library's device code and the array on the
 *     GPU, so the driver reserves the array's memory then: make one call at start-up, before a pool
 *     allocator takes the device's memory and before any stream capture on the device.  If the
 *     device has no room left for it, the call returns PAT_ENOMEM.
 *   - The plan tables are written with the legacy default stream and waited for before the solve,
 *     so `stream` may be any stream, non-blocking ones included.
 *   - Every call on a device shares that device's array, and the array keeps the last call's
 *     contents.  Calls that overlap on the same GPU (for example from several host threads) race
 *     on it: serialise them. */
pat_status pat_forward_static(const void* p0, const double* c, const double* rho, const double* alpha0,
                              int alpha0_is_scalar, double y, const pat_grid* grid,
                              const pat_sensors* sensor_mask, double dt, int Nt, pat_precision prec,
                              void* data, void* stream);

/* Phase-timeline trace of the persistent kernel (tracing).  After pat_plan_set_trace(plan, k0, nk)
 * (0 < nk <= 4096; nk = 0 turns it off), every solve records, for each CTA b and each grid barrier
 * k in [k0, k0 + nk) (counted from 0 in launch order), 8 device globaltimer stamps [ns]: [0] when
 * the CTA entered the barrier, [1] when it left it, [2..7] sub-phase marks of the phase that ends
 * at that barrier (row phase: spectra staged, packed, inverse x-FFT done, physics done, forward
 * x-FFT done, spectra written; column phase: tile loaded, forward FFT done, multiplied, inverse
 * FFT done; 0 = not reached).  pat_plan_read_trace copies them, synchronising the device, as
 * [grid][nk][8] unsigned 64-bit values into `out` (capacity `count` values) and sets *grid.
 * Plans on the per-phase graph path record nothing (*grid = 0). */
pat_status pat_plan_set_trace(pat_plan* plan, int k0, int nk);
pat_status pat_plan_read_trace(pat_plan* plan, unsigned long long* out, size_t count, int* grid);

/* pat_plan_set_fault -- failure-detection hook of the persistent path (no paper counterpart).
 * Every grid barrier of the plan's persistent kernels waits at most `wait_limit_s` seconds
 * (default 2; 0 < wait_limit_s <= 10) before the kernel records PAT_ETIMEOUT in the plan's status
 * word and every CTA returns (pat_plan_status reads it; the next launch clears it).  barrier_extra
 * = 1 makes every barrier wait for one arrival that never comes, so the limit runs out on the
 * first barrier: a host-side way to exercise the detection without faulting the GPU.  0 restores
 * normal operation.  No effect on the per-phase (graph) path, which has no device-side waits. */
pat_status pat_plan_set_fault(pat_plan* plan, int barrier_extra, double wait_limit_s);

/* pat_probe_fp32_peak -- measurement aid, not part of the method: *tflops = the FP32 FMA throughput
 * of the current device in TFLOP/s (best of three timed launches of eight independent FMA chains per
 * thread, 8 CTAs of 256 threads per SM), the denominator of the FP32 instruction roofline of the
 * spectral kernels.  Allocates and frees a few bytes on `stream`; synchronises it. */
pat_status pat_probe_fp32_peak(double* tflops, void* stream);

/* pat_last_error -- message describing the calling thread's last failed call ("" if none).
 * The pointer stays valid until the next pat_* call on the same thread. */
const char* pat_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PAT_H */
