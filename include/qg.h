/*
 * qg.h -- C-ABI of libqg: one time step of the forced-dissipative barotropic
 * quasi-geostrophic beta-plane vorticity equation with LES closures, Brinkman
 * volume penalisation and an inflow sponge, on one GB300 GPU (sm_103a).
 *
 * Model (Sec. II-A, Eq. 1):
 *     dw/dt + J(psi, w) = nu lap(w) - mu w - beta dpsi/dx + F_obs + F_sponge + Pi
 *     (u, v) = (-dpsi/dy, dpsi/dx),  w = lap(psi),
 * with a uniform inflow U added to the zeroth Fourier mode of u (Sec. II-D),
 * F_obs = -curl(chi_obs u / eta) (Eq. 2, u_obs = 0), F_sponge =
 * -rate chi_sponge (w - 0) (Eq. 3), and Pi = div(nu_e grad w) (Eq. 9) from one
 * of four closures: Smagorinsky (Eq. 10), Leith (Eq. 13) and their dynamic
 * Germano/Lilly variants (Eq. 11-12, 14).
 *
 * Discretisation (Sec. II-C): Fourier pseudo-spectral on an N x N doubly
 * periodic grid of [0, L)^2, products by collocation with the 2/3 rule
 * (square truncation |m_x|, |m_y| <= K = floor((N-1)/3)).  One step is the
 * Lie-Trotter split of Sec. II-E with these sub-step integrators:
 *   1. three SSP-RK3 (Shu-Osher) stages of L(w) = -J - beta v + C div(g grad w);
 *      a dynamic C is recomputed from every stage's field;
 *   2. the exact viscous/friction factor exp(-(nu |k|^2 + mu) dt);
 *   3. the exact Brinkman sub-step: total velocity times exp(-chi dt / eta),
 *      then w = T curl(u);
 *   4. the exact sponge sub-step: w times exp(-rate chi_s dt), then T;
 *   5. the mean mode set to zero.
 *
 * Conventions.  Physical arrays are row-major [y][x] (x fastest), x_i = i L/N.
 * Every call returns QG_OK (0) or a negative QG_ERR_* code and never throws;
 * qg_last_error() returns a thread-local message for the last failure.  Host
 * arrays passed in are copied before the call returns; device pointers
 * (on_device = 1) are borrowed for the duration of the call only.  The
 * library allocates and owns every device buffer it uses.  Work is enqueued
 * on the stream given at creation (NULL = the legacy default stream).
 */
#ifndef QG_H
#define QG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define QG_OK 0
#define QG_ERR_ARG (-1)       /* invalid argument: sizes, kinds, NULL pointers */
#define QG_ERR_CUDA (-2)      /* a CUDA runtime call failed (message has the CUDA error) */
#define QG_ERR_NONFINITE (-3) /* a non-finite value appeared in the state; stepping stopped */
#define QG_ERR_OOM (-4)       /* device allocation failed */
#define QG_ERR_TIMEOUT (-5)   /* a bounded device wait gave up (an async copy never arrived) */
#define QG_ERR_UNSUPPORTED (-6) /* valid request the library cannot serve on this device (e.g. shared memory) */
#define QG_ERR_BOUNDS (-7)    /* bounds-checked debug build (-DQG_CHECKED) only: a kernel met an index outside
                                 its array; the access was skipped and stepping stopped */

/* Working precision of the device fields. */
#define QG_FP64 0
#define QG_FP32 1

/* Closure kinds (Sec. III-A). */
#define QG_NONE 0
#define QG_SMAG 1   /* nu_e = (c_S Delta)^2 |S|,           Eq. 10 */
#define QG_LEITH 2  /* nu_e = (c_L Delta)^3 |grad w|,      Eq. 13 */
#define QG_DSMAG 3  /* (c_S Delta)^2 = <HM>/<MM>,          Eq. 11-12 */
#define QG_DLEITH 4 /* (c_L Delta)^3 = <HM>/<MM>,          Eq. 14 */

/* Grid: N even, N = 2^a 3^b, 16 <= N <= 4096; L > 0; precision QG_FP32/QG_FP64. */
typedef struct {
  int32_t n;
  int32_t precision;
  double L;
} qg_grid;

/* Closure: kind, the static constant c (c_S or c_L; ignored by dynamic
 * kinds) and the test-filter width ratio r = Delta~/Delta (2 in the paper,
 * Sec. III-A).  The test filter is sharp and radial: |m| <= N / (2 r). */
typedef struct {
  int32_t kind;
  int32_t reserved;
  double c;
  double test_ratio;
} qg_closure;

/* Time schemes.  QG_SCHEME_RK3_EXACT (default): SSP-RK3 for J, beta and the
 * SGS term, then exact viscous, Brinkman and sponge sub-steps.
 * QG_SCHEME_AB2CN: the paper's own scheme (Sec. II-E, Eq. 4): Crank-Nicolson on
 * nu lap - mu - beta d/dx, AB2 on the Jacobian, the SGS term and the Brinkman
 * forcing, then the sponge split advanced by AB2 with the w*, w** history;
 * the first step after qg_set_state is an Euler start.  AB2CN treats the
 * penalisation explicitly, so it needs eta > dt (Sec. II-E). */
#define QG_SCHEME_RK3_EXACT 0
#define QG_SCHEME_AB2CN 1

/* Time-step parameters: dt, viscosity nu = 1/Re, bottom friction mu,
 * porosity eta of the Brinkman term (Eq. 2), sponge rate = 1/eta_sponge
 * (Eq. 3) and the time scheme. */
typedef struct {
  double dt, nu, mu, eta, sponge_rate;
  int32_t scheme;
  int32_t reserved;
} qg_params;

/* Diagnostics of the current state.  energy = <|u'|^2>/2 of the perturbation
 * velocity, enstrophy = <w^2>/2 (both FP64 Parseval sums), coeff = the
 * closure coefficient C used in the last RK stage ((c Delta)^p), max_abs_omega
 * and finite from the physical field. */
typedef struct {
  double t, energy, enstrophy, coeff, max_abs_omega;
  int64_t step;
  int32_t finite;
  int32_t reserved;
} qg_diag;

typedef struct qg_handle qg_handle;

/* Create a solver on the current CUDA device.
 *   grid, closure, params: as above (copied).
 *   beta: the beta-plane parameter of Eq. 1;  U: uniform inflow along +x.
 *   mask:   chi_obs, N*N host doubles in [0, 1], or NULL for no obstacle.
 *   sponge: chi_sponge, N*N host doubles in [0, 1], or NULL for no sponge.
 *   cuda_stream: a cudaStream_t (as void*) all work is enqueued on.
 *   out: receives the handle.
 * The state starts at w = 0.  Errors: QG_ERR_ARG (bad sizes/kinds),
 * QG_ERR_UNSUPPORTED (the grid does not fit the kernels' shared memory),
 * QG_ERR_OOM, QG_ERR_CUDA. */
int qg_create(const qg_grid* grid, double beta, double U, const double* mask, const double* sponge,
              const qg_closure* closure, const qg_params* params, void* cuda_stream, qg_handle** out);

/* Set the state from a physical vorticity field of N*N values (dtype QG_FP64
 * = double, QG_FP32 = float; host if on_device = 0, device otherwise: read on
 * the handle's stream, see qg_stream).  The field is projected: w_hat =
 * T F[w] with the mean mode removed (Sec. II-C, II-D).  Resets the non-finite
 * flag; keeps t and step. */
int qg_set_state(qg_handle* h, const void* omega, int32_t on_device, int32_t dtype);

/* Write the physical vorticity of the current state (N*N, dtype as above).
 * Synchronises the handle's stream when omega is a host buffer; a device
 * buffer is written on the handle's stream (see qg_stream). */
int qg_get_state(qg_handle* h, void* omega, int32_t on_device, int32_t dtype);

/* The cudaStream_t (as void*) the handle enqueues its work on: the stream
 * given at create, or the handle's own stream for an ensemble member (NULL is
 * the legacy default stream).  Device buffers passed to qg_set_state,
 * qg_get_state and qg_step_vjp are read and written in the order of this
 * stream: the caller makes it wait for the producer of an input and makes the
 * consumer of an output wait for it.  No paper counterpart (plumbing). */
int qg_stream(qg_handle* h, void** stream);

/* Enqueue nsteps >= 0 steps (asynchronous).  Returns QG_ERR_NONFINITE without
 * enqueueing if an earlier step is already known to have produced a
 * non-finite value (kernels also stop by themselves once the device flag is
 * set).  Use qg_sync to wait and collect the status. */
int qg_step(qg_handle* h, int32_t nsteps);

/* Wait for all enqueued work; QG_ERR_NONFINITE if the state became non-finite. */
int qg_sync(qg_handle* h);

/* Synchronise and fill out (see qg_diag).  Returns QG_ERR_NONFINITE (with
 * out filled, finite = 0) if the state is not finite. */
int qg_diagnostics(qg_handle* h, qg_diag* out);

/* Release every device buffer of the handle (NULL is ignored). */
void qg_destroy(qg_handle* h);

/* A priori SGS analysis (Sec. III, Eq. 5-8, 15) of one fully resolved field.
 *   omega_fr: N_fr*N_fr host doubles (projected onto the 2/3 band first).
 *   n_fr, n_les: grid sizes, n_les <= n_fr, both valid grid sizes.
 *   mask_fr, sponge_fr: chi_obs, chi_sponge on the fine grid (NULL = absent).
 *   closure: the closure whose Pi model is correlated with the exact Pi.
 *   params: eta and sponge_rate enter F_obs and F_sponge (dt, nu, mu unused).
 *   U, beta: inflow and beta (beta does not enter Pi, its term is linear).
 *   flags: bit 0 set = omit the Gaussian factor of the grid filter.
 *   pi_exact, pi_model: n_les*n_les host doubles (output).
 *   pi_parts: 3*n_les*n_les host doubles (Jacobian, obstacle, sponge parts of
 *             Eq. 8), or NULL.
 *   pcc: receives PCC(pi_exact, pi_model) (NaN if the model term is zero).
 * Grid filter: exp(-k^2 Delta_FF^2 / 6) times the cut-off |k| <= pi/Delta_FF,
 * Delta_FF = L / n_les, then a spectral copy to the n_les grid.  Runs in FP64
 * on the current device; synchronous. */
int qg_sgs_apriori(const double* omega_fr, int32_t n_fr, int32_t n_les, double L, const double* mask_fr,
                   const double* sponge_fr, const qg_closure* closure, const qg_params* params, double U,
                   double beta, int32_t flags, double* pi_exact, double* pi_model, double* pi_parts, double* pcc);

/* The grid filter of Eq. 5 alone, applied to a series of fully resolved
 * fields: the filtered field omega_FF that an LES state is compared with a
 * posteriori (Sec. IV).
 *   omega_fr: nsnap >= 1 fields of n_fr*n_fr host doubles, row-major [y][x],
 *             each projected onto its 2/3 band with zero mean first.
 *   n_fr, n_les: grid sizes as for qg_sgs_apriori (n_les/2 - 1 must not exceed
 *             the fine band (n_fr - 1)/3: QG_ERR_UNSUPPORTED otherwise).
 *   flags: bit 0 set = omit the Gaussian factor.
 *   omega_les: nsnap fields of n_les*n_les host doubles (output).
 * Filter exp(-k^2 Delta^2 / 6) times the cut-off |k| <= pi/Delta, Delta =
 * L/n_les, spectral copy to the coarse grid, coarse 2/3 band kept.  FP64 on
 * the current device; synchronous; allocates its scratch per call. */
int qg_grid_filter(const double* omega_fr, int32_t nsnap, int32_t n_fr, int32_t n_les, double L, int32_t flags,
                   double* omega_les);

/* A posteriori comparison of two snapshot series on one grid (Sec. IV,
 * Eq. 15 and 16).
 *   les: n_les_snap fields, ff: n_ff_snap fields (1 .. 10^6 each), npts >= 1
 *        values per field, snapshot-major and contiguous; dtype QG_FP32 or
 *        QG_FP64 for both; on_device = 1: device pointers (borrowed, read
 *        only, used on stream), 0: host pointers (copied to the device).
 *   lag_min <= lag_max: lags phi in snapshot intervals (at most 2^16 lags,
 *        n_ff_snap * nlag <= 2^24); the pair (t, phi) compares les[t - phi]
 *        with ff[t].
 *   stream: a cudaStream_t, or NULL for the legacy default stream.
 * Outputs, host doubles, row t = ff snapshot, column j = phi - lag_min:
 *   dist[n_ff_snap * nlag]: sum over the points of (les[t-phi] - ff[t])^2;
 *   pcc[n_ff_snap * nlag] or NULL: PCC(les[t-phi], ff[t]) of Eq. 15 with
 *        population moments, NaN where either field is constant;
 *   entries whose t - phi lies outside [0, n_les_snap) are NaN in both;
 *   mean_dist[nlag] or NULL: the mean of each column of dist over its
 *        defined entries (NaN if none);
 *   phase or NULL: the lag of Eq. 16, the phi of the smallest mean_dist
 *        (ties: the smallest |phi|, then the negative lag).
 *   kernel_ms[4] or NULL: device milliseconds of the call's four kernel
 *        groups (moments, pairs, finish, phase), from CUDA events recorded
 *        on stream around them (-1 where an event could not be made).
 * QG_ERR_ARG if no lag in the range pairs two snapshots.  FP32 series are
 * differenced and multiplied in FP32, summed in short FMA chains that join
 * compensated per-thread totals, chunk sums and all means in FP64; FP64
 * series run in FP64.  Deterministic; synchronous.  Scratch (and the device
 * copy of host series) comes stream-ordered from a memory pool the library
 * keeps per device; the pool holds freed blocks for later calls until the
 * process ends. */
int qg_series_compare(const void* les, int32_t n_les_snap, const void* ff, int32_t n_ff_snap, int64_t npts,
                      int32_t dtype, int32_t on_device, int32_t lag_min, int32_t lag_max, void* stream, double* dist,
                      double* pcc, double* mean_dist, int32_t* phase, double* kernel_ms);

/* Ensembles of independent members (Sec. IV runs many LES of different
 * grids, closures and parameters; the paper gives no batching, this is the
 * batched form of qg_step).  Each member is a full qg_handle on a stream of
 * its own; a step of the ensemble advances every member by one step of its
 * own scheme.  After one eager step it is replayed as one CUDA graph in which
 * the members' steps are branches between a fork and a join on the
 * ensemble's stream, so members' kernels run side by side on the GPU.  A
 * member's results are bitwise those of the same member stepped alone.
 *
 * Launch form, chosen by a tuner at creation: the members run in L chains
 * (lanes) side by side, dealt longest-first by estimated cost (L = count:
 * every member in a branch of its own), with or without programmatic
 * dependent launch, and with the FP32 Germano reduction in its lean or
 * register form.  None of these changes a member's arithmetic.  The tuner
 * times a few replays of each candidate's graph, stepping the members from
 * their initial zero states, then restores those states, the step counters
 * and the status flags; the choice is cached per signature (grids,
 * precisions, closures, schemes, forcings, device) for later ensembles in the
 * process.  The environment can fix the form instead: QG_ENSEMBLE_LANES=L,
 * QG_ENSEMBLE_PDL=0|1, QG_ENSEMBLE_LEAN=0 (lean where it makes one wave) |
 * 1 (lean wherever it fits) | 2 (never), or QG_ENSEMBLE_TUNE=0 (no timing:
 * all members side by side, no PDL, lean where it makes one wave). */
typedef struct qg_ensemble qg_ensemble;

typedef struct {
  qg_grid grid;
  qg_closure closure;
  qg_params params;
  double beta;
  double U;
  const double* mask;   /* chi_obs, n*n host doubles, or NULL */
  const double* sponge; /* chi_sponge, n*n host doubles, or NULL */
} qg_member;            /* 120 bytes */

/* Create count >= 1 members as qg_create would (host masks copied; on error
 * nothing is left allocated and the message names the member).  stream: the
 * ensemble's cudaStream_t (capturable, i.e. not the legacy default stream),
 * or NULL to let the ensemble create one. */
int qg_ensemble_create(const qg_member* members, int32_t count, void* stream, qg_ensemble** out);

/* Borrow member i's handle for qg_set_state, qg_get_state, qg_diagnostics,
 * qg_profile, qg_kernel_times (valid until qg_ensemble_destroy; do not
 * qg_destroy it).  Work queued on it is ordered before the next ensemble step
 * and after the previous one. */
int qg_ensemble_handle(qg_ensemble* e, int32_t i, qg_handle** out);

/* Enqueue nsteps >= 0 steps of every member (asynchronous).  A member whose
 * state became non-finite stops computing (its kernels return at once); the
 * others go on. */
int qg_ensemble_step(qg_ensemble* e, int32_t nsteps);

/* Wait for all members; QG_ERR_NONFINITE (or QG_ERR_TIMEOUT) from the first
 * member that reports it, whose index goes to *first_bad (-1 if none; may be
 * NULL). */
int qg_ensemble_sync(qg_ensemble* e, int32_t* first_bad);

/* The ensemble's launch form: form[0] = lanes (1..count), form[1] = PDL
 * (0/1), form[2] = lean-reduction setting (0, 1, 2 as QG_ENSEMBLE_LEAN),
 * form[3] = 0 (default or fixed by the environment), 1 (timed at creation),
 * 2 (taken from the cache); *ms_per_step (may be NULL) = the chosen form's
 * timed ms per ensemble step (0 when not timed). */
int qg_ensemble_config(qg_ensemble* e, int32_t* form, double* ms_per_step);

/* Destroy every member and the ensemble's own streams (NULL is ignored). */
void qg_ensemble_destroy(qg_ensemble* e);

/* Discrete adjoint of one step: the vector-Jacobian product of the map
 * w_n -> w_{n+1} of the RK3 scheme (R1-R5: SSP-RK3, exact viscous factor,
 * exact Brinkman and sponge sub-steps, projection), for every closure: none,
 * Smagorinsky and Leith with a fixed coefficient (Eq. 10, 13) and their
 * dynamic forms, whose coefficient C = max(0, <HM>/<MM>) (Eq. 12, 14) is
 * differentiated through the quotient (zero gradient where it is clipped).
 * Inner products are sums over the grid points.
 *   omega_n:  N*N physical state at the start of the step (projected onto the
 *             2/3 band with zero mean first, as qg_set_state does).
 *   lam_next: N*N gradient of a loss with respect to the physical w_{n+1}
 *             (the field qg_get_state would return after the step).
 *   lam_n:    N*N gradient with respect to the physical input field (output;
 *             2/3 band, zero mean).
 *   on_device, dtype: as for qg_set_state, for all three buffers.
 *   grads[3] or NULL: d loss / dC summed over the three stages (C held
 *             fixed), d loss / dc for C = (c Delta)^p (0 for the dynamic
 *             closures), d loss / d sponge_rate.
 * The forward stages are recomputed from omega_n; the handle's own state and
 * stepping are untouched.  Synchronous on the handle's stream; the first call
 * allocates a workspace of 25 spectral, 37 physical and 6 mixed arrays (39,
 * 56 and 6 for the dynamic closures); later calls replay one captured CUDA
 * graph.
 * QG_ERR_UNSUPPORTED for the AB2CN scheme. */
int qg_step_vjp(qg_handle* h, const void* omega_n, const void* lam_next, void* lam_n, int32_t on_device,
                int32_t dtype, double* grads);

/* Kernel classes reported by qg_kernel_times. */
#define QG_K_ROW_STAGE 0   /* row pass of an RK stage (products of Eq. 1, 9-14) */
#define QG_K_COL_REDUCE 1  /* column pass: Germano partial sums (Eq. 12, 14) */
#define QG_K_COL_STAGE 2   /* column pass: RK combine + next stage's fields */
#define QG_K_ROW_BRINK 3   /* row pass of the Brinkman sub-step (Eq. 2) */
#define QG_K_COL_CURL 4    /* column pass: Brinkman curl */
#define QG_K_ROW_SPONGE 5  /* row pass of the sponge sub-step (Eq. 3) */
#define QG_K_COL_FINAL 6   /* column pass: projection of w^{n+1}, stage-1 fields */
#define QG_K_OTHER 7       /* state I/O and diagnostics */
#define QG_K_ADJ_ROW 8     /* qg_step_vjp: row passes (one field each, into or out of physical space) */
#define QG_K_ADJ_COL 9     /* qg_step_vjp: column passes (forward transforms, derived fields) */
#define QG_K_ADJ_PW 10     /* qg_step_vjp: pointwise products, spectral multipliers, inner products */
#define QG_NUM_KCLASS 11

/* Tracing.  enable = 1 clears the counters and starts recording a CUDA event
 * pair around every kernel launch on the handle's stream; 0 stops recording.
 * Launch counts are kept whether or not recording is on. */
int qg_profile(qg_handle* h, int32_t enable);

/* Per kernel class (index QG_K_*): counts[i] = launches since the last
 * qg_profile(h, 1) (or creation), ms[i] = summed device time of the recorded
 * launches.  Synchronises the handle's stream.  nclass <= QG_NUM_KCLASS. */
int qg_kernel_times(qg_handle* h, int32_t* counts, double* ms, int32_t nclass);

/* Energy, enstrophy, max |w| and finiteness of a physical vorticity field,
 * computed without allocating any device memory.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc where they need
 * these numbers, such as hosts whose framework owns all device memory through
 * its own allocator or a fixed budget, code that must not introduce the
 * device-wide synchronisation an allocation can cause, and real-time loops
 * that must not pay for or risk an allocation.
 *   omega: N*N device array of dtype (QG_FP32 = float, QG_FP64 = double),
 *          row-major [y][x]; read only.  The field is projected as by
 *          qg_set_state (2/3 band, zero mean) and the statistics are those
 *          qg_diagnostics reports for that state, computed in dtype with FP64
 *          sums.
 *   n: grid size, even, 2^a 3^b, 16 <= n <= 512;  L: box length (> 0).
 *   cuda_stream: cudaStream_t (as void*) the work is enqueued on; the call is
 *          asynchronous.
 *   stats: 4 device doubles (output): energy, enstrophy, max |w|, finite
 *          (1.0 or 0.0).
 * Scratch lives in one static device array of 5 MiB that every GPU loading
 * the library holds until the process exits.  All calls share it and it keeps
 * the last call's contents: calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and must be serialised by the
 * caller.  The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  CUDA loads a library's device code lazily by
 * default, so that first call on a device may also load this module, which
 * reserves the static array and other module memory and can synchronise the
 * device: a caller that needs the no-allocation guarantee from its very first
 * use makes one warm-up call per device at set-up time; every later call
 * allocates nothing.  Errors: QG_ERR_ARG for n > 512 or other bad arguments
 * (nothing is enqueued), QG_ERR_CUDA. */
int qg_field_stats_static(const void* omega, int32_t n, double L, int32_t dtype, void* cuda_stream, double* stats);

/* Measured fused multiply-add throughput of the current device in dtype
 * (QG_FP32 or QG_FP64): a kernel of independent FMA chains, 8 CTAs of 256
 * threads per SM, calibrated to about 50 ms and timed by CUDA events (best of
 * three launches).  The paper has no counterpart: it gives the arithmetic
 * peak that the FP64 form of the step (bound by FP64 arithmetic, not HBM, on
 * this GPU) is reported against.  Synchronous; allocates one scalar.
 *   flops_per_s: output, 2 flops per FMA;  ms: output (may be NULL), the
 *   duration of the best launch.
 * Changes no clock or device setting.  Errors: QG_ERR_ARG, QG_ERR_OOM,
 * QG_ERR_CUDA. */
int qg_probe_fma_rate(int32_t dtype, double* flops_per_s, double* ms);

/* Thread-local description of the last error (never NULL). */
const char* qg_last_error(void);

/* Library version string. */
const char* qg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QG_H */
