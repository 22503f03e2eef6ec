/*
 * rbc.h - C ABI of the GB300 Parareal fine propagator for 2D Rayleigh-Benard
 * convection (Clarke, Davies, Ruprecht, Tobias, Oishi: "Performance of
 * parallel-in-time integration for Rayleigh Benard Convection").
 *
 * Problem (Sec. 2.1, Eqs. 3-7): Oberbeck-Boussinesq equations, Prandtl number
 * Pr, Rayleigh number Ra, periodic x in [0, Lx), z in [-1/2, 1/2], no-slip walls
 * with T(-1/2) = 1, T(1/2) = 0 (or, by option, the fixed flux dT/dz = -1 of
 * Eq. 7); time in thermal-diffusion units.  The consistency diagnostics of
 * Sec. 2.2 come from rbc_diagnostics.
 * Discretisation (Sec. 3.2): Fourier modes in x, Chebyshev polynomials in z,
 * products in grid space (3/2-rule padded), linear terms implicit (ultraspherical
 * tau), nonlinear terms explicit, IMEX RK443 (Sec. 3.6).  Parareal (Sec. 3.1,
 * Eq. 20) with the defect and Nusselt stopping norms (Sec. 3.7, Eq. 9).
 *
 * Conventions
 *  - Every call returns rbc_status; nothing throws across the ABI.
 *  - Device buffers are owned by the caller (any allocator); the library reads
 *    and writes them on the stream passed in.  Handles own their operator
 *    tables and their workspace (device memory allocated at create/reserve).
 *  - Host arrays are owned by the caller and are copied before return.
 *  - A handle is not re-entrant: one stream at a time per handle.
 *  - Invalid arguments return RBC_EINVAL and change nothing.
 *
 * Spectral state layout (one time slice, "state"), 16*Nx*Nz bytes, FP64:
 *    double X[2][Nz][Nx/2][2]
 *    X[f][n][m][c]: field f (0 = temperature T, 1 = streamfunction psi),
 *    Chebyshev index n (T_n(2z)), Fourier index m (k = 2 pi m / Lx; the Nyquist
 *    mode is not stored), c = 0 real / 1 imaginary part.  The field value is
 *    f(x, z) = sum_{|m| < Nx/2} sum_n fhat_m,n T_n(2z) exp(i k x) (real field,
 *    fhat_{-m} = conj(fhat_m)).  The m = 0 slot of psi holds instead the
 *    Chebyshev coefficients of the mean horizontal velocity U(z) (real).
 *    u = d psi / dz (+ U), w = -d psi / dx.
 * Native grid (set/get_state): x_i = Lx i / Nx, z_j = -cos(pi j/(Nz-1))/2,
 *    arrays double g[Nz][Nx] (z-major, z ascending).
 */
#ifndef RBC_H
#define RBC_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbc_s* rbc_t;
typedef struct pr_s* parareal_t;

typedef enum {
  RBC_OK = 0,
  RBC_EINVAL = -1,      /* bad argument (sizes, null pointers, dt <= 0, ...)  */
  RBC_ENOMEM = -2,      /* device or host allocation failed                    */
  RBC_ECUDA = -3,       /* a CUDA runtime call failed (see rbc_last_error)     */
  RBC_EDIVERGED = -4,   /* a NaN/Inf appeared in a state (Sec. 3.6 warns that
                           Parareal can be unstable with stable F and G)       */
  RBC_ETIMEOUT = -5,    /* a bounded device-side wait gave up (the mbarrier
                           waits of the mixed-precision tensor-core kernels);
                           the states concerned are left as they were at the
                           start of the failing step                          */
  RBC_ENOTCONVERGED = 1 /* Parareal reached max_iters without meeting tol      */
} rbc_status;

enum { RBC_FP64 = 0, RBC_MIXED = 1, RBC_MIXED_BF16 = 2 };   /* rbc_opts.precision */
enum { RBC_FIXED_T = 0, RBC_FIXED_FLUX = 1 }; /* rbc_opts.bc (Eqs. 6, 7) */
enum { RBC_CRIT_FIXED = 0, RBC_CRIT_DEFECT = 1, RBC_CRIT_NU = 2, RBC_CRIT_STAT = 3 };
enum { RBC_RK443 = 0, RBC_RK222 = 1, RBC_RK111 = 2 };   /* rbc_opts.scheme (Sec. 3.6) */

typedef struct {
  int precision;   /* RBC_FP64: every step in FP64.  RBC_MIXED: transforms and
                      products in FP32, solves, RK combination, Parareal update
                      and norms in FP64; from Nz = 64 the z transforms run on
                      the tensor cores with TF32 operands split in hi and lo
                      parts (three products: about FP32 accuracy).
                      RBC_MIXED_BF16: the same with BF16 hi/lo operands (three
                      products of about 16-bit operands; the transforms' error
                      enters the state through dt times the explicit terms and
                      stays within the FP32 products' 1e-5 bound).           */
  int bc;          /* RBC_FIXED_T: T = 1, 0 at the bottom and top walls (Eq. 6).
                      RBC_FIXED_FLUX: dT/dz = -1 at both walls (Eq. 7); Ra is
                      then the flux Rayleigh number Ra_f of Eq. 8.  No-slip
                      walls in both.  With fixed flux, Nu_b = Nu_t = 1 and the
                      Nusselt number is 1 / (T_bottom - T_top) (the plane
                      means at the walls, rbc_diagnostics' profile ends).      */
  int eager;       /* 0: rbc_step_batch runs its steps as one graph launch (a
                      device-side loop); 1: every kernel is launched from the
                      host, so per-kernel profilers see each launch (slower).
                      Same results either way.                               */
  int scheme;      /* IMEX Runge-Kutta pair of Ascher, Ruuth & Spiteri (1997):
                      RBC_RK443 (4 stages, 3rd order; the paper's, Sec. 3.2),
                      or the lower-order coarse steppers Sec. 3.6 reports
                      trying: RBC_RK222 = ARS(2,2,2) (2 stages, 2nd order,
                      implicit diagonal 1 - 1/sqrt(2)) and RBC_RK111 =
                      ARS(1,1,1) (forward-backward Euler).  All three have an
                      explicit first stage and are stiffly accurate; a step
                      launches 4 kernels per stage.  Zero-initialise the
                      struct: 0 is RK443.                                    */
} rbc_opts;

/* Text of the last error seen by this thread (static storage, never NULL). */
const char* rbc_last_error(void);

/* rbc_create: build a propagator for (Ra, Pr, Lx, Nx, Nz, dt) (Sec. 2.1 Eqs.
 * 3-6 parameters, Sec. 3.2 resolution (Nx, Nz), Sec. 3.4 time step).  Builds
 * the operator tables on the host in FP64 and uploads them to the current
 * device.  Requirements: Nx a power of two, 4 <= Nx <= 1024, Nz even, 8 <= Nz <= 512,
 * dt > 0, Pr > 0, Lx > 0, Ra >= 0; opts may be NULL (FP64).               */
rbc_status rbc_create(double Ra, double Pr, double Lx, int Nx, int Nz, double dt,
                      const rbc_opts* opts, rbc_t* out);
void rbc_destroy(rbc_t h);

/* Bytes of one spectral state (16*Nx*Nz) and of the workspace per batched
 * state, for admission control by device memory.                          */
size_t rbc_state_bytes(rbc_t h);
size_t rbc_workspace_bytes_per_state(rbc_t h);

/* Grow the workspace to hold at least B states (rbc_step_batch grows it on
 * demand; call this first to keep allocation out of timed regions).        */
rbc_status rbc_reserve(rbc_t h, int B);

/* Native grid <-> spectral state.  h_T, h_u, h_w: host double[Nz][Nx]
 * (h_u, h_w may be NULL = zero).  psi is recovered from w (psi_m = i w_m / k,
 * m >= 1), U from the x-mean of u; the Nyquist column is dropped.  d_state is
 * a device state buffer.  Synchronous.                                     */
rbc_status rbc_set_state(rbc_t h, void* d_state, const double* h_T, const double* h_u,
                         const double* h_w);
rbc_status rbc_get_state(rbc_t h, const void* d_state, double* h_T, double* h_u, double* h_w);

/* rbc_step_batch: the fine (or coarse) propagator F of Eq. 20 applied to B
 * independent states at once (Sec. 3.1: the fine solves of all time slices
 * run in parallel).  d_states: B contiguous device states, advanced in place
 * by h_nsteps[b] RK443 steps each (host int[B], each >= 0; 0 leaves a state
 * untouched; uneven counts are allowed).  d_nu_integral (device double[B],
 * may be NULL) is overwritten with the trapezoid-rule integral over the run
 * of Nu_V(t) (Eq. 9) for each state.  Asynchronous on `stream` (the step
 * counts are copied before return); a NaN/Inf in a state is recorded in a
 * device flag and reported by rbc_check_diverged.                          */
rbc_status rbc_step_batch(rbc_t h, void* d_states, int B, const int* h_nsteps,
                          double* d_nu_integral, cudaStream_t stream);

/* rbc_step_batch_ra: rbc_step_batch with a Rayleigh number per state,
 * h_ra[b] (host double[B], each >= 0).  The implicit operators and their
 * factors do not depend on Ra (it enters the stage systems only through the
 * buoyancy coupling, Eq. 3), so one handle serves states of any Ra; the
 * handle's own Ra is ignored by this call.                                 */
rbc_status rbc_step_batch_ra(rbc_t h, void* d_states, int B, const int* h_nsteps, const double* h_ra,
                             double* d_nu_integral, cudaStream_t stream);

/* Synchronises `stream` and reports the device-side errors of the handle:
 * those of the states of the last rbc_step_batch call and those of every
 * call since the previous rbc_check_diverged (whose record it clears).
 * RBC_ETIMEOUT if a bounded device-side wait gave up (a state whose transform
 * timed out is left as it was at the start of the failing step and its Nu
 * integral is unspecified), else RBC_EDIVERGED if a state went non-finite,
 * else RBC_OK.                                                              */
rbc_status rbc_check_diverged(rbc_t h, cudaStream_t stream);

/* Test hook, outside the paper's method: the number of polls after which
 * every bounded mbarrier wait of the tensor-core kernels (RBC_MIXED) gives
 * up, on the current device and for every handle (a device variable, read
 * by each kernel launch, graph replays included).  0 makes each such wait
 * give up at once, so that a test can exercise the RBC_ETIMEOUT path without
 * a fault; a negative value restores the default (2^24 polls).  The waits
 * that drain work already issued before tensor memory is released always
 * keep the default limit.                                                  */
rbc_status rbc_set_wait_limit(long long polls);

/* rbc_nusselt: Nu_V (Eq. 9), Nu_b and Nu_t (Eqs. 10, 11) of one device state,
 * written to host out[3].  Synchronous on `stream`.  RBC_ETIMEOUT (out
 * unspecified) if a tensor-core transform gave up waiting; the record read by
 * rbc_check_diverged is not touched.                                        */
rbc_status rbc_nusselt(rbc_t h, const void* d_state, double out[3], cudaStream_t stream);

/* rbc_nusselt_static: the same three Nusselt numbers as rbc_nusselt, from a
 * call that allocates no device memory.  The paper has no counterpart: this
 * exists for callers that cannot allocate when they ask for a diagnostic, for
 * example an application whose pool allocator already owns the free device
 * memory (a raw cudaMalloc from the library would then fail), or a timed loop
 * that cannot afford the device synchronisation cudaMalloc/cudaFree may cause.
 * rbc_nusselt may grow the handle's workspace on first use; this call never
 * does: its scratch (about 132 * Nx * Nz bytes) lives in one file-scope
 * device array of 3 MiB that every GPU loading the library keeps until the
 * process exits.  Grids needing more scratch than that (Nx * Nz above about
 * 23000, e.g. 256 x 128) return RBC_EINVAL and do nothing.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All
 * calls share the array: calls whose work overlaps on the GPU (different
 * streams, or different host threads) race and must be serialised by the
 * caller.  Every element a call reads is written by that call first, so no
 * clearing is needed and the leftover contents of an earlier call do not
 * matter, except the call's error word, which it clears first.  Synchronous
 * on `stream`; out[3] = (Nu_V, Nu_b, Nu_t) on the host; RBC_ETIMEOUT (out
 * unspecified) if a tensor-core transform of a mixed-precision handle gave
 * up waiting.                                                               */
rbc_status rbc_nusselt_static(rbc_t h, const void* d_state, double out[3], cudaStream_t stream);

/* ||T||_{L2(Omega)} of one device state (exact in x and z), host out.       */
rbc_status rbc_l2_temperature(rbc_t h, const void* d_state, double* out, cudaStream_t stream);

/* rbc_diagnostics: the instantaneous averages behind the consistency checks
 * of Sec. 2.2, for B contiguous device states (read only), into the
 * caller-owned device array d_out[B][rbc_diag_size(h)] (FP64, row per state),
 * asynchronously on `stream`.  Per state:
 *   [0] <u^2 + w^2>_V      (the characteristic speed U is the time mean of its
 *                           square root; Re = U / Pr)
 *   [1] <u . lap u>_V       (viscous term of the energy balance, Eq. 14)
 *   [2] <w T>_V             (buoyancy production P = Ra <w T>_V, Eq. 14)
 *   [3] Nu_V  [4] Nu_b  [5] Nu_t   (Eqs. 9-11)
 *   [6, 6 + Mz)           <T>_x at the padded points z_j = cos(pi j/(Mz-1))/2
 *   [6 + Mz, 6 + 2 Mz)    <(T - <T>_x)^2>_x at the same points (the integrand
 *                         of T_rms, Eq. 16)
 * with Mz = 3 Nz / 2 and j ascending (z descending from the top wall).  The
 * x-means are exact (Parseval over the kept Fourier modes); z-integrals use
 * the Clenshaw-Curtis rule on the Mz padded Lobatto points (Lz = 1).  The
 * transforms run in FP64 whatever the handle's precision.  Uses the handle's
 * workspace and grows it to B states when it is smaller (as rbc_step_batch
 * does); RBC_EINVAL for a null handle or pointer or B < 0; B = 0 does nothing.
 * rbc_diag_size returns 6 + 2 Mz (0 for a null handle).                     */
size_t     rbc_diag_size(rbc_t h);
rbc_status rbc_diagnostics(rbc_t h, const void* d_states, int B, double* d_out, cudaStream_t stream);

/* Time statistics of Sec. 2.2 along a run.
 * rbc_step_batch_sampled: rbc_step_batch of B states by nsteps steps each,
 * with the averages of rbc_diagnostics taken at steps 0, every, 2 every, ...
 * and nsteps, and their trapezoid-rule time integrals written to the
 * caller-owned device array d_stat[B][rbc_diag_size(h)] (FP64) in the order
 *   [0] <u^2 + w^2>_V^(1/2)   [1] <u . lap u>_V   [2] <w T>_V
 *   [3] Nu_V  [4] Nu_b  [5] Nu_t
 *   [6, 6 + Mz)          <T>_x at the padded points (as rbc_diagnostics)
 *   [6 + Mz, 6 + 2 Mz)   <T^2>_x = <(T - <T>_x)^2>_x + <T>_x^2
 * (divided by the sampled duration they give the time means; reading: the
 * paper gives no sampling rule).  d_nu_integral (device double[B], may be
 * NULL) receives the Nu_V integral as rbc_step_batch would (summed over the
 * sampling intervals, so its last bits can differ from one unsampled call).
 * Asynchronous on `stream`; grows the handle's buffers on demand.  RBC_EINVAL
 * for every < 1, nsteps < 0 or a null pointer.                              */
rbc_status rbc_step_batch_sampled(rbc_t h, void* d_states, int B, int nsteps, int every,
                                  double* d_nu_integral, double* d_stat, cudaStream_t stream);

/* rbc_stat_summary: the quantities of Sec. 2.2 from time means (d_stat rows
 * divided by the duration, summed over slices first when there are several)
 * of a grid with Nz Chebyshev points, Rayleigh number Ra and Prandtl number
 * Pr, into host out[12 + 3 Nz / 2]:
 *   [0] U (characteristic speed)  [1] Re = U / Pr  [2] Nu_V  [3] Nu_b  [4] Nu_t
 *   [5] Nu_int = max pairwise |difference| / Nu_V (Eq. 13)
 *   [6] P = Ra <w T> (Eq. 14)  [7] eps_U = |<u . lap u>|  [8] |P - eps_U| / P (Eq. 15)
 *   [9] delta_t = 1 / (2 Nu_V) (Eq. 17)
 *   [10] delta_T: height above the bottom wall of the largest T_rms over the
 *        padded points of the lower half (the first from the wall on a tie)
 *   [11] N_BL: interior native Lobatto points within delta_T of the wall
 *   [12, 12 + Mz) T_rms (Eq. 16, read as the RMS about the time-mean plane
 *        average) at the padded points.
 * Host arithmetic only (no device, no handle).                              */
rbc_status rbc_stat_summary(int Nz, double Ra, double Pr, const double* means, double* out);

/* Building blocks of Eq. 20 for callers that drive Parareal themselves (the
 * serving engine interleaves many runs).  All act on B contiguous states on
 * `stream`, asynchronously; the coarse grid must be no finer than the fine.
 *  rbc_restrict:  coarse[b] = fine[b] truncated to the coarse modes (Sec. 3.6).
 *  rbc_prolong:   fine[b] = coarse[b] zero-padded to the fine modes.
 *  rbc_parareal_correct: U[b] = F[b] + (prolong(Gnew[b]) - prolong(Gold[b])),
 *                 elementwise in that order (fine F, U; coarse Gnew, Gold).
 *  rbc_l2_diff:   d_out[b] = ||A[b] - B[b]||^2 of the temperature field (L2 over
 *                 the domain, exact), or ||A[b]||^2 when d_B is NULL; device
 *                 double[B].                                                */
rbc_status rbc_restrict(rbc_t fine, rbc_t coarse, const void* d_fine, void* d_coarse, int B, cudaStream_t stream);
rbc_status rbc_prolong(rbc_t fine, rbc_t coarse, const void* d_coarse, void* d_fine, int B, cudaStream_t stream);
rbc_status rbc_parareal_correct(rbc_t fine, rbc_t coarse, const void* d_F, const void* d_Gnew, const void* d_Gold,
                                void* d_U, int B, cudaStream_t stream);
rbc_status rbc_l2_diff(rbc_t h, const void* d_A, const void* d_B, int B, double* d_out, cudaStream_t stream);

/* Parareal (Sec. 3.1, Eq. 20).  fine and coarse share Ra, Pr, Lx; the coarse
 * grid is no finer than the fine one.  [t0, t1] is cut into nslices equal
 * slices; each slice must be a whole number of fine and of coarse steps
 * (relative 1e-9), else RBC_EINVAL.  G = prolong o coarse o restrict, with
 * restriction = truncation of the coefficient arrays and prolongation =
 * zero padding.  criterion: RBC_CRIT_FIXED (max_iters iterations, the
 * paper's practice, Sec. 3.7), RBC_CRIT_DEFECT (stop when
 * max_n ||U_n^k - U_n^{k-1}|| / ||U_n^k|| <= tol, L2 norm of T), RBC_CRIT_NU
 * (stop when |Nu_k - Nu_{k-1}| / |Nu_k| <= tol, Nu_k = time average of Nu_V
 * over the second half of the slices along the fine trajectories from U^k),
 * RBC_CRIT_STAT (the statistical rule the paper leaves open, Sec. 3.7 and
 * Sec. 5.2, read as: stop at the first k >= 2 whose time means of Nu_V, Nu_b,
 * Nu_t, Re, P and eps_U over the averaging window all changed by at most tol
 * relative to iteration k - 1; the fine sweeps are then sampled, see
 * parareal_set_sampling).
 * The handles must outlive the Parareal handle.                            */
rbc_status parareal_create(rbc_t fine, rbc_t coarse, double t0, double t1, int nslices,
                           int criterion, double tol, parareal_t* out);
void parareal_destroy(parareal_t p);

/* Run up to max_iters Parareal iterations from the device state d_U0.
 * d_U: caller-owned device buffer of nslices+1 states; on return d_U[n] =
 * U_n^k (d_U[0] = U0).  Host outputs: *k_done iterations performed,
 * defects[k-1] = Defect_k, nus[k-1] = Nu_{k-1} (arrays of max_iters doubles,
 * either may be NULL).  Returns RBC_OK when the criterion was met (always for
 * RBC_CRIT_FIXED), RBC_ENOTCONVERGED when max_iters ran out, RBC_EDIVERGED on
 * a non-finite state, RBC_ETIMEOUT if a bounded device-side wait of a
 * tensor-core kernel gave up.  Iterations stop after k = nslices, where U^k is the
 * serial fine solution.  Synchronous on `stream` (a few small D2H per iteration).
 *
 * Schedule (the results do not depend on it, bit for bit).  Iteration k's
 * fine sweep F(U_n^{k-1}) runs in groups of slices; its correction sweep
 * U_{n+1}^k = F(U_n^{k-1}) + (G(U_n^k) - G(U_n^{k-1})) runs on its own coarse
 * handle and stream, each step fused with the step's norms (one kernel forms
 * U_{n+1}^k, the coarse input of the next step, the next iteration's fine
 * input and ||U_{n+1}^k - U_{n+1}^{k-1}||, ||U_{n+1}^k||).  Every step waits
 * only for the data it reads: the previous iteration's step n and the fine
 * group of slice n.  So the sweeps of one iteration overlap, and so do
 * successive iterations: the host evaluates iteration k (defect, Nu,
 * criterion) while iterations k+1 .. k+depth are already running; when the
 * criterion is met their step loops are stopped early and their results
 * dropped.  The library runs all of this on copies of the caller's handles
 * (sharing their tables); kernel timing (rbc_profile) of the caller's handles
 * covers the copies.  parareal_set_schedule and parareal_set_depth tune it.  */
rbc_status parareal_iterate(parareal_t p, const void* d_U0, void* d_U, int max_iters,
                            int* k_done, double* defects, double* nus, cudaStream_t stream);

/* Schedule of parareal_iterate (timing only; results are the same bit for bit):
 *  group:        largest fine group (default ceil(nslices / 4)); group >=
 *                nslices runs each fine sweep as one batch after the coarse
 *                sweep U^0 has finished;
 *  first_group:  size of the first fine group (1 <= first_group <= group);
 *                sizes then double up to group (default ceil(group / 4));
 *  fine_streams: 1 to 4 streams (and fine handles) per iteration that the
 *                groups alternate over (default 2);
 *  coarse_priority: 1 runs the sweeps on the coarse grid on high-priority
 *                streams (default 1);
 *  coarse_sms:   0 (default) shares all SMs; n > 0 keeps the fine groups
 *                off about n SMs (they run in a green context of the other
 *                SMs; n is rounded up to the device's partition granularity),
 *                while the sweeps on the coarse grid may use every SM, so
 *                that their latency-bound kernels always find free SMs.  The
 *                library's copies of the fine handle capture their step
 *                graphs in that partition.  RBC_ECUDA if the driver cannot
 *                partition the device (the schedule is then unchanged).
 * RBC_EINVAL outside these ranges.                                          */
rbc_status parareal_set_schedule(parareal_t p, int group, int first_group, int fine_streams, int coarse_priority,
                                 int coarse_sms);

/* Iterations parareal_iterate keeps enqueued beyond the one it evaluates
 * next (0 to 6, default 1).  0 runs one iteration after another; with depth
 * d, iteration k + 1 .. k + d run while the host waits for iteration k, and
 * run for nothing (stopped early) when iteration k meets the criterion.
 * Each extra level holds nslices + 1 and nslices fine states more.  Timing
 * only; RBC_EINVAL outside [0, 6].                                          */
rbc_status parareal_set_depth(parareal_t p, int depth);

/* Sampling of the Sec. 2.2 time statistics along parareal_iterate's fine
 * sweeps (rbc_step_batch_sampled): every > 0 samples every `every` fine steps
 * and at each slice end, 0 turns sampling off (not allowed with
 * RBC_CRIT_STAT, whose default is one sample per slice end); the averaging
 * window is the slices [window_first, nslices) (default nslices / 2).
 * parareal_stat_means writes the window means of the last iteration that
 * parareal_iterate evaluated (iteration k: the fine trajectories from
 * U^{k-1}), 6 + 2 Mz doubles in rbc_step_batch_sampled's order, to host
 * out; RBC_EINVAL before any sampled iteration.                             */
rbc_status parareal_set_sampling(parareal_t p, int every, int window_first);
rbc_status parareal_stat_means(parareal_t p, double* out);

/* SMs kept free of fine groups (0: none), -1 for a NULL handle.           */
int parareal_coarse_sms(parareal_t p);

/* Autotuner (outside the paper's method).  rbc_autotune times, on the device,
 * RK443 steps of a batch of B states with candidate launch shapes that leave
 * every result unchanged bit for bit (modes per stage-solve block, modes and
 * n-chunks per z-forward block, the clustered or the one-block-per-row x-FFT
 * kernel and the latter's block size and shared-memory layout; reduction
 * orders depend on the grid only), by a coordinate search
 * from the built-in heuristics, and keeps the fastest for batches of B states
 * on this handle (and on the library's copies of it that Parareal uses).
 * out_ms (may be NULL): the time per step with the heuristics and with the
 * shapes kept.  Synchronous on `stream`; allocates B scratch states for the
 * duration of the call; RBC_EINVAL for B < 1.  rbc_tuned_shapes writes the
 * shapes kept for B (0 / -1: the heuristic) to host out[6] = (solve modes,
 * z-forward modes, z-forward chunks, clustered rows, row-kernel threads,
 * row-kernel layout: 1 lean, 0 full).  rbc_set_shapes keeps the host array
 * in[6] (same order and meaning) for batches of B states without timing
 * anything; RBC_EINVAL if a shape is not valid for the grid (a power of two
 * up to 16 solve modes or 32 z-forward modes, 1-8 chunks, 256/512/1024 row
 * threads, a layout that fits).  Any valid shapes give the same bits.      */
rbc_status rbc_autotune(rbc_t h, int B, double out_ms[2], cudaStream_t stream);
rbc_status rbc_tuned_shapes(rbc_t h, int B, int out[6]);
rbc_status rbc_set_shapes(rbc_t h, int B, const int in[6]);

/* ---- Instrumentation (outside the paper's method) ----
 * Kernel kinds of one RK443 stage: z-inverse transform, row kernel (x-FFTs and
 * products), z-forward transform, stage solve. */
enum { RBC_KERNEL_ZINV = 0, RBC_KERNEL_ROWS = 1, RBC_KERNEL_ZFWD = 2, RBC_KERNEL_SOLVE = 3, RBC_NKERNELS = 4 };

/* rbc_profile(h, 1) starts recording a CUDA event pair on the launching stream
 * around every stage kernel that h launches (such calls run without their
 * CUDA graph) and clears the totals; (h, 2) records only the first 8 steps of
 * the next rbc_step_batch call (a sample: the rest of that call runs on its
 * graph as usual); (h, 0) stops recording.  rbc_profile_read synchronises the device and returns, per
 * kernel kind, the summed event time (ms), the launch count, and the
 * algorithmic FP operations and DRAM bytes of those launches (each operand
 * read once, each result written once, all B slices active).  Any of the
 * output arrays may be NULL. */
rbc_status rbc_profile(rbc_t h, int enable);
rbc_status rbc_profile_read(rbc_t h, double ms[4], long long launches[4], double flops[4], double bytes[4]);

/* Number of CUDA kernels this library has launched in this process. */
unsigned long long rbc_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* RBC_H */
