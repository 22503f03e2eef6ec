// Internal types shared by the host runtime (rbc_host.cpp) and the CUDA
// kernels (rbc_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <utility>
#include <vector>

#include "../../include/rbc.h"

namespace rbc {

// Largest coefficient count per Chebyshev parity solved with explicit inverses.
constexpr int kDenseSolveMaxNq = 16;

// Grid and physical parameters, passed to kernels by value.
struct Grid {
  int Nx, Nz;     // native resolution (Fourier points, Chebyshev points)
  int nm;         // Fourier modes kept, m = 0 .. nm-1 (nm = Nx/2, Nyquist dropped)
  int Mx, Mz;     // 3/2-padded product grid (uniform x, Chebyshev-Lobatto z)
  int nq;         // coefficients per Chebyshev parity (Nz/2)
  double Ra, Pr, Lx, dt;
  double kfac;    // 2 pi / Lx, k_m = kfac * m
  int mixed;      // 1: transforms and products in FP32 (RBC_MIXED, RBC_MIXED_BF16)
  int tcbf16;     // 1: the tensor-core z transforms with BF16 operands (RBC_MIXED_BF16), else TF32
  int bc;         // RBC_FIXED_T or RBC_FIXED_FLUX (temperature boundary rows)
  int scheme;     // RBC_RK443, RBC_RK222 or RBC_RK111 (index of the tableaux)
  int ns;         // implicit stages per step: 4, 2 or 1
  double gamma;   // the constant implicit diagonal of the scheme (1/2 for RK443)
  double inv_gamma;
};

// Right-hand side of the temperature boundary row of the mean profile (m = 0)
// for Chebyshev parity p.  The rows are the parity combinations
// (f(1) + f(-1)) / 2 (even n) and (f(1) - f(-1)) / 2 (odd n) of the wall
// values (Eq. 6: T(-1/2) = 1, T(1/2) = 0), or, with fixed flux, of the wall
// slopes in s = 2z with the even / odd roles swapped (Eq. 7: dT/ds = -1/2 at
// both walls): 1/2, -1/2 and 0, -1/2.
#ifdef __CUDACC__
__host__ __device__
#endif
inline double t_wall_rhs(const Grid& g, int p) {
  if (g.bc == RBC_FIXED_FLUX) return p == 0 ? 0.0 : -0.5;
  return p == 0 ? 0.5 : -0.5;
}

// Device-resident operator tables (built on the host in FP64 once per grid/dt).
// Parity-split tables are laid out [p][row][j][m] so that threads with
// consecutive Fourier index m read consecutive addresses.
struct Tables {
  const double* zinv;   // [4][Mz][Nz]  d^q T_n / ds^q at the padded Lobatto points, q = 0..3
  const double* zfwd;   // [Nz][Mz]     padded Lobatto values -> T coefficients n < Nz
  const double* cc;     // [Mz]         Clenshaw-Curtis weights on the padded points
  const double2* tw;    // [Mx]         exp(-2 pi i t / Mx)
  const double* s2;     // [2][nq][3]   C^(2) conversion S1 S0, tau row t, columns q = t..t+2
  const double* s4;     // [2][nq][5]   C^(4) conversion S3 S2 S1 S0, columns q = t..t+4
  const double* mp;     // [2][nq][5][nm] psi mass operator lap_k in C^(4)
  // UL factors of the stage matrices (M - dt/2 L) with boundary rows on top.
  // T: D = 1, [2][nq][1][nm]; P (psi, m >= 1): D = 2, [2][nq][2][nm];
  // U (mean flow, m = 0): D = 1, [2][nq][1][1].  Dinv: [2][D*D][nmod];
  // invd (reciprocal diagonal): [2][nq][nmod] for every system.
  const double *T_multB, *T_multD, *T_Dinv, *T_Lb, *T_invd;
  const double *P_multB, *P_multD, *P_Dinv, *P_Lb, *P_invd;
  const double *U_multB, *U_multD, *U_Dinv, *U_Lb, *U_invd;
  const double* gram;   // [Nz][Nz]  int_{-1}^{1} T_a T_b ds
  // native grid transforms
  const double2* twn;   // [Nx]      exp(-2 pi i t / Nx)
  const double* Vn;     // [Nz][Nz]  T_n(s_j) at the native points
  const double* Vn1;    // [Nz][Nz]  T_n'(s_j)
  const double* Wn;     // [Nz][Nz]  native values -> T coefficients (exact interpolation)
  // Explicit inverses of the parity systems, [2][nq][nq][nmod], built for grids
  // with nq <= kDenseSolveMaxNq only (otherwise nullptr): small systems are
  // solved by a parallel matrix-vector product instead of the sequential UL
  // recurrences, whose FP64 dependency chain dominates their latency.
  const double *T_inv, *P_inv, *U_inv;
  // FP32 copies of the transform tables (RBC_MIXED)
  const float* zinv32;  // [4][Mz][Nz]
  const float* zfwd32;  // [Nz][Mz]
  const float2* tw32;   // [Mx]
  // tensor-core z-inverse operands (RBC_MIXED): TF32 hi/lo images of the
  // interleaved operator rows, pre-swizzled per 128-row tile and 32-wide K-chunk
  const float *tcA_psi_hi, *tcA_psi_lo, *tcA_T_hi, *tcA_T_lo;
  // tensor-core z-forward operands (RBC_MIXED): TF32 hi/lo images of the rows
  // of the forward matrix of each Chebyshev parity, per 128-row tile and K-chunk
  const float *tcW_hi[2], *tcW_lo[2];
  // [5][5] dt * (explicit tableau entry) and, at [25], (gamma dt) Pr: products
  // the stage solve would otherwise form per element (same IEEE products, same bits)
  const double* dtae;
};

// Error bits a kernel sets for a state (Work::flags) and for the handle (Work::err).
constexpr int kFlagNonFinite = 1;   // a stage solve produced NaN/Inf
constexpr int kFlagTimeout = 2;     // a bounded device-side wait gave up

// Optional per-kernel CUDA-event timing (host side).  Event pairs come from a
// pool; when it runs out, the stream is synchronised and the elapsed times are
// folded into the totals so that the pool can be reused.
struct Prof {
  bool on = false;
  bool once = false;             // record the next rbc_step_batch call only
  std::vector<cudaEvent_t> ev;   // 2 per record
  std::vector<int> kind;         // kind of each recorded pair
  size_t used = 0;
  double ms[RBC_NKERNELS] = {};
  long long launches[RBC_NKERNELS] = {};
  double flops[RBC_NKERNELS] = {};
  double bytes[RBC_NKERNELS] = {};
  cudaError_t fold();
  void begin(int k, cudaStream_t s);
  void end(int k, cudaStream_t s, double fl, double by);
};

// Launch shapes that leave every result unchanged bit for bit (each column's
// solve, each z-forward sum and each row's arithmetic do not depend on them),
// picked per batch size by rbc_autotune; 0 (or -1 for rows_cl) keeps the
// built-in heuristic.
struct Shapes {
  int solve_tms = 0;   // Fourier modes per k_solve block (power of two, <= 16)
  int zfwd_tm = 0;     // Fourier modes per k_zfwd block (power of two, <= 32)
  int zfwd_nch = 0;    // chunks of the n range per k_zfwd block (1, 2, 4, 8)
  int rows_cl = -1;    // 1: the clustered row kernel, 0: one block per row
  int rows_threads = 0;   // threads of a k_rows block (256, 512 or 1024)
  int rows_lean = -1;  // 1: k_rows with 5 + 3 shared rows, 0: 5 + 5 (where either fits)
};

// Per-call workspace pointers (capacity >= B states).
struct Work {
  double* Xs;      // stage state, B states
  double* F;       // explicit-term coefficients, B states
  double* R;       // RK accumulators, [B][4] states (tau rows in the coefficient slots)
  double* Z;       // z-inverse output, [B][9][Mz][nm] complex (FP64, or FP32 in the first half)
  double* Q;       // row-kernel output, [B][2][Mz][nm] complex (FP64 or FP32)
  double* wT;      // [B][Mz] x-mean of w T
  int* maxs;       // [1] max over nsteps, right before nsteps (copied with it)
  int* nsteps;     // [B]
  int* step;       // [1] step counter of the running batch
  int* flags;      // [B] error bits of the running batch: kFlagNonFinite, kFlagTimeout
  int* err;        // [1] the same bits, OR-ed over every call since the last read (sticky)
  int* dflag;      // [1] error bits of a diagnostic call (rbc_nusselt)
  double* nu;      // [B] internal Nu integral when the caller passes none
  double* small;   // [16] scalars
  double* ra;      // [B] Rayleigh number of each state
  const int* cancel;   // device word that ends the step loops early when set, or nullptr
  const Shapes* shapes;   // tuned launch shapes of this batch size, or nullptr
  int pdl;         // 1: step kernels with programmatic dependent launch (batches of <= kPdlMaxBatch)
  Prof* prof;      // timing, or nullptr
};

// largest batch whose step kernels use programmatic dependent launch (below)
constexpr int kPdlMaxBatch = 2;

#ifdef __CUDACC__
#define RBC_HD __host__ __device__

// Programmatic dependent launch of the step kernels of small batches (at most
// kPdlMaxBatch states, the coarse sweeps): such a kernel is launched with
// programmatic stream serialisation and begins with pdl_wait(), which returns
// once the previous kernel on the stream has completed and its writes are
// visible (griddepcontrol.wait: a hardware dependency, like the stream order
// it replaces, not a spin).  No kernel triggers its dependents early, so the
// next kernel is launched as the previous one's blocks exit: its launch is
// hidden behind their tail, and its blocks are placed on an idle GPU as in
// plain stream order (triggering at kernel entry placed them beside running
// blocks and slowed single-slice steps by up to 10 %).  Launched without the
// attribute (larger batches, or first in a graph body) the wait is a no-op.
// The arithmetic, and so every bit, is that of plain stream order.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}
#else
#define RBC_HD
#endif
RBC_HD inline size_t state_doubles(const Grid& g) { return (size_t)2 * g.Nz * g.nm * 2; }
RBC_HD inline size_t z_doubles(const Grid& g) { return (size_t)9 * g.Mz * g.nm * 2; }
RBC_HD inline size_t q_doubles(const Grid& g) { return (size_t)2 * g.Mz * g.nm * 2; }

// ---- launchers (rbc_kernels.cu) ----
cudaError_t launch_stage(const Grid& g, const Tables& t, const Work& w, double* X, int B, int stage,
                         double* nu, cudaStream_t s);
cudaError_t launch_explicit(const Grid& g, const Tables& t, const Work& w, const double* X, int B,
                            bool all_active, cudaStream_t s);
cudaError_t launch_advance(const Work& w, cudaStream_t s);
// advance the step counter and keep the enclosing graph loop running while step < maxs
cudaError_t launch_advance_loop(const Work& w, cudaGraphConditionalHandle loop, cudaStream_t s);

cudaError_t launch_nu_final(const Grid& g, const Tables& t, const Work& w, const double* X, int B,
                            double* nu, cudaStream_t s);
cudaError_t launch_nusselt(const Grid& g, const Tables& t, const Work& w, const double* X, double* out3,
                           cudaStream_t s);
// Sec. 2.2 averages of B states into out[B][6 + 2 Mz] (layout as rbc_diagnostics)
cudaError_t launch_diagnostics(const Grid& g, const Tables& t, const Work& w, const double* X, int B, double* out,
                               cudaStream_t s);
// Time statistics of Sec. 2.2: sampled quantities from diagnostics rows (in
// place), trapezoid accumulation (acc += h2 (prev + cur); prev = cur), a += b.
cudaError_t launch_stat_sample(const Grid& g, double* d, int B, cudaStream_t s);
cudaError_t launch_stat_accum(double* acc, double* prev, const double* cur, double h2, long n, cudaStream_t s);
cudaError_t launch_add(double* a, const double* b, int n, cudaStream_t s);
cudaError_t launch_l2_diff(const Grid& g, const Tables& t, const double* A, const double* Bm, int nst,
                           double* out, cudaStream_t s);
cudaError_t launch_set_state(const Grid& g, const Tables& t, const double* gT, const double* gu,
                             const double* gw, double* scratch, double* X, cudaStream_t s);
cudaError_t launch_get_state(const Grid& g, const Tables& t, const double* X, double* scratch, double* gT,
                             double* gu, double* gw, cudaStream_t s);
cudaError_t launch_restrict(const Grid& gf, const Grid& gc, const double* Xf, double* Xc, int B, cudaStream_t s);
cudaError_t launch_correct(const Grid& gf, const Grid& gc, const double* Ff, const double* Gnew,
                           const double* Gold, double* Uout, int B, cudaStream_t s);
cudaError_t launch_prolong(const Grid& gf, const Grid& gc, const double* Xc, double* Xf, int B, cudaStream_t s);
// One slice of a Parareal sweep fused with its norms (mode 0: U^0 = prolong(Gnew);
// mode 1: the correction of Eq. 20); see k_correct_norm.  partial: 2 doubles
// per block (correct_norm_blocks), counter: one zeroed unsigned; launches on
// the same (partial, counter) must be ordered (one stream).
int correct_norm_blocks(const Grid& gf);
cudaError_t launch_correct_norm(const Grid& gf, const Grid& gc, const Tables& tf, int mode, const double* Ff,
                                const double* Gnew, double* Gold, double* C, const double* Uprev, double* U,
                                double* Fnext, double* partial, unsigned* counter, double* norms, cudaStream_t s);
size_t rows_smem_bytes(const Grid& g);
// whether a launch shape can run on this grid (shared memory, threads)
bool shapes_valid(const Grid& g, const Shapes& sh, size_t es);
size_t static_scratch_doubles_needed(const Grid& g);
constexpr size_t kStaticScratchCapacity = (size_t)3 << 17;   // doubles in the static scratch array (3 MiB)
// Nusselt numbers with all scratch in the static array; *host_flags receives
// the error bits of the call (kFlagTimeout when a bounded wait gave up).
cudaError_t launch_nusselt_static(const Grid& g, const Tables& t, const double* X, double* host_out3,
                                  int* host_flags, cudaStream_t s);
unsigned long long launches_so_far();
void add_launches(unsigned long long n);   // kernels launched through a replayed graph
// kernels of one captured step: 4 per stage + the step counter
inline int step_kernels(const Grid& g) { return 4 * g.ns + 1; }
// tableaux of the IMEX pairs (host copy), stage count and implicit diagonal
void scheme_tableau(int scheme, double AE[5][5], double AI[5][5], int* ns, double* gamma);
// copies the three schemes' tableaux to the device's constant memory
cudaError_t upload_schemes();
constexpr int kProfileSampleSteps = 8;     // steps recorded kernel by kernel in a sampled call
cudaError_t configure_kernels(const Grid& g);
// tensor-core z inverse transform (rbc_tcgen05.cu)
RBC_HD int tc_zinv_mtiles(const Grid& g, int nops);
RBC_HD int tc_zinv_kchunks(const Grid& g);
size_t tc_zinv_image_floats(const Grid& g, int nops);
void tc_zinv_build_images(const Grid& g, const double* zinv, int nops, float* hi, float* lo);
bool tc_zinv_supported(const Grid& g);
cudaError_t launch_zinv_tc(const Grid& g, const Tables& t, const Work& w, const double* X, int B, const int* ns,
                           cudaStream_t s);
// tensor-core z forward transform (rbc_tcgen05.cu)
RBC_HD int tc_zfwd_mtiles(const Grid& g);
RBC_HD int tc_zfwd_kchunks(const Grid& g);
size_t tc_zfwd_image_floats(const Grid& g);
void tc_zfwd_build_images(const Grid& g, const double* zfwd, int p, float* hi, float* lo);
bool tc_zfwd_supported(const Grid& g);
cudaError_t launch_zfwd_tc(const Grid& g, const Tables& t, const Work& w, int B, cudaStream_t s);
// Spin limit of the bounded mbarrier waits of the tensor-core kernels on the
// current device (limit < 0: the default).  Waits that drain work already
// issued before tensor memory is freed keep their own, default limit.
cudaError_t tc_set_wait_limit(long long limit);

}  // namespace rbc
