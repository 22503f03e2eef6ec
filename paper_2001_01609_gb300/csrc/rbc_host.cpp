// Host runtime of the RBC Parareal library: operator assembly and UL
// factorisation (FP64, once per grid and time step), workspace management,
// the RK443 step loop, and the Parareal control flow (Eq. 20).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "rbc_internal.h"

#include <cuda.h>   // driver types of SM partitions; the functions are resolved at run time

using namespace rbc;

namespace {

thread_local char g_err[512] = "";

rbc_status fail(rbc_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return fail(RBC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// Dense N x N operators on Chebyshev-T coefficients (row-major).
// Ultraspherical method (Olver & Townsend): conversions T -> C^(1) -> C^(2) ...
// and derivatives T -> C^(lambda).
// ---------------------------------------------------------------------------
using Mat = std::vector<double>;

Mat eye_like(int N) { return Mat((size_t)N * N, 0.0); }

// T_n = (C1_n - C1_{n-2}) / 2 (n >= 2), T_1 = C1_1 / 2, T_0 = C1_0.
Mat conv_T_C1(int N) {
  Mat S = eye_like(N);
  S[0] = 1.0;
  for (int j = 1; j < N; ++j) S[(size_t)j * N + j] = 0.5;
  for (int j = 0; j + 2 < N; ++j) S[(size_t)j * N + j + 2] = -0.5;
  return S;
}

// C^(l)_n = l/(n+l) (C^(l+1)_n - C^(l+1)_{n-2}).
Mat conv_C(int l, int N) {
  Mat S = eye_like(N);
  for (int j = 0; j < N; ++j) {
    S[(size_t)j * N + j] = (double)l / (j + l);
    if (j + 2 < N) S[(size_t)j * N + j + 2] = -(double)l / (j + l + 2);
  }
  return S;
}

// d^l T_n / ds^l = 2^(l-1) (l-1)! n C^(l)_{n-l}.
Mat deriv(int l, int N) {
  Mat D = eye_like(N);
  double c = std::ldexp(1.0, l - 1);
  for (int i = 2; i < l; ++i) c *= i;
  for (int j = 0; j + l < N; ++j) D[(size_t)j * N + j + l] = c * (j + l);
  return D;
}

Mat matmul(const Mat& A, const Mat& B, int N) {
  Mat C = eye_like(N);
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < N; ++k) {
      const double a = A[(size_t)i * N + k];
      if (a == 0.0) continue;
      for (int j = 0; j < N; ++j) C[(size_t)i * N + j] += a * B[(size_t)k * N + j];
    }
  return C;
}

// Values and derivatives (orders 0..Q) of T_0..T_{N-1} at s, by the
// three-term recurrence T_{n+1} = 2 s T_n - T_{n-1} differentiated q times:
// T^(q)_{n+1} = 2 s T^(q)_n + 2 q T^(q-1)_n - T^(q)_{n-1}.
void cheb_eval(double s, int N, int Q, std::vector<double>& out) {
  out.assign((size_t)(Q + 1) * N, 0.0);
  auto at = [&](int q, int n) -> double& { return out[(size_t)q * N + n]; };
  at(0, 0) = 1.0;
  if (N > 1) {
    at(0, 1) = s;
    if (Q >= 1) at(1, 1) = 1.0;
  }
  for (int n = 1; n + 1 < N; ++n)
    for (int q = 0; q <= Q; ++q)
      at(q, n + 1) = 2.0 * s * at(q, n) + (q > 0 ? 2.0 * q * at(q - 1, n) : 0.0) - at(q, n - 1);
}

// Exact interpolation on N Chebyshev-Lobatto points with angles theta_j:
// W[n][j] = 2/(N-1) * T_n(s_j) / (c_n c_j), c = 2 at the end points/indices.
Mat lobatto_interp(int N, const std::vector<double>& theta) {
  Mat W = eye_like(N);
  for (int n = 0; n < N; ++n)
    for (int j = 0; j < N; ++j) {
      const double cn = (n == 0 || n == N - 1) ? 2.0 : 1.0;
      const double cj = (j == 0 || j == N - 1) ? 2.0 : 1.0;
      W[(size_t)n * N + j] = 2.0 / (N - 1) * std::cos(n * theta[j]) / (cn * cj);
    }
  return W;
}

// ---------------------------------------------------------------------------
// UL factorisation of a parity-split stage matrix: D dense boundary rows on
// top, then tau rows whose nonzeros lie in columns r-D .. r+D (dominant
// derivative term on the diagonal).  Eliminating columns n-1 .. D from the
// bottom creates no fill; what remains is a D x D dense block and a lower
// band.  No pivoting; the residual is checked after factoring.
// ---------------------------------------------------------------------------
struct UL {
  int n = 0, D = 0;
  std::vector<double> multB, multD, Dinv, Lb, invd;  // [c][D], [c][D], [D*D], [r][D], [r]
};

bool ul_factor(Mat A, int n, int D, UL& f, std::string& why) {
  f.n = n;
  f.D = D;
  f.multB.assign((size_t)n * D, 0.0);
  f.multD.assign((size_t)n * D, 0.0);
  f.Lb.assign((size_t)n * D, 0.0);
  f.invd.assign(n, 0.0);
  f.Dinv.assign(D * D, 0.0);
  auto a = [&](int r, int c) -> double& { return A[(size_t)r * n + c]; };
  for (int c = n - 1; c >= D; --c) {
    const double piv = a(c, c);
    if (piv == 0.0 || !std::isfinite(piv)) {
      why = "zero pivot";
      return false;
    }
    for (int r = 0; r < c; ++r) {
      const double v = a(r, c);
      if (v == 0.0) continue;
      if (r >= D && r < c - D) {
        why = "band structure violated";
        return false;
      }
      const double mult = v / piv;
      for (int q = std::max(0, c - D); q < c; ++q) a(r, q) -= mult * a(c, q);
      a(r, c) = 0.0;
      if (r < D)
        f.multD[(size_t)c * D + r] = mult;
      else
        f.multB[(size_t)c * D + (r - (c - D))] = mult;
    }
  }
  for (int r = D; r < n; ++r) {
    for (int q = 0; q < r - D; ++q)
      if (a(r, q) != 0.0) {
        why = "lower band structure violated";
        return false;
      }
    for (int j = 0; j < D; ++j) f.Lb[(size_t)r * D + j] = a(r, r - D + j);
    f.invd[r] = 1.0 / a(r, r);
  }
  if (D == 1) {
    f.Dinv[0] = 1.0 / a(0, 0);
  } else {
    const double det = a(0, 0) * a(1, 1) - a(0, 1) * a(1, 0);
    if (det == 0.0) {
      why = "singular boundary block";
      return false;
    }
    f.Dinv[0] = a(1, 1) / det;
    f.Dinv[1] = -a(0, 1) / det;
    f.Dinv[2] = -a(1, 0) / det;
    f.Dinv[3] = a(0, 0) / det;
  }
  return true;
}

// Host mirror of the device solve, for the residual check.
void ul_solve(const UL& f, std::vector<double>& y, std::vector<double>& x) {
  const int n = f.n, D = f.D;
  for (int c = n - 1; c >= D; --c) {
    for (int j = 0; j < D; ++j) {
      const int r = c - D + j;
      if (r >= D) y[r] -= f.multB[(size_t)c * D + j] * y[c];
    }
    for (int r = 0; r < D; ++r) y[r] -= f.multD[(size_t)c * D + r] * y[c];
  }
  x.assign(n, 0.0);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) x[r] += f.Dinv[r * D + c] * y[c];
  for (int r = D; r < n; ++r) {
    double s = y[r];
    for (int j = 0; j < D; ++j) s -= f.Lb[(size_t)r * D + j] * x[r - D + j];
    x[r] = s * f.invd[r];
  }
}

double ul_residual(const Mat& A, const UL& f, unsigned seed) {
  const int n = f.n;
  std::vector<double> b(n), y, x;
  unsigned s = seed * 2654435761u + 12345u;
  for (int i = 0; i < n; ++i) {
    s = s * 1664525u + 1013904223u;
    b[i] = (double)(s >> 8) / (double)(1u << 24) - 0.5;
  }
  y = b;
  ul_solve(f, y, x);
  double rmax = 0.0, amax = 0.0, xmax = 0.0, bmax = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = -b[i], arow = 0.0;
    for (int j = 0; j < n; ++j) {
      r += A[(size_t)i * n + j] * x[j];
      arow += std::fabs(A[(size_t)i * n + j]);
    }
    rmax = std::max(rmax, std::fabs(r));
    amax = std::max(amax, arow);
    xmax = std::max(xmax, std::fabs(x[i]));
    bmax = std::max(bmax, std::fabs(b[i]));
  }
  return rmax / (amax * xmax + bmax);
}

}  // namespace

// ---------------------------------------------------------------------------
// Handle.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// SM partitions (green contexts).  The driver entry points are looked up at run
// time, so the library does not link libcuda and loads without a driver.
// ---------------------------------------------------------------------------
struct DriverApi {
  CUresult (*get_resource)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
  CUresult (*split)(CUdevResource*, unsigned*, const CUdevResource*, CUdevResource*, unsigned, unsigned) = nullptr;
  CUresult (*make_desc)(CUdevResourceDesc*, CUdevResource*, unsigned) = nullptr;
  CUresult (*green_create)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned) = nullptr;
  CUresult (*green_destroy)(CUgreenCtx) = nullptr;
  CUresult (*from_green)(CUcontext*, CUgreenCtx) = nullptr;
  CUresult (*ctx_get)(CUcontext*) = nullptr;
  CUresult (*ctx_set)(CUcontext) = nullptr;
  bool ok = false;
};

static const DriverApi& driver_api() {
  static const DriverApi api = [] {
    DriverApi a;
    auto get = [](const char* name, void** fn) {
      cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
      return cudaGetDriverEntryPointByVersion(name, fn, 13000, cudaEnableDefault, &q) == cudaSuccess &&
             q == cudaDriverEntryPointSuccess && *fn != nullptr;
    };
    a.ok = get("cuDeviceGetDevResource", reinterpret_cast<void**>(&a.get_resource)) &&
           get("cuDevSmResourceSplitByCount", reinterpret_cast<void**>(&a.split)) &&
           get("cuDevResourceGenerateDesc", reinterpret_cast<void**>(&a.make_desc)) &&
           get("cuGreenCtxCreate", reinterpret_cast<void**>(&a.green_create)) &&
           get("cuGreenCtxDestroy", reinterpret_cast<void**>(&a.green_destroy)) &&
           get("cuCtxFromGreenCtx", reinterpret_cast<void**>(&a.from_green)) &&
           get("cuCtxGetCurrent", reinterpret_cast<void**>(&a.ctx_get)) &&
           get("cuCtxSetCurrent", reinterpret_cast<void**>(&a.ctx_set));
    return a;
  }();
  return api;
}

// Makes `ctx` (a partition's context) current for the scope; nullptr keeps
// the current (primary) context.  ok() is false if the switch failed.
class CtxScope {
 public:
  explicit CtxScope(CUcontext ctx) {
    if (!ctx) return;
    const DriverApi& d = driver_api();
    if (!d.ok || d.ctx_get(&prev_) != CUDA_SUCCESS || d.ctx_set(ctx) != CUDA_SUCCESS) {
      failed_ = true;
      return;
    }
    switched_ = true;
  }
  ~CtxScope() {
    if (switched_) driver_api().ctx_set(prev_);
  }
  bool ok() const { return !failed_; }

 private:
  CUcontext prev_ = nullptr;
  bool switched_ = false, failed_ = false;
};

struct rbc_s {
  Grid g{};
  rbc_opts opts{};
  int device = 0;
  double max_residual = 0.0;
  double* d_tables = nullptr;
  Tables t{};
  int cap = 0;
  void* d_work = nullptr;
  Work w{};
  double* d_scratch = nullptr;   // set/get state and diagnostics, independent of B
  double* d_sbuf = nullptr;      // sampled runs: two rows of diagnostics per state and a Nu slot
  int sbuf_cap = 0;              // states d_sbuf holds
  int last_B = 0;
  // Pinned staging of each call's host arrays (Ra, step counts): a ring of
  // slots, each reused only after the copy that last read it has run, so the
  // host can queue several calls ahead of the device.
  static constexpr int kPinSlots = 8;
  char* pin = nullptr;
  size_t pin_slot = 0;
  cudaEvent_t pin_ev[kPinSlots] = {};
  bool pin_busy[kPinSlots] = {};
  int pin_next = 0;
  // what the workspace holds from the last upload: a call with the same
  // arrays (a serial sweep repeats them) queues no copy at all
  std::vector<int> up_ns;
  std::vector<double> up_ra;
  Prof prof;
  Prof* profp = nullptr;   // the timing record in use: its own, or its template's (Parareal's copies)
  // Launch shapes picked by rbc_autotune, per batch size; `gen` counts the
  // changes, so that step graphs captured with other shapes are not reused.
  struct Tuning {
    std::map<int, Shapes> byB;
    unsigned gen = 0;
  };
  Tuning tuning;
  Tuning* tunep = nullptr;   // its own table, or its template's (Parareal's copies)
  // Step loops: a graph whose one node is a device-side while loop over the
  // captured RK443 step (4 stages + counter), so a call of any length is one
  // launch.  A few bindings (states, B, nu) are kept, least recently used out.
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    const void* X = nullptr;
    const void* nu = nullptr;
    int B = -1;
    CUcontext ctx = nullptr;   // the SM partition it was captured in (nullptr: whole GPU)
    unsigned tune_gen = 0;     // the launch shapes it was captured with
    unsigned long long used = 0;
  };
  static constexpr int kGraphCache = 8;
  StepGraph graphs[kGraphCache];
  unsigned long long graph_clock = 0;
  // Step graphs are captured in `bind_ctx` (set by a Parareal schedule that
  // confines this handle to an SM partition), on a capture stream of that context.
  CUcontext bind_ctx = nullptr;
  struct CapStream {
    CUcontext ctx = nullptr;
    cudaStream_t s = nullptr;
  };
  static constexpr int kCapStreams = 4;
  CapStream caps[kCapStreams];
  bool use_graphs = true;
};

struct pr_s {
  rbc_t fine = nullptr, coarse = nullptr;   // the caller's handles: grids, time steps, options, tables
  double t0 = 0, t1 = 0;
  int N = 0, nf = 0, nc = 0, criterion = 0;
  double tol = 0;
  // Schedule (timing only; the results are the same bit for bit).
  int group = 0;              // largest fine group
  int first_group = 0;        // first fine group
  int fine_streams = 2;       // fine groups of an iteration alternate over this many streams
  int coarse_priority = 1;    // 1: the sweeps on the coarse grid run on high-priority streams
  int depth = 1;              // iterations enqueued beyond the one the host evaluates next
  // Sampled time statistics of Sec. 2.2 along the fine sweeps (every > 0):
  // diagnostics every `every` fine steps and at each slice end, trapezoid
  // integrals per slice; window = slices [window_first, N).
  int every = 0, window_first = 0;
  std::vector<double> stat_means;   // window means of the last evaluated iteration
  static constexpr int kFineStreams = 4;
  static constexpr int kMaxDepth = 6;
  // One slot per iteration in flight: iteration k uses slot k % R, R = depth + 2.
  // Its sweep on the coarse grid (k = 0: U^0; k >= 1: the correction of Eq. 20)
  // runs on the slot's coarse handle and stream; its fine groups on the slot's
  // fine handles and streams.  All handles are the library's own copies of the
  // caller's (sharing their tables), so that their step loops can be cancelled.
  struct Slot {
    rbc_t coarse = nullptr;
    rbc_t fines[kFineStreams] = {};
    cudaStream_t sC = nullptr, sC_hi = nullptr;   // the sweep: default / high priority
    cudaStream_t sF[kFineStreams] = {};
    cudaStream_t pC = nullptr;                    // the same in the SM partition (gctx[0], gctx[1])
    cudaStream_t pF[kFineStreams] = {};
    double* U = nullptr;        // [N+1] fine states: U^k
    double* Fin = nullptr;      // [N] fine states: inputs, then results, of the iteration's fine sweep
    double* C = nullptr;        // 1 coarse state: the sweep's coarse state
    double* I = nullptr;        // [N] Nu_V integrals of the fine sweep
    double* norms = nullptr;    // [N][2]: ||T(U^k_{n+1} - U^{k-1}_{n+1})||^2, ||T(U^k_{n+1})||^2
    double* stat = nullptr;     // [N][6 + 2 Mz]: sampled time integrals of the fine sweep (every > 0)
    double* partial = nullptr;  // block sums of the correction kernel
    unsigned* counter = nullptr;
    std::vector<cudaEvent_t> ev_step;    // [N] sweep step n done
    std::vector<cudaEvent_t> ev_group;   // [N] fine group j done
    std::vector<int> slice_group;        // fine group of each slice
    cudaEvent_t ev_join[1 + kFineStreams] = {};
    bool busy = false;                   // has work in the current call
  };
  std::vector<Slot> slots;
  double* d_Gold = nullptr;   // [N] coarse states G(U_n), updated in place by each sweep
  int* d_cancel = nullptr;    // read by the slots' step loops: set, they stop early
  cudaStream_t sCancel = nullptr;
  cudaEvent_t ev_begin = nullptr, ev_cancel = nullptr;
  // Optional SM reserve: the fine groups run in a green context of the SMs
  // outside `coarse_sms` reserved ones (gctx[1]; gctx[0] holds the reserve),
  // while the sweeps on the coarse grid run on the whole device, so that their
  // latency-bound kernels always find free SMs.
  int coarse_sms = 0;
  CUgreenCtx green[2] = {};
  CUcontext gctx[2] = {};
};

static void release_context(rbc_t h, CUcontext ctx);

// Remove the SM partition of a Parareal handle: its streams, the step graphs
// its handles captured in it, and the green contexts.
static void drop_partition(pr_s* p) {
  if (!p->gctx[0]) return;
  for (auto& S : p->slots)
    for (cudaStream_t* st : {&S.pC, &S.pF[0], &S.pF[1], &S.pF[2], &S.pF[3]})
      if (*st) {
        cudaStreamSynchronize(*st);
        cudaStreamDestroy(*st);
        *st = nullptr;
      }
  for (int i = 0; i < 2; ++i) {
    for (auto& S : p->slots) {
      release_context(S.coarse, p->gctx[i]);
      for (rbc_t h : S.fines) release_context(h, p->gctx[i]);
    }
    if (p->green[i]) driver_api().green_destroy(p->green[i]);
    p->green[i] = nullptr;
    p->gctx[i] = nullptr;
  }
  p->coarse_sms = 0;
}

static rbc_status make_partition(pr_s* p, int coarse_sms) {
  const DriverApi& d = driver_api();
  if (!d.ok) return fail(RBC_ECUDA, "SM partitions (green contexts) are not available");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CUdevResource all{}, grp{}, rest{};
  unsigned n = 1;
  if (d.get_resource((CUdevice)dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS ||
      d.split(&grp, &n, &all, &rest, 0, (unsigned)coarse_sms) != CUDA_SUCCESS || n != 1 || rest.sm.smCount == 0)
    return fail(RBC_ECUDA, "cannot split %d SMs off the device", coarse_sms);
  CUdevResourceDesc desc[2];
  if (d.make_desc(&desc[0], &grp, 1) != CUDA_SUCCESS || d.make_desc(&desc[1], &rest, 1) != CUDA_SUCCESS)
    return fail(RBC_ECUDA, "SM partition descriptors");
  for (int i = 0; i < 2; ++i)
    if (d.green_create(&p->green[i], desc[i], (CUdevice)dev, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS ||
        d.from_green(&p->gctx[i], p->green[i]) != CUDA_SUCCESS) {
      drop_partition(p);
      return fail(RBC_ECUDA, "green context creation");
    }
  p->coarse_sms = (int)grp.sm.smCount;
  return RBC_OK;
}

extern "C" const char* rbc_last_error(void) { return g_err; }

static rbc_status upload_tables(rbc_t h) {
  const Grid& g = h->g;
  const int N = g.Nz, Mz = g.Mz, nq = g.nq, nm = g.nm;
  std::vector<double> buf;
  std::vector<size_t> offs;
  auto add = [&](const std::vector<double>& v) {
    size_t o = buf.size();
    o = (o + 1) & ~(size_t)1;   // 16-byte alignment for double2 loads
    buf.resize(o);
    buf.insert(buf.end(), v.begin(), v.end());
    offs.push_back(o);
  };

  // ---- z transforms at the padded Lobatto points s_j = cos(pi j/(Mz-1)) ----
  std::vector<double> zinv((size_t)4 * Mz * N), ev;
  std::vector<double> thp(Mz);
  for (int j = 0; j < Mz; ++j) thp[j] = M_PI * j / (Mz - 1);
  for (int j = 0; j < Mz; ++j) {
    cheb_eval(std::cos(thp[j]), N, 3, ev);
    for (int q = 0; q < 4; ++q)
      for (int n = 0; n < N; ++n) zinv[((size_t)q * Mz + j) * N + n] = ev[(size_t)q * N + n];
  }
  Mat Wfull = lobatto_interp(Mz, thp);
  std::vector<double> zfwd((size_t)N * Mz), cc(Mz, 0.0);
  for (int n = 0; n < N; ++n)
    for (int j = 0; j < Mz; ++j) zfwd[(size_t)n * Mz + j] = Wfull[(size_t)n * Mz + j];
  for (int j = 0; j < Mz; ++j)
    for (int n = 0; n < Mz; n += 2) cc[j] += Wfull[(size_t)n * Mz + j] * 2.0 / (1.0 - (double)n * n);
  std::vector<double> tw((size_t)2 * g.Mx);
  for (int t = 0; t < g.Mx; ++t) {
    tw[2 * t] = std::cos(2.0 * M_PI * t / g.Mx);
    tw[2 * t + 1] = -std::sin(2.0 * M_PI * t / g.Mx);
  }

  // ---- ultraspherical operators ----
  const Mat S0 = conv_T_C1(N);
  const Mat S2 = matmul(conv_C(1, N), S0, N);
  const Mat C32 = matmul(conv_C(3, N), conv_C(2, N), N);
  const Mat S4 = matmul(C32, S2, N);
  const Mat D2 = deriv(2, N);
  const Mat S4D2 = matmul(C32, D2, N);
  const Mat D4 = deriv(4, N);
  auto el = [&](const Mat& M, int r, int c) -> double { return (c < N) ? M[(size_t)r * N + c] : 0.0; };
  // structural check: row j couples only columns j, j+2, ..., j+2*lam
  auto check_band = [&](const Mat& M, int rows, int lam) -> bool {
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < N; ++c) {
        const double v = M[(size_t)r * N + c];
        if (v != 0.0 && (c < r || c > r + 2 * lam || ((c - r) & 1))) return false;
      }
    return true;
  };
  if (!check_band(S2, N - 2, 2) || !check_band(D2, N - 2, 2) || !check_band(S4, N - 4, 4) ||
      !check_band(S4D2, N - 4, 4) || !check_band(D4, N - 4, 4))
    return fail(RBC_EINVAL, "operator band structure check failed");

  std::vector<double> s2((size_t)2 * nq * 3, 0.0), s4((size_t)2 * nq * 5, 0.0), mp((size_t)2 * nq * 5 * nm, 0.0);
  for (int p = 0; p < 2; ++p)
    for (int t = 0; t < nq; ++t) {
      const int r = 2 * t + p;
      for (int j = 0; j < 3; ++j)
        if (r < N - 2) s2[(p * nq + t) * 3 + j] = el(S2, r, 2 * (t + j) + p);
      for (int j = 0; j < 5; ++j)
        if (r < N - 4) s4[(p * nq + t) * 5 + j] = el(S4, r, 2 * (t + j) + p);
      for (int m = 0; m < nm; ++m) {
        const double k = g.kfac * m;
        for (int j = 0; j < 5; ++j)
          if (r < N - 4) {
            const int c = 2 * (t + j) + p;
            mp[((size_t)(p * nq + t) * 5 + j) * nm + m] = 4.0 * el(S4D2, r, c) - k * k * el(S4, r, c);
          }
      }
    }

  // ---- stage matrices and their UL factors ----
  const double hdt = g.gamma * g.dt;       // stage matrices M - gamma dt L
  auto layout = [&](std::vector<double>& dst, const std::vector<double>& src, int p, int rows, int D, int nmod,
                    int mi) {
    for (int c = 0; c < rows; ++c)
      for (int j = 0; j < D; ++j) dst[((size_t)(p * rows + c) * D + j) * nmod + mi] = src[(size_t)c * D + j];
  };
  std::vector<double> Tb((size_t)2 * nq * nm), Td(Tb.size()), TDi((size_t)2 * nm), TL(Tb.size()), Ti(Tb.size());
  std::vector<double> Pb((size_t)2 * nq * 2 * nm), Pd(Pb.size()), PDi((size_t)2 * 4 * nm), PL(Pb.size()),
      Pi((size_t)2 * nq * nm);
  std::vector<double> Ub((size_t)2 * nq), Ud(Ub.size()), UDi(2), UL_(Ub.size()), Ui(Ub.size());
  // explicit inverses of the parity systems of small grids, [p][r][q][m]
  const bool dense = nq <= kDenseSolveMaxNq;
  const size_t ninv = dense ? (size_t)2 * nq * nq : 0;
  std::vector<double> Tinv(ninv * nm), Pinv(ninv * nm), Uinv(ninv);
  auto inverse_into = [&](const UL& f, std::vector<double>& dst, int p, int nmod, int mi) {
    std::vector<double> y, x;
    for (int q = 0; q < nq; ++q) {
      y.assign(nq, 0.0);
      y[q] = 1.0;
      ul_solve(f, y, x);
      for (int r = 0; r < nq; ++r) dst[(((size_t)p * nq + r) * nq + q) * nmod + mi] = x[r];
    }
  };
  double worst = 0.0;
  std::string why;
  for (int p = 0; p < 2; ++p) {
    for (int m = 0; m < nm; ++m) {
      const double k = g.kfac * m;
      // temperature: BC row (wall values: all ones; wall slopes: n^2), tau rows
      // of S2 - h (4 D2 - k^2 S2)
      Mat A((size_t)nq * nq, 0.0);
      for (int q = 0; q < nq; ++q) {
        const double n = 2 * q + p;
        A[q] = (g.bc == RBC_FIXED_FLUX) ? n * n : 1.0;
      }
      for (int t = 0; t + 1 < nq; ++t)
        for (int q = 0; q < nq; ++q) {
          const int r = 2 * t + p, c = 2 * q + p;
          A[(size_t)(1 + t) * nq + q] = el(S2, r, c) - hdt * (4.0 * el(D2, r, c) - k * k * el(S2, r, c));
        }
      UL f;
      if (!ul_factor(A, nq, 1, f, why)) return fail(RBC_EINVAL, "T system m=%d p=%d: %s", m, p, why.c_str());
      worst = std::max(worst, ul_residual(A, f, 17 * m + p));
      layout(Tb, f.multB, p, nq, 1, nm, m);
      layout(Td, f.multD, p, nq, 1, nm, m);
      layout(TL, f.Lb, p, nq, 1, nm, m);
      for (int r = 0; r < nq; ++r) Ti[(size_t)(p * nq + r) * nm + m] = f.invd[r];
      TDi[(size_t)p * nm + m] = f.Dinv[0];
      if (dense) inverse_into(f, Tinv, p, nm, m);
      if (m == 0) {
        // mean flow: S2 - h 4 Pr D2
        Mat U((size_t)nq * nq, 0.0);
        for (int q = 0; q < nq; ++q) U[q] = 1.0;
        for (int t = 0; t + 1 < nq; ++t)
          for (int q = 0; q < nq; ++q) {
            const int r = 2 * t + p, c = 2 * q + p;
            U[(size_t)(1 + t) * nq + q] = el(S2, r, c) - hdt * 4.0 * g.Pr * el(D2, r, c);
          }
        UL fu;
        if (!ul_factor(U, nq, 1, fu, why)) return fail(RBC_EINVAL, "U system p=%d: %s", p, why.c_str());
        worst = std::max(worst, ul_residual(U, fu, 99 + p));
        layout(Ub, fu.multB, p, nq, 1, 1, 0);
        layout(Ud, fu.multD, p, nq, 1, 1, 0);
        layout(UL_, fu.Lb, p, nq, 1, 1, 0);
        for (int r = 0; r < nq; ++r) Ui[(size_t)p * nq + r] = fu.invd[r];
        UDi[p] = fu.Dinv[0];
        if (dense) inverse_into(fu, Uinv, p, 1, 0);
      } else {
        // streamfunction: BC rows (ones, n^2), tau rows of M - h L in C^(4)
        Mat P((size_t)nq * nq, 0.0);
        for (int q = 0; q < nq; ++q) {
          const double n = 2 * q + p;
          P[q] = 1.0;
          P[(size_t)nq + q] = n * n;
        }
        for (int t = 0; t + 2 < nq; ++t)
          for (int q = 0; q < nq; ++q) {
            const int r = 2 * t + p, c = 2 * q + p;
            const double M = 4.0 * el(S4D2, r, c) - k * k * el(S4, r, c);
            const double L =
                g.Pr * (16.0 * el(D4, r, c) - 8.0 * k * k * el(S4D2, r, c) + k * k * k * k * el(S4, r, c));
            P[(size_t)(2 + t) * nq + q] = M - hdt * L;
          }
        UL fp;
        if (!ul_factor(P, nq, 2, fp, why)) return fail(RBC_EINVAL, "psi system m=%d p=%d: %s", m, p, why.c_str());
        worst = std::max(worst, ul_residual(P, fp, 31 * m + p));
        layout(Pb, fp.multB, p, nq, 2, nm, m);
        layout(Pd, fp.multD, p, nq, 2, nm, m);
        layout(PL, fp.Lb, p, nq, 2, nm, m);
        for (int r = 0; r < nq; ++r) Pi[(size_t)(p * nq + r) * nm + m] = fp.invd[r];
        for (int e = 0; e < 4; ++e) PDi[((size_t)p * 4 + e) * nm + m] = fp.Dinv[e];
        if (dense) inverse_into(fp, Pinv, p, nm, m);
      }
    }
  }
  h->max_residual = worst;
  if (!(worst < 1e-9)) return fail(RBC_EINVAL, "stage solve residual %.3e too large (unpivoted UL)", worst);

  // ---- norms and native grid transforms ----
  std::vector<double> gram((size_t)N * N, 0.0);
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b)
      if (((a + b) & 1) == 0)
        gram[(size_t)a * N + b] = 1.0 / (1.0 - (double)(a + b) * (a + b)) + 1.0 / (1.0 - (double)(a - b) * (a - b));
  std::vector<double> twn((size_t)2 * g.Nx);
  for (int t = 0; t < g.Nx; ++t) {
    twn[2 * t] = std::cos(2.0 * M_PI * t / g.Nx);
    twn[2 * t + 1] = -std::sin(2.0 * M_PI * t / g.Nx);
  }
  std::vector<double> thn(N);  // native s_j = -cos(pi j/(N-1)) = cos(pi (N-1-j)/(N-1))
  for (int j = 0; j < N; ++j) thn[j] = M_PI * (N - 1 - j) / (N - 1);
  std::vector<double> Vn((size_t)N * N), Vn1((size_t)N * N);
  for (int j = 0; j < N; ++j) {
    cheb_eval(std::cos(thn[j]), N, 1, ev);
    for (int n = 0; n < N; ++n) {
      Vn[(size_t)j * N + n] = ev[n];
      Vn1[(size_t)j * N + n] = ev[(size_t)N + n];
    }
  }
  Mat Wn = lobatto_interp(N, thn);

  add(zinv); add(zfwd); add(cc); add(tw); add(s2); add(s4); add(mp);
  add(Tb); add(Td); add(TDi); add(TL); add(Ti);
  add(Pb); add(Pd); add(PDi); add(PL); add(Pi);
  add(Ub); add(Ud); add(UDi); add(UL_); add(Ui);
  add(gram); add(twn); add(Vn); add(Vn1); add(Wn);
  {
    // dt * (explicit tableau), then (gamma dt) Pr: the same IEEE products the
    // stage solve would form per element
    double ae[5][5], ai[5][5], gm;
    int ns;
    scheme_tableau(g.scheme, ae, ai, &ns, &gm);
    std::vector<double> dtae(26);
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) dtae[i * 5 + j] = g.dt * ae[i][j];
    dtae[25] = (g.gamma * g.dt) * g.Pr;
    add(dtae);
  }
  // FP32 copies of the transform tables, packed two floats per double slot
  auto add_f32 = [&](const std::vector<double>& v) {
    std::vector<double> packed((v.size() + 1) / 2, 0.0);
    float* f = reinterpret_cast<float*>(packed.data());
    for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
    add(packed);
  };
  add_f32(zinv); add_f32(zfwd); add_f32(tw);
  add(Tinv); add(Pinv); add(Uinv);
  // tensor-core z-inverse operator images (mixed precision only)
  const bool tc = g.mixed && tc_zinv_supported(g);
  auto add_floats = [&](const std::vector<float>& v) {
    std::vector<double> packed((v.size() + 1) / 2, 0.0);
    memcpy(packed.data(), v.data(), v.size() * sizeof(float));
    add(packed);
  };
  {
    std::vector<float> ph(tc ? tc_zinv_image_floats(g, 4) : 0), pl(ph.size());
    std::vector<float> th(tc ? tc_zinv_image_floats(g, 2) : 0), tl(th.size());
    if (tc) {
      tc_zinv_build_images(g, zinv.data(), 4, ph.data(), pl.data());
      tc_zinv_build_images(g, zinv.data(), 2, th.data(), tl.data());
    }
    add_floats(ph); add_floats(pl); add_floats(th); add_floats(tl);
  }
  // tensor-core z-forward images, one pair per Chebyshev parity (mixed precision only)
  const bool tcw = g.mixed && tc_zfwd_supported(g);
  for (int p = 0; p < 2; ++p) {
    std::vector<float> wh(tcw ? tc_zfwd_image_floats(g) : 0), wl(wh.size());
    if (tcw) tc_zfwd_build_images(g, zfwd.data(), p, wh.data(), wl.data());
    add_floats(wh);
    add_floats(wl);
  }
  CK(cudaMalloc(&h->d_tables, buf.size() * sizeof(double)));
  CK(cudaMemcpy(h->d_tables, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice));
  const double* b = h->d_tables;
  int i = 0;
  Tables& T = h->t;
  T.zinv = b + offs[i++];
  T.zfwd = b + offs[i++];
  T.cc = b + offs[i++];
  T.tw = reinterpret_cast<const double2*>(b + offs[i++]);
  T.s2 = b + offs[i++];
  T.s4 = b + offs[i++];
  T.mp = b + offs[i++];
  T.T_multB = b + offs[i++]; T.T_multD = b + offs[i++]; T.T_Dinv = b + offs[i++]; T.T_Lb = b + offs[i++]; T.T_invd = b + offs[i++];
  T.P_multB = b + offs[i++]; T.P_multD = b + offs[i++]; T.P_Dinv = b + offs[i++]; T.P_Lb = b + offs[i++]; T.P_invd = b + offs[i++];
  T.U_multB = b + offs[i++]; T.U_multD = b + offs[i++]; T.U_Dinv = b + offs[i++]; T.U_Lb = b + offs[i++]; T.U_invd = b + offs[i++];
  T.gram = b + offs[i++];
  T.twn = reinterpret_cast<const double2*>(b + offs[i++]);
  T.Vn = b + offs[i++];
  T.Vn1 = b + offs[i++];
  T.Wn = b + offs[i++];
  T.dtae = b + offs[i++];
  T.zinv32 = reinterpret_cast<const float*>(b + offs[i++]);
  T.zfwd32 = reinterpret_cast<const float*>(b + offs[i++]);
  T.tw32 = reinterpret_cast<const float2*>(b + offs[i++]);
  T.T_inv = dense ? b + offs[i] : nullptr;
  ++i;
  T.P_inv = dense ? b + offs[i] : nullptr;
  ++i;
  T.U_inv = dense ? b + offs[i] : nullptr;
  ++i;
  T.tcA_psi_hi = tc ? reinterpret_cast<const float*>(b + offs[i]) : nullptr;
  ++i;
  T.tcA_psi_lo = tc ? reinterpret_cast<const float*>(b + offs[i]) : nullptr;
  ++i;
  T.tcA_T_hi = tc ? reinterpret_cast<const float*>(b + offs[i]) : nullptr;
  ++i;
  T.tcA_T_lo = tc ? reinterpret_cast<const float*>(b + offs[i]) : nullptr;
  ++i;
  for (int p = 0; p < 2; ++p) {
    T.tcW_hi[p] = tcw ? reinterpret_cast<const float*>(b + offs[i]) : nullptr;
    ++i;
    T.tcW_lo[p] = tcw ? reinterpret_cast<const float*>(b + offs[i]) : nullptr;
    ++i;
  }
  return RBC_OK;
}

extern "C" rbc_status rbc_create(double Ra, double Pr, double Lx, int Nx, int Nz, double dt, const rbc_opts* opts,
                                 rbc_t* out) {
  if (!out) return fail(RBC_EINVAL, "out is NULL");
  *out = nullptr;
  if (Nx < 4 || Nx > 1024 || (Nx & 1) || Nz < 8 || Nz > 512 || (Nz & 1))
    return fail(RBC_EINVAL, "need even Nx in [4, 1024] and even Nz in [8, 512]");
  if (!(dt > 0) || !(Pr > 0) || !(Lx > 0) || !(Ra >= 0) || !std::isfinite(Ra) || !std::isfinite(dt))
    return fail(RBC_EINVAL, "need dt > 0, Pr > 0, Lx > 0, Ra >= 0");
  rbc_opts o{RBC_FP64, RBC_FIXED_T, 0, RBC_RK443};
  if (opts) o = *opts;
  if (o.eager != 0 && o.eager != 1) return fail(RBC_EINVAL, "eager must be 0 or 1");
  if (o.precision != RBC_FP64 && o.precision != RBC_MIXED && o.precision != RBC_MIXED_BF16)
    return fail(RBC_EINVAL, "precision mode %d not available", o.precision);
  if (o.bc != RBC_FIXED_T && o.bc != RBC_FIXED_FLUX) return fail(RBC_EINVAL, "boundary condition %d not available", o.bc);
  if (o.scheme != RBC_RK443 && o.scheme != RBC_RK222 && o.scheme != RBC_RK111)
    return fail(RBC_EINVAL, "time-stepping scheme %d not available", o.scheme);
  // padded x length 3 Nx / 2 must be 3 * 2^p for the FFT
  int Mx = 3 * Nx / 2, r = Mx / 3;
  if (Mx % 3 || (r & (r - 1))) return fail(RBC_EINVAL, "Nx must be a power of two (3/2-padded FFT length 3*2^p)");
  rbc_t h = new (std::nothrow) rbc_s();
  if (!h) return fail(RBC_ENOMEM, "host allocation");
  h->opts = o;
  h->profp = &h->prof;
  h->tunep = &h->tuning;
  h->use_graphs = (o.eager == 0);
  cudaGetDevice(&h->device);
  Grid& g = h->g;
  g.Nx = Nx;
  g.Nz = Nz;
  g.nm = Nx / 2;
  g.Mx = Mx;
  g.Mz = 3 * Nz / 2;
  g.nq = Nz / 2;
  g.Ra = Ra;
  g.Pr = Pr;
  g.Lx = Lx;
  g.dt = dt;
  g.kfac = 2.0 * M_PI / Lx;
  g.mixed = (o.precision == RBC_MIXED || o.precision == RBC_MIXED_BF16) ? 1 : 0;
  g.tcbf16 = (o.precision == RBC_MIXED_BF16) ? 1 : 0;
  g.bc = o.bc;
  g.scheme = o.scheme;
  {
    double ae[5][5], ai[5][5];
    scheme_tableau(o.scheme, ae, ai, &g.ns, &g.gamma);
    g.inv_gamma = 1.0 / g.gamma;
  }
  rbc_status s = upload_tables(h);
  if (s == RBC_OK) {
    cudaError_t e = configure_kernels(g);
    if (e == cudaSuccess) e = upload_schemes();
    if (e != cudaSuccess) s = fail(RBC_ECUDA, "configure: %s", cudaGetErrorString(e));
  }
  if (s == RBC_OK) {
    const size_t scratch = (size_t)3 * Nz * Nx + (size_t)3 * Nz * g.nm * 2 + 64;
    if (cudaMalloc(&h->d_scratch, scratch * sizeof(double)) != cudaSuccess) s = fail(RBC_ENOMEM, "scratch");
  }
  if (s != RBC_OK) {
    rbc_destroy(h);
    return s;
  }
  *out = h;
  return RBC_OK;
}

extern "C" void rbc_destroy(rbc_t h) {
  if (!h) return;
  for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
  for (auto& sg : h->graphs)
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
  for (auto& c : h->caps)
    if (c.s) cudaStreamDestroy(c.s);
  for (int i = 0; i < rbc_s::kPinSlots; ++i) {
    if (h->pin_busy[i]) cudaEventSynchronize(h->pin_ev[i]);
    if (h->pin_ev[i]) cudaEventDestroy(h->pin_ev[i]);
  }
  cudaFreeHost(h->pin);
  cudaFree(h->d_tables);
  cudaFree(h->d_work);
  cudaFree(h->d_scratch);
  cudaFree(h->d_sbuf);
  delete h;
}

extern "C" size_t rbc_state_bytes(rbc_t h) { return h ? state_doubles(h->g) * sizeof(double) : 0; }

static size_t work_doubles_per_state(const Grid& g) {
  const size_t S = state_doubles(g);
  return 6 * S + z_doubles(g) + q_doubles(g) + g.Mz + 5;   // Xs, F, R[4], Z, Q, wT, ints + nu + Ra
}

extern "C" size_t rbc_workspace_bytes_per_state(rbc_t h) {
  return h ? work_doubles_per_state(h->g) * sizeof(double) : 0;
}

extern "C" rbc_status rbc_reserve(rbc_t h, int B) {
  if (!h || B < 0) return fail(RBC_EINVAL, "bad handle or B");
  if (B <= h->cap) return RBC_OK;
  const Grid& g = h->g;
  const size_t S = state_doubles(g);
  const size_t tot = (size_t)B * work_doubles_per_state(g) + 80;
  void* p = nullptr;
  if (cudaMalloc(&p, tot * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(RBC_ENOMEM, "workspace for %d states (%zu bytes)", B, tot * sizeof(double));
  }
  cudaFree(h->d_work);
  h->d_work = p;
  h->cap = B;
  for (auto& sg : h->graphs) {   // bound to the old workspace
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    sg = rbc_s::StepGraph{};
  }
  h->up_ns.clear();
  h->up_ra.clear();
  double* d = static_cast<double*>(p);
  Work& w = h->w;
  w.Xs = d; d += (size_t)B * S;
  w.F = d; d += (size_t)B * S;
  w.R = d; d += (size_t)B * 4 * S;
  w.Z = d; d += (size_t)B * z_doubles(g);
  w.Q = d; d += (size_t)B * q_doubles(g);
  w.wT = d; d += (size_t)B * g.Mz;
  w.nu = d; d += B;
  w.ra = d; d += B;
  w.small = d; d += 16;
  int* ip = reinterpret_cast<int*>(d);
  w.maxs = ip; ip += 1;
  w.nsteps = ip; ip += B;
  w.flags = ip; ip += B;
  w.step = ip; ip += 1;
  w.err = ip; ip += 1;
  w.dflag = ip; ip += 1;
  // the counters start defined: an unset loop bound reads 0 (one step), never garbage
  if (cudaMemset(w.maxs, 0, (size_t)(ip - w.maxs) * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(RBC_ECUDA, "workspace counters");
  }
  w.prof = h->profp;
  return RBC_OK;
}

extern "C" rbc_status rbc_profile(rbc_t h, int enable) {
  if (!h) return fail(RBC_EINVAL, "null handle");
  Prof& p = h->prof;
  if (enable < 0 || enable > 2) return fail(RBC_EINVAL, "profile mode %d", enable);
  if (enable) {
    CK(p.fold());
    for (int k = 0; k < RBC_NKERNELS; ++k) {
      p.ms[k] = p.flops[k] = p.bytes[k] = 0.0;
      p.launches[k] = 0;
    }
  }
  p.on = enable != 0;
  p.once = enable == 2;
  return RBC_OK;
}

extern "C" rbc_status rbc_profile_read(rbc_t h, double ms[4], long long launches[4], double flops[4],
                                       double bytes[4]) {
  if (!h) return fail(RBC_EINVAL, "null handle");
  Prof& p = h->prof;
  CK(p.fold());
  for (int k = 0; k < RBC_NKERNELS; ++k) {
    if (ms) ms[k] = p.ms[k];
    if (launches) launches[k] = p.launches[k];
    if (flops) flops[k] = p.flops[k];
    if (bytes) bytes[k] = p.bytes[k];
  }
  return RBC_OK;
}

extern "C" unsigned long long rbc_launch_count(void) { return launches_so_far(); }

extern "C" rbc_status rbc_set_state(rbc_t h, void* d_state, const double* h_T, const double* h_u, const double* h_w) {
  if (!h || !d_state || !h_T) return fail(RBC_EINVAL, "null argument");
  const Grid& g = h->g;
  const size_t n = (size_t)g.Nz * g.Nx;
  double* gd = h->d_scratch;
  double* modes = gd + 3 * n;
  CK(cudaMemcpy(gd, h_T, n * sizeof(double), cudaMemcpyHostToDevice));
  if (h_u) CK(cudaMemcpy(gd + n, h_u, n * sizeof(double), cudaMemcpyHostToDevice));
  else CK(cudaMemset(gd + n, 0, n * sizeof(double)));
  if (h_w) CK(cudaMemcpy(gd + 2 * n, h_w, n * sizeof(double), cudaMemcpyHostToDevice));
  else CK(cudaMemset(gd + 2 * n, 0, n * sizeof(double)));
  CK(launch_set_state(g, h->t, gd, gd + n, gd + 2 * n, modes, static_cast<double*>(d_state), 0));
  CK(cudaStreamSynchronize(0));
  return RBC_OK;
}

extern "C" rbc_status rbc_get_state(rbc_t h, const void* d_state, double* h_T, double* h_u, double* h_w) {
  if (!h || !d_state) return fail(RBC_EINVAL, "null argument");
  const Grid& g = h->g;
  const size_t n = (size_t)g.Nz * g.Nx;
  double* gd = h->d_scratch;
  double* modes = gd + 3 * n;
  CK(launch_get_state(g, h->t, static_cast<const double*>(d_state), modes, gd, gd + n, gd + 2 * n, 0));
  CK(cudaStreamSynchronize(0));
  if (h_T) CK(cudaMemcpy(h_T, gd, n * sizeof(double), cudaMemcpyDeviceToHost));
  if (h_u) CK(cudaMemcpy(h_u, gd + n, n * sizeof(double), cudaMemcpyDeviceToHost));
  if (h_w) CK(cudaMemcpy(h_w, gd + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost));
  return RBC_OK;
}

// The step loop of this (states, B, nu) binding: a while node whose body is
// one RK443 step captured on the handle's own stream, ended by the counter
// kernel once step == maxs.  Cached per binding.
// Drop the step graphs and the capture stream a handle holds in `ctx`.
static void release_context(rbc_t h, CUcontext ctx) {
  if (!h || !ctx) return;
  for (auto& sg : h->graphs)
    if (sg.exec && sg.ctx == ctx) {
      cudaGraphExecDestroy(sg.exec);
      sg = rbc_s::StepGraph{};
    }
  for (auto& c : h->caps)
    if (c.s && c.ctx == ctx) {
      cudaStreamSynchronize(c.s);
      cudaStreamDestroy(c.s);
      c = rbc_s::CapStream{};
    }
  if (h->bind_ctx == ctx) h->bind_ctx = nullptr;
}

static rbc_status capture_stream(rbc_t h, cudaStream_t* out) {
  rbc_s::CapStream* free_slot = nullptr;
  for (auto& c : h->caps) {
    if (c.s && c.ctx == h->bind_ctx) {
      *out = c.s;
      return RBC_OK;
    }
    if (!c.s && !free_slot) free_slot = &c;
  }
  if (!free_slot) return fail(RBC_ECUDA, "no free capture stream slot");
  CtxScope scope(h->bind_ctx);
  if (!scope.ok()) return fail(RBC_ECUDA, "cannot enter the SM partition's context");
  CK(cudaStreamCreateWithFlags(&free_slot->s, cudaStreamNonBlocking));
  free_slot->ctx = h->bind_ctx;
  *out = free_slot->s;
  return RBC_OK;
}

static rbc_status step_graph(rbc_t h, double* X, int B, double* nu, cudaGraphExec_t* out) {
  ++h->graph_clock;
  rbc_s::StepGraph* victim = &h->graphs[0];
  for (auto& sg : h->graphs) {
    if (sg.exec && sg.X == X && sg.B == B && sg.nu == nu && sg.ctx == h->bind_ctx && sg.tune_gen == h->tunep->gen) {
      sg.used = h->graph_clock;
      *out = sg.exec;
      return RBC_OK;
    }
    if (!sg.exec || sg.used < victim->used) victim = &sg;
  }
  if (victim->exec) cudaGraphExecDestroy(victim->exec);
  *victim = rbc_s::StepGraph{};
  cudaStream_t cap = nullptr;
  rbc_status cs = capture_stream(h, &cap);
  if (cs != RBC_OK) return cs;
  // the graph, its loop handle and the captured kernels belong to the
  // handle's SM partition when it is bound to one
  CtxScope scope(h->bind_ctx);
  if (!scope.ok()) return fail(RBC_ECUDA, "cannot enter the SM partition's context");
  cudaGraph_t gr = nullptr;
  CK(cudaGraphCreate(&gr, 0));
  cudaGraphConditionalHandle loop;
  cudaError_t e = cudaGraphConditionalHandleCreate(&loop, gr, 1u, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, gr, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(gr);
    return fail(RBC_ECUDA, "step loop node: %s", cudaGetErrorString(e));
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const unsigned long long before = launches_so_far();
  e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int stage = 1; stage <= h->g.ns && e == cudaSuccess; ++stage)
      e = launch_stage(h->g, h->t, h->w, X, B, stage, nu, cap);
    if (e == cudaSuccess) e = launch_advance_loop(h->w, loop, cap);
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &captured);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(gr);
    return fail(RBC_ECUDA, "step loop capture: %s", cudaGetErrorString(e));
  }
  if (launches_so_far() - before != (unsigned long long)step_kernels(h->g)) {
    cudaGraphDestroy(gr);
    return fail(RBC_ECUDA, "step graph: unexpected kernel count");
  }
  add_launches(~0ull - (unsigned long long)step_kernels(h->g) + 1ull);   // captured, not executed
  e = cudaGraphInstantiate(&victim->exec, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) {
    victim->exec = nullptr;
    return fail(RBC_ECUDA, "step graph instantiate: %s", cudaGetErrorString(e));
  }
  victim->X = X;
  victim->B = B;
  victim->nu = nu;
  victim->ctx = h->bind_ctx;
  victim->tune_gen = h->tunep->gen;
  victim->used = h->graph_clock;
  *out = victim->exec;
  return RBC_OK;
}

// Copy the per-state step counts (and their maximum) and Rayleigh numbers
// into the workspace, through a pinned slot of the handle's ring.
static rbc_status upload_steps(rbc_t h, int B, const int* h_nsteps, const double* h_ra, int maxs,
                               cudaStream_t stream) {
  const Work& w = h->w;
  const size_t need = ((size_t)B * (sizeof(double) + sizeof(int)) + sizeof(int) + 255) & ~(size_t)255;
  if (need > h->pin_slot) {
    for (int i = 0; i < rbc_s::kPinSlots; ++i) {
      if (h->pin_busy[i]) CK(cudaEventSynchronize(h->pin_ev[i]));
      h->pin_busy[i] = false;
    }
    cudaFreeHost(h->pin);
    h->pin = nullptr;
    h->pin_slot = 0;
    if (cudaMallocHost(&h->pin, need * rbc_s::kPinSlots) != cudaSuccess) {
      cudaGetLastError();
      h->pin = nullptr;
      return fail(RBC_ENOMEM, "pinned staging for %d states", B);
    }
    h->pin_slot = need;
  }
  const int slot = h->pin_next;
  h->pin_next = (slot + 1) % rbc_s::kPinSlots;
  if (!h->pin_ev[slot]) CK(cudaEventCreateWithFlags(&h->pin_ev[slot], cudaEventDisableTiming));
  if (h->pin_busy[slot]) CK(cudaEventSynchronize(h->pin_ev[slot]));
  double* pin_ra = reinterpret_cast<double*>(h->pin + slot * h->pin_slot);
  int* pin_ns = reinterpret_cast<int*>(pin_ra + B);   // [maxs][nsteps B], as w.maxs, w.nsteps
  pin_ns[0] = maxs;
  for (int b = 0; b < B; ++b) {
    pin_ra[b] = h_ra ? h_ra[b] : h->g.Ra;
    pin_ns[1 + b] = h_nsteps[b];
  }
  static_assert(sizeof(int) == 4, "int layout");
  CK(cudaMemcpyAsync(w.ra, pin_ra, (size_t)B * sizeof(double), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(w.maxs, pin_ns, (size_t)(B + 1) * sizeof(int), cudaMemcpyHostToDevice, stream));
  CK(cudaEventRecord(h->pin_ev[slot], stream));
  h->pin_busy[slot] = true;
  h->up_ns.assign(pin_ns + 1, pin_ns + 1 + B);
  h->up_ns.push_back(maxs);
  h->up_ra.assign(pin_ra, pin_ra + B);
  return RBC_OK;
}

static rbc_status step_batch(rbc_t h, void* d_states, int B, const int* h_nsteps, const double* h_ra,
                             double* d_nu_integral, cudaStream_t stream) {
  if (!h || B < 0 || (B > 0 && (!d_states || !h_nsteps))) return fail(RBC_EINVAL, "null argument or B < 0");
  if (B == 0) return RBC_OK;
  int maxs = 0;
  for (int b = 0; b < B; ++b) {
    if (h_nsteps[b] < 0) return fail(RBC_EINVAL, "negative step count");
    maxs = std::max(maxs, h_nsteps[b]);
    if (h_ra && !(h_ra[b] >= 0 && std::isfinite(h_ra[b]))) return fail(RBC_EINVAL, "Rayleigh number must be >= 0");
  }
  rbc_status s = rbc_reserve(h, B);
  if (s != RBC_OK) return s;
  const Work& w = h->w;
  double* X = static_cast<double*>(d_states);
  double* nu = d_nu_integral ? d_nu_integral : w.nu;
  bool same = (int)h->up_ns.size() == B + 1 && h->up_ns[B] == maxs;
  for (int b = 0; same && b < B; ++b)
    same = h->up_ns[b] == h_nsteps[b] && h->up_ra[b] == (h_ra ? h_ra[b] : h->g.Ra);
  if (!same) {
    rbc_status us = upload_steps(h, B, h_nsteps, h_ra, maxs, stream);
    if (us != RBC_OK) return us;
  }
  {
    auto it = h->tunep->byB.find(B);
    h->w.shapes = it == h->tunep->byB.end() ? nullptr : &it->second;
  }
  h->w.pdl = B <= kPdlMaxBatch ? 1 : 0;
  CK(cudaMemsetAsync(w.step, 0, sizeof(int), stream));
  CK(cudaMemsetAsync(w.flags, 0, (size_t)B * sizeof(int), stream));
  CK(cudaMemsetAsync(nu, 0, (size_t)B * sizeof(double), stream));
  h->last_B = B;
  // Steps launched one kernel at a time: all of them while profiling every
  // call; the first kProfileSampleSteps of a sampled call (the rest continue
  // on the graph loop from the same device step counter); none otherwise.
  Prof& pr = *h->profp;
  const int eager = !pr.on ? 0 : pr.once ? std::min(maxs, kProfileSampleSteps) : maxs;
  for (int st = 0; st < eager; ++st) {
    for (int stage = 1; stage <= h->g.ns; ++stage) CK(launch_stage(h->g, h->t, w, X, B, stage, nu, stream));
    CK(launch_advance(w, stream));
  }
  if (pr.once) pr.on = false;
  const int rest = maxs - eager;
  if (rest >= 2 && h->use_graphs) {
    cudaGraphExec_t ex = nullptr;
    rbc_status gs = step_graph(h, X, B, nu, &ex);
    if (gs != RBC_OK) return gs;
    CK(cudaGraphLaunch(ex, stream));
    add_launches((unsigned long long)rest * step_kernels(h->g));
  } else {
    for (int st = 0; st < rest; ++st) {
      for (int stage = 1; stage <= h->g.ns; ++stage) CK(launch_stage(h->g, h->t, w, X, B, stage, nu, stream));
      CK(launch_advance(w, stream));
    }
  }
  if (maxs > 0) CK(launch_nu_final(h->g, h->t, w, X, B, nu, stream));
  if (pr.once) pr.on = pr.once = false;   // sampled profiling: this call only (its first steps)
  return RBC_OK;
}

extern "C" rbc_status rbc_step_batch(rbc_t h, void* d_states, int B, const int* h_nsteps, double* d_nu_integral,
                                     cudaStream_t stream) {
  return step_batch(h, d_states, B, h_nsteps, nullptr, d_nu_integral, stream);
}

extern "C" rbc_status rbc_step_batch_ra(rbc_t h, void* d_states, int B, const int* h_nsteps, const double* h_ra,
                                        double* d_nu_integral, cudaStream_t stream) {
  if (!h_ra) return fail(RBC_EINVAL, "h_ra is NULL");
  return step_batch(h, d_states, B, h_nsteps, h_ra, d_nu_integral, stream);
}

static bool compatible(rbc_t fine, rbc_t coarse) {
  return fine && coarse && coarse->g.Nx <= fine->g.Nx && coarse->g.Nz <= fine->g.Nz && coarse->g.bc == fine->g.bc;
}

extern "C" rbc_status rbc_restrict(rbc_t fine, rbc_t coarse, const void* d_fine, void* d_coarse, int B,
                                   cudaStream_t stream) {
  if (!compatible(fine, coarse) || B < 0 || (B > 0 && (!d_fine || !d_coarse)))
    return fail(RBC_EINVAL, "bad handles, buffers or B");
  CK(launch_restrict(fine->g, coarse->g, static_cast<const double*>(d_fine), static_cast<double*>(d_coarse), B,
                     stream));
  return RBC_OK;
}

extern "C" rbc_status rbc_prolong(rbc_t fine, rbc_t coarse, const void* d_coarse, void* d_fine, int B,
                                  cudaStream_t stream) {
  if (!compatible(fine, coarse) || B < 0 || (B > 0 && (!d_fine || !d_coarse)))
    return fail(RBC_EINVAL, "bad handles, buffers or B");
  CK(launch_prolong(fine->g, coarse->g, static_cast<const double*>(d_coarse), static_cast<double*>(d_fine), B,
                    stream));
  return RBC_OK;
}

extern "C" rbc_status rbc_parareal_correct(rbc_t fine, rbc_t coarse, const void* d_F, const void* d_Gnew,
                                           const void* d_Gold, void* d_U, int B, cudaStream_t stream) {
  if (!compatible(fine, coarse) || B < 0 || (B > 0 && (!d_F || !d_Gnew || !d_Gold || !d_U)))
    return fail(RBC_EINVAL, "bad handles, buffers or B");
  CK(launch_correct(fine->g, coarse->g, static_cast<const double*>(d_F), static_cast<const double*>(d_Gnew),
                    static_cast<const double*>(d_Gold), static_cast<double*>(d_U), B, stream));
  return RBC_OK;
}

extern "C" rbc_status rbc_l2_diff(rbc_t h, const void* d_A, const void* d_B, int B, double* d_out,
                                  cudaStream_t stream) {
  if (!h || B < 0 || (B > 0 && (!d_A || !d_out))) return fail(RBC_EINVAL, "null argument or B < 0");
  CK(launch_l2_diff(h->g, h->t, static_cast<const double*>(d_A), static_cast<const double*>(d_B), B, d_out, stream));
  return RBC_OK;
}

// Error bits of the handle: the per-state flags of the last rbc_step_batch
// call OR-ed with the sticky bits of every call since the last read, which
// are cleared.  Synchronises `stream`.
static rbc_status read_errors(rbc_t h, cudaStream_t stream, int* bits) {
  *bits = 0;
  CK(cudaStreamSynchronize(stream));
  if (h->cap == 0) return RBC_OK;
  std::vector<int> f((size_t)h->last_B + 1, 0);
  if (h->last_B > 0) CK(cudaMemcpy(f.data(), h->w.flags, (size_t)h->last_B * sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&f[h->last_B], h->w.err, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemset(h->w.err, 0, sizeof(int)));
  for (int v : f) *bits |= v;
  return RBC_OK;
}

static rbc_status status_of_bits(int bits) {
  if (bits & kFlagTimeout) return fail(RBC_ETIMEOUT, "a bounded device-side wait gave up");
  if (bits & kFlagNonFinite) return fail(RBC_EDIVERGED, "non-finite state");
  return RBC_OK;
}

extern "C" rbc_status rbc_check_diverged(rbc_t h, cudaStream_t stream) {
  if (!h) return fail(RBC_EINVAL, "null handle");
  int bits = 0;
  rbc_status s = read_errors(h, stream, &bits);
  return s != RBC_OK ? s : status_of_bits(bits);
}

extern "C" rbc_status rbc_set_wait_limit(long long polls) {
  CK(tc_set_wait_limit(polls));
  return RBC_OK;
}

extern "C" rbc_status rbc_nusselt(rbc_t h, const void* d_state, double out[3], cudaStream_t stream) {
  if (!h || !d_state || !out) return fail(RBC_EINVAL, "null argument");
  rbc_status s = rbc_reserve(h, 1);
  if (s != RBC_OK) return s;
  Work w = h->w;   // the call's own error bits, apart from the batch's
  w.flags = w.err = h->w.dflag;
  CK(cudaMemsetAsync(w.dflag, 0, sizeof(int), stream));
  CK(launch_nusselt(h->g, h->t, w, static_cast<const double*>(d_state), w.small, stream));
  int bits = 0;
  CK(cudaMemcpyAsync(out, w.small, 3 * sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaMemcpyAsync(&bits, w.dflag, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  return status_of_bits(bits);
}

extern "C" rbc_status rbc_nusselt_static(rbc_t h, const void* d_state, double out[3], cudaStream_t stream) {
  if (!h || !d_state || !out) return fail(RBC_EINVAL, "null argument");
  const size_t need = static_scratch_doubles_needed(h->g);
  if (need > kStaticScratchCapacity)
    return fail(RBC_EINVAL, "grid %dx%d needs %zu doubles of scratch; the static array holds %zu (3 MiB)",
                h->g.Nx, h->g.Nz, need, kStaticScratchCapacity);
  int bits = 0;
  CK(launch_nusselt_static(h->g, h->t, static_cast<const double*>(d_state), out, &bits, stream));
  return status_of_bits(bits);
}

extern "C" size_t rbc_diag_size(rbc_t h) { return h ? (size_t)6 + 2 * (size_t)h->g.Mz : 0; }

extern "C" rbc_status rbc_diagnostics(rbc_t h, const void* d_states, int B, double* d_out, cudaStream_t stream) {
  if (!h || B < 0 || (B > 0 && (!d_states || !d_out))) return fail(RBC_EINVAL, "null argument or B < 0");
  if (B == 0) return RBC_OK;
  rbc_status s = rbc_reserve(h, B);
  if (s != RBC_OK) return s;
  CK(launch_diagnostics(h->g, h->t, h->w, static_cast<const double*>(d_states), B, d_out, stream));
  return RBC_OK;
}

// Device time (ms) of `steps` RK443 steps of the B states X, launched kernel by
// kernel with the shapes `sh` (after one untimed step).
static rbc_status time_shapes(rbc_t h, double* X, int B, const Shapes& sh, int steps, cudaStream_t s, float* ms) {
  Work w = h->w;
  w.shapes = &sh;
  w.prof = nullptr;
  std::vector<int> ns(B, steps + 1);
  CK(cudaMemcpyAsync(w.nsteps, ns.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(w.step, 0, sizeof(int), s));
  CK(cudaMemsetAsync(w.flags, 0, (size_t)B * sizeof(int), s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaSuccess;
  for (int st = 0; st <= steps && e == cudaSuccess; ++st) {
    if (st == 1) e = cudaEventRecord(e0, s);
    for (int stage = 1; stage <= h->g.ns && e == cudaSuccess; ++stage) e = launch_stage(h->g, h->t, w, X, B, stage, w.nu, s);
    if (e == cudaSuccess) e = launch_advance(w, s);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(e);
  return RBC_OK;
}

extern "C" rbc_status rbc_autotune(rbc_t h, int B, double out_ms[2], cudaStream_t stream) {
  if (!h || B < 1) return fail(RBC_EINVAL, "null handle or B < 1");
  rbc_status s = rbc_reserve(h, B);
  if (s != RBC_OK) return s;
  const Grid& g = h->g;
  const size_t es = g.mixed ? 4 : 8;
  // a batch of conduction states (finite, and the timing does not depend on the values)
  double* X = nullptr;
  if (cudaMalloc(&X, (size_t)B * state_doubles(g) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(RBC_ENOMEM, "autotune states");
  }
  struct Free {
    double* p;
    ~Free() { cudaFree(p); }
  } fr{X};
  CK(cudaMemsetAsync(X, 0, (size_t)B * state_doubles(g) * sizeof(double), stream));
  CK(cudaMemsetAsync(h->w.ra, 0, (size_t)B * sizeof(double), stream));
  h->up_ns.clear();   // the step counts and Rayleigh numbers on the device are
  h->up_ra.clear();   // overwritten: the next rbc_step_batch uploads its own
  const int steps = 3;
  Shapes best;   // the heuristics
  float t_best = 0.f;
  s = time_shapes(h, X, B, best, steps, stream, &t_best);
  if (s != RBC_OK) return s;
  const float t_heur = t_best;
  // coordinate search: row kernel form, then z-forward tile and chunks, then solve tile
  auto trial = [&](Shapes c) -> rbc_status {
    if (!shapes_valid(g, c, es)) return RBC_OK;
    float t = 0.f;
    rbc_status r = time_shapes(h, X, B, c, steps, stream, &t);
    if (r != RBC_OK) return r;
    if (t < t_best) {
      t_best = t;
      best = c;
    }
    return RBC_OK;
  };
  for (int cl = 0; cl <= 1; ++cl) {
    Shapes c = best;
    c.rows_cl = cl;
    if ((s = trial(c)) != RBC_OK) return s;
  }
  for (int th = 512; th <= 1024; th *= 2) {   // block size of the one-block-per-row kernel
    Shapes c = best;
    c.rows_threads = th;
    if ((s = trial(c)) != RBC_OK) return s;
  }
  for (int ln = 0; ln <= 1; ++ln) {             // its shared-memory layout
    Shapes c = best;
    c.rows_lean = ln;
    if ((s = trial(c)) != RBC_OK) return s;
  }
  for (int tm = 4; tm <= 32; tm *= 2)
    for (int nch = 1; nch <= 8; nch *= 2) {
      Shapes c = best;
      c.zfwd_tm = tm;
      c.zfwd_nch = nch;
      if ((s = trial(c)) != RBC_OK) return s;
    }
  for (int tms = 1; tms <= 16; tms *= 2) {
    Shapes c = best;
    c.solve_tms = tms;
    if ((s = trial(c)) != RBC_OK) return s;
  }
  h->tunep->byB[B] = best;
  h->tunep->gen++;
  if (out_ms) {
    out_ms[0] = t_heur / steps;
    out_ms[1] = t_best / steps;
  }
  return RBC_OK;
}

extern "C" rbc_status rbc_tuned_shapes(rbc_t h, int B, int out[6]) {
  if (!h || !out) return fail(RBC_EINVAL, "null argument");
  const auto it = h->tunep->byB.find(B);
  const Shapes sh = it == h->tunep->byB.end() ? Shapes{} : it->second;
  out[0] = sh.solve_tms;
  out[1] = sh.zfwd_tm;
  out[2] = sh.zfwd_nch;
  out[3] = sh.rows_cl;
  out[4] = sh.rows_threads;
  out[5] = sh.rows_lean;
  return RBC_OK;
}

extern "C" rbc_status rbc_set_shapes(rbc_t h, int B, const int in[6]) {
  if (!h || !in || B < 1) return fail(RBC_EINVAL, "null argument or B < 1");
  Shapes sh;
  sh.solve_tms = in[0];
  sh.zfwd_tm = in[1];
  sh.zfwd_nch = in[2];
  sh.rows_cl = in[3];
  sh.rows_threads = in[4];
  sh.rows_lean = in[5];
  if (sh.solve_tms < 0 || sh.zfwd_tm < 0 || sh.zfwd_nch < 0 || sh.rows_cl < -1 || sh.rows_cl > 1 ||
      sh.rows_threads < 0 || !shapes_valid(h->g, sh, h->g.mixed ? 4 : 8))
    return fail(RBC_EINVAL, "launch shapes not valid for this grid");
  h->tunep->byB[B] = sh;
  h->tunep->gen++;
  return RBC_OK;
}

// Buffers of a sampled run of B states (grown on demand, as the workspace).
static rbc_status reserve_sampling(rbc_t h, int B) {
  if (B <= h->sbuf_cap) return RBC_OK;
  const size_t D = 6 + 2 * (size_t)h->g.Mz;
  void* p = nullptr;
  if (cudaMalloc(&p, (size_t)B * (2 * D + 1) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(RBC_ENOMEM, "sampling buffers for %d states", B);
  }
  cudaFree(h->d_sbuf);
  h->d_sbuf = static_cast<double*>(p);
  h->sbuf_cap = B;
  return RBC_OK;
}

extern "C" rbc_status rbc_step_batch_sampled(rbc_t h, void* d_states, int B, int nsteps, int every,
                                             double* d_nu_integral, double* d_stat, cudaStream_t stream) {
  if (!h || B < 0 || nsteps < 0 || every < 1 || (B > 0 && (!d_states || !d_stat)))
    return fail(RBC_EINVAL, "null argument, B < 0, nsteps < 0 or every < 1");
  if (B == 0) return RBC_OK;
  rbc_status s = rbc_reserve(h, B);
  if (s == RBC_OK) s = reserve_sampling(h, B);
  if (s != RBC_OK) return s;
  const Grid& g = h->g;
  const long D = 6 + 2 * (long)g.Mz;
  double* X = static_cast<double*>(d_states);
  double* prev = h->d_sbuf;
  double* cur = prev + (size_t)B * D;
  double* nuc = cur + (size_t)B * D;
  CK(cudaMemsetAsync(d_stat, 0, (size_t)B * D * sizeof(double), stream));
  if (d_nu_integral) CK(cudaMemsetAsync(d_nu_integral, 0, (size_t)B * sizeof(double), stream));
  CK(launch_diagnostics(g, h->t, h->w, X, B, prev, stream));
  CK(launch_stat_sample(g, prev, B, stream));
  std::vector<int> ns(B, 0);
  for (int done = 0; done < nsteps;) {
    const int c = std::min(every, nsteps - done);
    std::fill(ns.begin(), ns.end(), c);
    s = rbc_step_batch(h, X, B, ns.data(), nuc, stream);
    if (s != RBC_OK) return s;
    if (d_nu_integral) CK(launch_add(d_nu_integral, nuc, B, stream));
    CK(launch_diagnostics(g, h->t, h->w, X, B, cur, stream));
    CK(launch_stat_sample(g, cur, B, stream));
    CK(launch_stat_accum(d_stat, prev, cur, 0.5 * (c * g.dt), (long)B * D, stream));
    done += c;
  }
  return RBC_OK;
}

// Time means and the checks of Sec. 2.2 from window means of the sampled
// quantities (see include/rbc.h for the layout of both arrays).
extern "C" rbc_status rbc_stat_summary(int Nz, double Ra, double Pr, const double* means, double* out) {
  if (!means || !out || Nz < 8 || (Nz & 1) || !(Pr > 0)) return fail(RBC_EINVAL, "bad arguments");
  const int Mz = 3 * Nz / 2;
  const double U = means[0], eps = means[1], wT = means[2], NuV = means[3], Nub = means[4], Nut = means[5];
  const double* Tm = means + 6;
  const double* T2 = means + 6 + Mz;
  const double P = Ra * wT, epsU = std::fabs(eps);
  out[0] = U;
  out[1] = U / Pr;                                                               // Re
  out[2] = NuV;
  out[3] = Nub;
  out[4] = Nut;
  out[5] = std::max(std::fabs(Nub - NuV), std::max(std::fabs(Nub - Nut), std::fabs(NuV - Nut))) / NuV;   // Nu_int
  out[6] = P;
  out[7] = epsU;
  out[8] = P != 0.0 ? std::fabs(P - epsU) / P : NAN;                            // |P - eps_U| / P
  out[9] = 0.5 / NuV;                                                           // delta_t = 1 / (2 Nu)
  // T_rms at the padded points z_j = cos(pi j / (Mz - 1)) / 2 (descending), its
  // peak over the lower half from the bottom wall up (the first maximum), and
  // the interior native Lobatto points no farther from the wall than it
  double* Trms = out + 12;
  for (int j = 0; j < Mz; ++j) Trms[j] = std::sqrt(std::max(T2[j] - Tm[j] * Tm[j], 0.0));
  double best = 0.0, delta = NAN;
  for (int j = Mz - 1; j >= 0; --j) {
    const double z = 0.5 * std::cos(M_PI * j / (Mz - 1));
    if (!(z < 0.0)) continue;
    if (Trms[j] > best) {
      best = Trms[j];
      delta = z + 0.5;
    }
  }
  int nbl = 0;
  if (best > 0.0)
    for (int j = 1; j < Nz - 1; ++j)
      if (0.5 - 0.5 * std::cos(M_PI * j / (Nz - 1)) <= delta) ++nbl;
  out[10] = best > 0.0 ? delta : NAN;                                           // delta_T
  out[11] = nbl;                                                                // N_BL
  return RBC_OK;
}

extern "C" rbc_status rbc_l2_temperature(rbc_t h, const void* d_state, double* out, cudaStream_t stream) {
  if (!h || !d_state || !out) return fail(RBC_EINVAL, "null argument");
  rbc_status s = rbc_reserve(h, 1);
  if (s != RBC_OK) return s;
  CK(launch_l2_diff(h->g, h->t, static_cast<const double*>(d_state), nullptr, 1, h->w.small, stream));
  double v = 0.0;
  CK(cudaMemcpyAsync(&v, h->w.small, sizeof(double), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  *out = std::sqrt(v);
  return RBC_OK;
}

// ---------------------------------------------------------------------------
// Parareal (Sec. 3.1, Eq. 20).
// ---------------------------------------------------------------------------
static bool whole_steps(double len, double dt, int* n) {
  const double q = len / dt;
  const double r = std::round(q);
  if (r < 1 || std::fabs(q - r) > 1e-9 * r) return false;
  *n = (int)r;
  return true;
}

// A handle of the library's own on the grid, time step and options of `src`,
// sharing its device tables (src must outlive it), with a workspace of its own.
static rbc_status clone_handle(rbc_t src, rbc_t* out) {
  rbc_t h = new (std::nothrow) rbc_s();
  if (!h) return fail(RBC_ENOMEM, "host allocation");
  h->g = src->g;
  h->opts = src->opts;
  h->device = src->device;
  h->max_residual = src->max_residual;
  h->t = src->t;                  // d_tables stays null: the tables are src's
  h->profp = src->profp;          // kernel timing goes to the template's record
  h->tunep = src->tunep;          // and the template's launch shapes apply
  h->use_graphs = src->use_graphs;
  *out = h;
  return RBC_OK;
}

static void destroy_slot(pr_s::Slot& S) {
  for (cudaStream_t st : {S.sC, S.sC_hi, S.sF[0], S.sF[1], S.sF[2], S.sF[3], S.pC, S.pF[0], S.pF[1], S.pF[2], S.pF[3]})
    if (st) cudaStreamSynchronize(st);
  for (cudaEvent_t e : S.ev_step)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : S.ev_group)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : S.ev_join)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t st : {S.sC, S.sC_hi, S.sF[0], S.sF[1], S.sF[2], S.sF[3], S.pC, S.pF[0], S.pF[1], S.pF[2], S.pF[3]})
    if (st) cudaStreamDestroy(st);
  rbc_destroy(S.coarse);
  for (rbc_t h : S.fines) rbc_destroy(h);
  for (void* b : {(void*)S.U, (void*)S.Fin, (void*)S.C, (void*)S.I, (void*)S.norms, (void*)S.partial, (void*)S.counter,
                  (void*)S.stat})
    cudaFree(b);
  S = pr_s::Slot{};
}

extern "C" void parareal_destroy(parareal_t p) {
  if (!p) return;
  drop_partition(p);
  if (p->sCancel) cudaStreamSynchronize(p->sCancel);
  for (auto& S : p->slots) destroy_slot(S);
  for (cudaEvent_t e : {p->ev_begin, p->ev_cancel})
    if (e) cudaEventDestroy(e);
  if (p->sCancel) cudaStreamDestroy(p->sCancel);
  cudaFree(p->d_Gold);
  cudaFree(p->d_cancel);
  delete p;
}

// Buffers, handles, streams and events of slot i, for `fine_streams` fine
// streams and the current partition (made on first use).
static rbc_status ensure_slot(pr_s* p, int i) {
  if ((int)p->slots.size() <= i) p->slots.resize(i + 1);
  pr_s::Slot& S = p->slots[i];
  const Grid &gf = p->fine->g, &gc = p->coarse->g;
  const int N = p->N;
  const size_t Bf = state_doubles(gf) * sizeof(double), Bc = state_doubles(gc) * sizeof(double);
  if (!S.U) {
    bool ok = cudaMalloc(&S.U, (N + 1) * Bf) == cudaSuccess && cudaMalloc(&S.Fin, N * Bf) == cudaSuccess &&
              cudaMalloc(&S.C, Bc) == cudaSuccess && cudaMalloc(&S.I, N * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&S.norms, 2 * N * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&S.partial, 2 * correct_norm_blocks(gf) * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&S.counter, sizeof(unsigned)) == cudaSuccess &&
              cudaMemset(S.counter, 0, sizeof(unsigned)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      destroy_slot(S);
      return fail(RBC_ENOMEM, "Parareal buffers of an iteration");
    }
    S.ev_step.assign(N, nullptr);
    S.ev_group.assign(N, nullptr);
    S.slice_group.assign(N, 0);
    for (auto* v : {&S.ev_step, &S.ev_group})
      for (cudaEvent_t& e : *v) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (cudaEvent_t& e : S.ev_join) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (p->every > 0 && !S.stat) {
    if (cudaMalloc(&S.stat, (size_t)N * (6 + 2 * gf.Mz) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(RBC_ENOMEM, "Parareal statistics of an iteration");
    }
  }
  if (!S.coarse) {
    rbc_status s = clone_handle(p->coarse, &S.coarse);
    if (s == RBC_OK) s = rbc_reserve(S.coarse, 1);
    if (s != RBC_OK) return s;
    S.coarse->w.cancel = p->d_cancel;
  }
  for (int j = 0; j < p->fine_streams; ++j)
    if (!S.fines[j]) {
      rbc_status s = clone_handle(p->fine, &S.fines[j]);
      if (s == RBC_OK) s = rbc_reserve(S.fines[j], std::min(p->N, p->group));
      if (s != RBC_OK) return s;
      S.fines[j]->w.cancel = p->d_cancel;
    }
  for (int j = 0; p->every > 0 && j < p->fine_streams; ++j) {
    rbc_status s = reserve_sampling(S.fines[j], std::min(p->N, p->group));
    if (s != RBC_OK) return s;
  }
  int lo = 0, hi = 0;
  CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  if (!S.sC) CK(cudaStreamCreateWithFlags(&S.sC, cudaStreamNonBlocking));
  if (!S.sC_hi) CK(cudaStreamCreateWithPriority(&S.sC_hi, cudaStreamNonBlocking, hi));
  for (int j = 0; j < p->fine_streams; ++j)
    if (!S.sF[j]) CK(cudaStreamCreateWithFlags(&S.sF[j], cudaStreamNonBlocking));
  if (p->gctx[0]) {
    CtxScope scope(p->gctx[1]);
    if (!scope.ok()) return fail(RBC_ECUDA, "cannot enter the SM partition's context");
    for (int j = 0; j < p->fine_streams; ++j)
      if (!S.pF[j]) CK(cudaStreamCreateWithFlags(&S.pF[j], cudaStreamNonBlocking));
  }
  // handles capture their step graphs in the partition they run in
  S.coarse->bind_ctx = nullptr;   // the sweeps on the coarse grid may use every SM
  for (int j = 0; j < p->fine_streams; ++j) S.fines[j]->bind_ctx = p->gctx[1];
  return RBC_OK;
}

static cudaStream_t sweep_stream(const pr_s* p, const pr_s::Slot& S) {
  return p->coarse_priority ? S.sC_hi : S.sC;
}
static cudaStream_t fine_stream(const pr_s* p, const pr_s::Slot& S, int j) { return p->gctx[0] ? S.pF[j] : S.sF[j]; }

extern "C" rbc_status parareal_create(rbc_t fine, rbc_t coarse, double t0, double t1, int nslices, int criterion,
                                      double tol, parareal_t* out) {
  if (!out) return fail(RBC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!fine || !coarse || nslices < 1 || !(t1 > t0)) return fail(RBC_EINVAL, "bad handles, slices or interval");
  if (criterion < RBC_CRIT_FIXED || criterion > RBC_CRIT_STAT || !(tol >= 0)) return fail(RBC_EINVAL, "bad criterion");
  const Grid &gf = fine->g, &gc = coarse->g;
  if (gc.Nx > gf.Nx || gc.Nz > gf.Nz) return fail(RBC_EINVAL, "coarse grid finer than fine grid");
  if (gc.Ra != gf.Ra || gc.Pr != gf.Pr || gc.Lx != gf.Lx || gc.bc != gf.bc)
    return fail(RBC_EINVAL, "Ra, Pr, Lx or boundary conditions differ");
  const double len = (t1 - t0) / nslices;
  int nf = 0, nc = 0;
  if (!whole_steps(len, gf.dt, &nf)) return fail(RBC_EINVAL, "slice length is not a whole number of fine steps");
  if (!whole_steps(len, gc.dt, &nc)) return fail(RBC_EINVAL, "slice length is not a whole number of coarse steps");
  pr_s* p = new (std::nothrow) pr_s();
  if (!p) return fail(RBC_ENOMEM, "host allocation");
  p->fine = fine;
  p->coarse = coarse;
  p->t0 = t0;
  p->t1 = t1;
  p->N = nslices;
  p->nf = nf;
  p->nc = nc;
  p->criterion = criterion;
  p->tol = tol;
  // default schedule: largest fine group N/4, first group a quarter of that,
  // groups alternating over two fine streams, sweeps on the coarse grid at high
  // priority, one iteration enqueued ahead of the one being evaluated
  p->group = std::max(1, (nslices + 3) / 4);
  p->first_group = std::max(1, (p->group + 3) / 4);
  // the statistical criterion samples at the slice ends unless told otherwise
  p->every = criterion == RBC_CRIT_STAT ? nf : 0;
  p->window_first = nslices / 2;
  const size_t Bc = state_doubles(gc) * sizeof(double);
  bool ok = cudaMalloc(&p->d_Gold, nslices * Bc) == cudaSuccess && cudaMalloc(&p->d_cancel, sizeof(int)) == cudaSuccess &&
            cudaMemset(p->d_cancel, 0, sizeof(int)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&p->sCancel, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&p->ev_begin, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&p->ev_cancel, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    parareal_destroy(p);
    return fail(RBC_ENOMEM, "Parareal buffers");
  }
  rbc_status s = ensure_slot(p, 0);   // the coarse sweep U^0 and the first iteration
  if (s == RBC_OK) s = ensure_slot(p, 1);
  if (s != RBC_OK) {
    parareal_destroy(p);
    return s;
  }
  *out = p;
  return RBC_OK;
}

extern "C" rbc_status parareal_set_schedule(parareal_t p, int group, int first_group, int fine_streams,
                                            int coarse_priority, int coarse_sms) {
  if (!p || group < 1 || first_group < 1 || first_group > group || fine_streams < 1 ||
      fine_streams > pr_s::kFineStreams || coarse_priority < 0 || coarse_priority > 1 || coarse_sms < 0)
    return fail(RBC_EINVAL, "bad schedule");
  if (coarse_sms != p->coarse_sms) {
    drop_partition(p);
    if (coarse_sms > 0) {
      rbc_status st = make_partition(p, coarse_sms);
      if (st != RBC_OK) return st;
    }
  }
  p->group = std::min(group, p->N);
  p->first_group = std::min(first_group, p->group);
  p->fine_streams = fine_streams;
  p->coarse_priority = coarse_priority;
  for (int i = 0; i < (int)p->slots.size(); ++i) {
    rbc_status s = ensure_slot(p, i);
    if (s != RBC_OK) return s;
  }
  return RBC_OK;
}

extern "C" rbc_status parareal_set_depth(parareal_t p, int depth) {
  if (!p || depth < 0 || depth > pr_s::kMaxDepth) return fail(RBC_EINVAL, "depth must be in [0, %d]", pr_s::kMaxDepth);
  p->depth = depth;
  return RBC_OK;
}

extern "C" rbc_status parareal_set_sampling(parareal_t p, int every, int window_first) {
  if (!p || every < 0 || window_first < 0 || window_first >= p->N)
    return fail(RBC_EINVAL, "every must be >= 0 and window_first in [0, nslices)");
  if (every == 0 && p->criterion == RBC_CRIT_STAT) return fail(RBC_EINVAL, "the statistical criterion needs samples");
  p->every = every;
  p->window_first = window_first;
  for (int i = 0; i < (int)p->slots.size(); ++i) {
    rbc_status s = ensure_slot(p, i);
    if (s != RBC_OK) return s;
  }
  return RBC_OK;
}

extern "C" rbc_status parareal_stat_means(parareal_t p, double* out) {
  if (!p || !out) return fail(RBC_EINVAL, "null argument");
  if (p->stat_means.empty()) return fail(RBC_EINVAL, "no sampled iteration yet");
  std::copy(p->stat_means.begin(), p->stat_means.end(), out);
  return RBC_OK;
}

extern "C" int parareal_coarse_sms(parareal_t p) { return p ? p->coarse_sms : -1; }

// Fine groups of an iteration: slices n >= n0 cut into groups whose sizes
// start at first_group and double up to `group`: a small first group lets the
// correction sweep start early, larger later groups keep the fine sweep efficient.
// Returns the first slice of each group (plus N at the end).
static std::vector<int> fine_group_starts(const pr_s* p, int n0) {
  std::vector<int> a{n0};
  if (p->group >= p->N) {   // one batch
    a.push_back(p->N);
    return a;
  }
  int size = p->first_group;
  while (a.back() < p->N) {
    a.push_back(std::min(p->N, a.back() + size));
    size = std::min(p->group, 2 * size);
  }
  return a;
}

// Enqueue iteration k: for k = 0 the coarse sweep U^0_{n+1} = prolong(G(U^0_n));
// for k >= 1 the fine groups F(U^{k-1}_n), n >= k - 1, and the correction sweep
// U^k_{n+1} = F(U^{k-1}_n) + (G(U^k_n) - G(U^{k-1}_n)) with its norms.  Slices
// n < k - 1 are exact already: U^k_{n+1} = U^{k-1}_{n+1}.  Every step waits only
// for the data it reads: the previous iteration's step n (which wrote
// G(U^{k-1}_n) and U^{k-1}_{n+1}) and the fine group of slice n.  `last`: the
// final iteration that will be enqueued (it writes no fine inputs for k + 1).
static rbc_status enqueue_iteration(pr_s* p, int k, int last, const double* d_U0) {
  const int R = p->depth + 2, N = p->N;
  const Grid &gf = p->fine->g, &gc = p->coarse->g;
  const size_t Sf = state_doubles(gf), Sc = state_doubles(gc), Bf = Sf * sizeof(double);
  pr_s::Slot& S = p->slots[k % R];
  pr_s::Slot& X = p->slots[(k + 1) % R];
  const cudaStream_t sC = sweep_stream(p, S);
  S.busy = true;
  std::vector<int> ncv(1, p->nc);
  CK(cudaMemsetAsync(S.coarse->w.err, 0, sizeof(int), sC));   // this iteration's error bits
  if (k == 0) {
    CK(launch_restrict(gf, gc, static_cast<const double*>(d_U0), S.C, 1, sC));
    for (int n = 0; n < N; ++n) {
      rbc_status s = rbc_step_batch(S.coarse, S.C, 1, ncv.data(), nullptr, sC);
      if (s != RBC_OK) return s;
      double* Fnext = (n + 1 < N && last >= 1) ? X.Fin + (n + 1) * Sf : nullptr;
      CK(launch_correct_norm(gf, gc, p->fine->t, 0, nullptr, S.C, p->d_Gold + n * Sc, S.C, nullptr,
                             S.U + (n + 1) * Sf, Fnext, S.partial, S.counter, nullptr, sC));
      CK(cudaEventRecord(S.ev_step[n], sC));
    }
    return RBC_OK;
  }
  pr_s::Slot& P = p->slots[(k - 1) % R];
  const int n0 = k - 1;
  // the converged slices U^k_0 .. U^k_{k-1}
  if (k >= 2) CK(cudaStreamWaitEvent(sC, P.ev_step[k - 2], 0));
  CK(cudaMemcpyAsync(S.U, P.U, (size_t)k * Bf, cudaMemcpyDeviceToDevice, sC));
  // the fine groups: inputs S.Fin[n] written by the previous sweep at its step n - 1
  std::vector<int> nfv(N, p->nf);
  const std::vector<int> a = fine_group_starts(p, n0);
  for (int i = 0; i < p->fine_streams; ++i)
    CK(cudaMemsetAsync(S.fines[i]->w.err, 0, sizeof(int), fine_stream(p, S, i)));
  for (int j = 0; j + 1 < (int)a.size(); ++j) {
    const int cnt = a[j + 1] - a[j];
    const int i = j % p->fine_streams;
    const cudaStream_t st = fine_stream(p, S, i);
    const int last_in = a[j] + cnt - 2;
    if (last_in >= std::max(0, k - 2)) CK(cudaStreamWaitEvent(st, P.ev_step[last_in], 0));
    double* Fj = S.Fin + (size_t)a[j] * Sf;
    rbc_status s = p->every > 0 ? rbc_step_batch_sampled(S.fines[i], Fj, cnt, p->nf, p->every, S.I + a[j],
                                                         S.stat + (size_t)a[j] * (6 + 2 * gf.Mz), st)
                                : rbc_step_batch(S.fines[i], Fj, cnt, nfv.data(), S.I + a[j], st);
    if (s != RBC_OK) return s;
    CK(cudaEventRecord(S.ev_group[j], st));
    for (int n = a[j]; n < a[j + 1]; ++n) S.slice_group[n] = j;
  }
  // the correction sweep
  for (int n = n0; n < N; ++n) {
    if (n >= k) {   // G(U^k_n); S.C holds the coarse modes of U^k_n
      rbc_status s = rbc_step_batch(S.coarse, S.C, 1, ncv.data(), nullptr, sC);
      if (s != RBC_OK) return s;
    }
    CK(cudaStreamWaitEvent(sC, P.ev_step[n], 0));
    CK(cudaStreamWaitEvent(sC, S.ev_group[S.slice_group[n]], 0));
    double* Gold = p->d_Gold + n * Sc;
    const double* Gnew = n >= k ? S.C : Gold;   // U^k_{k-1} = U^{k-1}_{k-1}: G of it is Gold exactly
    double* Fnext = (n + 1 < N && k < last) ? X.Fin + (n + 1) * Sf : nullptr;
    CK(launch_correct_norm(gf, gc, p->fine->t, 1, S.Fin + n * Sf, Gnew, Gold, S.C, P.U + (n + 1) * Sf,
                           S.U + (n + 1) * Sf, Fnext, S.partial, S.counter, S.norms + 2 * n, sC));
    CK(cudaEventRecord(S.ev_step[n], sC));
  }
  return RBC_OK;
}

// Stop the step loops still running (speculative iterations past the one
// that met the criterion), copy U^k_final to the caller and join every stream
// of the call into `stream`, then clear the cancel word for the next call.
static rbc_status finish_iterations(pr_s* p, int final_k, void* d_U, cudaStream_t stream) {
  const int R = p->depth + 2;
  CK(cudaMemsetAsync(p->d_cancel, 1, sizeof(int), p->sCancel));
  CK(cudaEventRecord(p->ev_cancel, p->sCancel));
  if (final_k >= 0) {
    pr_s::Slot& F = p->slots[final_k % R];
    CK(cudaStreamWaitEvent(stream, F.ev_step[p->N - 1], 0));
    CK(cudaMemcpyAsync(d_U, F.U, (size_t)(p->N + 1) * state_doubles(p->fine->g) * sizeof(double),
                       cudaMemcpyDeviceToDevice, stream));
  }
  for (auto& S : p->slots) {
    if (!S.busy) continue;
    S.busy = false;
    CK(cudaEventRecord(S.ev_join[0], sweep_stream(p, S)));
    CK(cudaStreamWaitEvent(stream, S.ev_join[0], 0));
    for (int j = 0; j < p->fine_streams; ++j) {
      CK(cudaEventRecord(S.ev_join[1 + j], fine_stream(p, S, j)));
      CK(cudaStreamWaitEvent(stream, S.ev_join[1 + j], 0));
    }
  }
  CK(cudaStreamWaitEvent(stream, p->ev_cancel, 0));
  CK(cudaMemsetAsync(p->d_cancel, 0, sizeof(int), stream));
  return RBC_OK;
}

extern "C" rbc_status parareal_iterate(parareal_t p, const void* d_U0, void* d_U, int max_iters, int* k_done,
                                       double* defects, double* nus, cudaStream_t stream) {
  if (!p || !d_U0 || !d_U || max_iters < 1) return fail(RBC_EINVAL, "bad arguments");
  const Grid& gf = p->fine->g;
  const size_t Sf = state_doubles(gf), Bf = Sf * sizeof(double);
  const int N = p->N, R = p->depth + 2;
  const int K = std::min(max_iters, N);   // U^N is the serial fine solution
  if (k_done) *k_done = 0;
  for (int i = 0; i < std::min(R, K + 1); ++i) {
    rbc_status s = ensure_slot(p, i);
    if (s != RBC_OK) return s;
  }
  // U^0_0 = U0 (slot 0), and the first fine input of iteration 1
  CK(cudaMemcpyAsync(p->slots[0].U, d_U0, Bf, cudaMemcpyDeviceToDevice, stream));
  CK(cudaMemcpyAsync(p->slots[1].Fin, d_U0, Bf, cudaMemcpyDeviceToDevice, stream));
  CK(cudaEventRecord(p->ev_begin, stream));   // every stream of the call starts after the caller's work
  for (int i = 0; i < std::min(R, K + 1); ++i) {
    pr_s::Slot& S = p->slots[i];
    CK(cudaStreamWaitEvent(sweep_stream(p, S), p->ev_begin, 0));
    for (int j = 0; j < p->fine_streams; ++j) CK(cudaStreamWaitEvent(fine_stream(p, S, j), p->ev_begin, 0));
  }
  int final_k = 0;
  rbc_status result = (p->criterion == RBC_CRIT_FIXED) ? RBC_OK : RBC_ENOTCONVERGED;
  int enqueued = -1;
  auto enqueue_upto = [&](int kmax) -> rbc_status {
    for (int k = enqueued + 1; k <= std::min(kmax, K); ++k) {
      rbc_status s = enqueue_iteration(p, k, K, static_cast<const double*>(d_U0));
      if (s != RBC_OK) return s;
      enqueued = k;
    }
    return RBC_OK;
  };
  auto bail = [&](rbc_status s) {
    const std::string why = g_err;
    finish_iterations(p, final_k, d_U, stream);
    snprintf(g_err, sizeof(g_err), "%s", why.c_str());
    return s;
  };
  rbc_status s = enqueue_upto(1 + p->depth);
  if (s != RBC_OK) return bail(s);
  std::vector<double> Ih(N, 0.0), nrm(2 * N), In(N);
  double nu_prev = 0.0;
  const size_t D = 6 + 2 * (size_t)gf.Mz;
  std::vector<double> Sh(p->every > 0 ? (size_t)N * D : 0), means(D);
  double stat_prev[6] = {};
  p->stat_means.clear();
  const int n_half = N / 2;
  const double win = (p->t1 - p->t0) * (double)(N - n_half) / N;
  for (int k = 1; k <= K; ++k) {
    pr_s::Slot& S = p->slots[k % R];
    const int n0 = k - 1;
    CK(cudaEventSynchronize(S.ev_step[N - 1]));   // the sweep waited for every fine group of the iteration
    final_k = k;
    int bits = 0;
    for (rbc_t h : {S.coarse, S.fines[0], S.fines[1], S.fines[2], S.fines[3]}) {
      int b = 0;
      if (h && h->cap > 0) CK(cudaMemcpy(&b, h->w.err, sizeof(int), cudaMemcpyDeviceToHost));
      bits |= b;
    }
    if (bits & kFlagTimeout) return bail(status_of_bits(bits));
    CK(cudaMemcpy(nrm.data() + 2 * n0, S.norms + 2 * n0, 2 * (N - n0) * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(In.data() + n0, S.I + n0, (N - n0) * sizeof(double), cudaMemcpyDeviceToHost));
    // Defect_k = max_n ||U_n^k - U_n^{k-1}|| / ||U_n^k|| (L2 of T); the slices
    // n <= k - 1 are unchanged.  A non-finite fine or coarse result reaches U
    // through the correction and shows here.
    double defect = 0.0;
    for (int n = n0; n < N; ++n) {
      const double d2 = nrm[2 * n], u2 = nrm[2 * n + 1];
      if (!std::isfinite(d2) || !std::isfinite(u2)) return bail(fail(RBC_EDIVERGED, "non-finite iterate"));
      if (u2 > 0) defect = std::max(defect, std::sqrt(d2 / u2));
      if (!std::isfinite(In[n])) return bail(fail(RBC_EDIVERGED, "non-finite Nu integral"));
      Ih[n] = In[n];
    }
    double nu = 0.0;
    for (int n = n_half; n < N; ++n) nu += Ih[n];
    nu /= win;
    if (defects) defects[k - 1] = defect;
    if (nus) nus[k - 1] = nu;
    if (k_done) *k_done = k;
    bool stop = false;
    if (p->criterion == RBC_CRIT_DEFECT && defect <= p->tol) stop = true;
    if (p->criterion == RBC_CRIT_NU && k >= 2 && std::fabs(nu - nu_prev) <= p->tol * std::fabs(nu)) stop = true;
    nu_prev = nu;
    if (p->every > 0) {
      // window means of the sampled quantities (Sec. 2.2) over the fine
      // trajectories from U^{k-1}; slices n < k - 1 keep their last values
      CK(cudaMemcpy(Sh.data() + (size_t)n0 * D, S.stat + (size_t)n0 * D, (size_t)(N - n0) * D * sizeof(double),
                    cudaMemcpyDeviceToHost));
      std::fill(means.begin(), means.end(), 0.0);
      double dur = 0.0;
      for (int n = p->window_first; n < N; ++n) {
        for (size_t q = 0; q < D; ++q) means[q] += Sh[(size_t)n * D + q];
        dur += p->nf * gf.dt;
      }
      for (size_t q = 0; q < D; ++q) means[q] /= dur;
      p->stat_means = means;
      // reading R22: stop at the first k >= 2 at which Nu_V, Nu_b, Nu_t, Re, P
      // and eps_U all changed by at most tol relative to iteration k - 1
      const double st[6] = {means[3], means[4], means[5], means[0] / gf.Pr, gf.Ra * means[2], std::fabs(means[1])};
      double change = 0.0;
      for (int q = 0; q < 6; ++q) {
        if (!std::isfinite(st[q])) return bail(fail(RBC_EDIVERGED, "non-finite time statistics"));
        change = std::max(change, std::fabs(st[q] - stat_prev[q]) / std::fabs(st[q]));
      }
      if (p->criterion == RBC_CRIT_STAT && k >= 2 && change <= p->tol) stop = true;
      std::copy(st, st + 6, stat_prev);
    }
    if (stop) {
      result = RBC_OK;
      break;
    }
    s = enqueue_upto(k + 1 + p->depth);
    if (s != RBC_OK) return bail(s);
  }
  s = finish_iterations(p, final_k, d_U, stream);
  if (s != RBC_OK) return s;
  CK(cudaStreamSynchronize(stream));
  return result;
}
