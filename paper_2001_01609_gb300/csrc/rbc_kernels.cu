// CUDA kernels of the fine/coarse propagator (FP64 path) for sm_103a.
//
// One RK443 stage (Sec. 3.2, Sec. 3.6) of B batched time slices is four
// launches:
//   k_zinv   z inverse transform: Chebyshev coefficients -> 9 fields at the
//            3/2-padded Lobatto points, with the Fourier-mode factors ik;
//   k_rows   per (slice, padded z-row): packed inverse real FFTs in x
//            (shared memory, mixed-radix Stockham), advective products,
//            one packed forward FFT, truncation to the kept modes, x-means;
//   k_zfwd   z forward transform of the products to T coefficients n < Nz;
//   k_solve  per (slice, Fourier mode, Chebyshev parity): RK443 right-hand
//            side in tau rows, UL banded solve of the implicit system
//            (temperature first, then streamfunction with the implicit
//            buoyancy coupling), RK accumulator updates, Nu_V accumulation.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "rbc_internal.h"

namespace rbc {

// IMEX Runge-Kutta pairs of Ascher, Ruuth & Spiteri (1997), [scheme][i][j]:
// coefficient of stage j in stage i, stage 0 explicit, zero-padded to 5 x 5.
// RK443 is the paper's (Sec. 3.2, Sec. 3.6); ARS(2,2,2) and ARS(1,1,1) are the
// lower-order coarse steppers of Sec. 3.6.  Filled by upload_schemes().
__constant__ double c_AE[3][5][5];
__constant__ double c_AI[3][5][5];

void scheme_tableau(int scheme, double AE[5][5], double AI[5][5], int* ns, double* gamma) {
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) AE[i][j] = AI[i][j] = 0.0;
  if (scheme == RBC_RK222) {
    // gamma = 1 - 1/sqrt(2): second order and L-stable; delta = 1 - 1/(2 gamma)
    const double gm = 1.0 - 1.0 / std::sqrt(2.0), dl = 1.0 - 1.0 / (2.0 * gm);
    AI[1][1] = gm;
    AI[2][1] = 1.0 - gm;
    AI[2][2] = gm;
    AE[1][0] = gm;
    AE[2][0] = dl;
    AE[2][1] = 1.0 - dl;
    *ns = 2;
    *gamma = gm;
  } else if (scheme == RBC_RK111) {
    // explicit Euler for the nonlinear terms, implicit Euler for the linear ones
    AI[1][1] = 1.0;
    AE[1][0] = 1.0;
    *ns = 1;
    *gamma = 1.0;
  } else {
    const double ae[5][5] = {{0, 0, 0, 0, 0},
                             {1.0 / 2, 0, 0, 0, 0},
                             {11.0 / 18, 1.0 / 18, 0, 0, 0},
                             {5.0 / 6, -5.0 / 6, 1.0 / 2, 0, 0},
                             {1.0 / 4, 7.0 / 4, 3.0 / 4, -7.0 / 4, 0}};
    const double ai[5][5] = {{0, 0, 0, 0, 0},
                             {0, 1.0 / 2, 0, 0, 0},
                             {0, 1.0 / 6, 1.0 / 2, 0, 0},
                             {0, -1.0 / 2, 1.0 / 2, 1.0 / 2, 0},
                             {0, 3.0 / 2, -3.0 / 2, 1.0 / 2, 1.0 / 2}};
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) {
        AE[i][j] = ae[i][j];
        AI[i][j] = ai[i][j];
      }
    *ns = 4;
    *gamma = 0.5;
  }
}


cudaError_t upload_schemes() {
  double ae[3][5][5], ai[3][5][5];
  for (int sc = 0; sc < 3; ++sc) {
    int ns;
    double gm;
    scheme_tableau(sc, ae[sc], ai[sc], &ns, &gm);
  }
  cudaError_t e = cudaMemcpyToSymbol(c_AE, ae, sizeof(ae));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_AI, ai, sizeof(ai));
  return e;
}

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
// Roundings written out (explicit fma): the bits do not depend on how the
// compiler would contract a*b + c*d in each kernel that inlines this.
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 times_i(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Complex element (f, n, m) of a state, in doubles.
__device__ __forceinline__ size_t soff(const Grid& g, int f, int n, int m) {
  return ((size_t)(f * g.Nz + n) * g.nm + m) * 2;
}

__device__ __forceinline__ bool slice_active(const int* nsteps, const int* step, int b) {
  return nsteps == nullptr || *step < nsteps[b];
}
__device__ __forceinline__ bool slice_active_at(const int* nsteps, int stepidx, int b) {
  return nsteps == nullptr || stepidx < nsteps[b];
}


// ---------------------------------------------------------------------------
// Real-type generic complex helpers for the transform kernels, which run in
// FP64 (RBC_FP64) or in FP32 (RBC_MIXED); the state, the explicit terms F and
// the stage solve stay FP64 in both modes.
// ---------------------------------------------------------------------------
template <typename T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };
template <typename T> using C2 = typename Cx<T>::t;

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 times_i(float2 a) { return make_float2(-a.y, a.x); }

template <typename T> __device__ __forceinline__ C2<T> mk2(T x, T y);
template <> __device__ __forceinline__ double2 mk2<double>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 mk2<float>(float x, float y) { return make_float2(x, y); }
template <typename T> __device__ __forceinline__ C2<T> ldc(const T* p) { return *reinterpret_cast<const C2<T>*>(p); }
template <typename T> __device__ __forceinline__ void stc(T* p, C2<T> v) { *reinterpret_cast<C2<T>*>(p) = v; }
template <typename T> __device__ __forceinline__ C2<T> ldgc(const C2<T>* p) { return __ldg(p); }
template <typename T> __device__ __forceinline__ C2<T> cvt2(double2 a) { return mk2<T>((T)a.x, (T)a.y); }

// ---------------------------------------------------------------------------
// z inverse transform (k_zinv).  Block per (slice, padded row pair j / Mz-1-j,
// tile of 32 modes) with kp warps; warp w accumulates the coefficients n of its
// share of [0, Nz), and the kp partial sums are added in a fixed order.
// Even/odd split: the padded points are symmetric, s_{Mz-1-j} = -s_j, and
// T_n^(q)(-s) = (-1)^(n+q) T_n^(q)(s), so the sums E, O over even and odd n at
// s_j give f^(q)(s_j) = E + O and f^(q)(-s_j) = (-1)^q (E - O): half the
// multiply-adds of evaluating both rows.  psi-slot operators V, VD, VD^2, VD^3
// (d/ds) and T-slot V, VD; the epilogue forms, with d/dz = 2 d/ds, d/dx = ik:
//   u = d_z psi (m = 0: U),  w = -ik psi,  d_x omega, d_z omega (omega = -lap psi,
//   m = 0: omega = -U'),  d_x u,  d_z u,  T,  d_x T,  d_z T.
// Output Z[b][field][j][m] (complex, real type T), fields in that order.
// ---------------------------------------------------------------------------
// Field f (0..8, as listed above) of one output point from the operator sums
// P[q] = d^q psi / ds^q (q < 4), t0 = T, t1 = dT/ds.  The roundings are written
// out (explicit fma), so every kernel that forms a field gets the same bits.
template <typename T>
__device__ __forceinline__ C2<T> zinv_field(int f, int m, T k, const C2<T>* P, C2<T> t0, C2<T> t1) {
  using V = C2<T>;
  const T zero = 0;
  const V z = mk2<T>(zero, zero);
  switch (f) {
    case 0: return m == 0 ? mk2<T>(P[0].x, zero) : (T)2 * P[1];                 // u (m = 0: U)
    case 1: return m == 0 ? z : -k * times_i(P[0]);                             // w = -ik psi
    case 2: {                                                                   // d_x omega
      if (m == 0) return z;
      const T kk = k * k;                                                       // omega = k^2 psi - 4 d2(psi)
      const V om = mk2<T>(fma(kk, P[0].x, (T)-4 * P[2].x), fma(kk, P[0].y, (T)-4 * P[2].y));
      return k * times_i(om);
    }
    case 3: {                                                                   // d_z omega
      if (m == 0) return mk2<T>((T)-4 * P[2].x, zero);
      const T kk2 = ((T)2 * k) * k;                                             // 2 k^2 d(psi) - 8 d3(psi)
      return mk2<T>(fma(kk2, P[1].x, (T)-8 * P[3].x), fma(kk2, P[1].y, (T)-8 * P[3].y));
    }
    case 4: return m == 0 ? z : k * times_i((T)2 * P[1]);                       // d_x u
    case 5: return m == 0 ? mk2<T>((T)2 * P[1].x, zero) : (T)4 * P[2];          // d_z u
    case 6: return t0;                                                          // T
    case 7: return m == 0 ? z : k * times_i(t0);                                // d_x T
    case 8: return (T)2 * t1;                                                   // d_z T
    default: return z;
  }
}

// Fields of one output row (j, m); half = 0: fields 0-3, 1: fields 4-8, -1: all.
template <typename T>
__device__ __forceinline__ void zinv_store(const Grid& g, T* Zb, int j, int m, T k, const C2<T>* P, C2<T> t0,
                                           C2<T> t1, int half) {
  const size_t fs = (size_t)g.Mz * g.nm * 2;
  T* zb = Zb + ((size_t)j * g.nm + m) * 2;
  const int f0 = half == 1 ? 4 : 0, f1 = half == 0 ? 4 : 9;
  for (int f = f0; f < f1; ++f) stc<T>(zb + f * fs, zinv_field<T>(f, m, k, P, t0, t1));
}

template <typename T>
__device__ void zinv_item(const Grid& g, const T* __restrict__ Bz, const double* __restrict__ X, size_t S,
                          T* __restrict__ Z, int B, const int* nsteps, int stepidx, int blk, int kp) {
  using V = C2<T>;
  extern __shared__ __align__(16) unsigned char zsm[];
  V* part = reinterpret_cast<V*>(zsm);                 // [kp][12][32] when kp > 1
  const int Mh = (g.Mz + 1) / 2;
  const int mt = (g.nm + 31) / 32;
  const int b = blk / (Mh * mt);
  const int rem = blk - b * Mh * mt;
  const int j = rem / mt, m0 = (rem - j * mt) * 32;
  if (b >= B || !slice_active_at(nsteps, stepidx, b)) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = m0 + lane;
  const bool valid = m < g.nm;
  const bool wact = w < kp;                            // warps beyond kp, if any, idle
  const double* Xb = X + (size_t)b * S;
  const T* bq[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) bq[q] = Bz + (size_t)(q * g.Mz + j) * g.Nz;
  // share of the coefficient pairs (n, n+1) of this warp
  const int npair = g.Nz / 2;
  const int per = (npair + kp - 1) / kp;
  const int p0 = w * per, p1 = min(npair, p0 + per);
  V E[6], O[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) E[q] = O[q] = mk2<T>(0, 0);
  if (valid && wact) {
#pragma unroll 4
    for (int pp = p0; pp < p1; ++pp) {
      const int n = 2 * pp;
#pragma unroll
      for (int par = 0; par < 2; ++par) {
        const V xp = cvt2<T>(ld2(Xb + soff(g, 1, n + par, m)));
        const V xt = cvt2<T>(ld2(Xb + soff(g, 0, n + par, m)));
        V* A = par ? O : E;
        T v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __ldg(bq[q] + n + par);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          A[q].x = fma(v[q], xp.x, A[q].x);
          A[q].y = fma(v[q], xp.y, A[q].y);
        }
        A[4].x = fma(v[0], xt.x, A[4].x);
        A[4].y = fma(v[0], xt.y, A[4].y);
        A[5].x = fma(v[1], xt.x, A[5].x);
        A[5].y = fma(v[1], xt.y, A[5].y);
      }
    }
  }
  const T k = (T)(g.kfac * m);
  T* Zb = Z + (size_t)b * 9 * g.Mz * g.nm * 2;
  const int jr = g.Mz - 1 - j;
  if (kp > 1) {
    if (wact) {
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        part[(w * 12 + q) * 32 + lane] = E[q];
        part[(w * 12 + 6 + q) * 32 + lane] = O[q];
      }
    }
    __syncthreads();
    // accumulator a (E_0..5, O_0..5) is summed by warp a % kp, over the warps'
    // partial sums in warp order, into the first warp's slot
    for (int a = w; a < 12; a += kp) {
      V e = part[a * 32 + lane];
      for (int ww = 1; ww < kp; ++ww) e = e + part[(ww * 12 + a) * 32 + lane];
      part[a * 32 + lane] = e;
    }
    __syncthreads();
    if (!valid) return;
    // epilogue: warps take (row, half of the fields); with 2 warps one row each
    const int nt = kp >= 4 ? 4 : kp;
    for (int task = w; task < 4; task += nt) {
      const int row = task & 1, half = task >> 1;
      if (row == 1 && jr == j) continue;
      V Ev[6], Ov[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        Ev[q] = part[q * 32 + lane];
        Ov[q] = part[(6 + q) * 32 + lane];
      }
      V P[4];
      if (row == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) P[q] = Ev[q] + Ov[q];
        zinv_store<T>(g, Zb, j, m, k, P, Ev[4] + Ov[4], Ev[5] + Ov[5], half);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) P[q] = ((q & 1) ? (T)-1 : (T)1) * (Ev[q] - Ov[q]);
        zinv_store<T>(g, Zb, jr, m, k, P, Ev[4] - Ov[4], (T)-1 * (Ev[5] - Ov[5]), half);
      }
    }
    return;
  }
  if (w != 0 || !valid) return;
  V P[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) P[q] = E[q] + O[q];
  zinv_store<T>(g, Zb, j, m, k, P, E[4] + O[4], E[5] + O[5], -1);
  if (jr != j) {
#pragma unroll
    for (int q = 0; q < 4; ++q) P[q] = ((q & 1) ? (T)-1 : (T)1) * (E[q] - O[q]);
    zinv_store<T>(g, Zb, jr, m, k, P, E[4] - O[4], (T)-1 * (E[5] - O[5]), -1);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_zinv(Grid g, const T* __restrict__ Bz, const double* __restrict__ X, size_t S,
                                              T* __restrict__ Z, int B, const int* nsteps, const int* step) {
  pdl_wait();
  zinv_item<T>(g, Bz, X, S, Z, B, nsteps, nsteps ? *step : 0, blockIdx.x, blockDim.x / 32);
}

// Warps sharing the coefficient sum of one k_zinv row pair.  It fixes the order
// of the floating-point additions, so it depends on the grid only (every batch
// size gives the same bits): small grids, whose single-state launches are
// latency-bound, split the sum over up to 8 warps; large grids keep one warp.
static int zinv_warps(const Grid& g) {
  if ((long)g.Nx * g.Nz > 8192) return 1;
  int kp = 1;
  while (kp < 8 && (g.Nz / 2) / (2 * kp) >= 2) kp *= 2;
  return kp;
}

// ---------------------------------------------------------------------------
// Shared-memory mixed-radix Stockham FFT of length N = 3 * 2^p (radices
// 4, ..., 4, [2], 3) applied to na arrays of length N at once (array a at
// [a * N]).  y_q = sum_r x_r exp(sign 2 pi i q r / N), unnormalised.
// Ping-pongs between a and b; returns the buffer holding the results.
// ---------------------------------------------------------------------------
template <typename T>
__device__ C2<T>* fft_smem(C2<T>* a, C2<T>* b, int N, int na, int sign, const C2<T>* tw) {
  using V = C2<T>;
  int p = 0;
  for (int M = N / 3; M > 1; M >>= 1) ++p;
  const int nr = p / 2 + (p & 1) + 1;
  int Ns = 1, lns = 0;                                 // Ns = 2^lns
  V* x = a;
  V* y = b;
  const T s3 = (T)0.86602540378443864676 * (T)sign;   // sign * sqrt(3)/2
  const T sg = (T)sign;
  for (int pass = 0; pass < nr; ++pass) {
    const int R = (pass < p / 2) ? 4 : ((p & 1) && pass == p / 2) ? 2 : 3;
    // N = 3 2^p: N / R and N / (Ns R) by shifts (the radix-3 pass leaves 2^p)
    const int nb = R == 4 ? N >> 2 : R == 2 ? N >> 1 : 1 << p;
    const int stride = nb >> lns;
    for (int it = threadIdx.x; it < na * nb; it += blockDim.x) {
      const int arr = na == 1 ? 0 : it / nb, jj = it - arr * nb;   // one array: no division
      const V* xa = x + arr * N;
      V* ya = y + arr * N;
      const int k = jj & (Ns - 1);                  // Ns is a power of two (the radix-3 pass is last)
      V v[4];
      for (int r = 0; r < R; ++r) v[r] = xa[jj + r * nb];
      if (Ns > 1) {
        // k < Ns and r < R, so k r stride < Ns R stride = N: the index needs no reduction
        const int kstr = k * stride;
        for (int r = 1; r < R; ++r) {
          V wv = tw[kstr * r];
          if (sign > 0) wv.y = -wv.y;
          v[r] = cmul(v[r], wv);
        }
      }
      const int base = (jj - k) * R + k;            // (jj / Ns) Ns R + k
      if (R == 2) {
        ya[base] = v[0] + v[1];
        ya[base + Ns] = v[0] - v[1];
      } else if (R == 4) {
        const V a0 = v[0] + v[2], a1 = v[0] - v[2];
        const V b0 = v[1] + v[3], b1 = v[1] - v[3];
        const V ib1 = sg * times_i(b1);
        ya[base] = a0 + b0;
        ya[base + Ns] = a1 + ib1;
        ya[base + 2 * Ns] = a0 - b0;
        ya[base + 3 * Ns] = a1 - ib1;
      } else {
        const V t1 = v[1] + v[2], t2 = v[1] - v[2];
        const V m1 = v[0] - (T)0.5 * t1;
        // m1 +- s3 i t2 with one rounding per part (explicit fma)
        ya[base] = v[0] + t1;
        ya[base + Ns] = mk2<T>(fma(-s3, t2.y, m1.x), fma(s3, t2.x, m1.y));
        ya[base + 2 * Ns] = mk2<T>(fma(s3, t2.y, m1.x), fma(-s3, t2.x, m1.y));
      }
    }
    __syncthreads();
    V* tmp = x;
    x = y;
    y = tmp;
    Ns *= R;
    lns += R == 4 ? 2 : R == 2 ? 1 : 0;                // the radix-3 pass is the last
  }
  return x;
}

// Shared memory of k_rows: two ping-pong sets of 5 complex rows and the
// twiddles (11 Mx complex values); lean: 5 + 3 rows and the twiddles (9 Mx),
// the inverse FFTs in groups of three and two rows; or, when neither fits, two
// single rows, the twiddles and 9 real fields, with the five inverse FFTs in turn.
static size_t rows_bytes_batched(const Grid& g, size_t es) { return (size_t)g.Mx * 11 * 2 * es; }
static size_t rows_bytes_lean(const Grid& g, size_t es) { return (size_t)g.Mx * 9 * 2 * es; }
static size_t rows_bytes_serial(const Grid& g, size_t es) { return (size_t)g.Mx * (3 * 2 + 9) * es; }
static bool rows_batched(const Grid& g, size_t es) { return rows_bytes_batched(g, es) <= 200 * 1024; }
static size_t rows_smem_for(const Grid& g, size_t es, bool lean) {
  return rows_batched(g, es) ? (lean ? rows_bytes_lean(g, es) : rows_bytes_batched(g, es)) : rows_bytes_serial(g, es);
}
size_t rows_smem_bytes(const Grid& g) { return rows_smem_for(g, 8, false); }
// The lean layout by default where the full one leaves room for a single block
// per SM and the lean one for two.
static bool rows_lean_default(const Grid& g, size_t es) {
  return rows_batched(g, es) && rows_bytes_batched(g, es) > 113 * 1024 && rows_bytes_lean(g, es) <= 113 * 1024;
}

// Deterministic block sum: the fixed tree red[t] += red[t + s], s = blockDim/2
// down to 1 (blockDim a power of two, at least 32).  Levels s >= 32 go through
// shared memory, the last five through warp shuffles with the same pairings.
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s >= 32; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    double x = red[threadIdx.x];
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) x += __shfl_down_sync(0xffffffffu, x, s);
    if (threadIdx.x == 0) red[0] = x;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// Pair pr of real fields (2 pr, 2 pr + 1) of row j as one complex spectrum of
// length Mx: C = A + iB with the Hermitian extensions, zero beyond the kept modes.
template <typename T>
__device__ __forceinline__ C2<T> rows_packed(const Grid& g, const T* zrow, size_t fs, int pr, int x) {
  using V = C2<T>;
  const int fa = 2 * pr, fb = 2 * pr + 1, Mx = g.Mx, nm = g.nm;
  const T* za = zrow + fa * fs;
  const T* zb = zrow + fb * fs;
  V c = mk2<T>(0, 0);
  if (x < nm) {
    const V a = ldc<T>(za + 2 * x);
    const V bb = (fb < 9) ? ldc<T>(zb + 2 * x) : mk2<T>(0, 0);
    c = a + times_i(bb);
  } else if (x > Mx - nm) {
    const int m = Mx - x;
    const V a = ldc<T>(za + 2 * m);
    const V bb = (fb < 9) ? ldc<T>(zb + 2 * m) : mk2<T>(0, 0);
    c = conj2(a) + times_i(conj2(bb));
  }
  return c;
}

// Two block sums over the first 256 threads at once (the others pass nothing
// and only meet the barriers): for each value the tree of block_sum at 256
// threads, whatever blockDim is, with half the barriers of two calls.
__device__ double2 block_sum256_2(double a, double b, double2* red) {
  if (threadIdx.x < 256) red[threadIdx.x] = make_double2(a, b);
  __syncthreads();
  for (int s = 128; s >= 32; s >>= 1) {
    if ((int)threadIdx.x < s) {
      const double2 u = red[threadIdx.x], v = red[threadIdx.x + s];
      red[threadIdx.x] = make_double2(u.x + v.x, u.y + v.y);
    }
    __syncthreads();
  }
  if (threadIdx.x < 32) {
    double x = red[threadIdx.x].x, y = red[threadIdx.x].y;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, s);
      y += __shfl_down_sync(0xffffffffu, y, s);
    }
    if (threadIdx.x == 0) red[0] = make_double2(x, y);
  }
  __syncthreads();
  const double2 r = red[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Row kernel (k_rows).  Block per (slice, padded row j).  Pairs of real fields
// share one complex inverse FFT (C = A + iB with the Hermitian extensions);
// products in advective form (Eqs. 3, 5):
//   N_T = u T_x + w T_z,  N_omega = u omega_x + w omega_z,
//   <N_u>_x = <u u_x + w u_z>_x,  <w T>_x;
// one packed forward FFT (N_T + i N_omega), truncation to m < nm.
// Q[b][0][j][m] = N_T, Q[b][1][j][m] = N_omega (m >= 1), (<N_u>, 0) at m = 0.
// The x-means are summed in FP64 in both precision modes, from per-point
// terms staged in shared memory: thread t < 256 adds x = t, t + 256, ..., then
// a 256-wide tree, so the bits do not depend on the block size (256 to 1024
// threads, a launch shape) and equal those of k_rows_cl.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void rows_item(const Grid& g, const C2<T>* __restrict__ tw, const T* __restrict__ Z, T* __restrict__ Q,
                          double* __restrict__ wT, int B, int batched, int lean, const int* nsteps, int stepidx,
                          int blk) {
  using V = C2<T>;
  extern __shared__ __align__(16) unsigned char rsm[];
  const int b = blk / g.Mz, j = blk - b * g.Mz;
  if (b >= B || !slice_active_at(nsteps, stepidx, b)) return;
  const int Mx = g.Mx, nm = g.nm;
  __shared__ double2 red[256];
  const size_t fs = (size_t)g.Mz * nm * 2;
  const T* zrow = Z + (size_t)b * 9 * fs + (size_t)j * nm * 2;
  const V* fld;      // field value at x: real/imag parts of the five packed rows
  const V* fld3 = nullptr;   // rows 3 and 4 (batched: fld + 3 Mx unless lean)
  V* A;
  V* Bf;
  V* tws;
  V* P = nullptr;    // free rows after the inverse FFTs: products, scratch, x-mean terms
  V* P2 = nullptr;
  T* vU = nullptr;
  T* fr = nullptr;
  if (batched) {
    // the five packed rows and the FFT scratch: five more rows, or (lean) three,
    // the inverse FFTs then running in groups of three and two rows (the same
    // arithmetic per row; less shared memory, more blocks per SM)
    A = reinterpret_cast<V*>(rsm);
    Bf = A + 5 * Mx;
    tws = Bf + (lean ? 3 : 5) * Mx;
    for (int x = threadIdx.x; x < Mx; x += blockDim.x) tws[x] = ldgc<T>(tw + x);
    for (int pr = 0; pr < 5; ++pr)
      for (int x = threadIdx.x; x < Mx; x += blockDim.x) A[pr * Mx + x] = rows_packed<T>(g, zrow, fs, pr, x);
    __syncthreads();
    if (!lean) {
      fld = fft_smem<T>(A, Bf, Mx, 5, +1, tws);
      fld3 = fld + 3 * Mx;
      P = (fld == A) ? Bf : A;                 // the five rows not holding the fields
      vU = reinterpret_cast<T*>(P + Mx);
      P2 = (P == A) ? Bf : A;                  // a field row, free once the products are formed
    } else {
      fld = fft_smem<T>(A, Bf, Mx, 3, +1, tws);
      V* fr3 = fld == A ? Bf : A;              // rows free after the first group
      fld3 = fft_smem<T>(A + 3 * Mx, fr3, Mx, 2, +1, tws);
      // three free rows: the scratch (even pass count) or A[2..4] (odd)
      P = fld == A ? Bf : A + 2 * Mx;
      vU = reinterpret_cast<T*>(P + Mx);
      P2 = P + 2 * Mx;
    }
  } else {
    A = reinterpret_cast<V*>(rsm);
    Bf = A + Mx;
    tws = Bf + Mx;
    fr = reinterpret_cast<T*>(tws + Mx);
    for (int x = threadIdx.x; x < Mx; x += blockDim.x) tws[x] = ldgc<T>(tw + x);
    for (int pr = 0; pr < 5; ++pr) {
      for (int x = threadIdx.x; x < Mx; x += blockDim.x) A[x] = rows_packed<T>(g, zrow, fs, pr, x);
      __syncthreads();
      const V* res = fft_smem<T>(A, Bf, Mx, 1, +1, tws);
      for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
        fr[(2 * pr) * Mx + x] = res[x].x;
        if (pr < 4) fr[(2 * pr + 1) * Mx + x] = res[x].y;
      }
      __syncthreads();
    }
    fld = nullptr;
    P = A;
    P2 = Bf;
    vU = reinterpret_cast<T*>(P2);            // the scratch row holds the 2 Mx terms
  }
  auto field = [&](int fi, int x) -> T {
    if (fld) {
      const int k = fi >> 1;
      const V v = k < 3 ? fld[k * Mx + x] : fld3[(k - 3) * Mx + x];
      return (fi & 1) ? v.y : v.x;
    }
    return fr[fi * Mx + x];
  };
  // per-point x-mean terms (in T: each is the FP64 sum's exact input)
  T* vW = vU + Mx;
  for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
    const T u = field(0, x), w = field(1, x);
    const T nO = fma(u, field(2, x), w * field(3, x));
    vU[x] = fma(u, field(4, x), w * field(5, x));
    const T nT = fma(u, field(7, x), w * field(8, x));
    vW[x] = w * field(6, x);
    P[x] = mk2<T>(nT, nO);
  }
  __syncthreads();
  double nU = 0.0, wt = 0.0;
  if (threadIdx.x < 256)
    for (int x = threadIdx.x; x < Mx; x += 256) {
      nU += (double)vU[x];
      wt += (double)vW[x];
    }
  const double2 sUW = block_sum256_2(nU, wt, red);
  const double sU = sUW.x, sW = sUW.y;
  const V* C = fft_smem<T>(P, P2, Mx, 1, -1, tws);
  const T inv = (T)1 / (T)Mx;
  const T half = (T)0.5 * inv;
  const size_t qs = (size_t)g.Mz * nm * 2;
  T* q0 = Q + (size_t)b * 2 * qs + (size_t)j * nm * 2;
  T* q1 = q0 + qs;
  for (int m = threadIdx.x; m < nm; m += blockDim.x) {
    const V cm = C[m];
    const V cn = conj2(C[m == 0 ? 0 : Mx - m]);
    const V s = cm + cn, d = cm - cn;
    stc<T>(q0 + 2 * m, mk2<T>(half * s.x, half * s.y));
    if (m == 0)
      stc<T>(q1, mk2<T>((T)(sU / Mx), (T)0));
    else
      stc<T>(q1 + 2 * m, mk2<T>(half * d.y, -half * d.x));
  }
  if (threadIdx.x == 0) wT[(size_t)b * g.Mz + j] = sW / Mx;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_rows(Grid g, const C2<T>* __restrict__ tw, const T* __restrict__ Z,
                                              T* __restrict__ Q, double* __restrict__ wT, int B, int batched,
                                              int lean, const int* nsteps, const int* step) {
  pdl_wait();
  rows_item<T>(g, tw, Z, Q, wT, B, batched, lean, nsteps, nsteps ? *step : 0, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Row kernel for small batches (k_rows_cl): the same arithmetic as k_rows,
// spread over a cluster of five CTAs per row so that a single slice uses five
// times as many SMs' FP64 pipes.  CTA c runs the inverse FFT of field pair c
// (fields 2c, 2c+1) in its shared memory; after a cluster barrier every CTA
// forms the products for its share of the x points, reading the nine fields
// from the five CTAs through distributed shared memory, and writes them, with
// the per-point terms of the two x-means, into CTA 0.  After a second barrier
// CTA 0 sums the x-means with exactly the per-thread order and tree of k_rows
// (256 threads) and runs the forward FFT, so the results are bit for bit
// those of k_rows.
// ---------------------------------------------------------------------------
constexpr int kRowsCluster = 5;
constexpr int kRowsThreads = 256;

static size_t rows_cl_bytes(const Grid& g, size_t es) {
  // A, Bf, twiddles, P, P2 (complex) + two real per-point arrays (double)
  return (size_t)g.Mx * 5 * 2 * es + (size_t)2 * g.Mx * 8;
}
static bool rows_use_cluster(const Grid& g, int B, size_t es) {
  return (long)B * g.Mz <= 2L * 152 && rows_cl_bytes(g, es) <= 200 * 1024;
}

template <typename T>
__global__ void __cluster_dims__(kRowsCluster, 1, 1) __launch_bounds__(kRowsThreads)
    k_rows_cl(Grid g, const C2<T>* __restrict__ tw, const T* __restrict__ Z, T* __restrict__ Q,
              double* __restrict__ wT, int B, const int* nsteps, const int* step) {
  using V = C2<T>;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char csm[];
  __shared__ double2 red[kRowsThreads];
  pdl_wait();
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int row = blockIdx.x / kRowsCluster;
  const int b = row / g.Mz, j = row - b * g.Mz;
  // uniform over the cluster (same b and step): no CTA reaches a cluster barrier alone
  if (b >= B || !slice_active(nsteps, step, b)) return;
  const int Mx = g.Mx, nm = g.nm;
  V* A = reinterpret_cast<V*>(csm);
  V* Bf = A + Mx;
  V* tws = Bf + Mx;
  V* P = tws + Mx;
  V* P2 = P + Mx;
  double* vU = reinterpret_cast<double*>(P2 + Mx);
  double* vW = vU + Mx;
  const size_t fs = (size_t)g.Mz * nm * 2;
  const T* zrow = Z + (size_t)b * 9 * fs + (size_t)j * nm * 2;
  for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
    tws[x] = ldgc<T>(tw + x);
    A[x] = rows_packed<T>(g, zrow, fs, c, x);
  }
  __syncthreads();
  const V* res = fft_smem<T>(A, Bf, Mx, 1, +1, tws);   // same buffer in every CTA
  cl.sync();
  const V* fr[kRowsCluster];
#pragma unroll
  for (int r = 0; r < kRowsCluster; ++r) fr[r] = cl.map_shared_rank(res, r);
  V* P0 = cl.map_shared_rank(P, 0);
  double* vU0 = cl.map_shared_rank(vU, 0);
  double* vW0 = cl.map_shared_rank(vW, 0);
  auto field = [&](int fi, int x) -> T {
    const V v = fr[fi >> 1][x];
    return (fi & 1) ? v.y : v.x;
  };
  const int per = (Mx + kRowsCluster - 1) / kRowsCluster;
  const int x0 = c * per, x1 = min(Mx, x0 + per);
  for (int x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
    const T u = field(0, x), w = field(1, x);
    const T nO = fma(u, field(2, x), w * field(3, x));
    vU0[x] = (double)fma(u, field(4, x), w * field(5, x));
    const T nT = fma(u, field(7, x), w * field(8, x));
    vW0[x] = (double)(w * field(6, x));
    P0[x] = mk2<T>(nT, nO);
  }
  cl.sync();
  if (c != 0) return;
  // x-means: thread t adds x = t, t + 256, ... from 0, then the tree of k_rows
  double nU = 0.0, wt = 0.0;
  for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
    nU += vU[x];
    wt += vW[x];
  }
  const double2 sUW = block_sum256_2(nU, wt, red);   // kRowsThreads = 256: the same tree
  const double sU = sUW.x, sW = sUW.y;
  const V* C = fft_smem<T>(P, P2, Mx, 1, -1, tws);
  const T inv = (T)1 / (T)Mx;
  const T half = (T)0.5 * inv;
  const size_t qs = (size_t)g.Mz * nm * 2;
  T* q0 = Q + (size_t)b * 2 * qs + (size_t)j * nm * 2;
  T* q1 = q0 + qs;
  for (int m = threadIdx.x; m < nm; m += blockDim.x) {
    const V cm = C[m];
    const V cn = conj2(C[m == 0 ? 0 : Mx - m]);
    const V s2 = cm + cn, d = cm - cn;
    stc<T>(q0 + 2 * m, mk2<T>(half * s2.x, half * s2.y));
    if (m == 0)
      stc<T>(q1, mk2<T>((T)(sU / Mx), (T)0));
    else
      stc<T>(q1 + 2 * m, mk2<T>(half * d.y, -half * d.x));
  }
  if (threadIdx.x == 0) wT[(size_t)b * g.Mz + j] = sW / Mx;
}

// ---------------------------------------------------------------------------
// z forward transform (k_zfwd): F[b][f][n][m] = sum_j W[n][j] Q[b][f][j][m], n < Nz.
// W[n][Mz-1-j] = (-1)^n W[n][j] (symmetric points), so with the folds
// Ev_j = Q_j + Q_{Mz-1-j}, Od_j = Q_j - Q_{Mz-1-j} (the middle row, for odd Mz,
// once in Ev) F_n = sum_{j < ceil(Mz/2)} W[n][j] (n even ? Ev : Od)_j.  Block per
// (slice, field, tile of tm modes, chunk of the n range): the folds are staged
// in shared memory once per block and reused by every n of the chunk.  F is
// written in FP64 for the stage solve.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void zfwd_item(const Grid& g, const T* __restrict__ W, const T* __restrict__ Q, double* __restrict__ F,
                          size_t S, int B, int tm, int nch, const int* nsteps, int stepidx, int blk) {
  using V = C2<T>;
  extern __shared__ __align__(16) unsigned char fsm[];
  V* fold = reinterpret_cast<V*>(fsm);                 // [2][Mh][tm]
  const int Mh = (g.Mz + 1) / 2;
  const int mt = (g.nm + tm - 1) / tm;
  const int per_b = 2 * mt * nch;
  const int b = blk / per_b;
  int rem = blk - b * per_b;
  const int ch = rem % nch;
  rem /= nch;
  const int f = rem / mt, m0 = (rem - f * mt) * tm;
  if (b >= B || !slice_active_at(nsteps, stepidx, b)) return;
  const size_t qs = (size_t)g.Mz * g.nm * 2;
  const T* q = Q + (size_t)(b * 2 + f) * qs;
  const int ltm = __ffs(tm) - 1;             // tm is a power of two
  for (int it = threadIdx.x; it < Mh * tm; it += blockDim.x) {
    const int jh = it >> ltm, mi = it & (tm - 1), m = m0 + mi;
    V ev = mk2<T>(0, 0), od = mk2<T>(0, 0);
    if (m < g.nm) {
      const V a = ldc<T>(q + ((size_t)jh * g.nm + m) * 2);
      const int jr = g.Mz - 1 - jh;
      if (jr != jh) {
        const V c = ldc<T>(q + ((size_t)jr * g.nm + m) * 2);
        ev = a + c;
        od = a - c;
      } else {
        ev = a;
      }
    }
    fold[(size_t)jh * tm + mi] = ev;
    fold[(size_t)(Mh + jh) * tm + mi] = od;
  }
  __syncthreads();
  const int ng = blockDim.x >> ltm;
  const int mi = threadIdx.x & (tm - 1), n0 = threadIdx.x >> ltm;
  const int m = m0 + mi;
  if (m >= g.nm) return;
  const int nper = (g.Nz + nch - 1) / nch;
  const int nlo = ch * nper, nhi = min(g.Nz, nlo + nper);
  for (int n = nlo + n0; n < nhi; n += ng) {
    const V* src = fold + (size_t)((n & 1) ? Mh : 0) * tm + mi;
    const T* wr = W + (size_t)n * g.Mz;
    V acc = mk2<T>(0, 0);
#pragma unroll 4
    for (int jh = 0; jh < Mh; ++jh) {
      const T wv = __ldg(wr + jh);
      const V v = src[(size_t)jh * tm];
      acc.x = fma(wv, v.x, acc.x);
      acc.y = fma(wv, v.y, acc.y);
    }
    st2(F + (size_t)b * S + soff(g, f, n, m), make_double2((double)acc.x, (double)acc.y));
  }
}

template <typename T>
__global__ void k_zfwd(Grid g, const T* __restrict__ W, const T* __restrict__ Q, double* __restrict__ F, size_t S,
                       int B, int tm, int nch, const int* nsteps, const int* step) {
  pdl_wait();
  zfwd_item<T>(g, W, Q, F, S, B, tm, nch, nsteps, nsteps ? *step : 0, blockIdx.x);
}

static int zfwd_tile(const Grid& g, int B, size_t es) {
  const int Mh = (g.Mz + 1) / 2;
  int tm = 32;
  while (tm > 1 && (size_t)B * 2 * ((g.nm + tm - 1) / tm) < 2 * 152) tm >>= 1;
  while (tm > 4 && (size_t)2 * Mh * tm * 2 * es > 200 * 1024) tm >>= 1;
  return tm;
}
static int zfwd_chunks(const Grid& g, int B, int tm) {
  const long blocks = (long)B * 2 * ((g.nm + tm - 1) / tm);
  int nch = 1;
  while (nch < 8 && blocks * nch < 4L * 152 && g.Nz / (2 * nch) >= 128 / tm) nch *= 2;
  return nch;
}
static size_t zfwd_smem(const Grid& g, int B, size_t es) {
  return (size_t)2 * ((g.Mz + 1) / 2) * zfwd_tile(g, B, es) * 2 * es;
}

// ---------------------------------------------------------------------------
// Stage solve (k_solve).  Block per (slice, Chebyshev parity p, tile of tms
// Fourier modes); a column is one (mode m, real/imaginary part c) pair -- the
// stage matrices are real, so the two parts are independent systems except for
// the implicit buoyancy coupling -i k Pr Ra T (the imaginary part of T feeds
// the real part of psi and vice versa).  Per system (T first, then psi for
// m >= 1 or the mean flow U for m = 0):
//   phase 1 (all threads, one tau row of one column each): right-hand side of
//           the stage, updates of the later RK accumulators;
//   phase 2 (one thread per column): backward elimination with the UL factors;
//   phase 3 (same thread): boundary block, forward substitution;
//   phase 4 (all threads): dt L X_i = (M X_i - r_i) / gamma into later accumulators.
// Phase 1 reads F and the step-start state straight from global memory
// (consecutive threads take consecutive (m, re/im) columns, so the loads
// coalesce); the right-hand sides, r_i and T_i live in shared memory, three
// arrays of nq x 2 tms doubles, so that more blocks share an SM.
// ---------------------------------------------------------------------------
enum { KT = 0, KP = 1, KU = 2 };

struct SolveSmem {
  const double* F;   // explicit terms of this slice (global; read in phase 1, coalesced over the columns)
  const double* X;   // step-start state of this slice (global; stage 1)
  double* y;    // [nq][W] right-hand side, then solution
  double* r;    // [nq][W] r_i of the tau rows
  double* T;    // [nq][W] T_i, kept for the psi coupling; the dense path's solution of each system
  int W;        // columns = 2 * tms
  double Ra;    // Rayleigh number of this slice
  double cpl;   // ((gamma dt) Pr) Ra of this slice
};

template <int KIND>
struct Sys {
  static constexpr int D = (KIND == KP) ? 2 : 1;
  static constexpr int LAM = 2 * D;
  static __device__ __forceinline__ const double* multB(const Tables& tb) {
    return KIND == KT ? tb.T_multB : KIND == KP ? tb.P_multB : tb.U_multB;
  }
  static __device__ __forceinline__ const double* multD(const Tables& tb) {
    return KIND == KT ? tb.T_multD : KIND == KP ? tb.P_multD : tb.U_multD;
  }
  static __device__ __forceinline__ const double* Dinv(const Tables& tb) {
    return KIND == KT ? tb.T_Dinv : KIND == KP ? tb.P_Dinv : tb.U_Dinv;
  }
  static __device__ __forceinline__ const double* Lb(const Tables& tb) {
    return KIND == KT ? tb.T_Lb : KIND == KP ? tb.P_Lb : tb.U_Lb;
  }
  static __device__ __forceinline__ const double* invd(const Tables& tb) {
    return KIND == KT ? tb.T_invd : KIND == KP ? tb.P_invd : tb.U_invd;
  }
  static __device__ __forceinline__ double tapF(const Grid& g, const Tables& tb, int p, int t, int j) {
    return KIND == KP ? __ldg(tb.s4 + (p * g.nq + t) * 5 + j) : __ldg(tb.s2 + (p * g.nq + t) * 3 + j);
  }
  static __device__ __forceinline__ double tapM(const Grid& g, const Tables& tb, int p, int t, int j, int m) {
    return KIND == KP ? __ldg(tb.mp + ((size_t)(p * g.nq + t) * 5 + j) * g.nm + m)
                      : __ldg(tb.s2 + (p * g.nq + t) * 3 + j);
  }
};

// phase 1 for one (tau row t, column col)
template <int KIND>
__device__ __forceinline__ void solve_rhs(const Grid& g, const Tables& tb, int stage, int p, int m, int c, int t,
                                          int col, const SolveSmem& sm, double* __restrict__ R, size_t S) {
  using SY = Sys<KIND>;
  const int nq = g.nq, W = sm.W;
  const int f = (KIND == KT) ? 0 : 1;
  double fv = 0.0;
#pragma unroll
  for (int j = 0; j <= SY::LAM; ++j)
    if (t + j < nq) fv = fma(SY::tapF(g, tb, p, t, j), sm.F[soff(g, f, 2 * (t + j) + p, m) + c], fv);
  if (KIND != KP) fv = -fv;
  const int ns = g.ns;
  const size_t ro = soff(g, f, 2 * t + p, m) + c;
  double r;
  if (stage == 1) {
    double mx = 0.0;
#pragma unroll
    for (int j = 0; j <= SY::LAM; ++j)
      if (t + j < nq) mx = fma(SY::tapM(g, tb, p, t, j, m), sm.X[soff(g, f, 2 * (t + j) + p, m) + c], mx);
    r = fma(__ldg(tb.dtae + 5), fv, mx);
#pragma unroll
    for (int l = 2; l <= 4; ++l)
      if (l <= ns) R[(size_t)(l - 1) * S + ro] = fma(__ldg(tb.dtae + l * 5), fv, mx);
  } else {
    double Rl[3];
    const double Ri = *(R + (size_t)(stage - 1) * S + ro);
#pragma unroll
    for (int l = 0; l < 3; ++l) Rl[l] = (l + 2 > stage && l + 2 <= ns) ? *(R + (size_t)(l + 1) * S + ro) : 0.0;
    r = fma(__ldg(tb.dtae + stage * 5 + stage - 1), fv, Ri);
#pragma unroll
    for (int l = 0; l < 3; ++l)
      if (l + 2 > stage && l + 2 <= ns)
        R[(size_t)(l + 1) * S + ro] = fma(__ldg(tb.dtae + (l + 2) * 5 + stage - 1), fv, Rl[l]);
  }
  sm.r[t * W + col] = r;
  double bv = r;
  if (KIND == KP) {
    // + gamma dt (-i k Pr Ra) S4 T_i: real part + k.. Im(S4 T), imaginary part - k.. Re(S4 T)
    double st = 0.0;
#pragma unroll
    for (int j = 0; j <= 4; ++j)
      if (t + j < nq) st = fma(__ldg(tb.s4 + (p * nq + t) * 5 + j), sm.T[(t + j) * W + (col ^ 1)], st);
    // (+-1) gamma dt Pr Ra k with the roundings of that left-to-right product:
    // the sign is exact, so it may come last
    const double cpl = (c == 0 ? sm.cpl : -sm.cpl) * (g.kfac * m);
    bv = fma(cpl, st, bv);
  }
  sm.y[(t + SY::D) * W + col] = bv;
}

// phases 2 and 3 for one column
template <int KIND>
__device__ __forceinline__ bool solve_recurrence(const Grid& g, const Tables& tb, int p, int m, int c, int col,
                                                 const SolveSmem& sm, double* __restrict__ Xo) {
  using SY = Sys<KIND>;
  constexpr int D = SY::D;
  const int nq = g.nq, W = sm.W;
  const int f = (KIND == KT) ? 0 : 1;
  const int nmod = (KIND == KU) ? 1 : g.nm;
  const int mi = (KIND == KU) ? 0 : m;
  const double* multB = SY::multB(tb);
  const double* multD = SY::multD(tb);
  auto tix = [&](int cc, int jj) { return ((size_t)(p * nq + cc) * D + jj) * nmod + mi; };
  // The factor entries of RC consecutive steps are loaded together before the
  // steps run, so the sequential chain does not wait on one load per step.
  constexpr int RC = 8;
  double pend[D], bd[D];
#pragma unroll
  for (int jj = 0; jj < D; ++jj) pend[jj] = bd[jj] = 0.0;
  for (int c0 = nq - 1; c0 >= D; c0 -= RC) {
    double mb[RC][D], md[RC][D];
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      const int cc = c0 - k;
#pragma unroll
      for (int jj = 0; jj < D; ++jj) {
        mb[k][jj] = (cc >= D) ? __ldg(multB + tix(cc, jj)) : 0.0;
        md[k][jj] = (cc >= D) ? __ldg(multD + tix(cc, jj)) : 0.0;
      }
    }
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      const int cc = c0 - k;
      if (cc < D) break;
      const double bc = sm.y[cc * W + col] + pend[0];
      sm.y[cc * W + col] = bc;
#pragma unroll
      for (int jj = 0; jj < D - 1; ++jj) pend[jj] = fma(-mb[k][D - 1 - jj], bc, pend[jj + 1]);
      pend[D - 1] = -mb[k][0] * bc;
#pragma unroll
      for (int r2 = 0; r2 < D; ++r2) bd[r2] = fma(-md[k][r2], bc, bd[r2]);
    }
  }
  // boundary rows: parity combinations of the wall values (Eq. 6) or slopes (Eq. 7)
  if (KIND == KT && m == 0 && c == 0) bd[0] += t_wall_rhs(g, p);
  const double* Dinv = SY::Dinv(tb);
  const double* Lb = SY::Lb(tb);
  const double* invd = SY::invd(tb);
  double win[D];
  bool ok = true;
#pragma unroll
  for (int r2 = 0; r2 < D; ++r2) {
    double x = 0.0;
#pragma unroll
    for (int c2 = 0; c2 < D; ++c2) x = fma(__ldg(Dinv + ((size_t)(p * D * D) + r2 * D + c2) * nmod + mi), bd[c2], x);
    win[r2] = x;
    sm.y[r2 * W + col] = x;
    Xo[soff(g, f, 2 * r2 + p, m) + c] = x;
    if (KIND == KT) sm.T[r2 * W + col] = x;
    ok = ok && isfinite(x);
  }
  for (int r0 = D; r0 < nq; r0 += RC) {
    double lb[RC][D], iv[RC];
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      const int r2 = r0 + k;
#pragma unroll
      for (int jj = 0; jj < D; ++jj) lb[k][jj] = (r2 < nq) ? __ldg(Lb + tix(r2, jj)) : 0.0;
      iv[k] = (r2 < nq) ? __ldg(invd + (size_t)(p * nq + r2) * nmod + mi) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < RC; ++k) {
      const int r2 = r0 + k;
      if (r2 >= nq) break;
      double y = sm.y[r2 * W + col];
#pragma unroll
      for (int jj = 0; jj < D; ++jj) y = fma(-lb[k][jj], win[jj], y);
      const double x = iv[k] * y;
      sm.y[r2 * W + col] = x;
      Xo[soff(g, f, 2 * r2 + p, m) + c] = x;
      if (KIND == KT) sm.T[r2 * W + col] = x;
#pragma unroll
      for (int jj = 0; jj < D - 1; ++jj) win[jj] = win[jj + 1];
      win[D - 1] = x;
      ok = ok && isfinite(x);
    }
  }
  return ok;
}

// phases 2-3 for small grids: x_r = sum_q Ainv[r][q] b_q for one (row r, column
// col); b holds the boundary values in rows 0 .. D-1 and the tau right-hand
// sides below them.
template <int KIND>
__device__ __forceinline__ bool solve_dense(const Grid& g, const Tables& tb, int p, int m, int c, int r, int col,
                                            const SolveSmem& sm, double* __restrict__ Xo) {
  const int nq = g.nq, W = sm.W;
  const int f = (KIND == KT) ? 0 : 1;
  const int nmod = (KIND == KU) ? 1 : g.nm;
  const int mi = (KIND == KU) ? 0 : m;
  const double* inv = (KIND == KT) ? tb.T_inv : (KIND == KP) ? tb.P_inv : tb.U_inv;
  const double* row = inv + ((size_t)p * nq + r) * nq * nmod + mi;
  double acc0 = 0.0, acc1 = 0.0;                       // two partial sums: shorter chain
  for (int q = 0; q + 1 < nq; q += 2) {
    acc0 = fma(__ldg(row + (size_t)q * nmod), sm.y[q * W + col], acc0);
    acc1 = fma(__ldg(row + (size_t)(q + 1) * nmod), sm.y[(q + 1) * W + col], acc1);
  }
  if (nq & 1) acc0 = fma(__ldg(row + (size_t)(nq - 1) * nmod), sm.y[(nq - 1) * W + col], acc0);
  const double x = acc0 + acc1;
  sm.T[r * W + col] = x;
  Xo[soff(g, f, 2 * r + p, m) + c] = x;
  return isfinite(x);
}

// phase 4 for one (tau row t, column col)
template <int KIND>
__device__ __forceinline__ void solve_lx(const Grid& g, const Tables& tb, int stage, int p, int m, int c, int t,
                                         int col, const SolveSmem& sm, const double* xs, double* __restrict__ R,
                                         size_t S) {
  using SY = Sys<KIND>;
  const int nq = g.nq, W = sm.W;
  const int f = (KIND == KT) ? 0 : 1;
  double mx = 0.0;
#pragma unroll
  for (int j = 0; j <= SY::LAM; ++j)
    if (t + j < nq) mx = fma(SY::tapM(g, tb, p, t, j, m), xs[(t + j) * W + col], mx);
  const double lx2 = g.inv_gamma * (mx - sm.r[t * W + col]);   // dt (L X_i + coupling)
  const size_t ro = soff(g, f, 2 * t + p, m) + c;
#pragma unroll
  for (int l = 0; l < 3; ++l)
    if (l + 2 > stage && l + 2 <= g.ns) {
      double* Rl = R + (size_t)(l + 1) * S + ro;
      *Rl = fma(c_AI[g.scheme][l + 2][stage], lx2, *(Rl));
    }
}

__device__ void solve_item(const Grid& g, const Tables& tb, double* X, double* Xs, const double* F, double* R,
                           size_t S, const double* wT, double* nu, int* flags, int* err, int B, int stage, int tms,
                           const double* ra, const int* nsteps, int stepidx, int blk) {
  extern __shared__ double sbuf[];
  const int mt = (g.nm + tms - 1) / tms;
  const int b = blk / (2 * mt);
  const int rem = blk - b * 2 * mt;
  const int p = rem / mt;
  const int m0 = (rem - p * mt) * tms;
  if (b >= B || !slice_active_at(nsteps, stepidx, b)) return;   // uniform per block
  // a transform of this state gave up waiting (the tensor-core kernels): leave
  // the state as it was at the start of the failing step
  if (flags[b] & kFlagTimeout) return;
  const int nq = g.nq;
  const int W = 2 * tms;                         // a power of two (tms is)
  const int lw = __ffs(W) - 1;
  const int ncol = 2 * min(tms, g.nm - m0);
  SolveSmem sm;
  sm.W = W;
  sm.Ra = ra ? ra[b] : g.Ra;
  sm.cpl = __ldg(tb.dtae + 25) * sm.Ra;
  sm.y = sbuf;
  sm.r = sm.y + (size_t)nq * W;
  sm.T = sm.r + (size_t)nq * W;
  double* X0 = X + (size_t)b * S;
  double* Xo = (stage == g.ns) ? X0 : Xs + (size_t)b * S;   // stiffly accurate: last stage = new state
  const double* Fb = F + (size_t)b * S;
  sm.F = Fb;
  sm.X = X0;
  double* Rb = R + (size_t)b * 4 * S;
  if (stage == 1 && m0 == 0 && p == 1 && threadIdx.x < 32 && nu != nullptr) {
    // Nu_V(t_n) (Eq. 9) of the step-start state: wall temperature difference of
    // the mean profile + Clenshaw-Curtis integral of <wT>_x; trapezoid weight.
    // The first warp sums it: each lane a strided share of both sums, then a
    // fixed shuffle tree (the order depends on the grid only). The odd
    // coefficients read here belong to this block, which overwrites them only
    // after the barriers below (a one-stage scheme writes X0 here).
    const int lane = threadIdx.x;
    double cond = 0.0, adv = 0.0;
    for (int n = 2 * lane + 1; n < g.Nz; n += 64) cond -= 2.0 * *(X0 + soff(g, 0, n, 0));
    for (int jz = lane; jz < g.Mz; jz += 32) adv = fma(__ldg(tb.cc + jz), *(wT + (size_t)b * g.Mz + jz), adv);
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
      cond += __shfl_down_sync(0xffffffffu, cond, sh);
      adv += __shfl_down_sync(0xffffffffu, adv, sh);
    }
    if (lane == 0) nu[b] += ((stepidx == 0) ? 0.5 : 1.0) * g.dt * (cond + 0.5 * adv);
  }
  bool ok = true;
  for (int sys = 0; sys < 2; ++sys) {
    const int f = sys;                               // field 0 = T, 1 = psi / U
    // phase 1
    const int ntmax = nq - 1;
    for (int it = threadIdx.x; it < ntmax * W; it += blockDim.x) {
      const int t = it >> lw, col = it & (W - 1);
      if (col >= ncol) continue;
      const int m = m0 + col / 2, c = col & 1;
      if (sys == 0)
        solve_rhs<KT>(g, tb, stage, p, m, c, t, col, sm, Rb, S);
      else if (m == 0)
        solve_rhs<KU>(g, tb, stage, p, m, c, t, col, sm, Rb, S);
      else if (t < nq - 2)
        solve_rhs<KP>(g, tb, stage, p, m, c, t, col, sm, Rb, S);
    }
    __syncthreads();
    const bool dense = g.nq <= kDenseSolveMaxNq;
    if (dense) {
      // boundary rows of b: the mean temperature's wall values (Eq. 6) or
      // slopes (Eq. 7) in parity combinations; zero for T at m >= 1, psi and U
      for (int it = threadIdx.x; it < 2 * W; it += blockDim.x) {
        const int r = it >> lw, col = it & (W - 1);
        if (col >= ncol) continue;
        const int m = m0 + col / 2, c = col & 1;
        const int D = (sys == 1 && m != 0) ? 2 : 1;
        if (r >= D) continue;
        sm.y[r * W + col] = (sys == 0 && m == 0 && c == 0) ? t_wall_rhs(g, p) : 0.0;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < nq * W; it += blockDim.x) {
        const int r = it >> lw, col = it & (W - 1);
        if (col >= ncol) continue;
        const int m = m0 + col / 2, c = col & 1;
        bool o2;
        if (sys == 0)
          o2 = solve_dense<KT>(g, tb, p, m, c, r, col, sm, Xo);
        else if (m == 0)
          o2 = solve_dense<KU>(g, tb, p, m, c, r, col, sm, Xo);
        else
          o2 = solve_dense<KP>(g, tb, p, m, c, r, col, sm, Xo);
        ok = ok && o2;
      }
    } else if ((int)threadIdx.x < ncol) {
      // phases 2, 3: one column per thread, columns packed into the fewest warps
      // (an FP64 warp instruction occupies its sub-partition's FP64 pipe for the
      // same time however many lanes are active, so packing is cheapest)
      const int col = threadIdx.x, m = m0 + col / 2, c = col & 1;
      bool o2;
      if (sys == 0)
        o2 = solve_recurrence<KT>(g, tb, p, m, c, col, sm, Xo);
      else if (m == 0)
        o2 = solve_recurrence<KU>(g, tb, p, m, c, col, sm, Xo);
      else
        o2 = solve_recurrence<KP>(g, tb, p, m, c, col, sm, Xo);
      ok = ok && o2;
    }
    __syncthreads();
    const double* xs = dense ? sm.T : sm.y;
    // phase 4
    if (stage < g.ns) {
      for (int it = threadIdx.x; it < ntmax * W; it += blockDim.x) {
        const int t = it >> lw, col = it & (W - 1);
        if (col >= ncol) continue;
        const int m = m0 + col / 2, c = col & 1;
        if (sys == 0)
          solve_lx<KT>(g, tb, stage, p, m, c, t, col, sm, xs, Rb, S);
        else if (m == 0)
          solve_lx<KU>(g, tb, stage, p, m, c, t, col, sm, xs, Rb, S);
        else if (t < nq - 2)
          solve_lx<KP>(g, tb, stage, p, m, c, t, col, sm, xs, Rb, S);
      }
    }
    __syncthreads();
  }
  if (!ok) {
    atomicOr(flags + b, kFlagNonFinite);
    atomicOr(err, kFlagNonFinite);
  }
}

__global__ void __launch_bounds__(256) k_solve(Grid g, Tables tb, double* X, double* Xs, const double* F, double* R,
                                               size_t S, const double* wT, double* nu, int* flags, int* err, int B,
                                               int stage, int tms, const double* ra, const int* nsteps,
                                               const int* step) {
  pdl_wait();
  solve_item(g, tb, X, Xs, F, R, S, wT, nu, flags, err, B, stage, tms, ra, nsteps, nsteps ? *step : 0, blockIdx.x);
}

// Modes per k_solve block.  Every column's arithmetic is independent of the
// tiling, so a small batch (a coarse sweep) takes single-mode tiles and spreads
// over the SMs instead of leaving most of them idle.
// shared memory of a k_solve block: y, r and T, nq x 2 tms doubles each
static size_t solve_smem_tms(const Grid& g, int tms) { return (size_t)3 * g.nq * 2 * tms * 8; }
static int solve_tile(const Grid& g, int B) {
  int tms = 16;
  while (tms > 1 && (long)B * 2 * ((g.nm + tms - 1) / tms) < 2L * 152) tms >>= 1;
  if (tms > g.nm) tms = g.nm;
  while (tms > 1 && solve_smem_tms(g, tms) > 200 * 1024) tms >>= 1;
  return tms;
}
// threads of a k_solve block: one per (row, column) of the tile, whole warps, at most 256
static int solve_threads(const Grid& g, int tms) {
  const int items = g.nq * 2 * tms;
  return std::min(256, std::max(32, (items + 31) / 32 * 32));
}
static size_t solve_smem(const Grid& g, int B) { return solve_smem_tms(g, solve_tile(g, B)); }

// The shapes of a launch: the tuned ones where set, else the heuristics.
static int solve_tms_of(const Grid& g, const Work& w, int B) {
  return (w.shapes && w.shapes->solve_tms > 0) ? w.shapes->solve_tms : solve_tile(g, B);
}
static int zfwd_tm_of(const Grid& g, const Work& w, int B, size_t es) {
  return (w.shapes && w.shapes->zfwd_tm > 0) ? w.shapes->zfwd_tm : zfwd_tile(g, B, es);
}
static int zfwd_nch_of(const Grid& g, const Work& w, int B, int tm) {
  return (w.shapes && w.shapes->zfwd_nch > 0) ? w.shapes->zfwd_nch : zfwd_chunks(g, B, tm);
}
static bool rows_cl_of(const Grid& g, const Work& w, int B, size_t es) {
  return (w.shapes && w.shapes->rows_cl >= 0) ? w.shapes->rows_cl != 0 : rows_use_cluster(g, B, es);
}
static int rows_threads_of(const Work& w) {
  return (w.shapes && w.shapes->rows_threads > 0) ? w.shapes->rows_threads : kRowsThreads;
}
static bool rows_lean_of(const Grid& g, const Work& w, size_t es) {
  return (w.shapes && w.shapes->rows_lean >= 0) ? w.shapes->rows_lean != 0 : rows_lean_default(g, es);
}

bool shapes_valid(const Grid& g, const Shapes& sh, size_t es) {
  if (sh.solve_tms > 0 && (sh.solve_tms > 16 || (sh.solve_tms & (sh.solve_tms - 1)) ||
                           solve_smem_tms(g, sh.solve_tms) > 200 * 1024))
    return false;
  if (sh.zfwd_tm > 0 && (sh.zfwd_tm > 32 || (sh.zfwd_tm & (sh.zfwd_tm - 1)) ||
                         (size_t)2 * ((g.Mz + 1) / 2) * sh.zfwd_tm * 2 * es > 200 * 1024))
    return false;
  if (sh.zfwd_nch > 0 && (sh.zfwd_nch > 8 || (sh.zfwd_nch & (sh.zfwd_nch - 1)))) return false;
  if (sh.rows_cl == 1 && rows_cl_bytes(g, es) > 200 * 1024) return false;
  if (sh.rows_threads != 0 && sh.rows_threads != 256 && sh.rows_threads != 512 && sh.rows_threads != 1024)
    return false;
  if (sh.rows_lean < -1 || sh.rows_lean > 1 || (sh.rows_lean == 1 && !rows_batched(g, es))) return false;
  return true;
}

__global__ void k_advance(int* step) {
  pdl_wait();
  *step += 1;
}

// Body end of the device-side step loop: the loop ends once every state of the
// batch has taken its steps (maxs is written by the host before each launch).
// cancel (may be null): a word another stream sets to stop the loop early
// (work whose result is no longer wanted, e.g. a speculative Parareal iteration)
__global__ void k_advance_loop(int* step, const int* maxs, const int* cancel, cudaGraphConditionalHandle loop) {
  pdl_wait();
  const int s = *step + 1;
  *step = s;
  const bool stop = cancel != nullptr && *(const volatile int*)cancel != 0;
  cudaGraphSetConditional(loop, (s < *maxs && !stop) ? 1u : 0u);
}

static inline unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

static std::atomic<unsigned long long> g_launches{0};
unsigned long long launches_so_far() { return g_launches.load(); }
void add_launches(unsigned long long n) { g_launches.fetch_add(n); }
static inline void count(int n = 1) { g_launches.fetch_add(n); }

cudaError_t Prof::fold() {
  for (size_t i = 0; i < used; ++i) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    e = cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    ms[kind[i]] += t;
  }
  used = 0;
  return cudaSuccess;
}

void Prof::begin(int k, cudaStream_t s) {
  if (used * 2 + 2 > ev.size()) {
    if (ev.size() >= 8192) {
      fold();
    } else {
      for (int i = 0; i < 256; ++i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ev.push_back(e);
      }
      kind.resize(ev.size() / 2);
    }
  }
  kind[used] = k;
  cudaEventRecord(ev[2 * used], s);
}

void Prof::end(int k, cudaStream_t s, double fl, double by) {
  cudaEventRecord(ev[2 * used + 1], s);
  ++used;
  launches[k] += 1;
  flops[k] += fl;
  bytes[k] += by;
}

// Algorithmic work of one launch over B slices (all active).
static double zinv_flops(const Grid& g, int B) { return 24.0 * B * ((g.Mz + 1) / 2) * g.nm * g.Nz; }
static double zinv_bytes(const Grid& g, int B, size_t es = 8) {
  return 8.0 * B * state_doubles(g) + (double)es * B * z_doubles(g);
}
static double rows_flops(const Grid& g, int B) {
  return (double)B * g.Mz * (6.0 * 5.0 * g.Mx * std::log2((double)g.Mx) + 10.0 * g.Mx);
}
static double rows_bytes(const Grid& g, int B, size_t es = 8) {
  return (double)es * B * (z_doubles(g) + q_doubles(g)) + 8.0 * B * g.Mz;
}
static double zfwd_flops(const Grid& g, int B) { return 4.0 * B * g.Nz * g.nm * ((g.Mz + 1) / 2) * 2.0; }
static double zfwd_bytes(const Grid& g, int B, size_t es = 8) {
  return (double)es * B * q_doubles(g) + 8.0 * B * state_doubles(g);
}
// stage solve: per (m, parity) about 60 flops per coefficient row for T and psi;
// reads F, X and up to four accumulators, writes X and the accumulators
static double solve_flops(const Grid& g, int B) { return 120.0 * B * g.nm * 2.0 * g.nq * 2.0; }
static double solve_bytes(const Grid& g, int B) { return 8.0 * B * state_doubles(g) * 10.0; }

// The dynamic shared-memory allowance of k_rows only ever grows, so that a
// later handle on a smaller grid does not shrink it below an earlier one's need.
// The dynamic shared-memory allowances only ever grow, so that a later handle
// on a smaller grid does not shrink them below an earlier one's need.
template <typename F>
static cudaError_t allow_smem(F* fn, int need, int& allowed) {
  if (need <= allowed) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
  if (e == cudaSuccess) allowed = need;
  return e;
}

cudaError_t configure_kernels(const Grid& g) {
  static int a_rows_d = 48 * 1024, a_rows_f = 48 * 1024, a_solve = 48 * 1024;
  static int a_zfwd_d = 48 * 1024, a_zfwd_f = 48 * 1024;
  static int a_rcl_d = 48 * 1024, a_rcl_f = 48 * 1024;
  cudaError_t e = allow_smem(k_rows<double>, (int)rows_smem_for(g, 8, false), a_rows_d);
  if (e == cudaSuccess && rows_cl_bytes(g, 8) <= 200 * 1024)
    e = allow_smem(k_rows_cl<double>, (int)rows_cl_bytes(g, 8), a_rcl_d);
  if (e == cudaSuccess && rows_cl_bytes(g, 4) <= 200 * 1024)
    e = allow_smem(k_rows_cl<float>, (int)rows_cl_bytes(g, 4), a_rcl_f);
  if (e == cudaSuccess) e = allow_smem(k_rows<float>, (int)rows_smem_for(g, 4, false), a_rows_f);
  if (e == cudaSuccess)
    e = allow_smem(k_solve, (int)std::max(solve_smem(g, 1), solve_smem(g, 1 << 20)), a_solve);
  if (e == cudaSuccess)
    e = allow_smem(k_zfwd<double>, (int)std::max(zfwd_smem(g, 1, 8), zfwd_smem(g, 1 << 20, 8)), a_zfwd_d);
  if (e == cudaSuccess)
    e = allow_smem(k_zfwd<float>, (int)std::max(zfwd_smem(g, 1, 4), zfwd_smem(g, 1 << 20, 4)), a_zfwd_f);
  return e;
}

template <typename T>
static void launch_transforms_in(const Grid& g, const Tables& t, const T* Bz, const C2<T>* tw, const Work& w,
                                 const double* X, int B, const int* ns, Prof* pf, cudaStream_t s) {
  const size_t S = state_doubles(g);
  const int kp = zinv_warps(g);
  const unsigned zb = (unsigned)(B * ((g.Mz + 1) / 2) * ((g.nm + 31) / 32));
  T* Z = reinterpret_cast<T*>(w.Z);
  T* Q = reinterpret_cast<T*>(w.Q);
  if (pf) pf->begin(RBC_KERNEL_ZINV, s);
  if (sizeof(T) == 4 && t.tcA_psi_hi != nullptr)
    launch_zinv_tc(g, t, w, X, B, ns, s);              // tensor cores, TF32 with split compensation
  else
    launch_pdl(w.pdl != 0, k_zinv<T>, zb, 32 * kp, kp > 1 ? (size_t)kp * 12 * 32 * 2 * sizeof(T) : 0, s, g, Bz, X,
               S, Z, B, ns, w.step);
  if (pf) pf->end(RBC_KERNEL_ZINV, s, zinv_flops(g, B), zinv_bytes(g, B, sizeof(T)));
  const size_t es = sizeof(T);
  if (pf) pf->begin(RBC_KERNEL_ROWS, s);
  if (rows_cl_of(g, w, B, es))
    launch_pdl(w.pdl != 0, k_rows_cl<T>, (unsigned)(B * g.Mz * kRowsCluster), kRowsThreads, rows_cl_bytes(g, es), s,
               g, tw, Z, Q, w.wT, B, ns, w.step);
  else
    launch_pdl(w.pdl != 0, k_rows<T>, (unsigned)(B * g.Mz), rows_threads_of(w),
               rows_smem_for(g, es, rows_lean_of(g, w, es)), s, g, tw, Z, Q, w.wT, B, rows_batched(g, es) ? 1 : 0,
               rows_lean_of(g, w, es) ? 1 : 0, ns, w.step);
  if (pf) pf->end(RBC_KERNEL_ROWS, s, rows_flops(g, B), rows_bytes(g, B, sizeof(T)));
}

cudaError_t launch_explicit(const Grid& g, const Tables& t, const Work& w, const double* X, int B, bool all_active,
                            cudaStream_t s) {
  const int* ns = all_active ? nullptr : w.nsteps;
  Prof* pf = (w.prof && w.prof->on && !all_active) ? w.prof : nullptr;
  if (g.mixed)
    launch_transforms_in<float>(g, t, t.zinv32, t.tw32, w, X, B, ns, pf, s);
  else
    launch_transforms_in<double>(g, t, t.zinv, t.tw, w, X, B, ns, pf, s);
  count(2);
  return cudaGetLastError();
}

template <typename T>
static void launch_zfwd(const Grid& g, const T* W, const Work& w, int B, Prof* pf, cudaStream_t s) {
  const size_t S = state_doubles(g), es = sizeof(T);
  const int tm = zfwd_tm_of(g, w, B, es);
  const int mt = (g.nm + tm - 1) / tm;
  const int nch = zfwd_nch_of(g, w, B, tm);
  const size_t smem = (size_t)2 * ((g.Mz + 1) / 2) * tm * 2 * es;
  if (pf) pf->begin(RBC_KERNEL_ZFWD, s);
  launch_pdl(w.pdl != 0, k_zfwd<T>, (unsigned)(B * 2 * mt * nch), 128, smem, s, g, W, reinterpret_cast<const T*>(w.Q),
             w.F, S, B, tm, nch, w.nsteps, w.step);
  if (pf) pf->end(RBC_KERNEL_ZFWD, s, zfwd_flops(g, B), zfwd_bytes(g, B, es));
}

cudaError_t launch_stage(const Grid& g, const Tables& t, const Work& w, double* X, int B, int stage, double* nu,
                         cudaStream_t s) {
  const size_t S = state_doubles(g);
  const double* Xin = (stage == 1) ? X : w.Xs;
  cudaError_t e = launch_explicit(g, t, w, Xin, B, false, s);
  if (e != cudaSuccess) return e;
  Prof* pf = (w.prof && w.prof->on) ? w.prof : nullptr;
  if (g.mixed && t.tcW_hi[0] != nullptr) {
    // tensor cores, TF32 with split compensation
    if (pf) pf->begin(RBC_KERNEL_ZFWD, s);
    launch_zfwd_tc(g, t, w, B, s);
    if (pf) pf->end(RBC_KERNEL_ZFWD, s, zfwd_flops(g, B), zfwd_bytes(g, B, 4));
  } else if (g.mixed)
    launch_zfwd<float>(g, t.zfwd32, w, B, pf, s);
  else
    launch_zfwd<double>(g, t.zfwd, w, B, pf, s);
  const int tms = solve_tms_of(g, w, B);
  const int mtiles = (g.nm + tms - 1) / tms;
  if (pf) pf->begin(RBC_KERNEL_SOLVE, s);
  launch_pdl(w.pdl != 0, k_solve, (unsigned)(B * 2 * mtiles), solve_threads(g, tms), solve_smem_tms(g, tms), s, g, t,
             X, w.Xs, w.F, w.R, S, w.wT, nu, w.flags, w.err, B, stage, tms, w.ra, w.nsteps, w.step);
  if (pf) pf->end(RBC_KERNEL_SOLVE, s, solve_flops(g, B), solve_bytes(g, B));
  count(2);
  return cudaGetLastError();
}

cudaError_t launch_advance(const Work& w, cudaStream_t s) {
  launch_pdl(w.pdl != 0, k_advance, 1, 1, 0, s, w.step);
  count();
  return cudaGetLastError();
}

cudaError_t launch_advance_loop(const Work& w, cudaGraphConditionalHandle loop, cudaStream_t s) {
  launch_pdl(w.pdl != 0, k_advance_loop, 1, 1, 0, s, w.step, w.maxs, w.cancel, loop);
  count();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostics.
// ---------------------------------------------------------------------------
__global__ void k_nu_final(Grid g, const double* cc, const double* X, size_t S, const double* wT, double* nu,
                           const int* nsteps, const int* flags, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || nsteps[b] <= 0 || (flags[b] & kFlagTimeout)) return;
  const double* X0 = X + (size_t)b * S;
  double cond = 0.0;
  for (int n = 1; n < g.Nz; n += 2) cond -= 2.0 * X0[soff(g, 0, n, 0)];
  double adv = 0.0;
  for (int jz = 0; jz < g.Mz; ++jz) adv = fma(cc[jz], wT[(size_t)b * g.Mz + jz], adv);
  nu[b] += 0.5 * g.dt * (cond + 0.5 * adv);
}

cudaError_t launch_nu_final(const Grid& g, const Tables& t, const Work& w, const double* X, int B, double* nu,
                            cudaStream_t s) {
  cudaError_t e = launch_explicit(g, t, w, X, B, true, s);
  if (e != cudaSuccess) return e;
  k_nu_final<<<nblk(B, 128), 128, 0, s>>>(g, t.cc, X, state_doubles(g), w.wT, nu, w.nsteps, w.flags, B);
  count();
  return cudaGetLastError();
}

// (Nu_V, Nu_b, Nu_t) of one state whose <wT>_x profile is in wT[0..Mz).
__global__ void k_nusselt(Grid g, const double* cc, const double* X, const double* wT, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double cond = 0.0, nb = 0.0, nt = 0.0;
  for (int n = 0; n < g.Nz; ++n) {
    const double a = X[soff(g, 0, n, 0)];
    if (n & 1) cond -= 2.0 * a;
    const double n2 = (double)n * n;
    nb -= 2.0 * a * ((n & 1) ? n2 : -n2);   // -dT/dz at z = -1/2: T_n'(-1) = (-1)^(n+1) n^2
    nt -= 2.0 * a * n2;                     // -dT/dz at z = +1/2: T_n'(1) = n^2
  }
  double adv = 0.0;
  for (int jz = 0; jz < g.Mz; ++jz) adv = fma(cc[jz], wT[jz], adv);
  out[0] = cond + 0.5 * adv;
  out[1] = nb;
  out[2] = nt;
}

cudaError_t launch_nusselt(const Grid& g, const Tables& t, const Work& w, const double* X, double* out3,
                           cudaStream_t s) {
  cudaError_t e = launch_explicit(g, t, w, X, 1, true, s);
  if (e != cudaSuccess) return e;
  k_nusselt<<<1, 32, 0, s>>>(g, t.cc, X, w.wT, out3);
  count();
  return cudaGetLastError();
}

// Consistency-check averages of Sec. 2.2, pass 1.  Z holds the FP64 z inverse
// of every state (fields u, w, d_x omega, d_z omega, ..., T, ... at the padded
// rows).  Block per (state, padded row j): x-means by Parseval over the kept
// modes (weight 1 for m = 0, 2 otherwise; Re(a conj b) for a pair of fields):
//   u^2 + w^2,   u.lap u = -u d_z omega + w d_x omega,   w T,
//   (T - <T>_x)^2 (modes m >= 1),   <T>_x = Re T_0(s_j).
// rows[b][q][j], q = 0..4 in that order.
__global__ void __launch_bounds__(128) k_diag_rows(Grid g, const double* __restrict__ Z, double* __restrict__ rows) {
  __shared__ double red[128];
  const int b = blockIdx.x / g.Mz, j = blockIdx.x - b * g.Mz;
  const size_t fs = (size_t)g.Mz * g.nm * 2;
  const double* zb = Z + (size_t)b * 9 * fs + (size_t)j * g.nm * 2;
  double ke = 0.0, ep = 0.0, wt = 0.0, tv = 0.0;
  for (int m = threadIdx.x; m < g.nm; m += blockDim.x) {
    const double c = m == 0 ? 1.0 : 2.0;
    const double2 u = ld2(zb + 2 * m), w = ld2(zb + fs + 2 * m);
    const double2 dxo = ld2(zb + 2 * fs + 2 * m), dzo = ld2(zb + 3 * fs + 2 * m);
    const double2 t = ld2(zb + 6 * fs + 2 * m);
    ke += c * (u.x * u.x + u.y * u.y + w.x * w.x + w.y * w.y);
    ep += c * (w.x * dxo.x + w.y * dxo.y - u.x * dzo.x - u.y * dzo.y);
    wt += c * (w.x * t.x + w.y * t.y);
    if (m > 0) tv += 2.0 * (t.x * t.x + t.y * t.y);
  }
  ke = block_sum(ke, red);
  ep = block_sum(ep, red);
  wt = block_sum(wt, red);
  tv = block_sum(tv, red);
  if (threadIdx.x == 0) {
    double* r = rows + (size_t)b * 5 * g.Mz + j;
    r[0] = ke;
    r[g.Mz] = ep;
    r[2 * g.Mz] = wt;
    r[3 * g.Mz] = tv;
    r[4 * g.Mz] = zb[6 * fs];
  }
}

// Pass 2, block per state: <f>_V = (1/2) sum_j cc_j <f>_x(s_j) (Lz = 1) for the
// first three rows, the Nusselt numbers of Eqs. 9-11 (conduction part of Nu_V
// and the wall slopes from the mean temperature coefficients), the profiles.
__global__ void __launch_bounds__(128) k_diag_final(Grid g, const double* __restrict__ cc, const double* __restrict__ X,
                                                    const double* __restrict__ rows, double* __restrict__ out) {
  __shared__ double red[128];
  const int b = blockIdx.x;
  const double* r = rows + (size_t)b * 5 * g.Mz;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int j = threadIdx.x; j < g.Mz; j += blockDim.x) {
    const double c = cc[j];
    s0 += c * r[j];
    s1 += c * r[g.Mz + j];
    s2 += c * r[2 * g.Mz + j];
  }
  s0 = block_sum(s0, red);
  s1 = block_sum(s1, red);
  s2 = block_sum(s2, red);
  double* o = out + (size_t)b * (6 + 2 * g.Mz);
  if (threadIdx.x == 0) {
    const double* Xb = X + (size_t)b * state_doubles(g);
    double cond = 0.0, nb = 0.0, nt = 0.0;
    for (int n = 0; n < g.Nz; ++n) {
      const double a = Xb[soff(g, 0, n, 0)];
      if (n & 1) cond -= 2.0 * a;
      const double n2 = (double)n * n;
      nb -= 2.0 * a * ((n & 1) ? n2 : -n2);
      nt -= 2.0 * a * n2;
    }
    o[0] = 0.5 * s0;
    o[1] = 0.5 * s1;
    o[2] = 0.5 * s2;
    o[3] = cond + 0.5 * s2;
    o[4] = nb;
    o[5] = nt;
  }
  for (int j = threadIdx.x; j < g.Mz; j += blockDim.x) {
    o[6 + j] = r[4 * g.Mz + j];
    o[6 + g.Mz + j] = r[3 * g.Mz + j];
  }
}

cudaError_t launch_diagnostics(const Grid& g, const Tables& t, const Work& w, const double* X, int B, double* out,
                               cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int kp = zinv_warps(g);
  const unsigned zb = (unsigned)(B * ((g.Mz + 1) / 2) * ((g.nm + 31) / 32));
  // FP64 z inverse of all states (no step mask), whatever the handle's precision
  k_zinv<double><<<zb, 32 * kp, kp > 1 ? (size_t)kp * 12 * 32 * 2 * sizeof(double) : 0, s>>>(
      g, t.zinv, X, state_doubles(g), w.Z, B, nullptr, w.step);
  k_diag_rows<<<(unsigned)(B * g.Mz), 128, 0, s>>>(g, w.Z, w.Q);
  k_diag_final<<<(unsigned)B, 128, 0, s>>>(g, t.cc, X, w.Q, out);
  count(3);
  return cudaGetLastError();
}

// Sampled quantities of the time statistics of Sec. 2.2, in place over B rows
// of rbc_diagnostics (6 + 2 Mz each): the characteristic speed
// <u^2 + w^2>_V^(1/2) replaces <u^2 + w^2>_V, and the plane mean of T^2,
// <(T - <T>_x)^2>_x + <T>_x^2, replaces the plane variance.
__global__ void k_stat_sample(Grid g, double* d, int B) {
  const int D = 6 + 2 * g.Mz;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)B * D) return;
  const int i = (int)(idx % D);
  if (i == 0) {
    d[idx] = sqrt(d[idx]);
  } else if (i >= 6 + g.Mz) {
    const double tm = d[idx - g.Mz];
    d[idx] = __dadd_rn(d[idx], __dmul_rn(tm, tm));
  }
}

// Trapezoid rule over one sampling interval: acc += h2 (prev + cur), h2 = half
// the interval; then prev = cur (n values).
__global__ void k_stat_accum(double* acc, double* prev, const double* cur, double h2, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double c = cur[i];
  acc[i] = __dadd_rn(acc[i], __dmul_rn(h2, __dadd_rn(prev[i], c)));
  prev[i] = c;
}

// a += b (n values)
__global__ void k_add(double* a, const double* b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += b[i];
}

cudaError_t launch_stat_sample(const Grid& g, double* d, int B, cudaStream_t s) {
  const long n = (long)B * (6 + 2 * g.Mz);
  k_stat_sample<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, d, B);
  count();
  return cudaGetLastError();
}

cudaError_t launch_stat_accum(double* acc, double* prev, const double* cur, double h2, long n, cudaStream_t s) {
  k_stat_accum<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(acc, prev, cur, h2, n);
  count();
  return cudaGetLastError();
}

cudaError_t launch_add(double* a, const double* b, int n, cudaStream_t s) {
  k_add<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a, b, n);
  count();
  return cudaGetLastError();
}

// Squared L2(Omega) norms of temperature fields (the defect norm of Sec. 3.7):
// ||T||^2 = (Lx / 2) sum_m w_m Re(conj(c_m) . Gram c_m), w = 1 for m = 0, 2
// otherwise (Parseval in x), Gram the exact Chebyshev Gram matrix (z in
// [-1/2, 1/2]).  The sum runs over tiles of kCorrTile Fourier modes in tile
// order, each tile's terms summed by the block in a fixed order, with explicit
// roundings; rbc_l2_diff and the fused Parareal correction share this order,
// so both give the same bits.
constexpr int kCorrTile = 8;
constexpr int kCorrThreads = 256;

// w Re(conj(di) . s) added to acc, s = sum_j gram_ij d_j
__device__ __forceinline__ double l2_term(double acc, double w, double2 di, double2 s) {
  return fma(w, fma(di.x, s.x, __dmul_rn(di.y, s.y)), acc);
}
__device__ __forceinline__ double2 gram_acc(double2 s, double gij, double2 dj) {
  return make_double2(fma(gij, dj.x, s.x), fma(gij, dj.y, s.y));
}

// ||A_b - B_b||^2 (or ||A_b||^2 when Bm is null) of the temperature field of nst
// states, block (kCorrThreads threads) per state.
__global__ void __launch_bounds__(kCorrThreads) k_l2_diff(Grid g, const double* gram, const double* A, const double* Bm,
                                                          double* out) {
  __shared__ double red[kCorrThreads];
  const int b = blockIdx.x;
  const size_t S = state_doubles(g);
  const double* a = A + (size_t)b * S;
  const double* bb = Bm ? Bm + (size_t)b * S : nullptr;
  double tot = 0.0;
  for (int m0 = 0; m0 < g.nm; m0 += kCorrTile) {
    const int tm = min(kCorrTile, g.nm - m0);
    double acc = 0.0;
    for (int it = threadIdx.x; it < tm * g.Nz; it += blockDim.x) {
      const int dm = it % tm, i = it / tm, m = m0 + dm;
      double2 di = ld2(a + soff(g, 0, i, m));
      if (bb) di = di - ld2(bb + soff(g, 0, i, m));
      double2 s = {0.0, 0.0};
      for (int jn = (i & 1); jn < g.Nz; jn += 2) {
        double2 dj = ld2(a + soff(g, 0, jn, m));
        if (bb) dj = dj - ld2(bb + soff(g, 0, jn, m));
        s = gram_acc(s, __ldg(gram + (size_t)i * g.Nz + jn), dj);
      }
      acc = l2_term(acc, m == 0 ? 1.0 : 2.0, di, s);
    }
    tot += block_sum(acc, red);
  }
  if (threadIdx.x == 0) out[b] = 0.5 * g.Lx * tot;
}

cudaError_t launch_l2_diff(const Grid& g, const Tables& t, const double* A, const double* Bm, int nst, double* out,
                           cudaStream_t s) {
  if (nst <= 0) return cudaSuccess;
  k_l2_diff<<<nst, kCorrThreads, 0, s>>>(g, t.gram, A, Bm, out);
  count();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Native grid <-> spectral state.
// ---------------------------------------------------------------------------
// modes[fld][j][m] = (1/Nx) sum_i g[fld][j][i] exp(-i k_m x_i)
__global__ void k_grid_to_modes(Grid g, const double2* twn, const double* grid, double* modes) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3L * g.Nz * g.nm) return;
  const int m = idx % g.nm;
  const int j = (idx / g.nm) % g.Nz;
  const int fld = idx / ((long)g.nm * g.Nz);
  const double* row = grid + ((size_t)fld * g.Nz + j) * g.Nx;
  double2 acc = {0.0, 0.0};
  for (int i = 0; i < g.Nx; ++i) {
    const double2 w = twn[((long)m * i) % g.Nx];
    acc.x = fma(row[i], w.x, acc.x);
    acc.y = fma(row[i], w.y, acc.y);
  }
  st2(modes + idx * 2, (1.0 / g.Nx) * acc);
}

// coefficients by exact interpolation; psi_m = i w_m / k (m >= 1), U = <u>_x.
__global__ void k_modes_to_state(Grid g, const double* Wn, const double* modes, double* X) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)g.Nz * g.nm) return;
  const int m = idx % g.nm, n = idx / g.nm;
  double2 c[3];
  for (int fld = 0; fld < 3; ++fld) {
    double2 acc = {0.0, 0.0};
    for (int j = 0; j < g.Nz; ++j) {
      const double2 v = ld2(modes + (((size_t)fld * g.Nz + j) * g.nm + m) * 2);
      const double wv = Wn[(size_t)n * g.Nz + j];
      acc.x = fma(wv, v.x, acc.x);
      acc.y = fma(wv, v.y, acc.y);
    }
    c[fld] = acc;
  }
  double2 T = c[0];
  double2 P;
  if (m == 0) {
    T.y = 0.0;
    P = make_double2(c[1].x, 0.0);
  } else {
    const double k = g.kfac * m;
    P = (1.0 / k) * times_i(c[2]);
  }
  st2(X + soff(g, 0, n, m), T);
  st2(X + soff(g, 1, n, m), P);
}

cudaError_t launch_set_state(const Grid& g, const Tables& t, const double* gT, const double* gu, const double* gw,
                             double* scratch, double* X, cudaStream_t s) {
  // gT, gu, gw are consecutive [3][Nz][Nx] in device scratch (gT points at it)
  (void)gu;
  (void)gw;
  double* modes = scratch;
  k_grid_to_modes<<<nblk(3L * g.Nz * g.nm, 128), 128, 0, s>>>(g, t.twn, gT, modes);
  k_modes_to_state<<<nblk((long)g.Nz * g.nm, 128), 128, 0, s>>>(g, t.Wn, modes, X);
  count(2);
  return cudaGetLastError();
}

// native-point mode values of T, u, w: modes[fld][j][m]
__global__ void k_state_to_modes(Grid g, const double* Vn, const double* Vn1, const double* X, double* modes) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)g.Nz * g.nm) return;
  const int m = idx % g.nm, j = idx / g.nm;
  double2 T = {0, 0}, P = {0, 0}, P1 = {0, 0};
  for (int n = 0; n < g.Nz; ++n) {
    const double v = Vn[(size_t)j * g.Nz + n], v1 = Vn1[(size_t)j * g.Nz + n];
    const double2 xt = ld2(X + soff(g, 0, n, m)), xp = ld2(X + soff(g, 1, n, m));
    T = T + v * xt;
    P = P + v * xp;
    P1 = P1 + v1 * xp;
  }
  double2 u, w;
  if (m == 0) {
    u = make_double2(P.x, 0.0);
    w = make_double2(0.0, 0.0);
  } else {
    const double k = g.kfac * m;
    u = 2.0 * P1;
    w = -k * times_i(P);
  }
  const size_t fsz = (size_t)g.Nz * g.nm * 2;
  st2(modes + 0 * fsz + idx * 2, T);
  st2(modes + 1 * fsz + idx * 2, u);
  st2(modes + 2 * fsz + idx * 2, w);
}

// grid[fld][j][i] = Re c_0 + 2 sum_{m>=1} Re(c_m exp(i k_m x_i))
__global__ void k_modes_to_grid(Grid g, const double2* twn, const double* modes, double* grid) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3L * g.Nz * g.Nx) return;
  const int i = idx % g.Nx;
  const int j = (idx / g.Nx) % g.Nz;
  const int fld = idx / ((long)g.Nx * g.Nz);
  const double* c = modes + ((size_t)fld * g.Nz + j) * g.nm * 2;
  double acc = c[0];
  for (int m = 1; m < g.nm; ++m) {
    const double2 w = twn[((long)m * i) % g.Nx];     // exp(-i...) -> use conj
    const double2 cm = ld2(c + 2 * m);
    acc += 2.0 * (cm.x * w.x + cm.y * w.y);          // Re(c * conj(w))
  }
  grid[idx] = acc;
}

cudaError_t launch_get_state(const Grid& g, const Tables& t, const double* X, double* scratch, double* gT,
                             double* gu, double* gw, cudaStream_t s) {
  (void)gu;
  (void)gw;
  double* modes = scratch;
  k_state_to_modes<<<nblk((long)g.Nz * g.nm, 128), 128, 0, s>>>(g, t.Vn, t.Vn1, X, modes);
  k_modes_to_grid<<<nblk(3L * g.Nz * g.Nx, 128), 128, 0, s>>>(g, t.twn, modes, gT);
  count(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Parareal transfer and correction (Eq. 20).
// ---------------------------------------------------------------------------
__global__ void k_restrict(Grid gf, Grid gc, const double* Xf, double* Xc, int B) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = 2L * gc.Nz * gc.nm;
  if (idx >= per * B) return;
  const int b = (int)(idx / per);
  const long r = idx - (long)b * per;
  const int m = r % gc.nm;
  const int n = (r / gc.nm) % gc.Nz;
  const int f = r / ((long)gc.nm * gc.Nz);
  st2(Xc + (size_t)b * state_doubles(gc) + soff(gc, f, n, m), ld2(Xf + (size_t)b * state_doubles(gf) + soff(gf, f, n, m)));
}

cudaError_t launch_restrict(const Grid& gf, const Grid& gc, const double* Xf, double* Xc, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_restrict<<<nblk(2L * gc.Nz * gc.nm * B, 128), 128, 0, s>>>(gf, gc, Xf, Xc, B);
  count();
  return cudaGetLastError();
}

__global__ void k_prolong(Grid gf, Grid gc, const double* Xc, double* Xf, int B) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = 2L * gf.Nz * gf.nm;
  if (idx >= per * B) return;
  const int b = (int)(idx / per);
  const long r = idx - (long)b * per;
  const int m = r % gf.nm;
  const int n = (r / gf.nm) % gf.Nz;
  const int f = r / ((long)gf.nm * gf.Nz);
  double2 v = {0.0, 0.0};
  if (m < gc.nm && n < gc.Nz) v = ld2(Xc + (size_t)b * state_doubles(gc) + soff(gc, f, n, m));
  st2(Xf + (size_t)b * state_doubles(gf) + soff(gf, f, n, m), v);
}

cudaError_t launch_prolong(const Grid& gf, const Grid& gc, const double* Xc, double* Xf, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_prolong<<<nblk(2L * gf.Nz * gf.nm * B, 128), 128, 0, s>>>(gf, gc, Xc, Xf, B);
  count();
  return cudaGetLastError();
}

// U = F + (prolong(Gnew) - prolong(Gold)), elementwise in that order (Eq. 20).
__global__ void k_correct(Grid gf, Grid gc, const double* Ff, const double* Gnew, const double* Gold, double* U,
                          int B) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = 2L * gf.Nz * gf.nm;
  if (idx >= per * B) return;
  const int b = (int)(idx / per);
  const long r = idx - (long)b * per;
  const int m = r % gf.nm;
  const int n = (r / gf.nm) % gf.Nz;
  const int f = r / ((long)gf.nm * gf.Nz);
  const size_t Sf = state_doubles(gf), Sc = state_doubles(gc);
  double2 d = {0.0, 0.0};
  if (m < gc.nm && n < gc.Nz)
    d = ld2(Gnew + (size_t)b * Sc + soff(gc, f, n, m)) - ld2(Gold + (size_t)b * Sc + soff(gc, f, n, m));
  st2(U + (size_t)b * Sf + soff(gf, f, n, m), ld2(Ff + (size_t)b * Sf + soff(gf, f, n, m)) + d);
}

cudaError_t launch_correct(const Grid& gf, const Grid& gc, const double* Ff, const double* Gnew, const double* Gold,
                           double* Uout, int B, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_correct<<<nblk(2L * gf.Nz * gf.nm * B, 128), 128, 0, s>>>(gf, gc, Ff, Gnew, Gold, Uout, B);
  count();
  return cudaGetLastError();
}

// One slice of a Parareal sweep (Sec. 3.1, Eq. 20) fused with its norms (Sec. 3.7).
// mode 0 (the coarse sweep U^0):  U = prolong(Gnew).
// mode 1 (a correction):          U = F + (prolong(Gnew) - prolong(Gold)), elementwise in that order.
// Both: Gold <- Gnew (the coarse value of this iterate, which the next
// iteration subtracts); C <- restrict(U) (the next coarse step's input: the
// coarse modes of U; C may be the Gnew buffer, each element is read before
// it is written); Fnext <- U when not null (the next iteration's fine input);
// mode 1 with Uprev: norms[0] = ||T(U) - T(Uprev)||^2, norms[1] = ||T(U)||^2
// (L2 over the domain, in the order of k_l2_diff: the same bits).
// Block per tile of kCorrTile Fourier modes, all Chebyshev indices of both
// fields; the blocks' partial sums are added in block order by the last block
// to finish (partial[2 * gridDim.x], counter: left at zero).
__global__ void __launch_bounds__(kCorrThreads) k_correct_norm(
    Grid gf, Grid gc, const double* __restrict__ gram, int mode, const double* Ff, const double* Gnew, double* Gold,
    double* C, const double* __restrict__ Uprev, double* __restrict__ U, double* __restrict__ Fnext,
    double* partial, unsigned* counter, double* norms) {
  __shared__ double red[kCorrThreads];
  extern __shared__ double2 sd[];             // [kCorrTile][Nz]: T(U) - T(Uprev) of the tile's modes
  __shared__ bool last;
  const int m0 = blockIdx.x * kCorrTile;
  const int tm = min(kCorrTile, gf.nm - m0);
  const int per = 2 * gf.Nz * tm;
  const bool with_norms = mode == 1 && Uprev != nullptr;
  for (int it = threadIdx.x; it < per; it += blockDim.x) {
    const int dm = it % tm, n = (it / tm) % gf.Nz, f = it / (tm * gf.Nz);
    const int m = m0 + dm;
    const size_t o = soff(gf, f, n, m);
    const bool coarse = m < gc.nm && n < gc.Nz;
    const size_t oc = coarse ? soff(gc, f, n, m) : 0;
    double2 u;
    if (mode == 0) {
      u = coarse ? ld2(Gnew + oc) : make_double2(0.0, 0.0);
      if (coarse) st2(Gold + oc, u);
    } else {
      double2 d = {0.0, 0.0};
      if (coarse) {
        const double2 gn = ld2(Gnew + oc);
        d = gn - ld2(Gold + oc);
        st2(Gold + oc, gn);
      }
      u = ld2(Ff + o) + d;
      if (coarse) st2(C + oc, u);
    }
    st2(U + o, u);
    if (Fnext) st2(Fnext + o, u);
    if (with_norms && f == 0) sd[dm * gf.Nz + n] = u - ld2(Uprev + o);
  }
  if (!with_norms) return;
  __syncthreads();
  // sum_m w_m Re(conj(d_i) sum_j gram_ij d_j), i, j of equal parity; the same for U
  double acc_d = 0.0, acc_u = 0.0;
  for (int it = threadIdx.x; it < tm * gf.Nz; it += blockDim.x) {
    const int dm = it % tm, i = it / tm, m = m0 + dm;
    const double2 di = sd[dm * gf.Nz + i];
    const double2 ui = ld2(U + soff(gf, 0, i, m));
    double2 s = {0.0, 0.0}, t = {0.0, 0.0};
    for (int j = (i & 1); j < gf.Nz; j += 2) {
      const double gij = __ldg(gram + (size_t)i * gf.Nz + j);
      s = gram_acc(s, gij, sd[dm * gf.Nz + j]);
      t = gram_acc(t, gij, ld2(U + soff(gf, 0, j, m)));
    }
    const double w = m == 0 ? 1.0 : 2.0;
    acc_d = l2_term(acc_d, w, di, s);
    acc_u = l2_term(acc_u, w, ui, t);
  }
  acc_d = block_sum(acc_d, red);
  acc_u = block_sum(acc_u, red);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = acc_d;
    partial[2 * blockIdx.x + 1] = acc_u;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double sdiff = 0.0, su = 0.0;
  for (unsigned bidx = 0; bidx < gridDim.x; ++bidx) {
    sdiff += *((volatile double*)partial + 2 * bidx);
    su += *((volatile double*)partial + 2 * bidx + 1);
  }
  norms[0] = 0.5 * gf.Lx * sdiff;
  norms[1] = 0.5 * gf.Lx * su;
  *counter = 0u;
}

int correct_norm_blocks(const Grid& gf) { return (gf.nm + kCorrTile - 1) / kCorrTile; }

cudaError_t launch_correct_norm(const Grid& gf, const Grid& gc, const Tables& tf, int mode, const double* Ff,
                                const double* Gnew, double* Gold, double* C, const double* Uprev, double* U,
                                double* Fnext, double* partial, unsigned* counter, double* norms, cudaStream_t s) {
  static int allowed = 48 * 1024;
  const size_t smem = (size_t)kCorrTile * gf.Nz * sizeof(double2);
  cudaError_t e = allow_smem(k_correct_norm, (int)smem, allowed);
  if (e != cudaSuccess) return e;
  k_correct_norm<<<correct_norm_blocks(gf), kCorrThreads, smem, s>>>(gf, gc, tf.gram, mode, Ff, Gnew, Gold, C, Uprev,
                                                                     U, Fnext, partial, counter, norms);
  count();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Nusselt numbers without any allocation: the scratch of the explicit-term
// evaluation (z-inverse fields, row outputs, the <wT>_x profile and the three
// results) lives in one file-scope device array, shared by every call on a
// device.  Its device address is looked up once per device, with that device
// current, on the first call there.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_static_scratch[kStaticScratchCapacity];
constexpr int kMaxDevices = 64;
static std::atomic<double*> g_static_ptr[kMaxDevices] = {};

// Layout: Z, Q, the <wT>_x profile (Mz rounded up to even), then 8 doubles:
// the three Nusselt numbers and, in the fifth, the int error bits of the call.
size_t static_scratch_doubles_needed(const Grid& g) {
  return z_doubles(g) + q_doubles(g) + (size_t)((g.Mz + 1) & ~1) + 8;
}

cudaError_t launch_nusselt_static(const Grid& g, const Tables& t, const double* X, double* host_out3,
                                  int* host_flags, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  double* base = g_static_ptr[dev].load();
  if (base == nullptr) {
    // two threads may both look it up; they store the same address
    e = cudaGetSymbolAddress((void**)&base, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev].store(base);
  }
  Work w{};
  w.Z = base;
  w.Q = w.Z + z_doubles(g);
  w.wT = w.Q + q_doubles(g);
  w.small = w.wT + ((g.Mz + 1) & ~1);
  w.flags = reinterpret_cast<int*>(w.small + 4);   // the call's error bits (the tensor-core waits)
  w.err = w.flags;
  w.prof = nullptr;
  e = cudaMemsetAsync(w.flags, 0, sizeof(int), s);   // the only element read before this call writes it
  if (e != cudaSuccess) return e;
  e = launch_nusselt(g, t, w, X, w.small, s);
  if (e != cudaSuccess) return e;
  double res[5];
  e = cudaMemcpyAsync(res, w.small, sizeof(res), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 3; ++i) host_out3[i] = res[i];
  std::memcpy(host_flags, &res[4], sizeof(int));
  return cudaSuccess;
}

}  // namespace rbc
