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
#include <cuda_runtime.h>

#include <cstdint>

#include "rbc_internal.h"

namespace rbc {

// RK443 (Ascher, Ruuth & Spiteri 1997, the (4,4,3) pair; Sec. 3.6).
__constant__ double c_AE[5][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 2, 0, 0, 0, 0},
    {11.0 / 18, 1.0 / 18, 0, 0, 0},
    {5.0 / 6, -5.0 / 6, 1.0 / 2, 0, 0},
    {1.0 / 4, 7.0 / 4, 3.0 / 4, -7.0 / 4, 0}};
__constant__ double c_AI[5][5] = {
    {0, 0, 0, 0, 0},
    {0, 1.0 / 2, 0, 0, 0},
    {0, 1.0 / 6, 1.0 / 2, 0, 0},
    {0, -1.0 / 2, 1.0 / 2, 1.0 / 2, 0},
    {0, 3.0 / 2, -3.0 / 2, 1.0 / 2, 1.0 / 2}};

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
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

// ---------------------------------------------------------------------------
// z inverse transform (k_zinv).  Thread per (slice, padded row j, mode m).
// psi-slot operators V, VD, VD^2, VD^3 (d/ds) and T-slot V, VD; the epilogue
// forms, with d/dz = 2 d/ds and d/dx = ik:
//   u = d_z psi (m = 0: U),  w = -ik psi,  d_x omega, d_z omega (omega = -lap psi,
//   m = 0: omega = -U'),  d_x u,  d_z u,  T,  d_x T,  d_z T.
// Output Z[b][field][j][m] (complex), fields in that order.
// ---------------------------------------------------------------------------
__global__ void k_zinv(Grid g, const double* __restrict__ Bz, const double* __restrict__ X, size_t S,
                       double* __restrict__ Z, int B, const int* nsteps, const int* step) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = (long)g.Mz * g.nm;
  if (idx >= per * B) return;
  const int b = (int)(idx / per);
  if (!slice_active(nsteps, step, b)) return;
  const int rem = (int)(idx - (long)b * per);
  const int j = rem / g.nm, m = rem - j * g.nm;
  const double* Xb = X + (size_t)b * S;
  const double* b0 = Bz + (size_t)(0 * g.Mz + j) * g.Nz;
  const double* b1 = Bz + (size_t)(1 * g.Mz + j) * g.Nz;
  const double* b2 = Bz + (size_t)(2 * g.Mz + j) * g.Nz;
  const double* b3 = Bz + (size_t)(3 * g.Mz + j) * g.Nz;
  double2 p0 = {0, 0}, p1 = {0, 0}, p2 = {0, 0}, p3 = {0, 0}, t0 = {0, 0}, t1 = {0, 0};
  for (int n = 0; n < g.Nz; ++n) {
    const double2 xp = ld2(Xb + soff(g, 1, n, m));
    const double2 xt = ld2(Xb + soff(g, 0, n, m));
    const double v0 = __ldg(b0 + n), v1 = __ldg(b1 + n), v2 = __ldg(b2 + n), v3 = __ldg(b3 + n);
    p0.x = fma(v0, xp.x, p0.x); p0.y = fma(v0, xp.y, p0.y);
    p1.x = fma(v1, xp.x, p1.x); p1.y = fma(v1, xp.y, p1.y);
    p2.x = fma(v2, xp.x, p2.x); p2.y = fma(v2, xp.y, p2.y);
    p3.x = fma(v3, xp.x, p3.x); p3.y = fma(v3, xp.y, p3.y);
    t0.x = fma(v0, xt.x, t0.x); t0.y = fma(v0, xt.y, t0.y);
    t1.x = fma(v1, xt.x, t1.x); t1.y = fma(v1, xt.y, t1.y);
  }
  const double k = g.kfac * m;
  double2 u, w, dxo, dzo, dxu, dzu, T, dxT, dzT;
  if (m == 0) {
    u = make_double2(p0.x, 0.0);
    w = make_double2(0.0, 0.0);
    dxo = make_double2(0.0, 0.0);
    dzo = make_double2(-4.0 * p2.x, 0.0);
    dxu = make_double2(0.0, 0.0);
    dzu = make_double2(2.0 * p1.x, 0.0);
    T = t0;
    dxT = make_double2(0.0, 0.0);
    dzT = 2.0 * t1;
  } else {
    u = 2.0 * p1;
    w = -k * times_i(p0);                             // -ik psi
    const double2 om = (k * k) * p0 - 4.0 * p2;       // omega = -(4 psi'' - k^2 psi)
    dxo = k * times_i(om);
    dzo = (2.0 * k * k) * p1 - 8.0 * p3;              // -(8 psi''' - 2 k^2 psi')
    dxu = k * times_i(u);
    dzu = 4.0 * p2;
    T = t0;
    dxT = k * times_i(t0);
    dzT = 2.0 * t1;
  }
  const size_t fs = (size_t)g.Mz * g.nm * 2;
  double* zb = Z + (size_t)b * 9 * fs + ((size_t)j * g.nm + m) * 2;
  st2(zb + 0 * fs, u);
  st2(zb + 1 * fs, w);
  st2(zb + 2 * fs, dxo);
  st2(zb + 3 * fs, dzo);
  st2(zb + 4 * fs, dxu);
  st2(zb + 5 * fs, dzu);
  st2(zb + 6 * fs, T);
  st2(zb + 7 * fs, dxT);
  st2(zb + 8 * fs, dzT);
}

// ---------------------------------------------------------------------------
// Shared-memory mixed-radix Stockham FFT of length N = 3 * 2^p (radices
// 4, ..., 4, [2], 3).  y_q = sum_r x_r exp(sign 2 pi i q r / N), unnormalised.
// Ping-pongs between a and b; returns the buffer holding the result.
// ---------------------------------------------------------------------------
__device__ double2* fft_smem(double2* a, double2* b, int N, int sign, const double2* __restrict__ tw) {
  int p = 0;
  for (int M = N / 3; M > 1; M >>= 1) ++p;
  int nr = p / 2 + (p & 1) + 1;
  int Ns = 1;
  double2* x = a;
  double2* y = b;
  const double s3 = 0.86602540378443864676 * sign;   // sign * sqrt(3)/2
  for (int pass = 0; pass < nr; ++pass) {
    const int R = (pass < p / 2) ? 4 : ((p & 1) && pass == p / 2) ? 2 : 3;
    const int nb = N / R;
    const int stride = N / (Ns * R);
    for (int jj = threadIdx.x; jj < nb; jj += blockDim.x) {
      const int k = jj % Ns;
      double2 v[4];
      for (int r = 0; r < R; ++r) v[r] = x[jj + r * nb];
      if (Ns > 1) {
        for (int r = 1; r < R; ++r) {
          double2 wv = __ldg(tw + (k * r * stride) % N);
          if (sign > 0) wv.y = -wv.y;
          v[r] = cmul(v[r], wv);
        }
      }
      const int base = (jj / Ns) * Ns * R + k;
      if (R == 2) {
        y[base] = v[0] + v[1];
        y[base + Ns] = v[0] - v[1];
      } else if (R == 4) {
        const double2 a0 = v[0] + v[2], a1 = v[0] - v[2];
        const double2 b0 = v[1] + v[3], b1 = v[1] - v[3];
        const double2 ib1 = (double)sign * times_i(b1);
        y[base] = a0 + b0;
        y[base + Ns] = a1 + ib1;
        y[base + 2 * Ns] = a0 - b0;
        y[base + 3 * Ns] = a1 - ib1;
      } else {
        const double2 t1 = v[1] + v[2], t2 = v[1] - v[2];
        const double2 m1 = v[0] - 0.5 * t1;
        const double2 m2 = s3 * times_i(t2);
        y[base] = v[0] + t1;
        y[base + Ns] = m1 + m2;
        y[base + 2 * Ns] = m1 - m2;
      }
    }
    __syncthreads();
    double2* tmp = x;
    x = y;
    y = tmp;
    Ns *= R;
  }
  return x;
}

size_t rows_smem_bytes(const Grid& g) { return (size_t)g.Mx * (2 * 16 + 9 * 8); }

// Deterministic block sum (fixed tree over blockDim.x threads, blockDim a power of two).
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double r = red[0];
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
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rows(Grid g, const double2* __restrict__ tw, const double* __restrict__ Z,
                                              double* __restrict__ Q, double* __restrict__ wT, int B,
                                              const int* nsteps, const int* step) {
  extern __shared__ double sm[];
  const int b = blockIdx.x / g.Mz, j = blockIdx.x - b * g.Mz;
  if (!slice_active(nsteps, step, b)) return;
  const int Mx = g.Mx, nm = g.nm;
  double2* A = reinterpret_cast<double2*>(sm);
  double2* Bf = A + Mx;
  double* fr = reinterpret_cast<double*>(Bf + Mx);
  __shared__ double red[256];
  const size_t fs = (size_t)g.Mz * nm * 2;
  const double* zrow = Z + (size_t)b * 9 * fs + (size_t)j * nm * 2;
  for (int pr = 0; pr < 5; ++pr) {
    const int fa = 2 * pr, fb = 2 * pr + 1;
    const double* za = zrow + fa * fs;
    const double* zb = zrow + fb * fs;
    for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
      double2 c = make_double2(0.0, 0.0);
      if (x < nm) {
        const double2 a = ld2(za + 2 * x);
        const double2 bb = (fb < 9) ? ld2(zb + 2 * x) : make_double2(0.0, 0.0);
        c = a + times_i(bb);
      } else if (x > Mx - nm) {
        const int m = Mx - x;
        const double2 a = ld2(za + 2 * m);
        const double2 bb = (fb < 9) ? ld2(zb + 2 * m) : make_double2(0.0, 0.0);
        c = conj2(a) + times_i(conj2(bb));
      }
      A[x] = c;
    }
    __syncthreads();
    const double2* res = fft_smem(A, Bf, Mx, +1, tw);
    for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
      fr[fa * Mx + x] = res[x].x;
      if (fb < 9) fr[fb * Mx + x] = res[x].y;
    }
    __syncthreads();
  }
  double nU = 0.0, wt = 0.0;
  for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
    const double u = fr[0 * Mx + x], w = fr[1 * Mx + x];
    const double nO = u * fr[2 * Mx + x] + w * fr[3 * Mx + x];
    nU += u * fr[4 * Mx + x] + w * fr[5 * Mx + x];
    const double nT = u * fr[7 * Mx + x] + w * fr[8 * Mx + x];
    wt += w * fr[6 * Mx + x];
    A[x] = make_double2(nT, nO);
  }
  __syncthreads();
  const double sU = block_sum(nU, red);
  const double sW = block_sum(wt, red);
  const double2* C = fft_smem(A, Bf, Mx, -1, tw);
  const double inv = 1.0 / Mx;
  const size_t qs = (size_t)g.Mz * nm * 2;
  double* q0 = Q + (size_t)b * 2 * qs + (size_t)j * nm * 2;
  double* q1 = q0 + qs;
  for (int m = threadIdx.x; m < nm; m += blockDim.x) {
    const double2 cm = C[m];
    const double2 cn = conj2(C[m == 0 ? 0 : Mx - m]);
    const double2 s = cm + cn, d = cm - cn;
    st2(q0 + 2 * m, make_double2(0.5 * inv * s.x, 0.5 * inv * s.y));
    if (m == 0)
      st2(q1, make_double2(sU * inv, 0.0));
    else
      st2(q1 + 2 * m, make_double2(0.5 * inv * d.y, -0.5 * inv * d.x));
  }
  if (threadIdx.x == 0) wT[(size_t)b * g.Mz + j] = sW * inv;
}

// ---------------------------------------------------------------------------
// z forward transform (k_zfwd): F[b][f][n][m] = sum_j W[n][j] Q[b][f][j][m], n < Nz.
// ---------------------------------------------------------------------------
__global__ void k_zfwd(Grid g, const double* __restrict__ W, const double* __restrict__ Q, double* __restrict__ F,
                       size_t S, int B, const int* nsteps, const int* step) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = 2L * g.Nz * g.nm;
  if (idx >= per * B) return;
  const int b = (int)(idx / per);
  if (!slice_active(nsteps, step, b)) return;
  int rem = (int)(idx - (long)b * per);
  const int m = rem % g.nm;
  rem /= g.nm;
  const int n = rem % g.Nz, f = rem / g.Nz;
  const size_t qs = (size_t)g.Mz * g.nm * 2;
  const double* q = Q + (size_t)(b * 2 + f) * qs + (size_t)m * 2;
  const double* wr = W + (size_t)n * g.Mz;
  double2 acc = {0.0, 0.0};
  for (int jz = 0; jz < g.Mz; ++jz) {
    const double wv = __ldg(wr + jz);
    const double2 v = ld2(q + (size_t)jz * g.nm * 2);
    acc.x = fma(wv, v.x, acc.x);
    acc.y = fma(wv, v.y, acc.y);
  }
  st2(F + (size_t)b * S + soff(g, f, n, m), acc);
}

// ---------------------------------------------------------------------------
// Stage solve (k_solve).
// ---------------------------------------------------------------------------
enum { KT = 0, KP = 1, KU = 2 };

// One parity-split system of one field for one (slice, m, p).
//   tau row t (full row 2t+p) of (M - dt/2 L) X_i = r_i, boundary rows on top;
//   r_i = M X_0 + dt sum_{j<i} (aE_ij F_j + aI_ij L X_j) kept in accumulators:
//   R_i complete when stage i starts; dt L X_i = 2 (M X_i - r_i).
template <int KIND>
__device__ bool solve_system(const Grid& g, const Tables& tb, int stage, int p, int m, const double* X0, double* Xo,
                             const double* Fc, double* R, size_t S) {
  constexpr int D = (KIND == KP) ? 2 : 1;
  constexpr int LAM = 2 * D;
  const int nq = g.nq;
  const int f = (KIND == KT) ? 0 : 1;
  const int nmod = (KIND == KU) ? 1 : g.nm;
  const int mi = (KIND == KU) ? 0 : m;
  const double* multB = (KIND == KT) ? tb.T_multB : (KIND == KP) ? tb.P_multB : tb.U_multB;
  const double* multD = (KIND == KT) ? tb.T_multD : (KIND == KP) ? tb.P_multD : tb.U_multD;
  const double* Dinv = (KIND == KT) ? tb.T_Dinv : (KIND == KP) ? tb.P_Dinv : tb.U_Dinv;
  const double* Lb = (KIND == KT) ? tb.T_Lb : (KIND == KP) ? tb.P_Lb : tb.U_Lb;
  const double* invd = (KIND == KT) ? tb.T_invd : (KIND == KP) ? tb.P_invd : tb.U_invd;
  auto tix = [&](int c, int jj) { return ((size_t)(p * nq + c) * D + jj) * nmod + mi; };
  auto co = [&](int n) { return soff(g, f, n, m); };
  auto tapF = [&](int t, int jj) -> double {
    return (KIND == KP) ? __ldg(tb.s4 + (p * nq + t) * 5 + jj) : __ldg(tb.s2 + (p * nq + t) * 3 + jj);
  };
  auto tapM = [&](int t, int jj) -> double {
    return (KIND == KP) ? __ldg(tb.mp + ((size_t)(p * nq + t) * 5 + jj) * g.nm + m)
                        : __ldg(tb.s2 + (p * nq + t) * 3 + jj);
  };
  const double fsign = (KIND == KP) ? 1.0 : -1.0;
  const double dt = g.dt;
  const double cpl = 0.5 * dt * g.Pr * g.Ra * (g.kfac * m);
  double* Ri = R + (size_t)(stage - 1) * S;

  // pass 1: right-hand side rows, backward elimination of the upper band
  double2 pend[D];
  double2 bd[D];
  for (int jj = 0; jj < D; ++jj) {
    pend[jj] = make_double2(0.0, 0.0);
    bd[jj] = make_double2(0.0, 0.0);
  }
  for (int c = nq - 1; c >= D; --c) {
    const int t = c - D;
    double2 fv = {0.0, 0.0};
    for (int jj = 0; jj <= LAM; ++jj) {
      const int q = t + jj;
      if (q < nq) fv = fv + tapF(t, jj) * ld2(Fc + co(2 * q + p));
    }
    fv = fsign * fv;
    const size_t ro = co(2 * t + p);
    double2 r;
    if (stage == 1) {
      double2 mx = {0.0, 0.0};
      for (int jj = 0; jj <= LAM; ++jj) {
        const int q = t + jj;
        if (q < nq) mx = mx + tapM(t, jj) * ld2(X0 + co(2 * q + p));
      }
      r = mx + (dt * c_AE[1][0]) * fv;
      for (int l = 2; l <= 4; ++l) st2(R + (size_t)(l - 1) * S + ro, mx + (dt * c_AE[l][0]) * fv);
    } else {
      r = ld2(Ri + ro) + (dt * c_AE[stage][stage - 1]) * fv;
      for (int l = stage + 1; l <= 4; ++l) {
        double* Rl = R + (size_t)(l - 1) * S + ro;
        st2(Rl, ld2(Rl) + (dt * c_AE[l][stage - 1]) * fv);
      }
    }
    st2(Ri + ro, r);
    double2 bv = r;
    if (KIND == KP) {
      double2 st = {0.0, 0.0};
      for (int jj = 0; jj <= 4; ++jj) {
        const int q = t + jj;
        if (q < nq) st = st + __ldg(tb.s4 + (p * nq + t) * 5 + jj) * ld2(Xo + soff(g, 0, 2 * q + p, m));
      }
      bv.x += cpl * st.y;                               // + dt/2 (-i k Pr Ra) S4 T_i
      bv.y -= cpl * st.x;
    }
    const double2 bc = bv + pend[0];
    st2(Xo + co(2 * c + p), bc);
    for (int jj = 0; jj < D - 1; ++jj) pend[jj] = pend[jj + 1] - __ldg(multB + tix(c, D - 1 - jj)) * bc;
    pend[D - 1] = -__ldg(multB + tix(c, 0)) * bc;
    for (int r2 = 0; r2 < D; ++r2) bd[r2] = bd[r2] - __ldg(multD + tix(c, r2)) * bc;
  }
  // boundary rows (Eq. 6): parity combinations of f(1) +- f(-1)
  double2 bb[D];
  for (int r2 = 0; r2 < D; ++r2) bb[r2] = bd[r2];
  if (KIND == KT && m == 0) bb[0].x += (p == 0) ? 0.5 : -0.5;   // T(-1/2) = 1, T(1/2) = 0
  double2 win[D];
  bool ok = true;
  for (int r2 = 0; r2 < D; ++r2) {
    double2 x = {0.0, 0.0};
    for (int c2 = 0; c2 < D; ++c2)
      x = x + __ldg(Dinv + ((size_t)(p * D * D) + r2 * D + c2) * nmod + mi) * bb[c2];
    win[r2] = x;
    st2(Xo + co(2 * r2 + p), x);
    ok = ok && finite2(x);
  }
  // pass 2: forward substitution with the lower band
  for (int r2 = D; r2 < nq; ++r2) {
    double2 y = ld2(Xo + co(2 * r2 + p));
    for (int jj = 0; jj < D; ++jj) y = y - __ldg(Lb + tix(r2, jj)) * win[jj];
    const double2 x = __ldg(invd + (size_t)(p * nq + r2) * nmod + mi) * y;
    st2(Xo + co(2 * r2 + p), x);
    for (int jj = 0; jj < D - 1; ++jj) win[jj] = win[jj + 1];
    win[D - 1] = x;
    ok = ok && finite2(x);
  }
  // pass 3: dt aI_li L X_i = 2 aI_li (M X_i - r_i) into later accumulators
  if (stage < 4) {
    for (int t = 0; t < nq - D; ++t) {
      double2 mx = {0.0, 0.0};
      for (int jj = 0; jj <= LAM; ++jj) {
        const int q = t + jj;
        if (q < nq) mx = mx + tapM(t, jj) * ld2(Xo + co(2 * q + p));
      }
      const size_t ro = co(2 * t + p);
      const double2 lx2 = 2.0 * (mx - ld2(Ri + ro));
      for (int l = stage + 1; l <= 4; ++l) {
        double* Rl = R + (size_t)(l - 1) * S + ro;
        st2(Rl, ld2(Rl) + c_AI[l][stage] * lx2);
      }
    }
  }
  return ok;
}

__global__ void k_solve(Grid g, Tables tb, double* X, double* Xs, const double* F, double* R, size_t S,
                        const double* wT, double* nu, int* flags, int B, int stage, const int* nsteps,
                        const int* step) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long per = 2L * g.nm;
  if (idx >= per * B) return;
  const int b = (int)(idx / per);
  if (!slice_active(nsteps, step, b)) return;
  const int rem = (int)(idx - (long)b * per);
  const int p = rem / g.nm, m = rem - p * g.nm;
  double* X0 = X + (size_t)b * S;
  double* Xo = (stage == 4) ? X0 : Xs + (size_t)b * S;
  const double* Fb = F + (size_t)b * S;
  double* Rb = R + (size_t)b * 4 * S;
  if (stage == 1 && m == 0 && p == 0 && nu != nullptr) {
    // Nu_V(t_n) (Eq. 9) of the step-start state: wall temperature difference of
    // the mean profile + Clenshaw-Curtis integral of <wT>_x; trapezoid weight.
    double cond = 0.0;
    for (int n = 1; n < g.Nz; n += 2) cond -= 2.0 * X0[soff(g, 0, n, 0)];
    double adv = 0.0;
    for (int jz = 0; jz < g.Mz; ++jz) adv = fma(__ldg(tb.cc + jz), wT[(size_t)b * g.Mz + jz], adv);
    const double nuv = cond + 0.5 * adv;
    nu[b] += ((*step == 0) ? 0.5 : 1.0) * g.dt * nuv;
  }
  bool ok;
  if (m == 0) {
    ok = solve_system<KT>(g, tb, stage, p, 0, X0, Xo, Fb, Rb, S);
    ok = solve_system<KU>(g, tb, stage, p, 0, X0, Xo, Fb, Rb, S) && ok;
  } else {
    ok = solve_system<KT>(g, tb, stage, p, m, X0, Xo, Fb, Rb, S);
    ok = solve_system<KP>(g, tb, stage, p, m, X0, Xo, Fb, Rb, S) && ok;
  }
  if (!ok) flags[b] = 1;
}

__global__ void k_advance(int* step) { *step += 1; }

static inline unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

// The dynamic shared-memory allowance of k_rows only ever grows, so that a
// later handle on a smaller grid does not shrink it below an earlier one's need.
cudaError_t configure_kernels(const Grid& g) {
  static int allowed = 48 * 1024;
  const int need = (int)rows_smem_bytes(g);
  if (need <= allowed) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
  if (e == cudaSuccess) allowed = need;
  return e;
}

cudaError_t launch_explicit(const Grid& g, const Tables& t, const Work& w, const double* X, int B, bool all_active,
                            cudaStream_t s) {
  const int* ns = all_active ? nullptr : w.nsteps;
  const size_t S = state_doubles(g);
  const int T1 = 128;
  k_zinv<<<nblk((long)B * g.Mz * g.nm, T1), T1, 0, s>>>(g, t.zinv, X, S, w.Z, B, ns, w.step);
  const int T2 = (g.Mx >= 768) ? 256 : 128;
  k_rows<<<(unsigned)(B * g.Mz), T2, rows_smem_bytes(g), s>>>(g, t.tw, w.Z, w.Q, w.wT, B, ns, w.step);
  return cudaGetLastError();
}

cudaError_t launch_stage(const Grid& g, const Tables& t, const Work& w, double* X, int B, int stage, double* nu,
                         cudaStream_t s) {
  const size_t S = state_doubles(g);
  const double* Xin = (stage == 1) ? X : w.Xs;
  cudaError_t e = launch_explicit(g, t, w, Xin, B, false, s);
  if (e != cudaSuccess) return e;
  const int T1 = 128;
  k_zfwd<<<nblk((long)B * 2 * g.Nz * g.nm, T1), T1, 0, s>>>(g, t.zfwd, w.Q, w.F, S, B, w.nsteps, w.step);
  const int T3 = 64;
  k_solve<<<nblk((long)B * 2 * g.nm, T3), T3, 0, s>>>(g, t, X, w.Xs, w.F, w.R, S, w.wT, nu, w.flags, B, stage,
                                                      w.nsteps, w.step);
  return cudaGetLastError();
}

cudaError_t launch_advance(const Work& w, cudaStream_t s) {
  k_advance<<<1, 1, 0, s>>>(w.step);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostics.
// ---------------------------------------------------------------------------
__global__ void k_nu_final(Grid g, const double* cc, const double* X, size_t S, const double* wT, double* nu,
                           const int* nsteps, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || nsteps[b] <= 0) return;
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
  k_nu_final<<<nblk(B, 128), 128, 0, s>>>(g, t.cc, X, state_doubles(g), w.wT, nu, w.nsteps, B);
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
  return cudaGetLastError();
}

// ||A_b - B_b||^2 (or ||A_b||^2 when Bm is null) of the temperature field of nst
// states: Parseval in x (weights 1 for m = 0, 2 otherwise), exact Chebyshev
// Gram matrix in z, times Lx / 2 (z in [-1/2, 1/2]).  Block per state,
// deterministic reduction.
__global__ void __launch_bounds__(256) k_l2_diff(Grid g, const double* gram, const double* A, const double* Bm,
                                                 double* out) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  const size_t S = state_doubles(g);
  const double* a = A + (size_t)b * S;
  const double* bb = Bm ? Bm + (size_t)b * S : nullptr;
  double acc = 0.0;
  for (int it = threadIdx.x; it < g.nm * g.Nz; it += blockDim.x) {
    const int m = it % g.nm, i = it / g.nm;
    double2 di = ld2(a + soff(g, 0, i, m));
    if (bb) di = di - ld2(bb + soff(g, 0, i, m));
    double2 s = {0.0, 0.0};
    for (int jn = (i & 1); jn < g.Nz; jn += 2) {
      double2 dj = ld2(a + soff(g, 0, jn, m));
      if (bb) dj = dj - ld2(bb + soff(g, 0, jn, m));
      s = s + __ldg(gram + (size_t)i * g.Nz + jn) * dj;
    }
    acc += (m == 0 ? 1.0 : 2.0) * (di.x * s.x + di.y * s.y);
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) out[b] = 0.5 * g.Lx * tot;
}

cudaError_t launch_l2_diff(const Grid& g, const Tables& t, const double* A, const double* Bm, int nst, double* out,
                           cudaStream_t s) {
  if (nst <= 0) return cudaSuccess;
  k_l2_diff<<<nst, 256, 0, s>>>(g, t.gram, A, Bm, out);
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
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Parareal transfer and correction (Eq. 20).
// ---------------------------------------------------------------------------
__global__ void k_restrict(Grid gf, Grid gc, const double* Xf, double* Xc) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2L * gc.Nz * gc.nm) return;
  const int m = idx % gc.nm;
  const int n = (idx / gc.nm) % gc.Nz;
  const int f = idx / ((long)gc.nm * gc.Nz);
  st2(Xc + soff(gc, f, n, m), ld2(Xf + soff(gf, f, n, m)));
}

cudaError_t launch_restrict(const Grid& gf, const Grid& gc, const double* Xf, double* Xc, cudaStream_t s) {
  k_restrict<<<nblk(2L * gc.Nz * gc.nm, 128), 128, 0, s>>>(gf, gc, Xf, Xc);
  return cudaGetLastError();
}

__global__ void k_prolong(Grid gf, Grid gc, const double* Xc, double* Xf) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2L * gf.Nz * gf.nm) return;
  const int m = idx % gf.nm;
  const int n = (idx / gf.nm) % gf.Nz;
  const int f = idx / ((long)gf.nm * gf.Nz);
  double2 v = {0.0, 0.0};
  if (m < gc.nm && n < gc.Nz) v = ld2(Xc + soff(gc, f, n, m));
  st2(Xf + soff(gf, f, n, m), v);
}

cudaError_t launch_prolong(const Grid& gf, const Grid& gc, const double* Xc, double* Xf, cudaStream_t s) {
  k_prolong<<<nblk(2L * gf.Nz * gf.nm, 128), 128, 0, s>>>(gf, gc, Xc, Xf);
  return cudaGetLastError();
}

// U = F + (prolong(Gnew) - prolong(Gold)), elementwise in that order.
__global__ void k_correct(Grid gf, Grid gc, const double* Ff, const double* Gnew, const double* Gold, double* U) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2L * gf.Nz * gf.nm) return;
  const int m = idx % gf.nm;
  const int n = (idx / gf.nm) % gf.Nz;
  const int f = idx / ((long)gf.nm * gf.Nz);
  double2 d = {0.0, 0.0};
  if (m < gc.nm && n < gc.Nz) d = ld2(Gnew + soff(gc, f, n, m)) - ld2(Gold + soff(gc, f, n, m));
  st2(U + soff(gf, f, n, m), ld2(Ff + soff(gf, f, n, m)) + d);
}

cudaError_t launch_correct(const Grid& gf, const Grid& gc, const double* Ff, const double* Gnew, const double* Gold,
                           double* Uout, cudaStream_t s) {
  k_correct<<<nblk(2L * gf.Nz * gf.nm, 128), 128, 0, s>>>(gf, gc, Ff, Gnew, Gold, Uout);
  return cudaGetLastError();
}

}  // namespace rbc
