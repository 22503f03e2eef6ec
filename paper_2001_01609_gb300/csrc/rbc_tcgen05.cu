// Tensor-core (tcgen05) z inverse transform for the mixed-precision path.
//
// The z inverse transform of one slice and one field is a dense contraction:
// C[(j, op)][col] = sum_n A[(j, op)][n] X[n][col], with A the values of
// d^q T_n / ds^q at the padded Lobatto points (rows interleaved as j * nops + op,
// nops = 4 for psi: V, VD, VD^2, VD^3; nops = 2 for T: V, VD) and X the state's
// Chebyshev coefficients (columns = Fourier mode x real/imaginary part).  It runs
// on the 5th-generation tensor cores with TF32 operands and split compensation:
// a = a_hi + a_lo, x = x_hi + x_lo (each a TF32 value), and
// A X ~ A_hi X_hi + A_hi X_lo + A_lo X_hi, accumulated in FP32 in tensor memory,
// which keeps about FP32 accuracy (the mixed mode computes the transforms and
// products in FP32).
//
// CTA per (slice, tile of 64 columns, 128-row tile of one field's operator
// rows).  Thread 0 starts bulk (TMA) copies of the operator images' K-chunks
// (pre-swizzled on the host, 16 KB each, hi and lo) into a ring of up to four
// shared-memory stages, while all threads convert the X tile (all K) from FP64
// into hi/lo TF32 operands; thread 0 then issues the MMAs of each chunk as it
// lands and refills a stage once its MMAs are done, and the four warps read
// the 128 x 64 FP32 accumulator from tensor memory and form the fields of the
// z-inverse output with the ik factors (the epilogue of k_zinv).
// Operands are K-major with the 128-byte swizzle; every mbarrier wait is bounded
// and reports through the slice's error flag, and nothing (MMA or copy) is in
// flight when a kernel frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "rbc_internal.h"

namespace rbc {

namespace {

constexpr int kTileN = 64;       // columns per CTA (32 Fourier modes x re/im)
constexpr int kTileM = 128;      // rows per MMA tile
constexpr int kChunkFloats = kTileM * 32;   // one 128-row image chunk of 128-byte rows: 16 KB
// threads of a tensor-core CTA: kTcGroups groups of four warps; in the
// epilogue warp w reads the accumulator's lane quarter w % 4 (the quarter a
// warp may access) and the column range w / 4 of kTileN / kTcGroups columns,
// so that kTcGroups times as many stores are in flight as with four warps
constexpr int kTcGroups = 2;
constexpr int kTcThreads = 128 * kTcGroups;
constexpr long long kWaitLimit = 1LL << 24;   // default spin limit of a bounded wait

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-elements per 128-byte swizzle row: 32 TF32 or 64 BF16 values
__host__ __device__ inline int tc_ke(const Grid& g) { return g.tcbf16 ? 64 : 32; }

// byte offset of the element at byte `kb` (< 128) of row r in a K-major, 128B-swizzled tile
__host__ __device__ inline uint32_t swz_b(int r, int kb) {
  return (uint32_t)(r * 128 + (((kb >> 4) ^ (r & 7)) << 4) + (kb & 15));
}

// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 16, sbo = 1024;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

// instruction descriptor: kind::tf32, FP32 accumulator, K-major A and B, M x N
__device__ __forceinline__ uint32_t instr_desc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor: kind::f16 with BF16 A and B, FP32 accumulator, K-major, M x N
__device__ __forceinline__ uint32_t instr_desc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// 3 MMAs (hi*hi, hi*lo, lo*hi) of one 32-byte K-step of the A and X operands
__device__ __forceinline__ void mma3(bool bf, uint32_t tmem, uint32_t ah, uint32_t al, uint32_t xh, uint32_t xl,
                                     uint32_t idesc, uint32_t acc0) {
  if (bf) {
    mma_bf16(tmem, smem_desc(ah), smem_desc(xh), idesc, acc0);
    mma_bf16(tmem, smem_desc(ah), smem_desc(xl), idesc, 1u);
    mma_bf16(tmem, smem_desc(al), smem_desc(xh), idesc, 1u);
  } else {
    mma_tf32(tmem, smem_desc(ah), smem_desc(xh), idesc, acc0);
    mma_tf32(tmem, smem_desc(ah), smem_desc(xl), idesc, 1u);
    mma_tf32(tmem, smem_desc(al), smem_desc(xh), idesc, 1u);
  }
}

// hi/lo split of an FP32 value x into the operand type, stored at byte offset
// o of the hi and lo tiles: TF32 (cvt.rna) or BF16 (round to nearest even)
__device__ __forceinline__ void store_split(bool bf, float x, unsigned char* hi, unsigned char* lo, uint32_t o) {
  if (bf) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    *reinterpret_cast<__nv_bfloat16*>(hi + o) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + o) = l;
  } else {
    const uint32_t h = to_tf32(x);
    const uint32_t l = to_tf32(x - __uint_as_float(h));
    *reinterpret_cast<uint32_t*>(hi + o) = h;
    *reinterpret_cast<uint32_t*>(lo + o) = l;
  }
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(mbar)));
}

// arrive on an mbarrier, announcing `bytes` of bulk-copy transactions for the phase
__device__ __forceinline__ void arrive_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(mbar)), "r"(bytes) : "memory");
}

// bulk (TMA) copy of `bytes` contiguous bytes, global -> shared, completing on mbar
// (both addresses 16-byte aligned, bytes a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(mbar))
      : "memory");
}

// bounded wait for the completion of phase `parity` of an mbarrier: at most
// `limit` polls (limit 0: gives up at once)
__device__ __forceinline__ bool wait_parity(uint64_t* mbar, uint32_t parity, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(saddr(mbar)), "r"(parity));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ size_t soff2(const Grid& g, int f, int n, int m) {
  return ((size_t)(f * g.Nz + n) * g.nm + m) * 2;
}

__device__ __forceinline__ void store_c(float* Zb, const Grid& g, int field, int j, int m, float re, float im) {
  const size_t fs = (size_t)g.Mz * g.nm * 2;
  *reinterpret_cast<float2*>(Zb + field * fs + ((size_t)j * g.nm + m) * 2) = make_float2(re, im);
}

// Spin limit of the waits that wait for MMAs to complete before the kernel goes
// on (set by tc_set_wait_limit; tests lower it to make the waits give up).
__device__ long long g_wait_limit = kWaitLimit;

// Error bits of a state and of its handle (kFlagTimeout when a wait gave up).
__device__ __forceinline__ void flag_timeout(int* flags, int* err, int b) {
  atomicOr(flags + b, kFlagTimeout);
  if (err) atomicOr(err, kFlagTimeout);
}

}  // namespace

cudaError_t tc_set_wait_limit(long long limit) {
  const long long v = limit < 0 ? kWaitLimit : limit;
  return cudaMemcpyToSymbol(g_wait_limit, &v, sizeof(v));
}

// Number of 128-row tiles and K-chunks of the operator images (host and device agree).
__host__ __device__ int tc_zinv_mtiles(const Grid& g, int nops) { return (nops * g.Mz + kTileM - 1) / kTileM; }
__host__ __device__ int tc_zinv_kchunks(const Grid& g) { return (g.Nz + tc_ke(g) - 1) / tc_ke(g); }
size_t tc_zinv_image_floats(const Grid& g, int nops) {
  return (size_t)tc_zinv_mtiles(g, nops) * tc_zinv_kchunks(g) * kChunkFloats;
}

// hi/lo split of v into the operand type of the grid, written at byte offset
// `off` of the hi and lo chunks: TF32 (hi = v rounded to 10 mantissa bits, lo
// = the rest, rounded alike) or BF16 (hi = v rounded to nearest even on 7
// mantissa bits, lo = the rest, rounded alike).
static void split_store(const Grid& g, double v, float* hi, float* lo, int off) {
  if (g.tcbf16) {
    auto bf = [](float x) {
      uint32_t u;
      memcpy(&u, &x, 4);
      u += 0x7FFFu + ((u >> 16) & 1u);          // round to nearest, ties to even
      return (uint16_t)(u >> 16);
    };
    auto fl = [](uint16_t b) {
      const uint32_t u = (uint32_t)b << 16;
      float x;
      memcpy(&x, &u, 4);
      return x;
    };
    const uint16_t h = bf((float)v);
    const uint16_t l = bf((float)(v - (double)fl(h)));
    memcpy(reinterpret_cast<unsigned char*>(hi) + off, &h, 2);
    memcpy(reinterpret_cast<unsigned char*>(lo) + off, &l, 2);
    return;
  }
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float h;
  memcpy(&h, &u, 4);
  float l = (float)(v - (double)h);
  memcpy(&u, &l, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  memcpy(&l, &u, 4);
  memcpy(reinterpret_cast<unsigned char*>(hi) + off, &h, 4);
  memcpy(reinterpret_cast<unsigned char*>(lo) + off, &l, 4);
}

// Pre-swizzled hi/lo operator images for field f (nops operators per row j),
// [mtile][kchunk][128 x 32 swizzled].  d[q][j][n] = d^q T_n / ds^q at s_j.
void tc_zinv_build_images(const Grid& g, const double* zinv, int nops, float* hi, float* lo) {
  const int mt = tc_zinv_mtiles(g, nops), kc = tc_zinv_kchunks(g), ke = tc_ke(g), es = 128 / ke;
  for (int t = 0; t < mt; ++t)
    for (int c = 0; c < kc; ++c) {
      float* bh = hi + ((size_t)t * kc + c) * kChunkFloats;
      float* bl = lo + ((size_t)t * kc + c) * kChunkFloats;
      for (int r = 0; r < kTileM; ++r)
        for (int k = 0; k < ke; ++k) {
          const int row = t * kTileM + r, j = row / nops, q = row % nops, n = c * ke + k;
          double v = 0.0;
          if (j < g.Mz && n < g.Nz) v = zinv[((size_t)q * g.Mz + j) * g.Nz + n];
          split_store(g, v, bh, bl, (int)swz_b(r, k * es));
        }
    }
}

// Operator-image stages (16 KB hi + 16 KB lo per K-chunk) of k_zinv_tc: up to
// four, as many as fit beside the X tile in 200 KB of shared memory.
static int tc_zinv_stages(const Grid& g) {
  const int kc = tc_zinv_kchunks(g);
  for (int nb = std::min(kc, 4); nb > 1; --nb)
    if ((size_t)kc * kTileN * 128 * 2 + (size_t)nb * 2 * kTileM * 128 + 1024 <= 200 * 1024) return nb;
  return 1;
}

size_t tc_zinv_smem_bytes(const Grid& g) {
  // X tile hi/lo (all K), the A-chunk stages hi/lo, alignment slack
  return (size_t)tc_zinv_kchunks(g) * kTileN * 128 * 2 + (size_t)tc_zinv_stages(g) * 2 * kTileM * 128 + 1024;
}

// Output fields: psi (nops = 4): u, w, d_x omega, d_z omega, d_x u, d_z u (0..5);
// T (nops = 2): T, d_x T, d_z T (6..8).
// CTA per (slice, 64-column tile, field, group of 128-row tiles of the field's
// operator rows): one row tile per CTA when K is at most two 32-wide chunks
// (the X tile is cheap to convert, and a single slice spreads over more CTAs),
// all of the field's row tiles otherwise (the X tile, converted once, serves
// them all).  Thread 0 streams the K-chunks of the operator images, tile after
// tile, into a ring of NB shared-memory stages with bulk (TMA) copies while all
// threads convert the X tile to hi/lo TF32 operands; it issues 3 x 4 MMAs per
// chunk as each lands, refilling a stage once its MMAs completed (so the next
// tile's chunks arrive during the current tile's epilogue); after each tile
// the four warps read the accumulator and form the fields.
__host__ __device__ inline bool tc_zinv_tile_per_cta(const Grid& g) { return tc_zinv_kchunks(g) <= 2; }

__global__ void __launch_bounds__(kTcThreads) k_zinv_tc(Grid g, const float* __restrict__ Ahi_psi,
                                                 const float* __restrict__ Alo_psi, const float* __restrict__ Ahi_T,
                                                 const float* __restrict__ Alo_T, const double* __restrict__ X,
                                                 size_t S, float* __restrict__ Z, int B, const int* nsteps,
                                                 const int* step, int* flags, int* err, int NB) {
  pdl_wait();
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[4], empty[4], accb[1];
  __shared__ uint32_t tmem_base;
  const int ntile = (2 * g.nm + kTileN - 1) / kTileN;
  const int mt4 = tc_zinv_mtiles(g, 4), mt2 = tc_zinv_mtiles(g, 2);
  const bool one = tc_zinv_tile_per_cta(g);
  const int units = one ? mt4 + mt2 : 2;      // CTAs per (slice, column tile)
  const int per_b = ntile * units;
  const int b = blockIdx.x / per_b;
  int rem = blockIdx.x - b * per_b;
  const int ct = rem / units;
  const int q = rem - ct * units;
  const int fsel = one ? (q < mt4 ? 0 : 1) : q;   // 0: psi (nops 4), 1: T (nops 2)
  const int t0 = one ? (q < mt4 ? q : q - mt4) : 0;
  const int t1 = one ? t0 + 1 : (fsel == 0 ? mt4 : mt2);
  const int c0 = ct * kTileN;
  if (b >= B || !(nsteps == nullptr || *step < nsteps[b])) return;   // uniform per block
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nops = fsel == 0 ? 4 : 2;
  const int f = fsel == 0 ? 1 : 0;            // state field: psi slot 1, T slot 0
  const int kc = tc_zinv_kchunks(g);
  const int nchunks = (t1 - t0) * kc;         // the chunks this CTA streams, tile after tile
  const float* Ahi = (fsel == 0 ? Ahi_psi : Ahi_T) + (size_t)t0 * kc * kChunkFloats;
  const float* Alo = (fsel == 0 ? Alo_psi : Alo_T) + (size_t)t0 * kc * kChunkFloats;
  constexpr uint32_t kChunkBytes = kChunkFloats * 4;   // one image chunk, 16 KB
  const bool bf = g.tcbf16 != 0;
  const int ke = tc_ke(g), es = 128 / ke, lke = bf ? 6 : 5;   // ke = 2^lke
  unsigned char* sXhi = base;
  unsigned char* sXlo = sXhi + (size_t)kc * kTileN * 128;
  unsigned char* sA = sXlo + (size_t)kc * kTileN * 128;   // [stage][hi, lo][128 x 128 B]
  uint32_t seen_full[4] = {0, 0, 0, 0}, copies[4] = {0, 0, 0, 0};   // thread 0's bookkeeping
  uint32_t seen_empty[4] = {0, 0, 0, 0}, commits[4] = {0, 0, 0, 0};
  uint32_t acc_commits = 0, acc_seen = 0;
  if (tid == 0) {
    for (int i = 0; i < NB; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&accb[0])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    // the first NB chunks of the operator images start streaming in at once
    for (int c = 0; c < NB && c < nchunks; ++c) {
      unsigned char* ah = sA + (size_t)c * 2 * kTileM * 128;
      arrive_expect_tx(&full[c], 2 * kChunkBytes);
      bulk_g2s(ah, Ahi + (size_t)c * kChunkFloats, kChunkBytes, &full[c]);
      bulk_g2s(ah + kTileM * 128, Alo + (size_t)c * kChunkFloats, kChunkBytes, &full[c]);
      copies[c]++;
    }
  }
  if (warp == 0) {
    __syncwarp();                             // the warp converged again after thread 0's set-up
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // X tile -> hi/lo TF32 operands, K-major (row = column of the tile, k = n)
  // (four consecutive columns, two modes, per item: 16-byte loads, several in flight)
  const double* Xb = X + (size_t)b * S;
#pragma unroll 4
  for (int it = tid; it < kc * ke * (kTileN / 4); it += blockDim.x) {
    const int n = it / (kTileN / 4), col = (it - n * (kTileN / 4)) * 4;
    const int gc = c0 + col;                  // even: columns gc .. gc+3 are modes gc/2, gc/2 + 1
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    if (n < g.Nz) {
      const double* src = Xb + soff2(g, f, n, gc >> 1);
      if (gc + 3 < 2 * g.nm) {
        const double2 v0 = *reinterpret_cast<const double2*>(src);
        const double2 v1 = *reinterpret_cast<const double2*>(src + 2);
        v[0] = v0.x; v[1] = v0.y; v[2] = v1.x; v[3] = v1.y;
      } else {
        for (int e = 0; e < 4; ++e)
          if (gc + e < 2 * g.nm) v[e] = src[e];
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const uint32_t o = (uint32_t)(n >> lke) * kTileN * 128 + swz_b(col + e, (n & (ke - 1)) * es);
      store_split(bf, (float)v[e], sXhi, sXlo, o);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = bf ? instr_desc_bf16(kTileM, kTileN) : instr_desc_tf32(kTileM, kTileN);
  const long long limit = g_wait_limit;
  bool issued_all = true;
  bool ok = true;
  float* Zb = Z + (size_t)b * 9 * g.Mz * g.nm * 2;
  for (int t = t0; t < t1 && ok; ++t) {
    if (tid == 0) {
      for (int c = 0; c < kc; ++c) {
        const int gi = (t - t0) * kc + c, buf = gi % NB;
        if (!wait_parity(&full[buf], seen_full[buf] & 1, limit)) {
          issued_all = false;
          break;
        }
        seen_full[buf]++;
        asm volatile("tcgen05.fence::after_thread_sync;");
        unsigned char* ah = sA + (size_t)buf * 2 * kTileM * 128;
        unsigned char* al = ah + (size_t)kTileM * 128;
        const uint32_t xh = saddr(sXhi) + (uint32_t)c * kTileN * 128;
        const uint32_t xl = saddr(sXlo) + (uint32_t)c * kTileN * 128;
        for (int ks = 0; ks < 4; ++ks) {       // four 32-byte K-steps per 128-byte row
          const uint32_t o = ks * 32;
          const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
          mma3(bf, tmem, saddr(ah) + o, saddr(al) + o, xh + o, xl + o, idesc, acc0);
        }
        commit(&empty[buf]);
        commits[buf]++;
        if (gi + NB < nchunks) {              // refill the stage once its MMAs are done
          if (!wait_parity(&empty[buf], seen_empty[buf] & 1, limit)) {
            issued_all = false;
            break;
          }
          seen_empty[buf]++;
          arrive_expect_tx(&full[buf], 2 * kChunkBytes);
          bulk_g2s(ah, Ahi + (size_t)(gi + NB) * kChunkFloats, kChunkBytes, &full[buf]);
          bulk_g2s(al, Alo + (size_t)(gi + NB) * kChunkFloats, kChunkBytes, &full[buf]);
          copies[buf]++;
        }
      }
      if (issued_all) {
        commit(&accb[0]);
        acc_commits++;
      }
    }
    // accumulator of tile t ready (thread 0 committed it after the tile's last chunk)
    const bool acc_done = wait_parity(&accb[0], (uint32_t)(t - t0) & 1, limit);
    if (tid == 0 && acc_done) acc_seen++;
    ok = __syncthreads_and(acc_done && issued_all) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) break;
    const int rows_per_j = nops, jper = kTileM / nops;
    const int r = (warp & 3) * 32 + lane;     // tile row = TMEM lane
    const int jl = r / rows_per_j, op = r % rows_per_j;
    const int j = t * jper + jl;
    const int cbeg = (warp >> 2) * (kTileN / kTcGroups);
    for (int cc = cbeg; cc < cbeg + kTileN / kTcGroups; cc += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + cc, v);
      float P[4][16];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq)
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int src = (lane & ~(rows_per_j - 1)) | (qq & (rows_per_j - 1));
          P[qq][i] = __shfl_sync(0xffffffffu, v[i], src);
        }
      if (j >= g.Mz) continue;
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        const int gc = c0 + cc + i;
        if (gc >= 2 * g.nm) break;
        const int m = gc >> 1;
        const float k = (float)(g.kfac * m);
        if (nops == 4) {
          // P[q] = (re, im) of d^q psi/ds^q (m = 0: of U)
          const float p0r = P[0][i], p0i = P[0][i + 1], p1r = P[1][i], p1i = P[1][i + 1];
          const float p2r = P[2][i], p2i = P[2][i + 1], p3r = P[3][i], p3i = P[3][i + 1];
          if (m == 0) {
            if (op == 0) {
              store_c(Zb, g, 0, j, 0, p0r, 0.f);            // u = U
              store_c(Zb, g, 1, j, 0, 0.f, 0.f);            // w
            } else if (op == 1) {
              store_c(Zb, g, 2, j, 0, 0.f, 0.f);            // d_x omega
              store_c(Zb, g, 3, j, 0, -4.f * p2r, 0.f);     // d_z omega = -U_zz
            } else if (op == 2) {
              store_c(Zb, g, 4, j, 0, 0.f, 0.f);            // d_x u
              store_c(Zb, g, 5, j, 0, 2.f * p1r, 0.f);      // d_z u = U_z
            }
          } else if (op == 0) {
            store_c(Zb, g, 0, j, m, 2.f * p1r, 2.f * p1i);  // u = d_z psi
            store_c(Zb, g, 1, j, m, k * p0i, -k * p0r);     // w = -ik psi
          } else if (op == 1) {
            const float omr = k * k * p0r - 4.f * p2r, omi = k * k * p0i - 4.f * p2i;
            store_c(Zb, g, 2, j, m, -k * omi, k * omr);     // d_x omega = ik omega
            store_c(Zb, g, 3, j, m, 2.f * k * k * p1r - 8.f * p3r, 2.f * k * k * p1i - 8.f * p3i);
          } else if (op == 2) {
            store_c(Zb, g, 4, j, m, -k * 2.f * p1i, k * 2.f * p1r);   // d_x u = ik u
            store_c(Zb, g, 5, j, m, 4.f * p2r, 4.f * p2i);            // d_z u
          }
        } else {
          const float tr = P[0][i], ti = P[0][i + 1], dr = P[1][i], di = P[1][i + 1];
          if (op == 0) {
            store_c(Zb, g, 6, j, m, tr, ti);                          // T
            store_c(Zb, g, 7, j, m, m == 0 ? 0.f : -k * ti, m == 0 ? 0.f : k * tr);   // d_x T
          } else {
            store_c(Zb, g, 8, j, m, 2.f * dr, 2.f * di);              // d_z T
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();                          // accumulator read before the next tile overwrites it
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (!ok && tid == 0) flag_timeout(flags, err, b);   // a bounded wait gave up
  if (tid == 0) {
    // nothing may be in flight when the kernel frees tensor memory and exits:
    // the MMAs (their commits) and the bulk copies (their stages), with the
    // default limit, in order
    for (int i = 0; i < NB; ++i) {
      while (seen_full[i] < copies[i]) {
        if (!wait_parity(&full[i], seen_full[i] & 1, kWaitLimit)) break;
        seen_full[i]++;
      }
      while (seen_empty[i] < commits[i]) {
        if (!wait_parity(&empty[i], seen_empty[i] & 1, kWaitLimit)) break;
        seen_empty[i]++;
      }
    }
    if (acc_seen < acc_commits) wait_parity(&accb[0], acc_seen & 1, kWaitLimit);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// ---------------------------------------------------------------------------
// Tensor-core z forward transform for the mixed-precision path.
//
// For one slice, one field and one Chebyshev parity p the z-forward transform
// is F[n][col] = sum_{jh < ceil(Mz/2)} W[n][jh] fold_p[jh][col], n = 2r + p,
// with fold_0 = Q_j + Q_{Mz-1-j} and fold_1 = Q_j - Q_{Mz-1-j} (the middle row
// of an odd Mz once in fold_0) and col = (Fourier mode, real/imaginary part).
// CTA per (slice, field, parity, 64-column tile): the folds are formed in FP32
// from the row kernel's output, split into hi/lo TF32 operands in shared memory
// (K-major, 128-byte swizzle); the rows of W of parity p are pre-split images
// [mtile][kchunk][128 x 32]; three MMAs per 8-wide K step (hi*hi, hi*lo, lo*hi)
// accumulate in tensor memory; the epilogue writes F in FP64 for the solve.
// The waits, the drain and the tensor-memory release follow k_zinv_tc.
// ---------------------------------------------------------------------------
__host__ __device__ int tc_zfwd_mtiles(const Grid& g) { return (g.Nz / 2 + kTileM - 1) / kTileM; }
__host__ __device__ int tc_zfwd_kchunks(const Grid& g) { return ((g.Mz + 1) / 2 + tc_ke(g) - 1) / tc_ke(g); }
size_t tc_zfwd_image_floats(const Grid& g) { return (size_t)tc_zfwd_mtiles(g) * tc_zfwd_kchunks(g) * kChunkFloats; }

void tc_zfwd_build_images(const Grid& g, const double* zfwd, int p, float* hi, float* lo) {
  const int mt = tc_zfwd_mtiles(g), kc = tc_zfwd_kchunks(g), Mh = (g.Mz + 1) / 2, ke = tc_ke(g), es = 128 / ke;
  for (int t = 0; t < mt; ++t)
    for (int c = 0; c < kc; ++c) {
      float* bh = hi + ((size_t)t * kc + c) * kChunkFloats;
      float* bl = lo + ((size_t)t * kc + c) * kChunkFloats;
      for (int r = 0; r < kTileM; ++r)
        for (int k = 0; k < ke; ++k) {
          const int n = 2 * (t * kTileM + r) + p, jh = c * ke + k;
          const double v = (n < g.Nz && jh < Mh) ? zfwd[(size_t)n * g.Mz + jh] : 0.0;
          split_store(g, v, bh, bl, (int)swz_b(r, k * es));
        }
    }
}

// Image stages of k_zfwd_tc, as for k_zinv_tc.
static int tc_zfwd_stages(const Grid& g) {
  const int kc = tc_zfwd_kchunks(g);
  for (int nb = std::min(kc, 4); nb > 1; --nb)
    if ((size_t)kc * kTileN * 128 * 2 + (size_t)nb * 2 * kTileM * 128 + 1024 <= 200 * 1024) return nb;
  return 1;
}

size_t tc_zfwd_smem_bytes(const Grid& g) {
  return (size_t)tc_zfwd_kchunks(g) * kTileN * 128 * 2 + (size_t)tc_zfwd_stages(g) * 2 * kTileM * 128 + 1024;
}
// Grid-only choices (so a state gives the same bits in any batch): the tensor
// cores take grids with at least 64 Chebyshev coefficients whose operands fit
// in 200 KB of shared memory.  Below Nz = 64 a transform is one or two 32-wide
// K-chunks, and the FP32 CUDA-core kernels finish sooner (measured on a
// single 128 x 32 slice: 0.123 ms per RK443 step against 0.187 ms).
bool tc_zfwd_supported(const Grid& g) { return g.Nz >= 64 && tc_zfwd_smem_bytes(g) <= 200 * 1024; }

// CTA per (slice, field, parity, 64-column tile, 128-row tile of W's rows of
// that parity); the images stream in through the bulk-copy ring of k_zinv_tc.
__global__ void __launch_bounds__(kTcThreads) k_zfwd_tc(Grid g, const float* __restrict__ Whi0, const float* __restrict__ Wlo0,
                                                 const float* __restrict__ Whi1, const float* __restrict__ Wlo1,
                                                 const float* __restrict__ Q, double* __restrict__ F, size_t S, int B,
                                                 const int* nsteps, const int* step, int* flags, int* err, int NB) {
  pdl_wait();
  extern __shared__ __align__(1024) unsigned char tc_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[4], empty[4], accb[1];
  __shared__ uint32_t tmem_base;
  const int ntile = (2 * g.nm + kTileN - 1) / kTileN;
  const int mtiles = tc_zfwd_mtiles(g);
  const int per_b = 2 * 2 * ntile * mtiles;
  const int b = blockIdx.x / per_b;
  int rem = blockIdx.x - b * per_b;
  const int f = rem / (2 * ntile * mtiles);
  rem -= f * 2 * ntile * mtiles;
  const int p = rem / (ntile * mtiles);
  rem -= p * ntile * mtiles;
  const int ct = rem / mtiles, t = rem - ct * mtiles;
  const int c0 = ct * kTileN;
  if (b >= B || !(nsteps == nullptr || *step < nsteps[b])) return;   // uniform per block
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kc = tc_zfwd_kchunks(g), Mh = (g.Mz + 1) / 2;
  const float* Ahi = (p == 0 ? Whi0 : Whi1) + (size_t)t * kc * kChunkFloats;
  const float* Alo = (p == 0 ? Wlo0 : Wlo1) + (size_t)t * kc * kChunkFloats;
  constexpr uint32_t kChunkBytes = kChunkFloats * 4;
  const bool bf = g.tcbf16 != 0;
  const int ke = tc_ke(g), es = 128 / ke, lke = bf ? 6 : 5;   // ke = 2^lke
  unsigned char* sXhi = base;
  unsigned char* sXlo = sXhi + (size_t)kc * kTileN * 128;
  unsigned char* sA = sXlo + (size_t)kc * kTileN * 128;   // [stage][hi, lo][128 x 128 B]
  uint32_t seen_full[4] = {0, 0, 0, 0}, copies[4] = {0, 0, 0, 0};
  uint32_t seen_empty[4] = {0, 0, 0, 0}, commits[4] = {0, 0, 0, 0};
  uint32_t acc_commits = 0, acc_seen = 0;
  if (tid == 0) {
    for (int i = 0; i < NB; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&accb[0])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    for (int c = 0; c < NB && c < kc; ++c) {
      unsigned char* ah = sA + (size_t)c * 2 * kTileM * 128;
      arrive_expect_tx(&full[c], 2 * kChunkBytes);
      bulk_g2s(ah, Ahi + (size_t)c * kChunkFloats, kChunkBytes, &full[c]);
      bulk_g2s(ah + kTileM * 128, Alo + (size_t)c * kChunkFloats, kChunkBytes, &full[c]);
      copies[c]++;
    }
  }
  if (warp == 0) {
    __syncwarp();                             // the warp converged again after thread 0's set-up
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // folds of parity p -> hi/lo TF32 operands, K-major (row = column of the tile, k = jh)
  // (four consecutive columns per item: 16-byte loads, several in flight)
  const float* q = Q + (size_t)(b * 2 + f) * g.Mz * g.nm * 2;
  const bool vec = (2 * g.nm) % 4 == 0;
#pragma unroll 4
  for (int it = tid; it < kc * ke * (kTileN / 4); it += blockDim.x) {
    const int jh = it / (kTileN / 4), col = (it - jh * (kTileN / 4)) * 4;
    const int jr = g.Mz - 1 - jh;
    float a[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    if (jh < Mh) {
      const float* ra = q + (size_t)jh * g.nm * 2 + c0 + col;
      const float* rc = q + (size_t)jr * g.nm * 2 + c0 + col;
      if (vec && c0 + col + 3 < 2 * g.nm) {
        const float4 va = *reinterpret_cast<const float4*>(ra);
        a[0] = va.x; a[1] = va.y; a[2] = va.z; a[3] = va.w;
        if (jr != jh) {
          const float4 vc = *reinterpret_cast<const float4*>(rc);
          c[0] = vc.x; c[1] = vc.y; c[2] = vc.z; c[3] = vc.w;
        }
      } else {
        for (int e = 0; e < 4; ++e)
          if (c0 + col + e < 2 * g.nm) {
            a[e] = ra[e];
            if (jr != jh) c[e] = rc[e];
          }
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float x = 0.f;
      if (jh < Mh && c0 + col + e < 2 * g.nm) x = (jr != jh) ? (p == 0 ? a[e] + c[e] : a[e] - c[e]) : (p == 0 ? a[e] : 0.f);
      const uint32_t o = (uint32_t)(jh >> lke) * kTileN * 128 + swz_b(col + e, (jh & (ke - 1)) * es);
      store_split(bf, x, sXhi, sXlo, o);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = bf ? instr_desc_bf16(kTileM, kTileN) : instr_desc_tf32(kTileM, kTileN);
  const long long limit = g_wait_limit;
  bool issued_all = true;
  if (tid == 0) {
    for (int c = 0; c < kc; ++c) {
      const int buf = c % NB;
      if (!wait_parity(&full[buf], seen_full[buf] & 1, limit)) {
        issued_all = false;
        break;
      }
      seen_full[buf]++;
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned char* ah = sA + (size_t)buf * 2 * kTileM * 128;
      unsigned char* al = ah + (size_t)kTileM * 128;
      const uint32_t xh = saddr(sXhi) + (uint32_t)c * kTileN * 128;
      const uint32_t xl = saddr(sXlo) + (uint32_t)c * kTileN * 128;
      for (int ks = 0; ks < 4; ++ks) {         // four 32-byte K-steps per 128-byte row
        const uint32_t o = ks * 32;
        const uint32_t acc0 = (c > 0 || ks > 0) ? 1u : 0u;
        mma3(bf, tmem, saddr(ah) + o, saddr(al) + o, xh + o, xl + o, idesc, acc0);
      }
      commit(&empty[buf]);
      commits[buf]++;
      if (c + NB < kc) {
        if (!wait_parity(&empty[buf], seen_empty[buf] & 1, limit)) {
          issued_all = false;
          break;
        }
        seen_empty[buf]++;
        arrive_expect_tx(&full[buf], 2 * kChunkBytes);
        bulk_g2s(ah, Ahi + (size_t)(c + NB) * kChunkFloats, kChunkBytes, &full[buf]);
        bulk_g2s(al, Alo + (size_t)(c + NB) * kChunkFloats, kChunkBytes, &full[buf]);
        copies[buf]++;
      }
    }
    if (issued_all) {
      commit(&accb[0]);
      acc_commits = 1;
    }
  }
  const bool acc_done = wait_parity(&accb[0], 0, limit);
  if (tid == 0 && acc_done) acc_seen = 1;
  const bool ok = __syncthreads_and(acc_done && issued_all) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    double* Fb = F + (size_t)b * S;
    const int n = 2 * (t * kTileM + (warp & 3) * 32 + lane) + p;   // tile row = TMEM lane
    const int cbeg = (warp >> 2) * (kTileN / kTcGroups);
    for (int cc = cbeg; cc < cbeg + kTileN / kTcGroups; cc += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + cc, v);
      if (n >= g.Nz) continue;
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        const int gc = c0 + cc + i;
        if (gc >= 2 * g.nm) break;
        *reinterpret_cast<double2*>(Fb + soff2(g, f, n, gc >> 1)) = make_double2((double)v[i], (double)v[i + 1]);
      }
    }
  }
  if (!ok && tid == 0) flag_timeout(flags, err, b);   // a bounded wait gave up
  if (tid == 0) {
    for (int i = 0; i < NB; ++i) {
      while (seen_full[i] < copies[i]) {
        if (!wait_parity(&full[i], seen_full[i] & 1, kWaitLimit)) break;
        seen_full[i]++;
      }
      while (seen_empty[i] < commits[i]) {
        if (!wait_parity(&empty[i], seen_empty[i] & 1, kWaitLimit)) break;
        seen_empty[i]++;
      }
    }
    if (acc_seen < acc_commits) wait_parity(&accb[0], 0, kWaitLimit);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

cudaError_t launch_zfwd_tc(const Grid& g, const Tables& t, const Work& w, int B, cudaStream_t s) {
  static int allowed = 48 * 1024;
  const size_t smem = tc_zfwd_smem_bytes(g);
  if ((int)smem > allowed) {
    cudaError_t e = cudaFuncSetAttribute(k_zfwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    allowed = (int)smem;
  }
  const int ntile = (2 * g.nm + kTileN - 1) / kTileN;
  return launch_pdl(w.pdl != 0, k_zfwd_tc, (unsigned)(B * 2 * 2 * ntile * tc_zfwd_mtiles(g)), kTcThreads, smem, s, g,
                    t.tcW_hi[0], t.tcW_lo[0], t.tcW_hi[1], t.tcW_lo[1], reinterpret_cast<const float*>(w.Q), w.F,
                    state_doubles(g), B, w.nsteps, w.step, w.flags, w.err, tc_zfwd_stages(g));
}

cudaError_t launch_zinv_tc(const Grid& g, const Tables& t, const Work& w, const double* X, int B, const int* ns,
                           cudaStream_t s) {
  static int allowed = 48 * 1024;
  const size_t smem = tc_zinv_smem_bytes(g);
  if ((int)smem > allowed) {
    cudaError_t e = cudaFuncSetAttribute(k_zinv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    allowed = (int)smem;
  }
  const int ntile = (2 * g.nm + kTileN - 1) / kTileN;
  const int units = tc_zinv_tile_per_cta(g) ? tc_zinv_mtiles(g, 4) + tc_zinv_mtiles(g, 2) : 2;
  return launch_pdl(w.pdl != 0, k_zinv_tc, (unsigned)(B * ntile * units), kTcThreads, smem, s, g, t.tcA_psi_hi,
                    t.tcA_psi_lo, t.tcA_T_hi, t.tcA_T_lo, X, state_doubles(g), reinterpret_cast<float*>(w.Z), B, ns,
                    w.step, w.flags, w.err, tc_zinv_stages(g));
}

bool tc_zinv_supported(const Grid& g) { return g.Nz >= 64 && tc_zinv_smem_bytes(g) <= 200 * 1024; }

}  // namespace rbc
