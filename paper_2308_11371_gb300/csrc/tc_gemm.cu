// Grouped principal contractions on the 5th-generation tensor cores (tcgen05).
//
// The ROM operators of Eq. 43 are linear combinations of a few principal
// operators (Remark 7), so every cell's column is multiplied by the SAME
// principal matrices: Y[:, c] = sum_k coef_k(c) A_k X[:, c] (Eqs. 46a, 48, 49,
// Algorithm 3).  Written as one GEMM per use:
//   combine  : A = [A_1 ... A_nk] (K-concatenated), B column c = [coef_k(c) X_c]_k
//   separate : batch over k, B = X shared (Eq. 46a keeps every R column)
// with BF16 operands (optionally split into hi + lo BF16 terms, three products
// A_hi X_hi + A_hi X_lo + A_lo X_hi, for ~16-bit input precision) and FP32
// accumulation in TMEM.
//
// Kernel: one CTA per (n-tile, m-tile, batch); warp 0 lane 0 streams 128x64 A
// tiles and BNx64 B tiles with cp.async.bulk into a STAGES-deep mbarrier ring;
// warp 1 lane 0 issues tcgen05.mma (M=128, N=BN, K=16) and commits each stage
// back to the producer; all four warps drain the accumulator with tcgen05.ld.
// Operands are pre-packed in global memory in the canonical 128-byte-swizzled
// K-major layout, so a linear bulk copy lands the exact shared-memory image.
// Every mbarrier wait is bounded by the caller's budget (wait_ns of globaltimer,
// 1 s by default): on expiry the CTA sets an error flag and every role stops.
// Before TMEM is freed and the CTA exits, the copy issuer waits for each of its
// bulk copies to land and the MMA issuer commits a final barrier and waits for
// it (every MMA issued has completed, every earlier commit has arrived).  Those
// drain waits have their own fixed 1 s bound, independent of the budget, so even
// a budget of 1 ns leaves no asynchronous write aimed at a CTA that has exited.
#include <cuda_bf16.h>

#include <cstdint>
#include <cmath>

#include "common.cuh"

namespace fetidp {

namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;                     // bf16 elements per 128-byte row
constexpr int A_TILE = TC_BM * TC_BK * 2;     // 16 KB
constexpr unsigned long long kDrainNs = 1000000000ull;   // fixed bound of the exit drains

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false after wait_ns of globaltimer or when another role has aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long wait_ns) {
  const unsigned long long t0 = gtime();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63u) == 63u) {
      if (*abort_flag) return false;
      if (gtime() - t0 > wait_ns) return false;
    }
  }
}
// exit drain: wait for a phase that is certain to complete (an issued copy, a committed MMA
// batch), ignoring the abort flag, bounded by kDrainNs
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = gtime();
  while (!mbar_try(bar, parity) && gtime() - t0 < kDrainNs) {
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups
// 1024 bytes apart.  start address >> 4 in bits 0-13, SBO >> 4 in bits 32-45,
// descriptor version 1 at bit 46, layout type SWIZZLE_128B (2) in bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1)
// or f16 (0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, bool bf16) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row r, k-index q in [0, 64)) inside a SW128 K-major tile.
__host__ __device__ __forceinline__ uint32_t sw128_offset(int r, int q) {
  const int chunk = q >> 3;
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (r & 7)) << 4) + ((q & 7) << 1));
}

}  // namespace

struct TcParams {
  const uint8_t* A;
  const uint8_t* B;
  int m_tiles, n_tiles, k_tiles;
  long long a_batch_stride;   // bytes
  long long b_batch_stride;   // bytes
  int M;
  long long ncols, ncell;
  void* Y;
  int y_f64;
  long long y_rs;
  int y_cs;
  long long y_b_stride;
  double alpha, beta;
  int* err;
  unsigned long long wait_ns;          // bound of every pipeline wait
  long long a_bytes, b_bytes, y_ext;   // extents for checked builds
  int batch, bgroup;                   // operators, and operators per L2-resident group
};

namespace {

template <int BN, int STAGES>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(TcParams P) {
  constexpr int B_TILE = BN * TC_BK * 2;
  constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
  constexpr uint32_t IDESC = make_idesc(TC_BM, BN, true);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_TILE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + STAGES * B_TILE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTA order: groups of bgroup operators; within a group the column tile is the slowest index, so
  // consecutive CTAs share one B tile (read from DRAM once per group) while the group's A tiles
  // stay resident in L2 across the column tiles
  int nt, mt, bz;
  {
    const long long bid = blockIdx.x;
    const long long per_group = (long long)P.n_tiles * P.m_tiles * P.bgroup;
    const int g = (int)(bid / per_group);
    const long long r = bid - (long long)g * per_group;
    const int gb = min(P.bgroup, P.batch - g * P.bgroup);
    nt = (int)(r / ((long long)P.m_tiles * gb));
    const int r2 = (int)(r - (long long)nt * P.m_tiles * gb);
    bz = g * P.bgroup + r2 / P.m_tiles;
    mt = r2 - (r2 / P.m_tiles) * P.m_tiles;
  }
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int KT = P.k_tiles;
  const int rot = (int)(((long long)nt + mt + (long long)P.m_tiles * bz) % KT);
  const uint8_t* Ab = P.A + bz * P.a_batch_stride + (long long)mt * KT * A_TILE;
  const uint8_t* Bb = P.B + bz * P.b_batch_stride + (long long)nt * KT * B_TILE;
  if (warp == 0 && lane == 0) {
    // ---------------- producer: bulk copies into the ring
    int issued = 0;
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES, n = kt / STAGES;
      if (kt >= STAGES && !mbar_wait(empty0 + 8 * s, (uint32_t)((n - 1) & 1), abort_flag, P.wait_ns)) {
        *abort_flag = 1;
        atomicExch(P.err, 1);
        break;
      }
      // k tiles in rotated order: CTAs that share A tiles (same row tile and operator) differ
      // in nt, CTAs that share B tiles differ in (mt, bz); the rotation keeps them off the
      // same L2 lines at the same time (the accumulation order only changes rounding)
      const int kr = (kt + rot) % KT;
      const long long aoff = (Ab - P.A) + (long long)kr * A_TILE, boff = (Bb - P.B) + (long long)kr * B_TILE;
      if (!FD_INB(aoff + A_TILE - 1, P.a_bytes, 101) || !FD_INB(boff + B_TILE - 1, P.b_bytes, 102)) {
        *abort_flag = 1;
        atomicExch(P.err, 4);
        break;
      }
      mbar_expect_tx(full0 + 8 * s, A_TILE + B_TILE);
      bulk_g2s(smem_u32(sA + s * A_TILE), Ab + (long long)kr * A_TILE, A_TILE, full0 + 8 * s);
      bulk_g2s(smem_u32(sB + s * B_TILE), Bb + (long long)kr * B_TILE, B_TILE, full0 + 8 * s);
      ++issued;
    }
    // exit drain: every copy issued has landed (earlier stages were seen released before their
    // slot was reused).  The MMA thread drains its own commits; without an abort the last stages'
    // releases are also awaited here.
    for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
      mbar_drain(full0 + 8 * (kt % STAGES), (uint32_t)((kt / STAGES) & 1));
    for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued && !*abort_flag; ++kt)
      if (!mbar_wait(empty0 + 8 * (kt % STAGES), (uint32_t)((kt / STAGES) & 1), abort_flag, P.wait_ns))
        atomicExch(P.err, 5);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % STAGES, n = kt / STAGES;
      if (!mbar_wait(full0 + 8 * s, (uint32_t)(n & 1), abort_flag, P.wait_ns)) {
        *abort_flag = 1;
        atomicExch(P.err, 2);
        break;
      }
      tc_fence_after();
      const uint64_t ad = sw128_desc(smem_u32(sA + s * A_TILE));
      const uint64_t bd = sw128_desc(smem_u32(sB + s * B_TILE));
#pragma unroll
      for (int j = 0; j < TC_BK / 16; ++j)
        tc_mma(tmem, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), IDESC, (kt > 0 || j > 0) ? 1u : 0u);
      tc_commit(empty0 + 8 * s);
    }
    // every MMA issued has completed and every commit above has arrived before TMEM and shared
    // memory are released (the epilogue below may stop waiting early on an abort)
    tc_commit(done);
    mbar_drain(done, 0u);
  }
  __syncwarp();
  // ---------------- epilogue: TMEM -> registers -> global (rows = TMEM lanes)
  const bool ok = mbar_wait(done, 0u, abort_flag, P.wait_ns);
  tc_fence_after();
  if (!ok) atomicExch(P.err, 3);
  if (ok && !*abort_flag) {
    const int m = mt * TC_BM + warp * 32 + lane;
    // plain store (alpha = 1, beta = 0): no FP64 arithmetic in the epilogue
    const bool plain = P.alpha == 1.0 && P.beta == 0.0;
    for (int ch = 0; ch < BN / 32; ++ch) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), r);
      tmem_ld_wait();
      if (m < P.M) {
        // (rhs, cell) of the chunk's first column once, then stepped: no division per entry
        const long long c0 = (long long)nt * BN + ch * 32;
        int rhs = (int)(c0 / P.ncell);
        long long cell = c0 - (long long)rhs * P.ncell;
        for (int j = 0; j < 32; ++j, ++cell) {
          if (cell == P.ncell) { cell = 0; ++rhs; }
          if (c0 + j >= P.ncols) break;
          const long long off = bz * P.y_b_stride + rhs * P.y_rs + cell * P.y_cs + m;
          if (!FD_INB(off, P.y_ext, 103)) continue;
          const float a = __uint_as_float(r[j]);
          if (plain) {
            if (P.y_f64) reinterpret_cast<double*>(P.Y)[off] = (double)a;
            else reinterpret_cast<float*>(P.Y)[off] = a;
            continue;
          }
          const double v = P.alpha * (double)a;
          if (P.y_f64) {
            double* y = reinterpret_cast<double*>(P.Y) + off;
            *y = (P.beta == 0.0) ? v : v + P.beta * (*y);
          } else {
            float* y = reinterpret_cast<float*>(P.Y) + off;
            *y = (P.beta == 0.0) ? (float)v : (float)(v + P.beta * (double)(*y));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// ---- packing into SW128 K-major tiles
// A operand: nb batches x m_tiles x k_tiles tiles.  K index of batch b is a concatenation of
// nblk blocks of Kp (= k_tiles_op * 64) columns; block q uses operator op = q / nterm and split
// term t = q % nterm (t = 0 hi, t = 1 hi, t = 2 lo for three terms).  Element (row m, col kk) of
// operator op is src[op*op_stride + (r0 + m)*lda + c0 + kk] for m < M, kk < K.
__global__ void pack_A_kernel(const double* __restrict__ src, long long op_stride, int lda, int r0,
                              int c0, int M, int K, int nops_per_batch, int nterm, int k_tiles_op,
                              int m_tiles, int nb, uint8_t* __restrict__ out) {
  const int k_tiles = nops_per_batch * nterm * k_tiles_op;
  const long long total = (long long)nb * m_tiles * k_tiles * TC_BM * 8;   // 16-byte chunks
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int chunk = (int)(t & 7);
    long long rest = t >> 3;
    const int row = (int)(rest % TC_BM);
    rest /= TC_BM;
    const int kt = (int)(rest % k_tiles);
    rest /= k_tiles;
    const int mt = (int)(rest % m_tiles);
    const int b = (int)(rest / m_tiles);
    const int blk = kt / k_tiles_op, ktl = kt - blk * k_tiles_op;
    const int op = b * nops_per_batch + blk / nterm, term = blk % nterm;
    const int m = mt * TC_BM + row;
    alignas(16) __nv_bfloat16 v[8];
    for (int e = 0; e < 8; ++e) {
      const int kk = ktl * TC_BK + chunk * 8 + e;
      float x = 0.f;
      if (m < M && kk < K) {
        const double a = src[op * op_stride + (long long)(r0 + m) * lda + c0 + kk];
        const __nv_bfloat16 hi = __double2bfloat16(a);
        if (term == 2) x = (float)(a - (double)__bfloat162float(hi));
        else x = __bfloat162float(hi);
      }
      v[e] = __float2bfloat16_rn(x);
    }
    uint8_t* tile = out + (((long long)b * m_tiles + mt) * k_tiles + kt) * A_TILE;
    *reinterpret_cast<uint4*>(tile + sw128_offset(row, chunk * 8)) = *reinterpret_cast<uint4*>(v);
  }
}

// B operand: n_tiles x k_tiles tiles of BN rows (columns c = rhs*ncell + cell) x 64.  K block q
// = (op = q / nterm, term = q % nterm) holds coef[cell*ncoef + op] * X[c][kk] (coef may be null)
// as hi (terms 0, 2) or lo (term 1) bf16 part.
template <int BN>
__global__ void pack_B_kernel(const double* __restrict__ X, long long x_rs, int x_cs, int K,
                              const double* __restrict__ coef, int ncoef, int nops, int nterm,
                              int k_tiles_op, long long ncols, long long ncell, int n_tiles,
                              uint8_t* __restrict__ out, long long x_ext, long long out_bytes) {
  constexpr int B_TILE = BN * TC_BK * 2;
  const int k_tiles = nops * nterm * k_tiles_op;
  const long long total = (long long)n_tiles * k_tiles * BN * 8;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int chunk = (int)(t & 7);
    long long rest = t >> 3;
    const int row = (int)(rest % BN);
    rest /= BN;
    const int kt = (int)(rest % k_tiles);
    const int nt = (int)(rest / k_tiles);
    const int blk = kt / k_tiles_op, ktl = kt - blk * k_tiles_op;
    const int op = blk / nterm, term = blk % nterm;
    const long long cidx = (long long)nt * BN + row;
    alignas(16) __nv_bfloat16 v[8];
    if (cidx < ncols) {
      const int rhs = (int)(cidx / ncell);
      const long long cell = cidx - (long long)rhs * ncell;
      const double cf = coef ? coef[cell * ncoef + op] : 1.0;
      const double* xc = X + rhs * x_rs + cell * x_cs;
      for (int e = 0; e < 8; ++e) {
        const int kk = ktl * TC_BK + chunk * 8 + e;
        float x = 0.f;
        if (kk < K && FD_INB(rhs * x_rs + cell * x_cs + kk, x_ext, 104)) {
          const double a = cf * xc[kk];
          const __nv_bfloat16 hi = __double2bfloat16(a);
          if (term == 1) x = (float)(a - (double)__bfloat162float(hi));
          else x = __bfloat162float(hi);
        }
        v[e] = __float2bfloat16_rn(x);
      }
    } else {
      for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16_rn(0.f);
    }
    uint8_t* tile = out + ((long long)nt * k_tiles + kt) * B_TILE;
    if (!FD_INB(((long long)nt * k_tiles + kt) * B_TILE + sw128_offset(row, chunk * 8) + 15, out_bytes, 105))
      continue;
    *reinterpret_cast<uint4*>(tile + sw128_offset(row, chunk * 8)) = *reinterpret_cast<uint4*>(v);
  }
}

// Reference for the self-check: Y[c][m] = sum_kk A[m][kk] X[c][kk] in FP64 on bf16-rounded inputs.
__global__ void ref_gemm_kernel(const double* A, const double* X, int M, int K, int N, double* Y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)M * N;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / M), m = (int)(t % M);
    double s = 0.0;
    for (int kk = 0; kk < K; ++kk)
      s += (double)__bfloat162float(__double2bfloat16(A[(long long)m * K + kk])) *
           (double)__bfloat162float(__double2bfloat16(X[(long long)c * K + kk]));
    Y[t] = s;
  }
}

__global__ void fill_random_kernel(double* x, long long n, unsigned long long seed) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(t + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[t] = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
}

inline int gridn(long long work) {
  long long g = (work + 255) / 256;
  if (g > 152LL * 32) g = 152LL * 32;
  return (int)(g < 1 ? 1 : g);
}

template <int BN, int STAGES>
constexpr size_t tc_smem_bytes() {
  return (size_t)STAGES * (A_TILE + BN * TC_BK * 2) + 8 * (2 * STAGES + 1) + 16 + 1024;
}

template <int BN, int STAGES>
fetidp_status launch_tc(Ctx& c, const TcParams& P, int batch) {
  const size_t smem = tc_smem_bytes<BN, STAGES>();
  cudaFuncSetAttribute(tc_gemm_kernel<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long long nblk = (long long)P.n_tiles * P.m_tiles * batch;
  if (nblk >= (1LL << 31) || P.batch != batch || P.bgroup < 1) {
    set_error("tensor-core GEMM: grid too large");
    return FETIDP_EINVAL;
  }
  tc_gemm_kernel<BN, STAGES><<<(unsigned)nblk, 128, smem, c.stream>>>(P);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

}  // namespace

// ---------------------------------------------------------------- fused combine kernel
// Y[:, c] = sum_k coef_k(c, row) (A_k X)[:, c] without materialising scaled copies of X:
// X is packed once (hi [+ lo] BF16 parts) and stays resident in shared memory; the operators
// A_k stream through a TMA ring; the MMAs of operator k accumulate in TMEM buffer k & 1; four
// epilogue warps add coef * accumulator into FP32 registers while the MMA warp fills the other
// buffer.  Rows below msplit use coef0, the others coef1 (stacked operator sets).
// Warps 0-3 epilogue (TMEM lane quadrants), warp 4 producer, warp 5 MMA issuer.
constexpr int kCombStages = 12;                   // deepest operator-tile ring
constexpr int kCombBars = 2 * kCombStages + 8;    // barrier slots (8 bytes) before the coefficients
struct TcCombParams {
  const uint8_t* A;
  const uint8_t* B;
  int m_tiles, n_tiles, kto, nops, nA, nX, astages, tps;   // tps: operator tiles per ring stage
  int M, msplit;
  long long ncols, ncell;
  const double* coef0;
  const double* coef1;
  void* Y;
  int y_f64;
  long long y_rs;
  int y_cs;
  double alpha, beta;
  int* err;
  unsigned long long wait_ns;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(192, 1) tc_comb_kernel(TcCombParams P) {
  constexpr int B_TILE = BN * TC_BK * 2;
  constexpr uint32_t TMEM_COLS = 2 * BN < 32 ? 32 : 2 * BN;
  constexpr uint32_t IDESC = make_idesc(TC_BM, BN, true);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int KX = P.kto * P.nX;
  const int S = P.astages;
  uint8_t* sB = smem;
  uint8_t* sA = sB + (size_t)KX * B_TILE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + (size_t)S * P.tps * A_TILE);
  // bars: aFull[kCombStages], aEmpty[kCombStages], bFull, accFull[2], accEmpty[2], (TMEM slot and
  // abort flag), done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kCombStages + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* sCoef = reinterpret_cast<float*>(bars + kCombBars);   // [set][op][column], FP32
  const uint32_t aFull = smem_u32(bars), aEmpty = smem_u32(bars + kCombStages);
  const uint32_t bFull = smem_u32(bars + 2 * kCombStages);
  const uint32_t accFull = smem_u32(bars + 2 * kCombStages + 1), accEmpty = smem_u32(bars + 2 * kCombStages + 3);
  const uint32_t done = smem_u32(bars + 2 * kCombStages + 6);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = blockIdx.x, mt = blockIdx.y;
  // the tile's combination coefficients, once: 1 without coefficients, 0 past the last column
  const int csets = P.msplit < P.M ? 2 : 1;
  for (int t = threadIdx.x; t < csets * P.nops * BN; t += blockDim.x) {
    const int set = t / (P.nops * BN);
    const int rem = t - set * P.nops * BN;
    const int j = rem / P.nops, k = rem - j * P.nops;   // op fastest: coalesced coefficient reads
    const long long cidx = (long long)nt * BN + j;
    const double* cp = set ? P.coef1 : P.coef0;
    float v = 0.f;
    if (cidx < P.ncols) v = cp ? (float)cp[(cidx % P.ncell) * P.nops + k] : 1.f;
    sCoef[(set * P.nops + k) * BN + j] = v;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kCombStages; ++s) {
      mbar_init(aFull + 8 * s, 1);
      mbar_init(aEmpty + 8 * s, 1);
    }
    mbar_init(bFull, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(accFull + 8 * b, 1);
      mbar_init(accEmpty + 8 * b, 128);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int per_op = P.kto * P.nA;
  const int tps = P.tps, cpo = (per_op + tps - 1) / tps, nchunk = P.nops * cpo;
  const size_t stage_bytes = (size_t)tps * A_TILE;
  // Every column tile streams all operators.  Tile nt starts at operator nt mod nops, so at any
  // moment the CTAs read different operator tiles, spread over all L2 slices, instead of all
  // hitting the few slices that hold one tile.
  const int rot = nt % P.nops;
  if (warp == 4) {
    if (lane == 0) {
      // resident X tiles (one copy), then the operator ring.  A stage holds tps consecutive
      // tiles of one operator and arrives with one bulk copy: the copy rate per SM grows with
      // the bytes per copy, not with the number of copies in flight.
      const uint8_t* Bb = P.B + (long long)nt * KX * B_TILE;
      mbar_expect_tx(bFull, (uint32_t)(KX * B_TILE));
      bulk_g2s(smem_u32(sB), Bb, (uint32_t)(KX * B_TILE), bFull);
      int issued = 0;
      for (int c = 0; c < nchunk; ++c) {
        const int s = c % S, n = c / S;
        if (c >= S && !mbar_wait(aEmpty + 8 * s, (uint32_t)((n - 1) & 1), abort_flag, P.wait_ns)) {
          *abort_flag = 1;
          atomicExch(P.err, 11);
          break;
        }
        const int kk = c / cpo, r0 = (c - kk * cpo) * tps;   // tiles [r0, r0 + ntl) of the op
        const int ntl = min(tps, per_op - r0);
        const int k = (kk + rot) % P.nops;                    // operator of this step
        const uint8_t* src = P.A + (((long long)k * P.m_tiles + mt) * per_op + r0) * A_TILE;
        mbar_expect_tx(aFull + 8 * s, (uint32_t)(ntl * A_TILE));
        bulk_g2s(smem_u32(sA + (size_t)s * stage_bytes), src, (uint32_t)(ntl * A_TILE), aFull + 8 * s);
        ++issued;
      }
      // exit drain: every copy issued has landed (the MMA thread drains its own commits; without
      // an abort the last stages' releases are also awaited here)
      for (int c = (issued > S ? issued - S : 0); c < issued; ++c)
        mbar_drain(aFull + 8 * (c % S), (uint32_t)((c / S) & 1));
      mbar_drain(bFull, 0u);
      for (int c = (issued > S ? issued - S : 0); c < issued && !*abort_flag; ++c)
        if (!mbar_wait(aEmpty + 8 * (c % S), (uint32_t)((c / S) & 1), abort_flag, P.wait_ns))
          atomicExch(P.err, 16);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      bool ok = mbar_wait(bFull, 0u, abort_flag, P.wait_ns);
      if (!ok) { *abort_flag = 1; atomicExch(P.err, 12); }
      int c = 0;
      for (int k = 0; ok && k < P.nops; ++k) {
        const int b = k & 1;
        if (k >= 2 && !mbar_wait(accEmpty + 8 * b, (uint32_t)(((k >> 1) - 1) & 1), abort_flag, P.wait_ns)) {
          *abort_flag = 1;
          atomicExch(P.err, 13);
          ok = false;
          break;
        }
        tc_fence_after();
        bool first = true;
        const uint32_t dst = tmem + (uint32_t)(b * BN);
        for (int cc = 0; ok && cc < cpo; ++cc, ++c) {
          const int s = c % S, n = c / S;
          if (!mbar_wait(aFull + 8 * s, (uint32_t)(n & 1), abort_flag, P.wait_ns)) {
            *abort_flag = 1;
            atomicExch(P.err, 14);
            ok = false;
            break;
          }
          tc_fence_after();
          const int r0 = cc * tps, ntl = min(tps, per_op - r0);
          for (int t = 0; t < ntl; ++t) {
            const int rem = r0 + t, kt = rem / P.nA, part = rem - kt * P.nA;
            const uint64_t ad = sw128_desc(smem_u32(sA + (size_t)s * stage_bytes + (size_t)t * A_TILE));
            // A hi pairs with X hi (and X lo when split); A lo pairs with X hi
            const int nxp = (part == 0) ? P.nX : 1;
            for (int xp = 0; xp < nxp; ++xp) {
              const uint64_t bd = sw128_desc(smem_u32(sB + (size_t)(kt * P.nX + xp) * B_TILE));
#pragma unroll
              for (int j = 0; j < TC_BK / 16; ++j) {
                tc_mma(dst, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), IDESC, first ? 0u : 1u);
                first = false;
              }
            }
          }
          tc_commit(aEmpty + 8 * s);
        }
        if (ok) tc_commit(accFull + 8 * b);
      }
      // every MMA issued has completed and every commit above has arrived before TMEM and
      // shared memory are released
      tc_commit(done);
      mbar_drain(done, 0u);
    }
  } else {
    // ---------------- epilogue warps 0-3: one row per thread
    const int m = mt * TC_BM + warp * 32 + lane;
    const float* cset = (m < P.msplit || csets == 1) ? sCoef : sCoef + P.nops * BN;
    float acc[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) acc[j] = 0.f;
    bool ok = true;
    for (int kk = 0; kk < P.nops; ++kk) {
      const int b = kk & 1;
      const int k = (kk + rot) % P.nops;
      if (!mbar_wait(accFull + 8 * b, (uint32_t)((kk >> 1) & 1), abort_flag, P.wait_ns)) {
        *abort_flag = 1;
        atomicExch(P.err, 15);
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int ch = 0; ch < BN / 32; ++ch) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * BN + ch * 32), r);
        tmem_ld_wait();
        const float* ck = cset + k * BN + ch * 32;
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 c4 = *reinterpret_cast<const float4*>(ck + j);   // broadcast
          acc[ch * 32 + j] += c4.x * __uint_as_float(r[j]);
          acc[ch * 32 + j + 1] += c4.y * __uint_as_float(r[j + 1]);
          acc[ch * 32 + j + 2] += c4.z * __uint_as_float(r[j + 2]);
          acc[ch * 32 + j + 3] += c4.w * __uint_as_float(r[j + 3]);
        }
      }
      tc_fence_before();
      mbar_arrive(accEmpty + 8 * b);
    }
    if (ok && !*abort_flag && m < P.M) {
      // (rhs, cell) of the tile's first column once, then stepped: no division per entry
      const long long c0 = (long long)nt * BN;
      int rhs = (int)(c0 / P.ncell);
      long long cell = c0 - (long long)rhs * P.ncell;
#pragma unroll
      for (int j = 0; j < BN; ++j, ++cell) {
        if (cell == P.ncell) { cell = 0; ++rhs; }
        const long long cidx = c0 + j;
        if (cidx < P.ncols) {
          const long long off = rhs * P.y_rs + cell * P.y_cs + m;
          const double v = P.alpha * (double)acc[j];
          if (P.y_f64) {
            double* y = reinterpret_cast<double*>(P.Y) + off;
            *y = (P.beta == 0.0) ? v : v + P.beta * (*y);
          } else {
            float* y = reinterpret_cast<float*>(P.Y) + off;
            *y = (P.beta == 0.0) ? (float)v : (float)(v + P.beta * (double)(*y));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// Operator tiles for the combine kernel: tile ((op * m_tiles + mt) * kto + kt) * nA + part, part 0
// the bf16 value, part 1 the bf16 rounding remainder.  Rows [0, M0) come from src0, rows
// [M0, M0 + M1) from src1 (same K): element (m, kk) of op = srcX[op*strideX + (r0X + m)*ldaX + c0X + kk].
__global__ void pack_comb_A_kernel(const double* __restrict__ src0, long long st0, int lda0, int r00,
                                   int c00, int M0, const double* __restrict__ src1, long long st1,
                                   int lda1, int r01, int c01, int M1, int K, int nops, int nA, int kto,
                                   int m_tiles, uint8_t* __restrict__ out) {
  const long long total = (long long)nops * m_tiles * kto * nA * TC_BM * 8;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int chunk = (int)(t & 7);
    long long rest = t >> 3;
    const int row = (int)(rest % TC_BM);
    rest /= TC_BM;
    const int part = (int)(rest % nA);
    rest /= nA;
    const int kt = (int)(rest % kto);
    rest /= kto;
    const int mt = (int)(rest % m_tiles);
    const int op = (int)(rest / m_tiles);
    const int m = mt * TC_BM + row;
    alignas(16) __nv_bfloat16 v[8];
    for (int e = 0; e < 8; ++e) {
      const int kk = kt * TC_BK + chunk * 8 + e;
      float x = 0.f;
      if (kk < K && m < M0 + M1) {
        const double a = (m < M0) ? src0[op * st0 + (long long)(r00 + m) * lda0 + c00 + kk]
                                  : src1[op * st1 + (long long)(r01 + m - M0) * lda1 + c01 + kk];
        const __nv_bfloat16 hi = __double2bfloat16(a);
        x = (part == 1) ? (float)(a - (double)__bfloat162float(hi)) : __bfloat162float(hi);
      }
      v[e] = __float2bfloat16_rn(x);
    }
    uint8_t* tile = out + ((((long long)op * m_tiles + mt) * kto + kt) * nA + part) * A_TILE;
    *reinterpret_cast<uint4*>(tile + sw128_offset(row, chunk * 8)) = *reinterpret_cast<uint4*>(v);
  }
}

// X tiles for the combine kernel: tile (nt * kto + kt) * nX + part of BN columns.
template <int BN>
__global__ void pack_comb_X_kernel(const double* __restrict__ X, long long x_rs, int x_cs, int K, int nX,
                                   int kto, long long ncols, long long ncell, int n_tiles,
                                   uint8_t* __restrict__ out) {
  constexpr int B_TILE = BN * TC_BK * 2;
  const long long total = (long long)n_tiles * kto * nX * BN * 8;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int chunk = (int)(t & 7);
    long long rest = t >> 3;
    const int row = (int)(rest % BN);
    rest /= BN;
    const int part = (int)(rest % nX);
    rest /= nX;
    const int kt = (int)(rest % kto);
    const int nt = (int)(rest / kto);
    const long long cidx = (long long)nt * BN + row;
    alignas(16) __nv_bfloat16 v[8];
    if (cidx < ncols) {
      const int rhs = (int)(cidx / ncell);
      const long long cell = cidx - (long long)rhs * ncell;
      const double* xc = X + rhs * x_rs + cell * x_cs;
      for (int e = 0; e < 8; ++e) {
        const int kk = kt * TC_BK + chunk * 8 + e;
        float x = 0.f;
        if (kk < K) {
          const double a = xc[kk];
          const __nv_bfloat16 hi = __double2bfloat16(a);
          x = (part == 1) ? (float)(a - (double)__bfloat162float(hi)) : __bfloat162float(hi);
        }
        v[e] = __float2bfloat16_rn(x);
      }
    } else {
      for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16_rn(0.f);
    }
    uint8_t* tile = out + (((long long)nt * kto + kt) * nX + part) * B_TILE;
    *reinterpret_cast<uint4*>(tile + sw128_offset(row, chunk * 8)) = *reinterpret_cast<uint4*>(v);
  }
}

template <int BN>
size_t comb_smem_bytes(int kto, int nX, int astages, int tps, size_t coef_bytes) {
  return (size_t)kto * nX * BN * TC_BK * 2 + (size_t)astages * tps * A_TILE + 8 * kCombBars + coef_bytes + 1024;
}

// ---------------------------------------------------------------- host API
int tc_bn_for(long long ncols, int m_tiles, int batch) {
  // smallest tile width that still gives at least one wave of CTAs on 148 SMs
  const long long ctas256 = ((ncols + 255) / 256) * m_tiles * batch;
  if (ctas256 >= 148) return 256;
  const long long ctas128 = ((ncols + 127) / 128) * m_tiles * batch;
  if (ctas128 >= 148) return 128;
  return 64;
}

fetidp_status tc_pack_operator(Ctx& c, TcOperator& op, const double* src, long long op_stride, int lda,
                               int r0, int c0, int M, int K, int nops, bool separate, int nterm) {
  op.M = M;
  op.K = K;
  op.nops = nops;
  op.nterm = nterm;
  op.separate = separate;
  op.m_tiles = (M + TC_BM - 1) / TC_BM;
  op.k_tiles_op = (K + TC_BK - 1) / TC_BK;
  const int nb = separate ? nops : 1;
  const int per_batch = separate ? 1 : nops;
  op.k_tiles = per_batch * nterm * op.k_tiles_op;
  op.batch_bytes = (long long)op.m_tiles * op.k_tiles * A_TILE;
  FD_TRY(dalloc(c, reinterpret_cast<void**>(&op.tiles), (size_t)nb * op.batch_bytes));
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, (double)nb * op.batch_bytes);
  const long long work = (long long)nb * op.m_tiles * op.k_tiles * TC_BM * 8;
  pack_A_kernel<<<gridn(work), 256, 0, c.stream>>>(src, op_stride, lda, r0, c0, M, K, per_batch, nterm,
                                                  op.k_tiles_op, op.m_tiles, nb, op.tiles);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

void tc_free_operator(Ctx& c, TcOperator& op) {
  if (!op.tiles) return;
  cudaStreamSynchronize(c.stream);
  for (auto it = c.allocations.begin(); it != c.allocations.end(); ++it)
    if (*it == op.tiles) {
      c.allocations.erase(it);
      break;
    }
  c.device_bytes -= (size_t)(op.separate ? op.nops : 1) * op.batch_bytes;
  cudaFreeAsync(op.tiles, c.stream);
  op.tiles = nullptr;
}

// Y = alpha * op(X) (+ beta Y).  X: FP64 columns (rhs, cell), K values each.  coef: [ncell][nops]
// scaling of the K blocks (combine mode), or null.  Y: FP64 or FP32; separate mode writes batch k
// at Y + k * y_b_stride.
fetidp_status tc_apply(Ctx& c, const TcOperator& op, CCellVec X, const double* coef, void* Y,
                       bool y_f64, long long y_rs, int y_cs, long long y_b_stride, double alpha,
                       double beta, int nrhs, long long ncell, long long y_ext) {
  const long long ncols = ncell * nrhs;
  const int batch = op.separate ? op.nops : 1;
  const int BN = c.opt.tc_bn > 0 ? c.opt.tc_bn : tc_bn_for(ncols, op.m_tiles, batch);
  const int n_tiles = (int)((ncols + BN - 1) / BN);
  const int nops_b = op.separate ? 1 : op.nops;
  const int k_tiles = nops_b * op.nterm * op.k_tiles_op;
  const size_t b_bytes = (size_t)n_tiles * k_tiles * BN * TC_BK * 2;
  if (b_bytes > c.tc_bbuf_bytes) {
    set_error("tensor-core B staging buffer too small");
    return FETIDP_EINVAL;
  }
  {
    ProfScope ps(c, FETIDP_K_MAPS, 0.0, (double)ncols * op.K * 8.0 + (double)b_bytes);
    const long long work = (long long)n_tiles * k_tiles * BN * 8;
    if (BN == 256)
      pack_B_kernel<256><<<gridn(work), 256, 0, c.stream>>>(X.p, X.rs, X.cs, op.K, coef, op.nops, nops_b,
                                                           op.nterm, op.k_tiles_op, ncols, ncell, n_tiles,
                                                           c.tc_bbuf, X.ext, (long long)c.tc_bbuf_bytes);
    else if (BN == 128)
      pack_B_kernel<128><<<gridn(work), 256, 0, c.stream>>>(X.p, X.rs, X.cs, op.K, coef, op.nops, nops_b,
                                                           op.nterm, op.k_tiles_op, ncols, ncell, n_tiles,
                                                           c.tc_bbuf, X.ext, (long long)c.tc_bbuf_bytes);
    else
      pack_B_kernel<64><<<gridn(work), 256, 0, c.stream>>>(X.p, X.rs, X.cs, op.K, coef, op.nops, nops_b,
                                                          op.nterm, op.k_tiles_op, ncols, ncell, n_tiles,
                                                          c.tc_bbuf, X.ext, (long long)c.tc_bbuf_bytes);
    FD_CHECK_LAUNCH();
  }
  TcParams P;
  P.A = op.tiles;
  P.B = c.tc_bbuf;
  P.m_tiles = op.m_tiles;
  P.n_tiles = n_tiles;
  P.k_tiles = k_tiles;
  P.a_batch_stride = op.separate ? op.batch_bytes : 0;
  P.b_batch_stride = 0;
  P.M = op.M;
  P.ncols = ncols;
  P.ncell = ncell;
  P.Y = Y;
  P.y_f64 = y_f64 ? 1 : 0;
  P.y_rs = y_rs;
  P.y_cs = y_cs;
  P.y_b_stride = y_b_stride;
  P.alpha = alpha;
  P.beta = beta;
  P.err = c.tc_err;
  P.wait_ns = c.wait_ns;
  P.a_bytes = (long long)batch * op.batch_bytes;
  P.b_bytes = (long long)c.tc_bbuf_bytes;
  P.y_ext = y_ext;
  P.batch = batch;
  // operators per group: their A tiles (batch_bytes each) within about 48 MB of the 129 MB L2
  P.bgroup = (int)std::max<long long>(1, std::min<long long>(batch, (48LL << 20) / std::max<long long>(1, op.batch_bytes)));
  // algorithmic flops: one M x K product per operator and column (no padding, no split products)
  const double flops = 2.0 * op.M * (double)op.K * op.nops * (double)ncols;
  ProfScope ps(c, FETIDP_K_TC_GEMM, flops,
               (double)batch * op.batch_bytes + (double)b_bytes + (double)ncols * op.M * (y_f64 ? 8 : 4) * batch);
  if (BN == 256) return launch_tc<256, 4>(c, P, batch);
  if (BN == 128) return launch_tc<128, 6>(c, P, batch);
  return launch_tc<64, 8>(c, P, batch);
}

// Self-check of the tensor-core path: random A (M x K), X (N columns), compare with an FP64
// GEMM of the same bf16-rounded inputs.  Returns the max relative error in *rel_err.
fetidp_status tc_selfcheck(Ctx& c, int M, int K, int N, double* rel_err) {
  // the four buffers are freed on every return path
  struct Bufs {
    double *A = nullptr, *X = nullptr, *Yt = nullptr, *Yr = nullptr;
    ~Bufs() { cudaFree(A); cudaFree(X); cudaFree(Yt); cudaFree(Yr); }
  } b;
  FD_CUDA(cudaMalloc(&b.A, sizeof(double) * M * K));
  FD_CUDA(cudaMalloc(&b.X, sizeof(double) * (size_t)N * K));
  FD_CUDA(cudaMalloc(&b.Yt, sizeof(double) * (size_t)N * M));
  FD_CUDA(cudaMalloc(&b.Yr, sizeof(double) * (size_t)N * M));
  double *A = b.A, *X = b.X, *Yt = b.Yt, *Yr = b.Yr;
  fill_random_kernel<<<gridn((long long)M * K), 256, 0, c.stream>>>(A, (long long)M * K, 1234);
  fill_random_kernel<<<gridn((long long)N * K), 256, 0, c.stream>>>(X, (long long)N * K, 5678);
  FD_CHECK_LAUNCH();
  TcOperator op;
  FD_TRY(tc_pack_operator(c, op, A, 0, K, 0, 0, M, K, 1, false, 1));
  FD_TRY(tc_apply(c, op, CCellVec{X, 0, K}, nullptr, Yt, true, 0, M, 0, 1.0, 0.0, 1, N));
  ref_gemm_kernel<<<gridn((long long)M * N), 256, 0, c.stream>>>(A, X, M, K, N, Yr);
  FD_CHECK_LAUNCH();
  std::vector<double> ht((size_t)N * M), hr((size_t)N * M);
  FD_CUDA(cudaMemcpyAsync(ht.data(), Yt, sizeof(double) * ht.size(), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaMemcpyAsync(hr.data(), Yr, sizeof(double) * hr.size(), cudaMemcpyDeviceToHost, c.stream));
  int herr = 0;
  FD_CUDA(cudaMemcpyAsync(&herr, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  if (herr != 0) {
    set_error("tensor-core GEMM wait timed out (code " + std::to_string(herr) + ")");
    return FETIDP_ETIMEOUT;
  }
  // a non-finite difference counts as an infinite error (the rule of absmax_pair_kernel)
  double mx = 0.0, ref = 0.0;
  for (size_t i = 0; i < ht.size(); ++i) {
    const double dv = std::fabs(ht[i] - hr[i]);
    mx = std::isfinite(dv) ? std::max(mx, dv) : INFINITY;
    ref = std::max(ref, std::fabs(hr[i]));
  }
  *rel_err = mx / (ref > 0 ? ref : 1.0);
  return FETIDP_OK;
}


// ---------------------------------------------------------------- combine kernel host side
// shared bytes of the staged combination coefficients (one or two FP32 sets of nops x bn)
static size_t comb_coef_bytes(int bn, int nops, bool two_sets) {
  return (size_t)(two_sets ? 2 : 1) * nops * bn * sizeof(float);
}

// Operator ring of the combine kernel: tiles per stage (as many of one operator's per_op tiles
// as allow two stages) and the number of stages; stages = 0 when two stages of one tile do not fit.
static void comb_ring(int bn, int kto, int nX, int per_op, size_t coef_bytes, int* stages, int* tps) {
  const size_t budget = 220 * 1024;
  const size_t b = (size_t)kto * nX * bn * TC_BK * 2 + 8 * kCombBars + coef_bytes + 1024;
  *stages = 0;
  *tps = 1;
  if (b + 2 * (size_t)A_TILE > budget) return;
  const size_t avail = budget - b;
  int t = (int)std::min<size_t>((size_t)per_op, avail / (2 * (size_t)A_TILE));
  if (t < 1) t = 1;
  int st = (int)(avail / ((size_t)t * A_TILE));
  if (st > kCombStages) st = kCombStages;
  *tps = t;
  *stages = st;
}

// Column-tile width of the combine kernel: the widest of 128 / 64 / 32 that still gives a full
// wave of CTAs, narrowed while the resident x tiles leave no room for two ring stages (long K).
int tc_comb_bn(long long ncols, int m_tiles, int kto, int nX, int nops, bool two_sets) {
  int bn = 32;
  if (((ncols + 127) / 128) * m_tiles >= 148) bn = 128;
  else if (((ncols + 63) / 64) * m_tiles >= 148) bn = 64;
  for (; bn > 32; bn /= 2) {
    int st = 0, tps = 1;
    comb_ring(bn, kto, nX, kto * nX, comb_coef_bytes(bn, nops, two_sets), &st, &tps);
    if (st >= 2) break;
  }
  return bn;
}

bool tc_comb_fits(int K, int split, long long ncols, int m_tiles, int nops, bool two_sets) {
  const int kto = (K + TC_BK - 1) / TC_BK;
  const int nA = split == 3 ? 2 : 1;
  const int bn = tc_comb_bn(ncols, m_tiles, kto, nA, nops, two_sets);
  int st = 0, tps = 1;
  comb_ring(bn, kto, nA, kto * nA, comb_coef_bytes(bn, nops, two_sets), &st, &tps);
  return st >= 2;
}

fetidp_status tc_comb_pack(Ctx& c, TcComb& op, const double* src0, long long st0, int lda0, int r00, int c00,
                           int M0, const double* src1, long long st1, int lda1, int r01, int c01, int M1,
                           int K, int nops, int split) {
  op.M = M0 + M1;
  op.msplit = M0;
  op.K = K;
  op.nops = nops;
  op.nA = split == 3 ? 2 : 1;
  op.nX = split == 3 ? 2 : 1;
  op.m_tiles = (op.M + TC_BM - 1) / TC_BM;
  op.kto = (K + TC_BK - 1) / TC_BK;
  op.bytes = (long long)nops * op.m_tiles * op.kto * op.nA * A_TILE;
  FD_TRY(dalloc(c, reinterpret_cast<void**>(&op.tiles), (size_t)op.bytes));
  ProfScope ps(c, FETIDP_K_SETUP, 0.0, (double)op.bytes);
  const long long work = (long long)nops * op.m_tiles * op.kto * op.nA * TC_BM * 8;
  pack_comb_A_kernel<<<gridn(work), 256, 0, c.stream>>>(src0, st0, lda0, r00, c00, M0, src1, st1, lda1, r01, c01,
                                                       M1, K, nops, op.nA, op.kto, op.m_tiles, op.tiles);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

size_t tc_comb_staging_bytes(const TcComb& op, long long ncols) {
  const int bn = tc_comb_bn(ncols, op.m_tiles, op.kto, op.nX, op.nops, op.msplit < op.M);
  const long long n_tiles = (ncols + bn - 1) / bn;
  return (size_t)n_tiles * op.kto * op.nX * bn * TC_BK * 2;
}

template <int BN>
static fetidp_status comb_launch(Ctx& c, const TcComb& op, const TcCombParams& P0, CCellVec X, long long ncols,
                                 long long ncell) {
  TcCombParams P = P0;
  const int n_tiles = (int)((ncols + BN - 1) / BN);
  P.n_tiles = n_tiles;
  const size_t b_bytes = (size_t)n_tiles * op.kto * op.nX * BN * TC_BK * 2;
  if (b_bytes > c.tc_bbuf_bytes) {
    set_error("tensor-core X staging buffer too small");
    return FETIDP_EINVAL;
  }
  const size_t coef_bytes = comb_coef_bytes(BN, op.nops, op.msplit < op.M);
  comb_ring(BN, op.kto, op.nX, op.kto * op.nA, coef_bytes, &P.astages, &P.tps);
  if (P.astages < 2) {
    set_error("combine kernel: operand K too large for shared memory");
    return FETIDP_EINVAL;
  }
  {
    ProfScope ps(c, FETIDP_K_MAPS, 0.0, (double)ncols * op.K * 8.0 + (double)b_bytes);
    const long long work = (long long)n_tiles * op.kto * op.nX * BN * 8;
    pack_comb_X_kernel<BN><<<gridn(work), 256, 0, c.stream>>>(X.p, X.rs, X.cs, op.K, op.nX, op.kto, ncols,
                                                              ncell, n_tiles, c.tc_bbuf);
    FD_CHECK_LAUNCH();
  }
  // algorithmic flops: one M x K product per principal operator and column (no tile padding,
  // no hi / lo split products)
  const double flops = 2.0 * op.M * (double)op.K * op.nops * (double)ncols;
  ProfScope ps(c, FETIDP_K_TC_GEMM, flops,
               (double)op.bytes + (double)b_bytes + (double)ncols * op.M * (P.y_f64 ? 8 : 4));
  const size_t smem = comb_smem_bytes<BN>(op.kto, op.nX, P.astages, P.tps, coef_bytes);
  cudaFuncSetAttribute(tc_comb_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)n_tiles, (unsigned)op.m_tiles, 1);
  tc_comb_kernel<BN><<<grid, 192, smem, c.stream>>>(P);
  FD_CHECK_LAUNCH();
  return FETIDP_OK;
}

static fetidp_status comb2_apply(Ctx& c, const TcComb& op, CCellVec X, const double* coef, void* Y, bool y_f64,
                                 long long y_rs, int y_cs, double alpha, double beta, long long ncols,
                                 long long ncell);

fetidp_status tc_comb_apply(Ctx& c, const TcComb& op, CCellVec X, const double* coef0, const double* coef1,
                            void* Y, bool y_f64, long long y_rs, int y_cs, double alpha, double beta, int nrhs,
                            long long ncell) {
  const long long ncols = ncell * nrhs;
  if (tc_comb2_ok(op) && c.tc_xf && c.tc_yp)
    return comb2_apply(c, op, X, coef0, Y, y_f64, y_rs, y_cs, alpha, beta, ncols, ncell);
  TcCombParams P{};
  P.A = op.tiles;
  P.B = c.tc_bbuf;
  P.m_tiles = op.m_tiles;
  P.kto = op.kto;
  P.nops = op.nops;
  P.nA = op.nA;
  P.nX = op.nX;
  P.M = op.M;
  P.msplit = op.msplit;
  P.ncols = ncols;
  P.ncell = ncell;
  P.coef0 = coef0;
  P.coef1 = coef1;
  P.Y = Y;
  P.y_f64 = y_f64 ? 1 : 0;
  P.y_rs = y_rs;
  P.y_cs = y_cs;
  P.alpha = alpha;
  P.beta = beta;
  P.err = c.tc_err;
  P.wait_ns = c.wait_ns;
  const int bn = tc_comb_bn(ncols, op.m_tiles, op.kto, op.nX, op.nops, op.msplit < op.M);
  if (bn == 128) return comb_launch<128>(c, op, P, X, ncols, ncell);
  if (bn == 64) return comb_launch<64>(c, op, P, X, ncols, ncell);
  return comb_launch<32>(c, op, P, X, ncols, ncell);
}

// ---------------------------------------------------------------- resident-operator combination
// y_c = sum_k coef_k(c) A_k x_c for operators of one row tile (M <= 128, K <= 128): the Eq. 48 / 49
// combinations F_dd, S_dd of every inner PCG iteration.  Streaming all N_rb operators through
// every column tile (tc_comb_kernel) makes each CTA read the whole operator set; here a CTA keeps
// the operators of kG2 principals resident in shared memory and runs over a range of 64-column
// tiles instead.  Four warps form the scaled operand z = coef_k(c) x_c (FP32 product, split into
// BF16 hi + lo) in the SW128 layout, one thread issues the MMAs of all the CTA's principals into
// one TMEM accumulator per tile, and four warps move each accumulator to an FP32 partial sum of
// the principal group.  comb2_reduce_kernel adds the groups in a fixed order (deterministic).
constexpr int kG2 = 2;                       // principals per CTA
constexpr int kBN2 = 64;                     // columns per tile (MMA N)
constexpr int Z_TILE2 = kBN2 * TC_BK * 2;    // 8 KB
constexpr int kComb2Threads = 288;           // epilogue warps 0-3, operand warps 4-7, MMA warp 8
struct TcComb2Params {
  const uint8_t* A;       // operator tiles (tc_comb_pack layout, one row tile)
  const float* xf;        // [ncols][KP] x in FP32, zero past K
  const double* coef;     // [ncell][nops]
  float* yp;              // [ngroups][ncols][M] partial sums
  int nops, kto, nA, nZ, M, KP, n_tiles, tiles_per_cta;
  long long ncols, ncell;
  int* err;
  unsigned long long wait_ns;
};

__global__ void __launch_bounds__(kComb2Threads, 1) tc_comb2_kernel(TcComb2Params P) {
  constexpr uint32_t IDESC = make_idesc(TC_BM, kBN2, true);
  constexpr uint32_t TMEM_COLS = 2 * kBN2;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int g = blockIdx.y;
  const int k0 = g * kG2, ng = min(kG2, P.nops - k0);
  const int t_begin = blockIdx.x * P.tiles_per_cta;
  const int t_end = min(P.n_tiles, t_begin + P.tiles_per_cta);
  if (t_begin >= t_end || ng <= 0) return;          // uniform: before any barrier or TMEM use
  const int ntile = t_end - t_begin;
  const int per_op = P.kto * P.nA;
  const size_t zslot = (size_t)P.kto * P.nZ * Z_TILE2;
  const int xld = P.KP + 4;                         // staged x row stride (floats): 16-byte rows, 4-bank offset
  uint8_t* sA = smem;                               // [kG2][kto][nA] operator tiles
  uint8_t* sZ = sA + (size_t)kG2 * per_op * A_TILE; // [2 slots][kto][nZ] operand tiles
  float* sX = reinterpret_cast<float*>(sZ + 2 * zslot);   // [kBN2][xld] x of the next tile
  uint64_t* bars = reinterpret_cast<uint64_t*>(sX + (size_t)kBN2 * xld);
  // opFull, zFull[2], zEmpty[2], accFull[2], accEmpty[2], done, xsync (operand warps)
  const uint32_t opFull = smem_u32(bars), zFull = smem_u32(bars + 1), zEmpty = smem_u32(bars + 3);
  const uint32_t accFull = smem_u32(bars + 5), accEmpty = smem_u32(bars + 7), done = smem_u32(bars + 9);
  const uint32_t xsync = smem_u32(bars + 10);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 11);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(opFull, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(zFull + 8 * s, 128);
      mbar_init(zEmpty + 8 * s, 1);
      mbar_init(accFull + 8 * s, 1);
      mbar_init(accEmpty + 8 * s, 128);
    }
    mbar_init(done, 1);
    mbar_init(xsync, 128);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp == 8) {
    if (lane == 0) {
      mbar_expect_tx(opFull, (uint32_t)(ng * per_op * A_TILE));
      for (int kk = 0; kk < ng; ++kk)
        bulk_g2s(smem_u32(sA + (size_t)kk * per_op * A_TILE), P.A + (long long)(k0 + kk) * per_op * A_TILE,
                 (uint32_t)(per_op * A_TILE), opFull);
      bool ok = mbar_wait(opFull, 0u, abort_flag, P.wait_ns);
      if (!ok) { *abort_flag = 1; atomicExch(P.err, 21); }
      for (int t = 0; ok && t < ntile; ++t) {
        const int b = t & 1, use = t >> 1;
        if (use >= 1 && !mbar_wait(accEmpty + 8 * b, (uint32_t)((use - 1) & 1), abort_flag, P.wait_ns)) {
          *abort_flag = 1;
          atomicExch(P.err, 22);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dst = tmem + (uint32_t)(b * kBN2);
        bool first = true;
        for (int kk = 0; ok && kk < ng; ++kk) {
          const int z = t * ng + kk, s = z & 1, n = z >> 1;
          if (!mbar_wait(zFull + 8 * s, (uint32_t)(n & 1), abort_flag, P.wait_ns)) {
            *abort_flag = 1;
            atomicExch(P.err, 23);
            ok = false;
            break;
          }
          tc_fence_after();
          for (int kt = 0; kt < P.kto; ++kt)
            for (int part = 0; part < P.nA; ++part) {
              const uint64_t ad = sw128_desc(smem_u32(sA + ((size_t)(kk * P.kto + kt) * P.nA + part) * A_TILE));
              // A hi pairs with z hi (and z lo when split); A lo pairs with z hi
              const int nzp = (part == 0) ? P.nZ : 1;
              for (int zp = 0; zp < nzp; ++zp) {
                const uint64_t bd = sw128_desc(smem_u32(sZ + s * zslot + (size_t)(kt * P.nZ + zp) * Z_TILE2));
#pragma unroll
                for (int j = 0; j < TC_BK / 16; ++j) {
                  tc_mma(dst, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), IDESC, first ? 0u : 1u);
                  first = false;
                }
              }
            }
          tc_commit(zEmpty + 8 * s);
        }
        if (ok) tc_commit(accFull + 8 * b);
      }
      // every MMA issued has completed, and the operator copies have landed, before TMEM and
      // shared memory are released
      tc_commit(done);
      mbar_drain(done, 0u);
      mbar_drain(opFull, 0u);
    }
  } else if (warp >= 4) {
    // ---------------- operand warps: thread (column c, k tile kt) forms 64 entries of z.  The x of
    // a tile arrives in shared memory by cp.async while the previous tile is formed; the four
    // operand warps meet on the xsync mbarrier (bounded waits, so an abort never strands them).
    const int tt = threadIdx.x - 128, c = tt & 63, kt = tt >> 6;
    const int xchunks = kBN2 * P.KP / 4;           // 16-byte chunks of one tile's x
    auto prefetch = [&](int t) {
      const long long col0 = (long long)(t_begin + t) * kBN2;
      for (int q = tt; q < xchunks; q += 128) {
        const int cc = q / (P.KP / 4), k4 = q - cc * (P.KP / 4);
        const long long col = col0 + cc;
        const bool in = col < P.ncols;
        const float* src = P.xf + (in ? col : 0) * P.KP + 4 * k4;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(sX + (size_t)cc * xld + 4 * k4);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    auto coefs = [&](int t, float (&cf)[kG2]) {
      const long long col = (long long)(t_begin + t) * kBN2 + c;
      const bool live = col < P.ncols && kt < P.kto;
      const long long cell = live ? col % P.ncell : 0;
#pragma unroll
      for (int kk = 0; kk < kG2; ++kk) cf[kk] = (live && kk < ng) ? (float)P.coef[cell * P.nops + k0 + kk] : 0.f;
    };
    int nsync = 0;
    auto osync = [&]() -> bool {                   // all 128 operand threads, bounded
      mbar_arrive(xsync);
      const bool r = mbar_wait(xsync, (uint32_t)(nsync & 1), abort_flag, P.wait_ns);
      ++nsync;
      return r;
    };
    prefetch(0);
    float cfs[kG2];
    coefs(0, cfs);
    bool ok = true;
    for (int t = 0; ok && t < ntile; ++t) {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      if (!osync()) {                                       // tile t's x is in shared memory
        *abort_flag = 1;
        atomicExch(P.err, 26);
        break;
      }
      float xv[TC_BK];
      if (kt < P.kto) {
#pragma unroll
        for (int e4 = 0; e4 < TC_BK / 4; ++e4) {
          const float4 v = *reinterpret_cast<const float4*>(sX + (size_t)c * xld + kt * TC_BK + 4 * e4);
          xv[4 * e4] = v.x; xv[4 * e4 + 1] = v.y; xv[4 * e4 + 2] = v.z; xv[4 * e4 + 3] = v.w;
        }
      }
      if (!osync()) {                                       // every thread holds its x
        *abort_flag = 1;
        atomicExch(P.err, 26);
        break;
      }
      float cf[kG2];
#pragma unroll
      for (int kk = 0; kk < kG2; ++kk) cf[kk] = cfs[kk];
      if (t + 1 < ntile) {
        prefetch(t + 1);
        coefs(t + 1, cfs);
      }
      for (int kk = 0; kk < ng; ++kk) {
        const int z = t * ng + kk, s = z & 1, n = z >> 1;
        if (n >= 1 && !mbar_wait(zEmpty + 8 * s, (uint32_t)((n - 1) & 1), abort_flag, P.wait_ns)) {
          *abort_flag = 1;
          atomicExch(P.err, 24);
          ok = false;
          break;
        }
        if (kt < P.kto) {
          uint8_t* zh = sZ + s * zslot + (size_t)(kt * P.nZ) * Z_TILE2;
#pragma unroll
          for (int ch = 0; ch < TC_BK / 8; ++ch) {
            alignas(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float zv = cf[kk] * xv[ch * 8 + e];
              h[e] = __float2bfloat16_rn(zv);
              l[e] = __float2bfloat16_rn(zv - __bfloat162float(h[e]));
            }
            *reinterpret_cast<uint4*>(zh + sw128_offset(c, ch * 8)) = *reinterpret_cast<const uint4*>(h);
            if (P.nZ > 1)
              *reinterpret_cast<uint4*>(zh + Z_TILE2 + sw128_offset(c, ch * 8)) = *reinterpret_cast<const uint4*>(l);
          }
        }
        // generic-proxy writes made visible to the tensor core before the slot is signalled
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(zFull + 8 * s);
      }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // no copy in flight at exit
  } else {
    // ---------------- epilogue warps 0-3: one row per thread, FP32 partial of the group
    const int m = warp * 32 + lane;
    for (int t = 0; t < ntile; ++t) {
      const int b = t & 1, use = t >> 1;
      if (!mbar_wait(accFull + 8 * b, (uint32_t)(use & 1), abort_flag, P.wait_ns)) {
        *abort_flag = 1;
        atomicExch(P.err, 25);
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int ch = 0; ch < kBN2 / 32; ++ch) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * kBN2 + ch * 32), r);
        tmem_ld_wait();
        if (m < P.M) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const long long col = (long long)(t_begin + t) * kBN2 + ch * 32 + j;
            if (col < P.ncols) P.yp[((long long)g * P.ncols + col) * P.M + m] = __uint_as_float(r[j]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(accEmpty + 8 * b);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// x (FP64, view strides) -> [ncols][KP] FP32, zero past K
__global__ void pack_xf_kernel(const double* __restrict__ X, long long x_rs, int x_cs, int K, int KP,
                               long long ncols, long long ncell, float* __restrict__ xf) {
  const long long total = ncols * KP;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long col = t / KP;
    const int k = (int)(t - col * KP);
    const int rhs = (int)(col / ncell);
    const long long cell = col - (long long)rhs * ncell;
    xf[t] = k < K ? (float)X[rhs * x_rs + cell * x_cs + k] : 0.f;
  }
}

// y = alpha * sum_g yp[g] + beta * y, groups added in order
__global__ void comb2_reduce_kernel(const float* __restrict__ yp, int ngroups, long long ncols, int M,
                                    long long ncell, void* __restrict__ Y, int y_f64, long long y_rs, int y_cs,
                                    double alpha, double beta) {
  const long long total = ncols * M;
  const bool narrow = total < (1ll << 31) && ncell < (1ll << 31);   // 32-bit index arithmetic
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int gi = 0; gi < ngroups; ++gi) acc += yp[gi * total + t];
    long long col, cell;
    int m, rhs;
    if (narrow) {
      const unsigned tu = (unsigned)t, cu = tu / (unsigned)M;
      m = (int)(tu - cu * (unsigned)M);
      rhs = (int)(cu / (unsigned)ncell);
      col = cu;
      cell = (long long)(cu - (unsigned)rhs * (unsigned)ncell);
    } else {
      col = t / M;
      m = (int)(t - col * M);
      rhs = (int)(col / ncell);
      cell = col - (long long)rhs * ncell;
    }
    const long long off = rhs * y_rs + cell * y_cs + m;
    const double v = alpha * (double)acc;
    if (y_f64) {
      double* y = reinterpret_cast<double*>(Y) + off;
      *y = (beta == 0.0) ? v : v + beta * (*y);
    } else {
      float* y = reinterpret_cast<float*>(Y) + off;
      *y = (beta == 0.0) ? (float)v : (float)(v + beta * (double)(*y));
    }
  }
}

static size_t comb2_smem_bytes(const TcComb& op) {
  return (size_t)kG2 * op.kto * op.nA * A_TILE + 2 * (size_t)op.kto * op.nX * Z_TILE2 +
         (size_t)kBN2 * (op.kto * TC_BK + 4) * sizeof(float) + 128 + 1024;
}

bool tc_comb2_ok(const TcComb& op) {
  return op.m_tiles == 1 && op.kto <= 2 && op.msplit == op.M && comb2_smem_bytes(op) <= 227 * 1024;
}


size_t tc_comb2_xf_bytes(const TcComb& op, long long ncols) { return (size_t)ncols * op.kto * TC_BK * sizeof(float); }
size_t tc_comb2_yp_bytes(const TcComb& op, long long ncols) {
  return (size_t)((op.nops + kG2 - 1) / kG2) * ncols * op.M * sizeof(float);
}

static fetidp_status comb2_apply(Ctx& c, const TcComb& op, CCellVec X, const double* coef, void* Y, bool y_f64,
                                 long long y_rs, int y_cs, double alpha, double beta, long long ncols,
                                 long long ncell) {
  const int KP = op.kto * TC_BK;
  if (tc_comb2_xf_bytes(op, ncols) > c.tc_xf_bytes || tc_comb2_yp_bytes(op, ncols) > c.tc_yp_bytes) {
    set_error("resident-operator combination: staging buffers too small");
    return FETIDP_EINVAL;
  }
  const int ngroups = (op.nops + kG2 - 1) / kG2;
  const int n_tiles = (int)((ncols + kBN2 - 1) / kBN2);
  int nchunk = std::max(1, std::min(n_tiles, 148 / ngroups));
  const int tpc = (n_tiles + nchunk - 1) / nchunk;
  nchunk = (n_tiles + tpc - 1) / tpc;
  if (ngroups > 65535) {
    set_error("resident-operator combination: too many principal groups");
    return FETIDP_EINVAL;
  }
  {
    ProfScope ps(c, FETIDP_K_MAPS, 0.0, (double)ncols * op.K * 8.0 + (double)ncols * KP * 4.0);
    pack_xf_kernel<<<gridn(ncols * KP), 256, 0, c.stream>>>(X.p, X.rs, X.cs, op.K, KP, ncols, ncell, c.tc_xf);
    FD_CHECK_LAUNCH();
  }
  {
    const double flops = 2.0 * op.M * (double)op.K * op.nops * (double)ncols;
    ProfScope ps(c, FETIDP_K_TC_GEMM, flops,
                 (double)op.bytes + (double)ncols * KP * 4.0 + (double)ngroups * ncols * op.M * 4.0);
    TcComb2Params P{};
    P.A = op.tiles;
    P.xf = c.tc_xf;
    P.coef = coef;
    P.yp = c.tc_yp;
    P.nops = op.nops;
    P.kto = op.kto;
    P.nA = op.nA;
    P.nZ = op.nX;
    P.M = op.M;
    P.KP = KP;
    P.n_tiles = n_tiles;
    P.tiles_per_cta = tpc;
    P.ncols = ncols;
    P.ncell = ncell;
    P.err = c.tc_err;
  P.wait_ns = c.wait_ns;
    const size_t smem = comb2_smem_bytes(op);
    cudaFuncSetAttribute(tc_comb2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_comb2_kernel<<<dim3((unsigned)nchunk, (unsigned)ngroups, 1), kComb2Threads, smem, c.stream>>>(P);
    FD_CHECK_LAUNCH();
  }
  {
    ProfScope ps(c, FETIDP_K_MAPS, 0.0, (double)ngroups * ncols * op.M * 4.0 + (double)ncols * op.M * 8.0);
    comb2_reduce_kernel<<<gridn(ncols * op.M), 256, 0, c.stream>>>(c.tc_yp, ngroups, ncols, op.M, ncell, Y,
                                                                  y_f64 ? 1 : 0, y_rs, y_cs, alpha, beta);
    FD_CHECK_LAUNCH();
  }
  return FETIDP_OK;
}

// Reference for the resident-operator kernel: Y[c][m] = sum_k sum_kk bf16(A_k[m][kk]) bf16(f32(coef[c][k]) f32(X[c][kk]))
__global__ void ref_comb2_kernel(const double* A, const double* X, const double* coef, int M, int K, int N,
                                 int nops, double* Y) {
  const long long total = (long long)M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int cidx = (int)(t / M), m = (int)(t - (long long)cidx * M);
    double acc = 0.0;
    for (int k = 0; k < nops; ++k) {
      const float cf = (float)coef[(long long)cidx * nops + k];
      for (int kk = 0; kk < K; ++kk) {
        const double a = (double)__bfloat162float(__double2bfloat16(A[((long long)k * M + m) * K + kk]));
        const float zv = cf * (float)X[(long long)cidx * K + kk];
        acc += a * (double)__bfloat162float(__float2bfloat16_rn(zv));
      }
    }
    Y[(long long)cidx * M + m] = acc;
  }
}

// Reference for the combine self-check: Y[c][m] = sum_k coef_sel[c][k] sum_kk bf16(A_k[m][kk]) bf16(X[c][kk])
__global__ void ref_comb_kernel(const double* A, const double* X, const double* coef0, const double* coef1,
                                int M, int msplit, int K, int N, int nops, double* Y) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)M * N;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / M), m = (int)(t % M);
    const double* cf = (m < msplit) ? coef0 : coef1;
    double s = 0.0;
    for (int k = 0; k < nops; ++k) {
      double d = 0.0;
      for (int kk = 0; kk < K; ++kk)
        d += (double)__bfloat162float(__double2bfloat16(A[((long long)k * M + m) * K + kk])) *
             (double)__bfloat162float(__double2bfloat16(X[(long long)c * K + kk]));
      s += cf[(long long)c * nops + k] * d;
    }
    Y[t] = s;
  }
}

fetidp_status tc_comb_selfcheck(Ctx& c, int M0, int M1, int K, int N, int nops, double* rel_err) {
  const int M = M0 + M1;
  double *A = nullptr, *X = nullptr, *C0 = nullptr, *C1 = nullptr, *Yt = nullptr, *Yr = nullptr;
  FD_CUDA(cudaMalloc(&A, sizeof(double) * (size_t)nops * M * K));
  FD_CUDA(cudaMalloc(&X, sizeof(double) * (size_t)N * K));
  FD_CUDA(cudaMalloc(&C0, sizeof(double) * (size_t)N * nops));
  FD_CUDA(cudaMalloc(&C1, sizeof(double) * (size_t)N * nops));
  FD_CUDA(cudaMalloc(&Yt, sizeof(double) * (size_t)N * M));
  FD_CUDA(cudaMalloc(&Yr, sizeof(double) * (size_t)N * M));
  fill_random_kernel<<<gridn((long long)nops * M * K), 256, 0, c.stream>>>(A, (long long)nops * M * K, 11);
  fill_random_kernel<<<gridn((long long)N * K), 256, 0, c.stream>>>(X, (long long)N * K, 12);
  fill_random_kernel<<<gridn((long long)N * nops), 256, 0, c.stream>>>(C0, (long long)N * nops, 13);
  fill_random_kernel<<<gridn((long long)N * nops), 256, 0, c.stream>>>(C1, (long long)N * nops, 14);
  FD_CHECK_LAUNCH();
  TcComb op;
  // rows [0, M0) of each operator from the first M0 rows, rows [M0, M) from the rest (same array)
  FD_TRY(tc_comb_pack(c, op, A, (long long)M * K, K, 0, 0, M0, A, (long long)M * K, K, M0, 0, M1, K, nops, 1));
  c.tc_bbuf_bytes = tc_comb_staging_bytes(op, N);
  FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.tc_bbuf), c.tc_bbuf_bytes));
  FD_TRY(tc_comb_apply(c, op, CCellVec{X, 0, K}, C0, C1, Yt, true, 0, M, 1.0, 0.0, 1, N));
  ref_comb_kernel<<<gridn((long long)M * N), 256, 0, c.stream>>>(A, X, C0, C1, M, M0, K, N, nops, Yr);
  FD_CHECK_LAUNCH();
  std::vector<double> ht((size_t)N * M), hr((size_t)N * M);
  FD_CUDA(cudaMemcpyAsync(ht.data(), Yt, sizeof(double) * ht.size(), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaMemcpyAsync(hr.data(), Yr, sizeof(double) * hr.size(), cudaMemcpyDeviceToHost, c.stream));
  int herr = 0;
  FD_CUDA(cudaMemcpyAsync(&herr, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  cudaFree(A); cudaFree(X); cudaFree(C0); cudaFree(C1); cudaFree(Yt); cudaFree(Yr);
  if (herr != 0) {
    set_error("combine kernel wait timed out (code " + std::to_string(herr) + ")");
    return FETIDP_ETIMEOUT;
  }
  // a non-finite difference counts as an infinite error (the rule of absmax_pair_kernel)
  double mx = 0.0, ref = 0.0;
  for (size_t i = 0; i < ht.size(); ++i) {
    const double dv = std::fabs(ht[i] - hr[i]);
    mx = std::isfinite(dv) ? std::max(mx, dv) : INFINITY;
    ref = std::max(ref, std::fabs(hr[i]));
  }
  *rel_err = mx / (ref > 0 ? ref : 1.0);
  if (!tc_comb2_ok(op)) return FETIDP_OK;
  // one row tile, K <= 128: the resident-operator kernel too, against its own reference (the
  // scaled operand is rounded to BF16 after the FP32 product)
  c.tc_xf_bytes = tc_comb2_xf_bytes(op, N);
  c.tc_yp_bytes = tc_comb2_yp_bytes(op, N);
  FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.tc_xf), c.tc_xf_bytes));
  FD_TRY(dalloc(c, reinterpret_cast<void**>(&c.tc_yp), c.tc_yp_bytes));
  FD_CUDA(cudaMalloc(&A, sizeof(double) * (size_t)nops * M * K));
  FD_CUDA(cudaMalloc(&X, sizeof(double) * (size_t)N * K));
  FD_CUDA(cudaMalloc(&C0, sizeof(double) * (size_t)N * nops));
  FD_CUDA(cudaMalloc(&Yt, sizeof(double) * (size_t)N * M));
  FD_CUDA(cudaMalloc(&Yr, sizeof(double) * (size_t)N * M));
  fill_random_kernel<<<gridn((long long)nops * M * K), 256, 0, c.stream>>>(A, (long long)nops * M * K, 21);
  fill_random_kernel<<<gridn((long long)N * K), 256, 0, c.stream>>>(X, (long long)N * K, 22);
  fill_random_kernel<<<gridn((long long)N * nops), 256, 0, c.stream>>>(C0, (long long)N * nops, 23);
  FD_CHECK_LAUNCH();
  TcComb op2;
  FD_TRY(tc_comb_pack(c, op2, A, (long long)M * K, K, 0, 0, M, nullptr, 0, 0, 0, 0, 0, K, nops, 1));
  FD_TRY(tc_comb_apply(c, op2, CCellVec{X, 0, K}, C0, C0, Yt, true, 0, M, 1.0, 0.0, 1, N));
  ref_comb2_kernel<<<gridn((long long)M * N), 256, 0, c.stream>>>(A, X, C0, M, K, N, nops, Yr);
  FD_CHECK_LAUNCH();
  FD_CUDA(cudaMemcpyAsync(ht.data(), Yt, sizeof(double) * ht.size(), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaMemcpyAsync(hr.data(), Yr, sizeof(double) * hr.size(), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaMemcpyAsync(&herr, c.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  cudaFree(A); cudaFree(X); cudaFree(C0); cudaFree(Yt); cudaFree(Yr);
  if (herr != 0) {
    set_error("resident-operator combine kernel wait timed out (code " + std::to_string(herr) + ")");
    return FETIDP_ETIMEOUT;
  }
  mx = 0.0;
  ref = 0.0;
  for (size_t i = 0; i < ht.size(); ++i) {
    mx = std::max(mx, std::fabs(ht[i] - hr[i]));
    ref = std::max(ref, std::fabs(hr[i]));
  }
  *rel_err = std::max(*rel_err, mx / (ref > 0 ? ref : 1.0));
  return FETIDP_OK;
}

// ---------------------------------------------------------------- allocation-free self-check
// Scratch of fetidp_tc_selfcheck_static: a fixed array in this library's device image, so the
// probe calls no cudaMalloc / cudaFree.  Its address is looked up once per device.
static __device__ __align__(256) unsigned char g_tc_static_scratch[FETIDP_TC_STATIC_SCRATCH_BYTES];

namespace {

struct TcCheckSlot {   // results of one probe, written on the device
  double diff;         // max |Y_tc - Y_ref| (+inf if Y_tc holds a non-finite value)
  double ref;          // max |Y_ref|
  int err;             // tensor-core wait / bounds status: must be zero before the GEMM runs
  int pad;
};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte offsets of the probe's buffers inside the static scratch.
struct StaticLayout {
  size_t A, X, Yt, Yr, tiles, bbuf, slot, total;
  size_t bbuf_bytes;
  int m_tiles, k_tiles, bn;
};

StaticLayout static_layout(int M, int K, int N) {
  StaticLayout L{};
  L.m_tiles = (M + TC_BM - 1) / TC_BM;
  L.k_tiles = (K + TC_BK - 1) / TC_BK;
  L.bn = tc_bn_for(N, L.m_tiles, 1);
  const size_t n_tiles = ((size_t)N + L.bn - 1) / L.bn;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += round256(bytes); return o; };
  L.A = take((size_t)M * K * sizeof(double));
  L.X = take((size_t)N * K * sizeof(double));
  L.Yt = take((size_t)N * M * sizeof(double));
  L.Yr = take((size_t)N * M * sizeof(double));
  L.tiles = take((size_t)L.m_tiles * L.k_tiles * A_TILE);
  L.bbuf_bytes = n_tiles * L.k_tiles * L.bn * TC_BK * 2;
  L.bbuf = take(L.bbuf_bytes);
  L.slot = take(sizeof(TcCheckSlot));
  L.total = off;
  return L;
}

__device__ __forceinline__ void absmax_warp(double& d, double& r) {
  for (int o = 16; o > 0; o >>= 1) {
    d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  }
}

// One block: max |a - b| and max |b|.  A maximum is exact in any order, so the result is
// deterministic; a non-finite difference turns into +inf, which no later fmax undoes.
__global__ void __launch_bounds__(1024) absmax_pair_kernel(const double* a, const double* b, long long n,
                                                         TcCheckSlot* out) {
  __shared__ double sd[32], sr[32];
  double d = 0.0, r = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(a[i] - b[i]);
    d = isfinite(v) ? fmax(d, v) : INFINITY;
    r = fmax(r, fabs(b[i]));
  }
  absmax_warp(d, r);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sd[w] = d; sr[w] = r; }
  __syncthreads();
  if (w == 0) {
    const int nw = (int)(blockDim.x >> 5);
    d = l < nw ? sd[l] : 0.0;
    r = l < nw ? sr[l] : 0.0;
    absmax_warp(d, r);
    if (l == 0) { out->diff = d; out->ref = r; }
  }
}

}  // namespace

size_t tc_selfcheck_static_bytes(int M, int K, int N) { return static_layout(M, K, N).total; }

// Address of the static scratch on the current device, looked up on every call: a cached address
// would go stale if the device's primary context were reset and the module loaded again.
fetidp_status tc_static_scratch(uint8_t** p) {
  void* a = nullptr;
  FD_CUDA(cudaGetSymbolAddress(&a, g_tc_static_scratch));
  *p = static_cast<uint8_t*>(a);
  return FETIDP_OK;
}

// The probe of tc_selfcheck (same seeds, same kernels) with every buffer carved from the static
// scratch.  The caller has checked tc_selfcheck_static_bytes against the scratch size.
fetidp_status tc_selfcheck_static(Ctx& c, int M, int K, int N, double* rel_err) {
  const StaticLayout L = static_layout(M, K, N);
  if (L.total > (size_t)FETIDP_TC_STATIC_SCRATCH_BYTES) {
    set_error("tensor-core probe does not fit the static scratch");
    return FETIDP_EINVAL;
  }
  uint8_t* base = nullptr;
  FD_TRY(tc_static_scratch(&base));
  double* A = reinterpret_cast<double*>(base + L.A);
  double* X = reinterpret_cast<double*>(base + L.X);
  double* Yt = reinterpret_cast<double*>(base + L.Yt);
  double* Yr = reinterpret_cast<double*>(base + L.Yr);
  TcCheckSlot* slot = reinterpret_cast<TcCheckSlot*>(base + L.slot);
  FD_CUDA(cudaMemsetAsync(slot, 0, sizeof(TcCheckSlot), c.stream));
  c.tc_err = &slot->err;
  c.tc_bbuf = base + L.bbuf;
  c.tc_bbuf_bytes = L.bbuf_bytes;
  fill_random_kernel<<<gridn((long long)M * K), 256, 0, c.stream>>>(A, (long long)M * K, 1234);
  fill_random_kernel<<<gridn((long long)N * K), 256, 0, c.stream>>>(X, (long long)N * K, 5678);
  FD_CHECK_LAUNCH();
  TcOperator op;
  op.M = M;
  op.K = K;
  op.nops = 1;
  op.nterm = 1;
  op.separate = false;
  op.m_tiles = L.m_tiles;
  op.k_tiles_op = L.k_tiles;
  op.k_tiles = L.k_tiles;
  op.batch_bytes = (long long)L.m_tiles * L.k_tiles * A_TILE;
  op.tiles = base + L.tiles;
  pack_A_kernel<<<gridn((long long)L.m_tiles * L.k_tiles * TC_BM * 8), 256, 0, c.stream>>>(
      A, 0, K, 0, 0, M, K, 1, 1, L.k_tiles, L.m_tiles, 1, op.tiles);
  FD_CHECK_LAUNCH();
  FD_TRY(tc_apply(c, op, CCellVec{X, 0, K}, nullptr, Yt, true, 0, M, 0, 1.0, 0.0, 1, N));
  ref_gemm_kernel<<<gridn((long long)M * N), 256, 0, c.stream>>>(A, X, M, K, N, Yr);
  FD_CHECK_LAUNCH();
  absmax_pair_kernel<<<1, 1024, 0, c.stream>>>(Yt, Yr, (long long)M * N, slot);
  FD_CHECK_LAUNCH();
  TcCheckSlot h{};
  FD_CUDA(cudaMemcpyAsync(&h, slot, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
  FD_CUDA(cudaStreamSynchronize(c.stream));
  if (h.err != 0) {
    set_error("tensor-core GEMM wait timed out or left its bounds (code " + std::to_string(h.err) + ")");
    return FETIDP_ETIMEOUT;
  }
  *rel_err = h.diff / (h.ref > 0 ? h.ref : 1.0);
  return FETIDP_OK;
}

// ---------------------------------------------------------------- bounded-wait probe
// One thread waits, through the pipeline's own bounded wait, on phase 0 of an mbarrier that
// expects one arrival nobody makes: the wait must expire after wait_ns and set the error flag,
// exactly as an expired wait does in the tensor-core kernels.  Nothing asynchronous is in flight.
namespace {
__device__ int g_wait_probe_flag;

__global__ void wait_probe_kernel(unsigned long long wait_ns, int* flag) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    *flag = mbar_wait(smem_u32(&bar), 0u, reinterpret_cast<volatile int*>(&abort_flag), wait_ns) ? 0 : 31;
}
}  // namespace

fetidp_status wait_selfcheck(unsigned long long wait_ns, cudaStream_t stream) {
  void* a = nullptr;
  FD_CUDA(cudaGetSymbolAddress(&a, g_wait_probe_flag));
  int* flag = static_cast<int*>(a);
  FD_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), stream));
  wait_probe_kernel<<<1, 32, 0, stream>>>(wait_ns, flag);
  FD_CHECK_LAUNCH();
  int h = 0;
  FD_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
  FD_CUDA(cudaStreamSynchronize(stream));
  if (h != 0) {
    set_error("device wait expired after its budget (code " + std::to_string(h) + ")");
    return FETIDP_ETIMEOUT;
  }
  return FETIDP_OK;
}

FD_DEFINE_CHECK(fd_check_tc)

}  // namespace fetidp
