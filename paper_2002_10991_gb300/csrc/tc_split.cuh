// Split-precision WY application on the fifth-generation tensor cores:
// tcgen05.mma with BF16 digit operands in shared memory and FP32 accumulators
// in tensor memory (TMEM), operand tiles brought in by the bulk-copy engine.
//
// Same method as split_kernels.cuh (compact WY blocks of 32 reflectors,
// Z <- Z - U (V^T Z), exact digit products summed per level in FP32, levels
// combined in 64-bit integers), laid out for one CTA per SM that owns a strip
// of 128 columns of the eigenvector block:
//
//  * Z stays in registers. The block window (R = b + 31 rows, padded to 32 P
//    rows, P = 3 for b = 64 and 2 for b = 32) is cut into P parts of 32 rows;
//    thread group g (4 warps, one column per thread) holds part (g + t) mod P
//    of block t. Consecutive blocks of a sweep start 32 rows apart (blocks
//    are aligned to stages 32k .. 32k+31), so from one block to the next each
//    part moves down one place and the group of the part that leaves the
//    window stores it and takes the 32 new rows on top: no data moves between
//    threads.
//  * GEMM1 W^T = Z^T V' runs as M = 128 (strip columns) x N = 32 * (slices) x
//    K = window rows: one instruction per digit of Z and K step covers every V'
//    slice it pairs with, writing each slice into the TMEM columns of its
//    level (level l = i + k of the 0-based digit indices, 32 columns each).
//    The math warps write the six digit slices of Z into tensor memory
//    (tcgen05.st) as the A operand of these MMAs, one ready barrier per
//    digit, so the tensor core starts on a digit as soon as it is complete.
//  * W is combined per column by the thread that owns the column (no
//    shuffles), normalised, split into digits (the A operand of GEMM2).
//  * GEMM2 corr^T = W^T U'^T runs per part of 32 rows (M = 128, N = 32 *
//    slices, K = 32) into two TMEM regions used in turn; the group that owns
//    the part reads its accumulators and subtracts the correction.
//
// Exactness (digit positions 61 - 8k, k = 1..6, balanced digits): Z is fixed
// point with |Z| <= 2^61 (first digit |d| <= 256, others <= 128); V', U' and W
// are scaled to |x| <= 2^60 so that all their digits are <= 128. Before its
// digits are taken, each column's window of Z is shifted left by the most
// bits that keep |Z| < 2^61 and its 1-norm within 2^66 (the bound that keeps
// W in 64-bit range), so the digits hold the window's leading bits. A level sums
// at most 6 digit products over K terms: GEMM1 (K <= 96) stays below 2^24 and
// is read with an exact float->int conversion; GEMM2 (K = 32) stays below 2^22,
// where the add-magic-number conversion is exact.
//
// Digits are read from the offset form Z' = Z + C (C = sum_k 128 * 2^(61-8k) +
// 2^12): then digit k is the plain byte e_k of Z' at bit 61 - 8k and d_k =
// e_k - 128, so a digit costs a shift, a logic op and one FADD (the byte is
// placed in the mantissa of 2^23 and 2^23 + 128 subtracted). Z is kept in
// registers in that form.
//
// Dependencies between sweeps, the work-unit queue and the bounded waits are
// those of the FP64 kernel (one sweep of one strip per unit).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "apply_kernels.cuh"
#include "split_kernels.cuh"

namespace tbbt {
namespace tcs {

constexpr int NB = 32;       // reflectors per WY block
constexpr int S = 6;         // digits per operand
constexpr int LV = 7;        // levels kept (0-based l = i + k <= 6)
constexpr int WS = 128;      // strip columns = MMA M
constexpr int FIX = 61;      // fixed-point exponent of the eigenvector block
constexpr int FOP = 60;      // fixed-point exponent of V', U' and normalised W
constexpr int STG_ROWS = 16;  // rows per staging box (16 x 8 bytes = one 128-byte swizzle row per column)
constexpr int TMEM_COLS = 512;
constexpr int REG_B = 224;   // second TMEM region (first one starts at column 0)
constexpr int ZA_COL = 224;  // the Z digits (A operand of the first product), after its accumulators

// offset of the balanced-digit form: 128 at every digit position + half a unit
// of the last digit
constexpr long long kDigitOffset = (1LL << 60) + (1LL << 52) + (1LL << 44) + (1LL << 36) + (1LL << 28) +
                                   (1LL << 20) + (1LL << 12);

template <int B>
struct Geo {
  static constexpr int R = B + NB - 1;
  static constexpr int RP = (R + 31) / 32 * 32;  // window rows, padded
  static constexpr int P = RP / 32;              // parts of 32 rows
  static constexpr int KS1 = RP / 16;            // K steps of GEMM1
  static constexpr int H = 2;                    // threads per column and part
  static constexpr int RT = 32 / H;              // rows of a part held by one thread
  static constexpr int NSUB = P * H;             // thread sets covering all 128 columns
  static constexpr int NMATH = 4 * P * H * 32;   // threads of the math warps
  static constexpr int NTHREADS = NMATH + 32;    // + the producer warp
  static constexpr int SBO1 = (RP / 8) * 128;    // row-group stride of K = RP operands
  static constexpr int VBYTES = S * NB * RP * 2;         // V' digits [32 i + m][r]
  static constexpr int UCHUNK = S * NB * 32 * 2;         // U' digits of one part [32 i + rr][m]
  static constexpr int UBYTES = P * UCHUNK;
  static constexpr int EBYTES = 128;                     // per-row exponents of U (int8)
  static constexpr int BLOCK_BYTES = VBYTES + UBYTES + EBYTES;
  static constexpr int ZCOLS = RP / 2;                   // TMEM columns of one Z digit (bf16 pairs)
  static constexpr int WDIG = WS * NB * 2;               // one digit of W [c][m]
  static constexpr int OFF_W = 0;                        // S W digit buffers
  static constexpr int OFF_V = OFF_W + S * WDIG;
  static constexpr int OFF_U = OFF_V + VBYTES;
  static constexpr int OFF_STG = (OFF_U + UBYTES + 1023) / 1024 * 1024;  // two swizzled boxes [c][16 rows]
  // [NSUB][WS] partial maxima of |W|; before that, in the same place,
  // [2 NSUB][WS] partial maxima and 1-norms of the window's Z
  static constexpr int OFF_KMX = OFF_STG + 2 * WS * STG_ROWS * 8;
  static constexpr int SMEM = OFF_KMX + 2 * NSUB * WS * 8 + 1024;  // + room to align the base to 1024 bytes
};

// byte offset of element (row, k) of a K-major operand with kt values of k per
// row, in the no-swizzle core-matrix layout: 8 x 16-byte core matrices, cores
// adjacent in k 128 bytes apart (LBO), row groups kt/8 * 128 apart (SBO)
__host__ __device__ constexpr int kmaj(int row, int k, int kt) {
  return ((row >> 3) * (kt >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// ---------------------------------------------------------------------------
// tcgen05, mbarrier and bulk-copy primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;              // leading byte offset: next core in K
  d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;  // stride byte offset: next row group
  d |= (uint64_t)1 << 46;                       // descriptor version of tcgen05
  return d;                                     // base offset 0, no swizzle
}
// instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
// A operand in tensor memory: lane m = row m, K elements as bf16 pairs along the columns
__device__ __forceinline__ void tc_mma_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
template <int C>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[C]) {
  if constexpr (C == 16) tmem_ld16(taddr, r);
  else if constexpr (C == 8) tmem_ld8(taddr, r);
  else tmem_ld4(taddr, r);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// 2-D tiled TMA load (tensor map in kernel-parameter space) completing on an mbarrier
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

// Bounded wait for the completion of the phase with the given parity. Gives
// up (and sets the block's abort flag) on timeout or when another role of the
// block has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort, int *err,
                                          long long timeout_ns) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_test(bar, parity)) return true;
    if (*abort) return false;
    if ((it & 15) == 0 && globaltimer_ns() - t0 > timeout_ns) {
      atomicCAS(err, 0, 4 /* TBBT_ETIMEOUT */);
      *abort = 1;
      return false;
    }
  }
}

// ---------------------------------------------------------------------------
// digits
// ---------------------------------------------------------------------------
// Digit k (1-based) of a value in offset form, as the float d_k (exact).
template <int K>
__device__ __forceinline__ float digit_of(uint32_t lo, uint32_t hi) {
  if constexpr (K == 1) {
    const int32_t e = (int32_t)hi >> 21;  // bits 53.. of the offset value, signed
    return __int_as_float(0x4B400000 + e) - 12583040.0f;  // (1.5 * 2^23 + e) - (1.5 * 2^23 + 128)
  } else {
    constexpr int pos = 61 - 8 * K;  // 45, 37, 29, 21, 13
    uint32_t bits;
    if constexpr (pos >= 32)
      bits = hi >> (pos - 32);
    else if constexpr (pos + 8 <= 32)
      bits = lo >> pos;
    else
      bits = __funnelshift_r(lo, hi, pos);
    return __int_as_float((int)((bits & 0xFFu) | 0x4B000000u)) - 8388736.0f;  // (2^23 + e) - (2^23 + 128)
  }
}
// two floats whose low 16 bits are zero -> bf16x2 (first value in the low half)
__device__ __forceinline__ uint32_t pack_hi16(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}
template <int K>
__device__ __forceinline__ uint4 digits8(const int64_t *x) {
  uint32_t w[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const uint64_t a = (uint64_t)x[2 * e], b = (uint64_t)x[2 * e + 1];
    w[e] = pack_hi16(digit_of<K>((uint32_t)a, (uint32_t)(a >> 32)), digit_of<K>((uint32_t)b, (uint32_t)(b >> 32)));
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}
template <int K>
__device__ __forceinline__ uint2 digits4(const int64_t *x) {
  uint32_t w[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const uint64_t a = (uint64_t)x[2 * e], b = (uint64_t)x[2 * e + 1];
    w[e] = pack_hi16(digit_of<K>((uint32_t)a, (uint32_t)(a >> 32)), digit_of<K>((uint32_t)b, (uint32_t)(b >> 32)));
  }
  return make_uint2(w[0], w[1]);
}
// digit K of R consecutive rows of one column -> R / 2 TMEM columns of the
// thread's lane (bf16 pairs, the even row in the low half)
template <int K, int R>
__device__ __forceinline__ void tmem_digits(uint32_t taddr, const int64_t (&z)[R]) {
  uint32_t w[R / 2];
#pragma unroll
  for (int q = 0; q < R / 8; ++q) {
    const uint4 v = digits8<K>(z + 8 * q);
    w[4 * q] = v.x;
    w[4 * q + 1] = v.y;
    w[4 * q + 2] = v.z;
    w[4 * q + 3] = v.w;
  }
  if constexpr (R == 16) tmem_st8(taddr, w);
  else tmem_st16(taddr, w);
}
template <int R>
__device__ __forceinline__ void tmem_z_digit(int k, uint32_t taddr, const int64_t (&z)[R]) {
  switch (k) {
    case 1: tmem_digits<1, R>(taddr, z); break;
    case 2: tmem_digits<2, R>(taddr, z); break;
    case 3: tmem_digits<3, R>(taddr, z); break;
    case 4: tmem_digits<4, R>(taddr, z); break;
    case 5: tmem_digits<5, R>(taddr, z); break;
    default: tmem_digits<6, R>(taddr, z); break;
  }
}

// exact float -> int for integer values below 2^22 in magnitude
__device__ __forceinline__ int32_t f2i_small(float v) { return __float_as_int(v + 12582912.0f) - 0x4B400000; }
__device__ __forceinline__ int64_t shl_signed(int64_t x, int s) {
  return s >= 0 ? (int64_t)((uint64_t)x << s) : (x >> min(-s, 63));
}
__device__ __forceinline__ int64_t shl8_add(int64_t h, int32_t v) { return (int64_t)((uint64_t)h << 8) + v; }

// round(x * 2^sh) for |x * 2^sh| < 2^62, from the bits of x (integer unit only;
// halves round up); zero and subnormal x give 0
__device__ __forceinline__ int64_t fix_round(double x, int sh) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;
  const uint64_t mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // |x| = mant 2^(e - 1075)
  const int s = e - 1075 + sh;
  int64_t r;
  if (s >= 0) r = (int64_t)(mant << s);
  else if (s > -64) r = (int64_t)((mant + (1ull << (-s - 1))) >> (-s));
  else r = 0;
  return (b >> 63) ? -r : r;
}
// e with |x| < 2^e (the frexp exponent) of the largest magnitude whose
// bits (sign cleared) are m; 0 for m = 0
__device__ __forceinline__ int exp_of_bits(uint64_t m) { return m ? (int)(m >> 52) - 1022 : 0; }
__device__ __forceinline__ uint64_t abs_bits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// ---------------------------------------------------------------------------
// per-plan preparation: FP64 T and U = V T per block, digits in the operand
// layouts of the tensor-core kernel
// ---------------------------------------------------------------------------
// Blocks of sweep j cover stages 32k .. min(32k + 31, imax(j)), k = kt(j) ..
// 0 with kt(j) = imax(j) / 32; block id = block_start[j] + (kt(j) - k).
template <int B>
__global__ void __launch_bounds__(128) tc_prepare_kernel(const double *__restrict__ vstore, StoreGeom g, int32_t ldv,
                                                         const int64_t *__restrict__ block_start, int32_t J,
                                                         int64_t nblocks, unsigned char *__restrict__ slices,
                                                         int32_t *__restrict__ gvs) {
  using D = Geo<B>;
  constexpr int RP = D::RP;
  __shared__ double sV[RP][NB + 1];  // V, later U = V T
  __shared__ double sT[NB][NB + 1];
  __shared__ double sG[NB][NB + 1];  // Gram matrix V^T V (strict upper triangle)
  __shared__ double stau[NB];
  __shared__ uint64_t sred[4];
  __shared__ int sgu[RP];
  const int64_t blk = blockIdx.x;
  if (blk >= nblocks) return;
  int32_t lo = 0, hi = J - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (block_start[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const int32_t j = lo;
  const int32_t kk = g.imax(j) / NB - (int32_t)(blk - block_start[j]);
  const int32_t s_lo = kk * NB;
  const int32_t cnt = min(NB, g.imax(j) - s_lo + 1);
  const int tid = threadIdx.x;
  const int64_t base = g.sweep_offset(j) + g.imax(j);  // entry of stage s: base - s
  for (int idx = tid; idx < RP * NB; idx += blockDim.x) {
    const int m = idx / RP, r = idx - m * RP;  // consecutive threads read one entry's consecutive elements
    double val = 0.0;
    if (m < cnt) {
      const int32_t s = s_lo + m;
      const int32_t L = g.len(s, j);
      const int tt = r - m;
      if (tt == 0) val = 1.0;
      else if (tt > 0 && tt < L) val = vstore[(base - s) * ldv + tt];
    }
    sV[r][m] = val;
  }
  for (int m = tid; m < NB; m += blockDim.x) stau[m] = m < cnt ? vstore[(base - (s_lo + m)) * ldv] : 0.0;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) sT[idx / NB][idx % NB] = 0.0;
  __syncthreads();
  // compact WY of H_0 H_1 ... H_{cnt-1} (H_m of stage s_lo + m; the highest
  // stage acts first): T_mm = tau_m, T[0:m, m] = -tau_m T[0:m, 0:m] (V^T v_m).
  // Column k of V is zero outside rows k .. k + B - 1, so V^T v_m needs rows
  // m .. k + B - 1 only; all of V^T V first (in parallel), then the recurrence.
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int k = idx / NB, m = idx - k * NB;
    if (k < m && m < cnt) {
      double acc = 0.0;
      const int rend = min(k + B, RP);
      for (int r = m; r < rend; ++r) acc = fma(sV[r][k], sV[r][m], acc);
      sG[k][m] = acc;
    }
  }
  __syncthreads();
  for (int m = 0; m < cnt; ++m) {
    for (int k = tid; k < m; k += blockDim.x) {
      double acc = 0.0;
      for (int l = k; l < m; ++l) acc = fma(sT[k][l], sG[l][m], acc);
      sT[k][m] = -stau[m] * acc;
    }
    if (tid == 0) sT[m][m] = stau[m];
    __syncthreads();
  }
  unsigned char *out = slices + blk * (int64_t)D::BLOCK_BYTES;
  // V' = V 2^(60 - gv), |V| <= 2^gv (magnitudes compared as IEEE bit patterns)
  uint64_t mx = 0;
  for (int idx = tid; idx < RP * NB; idx += blockDim.x) {
    const uint64_t a = abs_bits(sV[idx / NB][idx % NB]);
    mx = a > mx ? a : mx;
  }
  for (int o = 16; o; o >>= 1) {
    const uint64_t a = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = a > mx ? a : mx;
  }
  if ((tid & 31) == 0) sred[tid >> 5] = mx;
  __syncthreads();
  mx = sred[0] > sred[1] ? sred[0] : sred[1];
  mx = sred[2] > mx ? sred[2] : mx;
  mx = sred[3] > mx ? sred[3] : mx;
  const int gv = exp_of_bits(mx);
  // each item: 8 consecutive rows of one column of V', one 16-byte chunk per digit
  for (int idx = tid; idx < NB * (RP / 8); idx += blockDim.x) {
    const int m = idx % NB, r0 = 8 * (idx / NB);
    int64_t x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = fix_round(sV[r0 + e][m], FOP - gv);
#pragma unroll
    for (int sl = 1; sl <= S; ++sl) {
      uint32_t wv[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn((float)split::peel_digit(x[2 * e], sl),
                                                         (float)split::peel_digit(x[2 * e + 1], sl));
        wv[e] = *reinterpret_cast<const uint32_t *>(&h2);
      }
      *reinterpret_cast<uint4 *>(out + kmaj(NB * (sl - 1) + m, r0, RP)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
  }
  __syncthreads();
  // U = V T: row r of V is zero outside columns r - B + 1 .. r; each thread
  // computes its outputs in registers, then all write them over V
  {
    constexpr int PER = RP * NB / 128;  // outputs per thread (128 threads)
    double u[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = tid + 128 * i;
      const int r = idx / NB, m = idx - r * NB;
      double acc = 0.0;
      const int k0 = max(0, r - B + 1), k1 = min(m, r);
      for (int k = k0; k <= k1; ++k) acc = fma(sV[r][k], sT[k][m], acc);
      u[i] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = tid + 128 * i;
      sV[idx / NB][idx % NB] = u[i];
    }
  }
  __syncthreads();
  // U' = U 2^(60 - gu[r]) per row, |U[r][:]| <= 2^gu[r]
  int8_t *rowexp = reinterpret_cast<int8_t *>(out + D::VBYTES + D::UBYTES);
  for (int r = tid; r < RP; r += blockDim.x) {
    uint64_t m2 = 0;
    for (int m = 0; m < NB; ++m) {
      const uint64_t a = abs_bits(sV[r][m]);
      m2 = a > m2 ? a : m2;
    }
    // rows below 2^-64 keep the scale of 2^-64 (their contribution is far
    // below the digit truncation); the exponent fits int8
    int e = exp_of_bits(m2);
    e = e < -64 ? -64 : (e > 100 ? 100 : e);
    sgu[r] = e;
    rowexp[r] = (int8_t)e;
  }
  for (int r = RP + tid; r < D::EBYTES; r += blockDim.x) rowexp[r] = 0;
  __syncthreads();
  // each item: 8 consecutive columns of one row of U', one 16-byte chunk per digit
  for (int idx = tid; idx < RP * (NB / 8); idx += blockDim.x) {
    const int r = idx % RP, m0 = 8 * (idx / RP);
    const int part = r >> 5, rr = r & 31;
    int64_t x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = fix_round(sV[r][m0 + e], FOP - sgu[r]);
#pragma unroll
    for (int sl = 1; sl <= S; ++sl) {
      uint32_t wv[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 h2 = __floats2bfloat162_rn((float)split::peel_digit(x[2 * e], sl),
                                                         (float)split::peel_digit(x[2 * e + 1], sl));
        wv[e] = *reinterpret_cast<const uint32_t *>(&h2);
      }
      *reinterpret_cast<uint4 *>(out + D::VBYTES + part * D::UCHUNK + kmaj(NB * (sl - 1) + rr, m0, NB)) =
          make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
  }
  if (tid == 0) gvs[blk] = gv;
}

// ---------------------------------------------------------------------------
// fixed point <-> FP64 (separate workspace: column c, row r at c * ldz + r + 1,
// so that every 32-row part of a block window starts on a 16-byte boundary)
// ---------------------------------------------------------------------------
__global__ void to_fixed_kernel(const double *__restrict__ q, int64_t ldq, int64_t *__restrict__ z, int64_t ldz,
                                int32_t n, int32_t nev, int32_t *__restrict__ col_exp) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nev) return;
  const double *col = q + c * ldq;
  double ss = 0.0;
  for (int32_t r = lane; r < n; r += 32) ss = fma(col[r], col[r], ss);
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  int e = 0;
  if (ss > 0.0) frexp(sqrt(ss), &e);
  if (lane == 0) col_exp[c] = e;
  int64_t *zc = z + c * ldz + 1;
  for (int32_t r = lane; r < n; r += 32) zc[r] = __double2ll_rn(ldexp(col[r], FIX - e));
}

__global__ void from_fixed_kernel(double *__restrict__ q, int64_t ldq, const int64_t *__restrict__ z, int64_t ldz,
                                  int32_t n, int32_t nev, const int32_t *__restrict__ col_exp) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nev) return;
  const int e = col_exp[c];
  const int64_t *zc = z + c * ldz + 1;
  double *col = q + c * ldq;
  for (int32_t r = lane; r < n; r += 32) col[r] = ldexp(__ll2double_rn(zc[r]), e - FIX);
}

// ---------------------------------------------------------------------------
// the apply kernel
// ---------------------------------------------------------------------------
struct TcArgs {
  int64_t *z;  // fixed-point workspace (see to_fixed_kernel)
  int64_t ldz;
  StoreGeom g;
  int32_t nev;
  int32_t strips;  // ceil(nev / 128)
  int32_t units;   // strips * sweeps
  const unsigned char *slices;
  const int32_t *gvs;
  const int64_t *block_start;  // per sweep
  int *flags;                  // per unit: lowest row final for its sweep
  unsigned *counter;
  int *err;
  long long timeout_ns;
  int withhold;  // test hook: unit that never publishes its progress (-1: none)
};

// Levels of W = V'^T Z for C consecutive reflectors of this thread's column,
// combined exactly (Horner in base 2^8 over levels 0..5, then the level-6
// term): W_int = sum_l a_l 2^(42 - 8 l).
template <int C>
__device__ __forceinline__ void w_levels(uint32_t taddr, int64_t *w) {
#pragma unroll
  for (int l = 0; l < LV; l += 2) {
    uint32_t r[2][C];
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (l + h < LV) {
        if constexpr (C == 8) tmem_ld8(taddr + 32 * (l + h), r[h]);
        else tmem_ld4(taddr + 32 * (l + h), r[h]);
      }
    tc_wait_ld();
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int i = 0; i < C; ++i) {
        if (l + h >= LV) continue;
        const int32_t v = __float2int_rn(__uint_as_float(r[h][i]));  // |v| < 2^24: exact
        if (l + h == 0) w[i] = v;
        else if (l + h < LV - 1) w[i] = shl8_add(w[i], v);
        else w[i] = (int64_t)((uint64_t)w[i] << 2) + (v >> 6);  // 4 h + floor(a_6 / 64)
      }
  }
}

// RT rows rb .. of one column of the fixed-point block (column pointer zc,
// row r at zc[r]), as 16-byte pairs where the address allows (it does for
// every window part: the parts start at odd rows, zc + r is then on a
// 16-byte boundary), scalar otherwise; rows >= n are skipped / read as `add`.
template <int RT>
__device__ __forceinline__ void tc_store_rows(int64_t *zc, int32_t rb, int32_t n, const int64_t (&z)[RT], int64_t sub) {
  const bool pairs = ((reinterpret_cast<uintptr_t>(zc + rb)) & 15) == 0;
#pragma unroll
  for (int i = 0; i < RT; i += 2) {
    const int32_t r = rb + i;
    if (pairs && r + 1 < n) {
      *reinterpret_cast<longlong2 *>(zc + r) = make_longlong2(z[i] - sub, z[i + 1] - sub);
    } else {
      if (r < n) zc[r] = z[i] - sub;
      if (r + 1 < n) zc[r + 1] = z[i + 1] - sub;
    }
  }
}
template <int RT>
__device__ __forceinline__ void tc_load_rows(const int64_t *zc, int32_t rb, int32_t n, bool valid, int64_t add,
                                             int64_t (&z)[RT]) {
  const bool pairs = ((reinterpret_cast<uintptr_t>(zc + rb)) & 15) == 0;
#pragma unroll
  for (int i = 0; i < RT; i += 2) {
    const int32_t r = rb + i;
    if (valid && pairs && r + 1 < n) {
      const longlong2 v = __ldcg(reinterpret_cast<const longlong2 *>(zc + r));
      z[i] = v.x + add;
      z[i + 1] = v.y + add;
    } else {
      z[i] = (valid && r < n) ? (int64_t)__ldcg((const long long *)(zc + r)) + add : add;
      z[i + 1] = (valid && r + 1 < n) ? (int64_t)__ldcg((const long long *)(zc + r + 1)) + add : add;
    }
  }
}

struct TcBarriers {
  uint64_t zfull[S], blk, g1, wfull, c[3], cfree, v, u, stage, drain;
};

template <int B>
__global__ void __launch_bounds__(Geo<B>::NTHREADS, 1) tc_apply_kernel(TcArgs a, const __grid_constant__ CUtensorMap zmap) {
  using D = Geo<B>;
  constexpr int P = D::P;
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  // the swizzled staging boxes need a 1024-byte aligned base
  unsigned char *const smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  __shared__ TcBarriers bars;
  __shared__ uint32_t s_tmem;
  __shared__ int s_unit;
  __shared__ int s_stop;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == 4 * P * D::H;
  const int grp = warp / (4 * D::H);        // math group (parts rotate over groups)
  const int hf = (warp >> 2) % D::H;        // which rows of the part: RT * hf ..
  const int col = (warp & 3) * 32 + lane;   // strip column of this math thread = its TMEM lane
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const StoreGeom &g = a.g;

  if (warp == 4 * P * D::H) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int k = 0; k < S; ++k) mbar_init(&bars.zfull[k], D::NMATH);
    mbar_init(&bars.blk, D::NMATH);
    mbar_init(&bars.g1, 1);
    mbar_init(&bars.wfull, D::NMATH);
    for (int p = 0; p < 3; ++p) mbar_init(&bars.c[p], 1);
    mbar_init(&bars.cfree, 128 * D::H);
    mbar_init(&bars.v, 1);
    mbar_init(&bars.u, 1);
    mbar_init(&bars.stage, 1);
    mbar_init(&bars.drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  // phase counters (each role counts the completions it waits for)
  uint32_t n_blk = 0;    // blocks processed so far (g1, wfull, c[*], cfree)
  uint32_t n_v = 0, n_u = 0;  // producer: completions of the operand loads waited for
  uint32_t n_st = 0;          // staged row loads (issued by the producer, counted by every math thread)
  uint32_t iss_v = 0, iss_u = 0, iss_st = 0;  // producer: loads issued (for the drain)

  for (;;) {
    if (tid == 0) {
      s_unit = (int)atomicAdd(a.counter, 1u);
      s_stop = (*(volatile int *)a.err != 0);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int u = s_unit;
    if (u >= a.units || s_stop || s_abort) break;
    const int32_t j = u / a.strips;
    const int32_t c0 = (u - j * a.strips) * WS;
    int *myflag = a.flags + u;
    const int *prevflag = j > 0 ? a.flags + (u - a.strips) : nullptr;
    const bool publish = u != a.withhold;
    const int32_t kt = g.imax(j) / NB;  // blocks k = kt .. 0
    const int32_t nblk = kt + 1;
    const int32_t jb = j * g.b;
    const int64_t blk0 = a.block_start[j];
    auto r0_of = [&](int32_t t) { return (kt - t) * NB + 1 + jb; };  // first window row of block t
    // every row of the first window must be final for the previous sweep
    if (tid == 0 && prevflag && wait_released_raw(a.err, a.timeout_ns, prevflag, r0_of(0))) s_abort = 1;
    __syncthreads();

    if (!s_abort) {
      if (producer) {
        if (warp == 4 * P * D::H && lane == 0) {
          // ------------------------------------------------------------ producer
          const unsigned char *blkp = a.slices + blk0 * (int64_t)D::BLOCK_BYTES;
          mbar_expect_tx(&bars.v, D::VBYTES);
          bulk_load(smem + D::OFF_V, blkp, D::VBYTES, &bars.v);
          ++iss_v;
          mbar_expect_tx(&bars.u, D::UBYTES);
          bulk_load(smem + D::OFF_U, blkp + D::VBYTES, D::UBYTES, &bars.u);
          ++iss_u;
          const uint32_t wbase = smem_u32(smem + D::OFF_W);
          const uint32_t vbase = smem_u32(smem + D::OFF_V);
          const uint32_t ubase = smem_u32(smem + D::OFF_U);
          for (int32_t t = 0; t < nblk && !s_abort; ++t) {
            const int32_t r0 = r0_of(t);
            if (!mbar_wait(&bars.v, n_v & 1, &s_abort, a.err, a.timeout_ns)) break;
            ++n_v;
            // GEMM1: level l = i + k (0-based), 32 TMEM columns per level
            bool ok = true;
            for (int k = 0; k < S; ++k) {
              if (!mbar_wait(&bars.zfull[k], n_blk & 1, &s_abort, a.err, a.timeout_ns)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const int ni = (S < LV - k) ? S : LV - k;  // V' slices paired with digit k
              const uint32_t za = tmem + ZA_COL + D::ZCOLS * k;
              for (int ks = 0; ks < D::KS1; ++ks) {
                const uint32_t bv = vbase + ks * 256;
                if (k == 1 && ks == 0) {
                  // levels 1..5 accumulate; level 6 starts here (slice 5)
                  tc_mma_ta(tmem + 32, za, smem_desc(bv, D::SBO1), idesc_bf16(5 * NB), 1);
                  tc_mma_ta(tmem + 32 * 6, za, smem_desc(bv + 20 * D::SBO1, D::SBO1), idesc_bf16(NB), 0);
                } else {
                  tc_mma_ta(tmem + 32 * k, za + 8 * ks, smem_desc(bv, D::SBO1), idesc_bf16(ni * NB),
                            (k > 0 || ks > 0) ? 1u : 0u);
                }
              }
            }
            if (!ok) break;
            tc_commit(&bars.g1);
            // V' is free once GEMM1 is done: bring in the next block's
            if (!mbar_wait(&bars.g1, n_blk & 1, &s_abort, a.err, a.timeout_ns)) break;
            if (t + 1 < nblk) {
              mbar_expect_tx(&bars.v, D::VBYTES);
              bulk_load(smem + D::OFF_V, blkp + (int64_t)(t + 1) * D::BLOCK_BYTES, D::VBYTES, &bars.v);
              ++iss_v;
            }
            // GEMM2 per part of 32 rows
            if (!mbar_wait(&bars.u, n_u & 1, &s_abort, a.err, a.timeout_ns)) break;
            ++n_u;
            if (!mbar_wait(&bars.wfull, n_blk & 1, &s_abort, a.err, a.timeout_ns)) break;
            tc_fence_after();
            // parts in the order P-1 (the part leaving the window: its group then
            // stores it and takes the new rows while the others are computed),
            // 0, 1; part 0 in region A (free since W was read), the others in
            // region B one after the other
            for (int o = 0; o < P && ok; ++o) {
              const int p = (o == 0) ? P - 1 : o - 1;
              if (o == 2) {
                if (!mbar_wait(&bars.cfree, n_blk & 1, &s_abort, a.err, a.timeout_ns)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
              }
              const uint32_t dreg = tmem + (p == 0 ? 0u : (uint32_t)REG_B);
              const uint32_t ub = ubase + p * D::UCHUNK;
              for (int k = 0; k < S; ++k) {
                const int ni = (S < LV - k) ? S : LV - k;
                for (int ks = 0; ks < 2; ++ks) {
                  const uint64_t ad = smem_desc(wbase + k * D::WDIG + ks * 256, 512);
                  const uint32_t bu = ub + ks * 256;
                  if (k == 1 && ks == 0) {
                    tc_mma(dreg + 32, ad, smem_desc(bu, 512), idesc_bf16(5 * NB), 1);
                    tc_mma(dreg + 32 * 6, ad, smem_desc(bu + 20 * 512, 512), idesc_bf16(NB), 0);
                  } else {
                    tc_mma(dreg + 32 * k, ad, smem_desc(bu, 512), idesc_bf16(ni * NB), (k > 0 || ks > 0) ? 1u : 0u);
                  }
                }
              }
              tc_commit(&bars.c[p]);
              if (o == 0 && t + 1 < nblk) {
                // rows of the next block's new part (the previous sweep must
                // have finished them): two boxes of 16 rows x 128 columns
                // (columns past nev read as zeros)
                const int32_t rn = r0 - NB;
                if (prevflag && wait_released_raw(a.err, a.timeout_ns, prevflag, rn)) {
                  s_abort = 1;
                  ok = false;
                  break;
                }
                mbar_expect_tx(&bars.stage, 2u * WS * STG_ROWS * 8);
                tma_load_2d(smem + D::OFF_STG, &zmap, rn + 1, c0, &bars.stage);
                tma_load_2d(smem + D::OFF_STG + WS * STG_ROWS * 8, &zmap, rn + 1 + STG_ROWS, c0, &bars.stage);
                ++iss_st;
              }
            }
            if (!ok) break;
            // U' is free once GEMM2 is done (the last part issued: 1, or 0 for P = 2)
            if (!mbar_wait(&bars.c[P == 3 ? 1 : 0], n_blk & 1, &s_abort, a.err, a.timeout_ns)) break;
            ++n_blk;
            if (t + 1 < nblk) {
              mbar_expect_tx(&bars.u, D::UBYTES);
              bulk_load(smem + D::OFF_U, blkp + (int64_t)(t + 1) * D::BLOCK_BYTES + D::VBYTES, D::UBYTES, &bars.u);
              ++iss_u;
            }
          }
        }
        __syncwarp();
      } else {
        // -------------------------------------------------------------- math
        constexpr int RT = D::RT;
        const int64_t C = kDigitOffset;
        const bool colok = c0 + col < a.nev;
        const int64_t *zcol = a.z + (int64_t)(c0 + col) * a.ldz + 1;
        int64_t z[RT];  // rows RT * hf .. of my part of the window, offset form
        tc_load_rows<RT>(zcol, r0_of(0) + 32 * grp + RT * hf, g.n, colok, C, z);
        // reflector range of this thread set in the W readout
        const int sub = D::H * grp + hf;
        int ca0, cw0, ca1, cw1;
        if (D::NSUB == 6) {  // 8 / 4 / 4 / 4 / 4 / 8
          ca0 = sub == 0 ? 0 : (sub == 5 ? 24 : 4 + 4 * sub);
          cw0 = (sub == 0 || sub == 5) ? 8 : 4;
          ca1 = 0;
          cw1 = 0;
        } else if (D::NSUB == 4) {  // 8 each
          ca0 = 8 * sub;
          cw0 = 8;
          ca1 = 0;
          cw1 = 0;
        } else if (D::NSUB == 3) {  // 12 / 12 / 8
          ca0 = sub == 0 ? 0 : (sub == 1 ? 12 : 24);
          cw0 = sub == 1 ? 4 : 8;
          ca1 = sub == 0 ? 8 : 16;
          cw1 = sub == 0 ? 4 : (sub == 1 ? 8 : 0);
        } else {  // 16 / 16
          ca0 = 16 * sub;
          cw0 = 8;
          ca1 = 16 * sub + 8;
          cw1 = 8;
        }
        for (int32_t t = 0; t < nblk; ++t) {
          const int32_t r0 = r0_of(t);
          const int p = (grp + t) % P;  // my part of this block's window
          const int prow = 32 * p + RT * hf;  // my first window row
          const int64_t blk = blk0 + t;
          // per-row exponents of U for my rows, and the block's V scale (read now, used late)
          uint32_t gu4[RT / 4];
          int gv;
          {
            const uint4 *gsrc = reinterpret_cast<const uint4 *>(a.slices + blk * (int64_t)D::BLOCK_BYTES + D::VBYTES +
                                                                D::UBYTES + prow);
#pragma unroll
            for (int i = 0; i < RT / 16; ++i) {
              const uint4 gq = __ldg(gsrc + i);
              gu4[4 * i] = gq.x;
              gu4[4 * i + 1] = gq.y;
              gu4[4 * i + 2] = gq.z;
              gu4[4 * i + 3] = gq.w;
            }
            gv = __ldg(a.gvs + blk);
          }
          // ---- digits of Z -> GEMM1 (A operand in tensor memory). The columns
          // are those of the previous block's second product: wait until every
          // thread has read its correction.
          bool ok = true;
          if (n_blk > 0) {
            if (!mbar_wait(&bars.blk, (n_blk - 1) & 1, &s_abort, a.err, a.timeout_ns)) break;
            tc_fence_after();
          }
          // ---- shift of this block's window, per column: the digits take the
          // leading bits of Z 2^zsh, not of Z (Z's fixed point is scaled to the
          // column's norm bound, far above the entries of a delocalised
          // column, whose low bits the digits would drop). zsh keeps every
          // entry below 2^61 (the digits' range) and the window's 1-norm
          // within 2^66, so that W = V'^T Z 2^-64 stays within 2^62 for any
          // reflector (|V'| <= 2^60).
          // Bounds from the high words: Z = z - C has high word h = hi(z) -
          // hi(C) - (borrow 0 or 1), so |Z| < (|hi(z) - hi(C)| + 2) 2^32 =: m 2^32.
          int zsh;
          {
            constexpr int32_t CHI = (int32_t)(kDigitOffset >> 32);
            uint32_t mz = 0, sz = 0;
#pragma unroll
            for (int i = 0; i < RT; ++i) {
              const int32_t h = (int32_t)((uint64_t)z[i] >> 32) - CHI;
              const uint32_t m = (uint32_t)(h < 0 ? -h : h) + 2u;  // < 2^30
              mz = m > mz ? m : mz;
              sz += (m + 31u) >> 5;  // >= m / 32; 96 terms stay below 2^32
            }
            uint32_t *kz = reinterpret_cast<uint32_t *>(smem + D::OFF_KMX);
            kz[sub * WS + col] = mz;
            kz[(D::NSUB + sub) * WS + col] = sz;
            named_sync(1, D::NMATH);
            mz = 0;
            sz = 0;
#pragma unroll
            for (int q = 0; q < D::NSUB; ++q) {
              const uint32_t o = kz[q * WS + col];
              mz = o > mz ? o : mz;
              sz += kz[(D::NSUB + q) * WS + col];
            }
            // every |Z| < 2^(32 + bits(mz)); the 1-norm < sz 2^37 < 2^(37 + bits(sz))
            const int zb = 32 + (32 - __clz((int)mz));
            const int sb = 37 + (32 - __clz((int)sz));
            zsh = min(min(FIX - zb, 66 - sb), 16);  // 16: more gains nothing at the column's scale
            zsh = zsh > 0 ? zsh : 0;
          }
          if (zsh > 0) {
#pragma unroll
            for (int i = 0; i < RT; ++i) z[i] = (int64_t)((uint64_t)(z[i] - C) << zsh) + C;
          }
          {
            const uint32_t zt = tmem + lane_base + ZA_COL + prow / 2;
#pragma unroll
            for (int k = 1; k <= S; ++k) {  // unrolled: the digit helpers take k as a constant
              tmem_z_digit<RT>(k, zt + D::ZCOLS * (k - 1), z);
              tc_wait_st();
              tc_fence_before();
              mbar_arrive(&bars.zfull[k - 1]);
            }
          }
          if (zsh > 0) {  // back to Z (exact: the low zsh bits are zero)
#pragma unroll
            for (int i = 0; i < RT; ++i) z[i] = ((z[i] - C) >> zsh) + C;
          }
          if (!ok) break;
          // ---- W = V'^T Z for my column and my reflector range
          if (!mbar_wait(&bars.g1, n_blk & 1, &s_abort, a.err, a.timeout_ns)) break;
          tc_fence_after();
          constexpr int NW = (D::H == 2) ? 8 : 16;  // W values this thread may hold
          int64_t w[NW];
          const uint32_t wt = tmem + lane_base;
          if (cw0 == 8) w_levels<8>(wt + ca0, w);
          else w_levels<4>(wt + ca0, w);
          if constexpr (NW == 16) {
            if (cw1 == 8) w_levels<8>(wt + ca1, w + 8);
            else if (cw1 == 4) w_levels<4>(wt + ca1, w + 8);
          }
          uint64_t mx = 0;
#pragma unroll
          for (int i = 0; i < NW; ++i) {
            if ((i < 8 && i < cw0) || (i >= 8 && i - 8 < cw1)) {
              const uint64_t ax = (uint64_t)(w[i] < 0 ? -w[i] : w[i]);
              mx = ax > mx ? ax : mx;
            }
          }
          uint64_t *kmx = reinterpret_cast<uint64_t *>(smem + D::OFF_KMX);
          kmx[sub * WS + col] = mx;
          named_sync(1, D::NMATH);
#pragma unroll
          for (int q = 0; q < D::NSUB; ++q) {
            const uint64_t o = kmx[q * WS + col];
            mx = o > mx ? o : mx;
          }
          const int bits = mx ? 64 - __clzll((long long)mx) : 0;
          const int kcol = (bits > 0 && bits < FOP) ? FOP - bits : 0;
          {
            unsigned char *wb = smem + D::OFF_W;
#pragma unroll
            for (int q = 0; q < NW / 8; ++q) {
              const int cw = q ? cw1 : cw0;
              int64_t *wq = w + 8 * q;
#pragma unroll
              for (int i = 0; i < 8; ++i) wq[i] = (int64_t)((uint64_t)wq[i] << kcol) + C;
              const int koff = kmaj(col, q ? ca1 : ca0, NB);
              if (cw == 8) {
                *reinterpret_cast<uint4 *>(wb + 0 * D::WDIG + koff) = digits8<1>(wq);
                *reinterpret_cast<uint4 *>(wb + 1 * D::WDIG + koff) = digits8<2>(wq);
                *reinterpret_cast<uint4 *>(wb + 2 * D::WDIG + koff) = digits8<3>(wq);
                *reinterpret_cast<uint4 *>(wb + 3 * D::WDIG + koff) = digits8<4>(wq);
                *reinterpret_cast<uint4 *>(wb + 4 * D::WDIG + koff) = digits8<5>(wq);
                *reinterpret_cast<uint4 *>(wb + 5 * D::WDIG + koff) = digits8<6>(wq);
              } else if (cw == 4) {
                *reinterpret_cast<uint2 *>(wb + 0 * D::WDIG + koff) = digits4<1>(wq);
                *reinterpret_cast<uint2 *>(wb + 1 * D::WDIG + koff) = digits4<2>(wq);
                *reinterpret_cast<uint2 *>(wb + 2 * D::WDIG + koff) = digits4<3>(wq);
                *reinterpret_cast<uint2 *>(wb + 3 * D::WDIG + koff) = digits4<4>(wq);
                *reinterpret_cast<uint2 *>(wb + 4 * D::WDIG + koff) = digits4<5>(wq);
                *reinterpret_cast<uint2 *>(wb + 5 * D::WDIG + koff) = digits4<6>(wq);
              }
            }
          }
          fence_proxy_async();
          tc_fence_before();
          mbar_arrive(&bars.wfull);
          // ---- corr of my rows: Z -= sum_l B_l 2^(rs + gu[r] - 8 l); levels in
          // pairs (a_l 2^8 + a_(l+1) is exact in 32 bits, |a| < 2^22), then
          // T = P01 2^16 + P23 and T2 = P45 2^8 + a_6 (exact in 64 bits)
          if (!mbar_wait(&bars.c[p], n_blk & 1, &s_abort, a.err, a.timeout_ns)) break;
          tc_fence_after();
          const int rs = 50 + gv - kcol - zsh;
          const uint32_t dreg = tmem + lane_base + (p == 0 ? 0u : (uint32_t)REG_B) + RT * hf;
          constexpr int PR = (RT >= 16) ? 4 : 8;  // rows per piece (register budget)
#pragma unroll
          for (int q = 0; q < RT / PR; ++q) {
            int64_t t1[PR], t2[PR];
            {
              uint32_t ra[PR], rb[PR];
              int32_t p01[PR];
              tmem_ld<PR>(dreg + PR * q, ra);
              tmem_ld<PR>(dreg + 32 + PR * q, rb);
              tc_wait_ld();
#pragma unroll
              for (int i = 0; i < PR; ++i)
                p01[i] = f2i_small(__uint_as_float(ra[i])) * 256 + f2i_small(__uint_as_float(rb[i]));
              tmem_ld<PR>(dreg + 64 + PR * q, ra);
              tmem_ld<PR>(dreg + 96 + PR * q, rb);
              tc_wait_ld();
#pragma unroll
              for (int i = 0; i < PR; ++i)
                t1[i] = (int64_t)((uint64_t)(int64_t)p01[i] << 16) +
                        (f2i_small(__uint_as_float(ra[i])) * 256 + f2i_small(__uint_as_float(rb[i])));
              tmem_ld<PR>(dreg + 128 + PR * q, ra);
              tmem_ld<PR>(dreg + 160 + PR * q, rb);
              tc_wait_ld();
#pragma unroll
              for (int i = 0; i < PR; ++i)
                p01[i] = f2i_small(__uint_as_float(ra[i])) * 256 + f2i_small(__uint_as_float(rb[i]));
              tmem_ld<PR>(dreg + 192 + PR * q, ra);
              tc_wait_ld();
#pragma unroll
              for (int i = 0; i < PR; ++i)
                t2[i] = (int64_t)((uint64_t)(int64_t)p01[i] << 8) + f2i_small(__uint_as_float(ra[i]));
            }
#pragma unroll
            for (int i = 0; i < PR; ++i) {
              const int r = PR * q + i;
              const int sh = rs + (int)(int8_t)(gu4[r >> 2] >> (8 * (r & 3)));
              z[r] -= shl_signed(t1[i], sh - 24) + shl_signed(t2[i], sh - 48);
            }
          }
          tc_fence_before();
          if (P == 3 && p == P - 1) mbar_arrive(&bars.cfree);  // region B is free for part 1
          mbar_arrive(&bars.blk);                                // my reads of this block's products are done
          ++n_blk;
          // ---- the part leaving the window: store it, take the new rows
          if (t + 1 < nblk && p == P - 1) {
            const int32_t rb = r0 + 32 * (P - 1) + RT * hf;
            if (colok) tc_store_rows<RT>(a.z + (int64_t)(c0 + col) * a.ldz + 1, rb, g.n, z, C);
            named_sync(2 + grp, 128 * D::H);  // then one release publishes the group's stores
            if ((warp & 3) == 0 && hf == 0 && lane == 0 && publish) st_release(myflag, rb);
            if (!mbar_wait(&bars.stage, n_st & 1, &s_abort, a.err, a.timeout_ns)) break;
            // 128-byte swizzle: the 16-byte chunk j of column c sits at chunk j ^ (c mod 8)
#pragma unroll
            for (int i2 = 0; i2 < RT / 2; ++i2) {
              const int r = RT * hf + 2 * i2;  // row within the new part (pairs)
              const unsigned char *src = smem + D::OFF_STG + (r >> 4) * (WS * STG_ROWS * 8) + col * 128 +
                                         ((((r & 15) >> 1) ^ (col & 7)) << 4);
              const longlong2 v2 = *reinterpret_cast<const longlong2 *>(src);
              z[2 * i2] = v2.x + C;
              z[2 * i2 + 1] = v2.y + C;
            }
          }
          if (t + 1 < nblk) ++n_st;  // every group counts every staged load
        }
        if (!s_abort) {
          // the whole last window is final
          const int32_t rb = r0_of(nblk - 1) + 32 * ((grp + nblk - 1) % P) + RT * hf;
          if (colok) tc_store_rows<RT>(a.z + (int64_t)(c0 + col) * a.ldz + 1, rb, g.n, z, C);
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (s_abort) break;
    if (tid == 0 && publish) st_release(myflag, r0_of(nblk - 1));
  }
  // drain: no copy or MMA of this block may still be in flight at exit
  if (s_abort && warp == 4 * P * D::H && lane == 0) {
    tc_commit(&bars.drain);
    volatile int never = 0;
    const long long lim = 2000000000LL;
    mbar_wait(&bars.drain, 0, &never, a.err, lim);
    // the last load issued on each barrier has landed once its phase completed
    if (iss_v) mbar_wait(&bars.v, (iss_v - 1) & 1, &never, a.err, lim);
    if (iss_u) mbar_wait(&bars.u, (iss_u - 1) & 1, &never, a.err, lim);
    if (iss_st) mbar_wait(&bars.stage, (iss_st - 1) & 1, &never, a.err, lim);
  }
  if (s_abort && tid == 0 && s_unit < a.units) st_release(a.flags + s_unit, kPoison);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 4 * P * D::H) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS)
                             : "memory");
}

}  // namespace tcs
}  // namespace tbbt
