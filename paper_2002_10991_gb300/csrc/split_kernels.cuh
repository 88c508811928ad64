// Split-precision (Ozaki-style) form of the back-transformation for real
// data: the reflectors of a sweep are blocked nb = 32 at a time into compact
// WY form, Q_blk = H_0 H_1 ... H_{nb-1} = I - V T V^T, and each block is
// applied as Z <- Z - U (V^T Z) with U = V T, two dense contractions done on
// BF16 tensor cores.
//
// Exactness. The eigenvector block is held in 64-bit fixed point per column:
// Zi = round(z * 2^(61 - e_c)) with ||x_c||_2 <= 2^e_c; the reflectors are
// unitary, so |z| <= ||x_c|| and |Zi| <= 2^61 for the whole run. V (scaled by
// 2^-gv per block) and U (2^-gu) are fixed point with the same 2^61 scale. A
// fixed-point value X is split into S signed digits,
//     X ~ sum_{j=1..S} d_j 2^(61 - 8 j),  |d_1| <= 256, |d_j| <= 128,
// each exact in BF16. A digit product is exact in FP32 (<= 2^16); the sum of
// all pairs (i, j) of one level l = i + j over K <= 96 stays below 2^24 (see
// split_level_bound), so every level accumulates exactly in FP32 whatever the
// summation order of the tensor core. Levels are combined in 64-bit integer
// arithmetic and the update Zi -= corr is an integer subtraction: no FP64
// operation on the hot path. Pairs with i + j > S + 2 are dropped: the lower
// digits are full-size, so the first dropped level is about 2^-8 of the last
// kept one, and keeping level S + 2 puts it below the digit truncation.
//
// T and U are computed per plan in FP64 (forward recurrence of compact WY:
// T_mm = tau_m, T[0:m, m] = -tau_m T[0:m, 0:m] (V[:, 0:m]^T v_m)).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "apply_kernels.cuh"

namespace tbbt {
namespace split {

constexpr int NB = 32;      // reflectors per WY block
constexpr int S = 6;        // digit slices per operand
constexpr int LV = S + 1;   // levels kept: l = i + j in [2, S + 2] (pairs of 1-based digit indices)
constexpr int WS = 64;      // columns per strip (8 warps x 8 columns)
constexpr int NWARPS = 8;
constexpr int ZLD = 66;     // row stride of the shared-memory ring (int64 elements; padded)
constexpr int FIX = 61;     // fixed-point scale exponent of |x| <= 1
constexpr int WSHIFT = 4;   // headroom of W_int: W = 2^(gv - F + WSHIFT) W_int

// Slice tiles are stored with padded rows (8 extra bf16 = 16 bytes) so that
// the 8 rows an ldmatrix reads fall in disjoint shared-memory bank groups
// (row strides of 208/144/80 bytes instead of 192/128/64).
template <int B>
struct Dims {
  static constexpr int R = B + NB - 1;             // window rows of one block
  static constexpr int RP = (R + 15) / 16 * 16;    // padded to the MMA K step
  static constexpr int KT = RP / 16;               // K steps of the first product
  static constexpr int MT = RP / 16;               // M tiles of the second product
  static constexpr int LD1 = RP + 8;               // row stride of a V' slice [m][r]
  static constexpr int LD2 = NB + 8;               // row stride of a U' slice [r][m]
  static constexpr int SLICE1 = NB * LD1;          // bf16 elements of one V' slice
  static constexpr int SLICE2 = RP * LD2;          // bf16 elements of one U' slice
  static constexpr int ROWSC = (RP + 15) / 16 * 16 / 2;  // bf16-sized room for RP int8 row scales of U
  static constexpr int PART1 = S * SLICE1;         // V' slices of a block
  static constexpr int PART2 = S * SLICE2 + ROWSC; // U' slices and row scales
  static constexpr int BLOCK_ELEMS = PART1 + PART2;
};

// 2^gv >= max |V| of the block; U is scaled per row (int8 exponents stored
// after the block's slices) so that small rows keep their precision.
struct BlockScale {
  int32_t gv, gu_unused;
};

// Largest |sum| of one level of digit products over K terms (for the
// exactness argument: must stay below 2^24).
constexpr long long split_level_bound(int K, int level) {
  long long s = 0;
  for (int i = 1; i <= S; ++i) {
    int j = level - i;
    if (j < 1 || j > S) continue;
    s += (long long)(i == 1 ? 256 : 128) * (j == 1 ? 256 : 128);
  }
  return s * K;
}

__device__ __forceinline__ int64_t round_shift(int64_t x, int sh) {
  return (x + ((int64_t)1 << (sh - 1))) >> sh;  // round(x / 2^sh), arithmetic shift
}
__device__ __forceinline__ int64_t shift_signed(int64_t x, int sh) { return sh >= 0 ? (x << sh) : (x >> (-sh)); }

// Digit j (1-based) of a fixed-point value, peeled from the running remainder.
__device__ __forceinline__ int32_t peel_digit(int64_t &rem, int j) {
  const int sh = FIX - 8 * j;
  int64_t d = round_shift(rem, sh);
  rem -= d << sh;
  return (int32_t)d;
}

__device__ __forceinline__ uint32_t pack_bf16x2(int32_t lo, int32_t hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn((float)lo, (float)hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// ---------------------------------------------------------------------------
// per-plan preparation: T, U = V T (FP64), scales, digit slices
// ---------------------------------------------------------------------------
// Block id -> (sweep j, step t) through block_start[j] (first block of sweep j).
template <int B>
__global__ void __launch_bounds__(128) wy_prepare_kernel(const double *__restrict__ vstore, StoreGeom g, int32_t ldv,
                                                         const int64_t *__restrict__ block_start, int32_t J,
                                                         int64_t nblocks, __nv_bfloat16 *__restrict__ slices,
                                                         BlockScale *__restrict__ scales) {
  using D = Dims<B>;
  __shared__ double sV[D::RP][NB + 1];  // V, later overwritten by U = V T
  __shared__ double sT[NB][NB + 1];
  __shared__ double sy[NB];
  __shared__ double stau[NB];
  __shared__ double sred[4];
  const int64_t blk = blockIdx.x;
  if (blk >= nblocks) return;
  int32_t lo = 0, hi = J - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (block_start[mid] <= blk) lo = mid;
    else hi = mid - 1;
  }
  const int32_t j = lo;
  const int32_t t = (int32_t)(blk - block_start[j]);
  const int32_t s_hi = g.imax(j) - t * NB;
  const int32_t s_lo = s_hi - NB + 1 > 0 ? s_hi - NB + 1 : 0;
  const int32_t cnt = s_hi - s_lo + 1;
  const int tid = threadIdx.x;
  // V: column m = stage s_lo + m, occupying window rows m .. m + L - 1
  for (int idx = tid; idx < D::RP * NB; idx += blockDim.x) {
    int r = idx / NB, m = idx - r * NB;
    double val = 0.0;
    if (m < cnt) {
      const int32_t s = s_lo + m;
      const int32_t L = g.len(s, j);
      const int tt = r - m;
      if (tt == 0) val = 1.0;
      else if (tt > 0 && tt < L) val = vstore[(g.sweep_offset(j) + (g.imax(j) - s)) * ldv + tt];
    }
    sV[r][m] = val;
  }
  for (int m = tid; m < NB; m += blockDim.x)
    stau[m] = m < cnt ? vstore[(g.sweep_offset(j) + (g.imax(j) - (s_lo + m))) * ldv] : 0.0;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) sT[idx / NB][idx % NB] = 0.0;
  __syncthreads();
  // forward recurrence of compact WY (product order H_0 H_1 ... H_{cnt-1},
  // H_m of stage s_lo + m; the highest stage acts first)
  for (int m = 0; m < cnt; ++m) {
    for (int k = tid; k < m; k += blockDim.x) {
      double acc = 0.0;
      for (int r = 0; r < D::RP; ++r) acc += sV[r][k] * sV[r][m];
      sy[k] = acc;
    }
    __syncthreads();
    for (int k = tid; k < m; k += blockDim.x) {
      double acc = 0.0;
      for (int l = k; l < m; ++l) acc += sT[k][l] * sy[l];
      sT[k][m] = -stau[m] * acc;
    }
    if (tid == 0) sT[m][m] = stau[m];
    __syncthreads();
  }
  auto block_max_exp = [&](bool of_v) -> int {
    double mx = 0.0;
    for (int idx = tid; idx < D::RP * NB; idx += blockDim.x) mx = fmax(mx, fabs(sV[idx / NB][idx % NB]));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) sred[tid >> 5] = mx;
    __syncthreads();
    mx = fmax(fmax(sred[0], sred[1]), fmax(sred[2], sred[3]));
    __syncthreads();
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx <= 2^e
    (void)of_v;
    return e;
  };
  __nv_bfloat16 *out = slices + blk * D::BLOCK_ELEMS;
  // digit slices of V' = V 2^-gv, as A1 = [m][r] (NB x RP)
  const int gv = block_max_exp(true);
  for (int idx = tid; idx < D::RP * NB; idx += blockDim.x) {
    int m = idx / D::RP, r = idx - m * D::RP;
    int64_t x = __double2ll_rn(ldexp(sV[r][m], FIX - gv));
    for (int sl = 1; sl <= S; ++sl) out[(sl - 1) * D::SLICE1 + m * D::LD1 + r] = __float2bfloat16_rn((float)peel_digit(x, sl));
  }
  __syncthreads();
  // U = V T in place: row r, columns from the last down (column m needs V[r][0..m])
  for (int r = tid; r < D::RP; r += blockDim.x)
    for (int m = NB - 1; m >= 0; --m) {
      double acc = 0.0;
      for (int k = 0; k <= m; ++k) acc += sV[r][k] * sT[k][m];
      sV[r][m] = acc;
    }
  __syncthreads();
  // digit slices of U' = U 2^-gu[r] per row, as A2 = [r][m] (RP x NB)
  __shared__ int sgu[D::RP];
  int8_t *rowsc = reinterpret_cast<int8_t *>(out + D::PART1 + S * D::SLICE2);
  for (int r = tid; r < D::RP; r += blockDim.x) {
    double mx = 0.0;
    for (int m = 0; m < NB; ++m) mx = fmax(mx, fabs(sV[r][m]));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    sgu[r] = e;
    rowsc[r] = (int8_t)e;
  }
  __syncthreads();
  for (int idx = tid; idx < D::RP * NB; idx += blockDim.x) {
    int r = idx / NB, m = idx - r * NB;
    int64_t x = __double2ll_rn(ldexp(sV[r][m], FIX - sgu[r]));
    for (int sl = 1; sl <= S; ++sl)
      out[D::PART1 + (sl - 1) * D::SLICE2 + r * D::LD2 + m] = __float2bfloat16_rn((float)peel_digit(x, sl));
  }
  if (tid == 0) scales[blk] = BlockScale{gv, 0};
}

// ---------------------------------------------------------------------------
// fixed point <-> FP64 of the eigenvector block (in place, column scales)
// ---------------------------------------------------------------------------
// One warp per column: e_c with ||x_c||_2 <= 2^e_c, then Zi = round(x 2^(FIX - e_c)).
__global__ void to_fixed_kernel(double *q, int64_t ldq, int32_t n, int32_t nev, int32_t *col_exp) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nev) return;
  double *col = q + c * ldq;
  double ss = 0.0;
  for (int32_t r = lane; r < n; r += 32) ss = fma(col[r], col[r], ss);
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  int e = 0;
  if (ss > 0.0) frexp(sqrt(ss), &e);
  if (lane == 0) col_exp[c] = e;
  int64_t *ci = reinterpret_cast<int64_t *>(col);
  for (int32_t r = lane; r < n; r += 32) ci[r] = __double2ll_rn(ldexp(col[r], FIX - e));
}

__global__ void from_fixed_kernel(double *q, int64_t ldq, int32_t n, int32_t nev, const int32_t *col_exp) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nev) return;
  double *col = q + c * ldq;
  const int64_t *ci = reinterpret_cast<const int64_t *>(col);
  const int e = col_exp[c];
  for (int32_t r = lane; r < n; r += 32) col[r] = ldexp(__ll2double_rn(ci[r]), e - FIX);
}

// ---------------------------------------------------------------------------
// the split-precision apply kernel (warp-level BF16 tensor-core MMA)
// ---------------------------------------------------------------------------
struct SplitArgs {
  int64_t *q;  // fixed-point view of the eigenvector block
  int64_t ldq;
  StoreGeom g;
  int32_t nev;
  int32_t strips;  // ceil(nev / WS)
  int32_t units;   // strips * sweeps
  int32_t ring;    // rows of the shared-memory ring
  const __nv_bfloat16 *slices;
  const BlockScale *scales;
  const int64_t *block_start;  // per sweep
  int *flags;
  unsigned *counter;
  int *err;
  long long timeout_ns;
};

// Not volatile: a pure function of its operands, so the compiler may
// interleave independent accumulations to hide the MMA latency.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *smem_row_addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(smem_row_addr)));
}

__device__ __forceinline__ uint32_t movmatrix_trans(uint32_t x) {
  uint32_t y;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;\n" : "=r"(y) : "r"(x));
  return y;
}

// A fragment of a 16x16 tile of a row-major bf16 matrix in shared memory
// (row stride ld elements) at (row0, col0).
__device__ __forceinline__ void load_a_frag(uint32_t (&a)[4], const __nv_bfloat16 *base, int ld, int row0, int col0,
                                            int lane) {
  const int q = lane >> 3;           // which 8x8 matrix this lane addresses
  const int r = row0 + ((q & 1) << 3) + (lane & 7);
  const int c = col0 + ((q >> 1) << 3);
  ldmatrix_x4(a, base + r * ld + c);
}

// Work unit = (strip of WS columns, sweep j); units of consecutive sweeps of a
// strip are chained exactly as the epochs of the FP64 kernel (one sweep per
// epoch, one WY block per step). Per step the 8 warps apply the block to
// their 8 columns each: GEMM1 W = V'^T Z (B fragments are digits of the
// fixed-point window), integer combine, digits of W (transposed into B
// fragments with movmatrix), GEMM2 corr = U' W, integer update of the window.
template <int B>
__global__ void __launch_bounds__(NWARPS * 32, 1) split_apply_kernel(SplitArgs a) {
  using D = Dims<B>;
  constexpr int KT = D::KT;          // k steps of GEMM1 (window rows / 16)
  constexpr int MT1 = NB / 16;       // m tiles of GEMM1 (reflectors / 16) = k steps of GEMM2
  constexpr int CH = (D::MT + 1) / 2;  // m tiles of GEMM2 per chunk (two chunks)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_unit;
  __shared__ int s_stop;
  int64_t *ring = reinterpret_cast<int64_t *>(smem_raw);
  __nv_bfloat16 *sA1 = reinterpret_cast<__nv_bfloat16 *>(ring + (int64_t)a.ring * ZLD);
  __nv_bfloat16 *sA2 = sA1 + D::PART1;
  const int8_t *sGu = reinterpret_cast<const int8_t *>(sA2 + S * D::SLICE2);  // U row exponents
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const StoreGeom &g = a.g;
  const int cw = warp * 8;  // this warp's first column within the strip
  const int bcol = cw + (lane >> 2);         // strip column of this lane's B fragments (GEMM1)
  const int ccol = cw + 2 * (lane & 3);      // first strip column of this lane's C fragments

  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = (int)atomicAdd(a.counter, 1u);
      s_stop = (*(volatile int *)a.err != 0);
    }
    __syncthreads();
    const int u = s_unit;
    if (u >= a.units || s_stop) break;
    const int32_t j = u / a.strips;  // one sweep per unit
    const int32_t c0 = (u - j * a.strips) * WS;
    int *myflag = a.flags + u;
    const int *prevflag = j > 0 ? a.flags + (u - a.strips) : nullptr;
    const Epoch ep = make_epoch(g, j, 1, NB);
    const int64_t blk0 = a.block_start[j];

    auto slot = [&](int32_t r, int c) -> int64_t { return (int64_t)(r % a.ring) * ZLD + c; };
    auto copy_slices = [&](__nv_bfloat16 *dst, int64_t blk, int part, bool doit) {
      if (doit) {
        const __nv_bfloat16 *src = a.slices + blk * D::BLOCK_ELEMS + part * D::PART1;
        const int nchunks = (part ? D::PART2 : D::PART1) * 2 / 16;  // U part carries its row scales
        for (int cidx = threadIdx.x; cidx < nchunks; cidx += blockDim.x)
          cp_async<16>(reinterpret_cast<char *>(dst) + 16 * cidx, reinterpret_cast<const char *>(src) + 16 * cidx);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    auto store_rows = [&](int32_t r0, int32_t r1) {
      const int32_t nrows = r1 - r0;
      for (int32_t idx = threadIdx.x; idx < nrows * WS; idx += blockDim.x) {
        int32_t c = idx / nrows, r = r0 + (idx - c * nrows);
        int32_t col = c0 + c;
        if (col < a.nev) a.q[(int64_t)col * a.ldq + r] = ring[slot(r, c)];
      }
    };

    int32_t top = step_min_row(g, ep, 0);
    if (threadIdx.x == 0) s_stop = prevflag ? wait_released_raw(a.err, a.timeout_ns, prevflag, top) : 0;
    __syncthreads();
    bool abandoned = s_stop != 0;
    if (!abandoned) {
      // prologue: rows of step 0 (L2 path: written by another SM) and the slices of block 0
      {
        const int32_t nrows = g.n - top;
        for (int32_t idx = threadIdx.x; idx < nrows * WS; idx += blockDim.x) {
          int32_t c = idx / nrows, r = top + (idx - c * nrows);
          int32_t col = c0 + c;
          ring[slot(r, c)] = col < a.nev ? (int64_t)__ldcg((const long long *)(a.q + (int64_t)col * a.ldq + r)) : 0;
        }
      }
      copy_slices(sA1, blk0, 0, true);
      copy_slices(sA2, blk0, 1, true);
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
      int32_t released = g.n;
      for (int32_t t = 0; t < ep.nsteps; ++t) {
        const int32_t s_hi = ep.sig_top - t * NB;
        const int32_t s_lo = s_hi - NB + 1 > 0 ? s_hi - NB + 1 : 0;
        const int32_t r0 = g.row(s_lo, j);
        const int32_t rmax = min(s_hi + j * g.b + g.b, g.n - 1);  // last row this block touches
        const BlockScale sc = a.scales[blk0 + t];
        // rows no block of this sweep touches from step t on go back to global memory
        const int32_t live = rows_live_max(g, ep, t);
        const int32_t rel = live + 1 > top ? live + 1 : top;
        if (rel < released) {
          store_rows(rel, released);
          released = rel;
        }
        const int32_t ntop = step_min_row(g, ep, t + 1);
        if (threadIdx.x == 0)
          s_stop = (prevflag && ntop < top) ? wait_released_raw(a.err, a.timeout_ns, prevflag, ntop) : 0;
        __syncthreads();
        if (s_stop) {
          abandoned = true;
          break;
        }
        if (threadIdx.x == 0) st_release(myflag, released);
        // rows of the next step: issue the loads now, store them after the arithmetic
        int64_t pfv[NB * WS / (NWARPS * 32)];
        {
          const int32_t nrows = top - ntop;
#pragma unroll
          for (int i = 0; i < NB * WS / (NWARPS * 32); ++i) {
            int32_t idx = threadIdx.x + i * blockDim.x;
            if (nrows > 0 && idx < nrows * WS) {
              int32_t c = idx / nrows, r = ntop + (idx - c * nrows);
              int32_t col = c0 + c;
              pfv[i] = col < a.nev ? (int64_t)__ldcg((const long long *)(a.q + (int64_t)col * a.ldq + r)) : 0;
            }
          }
        }

        // ---------------- GEMM1: W = V'^T Z (levels exact in FP32) ----------------
        uint32_t bz[S][KT][2];
        {
          int64_t rem[KT][4];
#pragma unroll
          for (int kt = 0; kt < KT; ++kt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int32_t r = r0 + 16 * kt + 2 * (lane & 3) + (e & 1) + ((e >> 1) << 3);
              rem[kt][e] = (r <= rmax) ? ring[slot(r, bcol)] : 0;
            }
#pragma unroll
          for (int sl = 0; sl < S; ++sl)
#pragma unroll
            for (int kt = 0; kt < KT; ++kt) {
              int32_t d0 = peel_digit(rem[kt][0], sl + 1), d1 = peel_digit(rem[kt][1], sl + 1);
              int32_t d2 = peel_digit(rem[kt][2], sl + 1), d3 = peel_digit(rem[kt][3], sl + 1);
              bz[sl][kt][0] = pack_bf16x2(d0, d1);
              bz[sl][kt][1] = pack_bf16x2(d2, d3);
            }
        }
        float acc1[LV][MT1][4];
#pragma unroll
        for (int l = 0; l < LV; ++l)
#pragma unroll
          for (int mt = 0; mt < MT1; ++mt) acc1[l][mt][0] = acc1[l][mt][1] = acc1[l][mt][2] = acc1[l][mt][3] = 0.f;
#pragma unroll
        for (int i = 0; i < S; ++i) {
          uint32_t af[MT1][KT][4];
#pragma unroll
          for (int mt = 0; mt < MT1; ++mt)
#pragma unroll
            for (int kt = 0; kt < KT; ++kt) load_a_frag(af[mt][kt], sA1 + i * D::SLICE1, D::LD1, 16 * mt, 16 * kt, lane);
          // K steps outermost: the (level, m tile) accumulators of one K step are independent
#pragma unroll
          for (int kt = 0; kt < KT; ++kt)
#pragma unroll
            for (int jj = 0; jj < S && i + jj < LV; ++jj)  // level i + jj (0-based)
#pragma unroll
              for (int mt = 0; mt < MT1; ++mt) mma_bf16(acc1[i + jj][mt], af[mt][kt], bz[jj][kt][0], bz[jj][kt][1]);
        }
        __syncthreads();  // every warp is done with the V' slices
        copy_slices(sA1, blk0 + t + 1, 0, t + 1 < ep.nsteps);

        // ---------------- integer combine, digits of W as GEMM2 B fragments ----------------
        // W is normalized per column (shifted left by kcol so its largest entry
        // fills the 2^61 fixed-point range) before it is split, so its digits
        // keep 48 bits relative to the column's own magnitude; the shift is
        // undone in the combine of GEMM2. The 32 entries of column
        // cw + 2 (lane & 3) + p sit in the 8 lanes sharing lane & 3.
        uint32_t bw[S][MT1][2];
        int kcol[2];
        {
          int64_t w[MT1][4];
#pragma unroll
          for (int mt = 0; mt < MT1; ++mt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              int64_t x = 0;
#pragma unroll
              for (int l = 0; l < LV; ++l) x += shift_signed((int64_t)(int32_t)acc1[l][mt][e], 41 - 8 * l);
              w[mt][e] = x;
            }
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            uint64_t mx = 0;
#pragma unroll
            for (int mt = 0; mt < MT1; ++mt)
#pragma unroll
              for (int e = p; e < 4; e += 2) {
                const int64_t x = w[mt][e];
                const uint64_t ax = (uint64_t)(x < 0 ? -x : x);
                mx = ax > mx ? ax : mx;
              }
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
              const uint64_t other = __shfl_xor_sync(0xffffffffu, mx, o);
              mx = other > mx ? other : mx;
            }
            const int bits = mx ? 64 - __clzll((long long)mx) : 0;
            kcol[p] = bits > 0 && bits < FIX ? FIX - bits : 0;
#pragma unroll
            for (int mt = 0; mt < MT1; ++mt)
#pragma unroll
              for (int e = p; e < 4; e += 2) w[mt][e] <<= kcol[p];
          }
#pragma unroll
          for (int sl = 0; sl < S; ++sl)
#pragma unroll
            for (int mt = 0; mt < MT1; ++mt) {
              int32_t d0 = peel_digit(w[mt][0], sl + 1), d1 = peel_digit(w[mt][1], sl + 1);
              int32_t d2 = peel_digit(w[mt][2], sl + 1), d3 = peel_digit(w[mt][3], sl + 1);
              bw[sl][mt][0] = movmatrix_trans(pack_bf16x2(d0, d1));
              bw[sl][mt][1] = movmatrix_trans(pack_bf16x2(d2, d3));
            }
        }
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this block's U' slices
        __syncthreads();

        // ---------------- GEMM2: corr = U' W, window -= corr ----------------
        const int cshift = 49 + sc.gv;  // + the row exponent of U
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          float acc2[LV][CH][4];
#pragma unroll
          for (int l = 0; l < LV; ++l)
#pragma unroll
            for (int mt = 0; mt < CH; ++mt) acc2[l][mt][0] = acc2[l][mt][1] = acc2[l][mt][2] = acc2[l][mt][3] = 0.f;
#pragma unroll
          for (int i = 0; i < S; ++i) {
            uint32_t af[CH][MT1][4];
#pragma unroll
            for (int mt = 0; mt < CH; ++mt)
#pragma unroll
              for (int kt = 0; kt < MT1; ++kt) {
                const int row0 = 16 * (ch * CH + mt);
                if (row0 < D::RP) load_a_frag(af[mt][kt], sA2 + i * D::SLICE2, D::LD2, row0, 16 * kt, lane);
              }
#pragma unroll
            for (int kt = 0; kt < MT1; ++kt)
#pragma unroll
              for (int jj = 0; jj < S && i + jj < LV; ++jj)
#pragma unroll
                for (int mt = 0; mt < CH; ++mt)
                  if (16 * (ch * CH + mt) < D::RP) mma_bf16(acc2[i + jj][mt], af[mt][kt], bw[jj][kt][0], bw[jj][kt][1]);
          }
#pragma unroll
          for (int mt = 0; mt < CH; ++mt) {
            if (16 * (ch * CH + mt) >= D::RP) continue;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int32_t r = r0 + 16 * (ch * CH + mt) + (lane >> 2) + ((e >> 1) << 3);
              if (r > rmax) continue;
              const int rs = cshift + sGu[16 * (ch * CH + mt) + (lane >> 2) + ((e >> 1) << 3)] - kcol[e & 1];
              int64_t corr = 0;
#pragma unroll
              for (int l = 0; l < LV; ++l) corr += shift_signed((int64_t)(int32_t)acc2[l][mt][e], rs - 8 * l);
              ring[slot(r, ccol + (e & 1))] -= corr;
            }
          }
        }
        __syncthreads();  // every warp is done with the U' slices and the window
        copy_slices(sA2, blk0 + t + 1, 1, t + 1 < ep.nsteps);
        {
          const int32_t nrows = top - ntop;
#pragma unroll
          for (int i = 0; i < NB * WS / (NWARPS * 32); ++i) {
            int32_t idx = threadIdx.x + i * blockDim.x;
            if (nrows > 0 && idx < nrows * WS) {
              int32_t c = idx / nrows, r = ntop + (idx - c * nrows);
              ring[slot(r, c)] = pfv[i];
            }
          }
        }
        top = ntop;
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // the next block's V' slices
        __syncthreads();
      }
      if (!abandoned) {
        store_rows(top, released);
        __syncthreads();
        if (threadIdx.x == 0) st_release(myflag, top);
      }
    }
    if (abandoned) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      if (threadIdx.x == 0) st_release(myflag, kPoison);
    }
    __syncthreads();
  }
}

}  // namespace split
}  // namespace tbbt
