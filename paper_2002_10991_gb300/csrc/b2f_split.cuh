// Split-precision form of the band -> full back-transformation (Eq. 6e) on
// the fifth-generation tensor cores, real data.
//
// The WY blocks of b2f.cuh, H_{32p} ... H_{32p+31} = I - V T V^T, are applied
// last-first as Y <- Y - U (V^T Y) with U = V T, by the exact digit-slice
// products of the tcgen05 form of Eq. 6d (tc_split.cuh): Y in 64-bit fixed
// point per column, V', U' and W in 6 balanced 8-bit digits on BF16 tensor
// cores, every digit product and level sum exact in FP32, levels combined
// in 64-bit integers.
//
// Unlike Eq. 6d's short reflectors, a block's reflectors run over all rows
// c + b .. n - 1, so W = V^T Y is a contraction over up to n rows. It is cut
// into batches of 96 rows (three 32-row tiles; a level stays exact for K <=
// 96), each batch's levels read out and summed into 64-bit integers. The
// rows are dealt to S_K CTAs per 128-column strip by interleaved tiles
// (tile t belongs to slot t mod S_K), so that every CTA reads and updates
// only its own tiles of Y, block after block: no exchange of Y between CTAs.
// Per block the slots publish their partial W in global memory (one buffer
// per slot and block parity), count themselves in on the block's counter,
// and every slot sums all partials once the counter says they are there
// (bounded wait); then each slot normalises W, splits it into digits and
// applies the update to its tiles. The counters are per block: a slot with
// no rows in block p skips it, so it may publish block p - 1 before block p
// is complete, and a counter shared across blocks would count that too.
//
// Per batch a CTA (24 math warps: three 32-row parts x two 16-row halves x
// 128 columns, one producer warp) runs, as the tcgen05 Eq. 6d kernel does
// per window:
//   pass A: rows -> per-column shift -> digits in tensor memory -> GEMM1
//           (levels of W^T = Y^T V') -> levels read out and accumulated;
//   pass C: GEMM2 per part (corr^T = W^T U'^T) -> corrections read out and
//           subtracted from the rows, which go back to global memory.
// The V' / U' digit slices of every (block, slot, batch) are prepared per
// call in FP64 (T and U = V T) by bfs_prepare_kernel, in the operand layouts
// of tc_split.cuh (96 K-rows of V', three 32-row parts of U'); the T factors
// come from Gram matrices summed over 512-row chunks (bfs_gram_kernel,
// bfs_tfactor_kernel). The fixed-point copy of Y is row-major, so that a
// warp's 32 columns of one row are 256 consecutive bytes.
#pragma once

#include "b2f.cuh"
#include "tc_split.cuh"

namespace tbbt {
namespace bfs {

using namespace tbbt::tcs;
using D = Geo<64>;  // RP = 96 rows per batch, P = 3 parts, 800 threads; the layouts only, not b

// One (block, slot, batch) of the prepared operands.
struct Item {
  int32_t p, k, beta, pad;
};

struct Layout {
  int32_t n, b, K1, P;   // P: WY blocks of 32 reflectors
  int32_t ntiles;        // 32-row tiles of Y
  int32_t SK;            // CTAs (slots) per strip
};

// First tile of block p (its rows start at 32 p + b) and the tiles slot k owns.
__host__ __device__ inline int32_t first_tile_of(const Layout &L, int32_t p) { return (32 * p + L.b) / 32; }
__host__ __device__ inline int32_t slot_first(const Layout &L, int32_t p, int32_t k) {
  const int32_t t0 = first_tile_of(L, p);
  return t0 + (((k - t0) % L.SK) + L.SK) % L.SK;
}
__host__ __device__ inline int32_t slot_count(const Layout &L, int32_t p, int32_t k) {
  const int32_t f = slot_first(L, p, k);
  return f < L.ntiles ? (L.ntiles - 1 - f) / L.SK + 1 : 0;
}
__host__ __device__ inline int32_t slot_batches(const Layout &L, int32_t p, int32_t k) {
  return (slot_count(L, p, k) + 2) / 3;
}

// T factors, balanced over the SMs. The Gram matrix G = V^T V of WY block p
// runs over rows 32 p + b .. n - 1; on one thread block (as in b2f.cuh) the
// first blocks' 32 x 32 x n FP64 products would each hold one SM's FP64 pipe
// for the whole step. Here every chunk of GCH rows of a block is a thread
// block of its own that writes its partial G to its own slot, and
// bfs_tfactor_kernel sums a block's partials in chunk order (so the result
// does not depend on scheduling), then runs the forward recurrence of the WY
// representation: T_kk = tau_k, T[0:k, k] = -tau_k T[0:k, 0:k] G[0:k, k].
// It also gives gv[p]: every reflector of block p has norm sqrt(G_kk) below
// 2^gv (a margin of 2^-40 covers the rounding of G_kk), so V' = V 2^(60 - gv)
// has every entry, and by Cauchy-Schwarz every partial W, in range.
constexpr int GCH = 512;  // rows per Gram chunk

__global__ void __launch_bounds__(256) bfs_gram_kernel(bf::Geo g, const int2 *__restrict__ pieces,
                                                       double *__restrict__ gpart) {
  constexpr int RC = 64;
  __shared__ double Vs[RC][NB + 1];
  const int2 pc = pieces[blockIdx.x];  // (block p, first row)
  const int p = pc.x, tid = threadIdx.x;
  const int k = tid % NB, l0 = tid / NB;  // owns G[k][l0 + 8 i]
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int32_t rend = min(pc.y + GCH, g.n);
  for (int32_t r0 = pc.y; r0 < rend; r0 += RC) {
#pragma unroll
    for (int i = 0; i < RC * NB / 256; ++i) {
      const int e = tid + 256 * i;
      const int r = e % RC, t = e / RC;
      Vs[r][t] = r0 + r < rend ? bf::vget<double>(g, r0 + r, p, t) : 0.0;
    }
    __syncthreads();
    for (int r = 0; r < RC; ++r) {
      const double vk = Vs[r][k];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fma(vk, Vs[r][l0 + 8 * i], acc[i]);
    }
    __syncthreads();
  }
  double *out = gpart + (int64_t)blockIdx.x * NB * NB;
#pragma unroll
  for (int i = 0; i < 4; ++i) out[k * NB + l0 + 8 * i] = acc[i];
}

__global__ void __launch_bounds__(256) bfs_tfactor_kernel(bf::Geo g, const double *__restrict__ gpart,
                                                          const int32_t *__restrict__ chunk_base,
                                                          double *__restrict__ Tws, int32_t *__restrict__ gvs) {
  __shared__ double Gs[NB][NB + 1];
  __shared__ double Ts[NB][NB + 1];
  const int p = blockIdx.x, tid = threadIdx.x;
  const int k = tid % NB, l0 = tid / NB;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int32_t j = chunk_base[p]; j < chunk_base[p + 1]; ++j) {
    const double *src = gpart + (int64_t)j * NB * NB + k * NB + l0;
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] += src[8 * i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) Gs[k][l0 + 8 * i] = acc[i];
  __syncthreads();
  if (tid < NB) {
    double mx = sqrt(fmax(Gs[tid][tid], 0.0));
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx * (1.0 + 0x1p-40), &e);
    if (tid == 0) gvs[p] = e;
    const int i = tid;
    const double *tau = reinterpret_cast<const double *>(g.tau);
    for (int kk = 0; kk < NB; ++kk) {
      const int32_t c = NB * p + kk;
      const double tk = c < g.K1 ? tau[c] : 0.0;
      double val = 0.0;
      if (i < kk) {
        double sum = 0.0;
        for (int l = i; l < kk; ++l) sum = fma(Ts[i][l], Gs[l][kk], sum);
        val = -(tk * sum);
      } else if (i == kk) {
        val = tk;
      }
      Ts[i][kk] = val;
      __syncwarp();
    }
    for (int kk = 0; kk < NB; ++kk) Tws[(int64_t)p * NB * NB + i + NB * kk] = Ts[i][kk];
  }
}

// The digit slices of one (block, slot, batch): V' (96 rows x 32 reflectors,
// K-major for GEMM1's B operand) and U' = (V T)' (three 32-row parts for
// GEMM2's B operand, per-row scales) in the byte layout of tc_split.cuh.
// One block of 128 threads per item.
__global__ void __launch_bounds__(128) bfs_prepare_kernel(bf::Geo g, Layout L, const Item *__restrict__ items,
                                                          const double *__restrict__ Tws,
                                                          const int32_t *__restrict__ gvs,
                                                          unsigned char *__restrict__ slices) {
  constexpr int RP = D::RP;
  __shared__ double sV[RP][NB + 1];  // V, later U = V T
  __shared__ double sT[NB][NB + 1];
  __shared__ int sgu[RP];
  const Item it = items[blockIdx.x];
  const int tid = threadIdx.x;
  const int32_t f = slot_first(L, it.p, it.k), cnt = slot_count(L, it.p, it.k);
  for (int idx = tid; idx < RP * NB; idx += blockDim.x) {
    const int m = idx / RP, rr = idx - m * RP;
    const int part = rr / 32, j = 3 * it.beta + part;
    double val = 0.0;
    if (j < cnt) {
      const int32_t row = 32 * (f + j * L.SK) + (rr & 31);
      if (row < L.n) val = bf::vget<double>(g, row, it.p, m);
    }
    sV[rr][m] = val;
  }
  for (int idx = tid; idx < NB * NB; idx += blockDim.x)
    sT[idx % NB][idx / NB] = Tws[(int64_t)it.p * NB * NB + idx];  // T(i, kk) at i + NB kk
  __syncthreads();
  const int gv = gvs[it.p];
  unsigned char *out = slices + (int64_t)blockIdx.x * D::BLOCK_BYTES;
  // V' = V 2^(60 - gv)
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
  // U = V T (T upper triangular)
  {
    constexpr int PER = RP * NB / 128;
    double u[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int idx = tid + 128 * i;
      const int r = idx / NB, m = idx - r * NB;
      double acc = 0.0;
      for (int kk = 0; kk <= m; ++kk) acc = fma(sV[r][kk], sT[kk][m], acc);
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
  // U' = U 2^(60 - gu[r]) per row, |U[r][:]| < 2^gu[r]
  int8_t *rowexp = reinterpret_cast<int8_t *>(out + D::VBYTES + D::UBYTES);
  for (int r = tid; r < RP; r += blockDim.x) {
    uint64_t m2 = 0;
    for (int m = 0; m < NB; ++m) {
      const uint64_t a = abs_bits(sV[r][m]);
      m2 = a > m2 ? a : m2;
    }
    int e = exp_of_bits(m2);
    e = e < -64 ? -64 : (e > 100 ? 100 : e);
    sgu[r] = e;
    rowexp[r] = (int8_t)e;
  }
  for (int r = RP + tid; r < D::EBYTES; r += blockDim.x) rowexp[r] = 0;
  __syncthreads();
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
}

// Shared memory of the apply kernel: W's digits (GEMM2's A operand), two
// buffers each of V' and U' (the next batch's operands load during the
// current batch's products), the partial maxima of the column exchanges.
constexpr int SM_W = 0;
constexpr int SM_V = SM_W + S * D::WDIG;
constexpr int SM_U = SM_V + 2 * D::VBYTES;
constexpr int SM_KMX = SM_U + 2 * D::UBYTES;
constexpr int SM_BYTES = SM_KMX + 2 * D::NSUB * WS * 8 + 1024;  // + room to align the base to 1024 bytes
static_assert(SM_BYTES <= 227 * 1024, "shared memory of the split band -> full kernel");

// The fixed-point Y is row-major (row r of the strip's 128 columns is 1 KB
// of consecutive memory), so that the 32 lanes of a warp, which hold 32
// consecutive columns, read and write 256 consecutive bytes per row. (With
// the caller's column-major layout every lane would touch its own cache
// line on each access.)
// 16 rows of one column (rows >= n and invalid tiles read as zero), plus `add`
__device__ __forceinline__ void load_rows16(const int64_t *zc, int64_t ldc, int32_t rb, int32_t n, bool valid,
                                            int64_t add, int64_t (&z)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int32_t r = rb + i;
    z[i] = (valid && r < n) ? (int64_t)__ldcg((const long long *)(zc + (int64_t)r * ldc)) + add : add;
  }
}
__device__ __forceinline__ void store_rows16(int64_t *zc, int64_t ldc, int32_t rb, int32_t n, const int64_t (&z)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i)
    if (rb + i < n) __stcg((long long *)(zc + (int64_t)(rb + i) * ldc), (long long)z[i]);
}

// q (column-major, n x nev) <-> the row-major fixed-point Y: Z(r, c) =
// round(q(r, c) 2^(FIX - e_c)), e_c the exponent of column c's norm (as
// tcs::to_fixed_kernel). 32 x 32 tiles through shared memory, so that both
// sides are read and written along their contiguous dimension.
__global__ void __launch_bounds__(256) bfs_colexp_kernel(const double *__restrict__ q, int64_t ldq, int32_t n,
                                                         int32_t nev, int32_t *__restrict__ col_exp) {
  const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= nev) return;
  const double *col = q + c * ldq;
  double ss = 0.0;
  for (int32_t r = lane; r < n; r += 32) ss = fma(col[r], col[r], ss);
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  int e = 0;
  if (ss > 0.0) frexp(sqrt(ss), &e);
  if (lane == 0) col_exp[c] = e;
}
__global__ void __launch_bounds__(256) bfs_to_fixed_kernel(const double *__restrict__ q, int64_t ldq,
                                                           int64_t *__restrict__ z, int64_t ldc, int32_t n,
                                                           int32_t nev, const int32_t *__restrict__ col_exp) {
  __shared__ int64_t t[32][33];
  const int32_t r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int32_t c = c0 + ty + 8 * j, r = r0 + tx;
    if (c < nev && r < n) t[ty + 8 * j][tx] = __double2ll_rn(ldexp(q[(int64_t)c * ldq + r], FIX - col_exp[c]));
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int32_t r = r0 + ty + 8 * j, c = c0 + tx;
    if (c < nev && r < n) z[(int64_t)r * ldc + c] = t[tx][ty + 8 * j];
  }
}
__global__ void __launch_bounds__(256) bfs_from_fixed_kernel(double *__restrict__ q, int64_t ldq,
                                                             const int64_t *__restrict__ z, int64_t ldc, int32_t n,
                                                             int32_t nev, const int32_t *__restrict__ col_exp) {
  __shared__ int64_t t[32][33];
  const int32_t r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int32_t r = r0 + ty + 8 * j, c = c0 + tx;
    if (c < nev && r < n) t[tx][ty + 8 * j] = z[(int64_t)r * ldc + c];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int32_t c = c0 + ty + 8 * j, r = r0 + tx;
    if (c < nev && r < n) q[(int64_t)c * ldq + r] = ldexp(__ll2double_rn(t[ty + 8 * j][tx]), col_exp[c] - FIX);
  }
}

struct BfsArgs {
  int64_t *z;  // fixed-point Y, row-major: row r, column c at r * ldc + c
  int64_t ldc;
  Layout L;
  int32_t nev, strips;
  const unsigned char *slices;   // items x BLOCK_BYTES
  const int32_t *gv;             // per WY block
  const int32_t *item_base;      // per (p, k): index of its first item
  const int32_t *need;           // per p: slots with rows in block p
  int64_t *wpart;                // [strips][2][SK][NB][WS]: partial W per block parity and slot
  unsigned *wcnt;                // [strips][P]: partial W of the block published so far
  int *err;
  long long timeout_ns;
  int32_t withhold;  // test hook: CTA whose W publications are not counted (-1: none)
};

struct BfsBarriers {
  uint64_t zfull[S], blk, g1, wfull, c[3], cfree, v[2], u[2], drain;
};

// Levels of W = V'^T Z for C consecutive reflectors of this thread's column
// (as tc_split.cuh's w_levels, one level at a time: fewer live registers),
// at the batch's shift zsh, rounded back to the unshifted scale and added to
// acc[0], acc[WS], ... (the block's sums in shared memory).
template <int C>
__device__ __forceinline__ void w_levels_acc(uint32_t taddr, int zsh, int64_t *acc) {
  int64_t w[C];
#pragma unroll
  for (int l = 0; l < LV; ++l) {
    uint32_t r[C];
    if constexpr (C == 8) tmem_ld8(taddr + 32 * l, r);
    else tmem_ld4(taddr + 32 * l, r);
    tc_wait_ld();
#pragma unroll
    for (int i = 0; i < C; ++i) {
      const int32_t v = __float2int_rn(__uint_as_float(r[i]));  // |v| < 2^24: exact
      if (l == 0) w[i] = v;
      else if (l < LV - 1) w[i] = shl8_add(w[i], v);
      else w[i] = (int64_t)((uint64_t)w[i] << 2) + (v >> 6);  // 4 h + floor(a_6 / 64)
    }
  }
#pragma unroll
  for (int i = 0; i < C; ++i) acc[i * WS] += zsh > 0 ? ((w[i] + ((int64_t)1 << (zsh - 1))) >> zsh) : w[i];
}

__global__ void __launch_bounds__(D::NTHREADS, 1) bfs_apply_kernel(BfsArgs a) {
  constexpr int P = D::P;
  constexpr int RT = D::RT;
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char *const smem = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  __shared__ BfsBarriers bars;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_stop;  // s_abort as every thread saw it at the last block boundary
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool producer = warp == 4 * P * D::H;
  const int grp = warp / (4 * D::H);       // math group = part of the batch
  const int hf = (warp >> 2) % D::H;       // which 16 rows of the part
  const int col = (warp & 3) * 32 + lane;  // strip column = TMEM lane
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const Layout &L = a.L;
  const int SK = L.SK;

  if (producer) {
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
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars.v[b], 1);
      mbar_init(&bars.u[b], 1);
    }
    mbar_init(&bars.drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_abort = 0;
    s_stop = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  // completed phases each role waits for (both roles count batches alike)
  uint32_t n_batch = 0;  // batches (pass A and pass C) completed: blk
  uint32_t n_a = 0;      // pass-A batches: zfull, g1
  uint32_t n_c = 0;      // pass-C batches: c[*], cfree
  uint32_t n_w = 0;      // blocks: wfull
  // operand loads: batch i of a pass (counted over the whole launch) uses
  // buffer i & 1 and is the (i >> 1)-th load into it
  uint32_t iss_v[2] = {0, 0}, iss_u[2] = {0, 0};  // loads issued per buffer (for the drain)
  bool pre_v = false;  // V' of the block's first batch is already on its way
  const int slot = blockIdx.x % SK;
  const int rounds_stride = gridDim.x / SK;

  for (int strip = blockIdx.x / SK; strip < a.strips; strip += rounds_stride) {
    const int32_t c0 = strip * WS;
    for (int32_t p = L.P - 1; p >= 0; --p) {
      const int32_t nbat = slot_batches(L, p, slot);
      const int32_t f = slot_first(L, p, slot);
      const int32_t cnt = slot_count(L, p, slot);
      const int64_t ib = a.item_base[p * SK + slot];
      const unsigned char *items0 = a.slices + ib * (int64_t)D::BLOCK_BYTES;
      if (producer) {
        if (lane == 0) {
          // ----------------------------------------------------------- producer
          const uint32_t wbase = smem_u32(smem + SM_W);
          auto load_v = [&](uint32_t i, int32_t bt, const unsigned char *it0) {
            const int bf = i & 1;
            mbar_expect_tx(&bars.v[bf], D::VBYTES);
            bulk_load(smem + SM_V + bf * D::VBYTES, it0 + (int64_t)bt * D::BLOCK_BYTES, D::VBYTES, &bars.v[bf]);
            ++iss_v[bf];
          };
          auto load_u = [&](uint32_t i, int32_t bt, const unsigned char *it0) {
            const int bf = i & 1;
            mbar_expect_tx(&bars.u[bf], D::UBYTES);
            bulk_load(smem + SM_U + bf * D::UBYTES, it0 + (int64_t)bt * D::BLOCK_BYTES + D::VBYTES, D::UBYTES,
                      &bars.u[bf]);
            ++iss_u[bf];
          };
          bool ok = true;
          // U' of this block's first pass-C batch: its buffer is free (every
          // earlier GEMM2 is complete)
          if (nbat > 0) load_u(n_c, 0, items0);
          // pass A: GEMM1 per batch
          for (int32_t bt = 0; bt < nbat && ok; ++bt) {
            if (bt == 0 && !pre_v) load_v(n_a, 0, items0);
            pre_v = false;
            // the other buffer's GEMM1 (batch n_a - 1) is complete
            if (bt + 1 < nbat) load_v(n_a + 1, bt + 1, items0);
            if (!mbar_wait(&bars.v[n_a & 1], (n_a >> 1) & 1, &s_abort, a.err, a.timeout_ns)) { ok = false; break; }
            const uint32_t vbase = smem_u32(smem + SM_V + (n_a & 1) * D::VBYTES);
            for (int k = 0; k < S; ++k) {
              if (!mbar_wait(&bars.zfull[k], n_a & 1, &s_abort, a.err, a.timeout_ns)) { ok = false; break; }
              tc_fence_after();
              const int ni = (S < LV - k) ? S : LV - k;
              const uint32_t za = tmem + ZA_COL + D::ZCOLS * k;
              for (int ks = 0; ks < D::KS1; ++ks) {
                const uint32_t bv = vbase + ks * 256;
                if (k == 1 && ks == 0) {
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
            if (!mbar_wait(&bars.g1, n_a & 1, &s_abort, a.err, a.timeout_ns)) { ok = false; break; }
            ++n_a;
            ++n_batch;
          }
          // V' of the next block's first batch: both buffers are free now
          if (ok && p > 0 && slot_batches(L, p - 1, slot) > 0) {
            load_v(n_a, 0, a.slices + (int64_t)a.item_base[(p - 1) * SK + slot] * D::BLOCK_BYTES);
            pre_v = true;
          }
          // pass C: GEMM2 per batch and part (part 0 -> region A, 1 -> region B,
          // 2 -> region A once part 0 is read)
          for (int32_t bt = 0; bt < nbat && ok; ++bt) {
            // the other buffer's GEMM2 (batch n_c - 1) is complete
            if (bt + 1 < nbat) load_u(n_c + 1, bt + 1, items0);
            if (!mbar_wait(&bars.u[n_c & 1], (n_c >> 1) & 1, &s_abort, a.err, a.timeout_ns)) { ok = false; break; }
            if (bt == 0 && !mbar_wait(&bars.wfull, n_w & 1, &s_abort, a.err, a.timeout_ns)) { ok = false; break; }
            // every thread read the previous batch's accumulators
            if (n_batch > 0 && !mbar_wait(&bars.blk, (n_batch - 1) & 1, &s_abort, a.err, a.timeout_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ubase = smem_u32(smem + SM_U + (n_c & 1) * D::UBYTES);
            for (int part = 0; part < P && ok; ++part) {
              if (part == 2) {
                if (!mbar_wait(&bars.cfree, n_c & 1, &s_abort, a.err, a.timeout_ns)) { ok = false; break; }
                tc_fence_after();
              }
              const uint32_t dreg = tmem + (part == 1 ? (uint32_t)REG_B : 0u);
              const uint32_t ub = ubase + part * D::UCHUNK;
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
              tc_commit(&bars.c[part]);
            }
            if (!ok) break;
            // U' is free once the last part's products are done
            if (!mbar_wait(&bars.c[2], n_c & 1, &s_abort, a.err, a.timeout_ns)) { ok = false; break; }
            ++n_c;
            ++n_batch;
          }
          if (ok && nbat > 0) ++n_w;
          if (!ok) s_abort = 1;
        }
        __syncwarp();
      } else {
        // --------------------------------------------------------------- math
        const int64_t C = kDigitOffset;
        const bool colok = c0 + col < a.nev;
        int64_t *const zcol = a.z + (c0 + col);
        const int sub = D::H * grp + hf;
        // reflector range of this thread set in the W readout (8 / 4 / 4 / 4 / 4 / 8)
        const int ca0 = sub == 0 ? 0 : (sub == 5 ? 24 : 4 + 4 * sub);
        const int cw0 = (sub == 0 || sub == 5) ? 8 : 4;
        // rows of my part of batch bt: tile f + (3 bt + grp) SK, rows RT hf ..
        auto my_row0 = [&](int32_t bt) -> int32_t {
          const int32_t j = 3 * bt + grp;
          return j < cnt ? 32 * (f + j * SK) + RT * hf : -1;
        };
        // the block's W sums of my column and reflectors, in the W-digit
        // buffer (free during pass A: the previous block's GEMM2 is complete
        // once the first blk wait below returns); entry (m, col) at m WS + col
        int64_t *const wacc = reinterpret_cast<int64_t *>(smem + SM_W) + ca0 * WS + col;
        // Every math thread runs the same sequence of named barriers whatever
        // happens: after an abort (ok false) the work is skipped, not the
        // barriers, so no warp is left waiting at one.
        bool ok = !s_abort;
        // ---- pass A (the next batch's rows load while this batch's GEMM1 runs)
        int64_t z[RT];
        if (nbat > 0) {
          const int32_t rb = my_row0(0);
          load_rows16(zcol, a.ldc, rb, L.n, ok && rb >= 0 && colok, C, z);
        }
        for (int32_t bt = 0; bt < nbat; ++bt) {
          if (ok && n_batch > 0) {
            ok = mbar_wait(&bars.blk, (n_batch - 1) & 1, &s_abort, a.err, a.timeout_ns);
            tc_fence_after();
          }
          if (bt == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (i < cw0) wacc[i * WS] = 0;
          }
          // per-column shift of this batch (as the Eq. 6d kernel's per window):
          // every entry below 2^61 and the batch's 1-norm within 2^66
          int zsh;
          {
            constexpr int32_t CHI = (int32_t)(kDigitOffset >> 32);
            uint32_t mz = 0, sz = 0;
#pragma unroll
            for (int i = 0; i < RT; ++i) {
              const int32_t h = (int32_t)((uint64_t)z[i] >> 32) - CHI;
              const uint32_t m = (uint32_t)(h < 0 ? -h : h) + 2u;
              mz = m > mz ? m : mz;
              sz += (m + 31u) >> 5;
            }
            uint32_t *kz = reinterpret_cast<uint32_t *>(smem + SM_KMX);
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
            const int zb = 32 + (32 - __clz((int)mz));
            const int sb = 37 + (32 - __clz((int)sz));
            zsh = min(min(FIX - zb, 66 - sb), 16);
            zsh = zsh > 0 ? zsh : 0;
          }
          if (ok) {
            if (zsh > 0) {
#pragma unroll
              for (int i = 0; i < RT; ++i) z[i] = (int64_t)((uint64_t)(z[i] - C) << zsh) + C;
            }
            const uint32_t zt = tmem + lane_base + ZA_COL + (32 * grp + RT * hf) / 2;
#pragma unroll
            for (int k = 1; k <= S; ++k) {
              tmem_z_digit<RT>(k, zt + D::ZCOLS * (k - 1), z);
              tc_wait_st();
              tc_fence_before();
              mbar_arrive(&bars.zfull[k - 1]);
            }
          }
          if (bt + 1 < nbat) {
            const int32_t rb = my_row0(bt + 1);
            load_rows16(zcol, a.ldc, rb, L.n, ok && rb >= 0 && colok, C, z);
          }
          if (ok) ok = mbar_wait(&bars.g1, n_a & 1, &s_abort, a.err, a.timeout_ns);
          if (ok) {
            tc_fence_after();
            // this batch's W levels, back to the unshifted scale, into the block's sum
            const uint32_t wt = tmem + lane_base;
            if (cw0 == 8) w_levels_acc<8>(wt + ca0, zsh, wacc);
            else w_levels_acc<4>(wt + ca0, zsh, wacc);
            tc_fence_before();
            mbar_arrive(&bars.blk);
          }
          ++n_a;
          ++n_batch;
        }
        if (nbat > 0) {
          // ---- this slot's partial W -> global memory; count it in on the
          // block's counter; wait (bounded) until every slot with rows in the
          // block has. Buffer parity: a slot writes block p - 2's partial only
          // after every slot with rows in p - 1 (a superset of those in p)
          // published p - 1, which each did after reading block p's.
          int64_t *wp = a.wpart + ((((int64_t)strip * 2 + (p & 1)) * SK) * NB) * WS;
          if (ok) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (i < cw0) __stcg((long long *)(wp + ((int64_t)slot * NB + ca0 + i) * WS + col), (long long)wacc[i * WS]);
          }
          named_sync(1, D::NMATH);
          if (tid == 0) {
            if (s_abort) {
              atomicCAS(a.err, 0, 4 /* TBBT_ETIMEOUT */);  // the other slots stop waiting for this one
            } else {
              unsigned *cnt_p = a.wcnt + (int64_t)strip * L.P + p;
              __threadfence();
              if ((int32_t)blockIdx.x != a.withhold) atomicAdd(cnt_p, 1u);
              const unsigned need = (unsigned)a.need[p];
              const long long t0 = globaltimer_ns();
              for (unsigned itr = 0;; ++itr) {
                unsigned v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(cnt_p) : "memory");
                if (v >= need) break;
                if (*(volatile int *)a.err != 0) { s_abort = 1; break; }
                if (globaltimer_ns() - t0 > a.timeout_ns) {
                  atomicCAS(a.err, 0, 4 /* TBBT_ETIMEOUT */);
                  s_abort = 1;
                  break;
                }
                __nanosleep(itr < 64 ? 64 : 256);
              }
            }
          }
          named_sync(1, D::NMATH);
          ok = ok && !s_abort;
          // ---- the block's W: sum of the partials, normalised per column,
          // split into digits -> the A operand of GEMM2 (as tc_split.cuh)
          // slots with rows in this block: tile t0 .. ntiles - 1 belongs to slot t mod S_K
          const int32_t t0b = first_tile_of(L, p);
          unsigned act = 0;
          for (int kk = 0; kk < SK; ++kk)
            if ((((kk - t0b) % SK) + SK) % SK < L.ntiles - t0b) act |= 1u << kk;
          int64_t w[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) w[i] = 0;
          if (ok) {
#pragma unroll 1
            for (int kk = 0; kk < SK; ++kk)
              if ((act >> kk) & 1u) {
                const int64_t *src = wp + ((int64_t)kk * NB + ca0) * WS + col;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                  if (i < cw0) w[i] += (int64_t)__ldcg((const long long *)(src + (int64_t)i * WS));
              }
          }
          uint64_t mx = 0;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint64_t ax = (uint64_t)(w[i] < 0 ? -w[i] : w[i]);
            mx = ax > mx ? ax : mx;
          }
          uint64_t *kmx = reinterpret_cast<uint64_t *>(smem + SM_KMX);
          kmx[sub * WS + col] = mx;
          named_sync(1, D::NMATH);
#pragma unroll
          for (int q = 0; q < D::NSUB; ++q) {
            const uint64_t o = kmx[q * WS + col];
            mx = o > mx ? o : mx;
          }
          const int bits = mx ? 64 - __clzll((long long)mx) : 0;
          const int kcol = (bits > 0 && bits < FOP) ? FOP - bits : 0;
          if (ok) {
            unsigned char *wb = smem + SM_W;
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = (int64_t)((uint64_t)w[i] << kcol) + C;
            const int koff = kmaj(col, ca0, NB);
            if (cw0 == 8) {
              *reinterpret_cast<uint4 *>(wb + 0 * D::WDIG + koff) = digits8<1>(w);
              *reinterpret_cast<uint4 *>(wb + 1 * D::WDIG + koff) = digits8<2>(w);
              *reinterpret_cast<uint4 *>(wb + 2 * D::WDIG + koff) = digits8<3>(w);
              *reinterpret_cast<uint4 *>(wb + 3 * D::WDIG + koff) = digits8<4>(w);
              *reinterpret_cast<uint4 *>(wb + 4 * D::WDIG + koff) = digits8<5>(w);
              *reinterpret_cast<uint4 *>(wb + 5 * D::WDIG + koff) = digits8<6>(w);
            } else {
              *reinterpret_cast<uint2 *>(wb + 0 * D::WDIG + koff) = digits4<1>(w);
              *reinterpret_cast<uint2 *>(wb + 1 * D::WDIG + koff) = digits4<2>(w);
              *reinterpret_cast<uint2 *>(wb + 2 * D::WDIG + koff) = digits4<3>(w);
              *reinterpret_cast<uint2 *>(wb + 3 * D::WDIG + koff) = digits4<4>(w);
              *reinterpret_cast<uint2 *>(wb + 4 * D::WDIG + koff) = digits4<5>(w);
              *reinterpret_cast<uint2 *>(wb + 5 * D::WDIG + koff) = digits4<6>(w);
            }
            fence_proxy_async();
            tc_fence_before();
            mbar_arrive(&bars.wfull);
          }
          ++n_w;
          // W is at the unshifted scale of Y: no batch shift in the exponent
          const int rs = 50 + a.gv[p] - kcol;
          // ---- pass C: corr of my rows, Z -= sum_l B_l 2^(rs + gu[r] - 8 l)
          for (int32_t bt = 0; bt < nbat && ok; ++bt) {
            const int32_t rb = my_row0(bt);
            load_rows16(zcol, a.ldc, rb, L.n, rb >= 0 && colok, 0, z);
            uint32_t gu4[RT / 4];
            {
              const uint4 *gsrc = reinterpret_cast<const uint4 *>(items0 + (int64_t)bt * D::BLOCK_BYTES + D::VBYTES +
                                                                  D::UBYTES + 32 * grp + RT * hf);
#pragma unroll
              for (int i = 0; i < RT / 16; ++i) {
                const uint4 gq = __ldg(gsrc + i);
                gu4[4 * i] = gq.x;
                gu4[4 * i + 1] = gq.y;
                gu4[4 * i + 2] = gq.z;
                gu4[4 * i + 3] = gq.w;
              }
            }
            if (!mbar_wait(&bars.c[grp], n_c & 1, &s_abort, a.err, a.timeout_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dreg = tmem + lane_base + (grp == 1 ? (uint32_t)REG_B : 0u) + RT * hf;
            constexpr int PR = 4;
#pragma unroll
            for (int q = 0; q < RT / PR; ++q) {
              int64_t t1[PR], t2[PR];
              {
                uint32_t ra[PR], rb2[PR];
                int32_t p01[PR];
                tmem_ld<PR>(dreg + PR * q, ra);
                tmem_ld<PR>(dreg + 32 + PR * q, rb2);
                tc_wait_ld();
#pragma unroll
                for (int i = 0; i < PR; ++i)
                  p01[i] = f2i_small(__uint_as_float(ra[i])) * 256 + f2i_small(__uint_as_float(rb2[i]));
                tmem_ld<PR>(dreg + 64 + PR * q, ra);
                tmem_ld<PR>(dreg + 96 + PR * q, rb2);
                tc_wait_ld();
#pragma unroll
                for (int i = 0; i < PR; ++i)
                  t1[i] = (int64_t)((uint64_t)(int64_t)p01[i] << 16) +
                          (f2i_small(__uint_as_float(ra[i])) * 256 + f2i_small(__uint_as_float(rb2[i])));
                tmem_ld<PR>(dreg + 128 + PR * q, ra);
                tmem_ld<PR>(dreg + 160 + PR * q, rb2);
                tc_wait_ld();
#pragma unroll
                for (int i = 0; i < PR; ++i)
                  p01[i] = f2i_small(__uint_as_float(ra[i])) * 256 + f2i_small(__uint_as_float(rb2[i]));
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
            if (grp == 0) mbar_arrive(&bars.cfree);  // region A is free for part 2
            mbar_arrive(&bars.blk);
            if (rb >= 0 && colok) store_rows16(zcol, a.ldc, rb, L.n, z);
            ++n_c;
            ++n_batch;
          }
        }
        if (!ok) s_abort = 1;
      }
      // The next block's rows of this slot are the same tiles (tile t belongs
      // to slot t mod S_K for every block), though a tile may move to another
      // thread; the barrier orders its stores before those loads.
      tc_fence_before();
      __syncthreads();
      if (tid == 0) s_stop = s_abort;
      __syncthreads();
      tc_fence_after();
      if (s_stop) break;
    }
    if (s_stop) break;
  }
  // drain: no copy or MMA of this block may still be in flight at exit
  if (s_stop && producer && lane == 0) {
    tc_commit(&bars.drain);
    volatile int never = 0;
    const long long lim = 2000000000LL;
    mbar_wait(&bars.drain, 0, &never, a.err, lim);
    for (int b = 0; b < 2; ++b) {  // the last load issued into each buffer has landed
      if (iss_v[b]) mbar_wait(&bars.v[b], (iss_v[b] - 1) & 1, &never, a.err, lim);
      if (iss_u[b]) mbar_wait(&bars.u[b], (iss_u[b] - 1) & 1, &never, a.err, lim);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (producer)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace bfs
}  // namespace tbbt
