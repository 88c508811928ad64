// Band -> full back-transformation of eigenvectors (Eq. 6e, Sec. 2.1):
// C = P^* Y = Q1 Y with Q1 = H_0 H_1 ... H_{K1-1} the reflectors of the
// full -> band reduction (Eq. 6a), one per column c = 0 .. n-b-1, acting on
// rows c+b .. n-1.
//
// Reflector store (LAPACK layout, as the full -> band step leaves it): the
// n x n column-major matrix `a` holds reflector c's v[0] = 1 implicitly at
// row c+b and v[1:] in a[c+b+1 : n, c]; tau[c]. Entries at or above the b-th
// sub-diagonal are not read.
//
// Unlike Eq. 6d (short reflectors on a sliding window) this step is dense:
// 32 consecutive reflectors form one WY block H_{c0} ... H_{c0+31} =
// I - V T V^H (V staircase, T upper triangular, built by the forward
// recurrence in FP64). Blocks are applied last-first. FP64 on GB300 runs at
// 2 DFMA per clock per SM, two orders of magnitude below shared-memory and
// L2 rates, so the kernel is FP64-pipe bound once the pipe is kept fed:
//   * one thread block per strip of <= 16 columns of Y (whole column
//     quads), grid sized to the SMs x resident blocks, applies every block
//     to its strip; strips of balanced quad counts keep each SM's FP64 pipe
//     equally loaded, and the four warps of a block split the rows so that
//     each sub-partition's pipe gets the same share;
//   * one pass over the rows per block boundary: the rows of a 64-row chunk
//     (32 for complex) get the update of block p+1, Y -= V_{p+1} W_{p+1},
//     and then feed W_p += V_p^H Y of the next block, so Y is read and
//     written once per block, not three times;
//   * the next chunk's Y and V are loaded into registers while the current
//     chunk is computed.
#pragma once

#include <stdint.h>

namespace tbbt {
namespace bf {

constexpr int NB = 32;        // reflectors per WY block
constexpr int THREADS = 256;  // threads of the T-factor kernel
constexpr int PADT = NB + 1;  // padded row length of t-major tiles

template <typename T>
struct Ops;

template <>
struct Ops<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ void mac(double &s, double x, double y) { s = fma(x, y, s); }
  static __device__ __forceinline__ void macc(double &s, double x, double y) { s = fma(x, y, s); }  // conj(x) y
  static __device__ __forceinline__ void msub(double &s, double x, double y) { s = fma(-x, y, s); }
  static __device__ __forceinline__ double neg_mul(double x, double y) { return -(x * y); }
  static __device__ __forceinline__ double ldro(const double *p) { return __ldg(p); }
  static __device__ __forceinline__ double add(double x, double y) { return x + y; }
};

template <>
struct Ops<zdouble> {
  static __device__ __forceinline__ zdouble zero() { return zdouble{0.0, 0.0}; }
  static __device__ __forceinline__ zdouble one() { return zdouble{1.0, 0.0}; }
  static __device__ __forceinline__ void mac(zdouble &s, zdouble x, zdouble y) {
    s.re = fma(x.re, y.re, s.re);
    s.re = fma(-x.im, y.im, s.re);
    s.im = fma(x.re, y.im, s.im);
    s.im = fma(x.im, y.re, s.im);
  }
  static __device__ __forceinline__ void macc(zdouble &s, zdouble x, zdouble y) {
    s.re = fma(x.re, y.re, s.re);
    s.re = fma(x.im, y.im, s.re);
    s.im = fma(x.re, y.im, s.im);
    s.im = fma(-x.im, y.re, s.im);
  }
  static __device__ __forceinline__ void msub(zdouble &s, zdouble x, zdouble y) {
    s.re = fma(-x.re, y.re, s.re);
    s.re = fma(x.im, y.im, s.re);
    s.im = fma(-x.re, y.im, s.im);
    s.im = fma(-x.im, y.re, s.im);
  }
  static __device__ __forceinline__ zdouble neg_mul(zdouble x, zdouble y) {
    return zdouble{-(x.re * y.re - x.im * y.im), -(x.re * y.im + x.im * y.re)};
  }
  static __device__ __forceinline__ zdouble add(zdouble x, zdouble y) { return zdouble{x.re + y.re, x.im + y.im}; }
  static __device__ __forceinline__ zdouble ldro(const zdouble *p) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return zdouble{v.x, v.y};
  }
};

struct Geo {
  const void *a;
  int64_t lda;
  const void *tau;
  int32_t n, b, K1, P;  // P = ceil(K1 / NB) blocks
};

// Entry (r, t) of the staircase V of block p: reflector c = NB p + t.
template <typename T>
__device__ __forceinline__ T vget(const Geo &g, int32_t r, int32_t p, int32_t t) {
  const int32_t c = NB * p + t;
  if (c >= g.K1 || r >= g.n) return Ops<T>::zero();
  const int32_t rr = r - (c + g.b);
  if (rr < 0) return Ops<T>::zero();
  if (rr == 0) return Ops<T>::one();
  return Ops<T>::ldro(reinterpret_cast<const T *>(g.a) + (int64_t)c * g.lda + r);
}

// T factor of every block (one thread block each): G = V^H V over the
// block's rows, then T_kk = tau_k, T[0:k, k] = -tau_k T[0:k, 0:k] G[0:k, k]
// (the forward recurrence of the WY representation). Tws: P x NB x NB,
// column-major per block.
template <typename T>
__global__ void __launch_bounds__(THREADS) bf_tfactor_kernel(Geo g, T *__restrict__ Tws) {
  constexpr int RC = sizeof(T) == 16 ? 32 : 64;  // static shared memory stays below 48 KB
  __shared__ T Vs[RC][PADT];
  __shared__ T Gs[NB][PADT];
  T(*Ts)[PADT] = Vs;  // the T factor reuses the V tile once G is complete
  const int p = blockIdx.x;
  const int tid = threadIdx.x;
  const int k = tid % NB, l0 = tid / NB;  // owns G[k][l0 + 8 i]
  T acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = Ops<T>::zero();
  const int32_t rs = NB * p + g.b;
  for (int32_t r0 = rs; r0 < g.n; r0 += RC) {
#pragma unroll
    for (int i = 0; i < RC * NB / THREADS; ++i) {
      const int e = tid + THREADS * i;
      const int r = e % RC, t = e / RC;
      Vs[r][t] = vget<T>(g, r0 + r, p, t);
    }
    __syncthreads();
    for (int r = 0; r < RC; ++r) {
      const T vk = Vs[r][k];
#pragma unroll
      for (int i = 0; i < 4; ++i) Ops<T>::macc(acc[i], vk, Vs[r][l0 + 8 * i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) Gs[k][l0 + 8 * i] = acc[i];  // G[k][l] = v_k^H v_l
  __syncthreads();
  if (tid < NB) {
    const int i = tid;
    const T *tau = reinterpret_cast<const T *>(g.tau);
    for (int kk = 0; kk < NB; ++kk) {
      const int32_t c = NB * p + kk;
      const T tk = c < g.K1 ? tau[c] : Ops<T>::zero();
      T val = Ops<T>::zero();
      if (i < kk) {
        T s = Ops<T>::zero();
        for (int l = i; l < kk; ++l) Ops<T>::mac(s, Ts[i][l], Gs[l][kk]);
        val = Ops<T>::neg_mul(tk, s);
      } else if (i == kk) {
        val = tk;
      }
      Ts[i][kk] = val;
      __syncwarp();
    }
    for (int kk = 0; kk < NB; ++kk) Tws[(int64_t)p * NB * NB + i + NB * kk] = Ts[i][kk];
  }
}

struct ApplyArgs {
  Geo g;
  const void *Tws;
  void *q;
  int64_t ldq;
  int32_t nev;
  int32_t base, extra;  // block i takes base + (i < extra) column quads
};

// Apply kernel geometry: 4 warps; a strip is 1 .. 4 column quads. Warp k
// takes rows 16k .. 16k+15 of every 64-row chunk (8k .. 8k+7 of a 32-row
// complex chunk) for all of the strip's quads, so the four warps, one per
// SM sub-partition, carry equal FP64 work whatever the strip width, and no
// DFMA is issued for a column the strip does not have. Within a warp,
// lane = 8 * (column in quad) + row (or reflector) group.
constexpr int ATHREADS = 128;
constexpr int AW = 16;  // columns per strip at most (4 quads)

template <typename T, int RC>
struct Smem {
  T Zs[AW][RC + 2];  // Y chunk, column-major, padded: the 4 columns of a quad in distinct banks
  T Vu[NB][RC];      // V of the updating block, t-major
  T Va[RC][PADT];    // V of the accumulating block, r-major
  T Wu[NB][AW + 1];  // T_u V_u^H Y of the updating block
  T Wt[NB][AW + 1];  // V_a^H Y of the accumulating block, before T (summed over the warps)
  T Ts[NB][PADT];    // T of the accumulating block
};

template <typename T, int RC>
__global__ void __launch_bounds__(ATHREADS, sizeof(T) == 16 ? 2 : (RC == 32 ? 4 : 3)) bf_apply_kernel(ApplyArgs A) {
  constexpr int RW = RC / 4;                    // rows per warp per chunk
  constexpr int RPT = RW / 8;                   // update rows per lane
  constexpr int NZ = AW * RW / 32;              // Y elements loaded per lane per chunk
  constexpr int NV = NB * RW / 32;              // V elements loaded per lane per chunk and block
  constexpr int LPR = 32 / RW;                  // lanes per row index in the loads
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T, RC> &S = *reinterpret_cast<Smem<T, RC> *>(smem_raw);
  const Geo &g = A.g;
  const int tid = threadIdx.x;
  // The blocks with one quad more are the first ones, which the block
  // scheduler spreads over distinct SMs before it places a second block on
  // any SM.
  const int32_t bi = (int32_t)blockIdx.x;
  const int32_t q0 = bi * A.base + min(bi, A.extra);
  const int nq = A.base + (bi < A.extra ? 1 : 0);  // 1 .. 4, uniform in the block
  const int32_t q1 = q0 + nq;
  const int32_t j0 = 4 * q0;
  const int32_t w = min(4 * q1, A.nev) - j0;  // 1 .. 16
  T *__restrict__ q = reinterpret_cast<T *>(A.q) + (int64_t)j0 * A.ldq;
  const T *__restrict__ Tws = reinterpret_cast<const T *>(A.Tws);

  const int warp = tid / 32, lane = tid % 32;
  const int rg = lane % 8;   // row group (update) / reflector group (accumulate)
  const int cq = lane / 8;   // column within a quad
  const int rbase = RW * warp;

  // Each warp loads, updates and accumulates only its own rows rbase ..
  // rbase+RW-1 of a chunk, so a pass over the rows needs no block barrier:
  // the warps run through the chunks independently and meet once per pass.
  const int lr = rbase + lane % RW;  // the chunk row this lane loads
  const int lc = lane / RW;          // first column (or reflector) it loads, then every LPR-th
  T zr[NZ], vur[NV], var[NV];
  auto load = [&](int32_t r0, int pu, int pa) {
    const int32_t row = r0 + lr;
#pragma unroll
    for (int i = 0; i < NZ; ++i) {
      const int cc = lc + LPR * i;
      zr[i] = (cc < w && row < g.n) ? q[(int64_t)cc * A.ldq + row] : Ops<T>::zero();
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int t = lc + LPR * i;
      vur[i] = pu >= 0 ? vget<T>(g, row, pu, t) : Ops<T>::zero();
      var[i] = pa >= 0 ? vget<T>(g, row, pa, t) : Ops<T>::zero();
    }
  };

  for (int pa = g.P - 1; pa >= -1; --pa) {
    const int pu = (pa + 1 <= g.P - 1) ? pa + 1 : -1;
    const int32_t rs = NB * (pa >= 0 ? pa : pu) + g.b;
    T wacc[4][4];  // [quad][i]: W_a[8 i + rg][4 quad + cq], this warp's rows only
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < 4; ++i) wacc[u][i] = Ops<T>::zero();
    load(rs, pu, pa);
    for (int32_t r0 = rs; r0 < g.n; r0 += RC) {
#pragma unroll
      for (int i = 0; i < NZ; ++i) S.Zs[lc + LPR * i][lr] = zr[i];
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        S.Vu[lc + LPR * i][lr] = vur[i];
        S.Va[lr][lc + LPR * i] = var[i];
      }
      __syncwarp();
      if (r0 + RC < g.n) load(r0 + RC, pu, pa);
      if (pu >= 0) {
        // Y[r][c] -= sum_t V_u[r][t] W_u[t][c], rows r = rbase + 8 j + rg
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < nq) {
            const int c = 4 * u + cq;
            T z[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) z[j] = S.Zs[c][rbase + 8 * j + rg];
#pragma unroll 8
            for (int t = 0; t < NB; ++t) {
              const T wt = S.Wu[t][c];
#pragma unroll
              for (int j = 0; j < RPT; ++j) Ops<T>::msub(z[j], S.Vu[t][rbase + 8 * j + rg], wt);
            }
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
              const int r = rbase + 8 * j + rg;
              S.Zs[c][r] = z[j];
              if (c < w && r0 + r < g.n) q[(int64_t)c * A.ldq + r0 + r] = z[j];
            }
          }
        }
      }
      __syncwarp();
      if (pa >= 0) {
        // W_a[t][c] += sum_r conj(V_a[r][t]) Y[r][c] over this warp's rows, t = 8 i + rg
        // (the quad loop is outside the row loop so that a quad the strip
        // lacks is skipped by a branch, not issued as predicated DFMAs)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (u < nq) {
            const int c = 4 * u + cq;
#pragma unroll 4
            for (int r = rbase; r < rbase + RW; ++r) {
              const T y = S.Zs[c][r];
#pragma unroll
              for (int i = 0; i < 4; ++i) Ops<T>::macc(wacc[u][i], S.Va[r][8 * i + rg], y);
            }
          }
        }
      }
      __syncwarp();
    }
    if (pa >= 0) {
      // sum the warps' partial V_a^H Y, then W_a <- T_a (V_a^H Y): the next pass's update
      for (int k = 0; k < 4; ++k) {
        if (warp == k) {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (u < nq) {
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                T &dst = S.Wt[8 * i + rg][4 * u + cq];
                if (k == 0) {
                  dst = wacc[u][i];
                } else {
                  dst = Ops<T>::add(dst, wacc[u][i]);
                }
              }
            }
        }
        __syncthreads();
      }
      for (int e = tid; e < NB * NB; e += ATHREADS) S.Ts[e % NB][e / NB] = Tws[(int64_t)pa * NB * NB + e];
      __syncthreads();
      {
        const int t = tid % NB, cg = tid / NB;  // columns cg, cg+4, cg+8, cg+12
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int c = cg + 4 * m;
          if (c < 4 * nq) {
            T sacc = Ops<T>::zero();
            for (int l = t; l < NB; ++l) Ops<T>::mac(sacc, S.Ts[t][l], S.Wt[l][c]);
            S.Wu[t][c] = sacc;
          }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace bf
}  // namespace tbbt
