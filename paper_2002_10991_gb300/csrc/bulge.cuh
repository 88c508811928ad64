// Band -> tridiagonal reduction by bulge chasing (Eq. 6b, Sec. 2.2.1): the
// step that produces the reflector store the back-transformation consumes,
// run on the GPU so that the store never leaves the device.
//
// Stage i (0-based) has ceil((n-i-2)/b) sweeps; sweep j works on rows
// r = i+1+j*b .. r+L-1, L = min(b, n-r): it builds the Householder reflector
// (LAPACK convention, H^H x = beta e_1, H = I - tau v v^H, v_0 = 1) of column
// c (c = i for j = 0, c = r-b otherwise: the first column of the bulge left by
// sweep j-1) and applies it two-sided (B <- H^H B H) to the entries of the
// band it reaches:
//   left:  rows r .. r+L-1, columns c+1 .. r-1          (A <- H^H A)
//   block: rows and columns r .. r+L-1                   (D <- H^H D H)
//   right: rows r+L .. min(r+L+b, n)-1, columns r .. r+L-1 (A <- A H)
// Hermitian problems get one more stage, n-2, whose length-1 reflector makes
// the last sub-diagonal entry real.
//
// Parallel schedule. Sweep j of stage i touches columns >= r_i(j) - b and
// rows >= r_i(j); sweep j' of stage i+1 touches columns < r_{i+1}(j') + 2b
// and rows < r_{i+1}(j') + 2b. So once stage i has finished sweeps 0 .. j'+2,
// none of its remaining sweeps touch what sweep j' of stage i+1 reads or
// writes, and all the sweeps that wrote it are done: stage i+1 runs sweep j'
// when stage i has published progress >= min(j'+3, sweeps of stage i).
// Persistent blocks claim stages in order from an atomic counter (a stage
// only waits for a smaller one, claimed earlier by a running block), keep the
// working band (lower storage, 2b+1 entries per column, L2-resident) in
// global memory, and publish their progress after every sweep with a
// release; the waits are bounded (TBBT_ETIMEOUT, then the block gives up).
//
// Within a sweep the three updates touch disjoint entries, so after the
// reflector is built the block's warps share them: warps 4..7 the left and
// right updates, warps 0..3 the diagonal block in shared memory. The
// right-update block of a sweep is the next sweep's generation column and
// left-update region; it stays in shared memory between the two. On GB300 a
// warp-level DFMA holds its sub-partition's FP64 unit for many cycles
// whatever the number of active lanes, so the updates are written to issue
// few warp-level FP64 instructions, spread over all four sub-partitions:
// FMA chains per column / row instead of shuffle reductions, and the
// diagonal block as the Hermitian rank-2 update D - w v^H - v w^H.
#pragma once
#include <stdint.h>

#include "apply_kernels.cuh"

namespace tbbt {
namespace bc {

template <typename T>
struct Ops;
template <>
struct Ops<double> {
  static __device__ __forceinline__ double conj(double x) { return x; }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
  static __device__ __forceinline__ double fms_(double a, double b, double c) { return fma(-a, b, c); }  // c - a b
  static __device__ __forceinline__ double re(double x) { return x; }
  static __device__ __forceinline__ double im(double) { return 0.0; }
  static __device__ __forceinline__ double make(double r, double) { return r; }
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double shfl_xor(double x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
};
template <>
struct Ops<zdouble> {
  static __device__ __forceinline__ zdouble conj(zdouble x) { return zdouble{x.re, -x.im}; }
  static __device__ __forceinline__ zdouble mul(zdouble a, zdouble b) {
    return zdouble{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
  }
  // a * b + c
  static __device__ __forceinline__ zdouble fma_(zdouble a, zdouble b, zdouble c) {
    zdouble r;
    r.re = fma(a.re, b.re, c.re);
    r.re = fma(-a.im, b.im, r.re);
    r.im = fma(a.re, b.im, c.im);
    r.im = fma(a.im, b.re, r.im);
    return r;
  }
  // c - a * b
  static __device__ __forceinline__ zdouble fms_(zdouble a, zdouble b, zdouble c) {
    zdouble r;
    r.re = fma(-a.re, b.re, c.re);
    r.re = fma(a.im, b.im, r.re);
    r.im = fma(-a.re, b.im, c.im);
    r.im = fma(-a.im, b.re, r.im);
    return r;
  }
  static __device__ __forceinline__ double re(zdouble x) { return x.re; }
  static __device__ __forceinline__ double im(zdouble x) { return x.im; }
  static __device__ __forceinline__ zdouble make(double r, double i) { return zdouble{r, i}; }
  static __device__ __forceinline__ zdouble zero() { return zdouble{0.0, 0.0}; }
  static __device__ __forceinline__ zdouble shfl_xor(zdouble x, int o) {
    return zdouble{__shfl_xor_sync(0xffffffffu, x.re, o), __shfl_xor_sync(0xffffffffu, x.im, o)};
  }
};
template <typename T>
__device__ __forceinline__ T add(T a, T b) {
  return Ops<T>::make(Ops<T>::re(a) + Ops<T>::re(b), Ops<T>::im(a) + Ops<T>::im(b));
}
template <typename T>
__device__ __forceinline__ T sub(T a, T b) {
  return Ops<T>::make(Ops<T>::re(a) - Ops<T>::re(b), Ops<T>::im(a) - Ops<T>::im(b));
}
template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = add(x, Ops<T>::shfl_xor(x, o));
  return x;
}

template <typename T>
struct BcArgs {
  T *w;             // working band, lower storage: (row, col) at w[(row - col) + col * ldw], ldw = 2b + 1
  int64_t ldw;
  StoreGeom g;
  T *hh_v;          // canonical store, K x b
  T *hh_tau;        // K
  const int64_t *stage_off;  // first reflector of each stage
  int32_t nstages;
  int *progress;    // per stage: sweeps finished (published with release); kPoison if abandoned
  unsigned *counter;
  int *err;
  long long timeout_ns;
};

constexpr int kBcMaxB = 128;

template <typename T>
__device__ __forceinline__ T *bat(const BcArgs<T> &a, int64_t row, int64_t col) {
  return a.w + (row - col) + col * a.ldw;
}
// The working band is written by other SMs: read and write it at L2 (no
// stale L1 lines from an earlier stage this block ran).
__device__ __forceinline__ double ldw(const double *p) { return __ldcg(p); }
__device__ __forceinline__ zdouble ldw(const zdouble *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return zdouble{v.x, v.y};
}
__device__ __forceinline__ void stw(double *p, double v) { __stcg(p, v); }
__device__ __forceinline__ void stw(zdouble *p, zdouble v) { __stcg(reinterpret_cast<double2 *>(p), make_double2(v.re, v.im)); }

// Hermitian entry (row, col) from the lower storage.
template <typename T>
__device__ __forceinline__ T hget(const BcArgs<T> &a, int64_t row, int64_t col) {
  return row >= col ? ldw(bat(a, row, col)) : Ops<T>::conj(ldw(bat(a, col, row)));
}

// Barrier among the first `count` threads of the block (id 1; id 0 is __syncthreads).
__device__ __forceinline__ void bar_sub(int count) { asm volatile("bar.sync 1, %0;\n" ::"r"(count) : "memory"); }

// Bounded wait until a stage's published progress reaches need (1: give up).
__device__ inline int wait_progress(int *err, long long timeout_ns, const int *flag, int need) {
  const long long t0 = globaltimer_ns();
  for (unsigned it = 0;; ++it) {
    const int v = ld_acquire(flag);
    if (v == kPoison) return 1;
    if (v >= need) return 0;
    if (*(volatile int *)err != 0) return 1;
    if (globaltimer_ns() - t0 > timeout_ns) {
      atomicCAS(err, 0, 4 /* TBBT_ETIMEOUT */);
      return 1;
    }
    __nanosleep(it < 64 ? 32 : 256);
  }
}

// Barrier among the 128 threads of warps 4..7 (id 2).
__device__ __forceinline__ void bar_upper() { asm volatile("bar.sync 2, 128;\n" ::: "memory"); }

// Shared memory of the bulge kernel, in elements of T: the reflector, the
// diagonal block, y = D v with its four partial sums, and (KEEP) the
// right-update block kept on chip for the next sweep (padded to b+1 rows)
// with the half dot products of its columns / rows.
__host__ __device__ constexpr int64_t bc_smem_elems(int b, bool keep) {
  return (int64_t)kBcMaxB * 6 + (int64_t)b * b + (keep ? (int64_t)b * (b + 1) + 2 * kBcMaxB : 0);
}

// KEEP: the right-update block of sweep j (rows r+L .. r+L+b-1, columns
// r .. r+L-1) stays in shared memory. It is exactly the next sweep's
// generation column and left-update columns, so sweep j+1 builds its
// reflector and runs its left update on chip, then writes the block back to
// L2 (before its progress release; stage i+1 first reads those entries at
// its sweep j, after progress j+3). The last sweep of a stage writes its
// right block (non-empty when n-i-2 is a multiple of b) straight to L2.
// Without KEEP (large b) every sweep reads and writes the band at L2.
template <typename T, bool KEEP>
__global__ void __launch_bounds__(256, 1) bulge_kernel(BcArgs<T> a) {
  using O = Ops<T>;
  constexpr int EPL = kBcMaxB / 32;  // elements per lane, at most
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.g.b;
  T *sv = reinterpret_cast<T *>(smem_raw);  // reflector, b
  T *sD = sv + kBcMaxB;                     // diagonal block, b x b (column-major, ld b)
  T *sy = sD + (int64_t)b * b;              // y = D v, b
  T *sy4 = sy + kBcMaxB;                    // partial sums of y, 4 x kBcMaxB
  T *sR = sy4 + 4 * kBcMaxB;                // KEEP: right block, sR[t + s ldr] = A[r + t, c + s] of the next sweep
  const int ldr = b + 1;                    // padded: a thread per row or per column reads without bank conflicts
  T *sPart = sR + (int64_t)b * ldr;         // KEEP: the two half dot products of each column / row
  __shared__ T s_tau;
  __shared__ int s_stage;
  __shared__ int s_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t n = a.g.n;
  for (;;) {
    if (tid == 0) {
      s_stage = (int)atomicAdd(a.counter, 1u);
      s_stop = (*(volatile int *)a.err != 0);
    }
    __syncthreads();
    const int i = s_stage;
    if (i >= a.nstages || s_stop) break;
    const int32_t nsweep = (i <= n - 3) ? (n - i - 2 + b - 1) / b : 1;
    const int32_t prev_sweeps = (i >= 1) ? ((i - 1 <= n - 3) ? (n - i - 1 + b - 1) / b : 1) : 0;
    int *mine = a.progress + i;
    bool abandoned = false;
    for (int32_t j = 0; j < nsweep; ++j) {
      // the previous stage must be 3 sweeps ahead (or finished)
      if (tid == 0 && i >= 1) {
        const int need = min(j + 3, prev_sweeps);
        s_stop = wait_progress(a.err, a.timeout_ns, a.progress + i - 1, need);
      }
      __syncthreads();
      if (s_stop) {
        abandoned = true;
        break;
      }
      const int64_t r = i + 1 + (int64_t)j * b;
      const int L = (int)((n - r < b) ? n - r : b);
      const int64_t c = (j == 0) ? i : r - b;
      const bool on_chip = KEEP && j > 0;  // generation and left-update columns are in sR
      // The right-update block is final once the previous stage is three
      // sweeps ahead (no sweep of this stage before j touches its rows, >= r+L),
      // so warps 4..7 issue the loads of their first HO elements of it now, into
      // registers, while warp 0 builds the reflector.
      constexpr int HO = sizeof(T) == 8 ? 32 : 16;
      T pre[HO];
      const int64_t rend0 = (r + L + b < n) ? r + L + b : n;
      const int nrr0 = (int)(rend0 - (r + L));  // right rows
      if (KEEP) {
        if (warp >= 4 && nrr0 > 0) {
          const int ut = tid - 128, tot = nrr0 * L;
#pragma unroll
          for (int u = 0; u < HO; ++u) {
            const int idx = ut + 128 * u;
            pre[u] = idx < tot ? ldw(bat(a, r + L + idx % nrr0, r + idx / nrr0)) : O::zero();
          }
        }
      }
      // ---- the reflector of column c, rows r .. r+L-1 (one warp)
      if (warp == 0) {
        T xv[EPL];
        double s2 = 0.0;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int t = lane + 32 * e;
          xv[e] = (t < L) ? (on_chip ? sR[t] : ldw(bat(a, r + t, c))) : O::zero();  // column 0 of sR
          if (t >= 1) {
            s2 = fma(O::re(xv[e]), O::re(xv[e]), s2);
            s2 = fma(O::im(xv[e]), O::im(xv[e]), s2);
          }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        const double ar = __shfl_sync(0xffffffffu, O::re(xv[0]), 0);
        const double ai = __shfl_sync(0xffffffffu, O::im(xv[0]), 0);
        T tau, scal;
        double beta;
        if (s2 == 0.0 && ai == 0.0) {
          tau = O::zero();
          beta = ar;
          scal = O::zero();
        } else {
          const double nrm = sqrt(ar * ar + ai * ai + s2);
          beta = ar >= 0.0 ? -nrm : nrm;
          // tau = (beta - alpha) / beta, scal = 1 / (alpha - beta)
          tau = O::make((beta - ar) / beta, -ai / beta);
          const double dr = ar - beta, di = ai;
          const double den = dr * dr + di * di;
          scal = O::make(dr / den, -di / den);
        }
        const bool zs = O::re(scal) == 0.0 && O::im(scal) == 0.0;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int t = lane + 32 * e;
          if (t < L) {
            sv[t] = (t == 0) ? O::make(1.0, 0.0) : (zs ? O::zero() : O::mul(xv[e], scal));
            const T piv = (t == 0) ? O::make(beta, 0.0) : O::zero();
            if (on_chip)
              sR[t] = piv;
            else
              stw(bat(a, r + t, c), piv);
          }
        }
        __syncwarp();
        if (lane == 0) s_tau = tau;
        // the canonical store
        const int64_t k = a.stage_off[i] + j;
        for (int t = lane; t < b; t += 32) a.hh_v[k * b + t] = (t < L) ? sv[t] : O::zero();
        if (lane == 0) a.hh_tau[k] = tau;
      }
      __syncthreads();
      const T tau = s_tau;
      const T ctau = O::conj(tau);
      // The left / right updates (warps 4..7) and the diagonal block (warps
      // 0..3) touch disjoint entries and run side by side.
      if (warp >= 4) {
        const int ut = tid - 128;  // 0 .. 127
        const int64_t rend = (r + L + b < n) ? r + L + b : n;
        const int nrr = (int)(rend - (r + L));  // right rows
        if constexpr (KEEP) {
          // Two threads per column (left) or row (right) of a padded on-chip
          // block, each taking half of the rows t: plain FMA chains, no
          // shuffle reductions, and all four warps (every sub-partition's
          // FP64 unit) carry an equal share.
          const int q = ut % 64, h = ut / 64;
          const int tlo = (L * h) / 2, thi = (L * (h + 1)) / 2;
          if (on_chip) {
            // ---- left, on chip: columns c+1 .. r-1 are sR columns 1 .. b-1
            for (int sc = 1 + q; sc < b; sc += 64) {
              const T *col = sR + (int64_t)sc * ldr;
              T wsum = O::zero();
              for (int t = tlo; t < thi; ++t) wsum = O::fma_(O::conj(sv[t]), col[t], wsum);
              sPart[h * kBcMaxB + sc] = wsum;
            }
            bar_upper();
            for (int sc = 1 + q; sc < b; sc += 64) {
              T *col = sR + (int64_t)sc * ldr;
              const T f = O::mul(ctau, add(sPart[sc], sPart[kBcMaxB + sc]));
              for (int t = tlo; t < thi; ++t) col[t] = O::fms_(f, sv[t], col[t]);
            }
            bar_upper();
            // the block is final for this stage: back to L2 (coalesced down each column)
            for (int idx = ut; idx < L * b; idx += 128) {
              const int t = idx % L, sc = idx / L;
              stw(bat(a, r + t, c + sc), sR[t + sc * ldr]);
            }
            bar_upper();  // every read of sR done before the right update refills it
          }
          if (nrr > 0) {
            // ---- right: rows r+L .. rend-1, columns r .. r+L-1 (A <- A H); the old
            // values land in sR (row k - (r+L), column t): the first HO per thread
            // from the loads issued before the reflector, the rest eight loads in
            // flight per thread
            const int tot = nrr * L;
#pragma unroll
            for (int u = 0; u < HO; ++u) {
              const int idx = ut + 128 * u;
              if (idx < tot) sR[idx % nrr + (idx / nrr) * ldr] = pre[u];
            }
            for (int base = 128 * HO; base < tot; base += 128 * 8) {
              T tmp[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int idx = base + ut + 128 * u;
                tmp[u] = idx < tot ? ldw(bat(a, r + L + idx % nrr, r + idx / nrr)) : O::zero();
              }
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int idx = base + ut + 128 * u;
                if (idx < tot) sR[idx % nrr + (idx / nrr) * ldr] = tmp[u];
              }
            }
            bar_upper();
            for (int kk = q; kk < nrr; kk += 64) {
              T wsum = O::zero();
              for (int t = tlo; t < thi; ++t) wsum = O::fma_(sR[kk + t * ldr], sv[t], wsum);
              sPart[h * kBcMaxB + kk] = wsum;
            }
            bar_upper();
            for (int kk = q; kk < nrr; kk += 64) {
              const T f = O::mul(tau, add(sPart[kk], sPart[kBcMaxB + kk]));
              for (int t = tlo; t < thi; ++t) sR[kk + t * ldr] = O::fms_(f, O::conj(sv[t]), sR[kk + t * ldr]);
            }
            if (j + 1 == nsweep) {
              // no later sweep of this stage consumes it: straight to L2
              bar_upper();
              for (int idx = ut; idx < tot; idx += 128)
                stw(bat(a, r + L + idx % nrr, r + idx / nrr), sR[idx % nrr + (idx / nrr) * ldr]);
            }
          }
        } else {
          // Wide bands: both updates at L2, a warp per batch of CB columns
          // (rows), loads issued together, values kept in registers.
          constexpr int CB = 4;
          const int w4 = warp - 4;
          // ---- left: rows r .. r+L-1, columns c+1 .. r-1
          for (int64_t s0 = c + 1 + CB * w4; s0 < r; s0 += CB * 4) {
            T x[CB][EPL];
#pragma unroll
            for (int q = 0; q < CB; ++q)
#pragma unroll
              for (int e = 0; e < EPL; ++e) {
                const int t = lane + 32 * e;
                x[q][e] = (s0 + q < r && t < L) ? ldw(bat(a, r + t, s0 + q)) : O::zero();
              }
#pragma unroll
            for (int q = 0; q < CB; ++q) {
              T wsum = O::zero();
#pragma unroll
              for (int e = 0; e < EPL; ++e) {
                const int t = lane + 32 * e;
                if (t < L) wsum = O::fma_(O::conj(sv[t]), x[q][e], wsum);
              }
              const T f = O::mul(ctau, warp_sum(wsum));
              if (s0 + q >= r) continue;
#pragma unroll
              for (int e = 0; e < EPL; ++e) {
                const int t = lane + 32 * e;
                if (t < L) stw(bat(a, r + t, s0 + q), O::fms_(f, sv[t], x[q][e]));
              }
            }
          }
          // ---- right: rows r+L .. rend-1, columns r .. r+L-1 (A <- A H)
          for (int64_t k0 = r + L + CB * w4; k0 < rend; k0 += CB * 4) {
            T x[CB][EPL];
#pragma unroll
            for (int q = 0; q < CB; ++q)
#pragma unroll
              for (int e = 0; e < EPL; ++e) {
                const int t = lane + 32 * e;
                x[q][e] = (k0 + q < rend && t < L) ? ldw(bat(a, k0 + q, r + t)) : O::zero();
              }
#pragma unroll
            for (int q = 0; q < CB; ++q) {
              T wsum = O::zero();
#pragma unroll
              for (int e = 0; e < EPL; ++e) {
                const int t = lane + 32 * e;
                if (t < L) wsum = O::fma_(x[q][e], sv[t], wsum);
              }
              const T f = O::mul(tau, warp_sum(wsum));
              const int64_t k = k0 + q;
              if (k >= rend) continue;
#pragma unroll
              for (int e = 0; e < EPL; ++e) {
                const int t = lane + 32 * e;
                if (t < L) stw(bat(a, k, r + t), O::fms_(f, O::conj(sv[t]), x[q][e]));
              }
            }
          }
        }
      } else {
        // ---- the diagonal block, D <- H^H D H = D - tau y v^H - conj(tau) v y^H
        // + |tau|^2 (v^H y) v v^H with y = D v (D Hermitian: v^H D = y^H)
        const int bt = tid;  // 0 .. 127
        for (int idx = bt; idx < L * L; idx += 128) {
          const int t = idx % L, s2 = idx / L;
          sD[t + s2 * b] = hget(a, r + t, r + s2);
        }
        bar_sub(128);
        // y = D v: warp w sums the quarter w of the columns, then the four add up
        {
          const int q0 = (L * warp) / 4, q1 = (L * (warp + 1)) / 4;
          for (int t = lane; t < L; t += 32) {
            T acc = O::zero();
            for (int s2 = q0; s2 < q1; ++s2) acc = O::fma_(sD[t + s2 * b], sv[s2], acc);
            sy4[warp * kBcMaxB + t] = acc;
          }
        }
        bar_sub(128);
        for (int t = bt; t < L; t += 128)
          sy[t] = add(add(sy4[t], sy4[kBcMaxB + t]), add(sy4[2 * kBcMaxB + t], sy4[3 * kBcMaxB + t]));
        bar_sub(128);
        double al = 0.0;  // v^H y (real), every warp reduces it for itself
        for (int t = lane; t < L; t += 32) al += O::re(O::mul(O::conj(sv[t]), sy[t]));
#pragma unroll
        for (int o = 16; o; o >>= 1) al += __shfl_xor_sync(0xffffffffu, al, o);
        const double tt2 = O::re(tau) * O::re(tau) + O::im(tau) * O::im(tau);
        const double half = 0.5 * tt2 * al;
        // H^H D H = D - w v^H - v w^H with w = tau y - (|tau|^2 (v^H y) / 2) v
        T *sw = sy4;  // the partial sums are consumed
        for (int t = bt; t < L; t += 128) sw[t] = O::fms_(O::make(half, 0.0), sv[t], O::mul(tau, sy[t]));
        bar_sub(128);
        for (int idx = bt; idx < L * L; idx += 128) {
          const int t = idx % L, s2 = idx / L;
          if (t < s2) continue;
          T dv = sD[t + s2 * b];
          dv = O::fms_(sw[t], O::conj(sv[s2]), dv);
          dv = O::fms_(sv[t], O::conj(sw[s2]), dv);
          if (t == s2) dv = O::make(O::re(dv), 0.0);
          stw(bat(a, r + t, r + s2), dv);
        }
      }
      __syncthreads();
      // sweep j of stage i is done: what the next stage may read next is in
      // L2 (the barrier above orders every thread's stores before this
      // release; with KEEP the block kept on chip is written back during
      // sweep j+1, before progress j+2)
      if (tid == 0) st_release(mine, j + 1);
    }
    if (abandoned && tid == 0) st_release(mine, kPoison);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Two-CTA form (the right block kept on chip): a cluster of two CTAs runs one
// stage. CTA 0 builds each sweep's reflector and applies the left and right
// updates with all eight warps (four threads per column / row); CTA 1
// applies the diagonal-block update D <- H^H D H with all eight warps. A
// sweep's FP64 work is thus split over two SMs, and the two halves run side
// by side:
//  * CTA 0 claims the stage and passes its index to CTA 1 (a store into CTA
//    1's shared memory and an arrival on its `stage` barrier);
//  * both wait for the previous stage's progress (the lag rule above);
//  * CTA 0's warp 0 writes the reflector and tau into CTA 1's shared memory
//    and arrives on its `refl` barrier (one arrival per lane, after the
//    lane's stores);
//  * CTA 1 loads D (it may run ahead: D of sweep j+1 shares no entry with
//    sweep j's updates), waits for the reflector, updates D, stores it to L2,
//    fences at GPU scope and arrives on CTA 0's `diag` barrier;
//  * CTA 0, after its own updates, waits for `diag` before it publishes the
//    sweep's progress.
// Every wait is bounded and also gives up when the device error word is set.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;\n" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, zdouble v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};\n" ::"r"(addr), "d"(v.re), "d"(v.im) : "memory");
}
__device__ __forceinline__ void st_cluster_i32(uint32_t addr, int v) {
  asm volatile("st.shared::cluster.b32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void bc_mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// arrival on a barrier in the peer CTA's shared memory (release at cluster scope)
__device__ __forceinline__ void bc_arrive_remote(uint32_t remote_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" ::"r"(remote_bar) : "memory");
}
__device__ __forceinline__ bool bc_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity (0: done; 1: gave up).
__device__ inline int bc_wait(uint64_t *bar, uint32_t parity, int *err, long long timeout_ns) {
  if (bc_try_wait(bar, parity)) return 0;
  const long long t0 = globaltimer_ns();
  for (unsigned it = 1;; ++it) {
    if (bc_try_wait(bar, parity)) return 0;
    if ((it & 15) == 0) {
      if (*(volatile int *)err != 0) return 1;
      if (globaltimer_ns() - t0 > timeout_ns) {
        atomicCAS(err, 0, 4 /* TBBT_ETIMEOUT */);
        return 1;
      }
    }
  }
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Shared memory of the two-CTA form, in elements of T: the reflector, then
// (CTA 0) the right block padded to b+1 rows and four partial dot products
// per column / row, or (CTA 1) the diagonal block, y and eight partial sums.
__host__ __device__ constexpr int64_t bc2_smem_elems(int b) {
  return (int64_t)kBcMaxB + (((int64_t)b * (b + 1) + 4 * kBcMaxB) > ((int64_t)b * b + 9 * kBcMaxB)
                                 ? ((int64_t)b * (b + 1) + 4 * kBcMaxB)
                                 : ((int64_t)b * b + 9 * kBcMaxB));
}

template <typename T>
__global__ void __launch_bounds__(256, 1) bulge_cluster_kernel(BcArgs<T> a) {
  using O = Ops<T>;
  constexpr int EPL = kBcMaxB / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.g.b;
  T *sv = reinterpret_cast<T *>(smem_raw);  // reflector (both CTAs: CTA 0 writes CTA 1's copy)
  // CTA 0
  T *sR = sv + kBcMaxB;                     // right block: sR[t + s ldr] = A[r + t, c + s] of the next sweep
  const int ldr = b + 1;
  T *sPart = sR + (int64_t)b * ldr;         // four partial dot products per column / row
  // CTA 1
  T *sD = sv + kBcMaxB;                     // diagonal block, b x b (column-major, ld b)
  T *sy = sD + (int64_t)b * b;              // y = D v
  T *sy8 = sy + kBcMaxB;                    // eight partial sums of y
  __shared__ __align__(8) uint64_t bar_stage, bar_refl, bar_diag;
  __shared__ T s_tau;
  __shared__ int s_stage;
  __shared__ int s_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t rank = cluster_ctarank();
  const int32_t n = a.g.n;
  if (tid == 0) {
    bc_mbar_init(&bar_stage, 1);  // CTA 1: the stage index arrived
    bc_mbar_init(&bar_refl, 32);  // CTA 1: the reflector arrived (one arrival per lane of CTA 0's warp 0)
    bc_mbar_init(&bar_diag, 1);   // CTA 0: CTA 1 stored the sweep's diagonal block
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  cluster_sync_all();  // the peer's barriers exist before anyone arrives on them
  const uint32_t peer = rank ^ 1u;
  const uint32_t r_stage = mapa_shared(smem_u32(&s_stage), peer);
  const uint32_t r_tau = mapa_shared(smem_u32(&s_tau), peer);
  const uint32_t r_sv = mapa_shared(smem_u32(sv), peer);
  const uint32_t r_bar_stage = mapa_shared(smem_u32(&bar_stage), peer);
  const uint32_t r_bar_refl = mapa_shared(smem_u32(&bar_refl), peer);
  const uint32_t r_bar_diag = mapa_shared(smem_u32(&bar_diag), peer);
  uint32_t n_stage = 0, n_sweep = 0;  // completed phases of the stage and per-sweep barriers
  for (;;) {
    // ---- the stage: CTA 0 claims it and passes it on
    if (tid == 0) {
      if (rank == 0) {
        const int st = (int)atomicAdd(a.counter, 1u);
        s_stage = st;
        s_stop = (*(volatile int *)a.err != 0);
        st_cluster_i32(r_stage, st);
        bc_arrive_remote(r_bar_stage);
      } else {
        s_stop = bc_wait(&bar_stage, n_stage & 1, a.err, a.timeout_ns);
      }
    }
    ++n_stage;
    __syncthreads();
    const int i = s_stage;
    if (s_stop || i >= a.nstages) break;
    const int32_t nsweep = (i <= n - 3) ? (n - i - 2 + b - 1) / b : 1;
    const int32_t prev_sweeps = (i >= 1) ? ((i - 1 <= n - 3) ? (n - i - 1 + b - 1) / b : 1) : 0;
    int *mine = a.progress + i;
    bool abandoned = false;
    for (int32_t j = 0; j < nsweep; ++j, ++n_sweep) {
      if (tid == 0 && i >= 1) s_stop = wait_progress(a.err, a.timeout_ns, a.progress + i - 1, min(j + 3, prev_sweeps));
      __syncthreads();
      if (s_stop) {
        abandoned = true;
        break;
      }
      const int64_t r = i + 1 + (int64_t)j * b;
      const int L = (int)((n - r < b) ? n - r : b);
      const int64_t c = (j == 0) ? i : r - b;
      const bool on_chip = j > 0;
      if (rank == 0) {
        // ---- right block: the first HO elements of each thread, loaded now
        constexpr int HO = 16;
        T pre[HO];
        const int64_t rend = (r + L + b < n) ? r + L + b : n;
        const int nrr = (int)(rend - (r + L));
        const int tot = nrr * L;
#pragma unroll
        for (int u = 0; u < HO; ++u) {
          const int idx = tid + 256 * u;
          pre[u] = idx < tot ? ldw(bat(a, r + L + idx % nrr, r + idx / nrr)) : O::zero();
        }
        // ---- the reflector of column c (warp 0), also into CTA 1
        if (warp == 0) {
          T xv[EPL];
          double s2 = 0.0;
#pragma unroll
          for (int e = 0; e < EPL; ++e) {
            const int t = lane + 32 * e;
            xv[e] = (t < L) ? (on_chip ? sR[t] : ldw(bat(a, r + t, c))) : O::zero();
            if (t >= 1) {
              s2 = fma(O::re(xv[e]), O::re(xv[e]), s2);
              s2 = fma(O::im(xv[e]), O::im(xv[e]), s2);
            }
          }
#pragma unroll
          for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
          const double ar = __shfl_sync(0xffffffffu, O::re(xv[0]), 0);
          const double ai = __shfl_sync(0xffffffffu, O::im(xv[0]), 0);
          T tau, scal;
          double beta;
          if (s2 == 0.0 && ai == 0.0) {
            tau = O::zero();
            beta = ar;
            scal = O::zero();
          } else {
            const double nrm = sqrt(ar * ar + ai * ai + s2);
            beta = ar >= 0.0 ? -nrm : nrm;
            tau = O::make((beta - ar) / beta, -ai / beta);
            const double dr = ar - beta, di = ai;
            const double den = dr * dr + di * di;
            scal = O::make(dr / den, -di / den);
          }
          const bool zs = O::re(scal) == 0.0 && O::im(scal) == 0.0;
#pragma unroll
          for (int e = 0; e < EPL; ++e) {
            const int t = lane + 32 * e;
            if (t < L) {
              const T vt = (t == 0) ? O::make(1.0, 0.0) : (zs ? O::zero() : O::mul(xv[e], scal));
              sv[t] = vt;
              st_cluster(r_sv + (uint32_t)(t * sizeof(T)), vt);
              const T piv = (t == 0) ? O::make(beta, 0.0) : O::zero();
              if (on_chip)
                sR[t] = piv;
              else
                stw(bat(a, r + t, c), piv);
            }
          }
          if (lane == 0) {
            s_tau = tau;
            st_cluster(r_tau, tau);
          }
          bc_arrive_remote(r_bar_refl);  // after this lane's stores into CTA 1
          const int64_t k = a.stage_off[i] + j;
          __syncwarp();
          for (int t = lane; t < b; t += 32) a.hh_v[k * b + t] = (t < L) ? sv[t] : O::zero();
          if (lane == 0) a.hh_tau[k] = tau;
        }
        __syncthreads();
        const T tau = s_tau;
        const T ctau = O::conj(tau);
        const int q = tid % 64, h = tid / 64;  // four threads per column / row
        const int tlo = (L * h) / 4, thi = (L * (h + 1)) / 4;
        if (on_chip) {
          // ---- left, on chip: columns c+1 .. r-1 are sR columns 1 .. b-1
          for (int sc = 1 + q; sc < b; sc += 64) {
            const T *col = sR + (int64_t)sc * ldr;
            T wsum = O::zero();
            for (int t = tlo; t < thi; ++t) wsum = O::fma_(O::conj(sv[t]), col[t], wsum);
            sPart[h * kBcMaxB + sc] = wsum;
          }
          __syncthreads();
          for (int sc = 1 + q; sc < b; sc += 64) {
            T *col = sR + (int64_t)sc * ldr;
            const T f = O::mul(ctau, add(add(sPart[sc], sPart[kBcMaxB + sc]),
                                         add(sPart[2 * kBcMaxB + sc], sPart[3 * kBcMaxB + sc])));
            for (int t = tlo; t < thi; ++t) col[t] = O::fms_(f, sv[t], col[t]);
          }
          __syncthreads();
          for (int idx = tid; idx < L * b; idx += 256) {
            const int t = idx % L, sc = idx / L;
            stw(bat(a, r + t, c + sc), sR[t + sc * ldr]);
          }
          __syncthreads();  // every read of sR done before the right update refills it
        }
        if (nrr > 0) {
          // ---- right: rows r+L .. rend-1, columns r .. r+L-1 (A <- A H)
#pragma unroll
          for (int u = 0; u < HO; ++u) {
            const int idx = tid + 256 * u;
            if (idx < tot) sR[idx % nrr + (idx / nrr) * ldr] = pre[u];
          }
          for (int base = 256 * HO; base < tot; base += 256 * 8) {
            T tmp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int idx = base + tid + 256 * u;
              tmp[u] = idx < tot ? ldw(bat(a, r + L + idx % nrr, r + idx / nrr)) : O::zero();
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int idx = base + tid + 256 * u;
              if (idx < tot) sR[idx % nrr + (idx / nrr) * ldr] = tmp[u];
            }
          }
          __syncthreads();
          for (int kk = q; kk < nrr; kk += 64) {
            T wsum = O::zero();
            for (int t = tlo; t < thi; ++t) wsum = O::fma_(sR[kk + t * ldr], sv[t], wsum);
            sPart[h * kBcMaxB + kk] = wsum;
          }
          __syncthreads();
          for (int kk = q; kk < nrr; kk += 64) {
            const T f = O::mul(tau, add(add(sPart[kk], sPart[kBcMaxB + kk]),
                                        add(sPart[2 * kBcMaxB + kk], sPart[3 * kBcMaxB + kk])));
            for (int t = tlo; t < thi; ++t) sR[kk + t * ldr] = O::fms_(f, O::conj(sv[t]), sR[kk + t * ldr]);
          }
          if (j + 1 == nsweep) {
            __syncthreads();
            for (int idx = tid; idx < tot; idx += 256)
              stw(bat(a, r + L + idx % nrr, r + idx / nrr), sR[idx % nrr + (idx / nrr) * ldr]);
          }
        }
        __syncthreads();
        // CTA 1's diagonal block of this sweep is in L2 before the progress release
        if (tid == 0) s_stop = bc_wait(&bar_diag, n_sweep & 1, a.err, a.timeout_ns);
        __syncthreads();
        if (s_stop) {
          abandoned = true;
          break;
        }
        if (tid == 0) st_release(mine, j + 1);
      } else {
        // ---- CTA 1: the diagonal block, D <- H^H D H = D - w v^H - v w^H
        for (int idx = tid; idx < L * L; idx += 256) {
          const int t = idx % L, s2 = idx / L;
          sD[t + s2 * b] = hget(a, r + t, r + s2);
        }
        if (tid == 0) s_stop = bc_wait(&bar_refl, n_sweep & 1, a.err, a.timeout_ns);
        __syncthreads();
        if (s_stop) {
          abandoned = true;
          break;
        }
        const T tau = s_tau;
        {
          // y = D v: warp w sums the eighth w of the columns, then the eight add up
          const int q0 = (L * warp) / 8, q1 = (L * (warp + 1)) / 8;
          for (int t = lane; t < L; t += 32) {
            T acc = O::zero();
            for (int s2 = q0; s2 < q1; ++s2) acc = O::fma_(sD[t + s2 * b], sv[s2], acc);
            sy8[warp * kBcMaxB + t] = acc;
          }
        }
        __syncthreads();
        for (int t = tid; t < L; t += 256) {
          T acc = sy8[t];
#pragma unroll
          for (int w8 = 1; w8 < 8; ++w8) acc = add(acc, sy8[w8 * kBcMaxB + t]);
          sy[t] = acc;
        }
        __syncthreads();
        double al = 0.0;  // v^H y (real), every warp reduces it for itself
        for (int t = lane; t < L; t += 32) al += O::re(O::mul(O::conj(sv[t]), sy[t]));
#pragma unroll
        for (int o = 16; o; o >>= 1) al += __shfl_xor_sync(0xffffffffu, al, o);
        const double tt2 = O::re(tau) * O::re(tau) + O::im(tau) * O::im(tau);
        const double half = 0.5 * tt2 * al;
        T *sw = sy8;  // the partial sums are consumed
        __syncthreads();
        for (int t = tid; t < L; t += 256) sw[t] = O::fms_(O::make(half, 0.0), sv[t], O::mul(tau, sy[t]));
        __syncthreads();
        for (int idx = tid; idx < L * L; idx += 256) {
          const int t = idx % L, s2 = idx / L;
          if (t < s2) continue;
          T dv = sD[t + s2 * b];
          dv = O::fms_(sw[t], O::conj(sv[s2]), dv);
          dv = O::fms_(sv[t], O::conj(sw[s2]), dv);
          if (t == s2) dv = O::make(O::re(dv), 0.0);
          stw(bat(a, r + t, r + s2), dv);
        }
        __syncthreads();
        if (tid == 0) {
          __threadfence();  // the stores above are visible GPU-wide before CTA 0 publishes
          bc_arrive_remote(r_bar_diag);
        }
      }
    }
    if (abandoned && rank == 0 && tid == 0) st_release(mine, kPoison);
    __syncthreads();
    if (abandoned) break;
  }
  cluster_sync_all();  // no access to the peer's shared memory after this
}

// Diagonal and (real) sub-diagonal of the reduced band.
template <typename T>
__global__ void bulge_extract_kernel(const T *w, int64_t ldw, int32_t n, double *d, double *e) {
  const int64_t cidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= n) return;
  d[cidx] = Ops<T>::re(w[cidx * ldw]);
  if (cidx + 1 < n) e[cidx] = Ops<T>::re(w[1 + cidx * ldw]);
}

// Working band from the caller's lower band storage (b+1) x n (ldb >= b+1);
// zero fill beyond, real diagonal.
template <typename T>
__global__ void bulge_load_kernel(const T *band, int64_t ldb, T *w, int64_t ldw, int32_t n, int32_t b) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)n * ldw;
  if (idx >= total) return;
  const int64_t col = idx / ldw, dd = idx - col * ldw;
  T val = Ops<T>::zero();
  if (dd <= b && col + dd < n) val = band[dd + col * ldb];
  if (dd == 0) val = Ops<T>::make(Ops<T>::re(val), 0.0);
  w[idx] = val;
}

}  // namespace bc
}  // namespace tbbt
