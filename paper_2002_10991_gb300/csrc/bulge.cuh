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
// reflector is built the block's warps share them: the left and right
// updates one column / row per warp, the diagonal block in shared memory.
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

template <typename T>
__global__ void __launch_bounds__(256, 1) bulge_kernel(BcArgs<T> a) {
  using O = Ops<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = a.g.b;
  T *sv = reinterpret_cast<T *>(smem_raw);  // reflector, b
  T *sD = sv + kBcMaxB;                     // diagonal block, b x b (column-major, ld b)
  T *sy = sD + (int64_t)b * b;              // work vector, b
  __shared__ T s_tau;
  __shared__ int s_stage;
  __shared__ int s_stop;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
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
      // ---- the reflector of column c, rows r .. r+L-1 (one warp)
      if (warp == 0) {
        double s2 = 0.0;
        for (int t = 1 + lane; t < L; t += 32) {
          const T x = ldw(bat(a, r + t, c));
          s2 = fma(O::re(x), O::re(x), s2);
          s2 = fma(O::im(x), O::im(x), s2);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        const T alpha = ldw(bat(a, r, c));
        T tau, scal;
        double beta;
        if (s2 == 0.0 && O::im(alpha) == 0.0) {
          tau = O::zero();
          beta = O::re(alpha);
          scal = O::zero();
        } else {
          const double nrm = sqrt(O::re(alpha) * O::re(alpha) + O::im(alpha) * O::im(alpha) + s2);
          beta = O::re(alpha) >= 0.0 ? -nrm : nrm;
          // tau = (beta - alpha) / beta, scal = 1 / (alpha - beta)
          tau = O::make((beta - O::re(alpha)) / beta, -O::im(alpha) / beta);
          const double dr = O::re(alpha) - beta, di = O::im(alpha);
          const double den = dr * dr + di * di;
          scal = O::make(dr / den, -di / den);
        }
        for (int t = lane; t < L; t += 32) {
          T vt;
          if (t == 0) vt = O::make(1.0, 0.0);
          else vt = (O::re(scal) == 0.0 && O::im(scal) == 0.0) ? O::zero() : O::mul(ldw(bat(a, r + t, c)), scal);
          sv[t] = vt;
        }
        __syncwarp();
        for (int t = lane; t < L; t += 32) stw(bat(a, r + t, c), (t == 0) ? O::make(beta, 0.0) : O::zero());
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
        // ---- left: rows r .. r+L-1, columns c+1 .. r-1, and right: rows
        // r+L .. min(r+L+b, n)-1, columns r .. r+L-1. A warp takes CB columns
        // (rows) at a time: all their loads are issued before the reductions,
        // and the values stay in registers for the update.
        constexpr int CB = 4;              // columns (rows) per batch
        constexpr int EPL = kBcMaxB / 32;  // elements per lane, at most
        const int64_t ncl = r - (c + 1);   // left columns
        const int64_t rend = (r + L + b < n) ? r + L + b : n;
        const int64_t nrr = rend - (r + L);  // right rows
        const int64_t nbl = (ncl + CB - 1) / CB, nbr = (nrr + CB - 1) / CB;
        for (int64_t bi = warp - 4; bi < nbl + nbr; bi += nw - 4) {
          const bool left = bi < nbl;
          const int64_t first = left ? c + 1 + bi * CB : r + L + (bi - nbl) * CB;
          const int64_t last = left ? r : rend;  // exclusive
          T x[CB][EPL];
#pragma unroll
          for (int q = 0; q < CB; ++q)
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
              const int t = lane + 32 * e;
              const int64_t k = first + q;
              x[q][e] = (k < last && t < L) ? ldw(left ? bat(a, r + t, k) : bat(a, k, r + t)) : O::zero();
            }
#pragma unroll
          for (int q = 0; q < CB; ++q) {
            const int64_t k = first + q;
            T wsum = O::zero();
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
              const int t = lane + 32 * e;
              if (t < L) wsum = left ? O::fma_(O::conj(sv[t]), x[q][e], wsum) : O::fma_(x[q][e], sv[t], wsum);
            }
            wsum = warp_sum(wsum);
            if (k >= last) continue;
            const T f = O::mul(left ? ctau : tau, wsum);
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
              const int t = lane + 32 * e;
              if (t < L) {
                if (left) stw(bat(a, r + t, k), sub(x[q][e], O::mul(f, sv[t])));
                else stw(bat(a, k, r + t), sub(x[q][e], O::mul(f, O::conj(sv[t]))));
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
        for (int t = bt; t < L; t += 128) {
          T acc = O::zero();
          for (int s2 = 0; s2 < L; ++s2) acc = O::fma_(sD[t + s2 * b], sv[s2], acc);
          sy[t] = acc;
        }
        bar_sub(128);
        double al = 0.0;  // v^H y (real)
        for (int t = 0; t < L; ++t) {
          const T p2 = O::mul(O::conj(sv[t]), sy[t]);
          al += O::re(p2);
        }
        const double tt2 = O::re(tau) * O::re(tau) + O::im(tau) * O::im(tau);
        const double cfac = tt2 * al;
        for (int idx = bt; idx < L * L; idx += 128) {
          const int t = idx % L, s2 = idx / L;
          if (t < s2) continue;
          T dv = sD[t + s2 * b];
          dv = sub(dv, O::mul(O::mul(tau, sy[t]), O::conj(sv[s2])));
          dv = sub(dv, O::mul(O::mul(ctau, sv[t]), O::conj(sy[s2])));
          dv = add(dv, O::mul(O::make(cfac, 0.0), O::mul(sv[t], O::conj(sv[s2]))));
          if (t == s2) dv = O::make(O::re(dv), 0.0);
          stw(bat(a, r + t, r + s2), dv);
        }
      }
      __syncthreads();
      // sweep j of stage i is done: its entries are final for the next stage
      // (the barrier above orders every thread's stores before this release)
      if (tid == 0) st_release(mine, j + 1);
    }
    if (abandoned && tid == 0) st_release(mine, kPoison);
    __syncthreads();
  }
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
