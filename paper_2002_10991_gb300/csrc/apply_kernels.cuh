// Kernels of the tridiagonal -> band back-transformation (Eq. 6d).
//
//   relayout_kernel  canonical store -> sweep-major store (tau folded in)
//   apply_kernel     applies every reflector to the columns of q (Eq. 8)
//
// Design (GB300): FP64 runs at 2 DFMA/clock/SM, one warp instruction per 64
// clocks per sub-partition, and a single warp with a dependent FMA chain
// already saturates it. So the kernel spends its FP64 issue slots on the
// 2L FMAs per column that Eq. 8 needs and on nothing else: one lane owns one
// column (dot product and update are serial per lane; no cross-lane
// reductions, which would cost extra FP64 adds), and parallelism beyond the
// columns comes from running several sweeps of a strip at once (see
// schedule.cuh). Rows of the 32-column strip live in a shared-memory ring
// indexed [row % ring][lane] (conflict-free 8/16-byte lane accesses); rows
// stream in through cp.async and are written back once the last sweep of
// the epoch has passed them. Reflectors stream per warp into double-buffered
// shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "schedule.cuh"

namespace tbbt {

struct alignas(16) zdouble {
  double re, im;
};

// ---------------------------------------------------------------------------
// arithmetic of one element type
// ---------------------------------------------------------------------------
template <typename T>
struct Arith;

template <>
struct Arith<double> {
  // s += conj(v) * x
  static __device__ __forceinline__ void dot(double &s, double v, double x) { s = fma(v, x, s); }
  // u = tau * s
  static __device__ __forceinline__ double scale(double tau, double s) { return tau * s; }
  // x -= u * v
  static __device__ __forceinline__ void axpy(double &x, double u, double v) { x = fma(-u, v, x); }
  static __device__ __forceinline__ void sub(double &x, double u) { x -= u; }
  static __device__ __forceinline__ double zero() { return 0.0; }
};

template <>
struct Arith<zdouble> {
  static __device__ __forceinline__ void dot(zdouble &s, zdouble v, zdouble x) {
    s.re = fma(v.re, x.re, s.re);
    s.re = fma(v.im, x.im, s.re);
    s.im = fma(v.re, x.im, s.im);
    s.im = fma(-v.im, x.re, s.im);
  }
  static __device__ __forceinline__ zdouble scale(zdouble t, zdouble s) {
    zdouble u;
    u.re = fma(t.re, s.re, -t.im * s.im);
    u.im = fma(t.re, s.im, t.im * s.re);
    return u;
  }
  static __device__ __forceinline__ void axpy(zdouble &x, zdouble u, zdouble v) {
    x.re = fma(-u.re, v.re, x.re);
    x.re = fma(u.im, v.im, x.re);
    x.im = fma(-u.re, v.im, x.im);
    x.im = fma(-u.im, v.re, x.im);
  }
  static __device__ __forceinline__ void sub(zdouble &x, zdouble u) {
    x.re -= u.re;
    x.im -= u.im;
  }
  static __device__ __forceinline__ zdouble zero() { return zdouble{0.0, 0.0}; }
};

// ---------------------------------------------------------------------------
// store re-layout
// ---------------------------------------------------------------------------
// The canonical store numbers reflectors in generation order (stage-major).
// The apply kernel reads them sweep-major: sweep j, stages imax(j) .. 0, so a
// warp streams consecutive reflectors of its sweep from one contiguous
// range. Entry layout (ldv = b rounded up to even, 16-byte aligned):
//   [tau, v1, v2, ..., v_{L-1}, 0, ...]      (v0 = 1 is implicit)
// stage_off[s] = generation index of reflector (s, 0).
template <typename T>
__global__ void relayout_kernel(const T *__restrict__ hh_v, const T *__restrict__ hh_tau,
                                const int64_t *__restrict__ stage_off, StoreGeom g, int32_t ldv,
                                T *__restrict__ out) {
  const int64_t K = g.num_reflectors();
  const int32_t J = g.num_sweeps();
  // one warp per destination entry
  int64_t entry = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (entry >= K) return;
  // find sweep j with sweep_offset(j) <= entry < sweep_offset(j+1)
  int32_t lo = 0, hi = J - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (g.sweep_offset(mid) <= entry)
      lo = mid;
    else
      hi = mid - 1;
  }
  int32_t j = lo;
  int32_t s = g.imax(j) - (int32_t)(entry - g.sweep_offset(j));
  int64_t k = stage_off[s] + j;
  int32_t L = g.len(s, j);
  const T *src = hh_v + k * g.b;
  T *dst = out + entry * ldv;
  for (int32_t t = lane; t < ldv; t += 32) {
    T val = Arith<T>::zero();
    if (t == 0)
      val = hh_tau[k];
    else if (t < L)
      val = src[t];
    dst[t] = val;
  }
}

// ---------------------------------------------------------------------------
// async-copy helpers (sm_80+ cp.async; completion by wait_all + barrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst_smem, const void *src_gmem) {
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst_smem)), "l"(src_gmem));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst_smem)), "l"(src_gmem));
  }
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Shared-memory load the compiler may not merge with other loads of the same
// address (keeps reflector entries from being cached in registers across the
// unrolled loops of the register-window variant, which would exhaust them).
__device__ __forceinline__ double lds_f64(const double *p) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];\n" : "=d"(v) : "r"(smem_u32(p)));
  return v;
}

// ---------------------------------------------------------------------------
// the apply kernel
// ---------------------------------------------------------------------------
// Work is split into units (strip of 32 columns, epoch of G sweeps), claimed
// by persistent blocks from an atomic counter in epoch-major order. Epoch e
// of a strip reads the rows epoch e-1 has finished; instead of waiting for the
// whole epoch, it follows it down the column: epoch e-1 publishes after
// every step the lowest row it has written back for good ("released"), and
// epoch e waits (bounded) until the rows it is about to load are released.
// A unit only ever waits for a unit with a smaller index, which was claimed
// earlier by a block that is already running, so the pipeline cannot
// deadlock, and all SMs stay busy even when the strips are fewer than SMs.
struct ApplyArgs {
  const void *vstore;  // sweep-major store, ldv elements per reflector
  void *q;
  int64_t ldq;
  StoreGeom g;
  int32_t nev;
  int32_t ldv;
  int32_t G;       // sweeps (warps) per block
  int32_t NB;      // stages per step
  int32_t ring;    // rows in the shared-memory ring
  int32_t strips;  // ceil(nev / 32)
  int32_t units;   // strips * epochs
  int *flags;      // per unit: lowest released row (INT_MAX at start), kPoison if abandoned
  unsigned *counter;
  int *err;
  long long timeout_ns;
  int withhold;  // test hook: unit whose progress is never published (-1: none)
};

constexpr int kPoison = -2;
constexpr int kMaxPrefetch = 4;  // rows-per-step * 32 <= kMaxPrefetch * threads

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// Bounded wait until the unit behind `flag` has released every row >= need.
// Returns 0 when it has, 1 if the producer was abandoned, an error was
// recorded elsewhere, or the wait timed out (which it records in *err).
__device__ inline int wait_released_raw(int *err, long long timeout_ns, const int *flag, int need) {
  long long t0 = globaltimer_ns();
  for (unsigned it = 0;; ++it) {
    int v = ld_acquire(flag);
    if (v == kPoison) return 1;
    if (v <= need) return 0;
    if (*(volatile int *)err != 0) return 1;
    if (globaltimer_ns() - t0 > timeout_ns) {
      atomicCAS(err, 0, 4 /* TBBT_ETIMEOUT */);
      return 1;
    }
    __nanosleep(it < 64 ? 64 : 512);
  }
}

__device__ __forceinline__ int wait_released(const ApplyArgs &a, const int *flag, int need) {
  return wait_released_raw(a.err, a.timeout_ns, flag, need);
}

// Element of ring slot sl (row sl of the ring) and strip column c. The
// lane-pair complex kernel (SWZ) moves the columns of odd slots by four
// (64 bytes): the two lanes of a pair touch adjacent rows of one column at
// the same time, which would otherwise fall on the same shared-memory banks.
template <bool SWZ>
__device__ __forceinline__ int64_t ring_slot(int32_t sl, int32_t c) {
  return (int64_t)sl * 32 + (SWZ ? (c ^ ((sl & 1) << 2)) : c);
}

template <typename T>
__device__ __forceinline__ T ld_cg(const T *p);
template <>
__device__ __forceinline__ double ld_cg<double>(const double *p) {
  return __ldcg(p);
}
template <>
__device__ __forceinline__ zdouble ld_cg<zdouble>(const zdouble *p) {
  double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return zdouble{v.x, v.y};
}

// Rows [r0, r1) of the strip, global -> ring, synchronously (L2 path: rows
// may have been written by another SM). Columns >= nev read as zero.
template <typename T, bool SWZ = false>
__device__ __forceinline__ void load_rows_now(const ApplyArgs &a, T *ring, int32_t r0, int32_t r1, int32_t c0) {
  const int32_t nrows = r1 - r0;
  if (nrows <= 0) return;
  const T *q = reinterpret_cast<const T *>(a.q);
  for (int32_t idx = threadIdx.x; idx < nrows * 32; idx += blockDim.x) {
    int32_t c = idx / nrows;
    int32_t r = r0 + (idx - c * nrows);
    int32_t col = c0 + c;
    ring[ring_slot<SWZ>(r % a.ring, c)] = col < a.nev ? ld_cg(q + (int64_t)col * a.ldq + r) : Arith<T>::zero();
  }
}

// The same split in two: issue the loads into registers now, write them to
// the ring after the step's arithmetic (hides the memory latency).
template <typename T, bool SWZ = false>
struct RowPrefetch {
  T val[kMaxPrefetch];
  __device__ __forceinline__ void issue(const ApplyArgs &a, int32_t r0, int32_t r1, int32_t c0) {
    const int32_t nrows = r1 - r0;
    const T *q = reinterpret_cast<const T *>(a.q);
#pragma unroll
    for (int i = 0; i < kMaxPrefetch; ++i) {
      int32_t idx = threadIdx.x + i * blockDim.x;
      if (nrows > 0 && idx < nrows * 32) {
        int32_t c = idx / nrows;
        int32_t r = r0 + (idx - c * nrows);
        int32_t col = c0 + c;
        val[i] = col < a.nev ? ld_cg(q + (int64_t)col * a.ldq + r) : Arith<T>::zero();
      }
    }
  }
  __device__ __forceinline__ void commit(const ApplyArgs &a, T *ring, int32_t r0, int32_t r1) {
    const int32_t nrows = r1 - r0;
#pragma unroll
    for (int i = 0; i < kMaxPrefetch; ++i) {
      int32_t idx = threadIdx.x + i * blockDim.x;
      if (nrows > 0 && idx < nrows * 32) {
        int32_t c = idx / nrows;
        int32_t r = r0 + (idx - c * nrows);
        ring[ring_slot<SWZ>(r % a.ring, c)] = val[i];
      }
    }
  }
};

// Rows [r0, r1): ring -> global.
template <typename T, bool SWZ = false>
__device__ __forceinline__ void store_rows(const ApplyArgs &a, const T *ring, int32_t r0, int32_t r1, int32_t c0) {
  const int32_t nrows = r1 - r0;
  if (nrows <= 0) return;
  T *q = reinterpret_cast<T *>(a.q);
  const int32_t total = nrows * 32;
  for (int32_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int32_t c = idx / nrows;
    int32_t r = r0 + (idx - c * nrows);
    int32_t col = c0 + c;
    if (col < a.nev) q[(int64_t)col * a.ldq + r] = ring[ring_slot<SWZ>(r % a.ring, c)];
  }
}

// Reflector entries of warp w for its block at step t -> its buffer slot
// (read-only data: asynchronous copies, completed by wait_all + barrier).
template <typename T>
__device__ __forceinline__ void load_reflectors(const ApplyArgs &a, const Epoch &ep, T *vbuf_w, int32_t w,
                                                int32_t t, int li, int nl) {
  int32_t hi, lo;
  warp_stages(a.g, ep, w, t, &hi, &lo);
  if (hi < lo) return;
  const int32_t j = ep.j0 + w;
  const int32_t sig = ep.sig_top - (t - w) * ep.nb;
  const T *src = reinterpret_cast<const T *>(a.vstore) + (a.g.sweep_offset(j) + (a.g.imax(j) - hi)) * a.ldv;
  T *dst = vbuf_w + (int64_t)(t & 1) * ep.nb * a.ldv + (int64_t)(sig - hi) * a.ldv;
  const int32_t nchunks = (hi - lo + 1) * a.ldv * (int32_t)sizeof(T) / 16;
  const char *s8 = reinterpret_cast<const char *>(src);
  char *d8 = reinterpret_cast<char *>(dst);
  for (int32_t c = li; c < nchunks; c += nl) cp_async<16>(d8 + 16 * c, s8 + 16 * c);
}

// Eq. 8 for one reflector on one column: x[r:r+L] -= tau * v * (v^H x[r:r+L]).
template <typename T>
__device__ __forceinline__ void apply_one(T *col, int32_t ring, int32_t r, int32_t L, const T *ent) {
  int32_t base = r % ring;
  T s = col[(int64_t)base * 32];
  {
    int32_t sl = base;
#pragma unroll 4
    for (int32_t t = 1; t < L; ++t) {
      sl = (sl + 1 == ring) ? 0 : sl + 1;
      Arith<T>::dot(s, ent[t], col[(int64_t)sl * 32]);
    }
  }
  const T u = Arith<T>::scale(ent[0], s);
  {
    T x0 = col[(int64_t)base * 32];
    Arith<T>::sub(x0, u);
    col[(int64_t)base * 32] = x0;
    int32_t sl = base;
#pragma unroll 4
    for (int32_t t = 1; t < L; ++t) {
      sl = (sl + 1 == ring) ? 0 : sl + 1;
      T x = col[(int64_t)sl * 32];
      Arith<T>::axpy(x, u, ent[t]);
      col[(int64_t)sl * 32] = x;
    }
  }
}

// Eq. 8 for one reflector on one complex column (strip column c), by a pair
// of lanes: lane h of the pair takes the rows t = h, h + 2, h + 4, ... of
// the window (v_0 = 1, so the row-0 term of lane 0 is x_0 itself), and the
// two partial sums of v^H x are added with one exchange inside the pair
// (both lanes form the same sum: addition commutes). Each lane's dependent
// chain is half as long, and a 32-column strip takes two warps per sweep,
// two per SM sub-partition. The ring is swizzled (ring_slot<true>): at every
// step the lanes of a pair touch adjacent rows, on different banks.
__device__ __forceinline__ void apply_pair(zdouble *ring, int32_t nring, int32_t c, int32_t r, int32_t L,
                                           const zdouble *ent, int h) {
  const int32_t base = r % nring;
  const int32_t t0 = h ? 1 : 2;
  int32_t sl0 = base + t0;
  if (sl0 >= nring) sl0 -= nring;
  zdouble s = h ? zdouble{0.0, 0.0} : ring[ring_slot<true>(base, c)];
  {
    int32_t sl = sl0;
#pragma unroll 4
    for (int32_t t = t0; t < L; t += 2) {
      Arith<zdouble>::dot(s, ent[t], ring[ring_slot<true>(sl, c)]);
      sl += 2;
      if (sl >= nring) sl -= nring;
    }
  }
  s.re += __shfl_xor_sync(0xffffffffu, s.re, 1);
  s.im += __shfl_xor_sync(0xffffffffu, s.im, 1);
  const zdouble u = Arith<zdouble>::scale(ent[0], s);
  if (!h) {
    zdouble x0 = ring[ring_slot<true>(base, c)];
    Arith<zdouble>::sub(x0, u);
    ring[ring_slot<true>(base, c)] = x0;
  }
  {
    int32_t sl = sl0;
#pragma unroll 4
    for (int32_t t = t0; t < L; t += 2) {
      zdouble x = ring[ring_slot<true>(sl, c)];
      Arith<zdouble>::axpy(x, u, ent[t]);
      ring[ring_slot<true>(sl, c)] = x;
      sl += 2;
      if (sl >= nring) sl -= nring;
    }
  }
  // the next reflector starts one row up: each lane then takes the rows the
  // other lane just wrote
  __syncwarp();
}

// Register-window variant of the stage loop for real data and b = B (32 or
// 64): the lane keeps rows r .. r+B-1 of its column in registers, so neither
// the dot-product chain nor the update touches shared memory. Per stage the
// lane reads the one new top row from the ring, applies Eq. 8, and writes the
// row that leaves the window at the bottom back to the ring (the next sweep
// reads it there). The window moves up one row per stage; the move is folded
// into the update, which runs from the bottom of the window up and writes
// each updated element into the register of the element below it (just
// consumed), so the window never needs a second copy. Rows >= n are held as
// zeros and meet zero reflector entries (the store is zero-padded to
// ldv = B), so they stay zero and are never written. Terms are summed and
// updated exactly as in apply_one, so both variants give the same bits.
template <int B>
__device__ __forceinline__ void apply_stages_regwin(double (&x)[B], double *ring_col, int32_t ring, const StoreGeom &g,
                                                    int32_t j, int32_t hi, int32_t lo, const double *vb,
                                                    int32_t sig, int32_t ldv) {
  const int32_t first = g.imax(j);
  for (int32_t s = hi; s >= lo; --s) {
    const int32_t r = g.row(s, j);
    if (s == first) {
      // first stage of the sweep: fill the whole window
      int32_t sl = r % ring;
#pragma unroll
      for (int32_t t = 0; t < B; ++t) {
        x[t] = (r + t < g.n) ? ring_col[(int64_t)sl * 32] : 0.0;
        sl = (sl + 1 == ring) ? 0 : sl + 1;
      }
    } else {
      x[0] = ring_col[(int64_t)(r % ring) * 32];  // rows r+1 .. r+B-1 are already in x[1..]
    }
    const double *ent = vb + (int64_t)(sig - s) * ldv;
    // Entries are loaded PF iterations ahead of their use (explicit software
    // pipeline: the loads are in-order, so this is what hides their latency).
    constexpr int PF = 4;
    double acc = x[0];
    {
      double v[PF];
#pragma unroll
      for (int k = 0; k < PF; ++k) v[k] = (1 + k < B) ? lds_f64(ent + 1 + k) : 0.0;
#pragma unroll
      for (int32_t t = 1; t < B; ++t) {
        const double vt = v[(t - 1) % PF];
        if (t + PF < B) v[(t - 1) % PF] = lds_f64(ent + t + PF);
        acc = fma(vt, x[t], acc);
      }
    }
    const double u = lds_f64(ent) * acc;
    if (s > 0) {
      // entries in the order the bottom-up update uses them: ent[B-1], ent[B-2], ..., ent[1]
      double w[PF];
#pragma unroll
      for (int k = 0; k < PF; ++k) w[k] = lds_f64(ent + B - 1 - k);
      const double out = fma(-u, w[0], x[B - 1]);  // row r+B-1 leaves the window
      if (PF <= B - 2) w[0] = lds_f64(ent + B - 1 - PF);
      if (r + B - 1 < g.n) ring_col[(int64_t)((r + B - 1) % ring) * 32] = out;
#pragma unroll
      for (int32_t k = 1; k <= B - 2; ++k) {  // element t = B - k takes entry ent[t-1]
        const double wk = w[k % PF];
        if (k + PF <= B - 2) w[k % PF] = lds_f64(ent + B - 1 - k - PF);
        x[B - k] = fma(-u, wk, x[B - k - 1]);
      }
      x[1] = x[0] - u;
    } else {
      // stage 0 ends the sweep: update in place; the whole window is final
      x[0] -= u;
#pragma unroll
      for (int32_t t = 1; t < B; ++t) x[t] = fma(-u, lds_f64(ent + t), x[t]);
      int32_t sl = r % ring;
#pragma unroll
      for (int32_t t = 0; t < B; ++t) {
        if (r + t < g.n) ring_col[(int64_t)sl * 32] = x[t];
        sl = (sl + 1 == ring) ? 0 : sl + 1;
      }
    }
  }
}

// 16-byte shared-memory load the compiler may not merge or hoist (as lds_f64).
__device__ __forceinline__ zdouble lds_z(const zdouble *p) {
  double re, im;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(re), "=d"(im) : "r"(smem_u32(p)));
  return zdouble{re, im};
}

// Register window for complex data and b = 2H, a lane pair per column
// (strip column c): lane h of the pair keeps rows r + H h .. r + H h + H - 1
// of its column's window in registers, so the dot product and the update
// run on registers, and the two halves of v^H x are added by one exchange
// inside the pair. The window moves up one row per stage; the update runs
// from the bottom of each half up and moves every element one register down:
// the element that leaves the lower lane's half enters the upper lane's by
// one exchange, the upper lane's last element leaves the window for the ring
// (the next sweep reads it there), and the lower lane takes the new top row
// from the ring at the next stage. Rows >= n are held as zeros and meet zero
// reflector entries, so they stay zero and are never written.
template <int H>
__device__ __forceinline__ void apply_stages_regwin_pair(zdouble (&x)[H], zdouble *ring, int32_t nring, int32_t c,
                                                         const StoreGeom &g, int32_t j, int32_t hi, int32_t lo,
                                                         const zdouble *vb, int32_t sig, int32_t ldv, int h) {
  constexpr int B = 2 * H;
  constexpr int PF = 4;
  const int32_t first = g.imax(j);
  const zdouble one{1.0, 0.0};
  for (int32_t s = hi; s >= lo; --s) {
    const int32_t r = g.row(s, j);
    if (s == first) {
      // first stage of the sweep: fill this lane's half of the window
      int32_t sl = (r + H * h) % nring;
#pragma unroll
      for (int32_t t = 0; t < H; ++t) {
        x[t] = (r + H * h + t < g.n) ? ring[ring_slot<true>(sl, c)] : Arith<zdouble>::zero();
        sl = (sl + 1 == nring) ? 0 : sl + 1;
      }
    } else if (h == 0) {
      x[0] = ring[ring_slot<true>(r % nring, c)];  // the upper lane's x[0] came by exchange
    }
    const zdouble *ent = vb + (int64_t)(sig - s) * ldv;  // [tau, v_1, ..., v_{B-1}]
    const zdouble *eh = ent + H * h;                       // this lane's entries: v_{H h + t}
    // v^H x over this lane's half (v_0 = 1: the lower lane's first entry)
    zdouble acc = Arith<zdouble>::zero();
    {
      zdouble v[PF];
#pragma unroll
      for (int k = 0; k < PF; ++k) v[k] = (k == 0 && h == 0) ? one : lds_z(eh + k);
#pragma unroll
      for (int32_t t = 0; t < H; ++t) {
        const zdouble vt = v[t % PF];
        if (t + PF < H) v[t % PF] = lds_z(eh + t + PF);
        Arith<zdouble>::dot(acc, vt, x[t]);
      }
    }
    acc.re += __shfl_xor_sync(0xffffffffu, acc.re, 1);
    acc.im += __shfl_xor_sync(0xffffffffu, acc.im, 1);
    const zdouble u = Arith<zdouble>::scale(lds_z(ent), acc);
    if (s > 0) {
      // bottom-up, entries v_{H h + H - 1} .. v_{H h}
      zdouble w[PF];
#pragma unroll
      for (int k = 0; k < PF; ++k) w[k] = lds_z(eh + H - 1 - k);
      zdouble out = x[H - 1];
      Arith<zdouble>::axpy(out, u, w[0]);  // this half's last row leaves it
      if (PF <= H - 1) w[0] = lds_z(eh + H - 1 - PF);
#pragma unroll
      for (int32_t k = 1; k <= H - 1; ++k) {  // element t = H - 1 - k moves to register t + 1
        zdouble wk = w[k % PF];
        if (k + PF <= H - 1) w[k % PF] = (h == 0 && H - 1 - k - PF == 0) ? one : lds_z(eh + H - 1 - k - PF);
        if (h == 0 && k == H - 1) wk = one;  // v_0
        zdouble xt = x[H - 1 - k];
        Arith<zdouble>::axpy(xt, u, wk);
        x[H - k] = xt;
      }
      zdouble in;
      in.re = __shfl_xor_sync(0xffffffffu, out.re, 1);
      in.im = __shfl_xor_sync(0xffffffffu, out.im, 1);
      if (h == 1) {
        x[0] = in;  // the lower half's last row is now the upper half's first
        if (r + B - 1 < g.n) ring[ring_slot<true>((r + B - 1) % nring, c)] = out;
      }
    } else {
      // stage 0 ends the sweep: update in place; the whole window is final
#pragma unroll
      for (int32_t t = 0; t < H; ++t) {
        const zdouble vt = (h == 0 && t == 0) ? one : lds_z(eh + t);
        Arith<zdouble>::axpy(x[t], u, vt);
      }
      int32_t sl = (r + H * h) % nring;
#pragma unroll
      for (int32_t t = 0; t < H; ++t) {
        if (r + H * h + t < g.n) ring[ring_slot<true>(sl, c)] = x[t];
        sl = (sl + 1 == nring) ? 0 : sl + 1;
      }
    }
  }
}

// One work unit: strip c0 .. c0+31 of the problem described by `a`, epoch e
// (sweeps e*G .. e*G+G-1). `myflag` receives this unit's progress, `prevflag`
// is the previous epoch's of the same strip (null for epoch 0). `s_stop` is a
// shared word used to broadcast waits that gave up. Returns false if the
// unit was abandoned.
template <typename T, int BW>
__device__ __forceinline__ bool process_unit(const ApplyArgs &a, int32_t e, int32_t c0, int *myflag,
                                             const int *prevflag, bool publish, unsigned char *smem_raw,
                                             int *s_stop) {
  T *ring = reinterpret_cast<T *>(smem_raw);
  T *vbuf = ring + (int64_t)a.ring * 32;
  const int lane = threadIdx.x & 31;
  // BW < 0 (complex): two warps per sweep; warp half cs of the pair takes
  // columns 16 cs .. 16 cs + 15, a lane pair per column
  const int w = BW < 0 ? (threadIdx.x >> 6) : (threadIdx.x >> 5);
  const int cs = (threadIdx.x >> 5) & 1;
  const int li = BW < 0 ? lane + 32 * cs : lane, nl = BW < 0 ? 64 : 32;
  const StoreGeom &g = a.g;
  T *vbuf_w = vbuf + (int64_t)w * 2 * a.NB * a.ldv;
  constexpr bool SWZ = BW < 0;  // the lane-pair kernel's ring is swizzled
  T *mycol = ring + lane;       // (shared-memory window and register-window kernels)
  const int32_t pcol = 16 * cs + (lane >> 1);  // lane pairs: strip column of this pair
  double xw[BW > 0 ? BW : 1];  // register window of the lane's column (BW > 0)
  (void)xw;
  zdouble xz[BW < -1 ? -BW / 2 : 1];  // complex register window: this lane's half (BW = -b)
  (void)xz;
  const Epoch ep = make_epoch(g, e, a.G, a.NB);

  // prologue: rows needed at step 0 and the reflectors of step 0
  int32_t top = step_min_row(g, ep, 0);
  if (threadIdx.x == 0) *s_stop = prevflag ? wait_released(a, prevflag, top) : 0;
  __syncthreads();
  bool abandoned = *s_stop != 0;
  if (!abandoned) {
    load_rows_now<T, SWZ>(a, ring, top, g.n, c0);
    load_reflectors<T>(a, ep, vbuf_w, w, 0, li, nl);
    cp_async_wait_all();
    __syncthreads();
    int32_t released = g.n;  // rows >= released are back in global memory
    RowPrefetch<T, SWZ> pf;
    for (int32_t t = 0; t < ep.nsteps; ++t) {
      // rows no warp touches from step t on go back to global memory
      int32_t live = rows_live_max(g, ep, t);
      int32_t rel = live + 1 > top ? live + 1 : top;
      if (rel < released) {
        store_rows<T, SWZ>(a, ring, rel, released, c0);
        released = rel;
      }
      // rows of step t+1 must have been released by the previous epoch
      const int32_t ntop = step_min_row(g, ep, t + 1);
      if (threadIdx.x == 0) *s_stop = (prevflag && ntop < top) ? wait_released(a, prevflag, ntop) : 0;
      __syncthreads();
      if (*s_stop) {
        abandoned = true;
        break;
      }
      if (threadIdx.x == 0 && publish) st_release(myflag, released);
      pf.issue(a, ntop, top, c0);
      load_reflectors<T>(a, ep, vbuf_w, w, t + 1, li, nl);
      // this warp's stages of step t
      int32_t hi, lo;
      warp_stages(g, ep, w, t, &hi, &lo);
      if (hi >= lo) {
        const int32_t j = ep.j0 + w;
        const int32_t sig = ep.sig_top - (t - w) * ep.nb;
        const T *vb = vbuf_w + (int64_t)(t & 1) * ep.nb * a.ldv;
        if constexpr (BW > 0) {
          apply_stages_regwin<BW>(xw, mycol, a.ring, g, j, hi, lo, vb, sig, a.ldv);
        } else if constexpr (BW < -1) {
          apply_stages_regwin_pair<-BW / 2>(xz, ring, a.ring, pcol, g, j, hi, lo, vb, sig, a.ldv, lane & 1);
        } else if constexpr (BW < 0) {
          for (int32_t s = hi; s >= lo; --s)
            apply_pair(ring, a.ring, pcol, g.row(s, j), g.len(s, j), vb + (int64_t)(sig - s) * a.ldv, lane & 1);
        } else {
          for (int32_t s = hi; s >= lo; --s)
            apply_one<T>(mycol, a.ring, g.row(s, j), g.len(s, j), vb + (int64_t)(sig - s) * a.ldv);
        }
      }
      pf.commit(a, ring, ntop, top);
      top = ntop;
      cp_async_wait_all();
      __syncthreads();
    }
    if (!abandoned) {
      // the rest of the strip is final for this epoch
      store_rows<T, SWZ>(a, ring, top, released, c0);
      __syncthreads();
      if (threadIdx.x == 0 && publish) st_release(myflag, top);
    }
  }
  if (abandoned) {
    cp_async_wait_all();
    if (threadIdx.x == 0) st_release(myflag, kPoison);
  }
  return !abandoned;
}

// Threads per block: real register windows 8 warps at most, the complex
// register window 4 sweeps (8 warps), the lane-pair and shared-memory
// windows 16 warps.
template <typename T, int BW>
__global__ void __launch_bounds__((BW > 0 || BW < -1) ? 256 : 512, 1) apply_kernel(ApplyArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_unit;
  __shared__ int s_stop;
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = (int)atomicAdd(a.counter, 1u);
      s_stop = (*(volatile int *)a.err != 0);
    }
    __syncthreads();
    const int u = s_unit;
    if (u >= a.units || s_stop) break;
    const int32_t e = u / a.strips;
    const int32_t c0 = (u - e * a.strips) * 32;
    process_unit<T, BW>(a, e, c0, a.flags + u, e > 0 ? a.flags + (u - a.strips) : nullptr, u != a.withhold,
                        smem_raw, &s_stop);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// batched form: many problems, one persistent launch
// ---------------------------------------------------------------------------
// Every problem keeps its own ApplyArgs (geometry, store, q, step length,
// ring size); the units of all problems form one queue whose order keeps
// every dependency pointing to an earlier unit (epoch-major across problems,
// longest problems first within an epoch), so the same no-deadlock argument
// holds. A block copies the arguments of its unit's problem into shared
// memory and dispatches on the problem's kind.
enum BatchKind : int32_t { kRealGeneric = 0, kReal32 = 1, kComplex = 3 };

struct BatchProblem {
  ApplyArgs a;  // flags/counter/err/units/strips fields unused here
  int32_t kind;
  int32_t pad;
};

struct BatchUnit {
  int32_t problem, strip, epoch, prev;  // prev: queue index of (problem, strip, epoch-1), or -1
};

struct BatchArgs {
  const BatchProblem *problems;
  const BatchUnit *units;
  int32_t nunits;
  int *flags;  // one per queue entry
  unsigned *counter;
  int *err;
};

__global__ void __launch_bounds__(256, 1) batch_kernel(BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_unit;
  __shared__ int s_stop;
  __shared__ BatchProblem s_prob;
  __shared__ BatchUnit s_u;
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = (int)atomicAdd(b.counter, 1u);
      s_stop = (*(volatile int *)b.err != 0);
    }
    __syncthreads();
    const int u = s_unit;
    if (u >= b.nunits || s_stop) break;
    // stage this unit's problem arguments in shared memory (word copy)
    {
      const int *src = reinterpret_cast<const int *>(b.problems + b.units[u].problem);
      int *dst = reinterpret_cast<int *>(&s_prob);
      for (int i = threadIdx.x; i < (int)(sizeof(BatchProblem) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
      if (threadIdx.x == 0) s_u = b.units[u];
    }
    __syncthreads();
    ApplyArgs a = s_prob.a;
    a.err = b.err;
    const int kind = s_prob.kind;
    const BatchUnit un = s_u;
    int *myflag = b.flags + u;
    const int *prevflag = un.prev >= 0 ? b.flags + un.prev : nullptr;
    const int32_t c0 = un.strip * 32;
    // (b = 64 real problems take the shared-memory window here: the 64-row
    // register window would not fit beside the other paths of this kernel.
    // Complex problems take one lane per column: two blocks of one warp per
    // sweep already share an SM here, which is what lane pairs buy the
    // single-problem kernel.)
    if (kind == kReal32)
      process_unit<double, 32>(a, un.epoch, c0, myflag, prevflag, true, smem_raw, &s_stop);
    else if (kind == kComplex)
      process_unit<zdouble, 0>(a, un.epoch, c0, myflag, prevflag, true, smem_raw, &s_stop);
    else
      process_unit<double, 0>(a, un.epoch, c0, myflag, prevflag, true, smem_raw, &s_stop);
    __syncthreads();
  }
}

}  // namespace tbbt
