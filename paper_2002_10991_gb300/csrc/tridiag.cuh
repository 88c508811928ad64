// Tridiagonal eigensolver for the nev lowest eigenpairs (Eq. 6c): the step
// between the bulge chase (Eq. 6b) and the back-transformation (Eq. 6d).
// ELPA computes only the wanted eigenvectors of the tridiagonal matrix
// (Sec. 2.1); here that is done with O(n * nev) work, the form that suits a
// GPU whose FP64 units are its scarce resource:
//
//  1. te_bounds_kernel: Gershgorin interval, ||T|| and e_i^2 (one block).
//  2. te_bisect_kernel: eigenvalue k by bisection on Sturm counts (the
//     number of negative pivots of the LDL^T factorisation of T - sigma I is
//     the number of eigenvalues below sigma). P threads share one eigenvalue
//     and evaluate P points of its bracket per round (multisection), so a
//     round shrinks the bracket (P + 1)-fold.
//  3. te_invit_kernel: eigenvector k by inverse iteration, one thread per
//     vector: Gaussian elimination with partial pivoting of T - lambda_k I
//     (the factor U has two super-diagonals), then solves from a
//     pseudo-random start, normalised after each. Factors and iterates are
//     stored [row][vector], so each step of the recurrences is one coalesced
//     access across the vectors of a warp.
//  4. te_tight_kernel: in groups of eigenvalues closer than TIGHT_TOL ||T||,
//     independent iterations from nearly equal shifts converge to nearly
//     parallel vectors, and orthogonalising those afterwards would amplify
//     their errors. There every vector after the first is iterated again,
//     its iterate orthogonalised against the group's earlier vectors after
//     every solve (a block per group; the solves run on one thread).
//  5. te_transpose_kernel: [row][vector] -> column-major X.
//  6. te_reorth_kernel: modified Gram-Schmidt (twice) inside each cluster of
//     eigenvalues closer than a fixed fraction of ||T||; a block per cluster.
//     Inverse iteration leaves vectors of well-separated eigenvalues
//     orthogonal to about eps ||T|| / gap; the clusters are where that bound
//     is loose.
#pragma once

#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

namespace tbbt {
namespace te {

constexpr int BOUNDS_THREADS = 256;
constexpr int INVIT_THREADS = 128;
constexpr int REORTH_THREADS = 256;
constexpr int TIGHT_THREADS = 256;
// eigenvalues closer than this fraction of ||T|| (chained) form a cluster
constexpr double CLUSTER_TOL = 1e-4;
// eigenvalues closer than this fraction of ||T|| (chained) form a tight group
constexpr double TIGHT_TOL = 1e-9;
// solves of inverse iteration per vector
constexpr int INVIT_STEPS = 3;

struct Bounds {
  double gl, gu;     // Gershgorin interval, widened
  double tnorm;      // max(|gl|, |gu|)
  double pivmin;     // smallest pivot magnitude allowed in a Sturm count
  double pert;       // replacement of a vanishing pivot in inverse iteration
  double sc;         // power of two with sc * tnorm <= 1 (scale of the FP32 copy)
};

// FP32 phase of the bisection: T sc in single precision (d and e^2), the
// smallest pivot magnitude of its Sturm counts, the bracket width it stops
// at and the margin its brackets get before the FP64 phase checks them.
// A single-precision Sturm count is exact for a matrix within a few units
// of FP32 rounding of T (relative to ||T||, so about 1e-7 ||T||); the
// margin is 2^-16 ||T||-scaled units, far beyond that.
constexpr float PIVMIN32 = 7.8886091e-31f;  // 2^-100
constexpr float STOP32 = 9.5367432e-7f;     // 2^-20
constexpr double MARGIN32 = 1.52587890625e-5;  // 2^-16

// Gershgorin bounds, e2 = e^2, the largest e^2 (one block of BOUNDS_THREADS).
__global__ void te_bounds_kernel(const double *__restrict__ d, const double *__restrict__ e, int32_t n,
                                 double *__restrict__ e2, Bounds *out, float *__restrict__ d32,
                                 float *__restrict__ e232) {
  __shared__ double s_lo[BOUNDS_THREADS], s_hi[BOUNDS_THREADS], s_e2[BOUNDS_THREADS];
  double lo = DBL_MAX, hi = -DBL_MAX, me2 = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double em = i > 0 ? fabs(e[i - 1]) : 0.0;
    const double ep = i + 1 < n ? fabs(e[i]) : 0.0;
    lo = fmin(lo, d[i] - em - ep);
    hi = fmax(hi, d[i] + em + ep);
    if (i + 1 < n) {
      const double s = e[i] * e[i];
      e2[i] = s;
      me2 = fmax(me2, s);
    }
  }
  s_lo[threadIdx.x] = lo;
  s_hi[threadIdx.x] = hi;
  s_e2[threadIdx.x] = me2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_lo[threadIdx.x] = fmin(s_lo[threadIdx.x], s_lo[threadIdx.x + w]);
      s_hi[threadIdx.x] = fmax(s_hi[threadIdx.x], s_hi[threadIdx.x + w]);
      s_e2[threadIdx.x] = fmax(s_e2[threadIdx.x], s_e2[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    Bounds b;
    const double eps = DBL_EPSILON;
    b.tnorm = fmax(fabs(s_lo[0]), fabs(s_hi[0]));
    b.pivmin = DBL_MIN * fmax(1.0, s_e2[0]);
    const double pad = 2.0 * eps * b.tnorm * (double)n + 2.0 * b.pivmin;
    b.gl = s_lo[0] - pad - DBL_MIN;
    b.gu = s_hi[0] + pad + DBL_MIN;
    b.pert = eps * fmax(b.tnorm, DBL_MIN);
    int ex = 0;
    frexp(fmax(b.tnorm, DBL_MIN), &ex);  // tnorm < 2^ex
    b.sc = ldexp(1.0, -ex);
    *out = b;
  }
  __syncthreads();
  const double sc = out->sc;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    d32[i] = (float)(d[i] * sc);
    if (i + 1 < n) e232[i] = (float)(e2[i] * sc * sc);
  }
}

// Number of eigenvalues of T below sigma: negative pivots of T - sigma I =
// L D L^T, q_0 = d_0 - sigma, q_i = d_i - sigma - e_{i-1}^2 / q_{i-1}, a
// pivot of magnitude below pivmin taken as -pivmin.
__device__ __forceinline__ int32_t sturm_count(const double *__restrict__ d, const double *__restrict__ e2,
                                               int32_t n, double sigma, double pivmin) {
  int32_t cnt = 0;
  double q = d[0] - sigma;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int32_t i = 1; i < n; ++i) {
    q = (d[i] - sigma) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

__device__ __forceinline__ int32_t sturm_count32(const float *__restrict__ d, const float *__restrict__ e2,
                                                 int32_t n, float sigma) {
  int32_t cnt = 0;
  float q = d[0] - sigma;
  if (fabsf(q) < PIVMIN32) q = -PIVMIN32;
  cnt += q < 0.0f;
  for (int32_t i = 1; i < n; ++i) {
    q = (d[i] - sigma) - __fdiv_rn(e2[i - 1], q);
    if (fabsf(q) < PIVMIN32) q = -PIVMIN32;
    cnt += q < 0.0f;
  }
  return cnt;
}

// FP32 phase: the multisection of te_bisect_kernel on T sc in single
// precision, down to a bracket of STOP32; writes the bracket widened by
// MARGIN32 on both sides, in the units of T, for the FP64 phase to check.
template <int P>
__global__ void te_bisect32_kernel(const float *__restrict__ d, const float *__restrict__ e2, int32_t n, int32_t nev,
                                   const Bounds *__restrict__ bounds, double *__restrict__ lo_out,
                                   double *__restrict__ hi_out) {
  static_assert(P >= 1 && P <= 32 && (32 % P) == 0, "group size must divide the warp");
  const int32_t lane = threadIdx.x & 31;
  const int32_t g = lane % P;
  const int32_t base = lane - g;
  const int32_t k = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / P);
  const bool active = k < nev;
  const Bounds B = *bounds;
  const unsigned gbits = (P == 32) ? 0xffffffffu : ((1u << P) - 1u);
  float lo = __double2float_rd(B.gl * B.sc), hi = __double2float_ru(B.gu * B.sc);
  bool done = !active;
  for (int round = 0; round < 256; ++round) {
    if (!done) done = hi - lo <= STOP32;
    if (__all_sync(0xffffffffu, done)) break;
    const float sigma = lo + (hi - lo) * ((float)(g + 1) / (float)(P + 1));
    const bool below = done || sturm_count32(d, e2, n, sigma) <= k;
    const unsigned grp = (__ballot_sync(0xffffffffu, below) >> base) & gbits;
    const int32_t lead = (grp == gbits) ? P : __ffs(~grp) - 1;
    const float s_lo = __shfl_sync(0xffffffffu, sigma, base + (lead > 0 ? lead - 1 : 0));
    const float s_hi = __shfl_sync(0xffffffffu, sigma, base + (lead < P ? lead : P - 1));
    if (!done) {
      const float nlo = lead > 0 ? s_lo : lo;
      const float nhi = lead < P ? s_hi : hi;
      if (nlo == lo && nhi == hi) done = true;
      lo = nlo;
      hi = nhi;
    }
  }
  if (active && g == 0) {
    lo_out[k] = ((double)lo - MARGIN32) / B.sc;
    hi_out[k] = ((double)hi + MARGIN32) / B.sc;
  }
}

// Eigenvalue k (0-based, ascending) by multisection: the P threads of a
// group (P divides 32; a warp holds whole groups) evaluate P interior points
// of the bracket [lo, hi], count(lo) <= k < count(hi), and keep the
// sub-interval between the last point of the leading run with count <= k
// and the point after it (so the invariant holds even where rounding makes
// the counts non-monotone). Stops when the bracket is within
// 2 eps max(|lo|, |hi|) + eps ||T||, or cannot shrink.
// With lo0 / hi0 (the FP32 phase's brackets) a group first checks both
// ends with FP64 counts and starts from each end that holds; an end that
// does not hold falls back to the Gershgorin bound.
template <int P>
__global__ void te_bisect_kernel(const double *__restrict__ d, const double *__restrict__ e2, int32_t n,
                                 int32_t nev, const Bounds *__restrict__ bounds, double *__restrict__ w,
                                 const double *__restrict__ lo0, const double *__restrict__ hi0) {
  static_assert(P >= 1 && P <= 32 && (32 % P) == 0, "group size must divide the warp");
  const int32_t lane = threadIdx.x & 31;
  const int32_t g = lane % P;     // index within the group
  const int32_t base = lane - g;  // first lane of the group
  const int32_t k = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / P);
  const bool active = k < nev;
  const Bounds B = *bounds;
  const double eps = DBL_EPSILON;
  const unsigned gbits = (P == 32) ? 0xffffffffu : ((1u << P) - 1u);
  double lo = B.gl, hi = B.gu;
  if (lo0 != nullptr) {
    const double l0 = active ? lo0[k] : 0.0, h0 = active ? hi0[k] : 0.0;
    bool okl, okh;
    if constexpr (P >= 2) {
      const int32_t c = (active && g < 2) ? sturm_count(d, e2, n, g == 0 ? l0 : h0, B.pivmin) : 0;
      okl = __shfl_sync(0xffffffffu, c, base) <= k;
      okh = __shfl_sync(0xffffffffu, c, base + 1) > k;
    } else {
      okl = active && sturm_count(d, e2, n, l0, B.pivmin) <= k;
      okh = active && sturm_count(d, e2, n, h0, B.pivmin) > k;
    }
    if (okl && l0 > lo) lo = l0;
    if (okh && h0 < hi) hi = h0;
  }
  bool done = !active;  // uniform within a group: lo and hi are
  for (int round = 0; round < 512; ++round) {
    if (!done) done = hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + eps * B.tnorm;
    if (__all_sync(0xffffffffu, done)) break;
    const double sigma = lo + (hi - lo) * ((double)(g + 1) / (double)(P + 1));
    const bool below = done || sturm_count(d, e2, n, sigma, B.pivmin) <= k;
    const unsigned grp = (__ballot_sync(0xffffffffu, below) >> base) & gbits;
    // leading run of points with count <= k
    const int32_t lead = (grp == gbits) ? P : __ffs(~grp) - 1;
    const double s_lo = __shfl_sync(0xffffffffu, sigma, base + (lead > 0 ? lead - 1 : 0));
    const double s_hi = __shfl_sync(0xffffffffu, sigma, base + (lead < P ? lead : P - 1));
    if (!done) {
      const double nlo = lead > 0 ? s_lo : lo;
      const double nhi = lead < P ? s_hi : hi;
      if (nlo == lo && nhi == hi) done = true;  // no representable progress
      lo = nlo;
      hi = nhi;
    }
  }
  if (active && g == 0) w[k] = 0.5 * (lo + hi);
}

// splitmix64 finaliser, for the pseudo-random start vectors
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct InvitArgs {
  const double *d, *e;
  int32_t n, nev;
  const double *w;
  const Bounds *bounds;
  // [row][vector] scratch, each n * nev: reciprocal of U's diagonal, U's
  // first and second super-diagonal, multipliers, the iterate; pivots
  // (1 = rows swapped)
  double *u0, *u1, *u2, *lm, *y;
  unsigned char *piv;
};

// Rows whose loads a solve issues together (the recurrences run one
// thread per vector, so the loads of a chunk hide each other's latency).
constexpr int CH = 8;

struct SolveOut {
  double amax;  // largest |y_i|
  double ss;    // sum of y_i^2 (inf if it overflowed)
  double sgn;   // sign of the first entry of largest magnitude
};

// One solve of inverse iteration for vector k, in place on its iterate:
// y <- U^-1 L^-1 P (fin y) with the factors of T - w_k I (fin: a scale
// still owed to the iterate, applied as it is read).
__device__ __forceinline__ SolveOut invit_solve(const InvitArgs &A, int32_t k, double fin) {
  const int32_t n = A.n;
  const size_t ld = (size_t)A.nev;
  auto at = [&](int32_t i) { return (size_t)i * ld + (size_t)k; };
  // forward: apply the row interchanges and multipliers to y
  double yk = A.y[at(0)] * fin;
  for (int32_t i0 = 0; i0 + 1 < n; i0 += CH) {
    double yy[CH], mm[CH];
    unsigned char pp[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int32_t i = i0 + u;
      if (i + 1 < n) {
        yy[u] = A.y[at(i + 1)] * fin;
        mm[u] = A.lm[at(i)];
        pp[u] = A.piv[at(i)];
      }
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int32_t i = i0 + u;
      if (i + 1 < n) {
        double yn = yy[u];
        if (pp[u]) {
          const double t = yk;
          yk = yn;
          yn = t - mm[u] * yk;
        } else {
          yn = yn - mm[u] * yk;
        }
        A.y[at(i)] = yk;
        yk = yn;
      }
    }
  }
  A.y[at(n - 1)] = yk;
  // back substitution with U (reciprocal diagonal, two super-diagonals)
  SolveOut o{0.0, 0.0, 1.0};
  double x1 = 0.0, x2 = 0.0;
  for (int32_t i0 = n - 1; i0 >= 0; i0 -= CH) {
    double yy[CH], a0[CH], a1[CH], a2[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int32_t i = i0 - u;
      if (i >= 0) {
        yy[u] = A.y[at(i)];
        a0[u] = A.u0[at(i)];
        a1[u] = A.u1[at(i)];
        a2[u] = A.u2[at(i)];
      }
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int32_t i = i0 - u;
      if (i >= 0) {
        const double x = (yy[u] - a1[u] * x1 - a2[u] * x2) * a0[u];
        A.y[at(i)] = x;
        // rows run downwards: >= keeps the first (lowest-index) largest entry
        if (fabs(x) >= o.amax) {
          o.amax = fabs(x);
          o.sgn = x < 0.0 ? -1.0 : 1.0;
        }
        o.ss = fma(x, x, o.ss);
        x2 = x1;
        x1 = x;
      }
    }
  }
  return o;
}

// Eigenvector k of T by inverse iteration (one thread per vector).
__global__ void te_invit_kernel(InvitArgs A) {
  const int32_t k = (int32_t)(blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if (k >= A.nev) return;
  const int32_t n = A.n;
  const size_t ld = (size_t)A.nev;
  const double lam = A.w[k];
  const double pert = A.bounds->pert;
  auto at = [&](int32_t i) { return (size_t)i * ld + (size_t)k; };
  // factor T - lam I = P L U with partial pivoting; a pivot below pert in
  // magnitude (T - lam I is singular to working precision there) is
  // replaced by +-pert
  {
    double a = A.d[0] - lam;
    double b = n > 1 ? A.e[0] : 0.0;
    for (int32_t i = 0; i + 1 < n; ++i) {
      const double c = A.e[i];             // row i+1, column i
      const double dn = A.d[i + 1] - lam;  // row i+1, column i+1
      const double bn = i + 2 < n ? A.e[i + 1] : 0.0;
      if (fabs(a) >= fabs(c)) {
        if (fabs(a) < pert) a = a < 0.0 ? -pert : pert;
        const double r = 1.0 / a;
        const double m = c * r;
        A.u0[at(i)] = r;
        A.u1[at(i)] = b;
        A.u2[at(i)] = 0.0;
        A.lm[at(i)] = m;
        A.piv[at(i)] = 0;
        a = dn - m * b;
        b = bn;
      } else {
        const double cp = fabs(c) < pert ? (c < 0.0 ? -pert : pert) : c;
        const double r = 1.0 / cp;
        const double m = a * r;
        A.u0[at(i)] = r;
        A.u1[at(i)] = dn;
        A.u2[at(i)] = bn;
        A.lm[at(i)] = m;
        A.piv[at(i)] = 1;
        a = b - m * dn;
        b = -m * bn;
      }
    }
    if (fabs(a) < pert) a = a < 0.0 ? -pert : pert;
    A.u0[at(n - 1)] = 1.0 / a;
    A.u1[at(n - 1)] = 0.0;
    A.u2[at(n - 1)] = 0.0;
  }
  // pseudo-random start in [-1, 1)
  const uint64_t key = mix64(0x2002109910ull ^ ((uint64_t)k * 0x9E3779B97F4A7C15ull));
  for (int32_t i = 0; i < n; ++i) {
    const uint64_t r = mix64(key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
    A.y[at(i)] = (double)(r >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
  // every solve is followed by a normalisation, folded into the next solve's
  // reads (and into one final pass): 1 / ||y||, or, if the sum of squares
  // overflowed, the same with y first scaled by its largest entry
  double f = 1.0, sgn = 1.0;
  for (int step = 0; step < INVIT_STEPS; ++step) {
    const SolveOut o = invit_solve(A, k, f);
    sgn = o.sgn;
    if (o.ss > 0.0 && o.ss <= DBL_MAX) {
      f = 1.0 / sqrt(o.ss);
    } else {
      const double s = o.amax > 0.0 ? 1.0 / o.amax : 1.0;
      double ss = 0.0;
      for (int32_t i = 0; i < n; ++i) {
        const double v = A.y[at(i)] * s;
        ss = fma(v, v, ss);
      }
      f = ss > 0.0 ? s / sqrt(ss) : 1.0;
    }
  }
  // sign: the first entry of largest magnitude is positive
  for (int32_t i = 0; i < n; ++i) A.y[at(i)] *= f * sgn;
}

__device__ __forceinline__ double block_sum(double v, double *red);

// Tight groups (eigenvalues chained by gaps below TIGHT_TOL ||T||) that
// start at vector blockIdx.x: vectors j0+1 .. j1-1 are iterated again from a
// new pseudo-random start, and after every solve the iterate is
// orthogonalised (twice) against the group's earlier vectors and
// normalised. Blocks at no group start, or of one-vector groups, return at
// once. Works on the [row][vector] iterates.
__global__ void te_tight_kernel(InvitArgs A) {
  __shared__ double red[TIGHT_THREADS / 32];
  __shared__ double s_scale;
  const int32_t j0 = blockIdx.x, nev = A.nev, n = A.n;
  const double tol = TIGHT_TOL * A.bounds->tnorm;
  if (j0 > 0 && A.w[j0] - A.w[j0 - 1] < tol) return;  // not a group start
  int32_t j1 = j0 + 1;
  while (j1 < nev && A.w[j1] - A.w[j1 - 1] < tol) ++j1;
  if (j1 - j0 < 2) return;
  const size_t ld = (size_t)nev;
  for (int32_t c = j0 + 1; c < j1; ++c) {
    double *yc = A.y + c;  // element i at yc[i * ld]
    const uint64_t key = mix64(0x7E5D1C0B3A29ull ^ ((uint64_t)c * 0x9E3779B97F4A7C15ull));
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint64_t r = mix64(key + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull);
      yc[(size_t)i * ld] = (double)(r >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    }
    __syncthreads();
    for (int step = 0; step < INVIT_STEPS; ++step) {
      if (threadIdx.x == 0) {
        const double amax = invit_solve(A, c, 1.0).amax;
        s_scale = amax > 0.0 ? 1.0 / amax : 1.0;
      }
      __syncthreads();
      const double sc = s_scale;
      for (int32_t i = threadIdx.x; i < n; i += blockDim.x) yc[(size_t)i * ld] *= sc;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass) {
        for (int32_t p = j0; p < c; ++p) {
          const double *yp = A.y + p;
          double s = 0.0;
          for (int32_t i = threadIdx.x; i < n; i += blockDim.x) s += yp[(size_t)i * ld] * yc[(size_t)i * ld];
          const double dot = block_sum(s, red);
          for (int32_t i = threadIdx.x; i < n; i += blockDim.x) yc[(size_t)i * ld] -= dot * yp[(size_t)i * ld];
          __syncthreads();
        }
      }
      double s = 0.0;
      for (int32_t i = threadIdx.x; i < n; i += blockDim.x) s += yc[(size_t)i * ld] * yc[(size_t)i * ld];
      const double nrm = sqrt(block_sum(s, red));
      const double f = nrm > 0.0 ? 1.0 / nrm : 0.0;
      for (int32_t i = threadIdx.x; i < n; i += blockDim.x) yc[(size_t)i * ld] *= f;
      __syncthreads();
    }
  }
}

// [row][vector] (ld = nev) -> column-major x (ldx), 32 x 32 tiles.
__global__ void te_transpose_kernel(const double *__restrict__ y, int32_t n, int32_t nev, double *__restrict__ x,
                                    int64_t ldx) {
  __shared__ double tile[32][33];
  const int32_t i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int32_t i = i0 + r, k = k0 + threadIdx.x;
    if (i < n && k < nev) tile[r][threadIdx.x] = y[(size_t)i * nev + k];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int32_t k = k0 + r, i = i0 + threadIdx.x;
    if (i < n && k < nev) x[(size_t)k * ldx + i] = tile[threadIdx.x][r];
  }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x / 32, nw = blockDim.x / 32;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Modified Gram-Schmidt, twice, inside the cluster that starts at vector
// blockIdx.x (vectors whose eigenvalues are chained by gaps below
// CLUSTER_TOL * ||T||); blocks at no cluster start, or of one-vector
// clusters, return at once.
__global__ void te_reorth_kernel(const double *__restrict__ w, int32_t n, int32_t nev,
                                 const Bounds *__restrict__ bounds, double *__restrict__ x, int64_t ldx) {
  __shared__ double red[REORTH_THREADS / 32];
  const int32_t j0 = blockIdx.x;
  const double tol = CLUSTER_TOL * bounds->tnorm;
  if (j0 > 0 && w[j0] - w[j0 - 1] < tol) return;  // not a cluster start
  int32_t j1 = j0 + 1;
  while (j1 < nev && w[j1] - w[j1 - 1] < tol) ++j1;
  if (j1 - j0 < 2) return;
  for (int32_t c = j0 + 1; c < j1; ++c) {
    double *xc = x + (size_t)c * ldx;
    for (int pass = 0; pass < 2; ++pass) {
      for (int32_t p = j0; p < c; ++p) {
        const double *xp = x + (size_t)p * ldx;
        double s = 0.0;
        for (int32_t i = threadIdx.x; i < n; i += blockDim.x) s += xp[i] * xc[i];
        const double dot = block_sum(s, red);
        for (int32_t i = threadIdx.x; i < n; i += blockDim.x) xc[i] -= dot * xp[i];
        __syncthreads();
      }
    }
    double s = 0.0;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) s += xc[i] * xc[i];
    const double nrm = sqrt(block_sum(s, red));
    const double f = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) xc[i] *= f;
    __syncthreads();
  }
}

// Real column-major xr (ld ldr) -> complex x (ld ldx), imaginary parts 0.
__global__ void te_to_complex_kernel(const double *__restrict__ xr, int64_t ldr, int32_t n, int32_t nev,
                                     double2 *__restrict__ x, int64_t ldx) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * nev) return;
  const int64_t k = t / n, i = t - k * n;
  x[k * ldx + i] = make_double2(xr[k * ldr + i], 0.0);
}

}  // namespace te
}  // namespace tbbt
