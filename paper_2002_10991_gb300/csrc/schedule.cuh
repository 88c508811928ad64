// Geometry of the reflector store and the block schedule of the apply kernel.
//
// Used by the kernels (device) and by host code (plan set-up and the schedule
// checker), so every function is __host__ __device__ and branch-light.
//
// Store geometry (Sec. 2.2.1): stage i = 0..n-3 has ceil((n-i-2)/b) sweeps;
// reflector (i, j) acts on rows r = i+1+j*b .. r+L-1, L = min(b, n-r). A
// Hermitian store adds (n-2, 0) with L = 1.
//
// Application order (Sec. 2.2.2, Sec. 3.2): the reverse of generation order
// is required only between reflectors whose row ranges overlap. Overlapping
// pairs (i, j), (i', j') with i > i' always have j <= j' (two reflectors of
// one stage are disjoint; (i, j+1) and (i', j) with i > i' are b+1 or more
// rows apart). So sweep j+1 may apply stage s once sweep j has applied every
// stage > s: the sweeps form a pipeline, each one stage behind the previous.
//
// Block schedule: a thread block owns a strip of 32 columns and processes the
// sweeps in epochs of G consecutive sweeps j0 .. j0+G-1, warp g taking sweep
// j0+g. Time advances in steps; at step t warp g applies the NB stages of
// block k = t-g, i.e. stages sigma(k) .. sigma(k)-NB+1 with
// sigma(k) = imax(j0) - k*NB (clipped to the stages its sweep has). Warp g is
// thus one block (NB stages) behind warp g-1: it never needs a row that warp
// g-1 has not finished, and within a step the row ranges of two warps are
// disjoint (one row apart).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define TBBT_HD __host__ __device__ __forceinline__
#else
#define TBBT_HD inline
#endif

namespace tbbt {

struct StoreGeom {
  int32_t n, b, cplx;

  // number of sweeps of stage 0 (the largest sweep index + 1)
  TBBT_HD int32_t num_sweeps() const {
    if (n >= 3) return (n - 2 + b - 1) / b;
    return (cplx && n == 2) ? 1 : 0;
  }
  // highest stage that has sweep j
  TBBT_HD int32_t imax(int32_t j) const { return (cplx && j == 0) ? n - 2 : n - 3 - j * b; }
  // reflectors of all sweeps before j in the sweep-major layout
  TBBT_HD int64_t sweep_offset(int32_t j) const {
    int64_t jj = j;
    int64_t o = jj * (int64_t)(n - 2) - (int64_t)b * jj * (jj - 1) / 2;
    if (cplx && j >= 1) o += 1;
    return o;
  }
  TBBT_HD int64_t num_reflectors() const { return sweep_offset(num_sweeps()); }
  // first row of reflector (s, j)
  TBBT_HD int32_t row(int32_t s, int32_t j) const { return s + 1 + j * b; }
  TBBT_HD int32_t len(int32_t s, int32_t j) const {
    int32_t r = row(s, j);
    return (n - r < b) ? n - r : b;
  }
};

struct Epoch {
  int32_t j0;      // first sweep
  int32_t ge;      // sweeps in this epoch (<= G)
  int32_t sig_top; // imax(j0)
  int32_t nb;      // stages per step
  int32_t nsteps;  // steps until the last warp has applied stage 0
};

TBBT_HD Epoch make_epoch(const StoreGeom &g, int32_t e, int32_t G, int32_t NB) {
  Epoch ep;
  ep.j0 = e * G;
  int32_t J = g.num_sweeps();
  ep.ge = (J - ep.j0 < G) ? J - ep.j0 : G;
  ep.sig_top = g.imax(ep.j0);
  ep.nb = NB;
  ep.nsteps = (ep.ge - 1) + (ep.sig_top + 1 + NB - 1) / NB;
  return ep;
}

// Stages [lo, hi] that warp w applies at step t (hi < lo if none).
TBBT_HD void warp_stages(const StoreGeom &g, const Epoch &ep, int32_t w, int32_t t, int32_t *hi, int32_t *lo) {
  int32_t k = t - w;
  *hi = -1;
  *lo = 0;
  if (w >= ep.ge || k < 0) return;
  int32_t sig = ep.sig_top - k * ep.nb;
  int32_t top = g.imax(ep.j0 + w);
  int32_t h = sig < top ? sig : top;
  int32_t l = sig - ep.nb + 1;
  if (l < 0) l = 0;
  *hi = h;
  *lo = l;
}

// Smallest row any warp touches at step t (rows below it must be resident).
TBBT_HD int32_t step_min_row(const StoreGeom &g, const Epoch &ep, int32_t t) {
  int32_t l = ep.sig_top - t * ep.nb - ep.nb + 1;
  if (l < 0) l = 0;
  return l + 1 + ep.j0 * g.b;
}

// Largest row any warp touches at steps >= t (rows above it are final for
// this epoch), or -1 if no warp has work left. Usually the lowest warp
// bounds it, but not always (the length-1 reflector of a Hermitian store
// sits on row n-1 in sweep 0), so every warp is asked.
TBBT_HD int32_t rows_live_max(const StoreGeom &g, const Epoch &ep, int32_t t) {
  int32_t best = -1;
  for (int32_t w = 0; w < ep.ge; ++w) {
    int32_t j = ep.j0 + w;
    int32_t top = g.imax(j);
    int32_t k = t - w;
    int32_t shi = top;
    if (k >= 0) {
      int32_t sig = ep.sig_top - k * ep.nb;
      shi = sig < top ? sig : top;
    }
    if (shi < 0) continue;
    int32_t m = shi + j * g.b + g.b;
    if (m > g.n - 1) m = g.n - 1;
    if (m > best) best = m;
  }
  return best;
}

}  // namespace tbbt
