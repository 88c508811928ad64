// Host side of libtbbt: argument checking, plans, the one-shot cache and the
// C ABI declared in include/tbbt.h. Every step of the computation runs in the
// kernels of apply_kernels.cuh; this file only validates, allocates and
// launches.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/tbbt.h"
#include "apply_kernels.cuh"
#include "split_kernels.cuh"
#include "tc_split.cuh"
#include "bulge.cuh"
#include "b2f.cuh"
#include "b2f_split.cuh"
#include "probe.cuh"
#include "tridiag.cuh"

using tbbt::StoreGeom;
using tbbt::zdouble;

namespace {

constexpr int32_t kMaxBand = 128;
// Dynamic shared memory a launch may use: the 227 KB opt-in limit of a block
// covers static plus dynamic shared memory, so leave 1 KB for the kernels'
// static variables.
constexpr int32_t kMaxSmem = 226 * 1024;

#define TBBT_CUDA_TRY(expr)                          \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) {                         \
      (void)cudaGetLastError();                      \
      return e_ == cudaErrorMemoryAllocation ? TBBT_ENOMEM : TBBT_ECUDA; \
    }                                                \
  } while (0)

// Device error word set by bounded in-kernel waits that gave up.
__device__ int g_tbbt_error = 0;

int32_t round_even(int32_t b) { return (b + 1) & ~1; }

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// Raise the kernel's dynamic shared memory limit to what the device allows
// beside its static shared memory (at least kMaxSmem on sm_103).
template <typename K>
cudaError_t allow_max_dynamic_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  int allowed = optin - (int)fa.sharedSizeBytes;
  if (allowed < kMaxSmem) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, allowed);
}

size_t elem_size(tbbt_dtype dt) { return dt == TBBT_COMPLEX128 ? 16 : 8; }

using ApplyFn = void (*)(tbbt::ApplyArgs);

// The apply kernel instance for a data type and register-window width.
ApplyFn apply_fn(tbbt_dtype dt, int32_t bw) {
  if (dt == TBBT_COMPLEX128) return bw == -64 ? tbbt::apply_kernel<zdouble, -64> : tbbt::apply_kernel<zdouble, -1>;
  if (bw == 64) return tbbt::apply_kernel<double, 64>;
  if (bw == 32) return tbbt::apply_kernel<double, 32>;
  return tbbt::apply_kernel<double, 0>;
}

int32_t ring_rows_for(int32_t b, int32_t G, int32_t NB) { return G * b + (G + 2) * NB + 8; }

size_t smem_bytes_for(tbbt_dtype dt, int32_t b, int32_t G, int32_t NB) {
  size_t es = elem_size(dt);
  return (size_t)ring_rows_for(b, G, NB) * 32 * es + (size_t)G * 2 * NB * round_even(b) * es;
}

// Register-window width of the apply kernel for a problem: real b = 32 or 64
// keep each column's window in registers, complex data take a lane pair per
// column (-1; b = 64 with the window in the pair's registers: -64), other
// widths the shared-memory window (0).
int32_t window_width(tbbt_dtype dt, int64_t nbw) {
  if (dt == TBBT_COMPLEX128) return nbw == 64 ? -64 : -1;
  return (nbw == 32 || nbw == 64) ? (int32_t)nbw : 0;
}

// Threads of one apply block: a warp per sweep (two for lane pairs).
int32_t apply_threads(int32_t G, int32_t bw) { return G * 32 * (bw < 0 ? 2 : 1); }

// Launch geometry: the requested sweeps per block (wantG) and stages per
// step (wantNB), lowered until the block's ring and reflector buffers fit in
// shared memory. Returns false if nothing fits.
bool fit_geometry(tbbt_dtype dt, int32_t nbw, int32_t bw, int32_t wantG, int32_t wantNB, int32_t *G_out,
                  int32_t *NB_out) {
  if (bw != 0 && wantG > 8) wantG = 8;  // register window: 256 threads; lane pairs: 512
  if (bw < -1 && wantG > 4) wantG = 4;  // complex register window: 256 threads
  if (wantG > 16) wantG = 16;
  int32_t G = wantG, NB = wantNB;
  if (NB > 4 * G) NB = 4 * G;  // the row prefetch holds at most 4 elements per thread
  while (smem_bytes_for(dt, nbw, G, NB) > (size_t)kMaxSmem) {
    if (G > 4 || (NB <= 2 && G > 1))
      --G;
    else if (NB > 2)
      NB /= 2;
    else
      break;
  }
  if (smem_bytes_for(dt, nbw, G, NB) > (size_t)kMaxSmem) return false;
  *G_out = G;
  *NB_out = NB;
  return true;
}

// Default launch geometry (sweeps per block, stages per step). Real data:
// 4 sweeps (one warp per SM sub-partition) and 8 stages per step, two blocks
// per SM. Complex data (lane pairs): one sweep and 2 stages per step, five
// small blocks per SM, whose step barriers cover one another (1.102 against
// 1.084 TFLOP/s for 4 x 8 at n = 20000, nev = 6000).
void default_geometry(tbbt_dtype dt, int32_t *G, int32_t *NB) {
  *G = dt == TBBT_COMPLEX128 ? 1 : 4;
  *NB = dt == TBBT_COMPLEX128 ? 2 : 8;
}

tbbt_status check_shape(int64_t n, int64_t nbw, int64_t nev) {
  if (n < 0 || n > (int64_t)1 << 30) return TBBT_EINVAL;
  if (nbw < 1 || nbw > kMaxBand) return TBBT_EINVAL;
  if (nev < 0 || nev > n) return TBBT_EINVAL;
  return TBBT_OK;
}

}  // namespace

struct tbbt_plan {
  tbbt_dtype dtype;
  StoreGeom g;
  int32_t nev;
  int64_t K;
  int32_t ldv;
  int32_t G, NB, ring;
  int32_t bw;  // register-window width of the apply kernel (0: shared-memory window)
  size_t smem;
  void *d_store = nullptr;       // re-laid reflectors, K * ldv elements
  int64_t *d_stage_off = nullptr;  // n entries
  int *d_err = nullptr;
  // persistent apply kernel: one progress flag per (strip, epoch) unit
  int32_t strips = 0, epochs = 0, units = 0, grid = 0;
  int *d_flags = nullptr;
  unsigned *d_counter = nullptr;
  long long timeout_ns = 20000000000LL;
  int withhold = -1;
  // split-precision variant
  int32_t variant = TBBT_VARIANT_FP64;
  int64_t s_blocks = 0;
  int32_t s_units = 0, s_grid = 0, s_ring = 0;
  size_t s_smem = 0;
  void *d_slices = nullptr;
  void *d_scales = nullptr;
  int64_t *d_block_start = nullptr;
  int32_t *d_colexp = nullptr;
  int *d_sflags = nullptr;
  int64_t *d_zfix = nullptr;  // tensor-core form: fixed-point copy of the eigenvector block
  int64_t ldz = 0;
  CUtensorMap zmap;           // tiled view of d_zfix: boxes of 16 rows x 128 columns, 128-byte swizzle
  // device copies used by the host-buffer entry points (allocated on demand)
  void *d_hv = nullptr, *d_ht = nullptr, *d_q = nullptr;
  int64_t d_q_ld = 0;
};

namespace {

template <int B>
size_t split_smem_bytes(int32_t ring) {
  using D = tbbt::split::Dims<B>;
  return (size_t)ring * tbbt::split::ZLD * sizeof(int64_t) + (size_t)D::BLOCK_ELEMS * 2;
}

template <int B>
tbbt_status split_setup_b(tbbt_plan *p) {
  using namespace tbbt::split;
  const int32_t J = p->g.num_sweeps();
  std::vector<int64_t> start((size_t)J + 1, 0);
  for (int32_t j = 0; j < J; ++j) start[(size_t)j + 1] = start[(size_t)j] + (p->g.imax(j) + 1 + NB - 1) / NB;
  p->s_blocks = start[(size_t)J];
  p->s_ring = p->g.b + 3 * NB + 8;  // ring_rows_for(b, 1, NB)
  p->s_smem = split_smem_bytes<B>(p->s_ring);
  const int32_t strips = (int32_t)((p->nev + WS - 1) / WS);
  p->s_units = strips * J;
  if (p->s_blocks == 0 || p->nev == 0) return TBBT_OK;
  const size_t slice_bytes = (size_t)p->s_blocks * Dims<B>::BLOCK_ELEMS * sizeof(__nv_bfloat16);
  if (cudaMalloc(&p->d_slices, slice_bytes) != cudaSuccess ||
      cudaMalloc(&p->d_scales, sizeof(BlockScale) * (size_t)p->s_blocks) != cudaSuccess ||
      cudaMalloc(&p->d_block_start, sizeof(int64_t) * ((size_t)J + 1)) != cudaSuccess ||
      cudaMalloc(&p->d_colexp, sizeof(int32_t) * (size_t)p->nev) != cudaSuccess ||
      cudaMalloc(&p->d_sflags, sizeof(int) * (size_t)p->s_units) != cudaSuccess) {
    (void)cudaGetLastError();
    return TBBT_ENOMEM;
  }
  TBBT_CUDA_TRY(cudaMemcpy(p->d_block_start, start.data(), sizeof(int64_t) * start.size(), cudaMemcpyHostToDevice));
  TBBT_CUDA_TRY(allow_max_dynamic_smem(split_apply_kernel<B>));
  int dev = 0, sms = 0, per_sm = 0;
  TBBT_CUDA_TRY(cudaGetDevice(&dev));
  TBBT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TBBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, split_apply_kernel<B>, NWARPS * 32, p->s_smem));
  if (per_sm < 1) return TBBT_ENOTSUP;
  const int64_t resident = (int64_t)sms * per_sm;
  p->s_grid = (int32_t)(p->s_units < resident ? p->s_units : resident);
  return TBBT_OK;
}

tbbt_status split_setup(tbbt_plan *p) {
  p->variant = TBBT_VARIANT_SPLIT_BF16;
  return p->g.b == 64 ? split_setup_b<64>(p) : split_setup_b<32>(p);
}

template <int B>
tbbt_status split_prepare(tbbt_plan *p, cudaStream_t s) {
  if (p->s_blocks == 0 || p->nev == 0) return TBBT_OK;
  tbbt::split::wy_prepare_kernel<B><<<(unsigned)p->s_blocks, 128, 0, s>>>(
      (const double *)p->d_store, p->g, p->ldv, p->d_block_start, p->g.num_sweeps(), p->s_blocks,
      (__nv_bfloat16 *)p->d_slices, (tbbt::split::BlockScale *)p->d_scales);
  TBBT_CUDA_TRY(cudaGetLastError());
  return TBBT_OK;
}

template <int B>
tbbt_status split_execute(tbbt_plan *p, void *q, int64_t ldq, cudaStream_t s) {
  using namespace tbbt::split;
  if (p->s_blocks == 0 || p->nev == 0) return TBBT_OK;
  const unsigned cblocks = (unsigned)((p->nev + 7) / 8);
  to_fixed_kernel<<<cblocks, 256, 0, s>>>((double *)q, ldq, p->g.n, p->nev, p->d_colexp);
  TBBT_CUDA_TRY(cudaGetLastError());
  TBBT_CUDA_TRY(cudaMemsetAsync(p->d_sflags, 0x7f, sizeof(int) * (size_t)p->s_units, s));
  TBBT_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned), s));
  SplitArgs a;
  a.q = (int64_t *)q;
  a.ldq = ldq;
  a.g = p->g;
  a.nev = p->nev;
  a.strips = (int32_t)((p->nev + WS - 1) / WS);
  a.units = p->s_units;
  a.ring = p->s_ring;
  a.slices = (const __nv_bfloat16 *)p->d_slices;
  a.scales = (const BlockScale *)p->d_scales;
  a.block_start = p->d_block_start;
  a.flags = p->d_sflags;
  a.counter = p->d_counter;
  a.err = p->d_err;
  a.timeout_ns = p->timeout_ns;
  split_apply_kernel<B><<<(unsigned)p->s_grid, NWARPS * 32, p->s_smem, s>>>(a);
  TBBT_CUDA_TRY(cudaGetLastError());
  from_fixed_kernel<<<cblocks, 256, 0, s>>>((double *)q, ldq, p->g.n, p->nev, p->d_colexp);
  TBBT_CUDA_TRY(cudaGetLastError());
  return TBBT_OK;
}


// tensor-core (tcgen05) form of the split-precision variant
template <int B>
tbbt_status tc_setup_b(tbbt_plan *p) {
  using namespace tbbt::tcs;
  using D = Geo<B>;
  int dev = 0, major = 0, sms = 0, per_sm = 0;
  TBBT_CUDA_TRY(cudaGetDevice(&dev));
  TBBT_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  if (major != 10) return TBBT_ENOTSUP;
  const int32_t J = p->g.num_sweeps();
  std::vector<int64_t> start((size_t)J + 1, 0);
  for (int32_t j = 0; j < J; ++j) start[(size_t)j + 1] = start[(size_t)j] + p->g.imax(j) / NB + 1;
  p->s_blocks = start[(size_t)J];
  p->s_smem = D::SMEM;
  const int32_t strips = (int32_t)((p->nev + WS - 1) / WS);
  p->s_units = strips * J;
  p->ldz = ((int64_t)p->g.n + 3) & ~(int64_t)1;  // even, >= n + 2
  if (p->s_blocks == 0 || p->nev == 0) return TBBT_OK;
  if (cudaMalloc(&p->d_slices, (size_t)p->s_blocks * D::BLOCK_BYTES) != cudaSuccess ||
      cudaMalloc(&p->d_scales, sizeof(int32_t) * (size_t)p->s_blocks) != cudaSuccess ||
      cudaMalloc(&p->d_block_start, sizeof(int64_t) * ((size_t)J + 1)) != cudaSuccess ||
      cudaMalloc(&p->d_colexp, sizeof(int32_t) * (size_t)p->nev) != cudaSuccess ||
      cudaMalloc(&p->d_sflags, sizeof(int) * (size_t)p->s_units) != cudaSuccess ||
      cudaMalloc(&p->d_zfix, sizeof(int64_t) * (size_t)p->nev * (size_t)p->ldz) != cudaSuccess) {
    (void)cudaGetLastError();
    return TBBT_ENOMEM;
  }
  TBBT_CUDA_TRY(cudaMemset(p->d_zfix, 0, sizeof(int64_t) * (size_t)p->nev * (size_t)p->ldz));
  TBBT_CUDA_TRY(cudaMemcpy(p->d_block_start, start.data(), sizeof(int64_t) * start.size(), cudaMemcpyHostToDevice));
  {
    // the tensor map of the fixed-point block (driver entry point, no link to libcuda)
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    TBBT_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr));
    if (qr != cudaDriverEntryPointSuccess || !fn) return TBBT_ENOTSUP;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t gdim[2] = {(cuuint64_t)p->ldz, (cuuint64_t)p->nev};
    const cuuint64_t gstride[1] = {(cuuint64_t)p->ldz * sizeof(int64_t)};
    const cuuint32_t box[2] = {(cuuint32_t)STG_ROWS, (cuuint32_t)WS};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&p->zmap, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, p->d_zfix, gdim, gstride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return TBBT_ECUDA;
  }
  TBBT_CUDA_TRY(allow_max_dynamic_smem(tc_apply_kernel<B>));
  TBBT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TBBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_apply_kernel<B>, D::NTHREADS, p->s_smem));
  if (per_sm < 1) return TBBT_ENOTSUP;
  // one block per SM: each holds all 512 columns of its SM's tensor memory
  p->s_grid = (int32_t)(p->s_units < sms ? p->s_units : sms);
  return TBBT_OK;
}

tbbt_status tc_setup(tbbt_plan *p) {
  p->variant = TBBT_VARIANT_SPLIT_BF16_TC;
  return p->g.b == 64 ? tc_setup_b<64>(p) : tc_setup_b<32>(p);
}

template <int B>
tbbt_status tc_prepare(tbbt_plan *p, cudaStream_t s) {
  if (p->s_blocks == 0 || p->nev == 0) return TBBT_OK;
  tbbt::tcs::tc_prepare_kernel<B><<<(unsigned)p->s_blocks, 128, 0, s>>>(
      (const double *)p->d_store, p->g, p->ldv, p->d_block_start, p->g.num_sweeps(), p->s_blocks,
      (unsigned char *)p->d_slices, (int32_t *)p->d_scales);
  TBBT_CUDA_TRY(cudaGetLastError());
  return TBBT_OK;
}

template <int B>
tbbt_status tc_execute(tbbt_plan *p, void *q, int64_t ldq, cudaStream_t s) {
  using namespace tbbt::tcs;
  using D = Geo<B>;
  if (p->s_blocks == 0 || p->nev == 0) return TBBT_OK;
  const unsigned cblocks = (unsigned)((p->nev + 7) / 8);
  to_fixed_kernel<<<cblocks, 256, 0, s>>>((const double *)q, ldq, p->d_zfix, p->ldz, p->g.n, p->nev, p->d_colexp);
  TBBT_CUDA_TRY(cudaGetLastError());
  TBBT_CUDA_TRY(cudaMemsetAsync(p->d_sflags, 0x7f, sizeof(int) * (size_t)p->s_units, s));
  TBBT_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned), s));
  TcArgs a;
  a.z = p->d_zfix;
  a.ldz = p->ldz;
  a.g = p->g;
  a.nev = p->nev;
  a.strips = (int32_t)((p->nev + WS - 1) / WS);
  a.units = p->s_units;
  a.slices = (const unsigned char *)p->d_slices;
  a.gvs = (const int32_t *)p->d_scales;
  a.block_start = p->d_block_start;
  a.flags = p->d_sflags;
  a.counter = p->d_counter;
  a.err = p->d_err;
  a.timeout_ns = p->timeout_ns;
  a.withhold = p->withhold;
  tc_apply_kernel<B><<<(unsigned)p->s_grid, D::NTHREADS, p->s_smem, s>>>(a, p->zmap);
  TBBT_CUDA_TRY(cudaGetLastError());
  from_fixed_kernel<<<cblocks, 256, 0, s>>>((double *)q, ldq, p->d_zfix, p->ldz, p->g.n, p->nev, p->d_colexp);
  TBBT_CUDA_TRY(cudaGetLastError());
  return TBBT_OK;
}

}  // namespace

extern "C" {

const char *tbbt_status_string(tbbt_status s) {
  switch (s) {
    case TBBT_OK: return "ok";
    case TBBT_EINVAL: return "invalid argument";
    case TBBT_ENOMEM: return "out of memory";
    case TBBT_ECUDA: return "CUDA error";
    case TBBT_ETIMEOUT: return "in-kernel wait timed out";
    case TBBT_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

int64_t tbbt_num_reflectors(int64_t n, int64_t b, int is_complex) {
  if (n < 0 || b < 1 || n > (int64_t)1 << 30 || b > (int64_t)1 << 30) return -1;
  StoreGeom g{(int32_t)n, (int32_t)b, is_complex ? 1 : 0};
  return g.num_reflectors();
}

int64_t tbbt_schedule_max_live_rows(int64_t n, int64_t nbw, int is_complex, int32_t G, int32_t NB) {
  if (n < 0 || nbw < 1 || G < 1 || NB < 1 || n > (int64_t)1 << 24) return -1;
  StoreGeom g{(int32_t)n, (int32_t)nbw, is_complex ? 1 : 0};
  const int32_t J = g.num_sweeps();
  int64_t worst = 0;
  std::vector<int32_t> done_stage;  // lowest stage applied so far per sweep
  std::vector<int64_t> count(J > 0 ? J : 1, 0);
  for (int32_t e = 0; e * G < J; ++e) {
    tbbt::Epoch ep = tbbt::make_epoch(g, e, G, NB);
    done_stage.assign(ep.ge, INT32_MAX);
    int32_t prev_live = g.n - 1;
    for (int32_t t = 0; t < ep.nsteps; ++t) {
      int32_t live = tbbt::rows_live_max(g, ep, t);
      int32_t top = tbbt::step_min_row(g, ep, t);
      int32_t ntop = tbbt::step_min_row(g, ep, t + 1);
      // ring must hold [ntop, prev_live] without aliasing
      int64_t need = (int64_t)prev_live - ntop + 1;
      if (need > worst) worst = need;
      int32_t last_max = -1;  // last row of the nearest active warp above
      for (int32_t w = 0; w < ep.ge; ++w) {
        int32_t hi, lo;
        tbbt::warp_stages(g, ep, w, t, &hi, &lo);
        if (hi < lo) continue;
        int32_t j = ep.j0 + w;
        int32_t rlo = g.row(lo, j);
        int32_t rhi = g.row(hi, j) + g.len(hi, j) - 1;
        if (rlo < top || rhi > live) return -1;  // outside the resident rows
        if (rlo <= last_max) return -1;  // overlaps the warp above
        last_max = rhi;
        for (int32_t s = hi; s >= lo; --s) {
          // sweep j-1 must have applied stage s+1 in an earlier step
          if (w > 0 && done_stage[w - 1] > s + 1) return -1;
          if (s > g.imax(j) || s < 0) return -1;
          count[j] += 1;
        }
      }
      for (int32_t w = 0; w < ep.ge; ++w) {
        int32_t hi, lo;
        tbbt::warp_stages(g, ep, w, t, &hi, &lo);
        if (hi >= lo) done_stage[w] = lo;
      }
      prev_live = live;
    }
    for (int32_t w = 0; w < ep.ge; ++w)
      if (done_stage[w] != 0) return -1;
  }
  for (int32_t j = 0; j < J; ++j)
    if (count[j] != (int64_t)g.imax(j) + 1) return -1;
  return worst;
}

tbbt_status tbbt_plan_create(tbbt_plan **plan, tbbt_dtype dtype, int64_t n, int64_t nbw, int64_t nev,
                             const tbbt_options *opt) {
  if (!plan) return TBBT_EINVAL;
  *plan = nullptr;
  if (dtype != TBBT_REAL64 && dtype != TBBT_COMPLEX128) return TBBT_EINVAL;
  tbbt_status st = check_shape(n, nbw, nev);
  if (st != TBBT_OK) return st;
  if (opt && opt->variant != TBBT_VARIANT_FP64 && opt->variant != TBBT_VARIANT_SPLIT_BF16 &&
      opt->variant != TBBT_VARIANT_SPLIT_BF16_TC)
    return TBBT_EINVAL;
  if (opt && opt->variant != TBBT_VARIANT_FP64 && (dtype != TBBT_REAL64 || (nbw != 32 && nbw != 64)))
    return TBBT_ENOTSUP;
  tbbt_plan *p = new (std::nothrow) tbbt_plan();
  if (!p) return TBBT_ENOMEM;
  p->dtype = dtype;
  p->g = StoreGeom{(int32_t)n, (int32_t)nbw, dtype == TBBT_COMPLEX128 ? 1 : 0};
  p->nev = (int32_t)nev;
  p->K = p->g.num_reflectors();
  p->ldv = round_even((int32_t)nbw);
  // real data with b = 32 or 64 keep each column's window in registers
  // complex data: two warps per sweep (a lane pair per column)
  p->bw = window_width(dtype, nbw);
  // launch geometry: the requested or default sweeps per block and stages
  // per step, lowered until they fit in shared memory; blocks that fit share
  // an SM, so one block's pipeline fill is covered by another
  int32_t G = 0, NB = 0, G0 = 0, NB0 = 0;
  default_geometry(dtype, &G0, &NB0);
  if (!fit_geometry(dtype, (int32_t)nbw, p->bw, opt && opt->sweeps_per_block > 0 ? opt->sweeps_per_block : G0,
                    opt && opt->stages_per_step > 0 ? opt->stages_per_step : NB0, &G, &NB)) {
    delete p;
    return TBBT_ENOTSUP;
  }
  p->G = G;
  p->NB = NB;
  p->ring = ring_rows_for((int32_t)nbw, G, NB);
  p->smem = smem_bytes_for(dtype, (int32_t)nbw, G, NB);
  if (opt && opt->wait_timeout_ms > 0) p->timeout_ns = (long long)opt->wait_timeout_ms * 1000000LL;
  if (opt && opt->debug_withhold_unit_plus1 > 0) p->withhold = opt->debug_withhold_unit_plus1 - 1;
  p->strips = (int32_t)((nev + 31) / 32);
  p->epochs = (p->g.num_sweeps() + G - 1) / G;
  p->units = p->strips * p->epochs;

  auto fail = [&](tbbt_status s) {
    tbbt_plan_destroy(p);
    return s;
  };
  cudaError_t e;
  if (p->K > 0) {
    e = cudaMalloc(&p->d_store, (size_t)p->K * p->ldv * elem_size(dtype));
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(TBBT_ENOMEM);
    }
    std::vector<int64_t> off((size_t)n + 1, 0);
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
      off[(size_t)i] = k;
      int64_t ns = (i + 3 <= n) ? (n - i - 2 + nbw - 1) / nbw : ((dtype == TBBT_COMPLEX128 && i == n - 2) ? 1 : 0);
      k += ns;
    }
    e = cudaMalloc(&p->d_stage_off, sizeof(int64_t) * ((size_t)n + 1));
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(TBBT_ENOMEM);
    }
    e = cudaMemcpy(p->d_stage_off, off.data(), sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(TBBT_ECUDA);
  }
  e = cudaGetSymbolAddress((void **)&p->d_err, g_tbbt_error);
  if (e != cudaSuccess) return fail(TBBT_ECUDA);
  // The attribute belongs to the kernel, not to the plan: raise it to the
  // largest size any plan may use, so that creating a plan with a smaller
  // footprint never invalidates the launches of an earlier, larger one.
  e = allow_max_dynamic_smem(apply_fn(dtype, p->bw));
  if (e != cudaSuccess) return fail(TBBT_ECUDA);
  if (p->units > 0) {
    e = cudaMalloc(&p->d_flags, sizeof(int) * (size_t)p->units);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_counter, sizeof(unsigned));
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(TBBT_ENOMEM);
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return fail(TBBT_ECUDA);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_fn(dtype, p->bw), apply_threads(G, p->bw),
                                                      p->smem);
    if (e != cudaSuccess || per_sm < 1) return fail(TBBT_ECUDA);
    int64_t resident = (int64_t)sms * per_sm;
    p->grid = (int32_t)(p->units < resident ? p->units : resident);
  }
  if (opt && opt->variant == TBBT_VARIANT_SPLIT_BF16) {
    tbbt_status sst = split_setup(p);
    if (sst != TBBT_OK) return fail(sst);
  }
  if (opt && opt->variant == TBBT_VARIANT_SPLIT_BF16_TC) {
    tbbt_status sst = tc_setup(p);
    if (sst != TBBT_OK) return fail(sst);
  }
  *plan = p;
  return TBBT_OK;
}

tbbt_status tbbt_plan_info(const tbbt_plan *p, int32_t *G, int32_t *NB, int32_t *ring, int32_t *smem,
                           int32_t *blocks) {
  if (!p) return TBBT_EINVAL;
  if (G) *G = p->G;
  if (NB) *NB = p->NB;
  if (ring) *ring = p->ring;
  if (smem) *smem = (int32_t)p->smem;
  if (blocks) *blocks = p->variant != TBBT_VARIANT_FP64 ? p->s_grid : p->grid;
  return TBBT_OK;
}

tbbt_status tbbt_plan_set_reflectors(tbbt_plan *p, const void *hh_v, const void *hh_tau, void *stream) {
  if (!p) return TBBT_EINVAL;
  if (p->K == 0) return TBBT_OK;
  if (!hh_v || !hh_tau) return TBBT_EINVAL;
  size_t es = elem_size(p->dtype);
  if (((uintptr_t)hh_v % es) || ((uintptr_t)hh_tau % es)) return TBBT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int threads = 256;
  const int64_t per_block = threads / 32;
  const int64_t blocks = (p->K + per_block - 1) / per_block;
  if (p->dtype == TBBT_COMPLEX128)
    tbbt::relayout_kernel<zdouble><<<(unsigned)blocks, threads, 0, s>>>(
        (const zdouble *)hh_v, (const zdouble *)hh_tau, p->d_stage_off, p->g, p->ldv, (zdouble *)p->d_store);
  else
    tbbt::relayout_kernel<double><<<(unsigned)blocks, threads, 0, s>>>(
        (const double *)hh_v, (const double *)hh_tau, p->d_stage_off, p->g, p->ldv, (double *)p->d_store);
  TBBT_CUDA_TRY(cudaGetLastError());
  if (p->variant == TBBT_VARIANT_SPLIT_BF16)
    return p->g.b == 64 ? split_prepare<64>(p, s) : split_prepare<32>(p, s);
  if (p->variant == TBBT_VARIANT_SPLIT_BF16_TC)
    return p->g.b == 64 ? tc_prepare<64>(p, s) : tc_prepare<32>(p, s);
  return TBBT_OK;
}

tbbt_status tbbt_plan_execute(tbbt_plan *p, void *q, int64_t ldq, void *stream) {
  if (!p) return TBBT_EINVAL;
  if (ldq < (p->g.n > 1 ? p->g.n : 1)) return TBBT_EINVAL;
  if (p->nev == 0 || p->K == 0) return TBBT_OK;
  if (!q) return TBBT_EINVAL;
  size_t es = elem_size(p->dtype);
  if ((uintptr_t)q % es) return TBBT_EINVAL;
  if (p->variant == TBBT_VARIANT_SPLIT_BF16)
    return p->g.b == 64 ? split_execute<64>(p, q, ldq, (cudaStream_t)stream)
                        : split_execute<32>(p, q, ldq, (cudaStream_t)stream);
  if (p->variant == TBBT_VARIANT_SPLIT_BF16_TC)
    return p->g.b == 64 ? tc_execute<64>(p, q, ldq, (cudaStream_t)stream)
                        : tc_execute<32>(p, q, ldq, (cudaStream_t)stream);
  tbbt::ApplyArgs a;
  a.vstore = p->d_store;
  a.q = q;
  a.ldq = ldq;
  a.g = p->g;
  a.nev = p->nev;
  a.ldv = p->ldv;
  a.G = p->G;
  a.NB = p->NB;
  a.ring = p->ring;
  a.strips = p->strips;
  a.units = p->units;
  a.flags = p->d_flags;
  a.counter = p->d_counter;
  a.err = p->d_err;
  a.timeout_ns = p->timeout_ns;
  a.withhold = p->withhold;
  cudaStream_t s = (cudaStream_t)stream;
  TBBT_CUDA_TRY(cudaMemsetAsync(p->d_flags, 0x7f, sizeof(int) * (size_t)p->units, s));
  TBBT_CUDA_TRY(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned), s));
  unsigned blocks = (unsigned)p->grid;
  apply_fn(p->dtype, p->bw)<<<blocks, apply_threads(p->G, p->bw), p->smem, s>>>(a);
  TBBT_CUDA_TRY(cudaGetLastError());
  return TBBT_OK;
}

tbbt_status tbbt_plan_destroy(tbbt_plan *p) {
  if (!p) return TBBT_OK;
  if (p->d_store || p->d_stage_off || p->d_flags || p->d_hv || p->d_ht || p->d_q) cudaDeviceSynchronize();
  if (p->d_store) cudaFree(p->d_store);
  if (p->d_stage_off) cudaFree(p->d_stage_off);
  if (p->d_flags) cudaFree(p->d_flags);
  if (p->d_counter) cudaFree(p->d_counter);
  if (p->d_slices) cudaFree(p->d_slices);
  if (p->d_scales) cudaFree(p->d_scales);
  if (p->d_block_start) cudaFree(p->d_block_start);
  if (p->d_colexp) cudaFree(p->d_colexp);
  if (p->d_sflags) cudaFree(p->d_sflags);
  if (p->d_zfix) cudaFree(p->d_zfix);
  if (p->d_hv) cudaFree(p->d_hv);
  if (p->d_ht) cudaFree(p->d_ht);
  if (p->d_q) cudaFree(p->d_q);
  delete p;
  return TBBT_OK;
}

tbbt_status tbbt_stream_check(void *stream) {
  TBBT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int h = 0;
  TBBT_CUDA_TRY(cudaMemcpyFromSymbol(&h, g_tbbt_error, sizeof(int)));
  if (h != 0) {
    int zero = 0;
    TBBT_CUDA_TRY(cudaMemcpyToSymbol(g_tbbt_error, &zero, sizeof(int)));
    return TBBT_ETIMEOUT;
  }
  return TBBT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// one-shot calls: plans cached by shape
// ---------------------------------------------------------------------------
namespace {
std::mutex g_cache_mu;
std::map<std::tuple<int, int64_t, int64_t, int64_t>, tbbt_plan *> g_cache;

tbbt_status cached_plan(tbbt_dtype dt, int64_t n, int64_t nbw, int64_t nev, tbbt_plan **out) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto key = std::make_tuple((int)dt, n, nbw, nev);
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    *out = it->second;
    return TBBT_OK;
  }
  tbbt_plan *p = nullptr;
  tbbt_status st = tbbt_plan_create(&p, dt, n, nbw, nev, nullptr);
  if (st != TBBT_OK) return st;
  g_cache[key] = p;
  *out = p;
  return TBBT_OK;
}

tbbt_status one_shot(tbbt_dtype dt, const void *hh_v, const void *hh_tau, int64_t n, int64_t nbw, int64_t nev,
                     void *q, int64_t ldq, void *stream) {
  tbbt_status st = check_shape(n, nbw, nev);
  if (st != TBBT_OK) return st;
  if (ldq < (n > 1 ? n : 1)) return TBBT_EINVAL;
  if (nev > 0 && n > 0 && !q) return TBBT_EINVAL;
  if (nev == 0) return TBBT_OK;
  tbbt_plan *p = nullptr;
  st = cached_plan(dt, n, nbw, nev, &p);
  if (st != TBBT_OK) return st;
  st = tbbt_plan_set_reflectors(p, hh_v, hh_tau, stream);
  if (st != TBBT_OK) return st;
  return tbbt_plan_execute(p, q, ldq, stream);
}

tbbt_status one_shot_host(tbbt_dtype dt, const void *hh_v, const void *hh_tau, int64_t n, int64_t nbw,
                          int64_t nev, void *q, int64_t ldq, void *stream) {
  tbbt_status st = check_shape(n, nbw, nev);
  if (st != TBBT_OK) return st;
  if (ldq < (n > 1 ? n : 1)) return TBBT_EINVAL;
  if (nev == 0) return TBBT_OK;
  if (!q) return TBBT_EINVAL;
  tbbt_plan *p = nullptr;
  st = cached_plan(dt, n, nbw, nev, &p);
  if (st != TBBT_OK) return st;
  const size_t es = elem_size(dt);
  cudaStream_t s = (cudaStream_t)stream;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (p->K > 0 && !p->d_hv) {
      TBBT_CUDA_TRY(cudaMalloc(&p->d_hv, (size_t)p->K * nbw * es));
      TBBT_CUDA_TRY(cudaMalloc(&p->d_ht, (size_t)p->K * es));
    }
    if (!p->d_q) {
      TBBT_CUDA_TRY(cudaMalloc(&p->d_q, (size_t)n * nev * es));
      p->d_q_ld = n;
    }
  }
  if (p->K > 0) {
    if (!hh_v || !hh_tau) return TBBT_EINVAL;
    TBBT_CUDA_TRY(cudaMemcpyAsync(p->d_hv, hh_v, (size_t)p->K * nbw * es, cudaMemcpyHostToDevice, s));
    TBBT_CUDA_TRY(cudaMemcpyAsync(p->d_ht, hh_tau, (size_t)p->K * es, cudaMemcpyHostToDevice, s));
  }
  TBBT_CUDA_TRY(cudaMemcpy2DAsync(p->d_q, (size_t)n * es, q, (size_t)ldq * es, (size_t)n * es, (size_t)nev,
                                  cudaMemcpyHostToDevice, s));
  st = tbbt_plan_set_reflectors(p, p->d_hv, p->d_ht, stream);
  if (st != TBBT_OK) return st;
  st = tbbt_plan_execute(p, p->d_q, n, stream);
  if (st != TBBT_OK) return st;
  TBBT_CUDA_TRY(cudaMemcpy2DAsync(q, (size_t)ldq * es, p->d_q, (size_t)n * es, (size_t)n * es, (size_t)nev,
                                  cudaMemcpyDeviceToHost, s));
  return TBBT_OK;
}
}  // namespace

extern "C" {

tbbt_status tbbt_trans_ev_tridi_to_band_d(const double *hh_v, const double *hh_tau, int64_t n, int64_t nbw,
                                          int64_t nev, double *q, int64_t ldq, void *stream) {
  return one_shot(TBBT_REAL64, hh_v, hh_tau, n, nbw, nev, q, ldq, stream);
}

tbbt_status tbbt_trans_ev_tridi_to_band_z(const void *hh_v, const void *hh_tau, int64_t n, int64_t nbw,
                                          int64_t nev, void *q, int64_t ldq, void *stream) {
  return one_shot(TBBT_COMPLEX128, hh_v, hh_tau, n, nbw, nev, q, ldq, stream);
}

tbbt_status tbbt_trans_ev_tridi_to_band_host_d(const double *hh_v, const double *hh_tau, int64_t n,
                                               int64_t nbw, int64_t nev, double *q, int64_t ldq, void *stream) {
  return one_shot_host(TBBT_REAL64, hh_v, hh_tau, n, nbw, nev, q, ldq, stream);
}

tbbt_status tbbt_trans_ev_tridi_to_band_host_z(const void *hh_v, const void *hh_tau, int64_t n, int64_t nbw,
                                               int64_t nev, void *q, int64_t ldq, void *stream) {
  return one_shot_host(TBBT_COMPLEX128, hh_v, hh_tau, n, nbw, nev, q, ldq, stream);
}

tbbt_status tbbt_release_cache(void) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (auto &kv : g_cache) tbbt_plan_destroy(kv.second);
  g_cache.clear();
  return TBBT_OK;
}

}  // extern "C"

#include "batch.cuh"

// ---------------------------------------------------------------------------
// Entry point that allocates nothing (no counterpart in the paper).
//
// Some callers cannot allocate device memory when they call us: every byte
// of the GPU may already belong to another allocator (a framework's caching
// allocator that reserved the device), or the caller runs in a loop where
// the host-device synchronisation implied by cudaMalloc/cudaFree is not
// acceptable (the cost the paper avoids by pre-allocating outside the work
// loop, Sec. 3.1), or it must never fail with out-of-memory at run time.
// This variant runs the same kernel instances, with the same default launch
// geometry, as the plan path but keeps all of their scratch -- the sweep-major store, the stage-offset table, the per-unit
// progress flags and the claim counter -- in one fixed array that exists
// from the moment the library's device code is loaded.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
struct NoAllocDevice {
  int ready;
  unsigned char *scratch;  // device address of g_noalloc_scratch on this device
  int sms;
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// Generation index of reflector (s, 0): the number of reflectors of stages
// 0..s-1, sum over m = n-1-s .. n-2 of ceil(m / b), from the closed form
// F(M) = sum_{m=1}^{M} ceil(m/b) = b q (q+1)/2 + r (q+1), M = q b + r.
__global__ void fill_stage_offsets_kernel(int64_t *off, StoreGeom g) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > (int64_t)g.n - 2) return;
  auto F = [&](int64_t M) -> int64_t {
    int64_t q = M / g.b, r = M - q * g.b;
    return g.b * q * (q + 1) / 2 + r * (q + 1);
  };
  off[s] = F((int64_t)g.n - 2) - F((int64_t)g.n - 2 - s);
}

// Per-device set-up, done by the first call on each device with that device
// current: resolve the array's device address (the host-side name of a
// __device__ array is only a stand-in) and allow the apply kernel the
// largest dynamic shared memory any launch uses.
tbbt_status noalloc_device(int *dev_out, NoAllocDevice **out) {
  int dev = 0;
  TBBT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return TBBT_ENOTSUP;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  NoAllocDevice &d = g_noalloc_dev[dev];
  if (!d.ready) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      (void)cudaGetLastError();
      return TBBT_ECUDA;
    }
    int sms = 0;
    TBBT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    TBBT_CUDA_TRY(allow_max_dynamic_smem(apply_fn(TBBT_REAL64, 0)));
    TBBT_CUDA_TRY(allow_max_dynamic_smem(apply_fn(TBBT_REAL64, 32)));
    TBBT_CUDA_TRY(allow_max_dynamic_smem(apply_fn(TBBT_REAL64, 64)));
    TBBT_CUDA_TRY(allow_max_dynamic_smem(apply_fn(TBBT_COMPLEX128, -1)));
    TBBT_CUDA_TRY(allow_max_dynamic_smem(apply_fn(TBBT_COMPLEX128, -64)));
    d.scratch = (unsigned char *)ptr;
    d.sms = sms;
    d.ready = 1;
  }
  *dev_out = dev;
  *out = &d;
  return TBBT_OK;
}

template <typename T>
tbbt_status noalloc_launch(NoAllocDevice &d, tbbt_dtype dtype, const void *hh_v, const void *hh_tau, int64_t n,
                           int64_t nbw, int64_t nev, void *q, int64_t ldq, cudaStream_t s) {
  const StoreGeom g{(int32_t)n, (int32_t)nbw, dtype == TBBT_COMPLEX128 ? 1 : 0};
  const int64_t K = g.num_reflectors();
  if (K == 0 || nev == 0) return TBBT_OK;
  const size_t es = elem_size(dtype);
  const int32_t ldv = round_even((int32_t)nbw);
  // the kernel instance and default launch geometry of the plan path
  const int32_t bw = window_width(dtype, nbw);
  int32_t G = 0, NB = 0, G0 = 0, NB0 = 0;
  default_geometry(dtype, &G0, &NB0);
  if (!fit_geometry(dtype, (int32_t)nbw, bw, G0, NB0, &G, &NB)) return TBBT_ENOTSUP;
  const size_t smem = smem_bytes_for(dtype, (int32_t)nbw, G, NB);
  const ApplyFn kern = apply_fn(dtype, bw);
  const int32_t strips = (int32_t)((nev + 31) / 32);
  const int32_t epochs = (g.num_sweeps() + G - 1) / G;
  const int64_t units = (int64_t)strips * epochs;
  // scratch layout: [store][stage offsets][flags][counter]
  const size_t b_store = round256((size_t)K * ldv * es);
  const size_t b_off = round256(sizeof(int64_t) * ((size_t)n + 1));
  const size_t b_flags = round256(sizeof(int) * (size_t)units);
  if (b_store + b_off + b_flags + sizeof(unsigned) > kNoAllocScratchBytes) return TBBT_ENOTSUP;
  unsigned char *base = d.scratch;
  T *store = reinterpret_cast<T *>(base);
  int64_t *off = reinterpret_cast<int64_t *>(base + b_store);
  int *flags = reinterpret_cast<int *>(base + b_store + b_off);
  unsigned *counter = reinterpret_cast<unsigned *>(base + b_store + b_off + b_flags);

  int per_sm = 0;
  TBBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, apply_threads(G, bw), smem));
  if (per_sm < 1) return TBBT_ENOTSUP;

  fill_stage_offsets_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(off, g);
  TBBT_CUDA_TRY(cudaGetLastError());
  const int threads = 256;
  const int64_t rblocks = (K + threads / 32 - 1) / (threads / 32);
  tbbt::relayout_kernel<T><<<(unsigned)rblocks, threads, 0, s>>>((const T *)hh_v, (const T *)hh_tau, off, g, ldv,
                                                                 store);
  TBBT_CUDA_TRY(cudaGetLastError());
  // the array keeps the previous call's contents: progress flags start at
  // "nothing released" and the claim counter at zero on every call
  TBBT_CUDA_TRY(cudaMemsetAsync(flags, 0x7f, sizeof(int) * (size_t)units, s));
  TBBT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  int *err = nullptr;
  TBBT_CUDA_TRY(cudaGetSymbolAddress((void **)&err, g_tbbt_error));
  tbbt::ApplyArgs a;
  a.vstore = store;
  a.q = q;
  a.ldq = ldq;
  a.g = g;
  a.nev = (int32_t)nev;
  a.ldv = ldv;
  a.G = G;
  a.NB = NB;
  a.ring = ring_rows_for((int32_t)nbw, G, NB);
  a.strips = strips;
  a.units = (int32_t)units;
  a.flags = flags;
  a.counter = counter;
  a.err = err;
  a.timeout_ns = 20000000000LL;
  a.withhold = -1;
  const int64_t resident = (int64_t)d.sms * per_sm;
  const unsigned grid = (unsigned)(units < resident ? units : resident);
  kern<<<grid, apply_threads(G, bw), smem, s>>>(a);
  TBBT_CUDA_TRY(cudaGetLastError());
  return TBBT_OK;
}

}  // namespace

extern "C" tbbt_status tbbt_trans_ev_tridi_to_band_noalloc(tbbt_dtype dtype, const void *hh_v, const void *hh_tau,
                                                           int64_t n, int64_t nbw, int64_t nev, void *q,
                                                           int64_t ldq, void *stream) {
  if (dtype != TBBT_REAL64 && dtype != TBBT_COMPLEX128) return TBBT_EINVAL;
  tbbt_status st = check_shape(n, nbw, nev);
  if (st != TBBT_OK) return st;
  if (ldq < (n > 1 ? n : 1)) return TBBT_EINVAL;
  const size_t es = elem_size(dtype);
  const int64_t K = StoreGeom{(int32_t)n, (int32_t)nbw, dtype == TBBT_COMPLEX128 ? 1 : 0}.num_reflectors();
  if (nev > 0 && (!q || (uintptr_t)q % es)) return TBBT_EINVAL;
  if (nev > 0 && K > 0 && (!hh_v || !hh_tau || (uintptr_t)hh_v % es || (uintptr_t)hh_tau % es)) return TBBT_EINVAL;
  if (nev == 0 || K == 0) return TBBT_OK;
  int dev = 0;
  NoAllocDevice *d = nullptr;
  st = noalloc_device(&dev, &d);
  if (st != TBBT_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == TBBT_COMPLEX128) return noalloc_launch<zdouble>(*d, dtype, hh_v, hh_tau, n, nbw, nev, q, ldq, s);
  return noalloc_launch<double>(*d, dtype, hh_v, hh_tau, n, nbw, nev, q, ldq, s);
}

// ---------------------------------------------------------------------------
// band -> tridiagonal reduction (bulge chasing) on the GPU
// ---------------------------------------------------------------------------
namespace {
template <typename T>
tbbt_status bulge_chase_impl(const T *band, int64_t ldb, int64_t n, int64_t nbw, T *hh_v, T *hh_tau, double *d,
                             double *e, cudaStream_t s) {
  const bool cplx = sizeof(T) == 16;
  tbbt_status st = check_shape(n, nbw, 0);
  if (st != TBBT_OK) return st;
  if (ldb < nbw + 1) return TBBT_EINVAL;
  if (n == 0) return TBBT_OK;
  if (!band || !d) return TBBT_EINVAL;
  if (n > 1 && !e) return TBBT_EINVAL;
  const StoreGeom g{(int32_t)n, (int32_t)nbw, cplx ? 1 : 0};
  const int64_t K = g.num_reflectors();
  if (K > 0 && (!hh_v || !hh_tau)) return TBBT_EINVAL;
  // the right-update block stays on chip when it fits beside the diagonal block
  const size_t smem_keep = (size_t)tbbt::bc::bc_smem_elems((int)nbw, true) * sizeof(T);
  const bool keep = smem_keep <= (size_t)kMaxSmem;
  const size_t smem = keep ? smem_keep : (size_t)tbbt::bc::bc_smem_elems((int)nbw, false) * sizeof(T);
  if (smem > (size_t)kMaxSmem) return TBBT_ENOTSUP;
  const int64_t ldw = 2 * nbw + 1;
  const int32_t nstages = cplx ? (n >= 2 ? (int32_t)n - 1 : 0) : (n >= 3 ? (int32_t)n - 2 : 0);
  std::vector<int64_t> off((size_t)std::max<int32_t>(nstages, 1), 0);
  {
    int64_t k = 0;
    for (int32_t i = 0; i < nstages; ++i) {
      off[(size_t)i] = k;
      k += (i <= n - 3) ? (n - i - 2 + nbw - 1) / nbw : 1;
    }
  }
  T *w = nullptr;
  int64_t *d_off = nullptr;
  int *progress = nullptr;  // nstages flags + the claim counter
  TBBT_CUDA_TRY(cudaMallocAsync((void **)&w, sizeof(T) * (size_t)ldw * (size_t)n, s));
  cudaError_t ce = cudaMallocAsync((void **)&d_off, sizeof(int64_t) * off.size(), s);
  if (ce == cudaSuccess) ce = cudaMallocAsync((void **)&progress, sizeof(int) * ((size_t)nstages + 1), s);
  if (ce != cudaSuccess) {
    (void)cudaGetLastError();
    if (w) cudaFreeAsync(w, s);
    if (d_off) cudaFreeAsync(d_off, s);
    return TBBT_ENOMEM;
  }
  tbbt_status rs = TBBT_OK;
  do {
    if (cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(progress, 0, sizeof(int) * ((size_t)nstages + 1), s) != cudaSuccess) {
      rs = TBBT_ECUDA;
      break;
    }
    const int64_t total = ldw * n;
    tbbt::bc::bulge_load_kernel<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(band, ldb, w, ldw, (int32_t)n,
                                                                                 (int32_t)nbw);
    if (cudaGetLastError() != cudaSuccess) {
      rs = TBBT_ECUDA;
      break;
    }
    if (nstages > 0) {
      auto kern = keep ? tbbt::bc::bulge_kernel<T, true> : tbbt::bc::bulge_kernel<T, false>;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        rs = TBBT_ECUDA;
        break;
      }
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      tbbt::bc::BcArgs<T> a;
      a.w = w;
      a.ldw = ldw;
      a.g = g;
      a.hh_v = hh_v;
      a.hh_tau = hh_tau;
      a.stage_off = d_off;
      a.nstages = nstages;
      a.progress = progress;
      a.counter = reinterpret_cast<unsigned *>(progress + nstages);
      int *err = nullptr;
      cudaGetSymbolAddress((void **)&err, g_tbbt_error);
      a.err = err;
      a.timeout_ns = 20000000000LL;
      const size_t smem2 = (size_t)tbbt::bc::bc2_smem_elems((int)nbw) * sizeof(T);
      if (keep && smem2 <= (size_t)kMaxSmem) {
        // two-CTA form: clusters of two CTAs, one stage each
        auto kern2 = tbbt::bc::bulge_cluster_kernel<T>;
        if (cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2) != cudaSuccess) {
          rs = TBBT_ECUDA;
          break;
        }
        const int clusters = std::min<int32_t>(nstages, std::max(sms / 2, 1));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(2 * clusters));
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem2;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, kern2, a) != cudaSuccess) {
          rs = TBBT_ECUDA;
          break;
        }
      } else {
        const int grid = std::min<int32_t>(nstages, sms > 0 ? sms : 1);
        kern<<<grid, 256, smem, s>>>(a);
      }
      if (cudaGetLastError() != cudaSuccess) {
        rs = TBBT_ECUDA;
        break;
      }
    }
    tbbt::bc::bulge_extract_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, ldw, (int32_t)n, d, e);
    if (cudaGetLastError() != cudaSuccess) rs = TBBT_ECUDA;
  } while (0);
  cudaFreeAsync(w, s);
  cudaFreeAsync(d_off, s);
  cudaFreeAsync(progress, s);
  return rs;
}
// Band -> full back-transformation (Eq. 6e): T factors of the 32-reflector
// blocks, then one pass per block boundary over every column strip.
namespace bfh {
namespace bf = tbbt::bf;

// Strips of whole column quads (<= 4 each). The FP64 pipe of an SM is shared
// by its resident blocks, so the time is set by the SM with the most quads:
// choose the blocks per SM (k <= per_sm) that minimise that maximum, the
// larger k on a tie (more warps to hide latency).
int64_t pick_grid(int64_t quads, int64_t nsm, int per_sm) {
  int64_t grid = 0, best_load = 0;
  for (int k = per_sm; k >= 1; --k) {
    const int64_t G = std::min<int64_t>(quads, nsm * k);
    const int64_t base = quads / G, extra = quads % G;
    if (base + (extra ? 1 : 0) > 4) continue;
    const int64_t rounds = (G + nsm - 1) / nsm;  // blocks per SM
    const int64_t load = rounds * base + (extra + nsm - 1) / nsm;
    if (grid == 0 || load < best_load) {
      grid = G;
      best_load = load;
    }
  }
  return grid ? grid : (quads + 3) / 4;  // more than 4 quads per SM slot: several waves of 4-quad strips
}

template <typename T, int RC>
tbbt_status launch_apply(const bf::Geo &g, const T *Tws, T *q, int64_t ldq, int64_t nev, int sms, cudaStream_t s) {
  const size_t smem = sizeof(bf::Smem<T, RC>);
  int per_sm = 0;
  if (cudaFuncSetAttribute(bf::bf_apply_kernel<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf::bf_apply_kernel<T, RC>, bf::ATHREADS, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return TBBT_ECUDA;
  const int64_t quads = (nev + 3) / 4;
  const int64_t grid = pick_grid(quads, std::max(sms, 1), per_sm);
  bf::ApplyArgs A;
  A.g = g;
  A.Tws = Tws;
  A.q = q;
  A.ldq = ldq;
  A.nev = (int32_t)nev;
  A.base = (int32_t)(quads / grid);
  A.extra = (int32_t)(quads % grid);
  bf::bf_apply_kernel<T, RC><<<(unsigned)grid, bf::ATHREADS, smem, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? TBBT_OK : TBBT_ECUDA;
}
}  // namespace bfh

template <typename T>
tbbt_status band_to_full_impl(const T *a, int64_t lda, const T *tau, int64_t n, int64_t nbw, int64_t nev, T *q,
                              int64_t ldq, cudaStream_t s) {
  if (n < 0 || n > (int64_t)1 << 30 || nbw < 1 || nev < 0 || nev > n) return TBBT_EINVAL;
  if (lda < std::max<int64_t>(1, n) || ldq < std::max<int64_t>(1, n)) return TBBT_EINVAL;
  const int64_t K1 = n > nbw ? n - nbw : 0;
  if (K1 == 0 || nev == 0) return TBBT_OK;
  if (!a || !tau || !q) return TBBT_EINVAL;
  if (((uintptr_t)q | (uintptr_t)a | (uintptr_t)tau) % alignof(T) != 0) return TBBT_EINVAL;
  namespace bf = tbbt::bf;
  const int32_t P = (int32_t)((K1 + bf::NB - 1) / bf::NB);
  T *Tws = nullptr;
  TBBT_CUDA_TRY(cudaMallocAsync((void **)&Tws, sizeof(T) * (size_t)P * bf::NB * bf::NB, s));
  tbbt_status rs = TBBT_OK;
  do {
    bf::Geo g;
    g.a = a;
    g.lda = lda;
    g.tau = tau;
    g.n = (int32_t)n;
    g.b = (int32_t)std::min<int64_t>(nbw, n);
    g.K1 = (int32_t)K1;
    g.P = P;
    bf::bf_tfactor_kernel<T><<<P, bf::THREADS, 0, s>>>(g, Tws);
    if (cudaGetLastError() != cudaSuccess) {
      rs = TBBT_ECUDA;
      break;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // Complex data and narrow strips (under two quads per block at three
    // blocks per SM) take 32-row chunks: more resident blocks, less fixed
    // work per pass. Wide real strips take 64-row chunks.
    const int64_t quads = (nev + 3) / 4;
    if constexpr (sizeof(T) == 16) {
      rs = bfh::launch_apply<T, 32>(g, Tws, q, ldq, nev, sms, s);
    } else {
      if (quads < 6 * (int64_t)std::max(sms, 1))
        rs = bfh::launch_apply<T, 32>(g, Tws, q, ldq, nev, sms, s);
      else
        rs = bfh::launch_apply<T, 64>(g, Tws, q, ldq, nev, sms, s);
    }
  } while (0);
  cudaFreeAsync(Tws, s);
  return rs;
}
}  // namespace

extern "C" {
tbbt_status tbbt_trans_ev_band_to_full_d(const double *a, int64_t lda, const double *tau, int64_t n, int64_t nbw,
                                         int64_t nev, double *q, int64_t ldq, void *stream) {
  return band_to_full_impl<double>(a, lda, tau, n, nbw, nev, q, ldq, (cudaStream_t)stream);
}
tbbt_status tbbt_trans_ev_band_to_full_z(const void *a, int64_t lda, const void *tau, int64_t n, int64_t nbw,
                                         int64_t nev, void *q, int64_t ldq, void *stream) {
  return band_to_full_impl<zdouble>((const zdouble *)a, lda, (const zdouble *)tau, n, nbw, nev, (zdouble *)q, ldq,
                                    (cudaStream_t)stream);
}
tbbt_status tbbt_bulge_chase_d(const double *band, int64_t ldb, int64_t n, int64_t nbw, double *hh_v, double *hh_tau,
                               double *d, double *e, void *stream) {
  return bulge_chase_impl<double>(band, ldb, n, nbw, hh_v, hh_tau, d, e, (cudaStream_t)stream);
}
tbbt_status tbbt_bulge_chase_z(const void *band, int64_t ldb, int64_t n, int64_t nbw, void *hh_v, void *hh_tau,
                               double *d, double *e, void *stream) {
  return bulge_chase_impl<zdouble>((const zdouble *)band, ldb, n, nbw, (zdouble *)hh_v, (zdouble *)hh_tau, d, e,
                                   (cudaStream_t)stream);
}
}  // extern "C"


// ---------------------------------------------------------------------------
// FP64 rate probes (the FP64 roofline's denominators, measured)
// ---------------------------------------------------------------------------
extern "C" tbbt_status tbbt_fp64_probe(int32_t kind, int32_t blocks, int32_t threads, int64_t iters, double *d_sink,
                                       double *flops, void *stream) {
  if (kind != 0 && kind != 1) return TBBT_EINVAL;
  if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !d_sink || !flops)
    return TBBT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0) {
    tbbt::probe::fma_probe_kernel<<<blocks, threads, 0, s>>>(d_sink, iters, 0.999999, 1e-6);
    *flops = 2.0 * tbbt::probe::kChains * (double)iters * (double)blocks * threads;
  } else {
    tbbt::probe::mma_probe_kernel<<<blocks, threads, 0, s>>>(d_sink, iters, 0.5);
    *flops = 512.0 * tbbt::probe::kMmaAcc * (double)iters * (double)blocks * (threads / 32);
  }
  TBBT_CUDA_TRY(cudaGetLastError());
  return TBBT_OK;
}

// ---------------------------------------------------------------------------
// Tridiagonal eigensolver for the nev lowest eigenpairs (Eq. 6c)
// ---------------------------------------------------------------------------
namespace {
// Threads per eigenvalue in the multisection: the fewest (least FP64 work)
// that still give every SM sub-partition about one warp.
int32_t bisect_group(int64_t nev, int sms) {
  const int64_t want = (int64_t)std::max(sms, 1) * 4 * 32 * 8 / 10;
  int32_t P = 1;
  while (P < 32 && nev * P < want) P *= 2;
  return P;
}

tbbt_status tridiag_eig_impl(const double *d, const double *e, int64_t n, int64_t nev, double *w, void *x,
                             int64_t ldx, tbbt_dtype xt, cudaStream_t s) {
  namespace te = tbbt::te;
  if (n < 0 || n > ((int64_t)1 << 30) || nev < 0 || nev > n) return TBBT_EINVAL;
  if (xt != TBBT_REAL64 && xt != TBBT_COMPLEX128) return TBBT_EINVAL;
  if (ldx < std::max<int64_t>(1, n)) return TBBT_EINVAL;
  if (n == 0 || nev == 0) return TBBT_OK;
  if (!d || !w || !x || (n > 1 && !e)) return TBBT_EINVAL;
  const size_t xs = xt == TBBT_COMPLEX128 ? 16 : 8;
  if (((uintptr_t)d | (uintptr_t)w | (uintptr_t)(n > 1 ? e : d)) % 8 || (uintptr_t)x % xs) return TBBT_EINVAL;
  const size_t nn = (size_t)n * (size_t)nev;
  int dev = 0, sms = 0;
  TBBT_CUDA_TRY(cudaGetDevice(&dev));
  TBBT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // workspace: e^2, bounds, five [row][vector] arrays, pivots, and a real
  // column-major copy of X when the output is complex
  const size_t b_e2 = round256(sizeof(double) * (size_t)std::max<int64_t>(n, 1));
  const size_t b_bounds = round256(sizeof(te::Bounds));
  const size_t b_f32 = round256(sizeof(float) * (size_t)std::max<int64_t>(n, 1));  // d and e^2 in FP32
  const size_t b_br = round256(sizeof(double) * (size_t)nev);                        // brackets of the FP32 phase
  const size_t b_arr = round256(sizeof(double) * nn);
  const size_t b_piv = round256(nn);
  const size_t b_xr = xt == TBBT_COMPLEX128 ? b_arr : 0;
  const size_t total = b_e2 + b_bounds + 2 * b_f32 + 2 * b_br + 5 * b_arr + b_piv + b_xr;
  unsigned char *ws = nullptr;
  TBBT_CUDA_TRY(cudaMallocAsync((void **)&ws, total, s));
  tbbt_status rs = TBBT_OK;
  do {
    double *e2 = (double *)ws;
    te::Bounds *bounds = (te::Bounds *)(ws + b_e2);
    float *d32 = (float *)(ws + b_e2 + b_bounds);
    float *e232 = (float *)(ws + b_e2 + b_bounds + b_f32);
    double *blo = (double *)(ws + b_e2 + b_bounds + 2 * b_f32);
    double *bhi = (double *)(ws + b_e2 + b_bounds + 2 * b_f32 + b_br);
    unsigned char *p = ws + b_e2 + b_bounds + 2 * b_f32 + 2 * b_br;
    te::InvitArgs A;
    A.d = d;
    A.e = e;
    A.n = (int32_t)n;
    A.nev = (int32_t)nev;
    A.w = w;
    A.bounds = bounds;
    A.u0 = (double *)p;
    A.u1 = (double *)(p + b_arr);
    A.u2 = (double *)(p + 2 * b_arr);
    A.lm = (double *)(p + 3 * b_arr);
    A.y = (double *)(p + 4 * b_arr);
    A.piv = p + 5 * b_arr;
    double *xr = xt == TBBT_COMPLEX128 ? (double *)(p + 5 * b_arr + b_piv) : (double *)x;
    const int64_t ldr = xt == TBBT_COMPLEX128 ? n : ldx;
    te::te_bounds_kernel<<<1, te::BOUNDS_THREADS, 0, s>>>(d, n > 1 ? e : d, (int32_t)n, e2, bounds, d32, e232);
    if (cudaGetLastError() != cudaSuccess) { rs = TBBT_ECUDA; break; }
    const int32_t P = bisect_group(nev, sms);
    const int64_t bthreads = 128;
    const unsigned bblocks = (unsigned)((nev * P + bthreads - 1) / bthreads);
    // FP32 phase (brackets of about 1e-5 ||T||), then the FP64 phase from them
#define TBBT_BISECT(PP)                                                                                         \
  te::te_bisect32_kernel<PP><<<bblocks, bthreads, 0, s>>>(d32, e232, (int32_t)n, (int32_t)nev, bounds, blo, bhi); \
  te::te_bisect_kernel<PP><<<bblocks, bthreads, 0, s>>>(d, e2, (int32_t)n, (int32_t)nev, bounds, w, blo, bhi)
    switch (P) {
      case 1: TBBT_BISECT(1); break;
      case 2: TBBT_BISECT(2); break;
      case 4: TBBT_BISECT(4); break;
      case 8: TBBT_BISECT(8); break;
      case 16: TBBT_BISECT(16); break;
      default: TBBT_BISECT(32); break;
    }
#undef TBBT_BISECT
    if (cudaGetLastError() != cudaSuccess) { rs = TBBT_ECUDA; break; }
    te::te_invit_kernel<<<(unsigned)((nev + te::INVIT_THREADS - 1) / te::INVIT_THREADS), te::INVIT_THREADS, 0, s>>>(A);
    if (cudaGetLastError() != cudaSuccess) { rs = TBBT_ECUDA; break; }
    te::te_tight_kernel<<<(unsigned)nev, te::TIGHT_THREADS, 0, s>>>(A);
    if (cudaGetLastError() != cudaSuccess) { rs = TBBT_ECUDA; break; }
    dim3 tg((unsigned)((n + 31) / 32), (unsigned)((nev + 31) / 32));
    te::te_transpose_kernel<<<tg, dim3(32, 8), 0, s>>>(A.y, (int32_t)n, (int32_t)nev, xr, ldr);
    if (cudaGetLastError() != cudaSuccess) { rs = TBBT_ECUDA; break; }
    te::te_reorth_kernel<<<(unsigned)nev, te::REORTH_THREADS, 0, s>>>(w, (int32_t)n, (int32_t)nev, bounds, xr, ldr);
    if (cudaGetLastError() != cudaSuccess) { rs = TBBT_ECUDA; break; }
    if (xt == TBBT_COMPLEX128) {
      te::te_to_complex_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(xr, ldr, (int32_t)n, (int32_t)nev,
                                                                        (double2 *)x, ldx);
      if (cudaGetLastError() != cudaSuccess) { rs = TBBT_ECUDA; break; }
    }
  } while (0);
  cudaFreeAsync(ws, s);
  return rs;
}
}  // namespace

extern "C" tbbt_status tbbt_tridiag_eig(const double *d, const double *e, int64_t n, int64_t nev, double *w,
                                        void *x, int64_t ldx, tbbt_dtype xtype, void *stream) {
  return tridiag_eig_impl(d, e, n, nev, w, x, ldx, xtype, (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// Band -> full back-transformation (Eq. 6e), split-precision form on tcgen05
// ---------------------------------------------------------------------------
namespace {
// Host side of the split form's layout: S_K, the (block, slot, batch) items
// in the order the slices are laid out, each (block, slot)'s first item, and
// per block the number of slots with rows (the target of its W counter).
struct BfsPlan {
  tbbt::bfs::Layout L;
  int32_t strips = 0, grid = 0;
  std::vector<tbbt::bfs::Item> items;
  std::vector<int32_t> item_base, need;
};
void bfs_make_plan(int64_t n, int64_t nbw, int64_t nev, int32_t sms, BfsPlan &pl) {
  namespace bfs = tbbt::bfs;
  bfs::Layout &L = pl.L;
  const int64_t K1 = n > nbw ? n - nbw : 0;
  L.n = (int32_t)n;
  L.b = (int32_t)std::min<int64_t>(nbw, n);
  L.K1 = (int32_t)K1;
  L.P = (int32_t)((K1 + tbbt::bf::NB - 1) / tbbt::bf::NB);
  L.ntiles = (int32_t)((n + 31) / 32);
  pl.strips = (int32_t)((nev + tbbt::tcs::WS - 1) / tbbt::tcs::WS);
  // S_K CTAs per strip, one CTA per SM: the fewest rounds of strips per CTA
  // group, each round taking about 1 / S_K of a strip's work (ties: fewer
  // slots, less exchange)
  double best = 0.0;
  L.SK = 1;
  for (int32_t sk = 1; sk <= 8 && sk <= sms; ++sk) {
    const int32_t conc = std::max(sms / sk, 1);
    const double t = (double)((pl.strips + conc - 1) / conc) / sk;
    if (sk == 1 || t < best * 0.999) {
      best = t;
      L.SK = sk;
    }
  }
  pl.grid = L.SK * std::min(pl.strips, std::max(sms / L.SK, 1));  // <= sms
  pl.items.clear();
  pl.item_base.assign((size_t)L.P * L.SK, 0);
  pl.need.assign((size_t)L.P, 0);
  for (int32_t p = 0; p < L.P; ++p)
    for (int32_t k = 0; k < L.SK; ++k) {
      pl.item_base[(size_t)p * L.SK + k] = (int32_t)pl.items.size();
      const int32_t nb = bfs::slot_batches(L, p, k);
      for (int32_t bt = 0; bt < nb; ++bt) pl.items.push_back(bfs::Item{p, k, bt, 0});
      pl.need[(size_t)p] += nb > 0;
    }
}

tbbt_status band_to_full_split_impl(const double *a, int64_t lda, const double *tau, int64_t n, int64_t nbw,
                                    int64_t nev, double *q, int64_t ldq, int32_t wait_timeout_ms,
                                    int32_t debug_withhold_cta, cudaStream_t s) {
  namespace bfs = tbbt::bfs;
  namespace bf = tbbt::bf;
  namespace tcs = tbbt::tcs;
  using D = bfs::D;
  if (n < 0 || n > (int64_t)1 << 30 || nbw < 1 || nev < 0 || nev > n) return TBBT_EINVAL;
  if (lda < std::max<int64_t>(1, n) || ldq < std::max<int64_t>(1, n)) return TBBT_EINVAL;
  if (wait_timeout_ms < 0 || debug_withhold_cta < -1) return TBBT_EINVAL;
  const int64_t K1 = n > nbw ? n - nbw : 0;
  if (K1 == 0 || nev == 0) return TBBT_OK;
  if (!a || !tau || !q) return TBBT_EINVAL;
  if (((uintptr_t)q | (uintptr_t)a | (uintptr_t)tau) % alignof(double) != 0) return TBBT_EINVAL;
  int dev = 0, major = 0, sms = 0;
  TBBT_CUDA_TRY(cudaGetDevice(&dev));
  TBBT_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  if (major != 10) return TBBT_ENOTSUP;
  TBBT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // layout: 32-reflector blocks, 32-row tiles dealt to S_K slots per 128-column strip
  if ((nev + 31) / 32 > 65535) return TBBT_ENOTSUP;  // grid of the layout transposes
  BfsPlan pl;
  bfs_make_plan(n, nbw, nev, sms, pl);
  const bfs::Layout &L = pl.L;
  const int32_t strips = pl.strips, grid = pl.grid;
  const std::vector<bfs::Item> &items = pl.items;
  const std::vector<int32_t> &item_base = pl.item_base, &need = pl.need;
  const int64_t ldc = (int64_t)strips * tcs::WS;  // row length of the row-major fixed-point Y
  // Gram chunks of the T factors: GCH rows each, block after block
  std::vector<int2> pieces;
  std::vector<int32_t> chunk_base((size_t)L.P + 1, 0);
  for (int32_t p = 0; p < L.P; ++p) {
    for (int64_t r = 32 * (int64_t)p + L.b; r < n; r += bfs::GCH) pieces.push_back(make_int2(p, (int32_t)r));
    chunk_base[(size_t)p + 1] = (int32_t)pieces.size();
  }
  // workspace (stream-ordered)
  const size_t b_T = round256(sizeof(double) * (size_t)L.P * bf::NB * bf::NB);
  const size_t b_gv = round256(sizeof(int32_t) * (size_t)L.P);
  const size_t b_items = round256(sizeof(bfs::Item) * items.size());
  const size_t b_base = round256(sizeof(int32_t) * item_base.size());
  const size_t b_need = round256(sizeof(int32_t) * need.size());
  const size_t b_sl = round256((size_t)D::BLOCK_BYTES * items.size());
  const size_t b_z = round256(sizeof(int64_t) * (size_t)n * (size_t)ldc);
  const size_t b_ce = round256(sizeof(int32_t) * (size_t)nev);
  const size_t b_wp = round256(sizeof(int64_t) * (size_t)strips * 2 * L.SK * bf::NB * tcs::WS);
  const size_t b_wc = round256(sizeof(unsigned) * (size_t)strips * L.P);
  const size_t b_pc = round256(sizeof(int2) * pieces.size());
  const size_t b_cb = round256(sizeof(int32_t) * chunk_base.size());
  const size_t b_gp = round256(sizeof(double) * pieces.size() * bf::NB * bf::NB);
  const size_t total = b_T + b_gv + b_items + b_base + b_need + b_sl + b_z + b_ce + b_wp + b_wc + b_pc + b_cb + b_gp;
  unsigned char *ws = nullptr;
  TBBT_CUDA_TRY(cudaMallocAsync((void **)&ws, total, s));
  tbbt_status rs = TBBT_OK;
  do {
    unsigned char *p0 = ws;
    double *Tws = (double *)p0; p0 += b_T;
    int32_t *gv = (int32_t *)p0; p0 += b_gv;
    bfs::Item *d_items = (bfs::Item *)p0; p0 += b_items;
    int32_t *d_base = (int32_t *)p0; p0 += b_base;
    int32_t *d_need = (int32_t *)p0; p0 += b_need;
    unsigned char *slices = p0; p0 += b_sl;
    int64_t *zfix = (int64_t *)p0; p0 += b_z;
    int32_t *colexp = (int32_t *)p0; p0 += b_ce;
    int64_t *wpart = (int64_t *)p0; p0 += b_wp;
    unsigned *wcnt = (unsigned *)p0; p0 += b_wc;
    int2 *d_pieces = (int2 *)p0; p0 += b_pc;
    int32_t *d_cbase = (int32_t *)p0; p0 += b_cb;
    double *gpart = (double *)p0;
    // the host vectors live until the end of this call: the copies below are
    // ordered on s before any kernel that reads them, and are from pageable
    // memory, which the runtime stages before returning
    if (cudaMemcpyAsync(d_items, items.data(), sizeof(bfs::Item) * items.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_base, item_base.data(), sizeof(int32_t) * item_base.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_need, need.data(), sizeof(int32_t) * need.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_pieces, pieces.data(), sizeof(int2) * pieces.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_cbase, chunk_base.data(), sizeof(int32_t) * chunk_base.size(), cudaMemcpyHostToDevice,
                        s) != cudaSuccess ||
        cudaMemsetAsync(wcnt, 0, sizeof(unsigned) * (size_t)strips * L.P, s) != cudaSuccess) {
      rs = TBBT_ECUDA;
      break;
    }
    bf::Geo g;
    g.a = a;
    g.lda = lda;
    g.tau = tau;
    g.n = (int32_t)n;
    g.b = L.b;
    g.K1 = (int32_t)K1;
    g.P = L.P;
    bfs::bfs_gram_kernel<<<(unsigned)pieces.size(), 256, 0, s>>>(g, d_pieces, gpart);
    bfs::bfs_tfactor_kernel<<<L.P, 256, 0, s>>>(g, gpart, d_cbase, Tws, gv);
    bfs::bfs_prepare_kernel<<<(unsigned)items.size(), 128, 0, s>>>(g, L, d_items, Tws, gv, slices);
    const unsigned cblocks = (unsigned)((nev + 7) / 8);
    const dim3 tgrid((unsigned)((n + 31) / 32), (unsigned)((nev + 31) / 32));
    bfs::bfs_colexp_kernel<<<cblocks, 256, 0, s>>>(q, ldq, (int32_t)n, (int32_t)nev, colexp);
    bfs::bfs_to_fixed_kernel<<<tgrid, 256, 0, s>>>(q, ldq, zfix, ldc, (int32_t)n, (int32_t)nev, colexp);
    if (cudaGetLastError() != cudaSuccess) { rs = TBBT_ECUDA; break; }
    if (allow_max_dynamic_smem(bfs::bfs_apply_kernel) != cudaSuccess) { rs = TBBT_ECUDA; break; }
    bfs::BfsArgs A;
    A.z = zfix;
    A.ldc = ldc;
    A.L = L;
    A.nev = (int32_t)nev;
    A.strips = strips;
    A.slices = slices;
    A.gv = gv;
    A.item_base = d_base;
    A.need = d_need;
    A.wpart = wpart;
    A.wcnt = wcnt;
    int *err = nullptr;
    if (cudaGetSymbolAddress((void **)&err, g_tbbt_error) != cudaSuccess) { rs = TBBT_ECUDA; break; }
    A.err = err;
    A.timeout_ns = (wait_timeout_ms > 0 ? (long long)wait_timeout_ms : 20000LL) * 1000000LL;
    A.withhold = debug_withhold_cta;
    // the slots of a strip wait for one another: a cooperative launch
    // guarantees that all CTAs are resident at once (or fails)
    void *kargs[] = {&A};
    if (cudaLaunchCooperativeKernel((const void *)bfs::bfs_apply_kernel, dim3((unsigned)grid), dim3(D::NTHREADS),
                                    kargs, (size_t)bfs::SM_BYTES, s) != cudaSuccess) {
      rs = TBBT_ECUDA;
      break;
    }
    bfs::bfs_from_fixed_kernel<<<tgrid, 256, 0, s>>>(q, ldq, zfix, ldc, (int32_t)n, (int32_t)nev, colexp);
    if (cudaGetLastError() != cudaSuccess) rs = TBBT_ECUDA;
  } while (0);
  cudaFreeAsync(ws, s);
  return rs;
}
}  // namespace

extern "C" tbbt_status tbbt_trans_ev_band_to_full_split_d(const double *a, int64_t lda, const double *tau, int64_t n,
                                                          int64_t nbw, int64_t nev, double *q, int64_t ldq,
                                                          void *stream) {
  return band_to_full_split_impl(a, lda, tau, n, nbw, nev, q, ldq, 0, -1, (cudaStream_t)stream);
}
extern "C" tbbt_status tbbt_trans_ev_band_to_full_split_opts_d(const double *a, int64_t lda, const double *tau,
                                                               int64_t n, int64_t nbw, int64_t nev, double *q,
                                                               int64_t ldq, int32_t wait_timeout_ms,
                                                               int32_t debug_withhold_cta, void *stream) {
  return band_to_full_split_impl(a, lda, tau, n, nbw, nev, q, ldq, wait_timeout_ms, debug_withhold_cta,
                                 (cudaStream_t)stream);
}

// Host-side check of the split form's layout (no GPU needed): the layout the
// launcher would use for these sizes and SM count, walked as the kernels walk
// it. Returns 0 if every row of every WY block (rows 32 p + nbw .. n - 1)
// belongs to exactly one (slot, batch, part, half, row) of the apply kernel,
// the preparation kernel maps every item's rows the same way, the items and
// their first indices agree, each block's counter target is its number of
// slots with rows (which only grows from the last block to the first), the
// in-kernel test of a slot's rows agrees with slot_batches, and every
// (strip, slot) has one CTA; a negative code names the first check that
// fails. *slots_per_strip and *items receive S_K and the item count.
extern "C" int64_t tbbt_b2f_split_layout_check(int64_t n, int64_t nbw, int64_t nev, int32_t sms,
                                              int32_t *slots_per_strip, int64_t *items_out) {
  namespace bfs = tbbt::bfs;
  if (n < 1 || nbw < 1 || nev < 1 || nev > n || sms < 1) return -1;
  if (n <= nbw) return 0;
  BfsPlan pl;
  bfs_make_plan(n, nbw, nev, sms, pl);
  const bfs::Layout &L = pl.L;
  if (slots_per_strip) *slots_per_strip = L.SK;
  if (items_out) *items_out = (int64_t)pl.items.size();
  if (pl.grid > sms || pl.grid % L.SK) return -2;
  // every (strip, slot) taken by exactly one CTA (blockIdx / S_K, stepping by grid / S_K)
  std::vector<int32_t> owner((size_t)pl.strips * L.SK, 0);
  for (int32_t bx = 0; bx < pl.grid; ++bx)
    for (int32_t st = bx / L.SK; st < pl.strips; st += pl.grid / L.SK) ++owner[(size_t)st * L.SK + bx % L.SK];
  for (int32_t c : owner)
    if (c != 1) return -3;
  std::vector<int32_t> seen((size_t)n);
  int32_t prev_active = 0;
  for (int32_t p = L.P - 1; p >= 0; --p) {
    std::fill(seen.begin(), seen.end(), 0);
    int32_t active = 0;
    const int32_t t0 = bfs::first_tile_of(L, p);
    for (int32_t k = 0; k < L.SK; ++k) {
      const int32_t f = bfs::slot_first(L, p, k), cnt = bfs::slot_count(L, p, k), nb = bfs::slot_batches(L, p, k);
      const bool has = ((((k - t0) % L.SK) + L.SK) % L.SK) < L.ntiles - t0;  // the apply kernel's mask
      if (has != (nb > 0)) return -4;
      active += nb > 0;
      const int64_t ib = pl.item_base[(size_t)p * L.SK + k];
      if (ib + nb > (int64_t)pl.items.size()) return -5;
      for (int32_t bt = 0; bt < nb; ++bt) {
        const bfs::Item &it = pl.items[(size_t)(ib + bt)];
        if (it.p != p || it.k != k || it.beta != bt) return -6;
        for (int32_t grp = 0; grp < 3; ++grp)
          for (int32_t hf = 0; hf < 2; ++hf) {
            const int32_t j = 3 * bt + grp;
            const int32_t rb = j < cnt ? 32 * (f + j * L.SK) + 16 * hf : -1;  // the apply kernel's rows
            for (int32_t i = 0; i < 16; ++i) {
              const int32_t rr = 32 * grp + 16 * hf + i;  // the item's row (the preparation kernel's)
              const int32_t jp = 3 * bt + rr / 32;
              const int32_t row_prep = jp < cnt ? 32 * (f + jp * L.SK) + (rr & 31) : -1;
              const int32_t row = rb >= 0 ? rb + i : -1;
              if (row != row_prep) return -7;
              if (row >= 0 && (row / 32) % L.SK != k) return -8;  // tile t belongs to slot t mod S_K
              if (row >= 0 && row < n) ++seen[(size_t)row];
            }
          }
      }
    }
    if (active != pl.need[(size_t)p] || active < prev_active) return -9;
    prev_active = active;
    for (int64_t r = 0; r < n; ++r) {
      const bool in_block = r >= 32 * (int64_t)p + L.b;
      if (seen[(size_t)r] > 1 || (in_block && seen[(size_t)r] != 1) || (r < 32 * (int64_t)t0 && seen[(size_t)r])) return -10;
    }
  }
  return 0;
}
