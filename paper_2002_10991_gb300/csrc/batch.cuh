// Host side of the batched form (included by tbbt.cu, one translation unit):
// many independent problems of uneven size, real and complex mixed, applied
// by one persistent launch of batch_kernel, captured with the re-layout of
// every store into one CUDA graph, with launch geometry chosen by timing.
#pragma once

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <string>

namespace {

// Default: 4 sweeps per block, 16 stages per step for real and 4 for complex
// problems (the tuner's choice on the 64-problem KS-DFT-like mix: the small
// complex step lets two blocks share an SM).
struct BatchGeom {
  int32_t G = 4, nb_real = 16, nb_cplx = 4;
};

struct BatchProblemHost {
  tbbt_problem p;
  StoreGeom g;
  int64_t K = 0;
  int32_t ldv = 0, nb = 0, ring = 0, strips = 0, epochs = 0, kind = 0;
  int32_t G = 0;  // sweeps per block
  size_t smem = 0;
  size_t store_off = 0, stage_off = 0;  // byte offsets in the shared buffers
};

}  // namespace

struct tbbt_batch {
  std::vector<BatchProblemHost> probs;
  BatchGeom geom;
  int tuned = 0;
  size_t smem = 0;
  int32_t threads = 0;  // one warp per sweep of a block
  int32_t grid = 0;
  int64_t nunits = 0;
  long long timeout_ns = 20000000000LL;
  void *d_store = nullptr;
  void *d_stage = nullptr;
  tbbt::BatchProblem *d_probs = nullptr;
  tbbt::BatchUnit *d_units = nullptr;
  int *d_flags = nullptr;
  unsigned *d_counter = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, BatchGeom> g_tune_cache;

void batch_free_device(tbbt_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->d_store) cudaFree(b->d_store);
  if (b->d_stage) cudaFree(b->d_stage);
  if (b->d_probs) cudaFree(b->d_probs);
  if (b->d_units) cudaFree(b->d_units);
  if (b->d_flags) cudaFree(b->d_flags);
  if (b->d_counter) cudaFree(b->d_counter);
  b->exec = nullptr;
  b->d_store = b->d_stage = nullptr;
  b->d_probs = nullptr;
  b->d_units = nullptr;
  b->d_flags = nullptr;
  b->d_counter = nullptr;
}

// A string that identifies the batch's shapes (not its pointers) on this GPU.
std::string batch_signature(const tbbt_batch *b) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string sig = (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) ? std::string(prop.name) : "gpu";
  std::vector<std::string> parts;
  for (const auto &h : b->probs) {
    char buf[96];
    snprintf(buf, sizeof buf, "%d:%lld:%lld:%lld", (int)h.p.dtype, (long long)h.p.n, (long long)h.p.nbw,
             (long long)h.p.nev);
    parts.push_back(buf);
  }
  std::sort(parts.begin(), parts.end());
  for (auto &s : parts) sig += "|" + s;
  return sig;
}

// Geometry and sizes of every problem for a candidate launch geometry.
tbbt_status batch_layout(tbbt_batch *b, const BatchGeom &geo) {
  b->geom = geo;
  size_t smem = 0, store = 0, stage = 0;
  int32_t warps = 1;
  int64_t units = 0;
  for (auto &h : b->probs) {
    const bool cplx = h.p.dtype == TBBT_COMPLEX128;
    h.g = StoreGeom{(int32_t)h.p.n, (int32_t)h.p.nbw, cplx ? 1 : 0};
    h.K = h.g.num_reflectors();
    h.ldv = round_even((int32_t)h.p.nbw);
    h.G = geo.G;
    h.nb = cplx ? geo.nb_cplx : geo.nb_real;
    if (h.nb > 4 * h.G) h.nb = 4 * h.G;
    h.ring = ring_rows_for((int32_t)h.p.nbw, h.G, h.nb);
    h.smem = smem_bytes_for(h.p.dtype, (int32_t)h.p.nbw, h.G, h.nb);
    if (h.smem > (size_t)kMaxSmem) return TBBT_ENOTSUP;
    smem = std::max(smem, h.smem);
    warps = std::max(warps, h.G);
    h.kind = cplx ? tbbt::kComplex : (h.p.nbw == 32 ? tbbt::kReal32 : tbbt::kRealGeneric);
    h.strips = (int32_t)((h.p.nev + 31) / 32);
    h.epochs = (h.g.num_sweeps() + h.G - 1) / h.G;
    if (h.p.nev == 0 || h.K == 0) h.strips = h.epochs = 0;
    h.store_off = store;
    store += round256((size_t)h.K * h.ldv * elem_size(h.p.dtype));
    h.stage_off = stage;
    stage += round256(sizeof(int64_t) * ((size_t)h.p.n + 1));
    units += (int64_t)h.strips * h.epochs;
  }
  b->smem = smem;
  b->threads = 32 * warps;
  b->nunits = units;
  return TBBT_OK;
}

// Allocate device arrays, build the unit queue, capture the graph, for the
// given q pointers (the caller's, or scratch copies while tuning).
tbbt_status batch_build(tbbt_batch *b, const std::vector<void *> &qs, const std::vector<int64_t> &ldqs) {
  size_t store_bytes = 0, stage_bytes = 0;
  for (auto &h : b->probs) {
    store_bytes = std::max(store_bytes, h.store_off + round256((size_t)h.K * h.ldv * elem_size(h.p.dtype)));
    stage_bytes = std::max(stage_bytes, h.stage_off + round256(sizeof(int64_t) * ((size_t)h.p.n + 1)));
  }
  const size_t np = b->probs.size();
  if (cudaMalloc(&b->d_store, std::max<size_t>(store_bytes, 256)) != cudaSuccess ||
      cudaMalloc(&b->d_stage, std::max<size_t>(stage_bytes, 256)) != cudaSuccess ||
      cudaMalloc(&b->d_probs, sizeof(tbbt::BatchProblem) * np) != cudaSuccess ||
      cudaMalloc(&b->d_units, sizeof(tbbt::BatchUnit) * std::max<int64_t>(b->nunits, 1)) != cudaSuccess ||
      cudaMalloc(&b->d_flags, sizeof(int) * std::max<int64_t>(b->nunits, 1)) != cudaSuccess ||
      cudaMalloc(&b->d_counter, sizeof(unsigned)) != cudaSuccess) {
    (void)cudaGetLastError();
    return TBBT_ENOMEM;
  }
  int *err = nullptr;
  TBBT_CUDA_TRY(cudaGetSymbolAddress((void **)&err, g_tbbt_error));
  // per-problem stage offsets and kernel arguments
  std::vector<tbbt::BatchProblem> hp(np);
  for (size_t i = 0; i < np; ++i) {
    const auto &h = b->probs[i];
    std::vector<int64_t> off((size_t)h.p.n + 1, 0);
    int64_t k = 0;
    for (int64_t s = 0; s < h.p.n; ++s) {
      off[(size_t)s] = k;
      k += (s + 3 <= h.p.n) ? (h.p.n - s - 2 + h.p.nbw - 1) / h.p.nbw : ((h.g.cplx && s == h.p.n - 2) ? 1 : 0);
    }
    TBBT_CUDA_TRY(cudaMemcpy((char *)b->d_stage + h.stage_off, off.data(), sizeof(int64_t) * off.size(),
                             cudaMemcpyHostToDevice));
    tbbt::ApplyArgs &a = hp[i].a;
    memset(&a, 0, sizeof a);
    a.vstore = (char *)b->d_store + h.store_off;
    a.q = qs[i];
    a.ldq = ldqs[i];
    a.g = h.g;
    a.nev = (int32_t)h.p.nev;
    a.ldv = h.ldv;
    a.G = h.G;
    a.NB = h.nb;
    a.ring = h.ring;
    a.strips = h.strips;
    a.err = err;
    a.timeout_ns = b->timeout_ns;
    a.withhold = -1;
    hp[i].kind = h.kind;
  }
  TBBT_CUDA_TRY(cudaMemcpy(b->d_probs, hp.data(), sizeof(tbbt::BatchProblem) * np, cudaMemcpyHostToDevice));
  // the queue: epoch-major; within an epoch, problems with the longest
  // columns (largest n, the longest dependency chains) first
  std::vector<size_t> order(np);
  for (size_t i = 0; i < np; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](size_t x, size_t y) { return b->probs[x].p.n > b->probs[y].p.n; });
  int32_t max_e = 0;
  for (auto &h : b->probs) max_e = std::max(max_e, h.epochs);
  std::vector<tbbt::BatchUnit> units;
  units.reserve((size_t)b->nunits);
  std::vector<std::vector<int32_t>> last(np);  // queue index of (problem, strip) in the previous epoch
  for (size_t i = 0; i < np; ++i) last[i].assign((size_t)b->probs[i].strips, -1);
  for (int32_t ep = 0; ep < max_e; ++ep)
    for (size_t oi = 0; oi < np; ++oi) {
      const size_t i = order[oi];
      if (ep >= b->probs[i].epochs) continue;
      for (int32_t s = 0; s < b->probs[i].strips; ++s) {
        tbbt::BatchUnit un{(int32_t)i, s, ep, last[i][(size_t)s]};
        last[i][(size_t)s] = (int32_t)units.size();
        units.push_back(un);
      }
    }
  if (!units.empty())
    TBBT_CUDA_TRY(cudaMemcpy(b->d_units, units.data(), sizeof(tbbt::BatchUnit) * units.size(),
                             cudaMemcpyHostToDevice));
  // launch geometry of the persistent kernel
  TBBT_CUDA_TRY(allow_max_dynamic_smem(tbbt::batch_kernel));
  int dev = 0, sms = 0, per_sm = 0;
  TBBT_CUDA_TRY(cudaGetDevice(&dev));
  TBBT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TBBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tbbt::batch_kernel, b->threads, b->smem));
  if (per_sm < 1) return TBBT_ENOTSUP;
  const int64_t resident = (int64_t)sms * per_sm;
  b->grid = (int32_t)std::max<int64_t>(1, std::min<int64_t>(b->nunits, resident));
  // capture: re-lay every store, reset the queue, one persistent launch
  cudaStream_t cs;
  TBBT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  tbbt_status st = TBBT_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return TBBT_ECUDA;
  }
  for (size_t i = 0; i < np; ++i) {
    const auto &h = b->probs[i];
    if (h.K == 0 || h.p.nev == 0) continue;
    const int threads = 256;
    const int64_t rblocks = (h.K + threads / 32 - 1) / (threads / 32);
    const int64_t *off = (const int64_t *)((char *)b->d_stage + h.stage_off);
    void *dst = (char *)b->d_store + h.store_off;
    if (h.g.cplx)
      tbbt::relayout_kernel<zdouble><<<(unsigned)rblocks, threads, 0, cs>>>(
          (const zdouble *)h.p.hh_v, (const zdouble *)h.p.hh_tau, off, h.g, h.ldv, (zdouble *)dst);
    else
      tbbt::relayout_kernel<double><<<(unsigned)rblocks, threads, 0, cs>>>(
          (const double *)h.p.hh_v, (const double *)h.p.hh_tau, off, h.g, h.ldv, (double *)dst);
  }
  if (b->nunits > 0) {
    cudaMemsetAsync(b->d_flags, 0x7f, sizeof(int) * (size_t)b->nunits, cs);
    cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned), cs);
    tbbt::BatchArgs ba{b->d_probs, b->d_units, (int32_t)b->nunits, b->d_flags, b->d_counter, err};
    tbbt::batch_kernel<<<(unsigned)b->grid, b->threads, b->smem, cs>>>(ba);
  }
  if (cudaStreamEndCapture(cs, &graph) != cudaSuccess || !graph) st = TBBT_ECUDA;
  if (st == TBBT_OK && cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess) st = TBBT_ECUDA;
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  (void)cudaGetLastError();
  return st;
}

// Times one candidate geometry on scratch copies of every q (the caller's
// data stay untouched). Returns milliseconds per execution, or < 0.
double batch_time_candidate(tbbt_batch *b, const BatchGeom &geo, const std::vector<void *> &scratch,
                            const std::vector<int64_t> &lds) {
  if (batch_layout(b, geo) != TBBT_OK) return -1.0;
  if (batch_build(b, scratch, lds) != TBBT_OK) {
    batch_free_device(b);
    return -1.0;
  }
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    batch_free_device(b);
    return -1.0;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaGraphLaunch(b->exec, s);  // warm-up
  cudaEventRecord(e0, s);
  cudaGraphLaunch(b->exec, s);
  cudaEventRecord(e1, s);
  float ms = -1.0f;
  if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  int h = 0;
  cudaMemcpyFromSymbol(&h, g_tbbt_error, sizeof(int));
  batch_free_device(b);
  (void)cudaGetLastError();
  return h != 0 ? -1.0 : (double)ms;
}

bool read_tune_file(const char *path, const std::string &sig, BatchGeom *out) {
  if (!path || !*path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[8192];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    std::string s(line);
    size_t tab = s.find('\t');
    if (tab == std::string::npos || s.substr(0, tab) != sig) continue;
    BatchGeom g;
    if (sscanf(s.c_str() + tab + 1, "%d %d %d", &g.G, &g.nb_real, &g.nb_cplx) == 3) {
      *out = g;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void append_tune_file(const char *path, const std::string &sig, const BatchGeom &g) {
  if (!path || !*path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%d %d %d\n", sig.c_str(), g.G, g.nb_real, g.nb_cplx);
  fclose(f);
}

}  // namespace

extern "C" {

tbbt_status tbbt_batch_create(tbbt_batch **out, int32_t count, const tbbt_problem *problems,
                              const tbbt_batch_options *opt) {
  if (!out) return TBBT_EINVAL;
  *out = nullptr;
  if (count < 1 || !problems) return TBBT_EINVAL;
  tbbt_batch *b = new (std::nothrow) tbbt_batch();
  if (!b) return TBBT_ENOMEM;
  for (int32_t i = 0; i < count; ++i) {
    const tbbt_problem &p = problems[i];
    const size_t es = p.dtype == TBBT_COMPLEX128 ? 16 : 8;
    tbbt_status st = (p.dtype == TBBT_REAL64 || p.dtype == TBBT_COMPLEX128) ? check_shape(p.n, p.nbw, p.nev)
                                                                            : TBBT_EINVAL;
    if (st == TBBT_OK && p.ldq < (p.n > 1 ? p.n : 1)) st = TBBT_EINVAL;
    const int64_t K = StoreGeom{(int32_t)p.n, (int32_t)p.nbw, p.dtype == TBBT_COMPLEX128 ? 1 : 0}.num_reflectors();
    if (st == TBBT_OK && p.nev > 0 && (!p.q || (uintptr_t)p.q % es)) st = TBBT_EINVAL;
    if (st == TBBT_OK && p.nev > 0 && K > 0 &&
        (!p.hh_v || !p.hh_tau || (uintptr_t)p.hh_v % es || (uintptr_t)p.hh_tau % es))
      st = TBBT_EINVAL;
    if (st != TBBT_OK) {
      delete b;
      return st;
    }
    BatchProblemHost h;
    h.p = p;
    b->probs.push_back(h);
  }
  if (opt && opt->wait_timeout_ms > 0) b->timeout_ns = (long long)opt->wait_timeout_ms * 1000000LL;
  std::vector<void *> qs;
  std::vector<int64_t> lds;
  for (auto &h : b->probs) {
    qs.push_back(h.p.q);
    lds.push_back(h.p.ldq);
  }
  BatchGeom geo;
  if (opt && opt->sweeps_per_block > 0) geo.G = opt->sweeps_per_block;
  if (opt && opt->stages_per_step_real > 0) geo.nb_real = opt->stages_per_step_real;
  if (opt && opt->stages_per_step_complex > 0) geo.nb_cplx = opt->stages_per_step_complex;
  if (geo.G > 4) geo.G = geo.G >= 8 ? 8 : 4;  // one or two warps per SM sub-partition
  // a geometry that fits, preferably two blocks per SM
  while (batch_layout(b, geo) == TBBT_ENOTSUP && (geo.nb_cplx > 1 || geo.nb_real > 1)) {
    if (geo.nb_cplx > 1) geo.nb_cplx /= 2;
    else geo.nb_real /= 2;
  }
  if (!(opt && (opt->stages_per_step_real > 0 || opt->stages_per_step_complex > 0))) {
    while (b->smem > (size_t)kMaxSmem / 2 && (geo.nb_cplx > 2 || geo.nb_real > 2)) {
      if (geo.nb_cplx > 2) geo.nb_cplx /= 2;
      else geo.nb_real /= 2;
      if (batch_layout(b, geo) != TBBT_OK) break;
    }
  }
  tbbt_status st = batch_layout(b, geo);
  if (st != TBBT_OK) {
    delete b;
    return st;
  }
  if (opt && opt->autotune) {
    const std::string sig = batch_signature(b);
    const char *path = opt->autotune_cache ? opt->autotune_cache : getenv("TBBT_AUTOTUNE_CACHE");
    BatchGeom best;
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(sig);
      if (it != g_tune_cache.end()) {
        best = it->second;
        have = true;
      }
    }
    if (!have && read_tune_file(path, sig, &best)) have = true;
    if (!have) {
      // Candidates are timed on a proxy of the batch: the same problems with
      // 1/16 of their columns (whole 32-column strips, at least one), on
      // scratch copies of those columns (the caller's data stay untouched).
      // Every unit's work is unchanged and there are still far more units
      // than resident blocks, so the proxy ranks geometries as the batch
      // does, at a sixteenth of the cost.
      tbbt_batch px;
      px.probs = b->probs;
      px.timeout_ns = b->timeout_ns;
      std::vector<void *> scratch(px.probs.size(), nullptr);
      std::vector<int64_t> sld(px.probs.size(), 1);
      bool ok = true;
      for (size_t i = 0; i < px.probs.size() && ok; ++i) {
        auto &h = px.probs[i];
        const size_t es = elem_size(h.p.dtype);
        sld[i] = std::max<int64_t>(1, h.p.n);
        if (h.p.nev == 0) continue;
        h.p.nev = std::min<int64_t>(h.p.nev, std::max<int64_t>(32, (h.p.nev / 16 + 31) / 32 * 32));
        ok = cudaMalloc(&scratch[i], (size_t)sld[i] * h.p.nev * es) == cudaSuccess &&
             cudaMemcpy2D(scratch[i], (size_t)sld[i] * es, h.p.q, (size_t)h.p.ldq * es, (size_t)h.p.n * es,
                          (size_t)h.p.nev, cudaMemcpyDeviceToDevice) == cudaSuccess;
      }
      double best_ms = -1.0;
      const BatchGeom cands[] = {{4, 8, 8}, {4, 8, 4}, {4, 16, 4}, {4, 4, 4}, {8, 8, 4}, {8, 16, 8}};
      for (const BatchGeom &c : cands) {
        if (!ok) break;
        double ms = batch_time_candidate(&px, c, scratch, sld);
        if (ms > 0 && (best_ms < 0 || ms < best_ms)) {
          best_ms = ms;
          best = c;
        }
      }
      for (void *p : scratch)
        if (p) cudaFree(p);
      (void)cudaGetLastError();
      if (best_ms > 0) {
        have = true;
        append_tune_file(path, sig, best);
      }
    }
    if (have) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[sig] = best;
      geo = best;
      b->tuned = 1;
    }
    st = batch_layout(b, geo);
    if (st != TBBT_OK) {
      delete b;
      return st;
    }
  }
  st = batch_build(b, qs, lds);
  if (st != TBBT_OK) {
    batch_free_device(b);
    delete b;
    return st;
  }
  *out = b;
  return TBBT_OK;
}

tbbt_status tbbt_batch_execute(tbbt_batch *b, void *stream) {
  if (!b || !b->exec) return TBBT_EINVAL;
  TBBT_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return TBBT_OK;
}

tbbt_status tbbt_batch_info(const tbbt_batch *b, int32_t *sweeps_per_block, int32_t *stages_real,
                            int32_t *stages_complex, int32_t *blocks, int64_t *units, int32_t *tuned) {
  if (!b) return TBBT_EINVAL;
  if (sweeps_per_block) *sweeps_per_block = b->geom.G;
  if (stages_real) *stages_real = b->geom.nb_real;
  if (stages_complex) *stages_complex = b->geom.nb_cplx;
  if (blocks) *blocks = b->grid;
  if (units) *units = b->nunits;
  if (tuned) *tuned = b->tuned;
  return TBBT_OK;
}

tbbt_status tbbt_batch_destroy(tbbt_batch *b) {
  if (!b) return TBBT_OK;
  cudaDeviceSynchronize();
  batch_free_device(b);
  delete b;
  return TBBT_OK;
}

}  // extern "C"
