// FP64 rate probes: the denominators of the FP64 roofline, measured on the
// device the library runs on. Not part of any computation of the paper.
//
//  * fma probe: every thread runs 8 independent FP64 fused multiply-add
//    chains, a <- a * m + c with 0 < m < 1 (the chains converge to
//    c / (1 - m), so no value overflows or goes subnormal). 2 flops per FMA.
//  * mma probe: every warp runs 4 independent FP64 tensor-core products
//    (mma.sync m8n8k4, D = A B + D), 2 * 8 * 8 * 4 = 512 flops each.
//
// The caller times the launch with events on its stream; the kernels write
// one value per thread to a sink so that no work is removed by the compiler.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tbbt {
namespace probe {

constexpr int kChains = 8;
constexpr int kMmaAcc = 4;

__global__ void fma_probe_kernel(double *sink, int64_t iters, double m, double c) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 1e-3 * (double)(threadIdx.x & 31) + (double)i;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void mma_probe_kernel(double *sink, int64_t iters, double m) {
  const int lane = threadIdx.x & 31;
  double a = m * (1.0 + 1e-3 * lane), b = 1.0 / 64.0 - 1e-5 * lane;
  double d[kMmaAcc][2];
#pragma unroll
  for (int i = 0; i < kMmaAcc; ++i) d[i][0] = d[i][1] = 1e-3 * i;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kMmaAcc; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(d[i][0]), "+d"(d[i][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kMmaAcc; ++i) s += d[i][0] + d[i][1];
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace probe
}  // namespace tbbt
