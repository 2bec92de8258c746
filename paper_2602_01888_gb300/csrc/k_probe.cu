// FMA-rate probe: the arithmetic peak that the FP64 stencils are measured against.
//
// GB300's FP64 rate is a small fraction of its FP32 rate, so the FP64 smoothers are bound by
// the FP64 pipe rather than by HBM; their roofline fraction needs that pipe's peak, which no
// library routine reports.  Every thread runs kChains independent dependent-FMA chains in
// registers (enough independent work to cover the pipe latency), `iters` times, and writes
// one value so that nothing is optimised away.  Work per launch: 2 flop x kChains x iters x
// threads.  The caller times the launch with CUDA events on the stream.
#include <cuda_runtime.h>

#include "mg_kernels.h"

namespace mg {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T* __restrict__ out) {
  const T b = T(0.999999), c = T(1e-7);
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace mg

extern "C" int mgk_fma_rate(int f64, int blocks, int iters, void* out, void* stream) {
  if (blocks < 1 || iters < 1 || !out) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (f64)
    mg::k_fma_rate<double><<<blocks, 256, 0, s>>>(iters, (double*)out);
  else
    mg::k_fma_rate<float><<<blocks, 256, 0, s>>>(iters, (float*)out);
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

extern "C" double mgk_fma_rate_flops(int blocks, int iters) {
  return 2.0 * mg::kChains * (double)iters * 256.0 * (double)blocks;
}
