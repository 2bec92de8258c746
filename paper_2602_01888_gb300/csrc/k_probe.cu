// FMA-rate probe: the arithmetic peak that the FP64 stencils are measured against.
//
// GB300's FP64 rate is a small fraction of its FP32 rate, so the FP64 smoothers are bound by
// the FP64 pipe rather than by HBM; their roofline fraction needs that pipe's peak, which no
// library routine reports.  Every thread runs CH independent dependent-FMA chains in
// registers (enough independent work to cover the pipe latency), `iters` times, and writes
// one value so that nothing is optimised away.  Work per launch: 2 flop x CH x iters x
// threads.  The caller times the launch with CUDA events on the stream.
#include <cuda_runtime.h>

#include "mg_kernels.h"

namespace mg {

constexpr int kProbeThreads = 256;

template <typename T, int CH>
__global__ void __launch_bounds__(kProbeThreads) k_fma_rate(int iters, T* __restrict__ out) {
  const T b = T(0.999999), c = T(1e-7);
  T a[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CH; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
static cudaError_t launch_rate(int chains, int blocks, int iters, T* out, cudaStream_t s) {
  switch (chains) {
    case 4: k_fma_rate<T, 4><<<blocks, kProbeThreads, 0, s>>>(iters, out); break;
    case 8: k_fma_rate<T, 8><<<blocks, kProbeThreads, 0, s>>>(iters, out); break;
    case 16: k_fma_rate<T, 16><<<blocks, kProbeThreads, 0, s>>>(iters, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mg

extern "C" int mgk_fma_rate(int f64, int chains, int blocks, int iters, void* out, void* stream) {
  if (blocks < 1 || iters < 1 || !out) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = f64 ? mg::launch_rate<double>(chains, blocks, iters, (double*)out, s)
                            : mg::launch_rate<float>(chains, blocks, iters, (float*)out, s);
  if (e == cudaErrorInvalidValue) return 1;
  return e == cudaSuccess ? 0 : 4;
}

extern "C" double mgk_fma_rate_flops(int chains, int blocks, int iters) {
  return 2.0 * chains * (double)iters * mg::kProbeThreads * (double)blocks;
}
