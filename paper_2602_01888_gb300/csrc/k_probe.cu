// FMA-rate probe: the arithmetic peak that the FP64 stencils are measured against.
//
// GB300's FP64 rate is a small fraction of its FP32 rate, so the FP64 smoothers are bound by
// the FP64 pipe rather than by HBM; their roofline fraction needs that pipe's peak, which no
// library routine reports.  Every thread runs CH independent chains of fused multiply-adds in
// registers (enough independent work to cover the pipe latency), `iters` times, and writes
// one value so that nothing is optimised away.  Two operand patterns, since the issue rate
// can depend on which registers an FMA reads: PAT 0 multiplies every chain by the same two
// constants (a = a b + c); PAT 1 accumulates products of per-chain operands the way a stencil
// row sum does (a = x y + a, x and y distinct registers per chain).  Work per launch:
// 2 flop x CH x iters x threads.  The caller times the launch with CUDA events.
#include <cuda_runtime.h>

#include "mg_kernels.h"

namespace mg {

constexpr int kProbeThreads = 256;

template <typename T, int CH, int PAT>
__global__ void __launch_bounds__(kProbeThreads) k_fma_rate(int iters, T* __restrict__ out) {
  T a[CH], x[CH], y[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    a[k] = T(threadIdx.x + k) * T(1e-3);
    x[k] = T(0.999999) - T(k) * T(1e-9);
    y[k] = T(1e-7) * T(k + 1);
  }
  const T b = T(0.999999), c = T(1e-7);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CH; ++k) {
      if constexpr (PAT == 0)
        a[k] = fma(a[k], b, c);
      else
        a[k] = fma(x[k], y[k], a[k]);
    }
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < CH; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T, int PAT>
static cudaError_t launch_rate(int chains, int blocks, int iters, T* out, cudaStream_t s) {
  switch (chains) {
    case 4: k_fma_rate<T, 4, PAT><<<blocks, kProbeThreads, 0, s>>>(iters, out); break;
    case 8: k_fma_rate<T, 8, PAT><<<blocks, kProbeThreads, 0, s>>>(iters, out); break;
    case 16: k_fma_rate<T, 16, PAT><<<blocks, kProbeThreads, 0, s>>>(iters, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_pat(int pattern, int chains, int blocks, int iters, T* out, cudaStream_t s) {
  if (pattern == 0) return launch_rate<T, 0>(chains, blocks, iters, out, s);
  if (pattern == 1) return launch_rate<T, 1>(chains, blocks, iters, out, s);
  return cudaErrorInvalidValue;
}

}  // namespace mg

extern "C" int mgk_fma_rate(int f64, int pattern, int chains, int blocks, int iters, void* out,
                            void* stream) {
  if (blocks < 1 || iters < 1 || !out) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = f64 ? mg::launch_pat<double>(pattern, chains, blocks, iters, (double*)out, s)
                            : mg::launch_pat<float>(pattern, chains, blocks, iters, (float*)out, s);
  if (e == cudaErrorInvalidValue) return 1;
  return e == cudaSuccess ? 0 : 4;
}

extern "C" double mgk_fma_rate_flops(int chains, int blocks, int iters) {
  return 2.0 * chains * (double)iters * mg::kProbeThreads * (double)blocks;
}
