// Weighted-Jacobi smoothing that allocates nothing: the residual scratch array that
// mgk_jacobi_f64 takes from its caller lives here in a fixed device array instead.
//
// Some callers cannot allocate device memory when they call the smoother: code that runs
// in a latency-critical loop where a cudaMalloc/cudaFree would synchronise the device, or
// an application whose device memory is entirely owned by another allocator (a
// framework's caching pool, a fixed arena sized at start-up).  They pass only the operator,
// the iterate and the right-hand side.
//
// The array below exists once per device that loads this library and stays allocated
// until the process exits.  All calls on a device share it and it keeps whatever the last
// call left there; every element the smoother reads is written earlier in the same call,
// so nothing needs to start at zero.  Calls whose work overlaps on the GPU (different
// streams, or concurrent host threads) would use the array at the same time and race.
#include <cuda_runtime.h>

#include "mg_internal_host.h"
#include "mg_kernels.h"
#include "mg_launch.h"

namespace mg {

constexpr size_t kStaticScratchElems = size_t(1) << 20;  // 8 MiB of doubles
static __device__ __align__(256) double g_jacobi_scratch[kStaticScratchElems];

// Device address of g_jacobi_scratch in the current device's context.  The host-side
// symbol is only a stand-in; the address comes from the runtime, looked up on every call
// (cheap next to the launches) so that a context created again after cudaDeviceReset,
// where the module may load at another address, never gets a stale pointer.
static cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_jacobi_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace mg

using namespace mg;

extern "C" size_t mgk_jacobi_f64_static_capacity(void) { return kStaticScratchElems; }

extern "C" int mgk_jacobi_f64_static(const mgk_op_f64* A, double* phi, const double* b, int sweeps,
                                     double omega, void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !A->cE || !A->cN || !A->cNE || !A->cNW ||
      !A->diag || !A->dinv || !phi || !b || sweeps < 0)
    return 1;
  const size_t need = (size_t)A->pitch * (size_t)(A->periodic ? A->ny - 1 : A->ny);
  if (need > kStaticScratchElems) {
    set_error(MG_ERR_SIZE,
              "mgk_jacobi_f64_static: grid needs %zu scratch doubles (pitch x rows), the static "
              "array holds %zu",
              need, kStaticScratchElems);
    return 2;
  }
  double* tmp = nullptr;
  if (scratch_address(&tmp) != cudaSuccess) return 4;
  return launch_jacobi<double>(op_from(*A), phi, b, tmp, sweeps, omega, nullptr,
                               (cudaStream_t)stream) == cudaSuccess ? 0 : 4;
}
