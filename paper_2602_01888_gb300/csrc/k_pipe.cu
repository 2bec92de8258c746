// Persistent, copy-engine-pipelined fused smoother (Sec. 2.1 Gauss-Seidel, omega = 1,
// four colours; optional prolongation-correction of Eq. 24 first).
//
// Each CTA walks a strided list of TX x TY tiles.  A tile plus a halo of 4 NS nodes of
// all seven arrays (iterate, right-hand side, E/N/NE/NW couplings, 1/diag) is brought
// into one of two shared-memory stages by 2-D tensor-map copies (TMA: one box per array,
// or per CH-row chunk on a periodic level so that no box straddles the seam), completed
// on an mbarrier, while the previous tile is smoothed from the other stage.  NS sweeps of four colour phases run in shared memory;
// the valid region shrinks by one node per phase, so the tile interior is exact.  The
// iterate is read from xin and written to xout.
//
// Out-of-grid parts of a box are filled with zeros by the copy engine; they are never
// used: only unknowns are updated, and every neighbour of an unknown lies inside the grid.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "mg_common.cuh"
#include "mg_fused.h"
#include "mg_launch.h"
#include "mg_pipe.h"
#include "mg_tile.h"

namespace mg {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait on an mbarrier phase: gives up after kPipeSpinLimit polls, records the
// failure in *err (if given) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* err) {
  for (long long k = 0; k < kPipeSpinLimit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) atomicExch(err, 1);
  return false;
}

template <typename T, int TX, int TY, int NS>
struct PipeGeom {
  static constexpr int H = 4 * NS;
  static constexpr int RX = TX + 2 * H, RY = TY + 2 * H, RN = RX * RY;
  static constexpr size_t stage_bytes = (size_t)7 * RN * sizeof(T);
  static_assert((RX * sizeof(T)) % 16 == 0, "row of a stage must be a multiple of 16 bytes");
  static_assert((H * sizeof(T)) % 16 == 0, "halo must keep 16-byte column alignment");
  static_assert((TX * sizeof(T)) % 16 == 0, "tile width must keep 16-byte column alignment");
};

// The seven tensor maps of a launch (iterate, b, cE, cN, cNE, cNW, dinv).
struct PipeMaps {
  CUtensorMap m[7];
};

template <typename T, int TX, int TY, int NS>
__global__ void __launch_bounds__(kPipeThreads, 1)
    k_smooth_pipe(const __grid_constant__ PipeMaps maps, Lvl<T> L, T* __restrict__ xout, int rev,
                  const T* __restrict__ eH, int pitchc, int nyrc, int tiles_x, int ntiles,
                  int chunk, const int* __restrict__ skip, int* err) {
  if (skip && *skip) return;
  using G = PipeGeom<T, TX, TY, NS>;
  constexpr int H = G::H, RX = G::RX, RY = G::RY, RN = G::RN;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[2];
  const int p = L.pitch;

  if (smem_u32(smem_raw) % 128 != 0) {  // copy destinations must be 128-byte aligned
    if (threadIdx.x == 0 && err) atomicExch(err, 2);
    return;
  }
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // one thread issues the box copies of a tile into stage s
  auto issue = [&](int tile, int s) {
    T* st = reinterpret_cast<T*>(smem_raw + s * G::stage_bytes);
    const int bx = tile % tiles_x, by = tile / tiles_x;
    const int i0 = bx * TX - H, j0 = by * TY - H;
    mbar_arrive_expect_tx(&full[s], (unsigned)G::stage_bytes);
#pragma unroll 1
    for (int a = 0; a < 7; ++a) {
      if (chunk == 0) {
        tma_load_2d(st + (size_t)a * RN, &maps.m[a], i0, j0, &full[s]);
      } else {
        for (int c = 0; c < RY / chunk; ++c) {
          int y = (j0 + c * chunk) % L.nyr;
          if (y < 0) y += L.nyr;
          tma_load_2d(st + (size_t)a * RN + (size_t)c * chunk * RX, &maps.m[a], i0, y, &full[s]);
        }
      }
    }
  };

  int tile = blockIdx.x;
  if (tile < ntiles && threadIdx.x == 0) issue(tile, 0);
  unsigned parity[2] = {0u, 0u};
  for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int s = k & 1;
    const int next = tile + gridDim.x;
    if (next < ntiles && threadIdx.x == 0) {
      // order this CTA's earlier shared-memory accesses to stage s^1 before the copies
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(next, s ^ 1);
    }
    if (!mbar_wait_bounded(&full[s], parity[s], err)) {
      // give up on this launch; first let copies already issued into the other stage land
      if (next < ntiles) mbar_wait_bounded(&full[s ^ 1], parity[s ^ 1], nullptr);
      return;
    }
    parity[s] ^= 1u;
    T* sx = reinterpret_cast<T*>(smem_raw + s * G::stage_bytes);
    T* sb = sx + RN;
    T* sE = sb + RN;
    T* sN = sE + RN;
    T* sNE = sN + RN;
    T* sNW = sNE + RN;
    T* sD = sNW + RN;
    const int bx = tile % tiles_x, by = tile / tiles_x;
    const int i0 = bx * TX - H, j0 = by * TY - H;
    if (eH) {  // prolongation-correction of the whole staged region
      for (int t = threadIdx.x; t < RN; t += blockDim.x) {
        const int lx = t % RX, ly = t / RX;
        const int i = i0 + lx;
        int j = j0 + ly;
        if (L.periodic) j = j < 0 ? j + L.nyr : (j >= L.nyr ? j - L.nyr : j);
        else if (j < 0 || j >= L.nyr) continue;
        if (!is_unknown(L, i, j)) continue;
        const int I = i >> 1, J = j >> 1;
        const int Jp = (J + 1 == nyrc) ? 0 : J + 1;
        const size_t a0 = (size_t)J * pitchc + I, c0 = (size_t)Jp * pitchc + I;
        T v;
        if (!(i & 1) && !(j & 1)) v = eH[a0];
        else if ((i & 1) && !(j & 1)) v = T(0.5) * (eH[a0] + eH[a0 + 1]);
        else if (!(i & 1)) v = T(0.5) * (eH[a0] + eH[c0]);
        else v = T(0.25) * ((eH[a0] + eH[a0 + 1]) + (eH[c0] + eH[c0 + 1]));
        sx[t] += v;
      }
      __syncthreads();
    }
#pragma unroll 1
    for (int ph = 0; ph < 4 * NS; ++ph) {
      const int c = rev ? 3 - (ph & 3) : (ph & 3);
      const int ci = colour_ci(c), cj = colour_cj(c);
      const int lo = ph + 1, hx = RX - 2 - ph, hy = RY - 2 - ph;
      const int sx0 = lo + ((ci - i0 - lo) & 1), sy0 = lo + ((cj - j0 - lo) & 1);
      const int ncx = hx >= sx0 ? (hx - sx0) / 2 + 1 : 0;
      const int ncy = hy >= sy0 ? (hy - sy0) / 2 + 1 : 0;
      for (int t = threadIdx.x; t < ncx * ncy; t += blockDim.x) {
        const int ty = t / ncx;
        const int lx = sx0 + 2 * (t - ty * ncx), ly = sy0 + 2 * ty;
        const int i = i0 + lx;
        int j = j0 + ly;
        if (L.periodic) j = j < 0 ? j + L.nyr : (j >= L.nyr ? j - L.nyr : j);
        else if (j < 0 || j >= L.nyr) continue;
        if (!is_unknown(L, i, j)) continue;
        const int kk = ly * RX + lx;
        T acc = sE[kk] * sx[kk + 1];
        acc = fma(sE[kk - 1], sx[kk - 1], acc);
        acc = fma(sN[kk], sx[kk + RX], acc);
        acc = fma(sN[kk - RX], sx[kk - RX], acc);
        acc = fma(sNE[kk], sx[kk + RX + 1], acc);
        acc = fma(sNE[kk - RX - 1], sx[kk - RX - 1], acc);
        acc = fma(sNW[kk], sx[kk + RX - 1], acc);
        acc = fma(sNW[kk - RX + 1], sx[kk - RX + 1], acc);
        sx[kk] = (sb[kk] - acc) * sD[kk];
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
      const int ty = t / TX;
      const int lx = H + (t - ty * TX), ly = H + ty;
      const int i = i0 + lx, j = j0 + ly;  // unwrapped: every node is written by one tile
      if (i >= L.nx || j >= L.nyr) continue;
      xout[(size_t)j * p + i] = sx[ly * RX + lx];
    }
    __syncthreads();  // stage s may be refilled from the next iteration on
  }
}

// ------------------------------------------------------------------ launcher
// Variants (owned tile, sweeps per launch).  Two stages of (tx + 8 ns) x (ty + 8 ns) nodes of
// seven arrays must fit in shared memory; on a periodic level the boxes are copied in chunks
// of 32 bytes' worth of rows, which the halo must be a multiple of (FP32: two sweeps).
constexpr SmoothVariant kPipeTableF64[] = {{32, 32, 1}, {64, 16, 1}};
constexpr SmoothVariant kPipeTableF32[] = {{64, 24, 2}, {32, 32, 2}, {64, 16, 2}};

template <typename T>
int pipe_variants() {
  return sizeof(T) == 8 ? 2 : 3;
}

template <typename T>
SmoothVariant pipe_variant(int v) {
  if (v < 0 || v >= pipe_variants<T>()) v = 0;
  return sizeof(T) == 8 ? kPipeTableF64[v] : kPipeTableF32[v];
}

template <typename T>
int pipe_sweeps(int v) {
  return pipe_variant<T>(v).ns;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

// 2-D map of an nx x nyr pitched array with a box of bx x by elements (zero fill outside).
template <typename T>
static bool make_map(CUtensorMap* m, const T* base, int nx, int nyr, int pitch, int bx, int by) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)nyr};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(T)};
  const cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
  const cuuint32_t es[2] = {1, 1};
  return fn(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
            (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, int TX, int TY, int NS>
static cudaError_t pipe_impl(const Op<T>& A, const T* xin, T* xout, const T* b, int rev, const T* eH,
                             int pitch_c, const int* skip, int* err, cudaStream_t s) {
  using G = PipeGeom<T, TX, TY, NS>;
  constexpr int CH = 32 / (int)sizeof(T);  // chunk rows on periodic levels (8 FP32, 4 FP64)
  static_assert(2 * G::stage_bytes <= 227 * 1024, "two stages must fit in shared memory");
  const int nyr = rows_stored(A.ny, A.periodic);
  if (A.pitch % (16 / (int)sizeof(T)) != 0) return cudaErrorInvalidValue;  // 16-byte row strides
  if (((uintptr_t)xin | (uintptr_t)b | (uintptr_t)A.cE | (uintptr_t)A.cN | (uintptr_t)A.cNE |
       (uintptr_t)A.cNW | (uintptr_t)A.dinv) % 16 != 0)
    return cudaErrorInvalidValue;
  static_assert(TY % CH == 0 && G::H % CH == 0 && G::RY % CH == 0, "chunks must tile the box");
  const int chunk = A.periodic ? CH : 0;
  if (A.periodic && nyr % CH != 0) return cudaErrorInvalidValue;
  PipeMaps maps;
  const T* arr[7] = {xin, b, A.cE, A.cN, A.cNE, A.cNW, A.dinv};
  for (int a = 0; a < 7; ++a)
    if (!make_map<T>(&maps.m[a], arr[a], A.nx, nyr, A.pitch, G::RX, chunk ? CH : G::RY))
      return cudaErrorInvalidValue;
  auto kern = k_smooth_pipe<T, TX, TY, NS>;
  const size_t sm = 2 * G::stage_bytes;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  });
  if (attr != cudaSuccess) return attr;
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  const Lvl<T> L = lvl_of(A);
  const int tx = (L.nx + TX - 1) / TX, ty = (L.nyr + TY - 1) / TY;
  const int ntiles = tx * ty;
  const int grid = ntiles < nsm ? ntiles : nsm;
  const int nyc = (A.ny - 1) / 2 + 1;
  kern<<<grid, kPipeThreads, sm, s>>>(maps, L, xout, rev, eH, pitch_c,
                                      eH ? rows_stored(nyc, A.periodic) : 0, tx, ntiles, chunk, skip,
                                      err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth_pipe(const Op<T>& A, const T* xin, T* xout, const T* b, int rev,
                               const T* eH, int pitch_c, const int* skip, int* err,
                               cudaStream_t s, int v) {
  if (v < 0 || v >= pipe_variants<T>()) v = 0;
  if constexpr (sizeof(T) == 8) {
    if (v == 1) return pipe_impl<T, 64, 16, 1>(A, xin, xout, b, rev, eH, pitch_c, skip, err, s);
    return pipe_impl<T, 32, 32, 1>(A, xin, xout, b, rev, eH, pitch_c, skip, err, s);
  } else {
    if (v == 1) return pipe_impl<T, 32, 32, 2>(A, xin, xout, b, rev, eH, pitch_c, skip, err, s);
    if (v == 2) return pipe_impl<T, 64, 16, 2>(A, xin, xout, b, rev, eH, pitch_c, skip, err, s);
    return pipe_impl<T, 64, 24, 2>(A, xin, xout, b, rev, eH, pitch_c, skip, err, s);
  }
}

template int pipe_sweeps<float>(int);
template int pipe_sweeps<double>(int);
template int pipe_variants<float>();
template int pipe_variants<double>();
template SmoothVariant pipe_variant<float>(int);
template SmoothVariant pipe_variant<double>(int);
template cudaError_t launch_smooth_pipe<float>(const Op<float>&, const float*, float*, const float*,
                                               int, const float*, int, const int*, int*,
                                               cudaStream_t, int);
template cudaError_t launch_smooth_pipe<double>(const Op<double>&, const double*, double*,
                                                const double*, int, const double*, int, const int*,
                                                int*, cudaStream_t, int);

}  // namespace mg
