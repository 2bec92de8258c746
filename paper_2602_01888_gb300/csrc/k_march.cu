// Row-marching temporally blocked smoother: NS four-colour Gauss-Seidel sweeps (Sec. 2.1,
// omega = 1) in one pass over the level, with an optional prolongation-correction
// (Eq. 24) of the iterate as it is read.
//
// Each CTA owns a strip of W = C - 2 HX columns and a segment of S rows.  It streams the
// rows of the strip plus a halo of HX columns and HY = 4 NS rows on each side from the
// bottom up through a ring of R rows in shared memory (all seven arrays: iterate, b, E,
// N, NE, NW couplings, 1/diag).  Each ring row is stored de-interleaved (even columns,
// then odd columns) so that the nodes of one colour and their neighbours are unit-stride.
//
// Phase ph (0 <= ph < 4 NS, colour ph mod 4, or reversed) runs on local row s - 2 ph at
// step s.  Lagging consecutive phases by two rows makes the phases of one step touch
// disjoint row triples: phase ph at row q reads rows q-1..q+1, which by then hold
// exactly the state after phase ph-1 there (phase ph-1 ran on row q+1 one step earlier,
// on row q-1 three steps earlier) and that phase ph+1 has not yet overwritten (it reaches
// row q-1 one step later).  So a step needs one barrier, and at each step only the
// phases whose colour lives on rows of the step's parity do work, 2 NS of them, one
// thread group each.  As in a tile of the same halo, phase ph updates only rows and
// columns at distance > ph from the loaded edge; after 4 NS phases the owned rows and
// columns hold exactly the result of NS sequential sweeps.
//
// Geometry per precision: FP32 two sweeps a pass on 256-column strips, FP64 one sweep a
// pass on 128-column strips by default; the other depth of each is a variant the autotuner
// may pick (MarchGeom below).
//
// The threads of a CTA have one role each, in whole warps: compute threads run the
// phases; loader threads request rows D steps ahead with asynchronous 16-byte copies into
// a small staging ring (a barrier does not wait for these, unlike for plain loads, so the
// copies stay in flight across steps) and de-interleave a landed row into the main ring;
// writer threads copy finished owned rows out.  The iterate is read from xin and written
// to xout (halos of neighbouring CTAs overlap).
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "mg_common.cuh"
#include "mg_launch.h"
#include "mg_march.h"
#include "mg_tile.h"

namespace mg {

template <typename T, int CFG>
struct MarchGeom;

// Geometries, by precision and configuration number (FP32: configuration 0 is the default;
// FP64: configuration 3, see f64_cfg).  C loaded columns (C/2 per parity), HX halo columns and HY = 4 NS halo rows each
// side, R ring rows, D rows in flight, LCH 16-byte chunks per loader thread and row.
//
// FP32 0: two sweeps a pass.  1024 threads: 512 compute (4 active phases x 128 nodes), 448
// loaders (one chunk of each of the 7 arrays' rows each) and 64 writers (60 copy the owned 240
// columns of a finished row).
template <>
struct MarchGeom<float, 0> {
  static constexpr int NS = 2, C = 256, HX = 8, W = C - 2 * HX, HY = 8, R = 20, D = 6, NPT = 1, LCH = 1;
  static constexpr int THREADS = 1024, CTAS_PER_SM = 1;
};
// FP32 1: one sweep a pass; the x halo stays 8 columns (the coarse-correction copies need
// strips that start on a multiple of 8 fine columns).  768 threads (256 compute, 448 loaders,
// 60 writers).
template <>
struct MarchGeom<float, 1> {
  static constexpr int NS = 1, C = 256, HX = 8, W = C - 2 * HX, HY = 4, R = 12, D = 6, NPT = 1, LCH = 1;
  static constexpr int THREADS = 768, CTAS_PER_SM = 1;
};
// FP32 2: two sweeps a pass on 128-column strips (112 owned), two CTAs resident per SM (98 KB
// each) so that one CTA's per-row barrier overlaps the other's work.  512 threads: 256
// compute, 224 loaders, 32 writers (28 copy the owned columns).
template <>
struct MarchGeom<float, 2> {
  static constexpr int NS = 2, C = 128, HX = 8, W = C - 2 * HX, HY = 8, R = 20, D = 6, NPT = 1, LCH = 1;
  static constexpr int THREADS = 512, CTAS_PER_SM = 2;
};
// FP32 3 and 4: configuration 0 with fewer, busier threads, which spreads each thread's
// per-step bookkeeping (row and ring-slot arithmetic, loop control, the barrier) over more
// nodes: two chunks per loader thread (224 loaders), and in 3 also two nodes per compute
// thread (256 compute threads).
template <>
struct MarchGeom<float, 3> {
  static constexpr int NS = 2, C = 256, HX = 8, W = C - 2 * HX, HY = 8, R = 20, D = 6, NPT = 2, LCH = 2;
  static constexpr int THREADS = 544, CTAS_PER_SM = 1;
};
template <>
struct MarchGeom<float, 4> {
  static constexpr int NS = 2, C = 256, HX = 8, W = C - 2 * HX, HY = 8, R = 20, D = 6, NPT = 1, LCH = 2;
  static constexpr int THREADS = 800, CTAS_PER_SM = 1;
};
// FP64 0: one sweep a pass on 128-column strips.  FP64 smoothing is bound by the FP64 pipe,
// not by HBM, once each array is read once per sweep, so extra sweeps per pass mostly add
// redundant halo work.  640 threads: 128 compute (2 active phases x 64 nodes), 448 loaders
// and 64 writers (60 copy the owned 120 columns).
template <>
struct MarchGeom<double, 0> {
  static constexpr int NS = 1, C = 128, HX = 4, W = C - 2 * HX, HY = 4, R = 12, D = 4, NPT = 1, LCH = 1;
  static constexpr int THREADS = 640, CTAS_PER_SM = 1;
};
// FP64 1: two sweeps a pass: 8-column halo, 112 owned columns, a 20-row ring (184 KB); 768
// threads (256 compute, 448 loaders, 56 writers).
template <>
struct MarchGeom<double, 1> {
  static constexpr int NS = 2, C = 128, HX = 8, W = C - 2 * HX, HY = 8, R = 20, D = 4, NPT = 1, LCH = 1;
  static constexpr int THREADS = 768, CTAS_PER_SM = 1;
};
// FP64 2: one sweep a pass on 256-column strips: twice the compute warps of configuration 0
// (two per scheduler, so one warp's dependent FMA chain hides behind the other's) and half
// its redundant halo; an 11-row ring and 3 rows in flight fit 223 KB.  832 threads: 256
// compute, 448 loaders (two chunks each), 128 writers (124 copy the owned 248 columns).
template <>
struct MarchGeom<double, 2> {
  static constexpr int NS = 1, C = 256, HX = 4, W = C - 2 * HX, HY = 4, R = 11, D = 3, NPT = 1, LCH = 2;
  static constexpr int THREADS = 832, CTAS_PER_SM = 1;
};
// FP64 3: configuration 0's strips with two CTAs resident per SM (112 KB each): 416 threads
// (128 compute, 224 loaders of two chunks, 64 writers), so one CTA's barrier overlaps the
// other's compute.
template <>
struct MarchGeom<double, 3> {
  static constexpr int NS = 1, C = 128, HX = 4, W = C - 2 * HX, HY = 4, R = 11, D = 3, NPT = 1, LCH = 2;
  static constexpr int THREADS = 416, CTAS_PER_SM = 2;
};

template <typename T, int CFG>
struct MarchLayout {
  using G = MarchGeom<T, CFG>;
  static constexpr int NS = G::NS;
  static constexpr int M = G::C / 2;              // nodes per parity half
  static constexpr int VEC = 16 / sizeof(T);      // elements per 16-byte chunk
  static constexpr int CHUNKS = G::C / VEC;       // chunks per array row
  static constexpr int LPA = CHUNKS / G::LCH;     // loader threads per array
  static constexpr int NPT = G::NPT;              // nodes per compute thread (m + k M/NPT)
  static constexpr int COMPUTE = 2 * NS * M / NPT;  // compute threads of the active phases
  static constexpr int LOADERS = 7 * LPA;         // threads moving one row of all arrays
  static constexpr int WRITERS = G::W / VEC;      // threads writing one owned row
  static constexpr int ROW = 7 * G::C;            // elements of one ring row
  static constexpr int RAWS = G::D + 1;           // staging slots: rows in flight + the landed one
  // coarse correction staged per staging slot: the two coarse rows a fine row interpolates
  // from, CW values each (the strip's C/2 + 1 coarse columns, rounded up to whole chunks)
  static constexpr int CW = G::C / 2 + VEC, CCHUNKS = 2 * CW / VEC;
  static constexpr int ESTAGE = 2 * CW;
  static constexpr size_t smem_elems =
      (size_t)G::R * ROW + (size_t)RAWS * ROW + (size_t)RAWS * ESTAGE;
  static constexpr size_t smem_bytes = smem_elems * sizeof(T);
  static_assert(COMPUTE + LOADERS + WRITERS <= G::THREADS, "one role per thread");
  static_assert(COMPUTE % 32 == 0 && LOADERS % 32 == 0 && LPA % 32 == 0, "roles are whole warps");
  static_assert(CHUNKS % G::LCH == 0, "loader threads share a row's chunks evenly");
  static_assert(G::HY == 4 * NS && G::HX >= 4 * NS, "halo must cover the dependency cone");
  static_assert((G::HX * sizeof(T)) % 16 == 0, "strip start must stay 16-byte aligned");
  // rows touched at step s: s - 2 (4 NS - 1) - 2 (written out) .. s + 2 (de-interleaved)
  static_assert(G::R >= 2 * (4 * NS - 1) + 5, "ring must hold the live rows");
  static_assert(VEC % 2 == 0, "a 16-byte chunk holds whole even/odd column pairs");
  static_assert(smem_bytes * G::CTAS_PER_SM <= 226 * 1024, "resident CTAs must fit in shared memory");
};

// 16-byte vector of T: a chunk of VEC consecutive columns.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  __device__ static void split(const float4& v, float* e) { e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w; }
  __device__ static float4 join(const float* e) { return make_float4(e[0], e[1], e[2], e[3]); }
};
template <>
struct Vec16<double> {
  using type = double2;
  __device__ static void split(const double2& v, double* e) { e[0] = v.x; e[1] = v.y; }
  __device__ static double2 join(const double* e) { return make_double2(e[0], e[1]); }
};

// VEC/2 consecutive elements of one parity half of a ring row (8-byte aligned for FP32
// pairs, one element for FP64).
template <typename T, int K>
__device__ __forceinline__ void put_half(T* dst, const T* e) {
  if constexpr (K == 2) {
    *reinterpret_cast<float2*>(dst) = make_float2(e[0], e[1]);
  } else {
    static_assert(K == 1, "half chunks of 1 (FP64) or 2 (FP32) elements");
    dst[0] = e[0];
  }
}
template <typename T, int K>
__device__ __forceinline__ void get_half(const T* src, T* e) {
  if constexpr (K == 2) {
    const float2 v = *reinterpret_cast<const float2*>(src);
    e[0] = v.x;
    e[1] = v.y;
  } else {
    e[0] = src[0];
  }
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Asynchronous global-to-shared copy of 4 or 16 bytes (zero-filled when src_bytes is 0).
// Unlike a plain load it does not hold up the next barrier: its completion is awaited
// with cp.async.wait_group, so copies stay in flight across steps.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Dynamic shared memory of the kernel.  Every access below goes through a 32-bit shared
// address (base + byte offset) so that no generic 64-bit pointer arithmetic is spent on it.
extern __shared__ __align__(16) float march_smem[];

// Shared-memory loads and stores at a 32-bit address plus a compile-time byte offset.  The
// "memory" clobber keeps them ordered against the barriers and against each other.
template <int OFF = 0>
__device__ __forceinline__ float lds_f(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF) : "memory");
  return v;
}
template <int OFF = 0>
__device__ __forceinline__ double lds_d(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1+%2];" : "=d"(v) : "r"(a), "n"(OFF) : "memory");
  return v;
}
template <typename T, int OFF = 0>
__device__ __forceinline__ T lds(uint32_t a) {
  if constexpr (sizeof(T) == 4)
    return lds_f<OFF>(a);
  else
    return lds_d<OFF>(a);
}
template <typename T>
__device__ __forceinline__ void sts(uint32_t a, T v) {
  if constexpr (sizeof(T) == 4)
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
  else
    asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
// 16 bytes (one chunk of VEC elements) from shared memory into e[VEC].
template <typename T>
__device__ __forceinline__ void lds16(uint32_t a, T* e) {
  if constexpr (sizeof(T) == 4)
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(e[0]), "=f"(e[1]), "=f"(e[2]), "=f"(e[3])
                 : "r"(a)
                 : "memory");
  else
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(e[0]), "=d"(e[1]) : "r"(a) : "memory");
}
// VEC/2 consecutive elements (8 bytes for FP32 pairs, one FP64) to / from shared memory.
template <typename T>
__device__ __forceinline__ void sts_half(uint32_t a, const T* e) {
  if constexpr (sizeof(T) == 4)
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(e[0]), "f"(e[1]) : "memory");
  else
    asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(e[0]) : "memory");
}
template <typename T>
__device__ __forceinline__ void lds_half(uint32_t a, T* e) {
  if constexpr (sizeof(T) == 4)
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(e[0]), "=f"(e[1]) : "r"(a) : "memory");
  else
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(e[0]) : "r"(a) : "memory");
}
__device__ __forceinline__ void cp_async16_s(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}

// Per-thread constants of one phase parity: which phase the thread's group runs on steps
// of that parity and where its node and the node's left/right neighbours sit in a ring row.
struct MarchLane {
  int ph;                // phase index
  int own, left, right;  // byte offsets in a ring row (parity half * M + index, times the element size)
  int qlo, qhi;          // local rows the phase may update (halo shrink, grid rows)
  bool col_ok;           // column inside the shrinking halo and an interior grid column
};

template <typename T, int CFG>
__global__ void __launch_bounds__(MarchGeom<T, CFG>::THREADS, MarchGeom<T, CFG>::CTAS_PER_SM)
    k_smooth_march(Lvl<T> L, const T* __restrict__ xin, T* __restrict__ xout,
                   const T* __restrict__ b, int rev, const T* __restrict__ eH, int pitchc,
                   int nyrc, int S, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using G = MarchGeom<T, CFG>;
  using Y = MarchLayout<T, CFG>;
  constexpr int NS = G::NS;
  constexpr int C = G::C, HX = G::HX, W = G::W, HY = G::HY, D = G::D, M = Y::M, VEC = Y::VEC;
  constexpr int R = G::R, ROW = Y::ROW, RAWS = Y::RAWS;
  constexpr int LAG = 2 * (4 * NS - 1);  // rows between phase 0 and the last phase
  constexpr int E = (int)sizeof(T);      // bytes per element
  constexpr int ROWB = ROW * E;          // bytes of one ring (or staging) row
  constexpr int CB = C * E;              // bytes of one array's part of a ring row
  // shared-memory layout (byte addresses): ring of R rows, RAWS staging rows, coarse staging
  const uint32_t s_ring = smem_addr(march_smem);
  const uint32_t s_raw = s_ring + R * ROWB;
  const uint32_t s_est = s_raw + RAWS * ROWB;

  const int t = threadIdx.x;
  const int X0 = blockIdx.x * W, Y0 = blockIdx.y * S;
  const int Seff = min(S, L.nyr - Y0);
  const int Q = Seff + 2 * HY;  // loaded rows, local q <-> global row jb + q
  const int jb = Y0 - HY;       // global row of local row 0 (before periodic wrap)
  const int xl0 = X0 - HX;      // global column of local column 0 (even)
  const int p = L.pitch;
  auto wrapR = [](int x) { return x < 0 ? x + R : (x >= R ? x - R : x); };

  const bool computer = t < Y::COMPUTE;
  const int lt = t - Y::COMPUTE;
  const bool loader = lt >= 0 && lt < Y::LOADERS;
  const int wt = t - Y::COMPUTE - Y::LOADERS;
  const bool writer = wt >= 0 && wt < Y::WRITERS;

  // ---- loader role: array la, chunks lcb + k LPA (k < LCH; VEC consecutive columns each) of
  // every row
  constexpr int LCH = G::LCH, LPA = Y::LPA;
  const int la = loader ? lt / LPA : 0, lcb = loader ? lt % LPA : 0;
  const T* const lsrc = la == 0 ? xin : la == 1 ? b : la == 2 ? L.cE : la == 3 ? L.cN
                       : la == 4 ? L.cNE : la == 5 ? L.cNW : L.dinv;
  const bool corr = loader && la == 0 && eH != nullptr;
  const int I0b = xl0 >> 1;  // global coarse column of coarse staging column 0 (multiple of VEC)
  // per chunk of the thread: first global column, whether it lies in the array, byte offsets
  // in a staging row and (first even column) in a ring row
  int lcol[LCH];
  uint32_t raw_off[LCH], put_off[LCH];
  bool lcol_ok[LCH];
#pragma unroll
  for (int k = 0; k < LCH; ++k) {
    const int lc = lcb + k * LPA;
    lcol[k] = xl0 + lc * VEC;
    lcol_ok[k] = lcol[k] >= 0 && lcol[k] + VEC <= p;
    raw_off[k] = (uint32_t)((la * C + lc * VEC) * E);
    put_off[k] = (uint32_t)((la * C + lc * (VEC / 2)) * E);
  }

  // global row of local row q (wrapped on a periodic level), -1 outside a non-periodic grid
  auto grow = [&](int q) -> int {
    const int j = jb + q;
    if (L.periodic) return j < 0 ? j + L.nyr : (j >= L.nyr ? j - L.nyr : j);
    return (j >= 0 && j < L.nyr) ? j : -1;
  };
  // request local row q into staging slot rs, committed as one copy group
  auto issue = [&](int q, int rs) {
    if (q < Q) {
      const int j = grow(q);
      const T* const rowp = lsrc + (size_t)(j < 0 ? 0 : j) * p;
#pragma unroll
      for (int k = 0; k < LCH; ++k) {
        const bool ok = lcol_ok[k] && j >= 0;
        cp_async16_s(s_raw + rs * ROWB + raw_off[k], ok ? rowp + lcol[k] : lsrc, ok ? 16 : 0);
      }
      if (corr) {
        // coarse rows J = j >> 1 and the next one (wrapped when periodic) over the strip's
        // coarse columns, in 16-byte chunks shared out among the x-loader threads
        const int J = j >> 1;
        int Jp = J + 1;
        if (Jp == nyrc) Jp = L.periodic ? 0 : -1;
        const uint32_t ed = s_est + rs * (Y::ESTAGE * E);
        for (int c = lcb; c < Y::CCHUNKS; c += LPA) {
          const int k = c / (Y::CW / VEC), cc = c % (Y::CW / VEC);
          const int JJ = k ? Jp : J, I = I0b + cc * VEC;
          const bool ev = j >= 0 && JJ >= 0 && I >= 0 && I + VEC <= pitchc;
          cp_async16_s(ed + (k * Y::CW + cc * VEC) * E, ev ? eH + (size_t)JJ * pitchc + I : eH, ev ? 16 : 0);
        }
      }
    }
    cp_async_commit();
  };
  // the landed local row q (staging slot rs) into ring slot sr, de-interleaved; the
  // x-loaders add P eH (bilinear, Eq. 24) to their chunks on the way.  The coarse correction
  // is zero on the coarse boundary ring, so P eH vanishes at every fine node that is not an
  // unknown and needs no mask.  The coarse rows were brought by the x-loaders' copies of
  // the same group, so the x-loader warps wait for all of them (named barrier 1).
  auto settle = [&](int q, int rs, int sr) {
    if (q >= Q) return;
    constexpr int K = VEC / 2;  // even (and odd) columns of a chunk
    int j = -1;
    if (corr) {
      asm volatile("bar.sync 1, %0;" ::"n"(LPA) : "memory");
      j = grow(q);
    }
#pragma unroll
    for (int kk = 0; kk < LCH; ++kk) {
      const int lc = lcb + kk * LPA;
      T v[VEC];
      lds16<T>(s_raw + rs * ROWB + raw_off[kk], v);
      if (j >= 0) {
        // local coarse columns K lc .. K lc + K of rows J (a) and J + 1 (c)
        const uint32_t ed = s_est + rs * (Y::ESTAGE * E) + K * lc * E;
        T a[K + 1], c[K + 1];
#pragma unroll
        for (int e = 0; e <= K; ++e) a[e] = lds<T>(ed + e * E);
        if (!(j & 1)) {
#pragma unroll
          for (int e = 0; e < K; ++e) {
            v[2 * e] += a[e];
            v[2 * e + 1] += T(0.5) * (a[e] + a[e + 1]);
          }
        } else {
#pragma unroll
          for (int e = 0; e <= K; ++e) c[e] = lds<T>(ed + (Y::CW + e) * E);
#pragma unroll
          for (int e = 0; e < K; ++e) {
            v[2 * e] += T(0.5) * (a[e] + c[e]);
            v[2 * e + 1] += T(0.25) * ((a[e] + a[e + 1]) + (c[e] + c[e + 1]));
          }
        }
      }
      T ev[K], od[K];
#pragma unroll
      for (int e = 0; e < K; ++e) {
        ev[e] = v[2 * e];
        od[e] = v[2 * e + 1];
      }
      const uint32_t row = s_ring + sr * ROWB + put_off[kk];
      sts_half<T>(row, ev);          // even columns
      sts_half<T>(row + M * E, od);  // odd columns
    }
  };

  // ---- compute role: group grp runs phase 2 grp + parity on node m of a parity half
  constexpr int MH = M / Y::NPT;  // compute threads per phase group
  const int grp = computer ? t / MH : 0, m = computer ? t % MH : 0;
  // rows a phase may touch: global unknown rows (all rows when periodic)
  const int qrow_lo = L.periodic ? 0 : 1 - jb, qrow_hi = L.periodic ? Q : L.ny - 2 - jb;
  // node mm of a parity half (mm = m or m + MH) for phase parity par
  auto lane = [&](int par, int mm) {
    MarchLane z;
    z.ph = 2 * grp + par;
    const int c = rev ? 3 - (z.ph & 3) : (z.ph & 3);
    const int ci = colour_ci(c);
    const int i = 2 * mm + ci;  // local column; its global column xl0 + i has parity ci
    const int h = ci, o = 1 - ci;
    z.own = (h * M + mm) * E;  // byte offsets in a ring row
    z.left = (o * M + mm - 1 + ci) * E;
    z.right = (o * M + mm + ci) * E;
    z.col_ok = computer && i >= 1 + z.ph && i <= C - 2 - z.ph && xl0 + i >= 1 && xl0 + i <= L.nx - 2;
    z.qlo = max(1 + z.ph, qrow_lo);
    z.qhi = min(Q - 2 - z.ph, qrow_hi);
    return z;
  };
  // lanes of the steps with s even and s odd (the phase parity is that of s + rev), for
  // each of the thread's nodes
  MarchLane l_even[Y::NPT], l_odd[Y::NPT];
#pragma unroll
  for (int k = 0; k < Y::NPT; ++k) {
    l_even[k] = lane(rev & 1, m + k * MH);
    l_odd[k] = lane((rev & 1) ^ 1, m + k * MH);
  }

  // ---- writer role: chunk wt of the owned columns of a finished row
  const int wl = HX + wt * VEC;  // even local column of the chunk
  const int wcol = xl0 + wl;
  T* const wdst = xout + wcol;

  // prologue: rows 0 and 1 settled, rows 2 .. D + 1 in flight (row r stages in slot r mod
  // RAWS; RAWS = D + 1 slots hold the D rows in flight and the one being settled)
  if (loader) {
    issue(0, 0);
    issue(1, 1);
    cp_async_wait<0>();
    settle(0, 0, 0);
    settle(1, 1, 1);
#pragma unroll 1
    for (int q = 2; q < D + 2; ++q) issue(q, q % RAWS);
  }
  __syncthreads();

  const int last_step = HY + Seff - 1 + LAG + 2;  // the last owned row is written at this step
  int sbase = 0;     // s mod R at the start of each unrolled block
  int rsn = 2 % RAWS;  // staging slot of row s + 2
#pragma unroll 1
  for (int s0 = 0; s0 <= last_step; s0 += 2) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int s = s0 + u;
      // phase ph of the thread's group on local row s - 2 ph, for each of its nodes (they
      // share the phase, hence the row and the ring slots).  Roles are whole warps, so the
      // other roles' warps branch past this block instead of issuing it predicated off.
      if (computer) {
        const MarchLane* zz = u ? l_odd : l_even;
        const MarchLane& za = zz[0];
        const int q = s - 2 * za.ph;
        if (q >= za.qlo && q <= za.qhi) {
          const int sq = wrapR(sbase + u - 2 * za.ph);
          const uint32_t bR = s_ring + sq * ROWB;  // ring rows q, q + 1, q - 1
          const uint32_t bU = s_ring + (sq + 1 == R ? 0 : sq + 1) * ROWB;
          const uint32_t bD = s_ring + (sq == 0 ? R - 1 : sq - 1) * ROWB;
          // arrays at byte offsets a CB in a ring row: 0 iterate, 1 b, 2 E, 3 N, 4 NE, 5 NW, 6 1/diag
          auto update = [&](const MarchLane& z) {
            const uint32_t r0o = bR + z.own, r0l = bR + z.left, r0r = bR + z.right;
            const uint32_t ruo = bU + z.own, rul = bU + z.left, rur = bU + z.right;
            const uint32_t rdo = bD + z.own, rdl = bD + z.left, rdr = bD + z.right;
            T acc = lds<T, 2 * CB>(r0o) * lds<T>(r0r);
            acc = fma(lds<T, 2 * CB>(r0l), lds<T>(r0l), acc);
            acc = fma(lds<T, 3 * CB>(r0o), lds<T>(ruo), acc);
            acc = fma(lds<T, 3 * CB>(rdo), lds<T>(rdo), acc);
            acc = fma(lds<T, 4 * CB>(r0o), lds<T>(rur), acc);
            acc = fma(lds<T, 4 * CB>(rdl), lds<T>(rdl), acc);
            acc = fma(lds<T, 5 * CB>(r0o), lds<T>(rul), acc);
            acc = fma(lds<T, 5 * CB>(rdr), lds<T>(rdr), acc);
            return (lds<T, CB>(r0o) - acc) * lds<T, 6 * CB>(r0o);
          };
          // every lane computes (its addresses are inside the ring row whatever its column), and
          // only lanes of updatable columns store: no divergent branch around the loads
          T v[Y::NPT];
#pragma unroll
          for (int k = 0; k < Y::NPT; ++k) v[k] = update(zz[k]);
#pragma unroll
          for (int k = 0; k < Y::NPT; ++k)
            if (zz[k].col_ok) sts<T>(bR + zz[k].own, v[k]);
        }
      }
      // write-out: local row s - LAG - 2 is final (its last phase ran at step s - 2 at the
      // latest); owned rows never wrap
      if (writer) {
        const int qo = s - LAG - 2;
        if (qo >= HY && qo < HY + Seff) {
          constexpr int K = VEC / 2;
          const uint32_t xr = s_ring + wrapR(sbase + u - LAG - 2) * ROWB;
          T ev[K], od[K], e[VEC];
          lds_half<T>(xr + (wl / 2) * E, ev);
          lds_half<T>(xr + (M + wl / 2) * E, od);
#pragma unroll
          for (int k = 0; k < K; ++k) {
            e[2 * k] = ev[k];
            e[2 * k + 1] = od[k];
          }
          T* dst = wdst + (size_t)(jb + qo) * p;
          if (wcol + VEC <= L.nx) {
            *reinterpret_cast<typename Vec16<T>::type*>(dst) = Vec16<T>::join(e);
          } else {
#pragma unroll
            for (int v = 0; v < VEC; ++v)
              if (wcol + v < L.nx) dst[v] = e[v];
          }
        }
      }
      // loaders: request row s + 2 + D into the staging slot that row s + 1 left, then
      // settle row s + 2 (requested D steps ago) into its ring slot, which last held row
      // s + 2 - R, no longer read
      if (loader) {
        const int rs_new = rsn == 0 ? RAWS - 1 : rsn - 1;  // slot of row s + 1
        issue(s + 2 + D, rs_new);
        cp_async_wait<D>();
        settle(s + 2, rsn, wrapR(sbase + u + 2));
        rsn = rsn + 1 == RAWS ? 0 : rsn + 1;
      }
      __syncthreads();
    }
    sbase = wrapR(sbase + 2);
  }
}

// Variants: the configurations of MarchGeom; variant 0 is each precision's default.
template <typename T>
int march_variants() {
  return sizeof(T) == 8 ? 4 : 5;
}

template <typename T, int CFG>
static SmoothVariant march_cfg() {
  return {MarchGeom<T, CFG>::W, 0, MarchGeom<T, CFG>::NS};
}

// FP64 variant -> configuration: variant 0 (the default) is configuration 3, measured the
// fastest at 2049^2-8193^2 (1.46 ms a sweep at 8193^2 against 1.69 for configuration 2 and
// 2.26 for configuration 0, whose four compute warps leave the FP64 pipe waiting on their
// dependent FMA chains).
static int f64_cfg(int v) {
  constexpr int cfg[4] = {3, 1, 2, 0};
  return cfg[(v < 0 || v >= 4) ? 0 : v];
}

template <typename T>
SmoothVariant march_variant(int v) {
  if (v < 0 || v >= march_variants<T>()) v = 0;
  if constexpr (sizeof(T) == 8) {
    switch (f64_cfg(v)) {
      case 1: return march_cfg<double, 1>();
      case 2: return march_cfg<double, 2>();
      case 3: return march_cfg<double, 3>();
      default: return march_cfg<double, 0>();
    }
  } else {
    switch (v) {
      case 1: return march_cfg<float, 1>();
      case 2: return march_cfg<float, 2>();
      case 3: return march_cfg<float, 3>();
      case 4: return march_cfg<float, 4>();
      default: return march_cfg<float, 0>();
    }
  }
}

template <typename T>
int march_sweeps(int v) {
  return march_variant<T>(v).ns;
}

template <typename T>
int march_strip_width(int v) {
  return march_variant<T>(v).tx;
}

template <typename T, int CFG>
static cudaError_t march_impl(const Op<T>& A, const T* xin, T* xout, const T* b, int rev, const T* eH,
                              int pitch_c, const int* skip, cudaStream_t s) {
  using G = MarchGeom<T, CFG>;
  using Y = MarchLayout<T, CFG>;
  constexpr int NS = G::NS;
  static_assert(Y::smem_bytes <= 227 * 1024, "ring and staging rows must fit in shared memory");
  if (A.pitch % Y::VEC != 0) return cudaErrorInvalidValue;
  if (((uintptr_t)xin | (uintptr_t)xout | (uintptr_t)b | (uintptr_t)A.cE | (uintptr_t)A.cN |
       (uintptr_t)A.cNE | (uintptr_t)A.cNW | (uintptr_t)A.dinv | (uintptr_t)eH) % 16 != 0)
    return cudaErrorInvalidValue;
  if (eH && pitch_c % Y::VEC != 0) return cudaErrorInvalidValue;
  if (xin == xout) return cudaErrorInvalidValue;
  auto kern = k_smooth_march<T, CFG>;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [&] {
    attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Y::smem_bytes);
    // all of the SM's unified memory as shared memory, so CTAS_PER_SM rings fit side by side
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared);
  });
  if (attr != cudaSuccess) return attr;
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  const Lvl<T> L = lvl_of(A);
  const int strips = (L.nx + G::W - 1) / G::W;
  // segment height S (even, so that local and global row parities agree): the choice with
  // the least estimated time, counting the redundant halo rows of each segment and the
  // idle SMs of a partly filled last wave (CTAS_PER_SM resident CTAs per SM)
  int S = 0;
  double best = 1e300;
  for (int segs = 1; segs <= 256; ++segs) {
    int s2 = (L.nyr + segs - 1) / segs;
    s2 = (s2 + 1) & ~1;
    if (s2 < 4 * G::HY && segs > 1) break;
    const int n = (L.nyr + s2 - 1) / s2;
    const int slots = nsm * G::CTAS_PER_SM;
    const int waves = (strips * n + slots - 1) / slots;
    const double cost = (double)waves * (s2 + 2 * G::HY + 2 * (4 * NS - 1));
    if (cost < best) {
      best = cost;
      S = s2;
    }
  }
  const int segs = (L.nyr + S - 1) / S;
  const int nyc = (A.ny - 1) / 2 + 1;
  kern<<<dim3(strips, segs), G::THREADS, Y::smem_bytes, s>>>(
      L, xin, xout, b, rev, eH, pitch_c, eH ? rows_stored(nyc, A.periodic) : 0, S, skip);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth_march(const Op<T>& A, const T* xin, T* xout, const T* b, int rev,
                                const T* eH, int pitch_c, const int* skip, cudaStream_t s, int v) {
  if (v < 0 || v >= march_variants<T>()) v = 0;
  if constexpr (sizeof(T) == 8) {
    switch (f64_cfg(v)) {
      case 1: return march_impl<double, 1>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
      case 2: return march_impl<double, 2>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
      case 3: return march_impl<double, 3>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
      default: return march_impl<double, 0>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
    }
  } else {
    switch (v) {
      case 1: return march_impl<float, 1>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
      case 2: return march_impl<float, 2>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
      case 3: return march_impl<float, 3>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
      case 4: return march_impl<float, 4>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
      default: return march_impl<float, 0>(A, xin, xout, b, rev, eH, pitch_c, skip, s);
    }
  }
}

template int march_sweeps<float>(int);
template int march_sweeps<double>(int);
template int march_strip_width<float>(int);
template int march_strip_width<double>(int);
template int march_variants<float>();
template int march_variants<double>();
template SmoothVariant march_variant<float>(int);
template SmoothVariant march_variant<double>(int);
template cudaError_t launch_smooth_march<float>(const Op<float>&, const float*, float*,
                                                const float*, int, const float*, int, const int*,
                                                cudaStream_t, int);
template cudaError_t launch_smooth_march<double>(const Op<double>&, const double*, double*,
                                                 const double*, int, const double*, int, const int*,
                                                 cudaStream_t, int);

}  // namespace mg
