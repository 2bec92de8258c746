// One multigrid V(nu1, nu2) cycle (Sec. 3, Eqs. 19-24) enqueued on a stream.  Smoothing
// per level, by size: the largest levels use the row-marching kernel (FP32 two sweeps a
// pass, FP64 one), other large FP32 levels the pipelined tile kernel, other large FP64
// levels the per-colour kernels, mid-size levels the fused tile kernel (NS sweeps per launch,
// ping-pong iterates); the residual is fused with full-weighting restriction; the levels
// at and below the tail threshold run in one single-CTA tail kernel that ends with the
// coarsest dense solve.  The weighted-Jacobi smoother uses the per-sweep kernels on every
// level, the zebra x-line smoother its two launches a sweep on every level but the coarsest.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "mg.h"
#include "mg_fused.h"
#include "mg_internal_host.h"
#include "mg_kernels.h"
#include "mg_launch.h"
#include "mg_pipe.h"
#include "mg_line.h"
#include "mg_march.h"
#include "mg_tile.h"
#include "mg_vcycle.h"

namespace mg {

template <typename T>
static int default_tail_nodes() {
  // One SM runs the tail, so its phases are limited by one SM's issue rate (and, in FP64,
  // by its 2 FMA/clk), but each level it takes over saves about six launches.  Measured on
  // the 1025^2 inclusion workload: levels up to 33^2 (1200 nodes) in the tail give the
  // fastest cycle in both precisions (FP64 0.440 -> 0.414 ms, FP32 0.237 -> 0.225 ms);
  // taking 65^2 too gains nothing in FP64 and loses in FP32.
  return 1200;
}

template <typename T>
int tail_nodes() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv(sizeof(T) == 8 ? "MG_TAIL_NODES_F64" : "MG_TAIL_NODES_F32");
    v = e ? atoi(e) : default_tail_nodes<T>();
  }
  return v;
}

// Largest level the zebra x-line cycle leaves to the tail kernel (its levels must also fit the
// tail's shared memory together).  Measured on the 8193^2 annulus cycle: FP32 2.730 ms with no
// tail, 2.713 ms with the levels up to 33^2 (1200 nodes) in it, 2.742 ms up to 65^2 (the
// single CTA's sequential row solves then cost more than the launches they replace); FP64
// 6.164 ms with no tail, 6.254 ms up to 33^2, so FP64 keeps the launches.
template <typename T>
int line_tail_nodes() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv(sizeof(T) == 8 ? "MG_LINE_TAIL_NODES_F64" : "MG_LINE_TAIL_NODES_F32");
    v = e ? atoi(e) : (sizeof(T) == 8 ? 0 : 1200);
  }
  return v;
}

// Levels with more nodes than this use the per-colour smoothing kernels (four launches
// a sweep); smaller levels above the tail use the fused tile kernel.
template <typename T>
int colour_nodes() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv(sizeof(T) == 8 ? "MG_COLOUR_NODES_F64" : "MG_COLOUR_NODES_F32");
    v = e ? atoi(e) : 40000;
  }
  return v;
}

// Levels with at least this many nodes use the row-marching smoother; below it the grid has
// too few strips and segments to fill the GPU.
inline long long march_nodes() {
  static long long v = -1;
  if (v < 0) {
    const char* e = getenv("MG_MARCH_NODES");
    v = e ? atoll(e) : 2000000;
  }
  return v;
}

int SmoothPolicy::lookup(long long nodes, int* var_out) const {
  if (var_out) *var_out = -1;
  if (n <= 0 || nodes <= 0) return SK_DEFAULT;
  int best = 0;
  double bd = 1e300;
  for (int k = 0; k < n; ++k) {
    const double d = fabs(log((double)nodes) - 2.0 * log((double)side[k]));
    if (d < bd) {
      bd = d;
      best = k;
    }
  }
  if (var_out) *var_out = var[best];
  return kind[best];
}

template <typename T>
cudaError_t emit_vcycle(const VLevels<T>& V, int smoother, int nu1, int nu2, double omega,
                        const int* skip, cudaStream_t s, T** result, bool x0_zero) {
  const int L = V.L;
  T* cur[kMaxLevels];
  T* alt[kMaxLevels];
  for (int l = 0; l < L; ++l) {
    cur[l] = V.x[l];
    alt[l] = V.t[l];
  }
  cudaError_t e;
  if (smoother == MG_SMOOTH_JACOBI) {
    for (int l = 0; l < L - 1; ++l) {
      if ((e = launch_jacobi(V.A[l], cur[l], V.b[l], alt[l], nu1, omega, skip, s))) return e;
      if ((e = launch_resid_restrict(V.A[l], cur[l], V.b[l], V.b[l + 1], cur[l + 1],
                                     V.A[l + 1].pitch, skip, s)))
        return e;
    }
    if ((e = launch_coarse_solve(V.A[L - 1], V.inv, V.b[L - 1], cur[L - 1], skip, s))) return e;
    for (int l = L - 2; l >= 0; --l) {
      if ((e = launch_prolong_add(V.A[l], cur[l], cur[l + 1], V.A[l + 1].pitch, skip, s))) return e;
      if ((e = launch_jacobi(V.A[l], cur[l], V.b[l], alt[l], nu2, omega, skip, s))) return e;
    }
    *result = cur[0];
    return cudaSuccess;
  }
  if (smoother == MG_SMOOTH_XLINE) {
    // zebra x-line Gauss-Seidel on every level but the coarsest.  A coarse level's iterate
    // starts at zero, so with pre-smoothing its first half-sweep reads no iterate and the
    // restriction need not clear it; the coarse correction is added to the even rows only,
    // just before the first post-smoothing half-sweep solves the odd rows from them (see
    // launch_line_rows): identical values, one pass over half of each level's iterate.
    // The smallest levels (at most line_tail_nodes each, all in the tail kernel's shared
    // memory) run with the coarsest solve in the single-CTA tail kernel, which smooths them
    // row by row: one launch instead of about six per level, each of them latency-bound.
    const bool zs = nu1 > 0;
    int t = L - 1;
    const int thr = line_tail_nodes<T>();
    for (int l = 1; l < L - 1; ++l) {
      const long long nodes = (long long)V.A[l].nx * rows_stored(V.A[l].ny, V.A[l].periodic);
      size_t bytes = 0;
      for (int q = l; q < L; ++q)
        bytes += (size_t)9 * sizeof(T) * V.A[q].nx * rows_stored(V.A[q].ny, V.A[q].periodic);
      if (nodes <= thr && L - l <= kMaxTail && bytes <= kTailSmemMax) {
        t = l;
        break;
      }
    }
    for (int l = 0; l < t; ++l) {
      const int zero = l == 0 ? (x0_zero && zs) : zs;
      if ((e = launch_line_smooth(V.A[l], V.lf[l], cur[l], V.b[l], nu1, 0, skip, s, (const T*)nullptr, 0, zero)))
        return e;
      // the tail kernel reads the iterate of its first level: clear it there.  After
      // pre-smoothing, whose last half-sweep solved the odd rows, only the even rows'
      // residual is restricted (launch_resid_restrict_even).
      T* const xc = zs && l + 1 < t ? nullptr : cur[l + 1];
      if ((e = zs ? launch_resid_restrict_even(V.A[l], cur[l], V.b[l], V.b[l + 1], xc, V.A[l + 1].pitch, skip, s)
                  : launch_resid_restrict(V.A[l], cur[l], V.b[l], V.b[l + 1], xc, V.A[l + 1].pitch, skip, s)))
        return e;
    }
    if (t == L - 1) {
      if ((e = launch_coarse_solve(V.A[L - 1], V.inv, V.b[L - 1], cur[L - 1], skip, s))) return e;
    } else {
      TailArgs<T> ta;
      memset(&ta, 0, sizeof ta);
      ta.nlev = L - t;
      ta.nu1 = nu1;
      ta.nu2 = nu2;
      ta.line = 1;
      ta.inv = V.inv;
      for (int l = t; l < L; ++l) {
        ta.lv[l - t].L = lvl_of(V.A[l]);
        ta.lv[l - t].x = cur[l];
        ta.lv[l - t].b = V.b[l];
        ta.lv[l - t].t = alt[l];
      }
      if ((e = launch_tail(ta, skip, s))) return e;
    }
    for (int l = t - 1; l >= 0; --l) {
      if (nu2 > 0) {
        if ((e = launch_line_smooth(V.A[l], V.lf[l], cur[l], V.b[l], nu2, 1, skip, s, (const T*)cur[l + 1],
                                    V.A[l + 1].pitch, 0)))
          return e;
      } else if ((e = launch_prolong_add(V.A[l], cur[l], cur[l + 1], V.A[l + 1].pitch, skip, s))) {
        return e;
      }
    }
    *result = cur[0];
    return cudaSuccess;
  }
  // first level handled by the tail kernel
  // the tail starts at the first level that is small enough and whose levels fit in
  // the tail kernel's shared memory
  int t = L - 1;
  const int thr = tail_nodes<T>();
  for (int l = 0; l < L; ++l) {
    const long long nodes = (long long)V.A[l].nx * rows_stored(V.A[l].ny, V.A[l].periodic);
    size_t bytes = 0;
    for (int q = l; q < L; ++q)
      bytes += (size_t)9 * sizeof(T) * V.A[q].nx * rows_stored(V.A[q].ny, V.A[q].periodic);
    if ((nodes <= thr || l == L - 1) && L - l <= kMaxTail && bytes <= kTailSmemMax) {
      t = l;
      break;
    }
  }
  const long long cthr = colour_nodes<T>();
  auto smooth = [&](int l, int sweeps, int rev, const T* eH) -> cudaError_t {
    cudaError_t err;
    const long long nodes = (long long)V.A[l].nx * rows_stored(V.A[l].ny, V.A[l].periodic);
    const int nyr = rows_stored(V.A[l].ny, V.A[l].periodic);
    const int pc = eH ? V.A[l + 1].pitch : 0;
    // which families (in a given variant) can run this level with this many sweeps
    auto can = [&](int kind, int v) {
      if (sweeps <= 0) return kind == SK_COLOUR;
      switch (kind) {
        case SK_MARCH:
          return sweeps % march_sweeps<T>(v) == 0 && V.A[l].pitch % (16 / (int)sizeof(T)) == 0 && nyr >= 128;
        case SK_PIPE:
          return sweeps % pipe_sweeps<T>(v) == 0 && nyr >= 64 && V.A[l].nx >= 160 &&
                 V.A[l].pitch % (16 / (int)sizeof(T)) == 0 &&
                 (!V.A[l].periodic || nyr % (32 / (int)sizeof(T)) == 0);
        case SK_FUSED:
          return sweeps % fused_sweeps<T>(v) == 0;
        default:
          return kind == SK_COLOUR;
      }
    };
    // size-threshold rule, default variants
    int kind, var = -1;
    if (nodes >= march_nodes() && can(SK_MARCH, -1))
      kind = SK_MARCH;
    else if (sizeof(T) == 4 && nodes > cthr && can(SK_PIPE, -1))
      kind = SK_PIPE;
    else if (!can(SK_FUSED, -1) || nodes > cthr)
      kind = SK_COLOUR;
    else
      kind = SK_FUSED;
    // measured choice, where it can run
    if (V.pol) {
      int v = -1;
      const int k = V.pol->lookup(nodes, &v);
      if (k != SK_DEFAULT && can(k, v)) {
        kind = k;
        var = v;
      }
    }
    auto swap_cur = [&]() {
      T* tmp = cur[l];
      cur[l] = alt[l];
      alt[l] = tmp;
    };
    if (kind == SK_MARCH) {
      for (int k = 0; k < sweeps / march_sweeps<T>(var); ++k) {
        err = launch_smooth_march<T>(V.A[l], cur[l], alt[l], V.b[l], rev, k == 0 ? eH : nullptr, pc, skip, s,
                                     var);
        if (err) return err;
        swap_cur();
      }
      return cudaSuccess;
    }
    if (kind == SK_PIPE) {
      for (int k = 0; k < sweeps / pipe_sweeps<T>(var); ++k) {
        err = launch_smooth_pipe<T>(V.A[l], cur[l], alt[l], V.b[l], rev, k == 0 ? eH : nullptr, pc, skip,
                                    V.err, s, var);
        if (err) return err;
        swap_cur();
      }
      return cudaSuccess;
    }
    if (kind == SK_COLOUR) {  // per-colour kernels, in place
      if (eH && (err = launch_prolong_add(V.A[l], cur[l], eH, pc, skip, s))) return err;
      return launch_smooth(V.A[l], cur[l], V.b[l], sweeps, rev, skip, s);
    }
    for (int k = 0; k < sweeps / fused_sweeps<T>(var); ++k) {
      err = launch_smooth_fused(V.A[l], cur[l], alt[l], V.b[l], rev, k == 0 ? eH : nullptr, pc, skip, s, var);
      if (err) return err;
      swap_cur();
    }
    if (sweeps == 0 && eH) return launch_prolong_add(V.A[l], cur[l], eH, pc, skip, s);
    return cudaSuccess;
  };
  for (int l = 0; l < t; ++l) {
    if ((e = smooth(l, nu1, 0, nullptr))) return e;
    if ((e = launch_resid_restrict(V.A[l], cur[l], V.b[l], V.b[l + 1], cur[l + 1], V.A[l + 1].pitch,
                                   skip, s)))
      return e;
  }
  {
    TailArgs<T> ta;
    memset(&ta, 0, sizeof ta);
    ta.nlev = L - t;
    ta.nu1 = nu1;
    ta.nu2 = nu2;
    ta.inv = V.inv;
    for (int l = t; l < L; ++l) {
      ta.lv[l - t].L = lvl_of(V.A[l]);
      ta.lv[l - t].x = cur[l];
      ta.lv[l - t].b = V.b[l];
      ta.lv[l - t].t = alt[l];
    }
    if ((e = launch_tail(ta, skip, s))) return e;
  }
  for (int l = t - 1; l >= 0; --l)
    if ((e = smooth(l, nu2, 1, cur[l + 1]))) return e;
  *result = cur[0];
  return cudaSuccess;
}

template int tail_nodes<double>();
template int tail_nodes<float>();
template cudaError_t emit_vcycle<double>(const VLevels<double>&, int, int, int, double, const int*,
                                         cudaStream_t, double**, bool);
template cudaError_t emit_vcycle<float>(const VLevels<float>&, int, int, int, double, const int*,
                                        cudaStream_t, float**, bool);

}  // namespace mg

using namespace mg;

template <typename T, typename OPK>
static int vcycle_abi(int nlev, const OPK* ops, T* const* x, T* const* b, T* const* t,
                      const double* inv, T* const* lf, int nu1, int nu2, int smoother, void* stream) {
  if (nlev < 1 || nlev > kMaxLevels || !ops || !x || !b || !t || !inv || nu1 < 0 || nu2 < 0 ||
      nu1 + nu2 == 0)
    return 1;
  if (smoother != MG_SMOOTH_GS4 && smoother != MG_SMOOTH_JACOBI && smoother != MG_SMOOTH_XLINE) return 1;
  if ((smoother == MG_SMOOTH_XLINE) != (lf != nullptr)) return 1;
  VLevels<T> V;
  V.L = nlev;
  V.inv = inv;
  for (int l = 0; l < nlev; ++l) {
    const OPK& o = ops[l];
    if (o.nx < 3 || o.ny < 3 || o.pitch < o.nx || !x[l] || !b[l] || !t[l]) return 1;
    if (l > 0 && (o.nx != (ops[l - 1].nx - 1) / 2 + 1 || o.ny != (ops[l - 1].ny - 1) / 2 + 1))
      return 1;
    V.A[l] = op_from(o);
    V.x[l] = x[l];
    V.b[l] = b[l];
    V.t[l] = t[l];
    if (lf && l < nlev - 1) {
      if (!lf[l] || !line_supported<T>(o.nx)) return 1;
      V.lf[l] = line_factors_at<T>(lf[l], o.nx, o.ny, o.periodic);
    }
  }
  if (coarse_unknowns(ops[nlev - 1].nx, ops[nlev - 1].ny, ops[nlev - 1].periodic) > kCoarseMax) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  T* res = nullptr;
  if (emit_vcycle<T>(V, smoother, nu1, nu2, 0.8, nullptr, s, &res) != cudaSuccess) return 4;
  if (res != x[0]) {
    const size_t bytes = (size_t)ops[0].pitch * rows_stored(ops[0].ny, ops[0].periodic) * sizeof(T);
    if (cudaMemcpyAsync(x[0], res, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return 4;
  }
  return 0;
}

extern "C" int mgk_vcycle_f64(int nlev, const mgk_op_f64* ops, double* const* x, double* const* b,
                              double* const* t, const double* inv, int nu1, int nu2, int smoother,
                              void* stream) {
  return vcycle_abi<double>(nlev, ops, x, b, t, inv, nullptr, nu1, nu2, smoother, stream);
}

extern "C" int mgk_vcycle_f32(int nlev, const mgk_op_f32* ops, float* const* x, float* const* b,
                              float* const* t, const double* inv, int nu1, int nu2, int smoother,
                              void* stream) {
  return vcycle_abi<float>(nlev, ops, x, b, t, inv, nullptr, nu1, nu2, smoother, stream);
}

extern "C" int mgk_vcycle_line_f64(int nlev, const mgk_op_f64* ops, double* const* x, double* const* b,
                                   double* const* t, const double* inv, double* const* factors, int nu1,
                                   int nu2, void* stream) {
  if (!factors) return 1;
  return vcycle_abi<double>(nlev, ops, x, b, t, inv, factors, nu1, nu2, MG_SMOOTH_XLINE, stream);
}

extern "C" int mgk_vcycle_line_f32(int nlev, const mgk_op_f32* ops, float* const* x, float* const* b,
                                   float* const* t, const double* inv, float* const* factors, int nu1,
                                   int nu2, void* stream) {
  if (!factors) return 1;
  return vcycle_abi<float>(nlev, ops, x, b, t, inv, factors, nu1, nu2, MG_SMOOTH_XLINE, stream);
}

// Single fused smoothing launch on caller memory (testing and profiling).
template <typename T, typename OPK>
static int fused_abi(const OPK* A, const T* xin, T* xout, const T* b, int rev, const T* eH,
                     int pitch_c, void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !xin || !xout || !b || xin == xout)
    return 1;
  if (eH && ((A->nx - 1) % 2 || (A->ny - 1) % 2 || pitch_c < (A->nx - 1) / 2 + 1)) return 1;
  return launch_smooth_fused<T>(op_from(*A), xin, xout, b, rev, eH, pitch_c, nullptr,
                                (cudaStream_t)stream) == cudaSuccess ? 0 : 4;
}

extern "C" int mgk_smooth_fused_f64(const mgk_op_f64* A, const double* xin, double* xout,
                                    const double* b, int reverse, const double* eH, int pitch_c,
                                    void* stream) {
  return fused_abi<double>(A, xin, xout, b, reverse, eH, pitch_c, stream);
}

extern "C" int mgk_smooth_fused_f32(const mgk_op_f32* A, const float* xin, float* xout,
                                    const float* b, int reverse, const float* eH, int pitch_c,
                                    void* stream) {
  return fused_abi<float>(A, xin, xout, b, reverse, eH, pitch_c, stream);
}

extern "C" int mgk_fused_sweeps(int f32) { return f32 ? fused_sweeps<float>() : fused_sweeps<double>(); }

template <typename T, typename OPK>
static int pipe_abi(const OPK* A, const T* xin, T* xout, const T* b, int rev, const T* eH,
                    int pitch_c, int* err, void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !xin || !xout || !b || xin == xout)
    return 1;
  if (eH && ((A->nx - 1) % 2 || (A->ny - 1) % 2 || pitch_c < (A->nx - 1) / 2 + 1)) return 1;
  const cudaError_t e = launch_smooth_pipe<T>(op_from(*A), xin, xout, b, rev, eH, pitch_c, nullptr,
                                              err, (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue) return 1;
  return e == cudaSuccess ? 0 : 4;
}

extern "C" int mgk_smooth_pipe_f64(const mgk_op_f64* A, const double* xin, double* xout,
                                   const double* b, int reverse, const double* eH, int pitch_c,
                                   int* err, void* stream) {
  return pipe_abi<double>(A, xin, xout, b, reverse, eH, pitch_c, err, stream);
}

extern "C" int mgk_smooth_pipe_f32(const mgk_op_f32* A, const float* xin, float* xout,
                                   const float* b, int reverse, const float* eH, int pitch_c,
                                   int* err, void* stream) {
  return pipe_abi<float>(A, xin, xout, b, reverse, eH, pitch_c, err, stream);
}

extern "C" int mgk_pipe_sweeps(int f32) { return f32 ? pipe_sweeps<float>() : pipe_sweeps<double>(); }

template <typename T, typename OPK>
static int march_abi(const OPK* A, const T* xin, T* xout, const T* b, int reverse, const T* eH, int pitch_c,
                     void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !xin || !xout || !b || xin == xout)
    return 1;
  if (A->periodic && (A->ny - 1) % 2) return 1;
  if (eH && ((A->nx - 1) % 2 || (A->ny - 1) % 2 || pitch_c < (A->nx - 1) / 2 + 1)) return 1;
  const cudaError_t e = launch_smooth_march<T>(op_from(*A), xin, xout, b, reverse, eH, pitch_c, nullptr,
                                               (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue) return 1;
  return e == cudaSuccess ? 0 : 4;
}

extern "C" int mgk_smooth_march_f32(const mgk_op_f32* A, const float* xin, float* xout, const float* b,
                                    int reverse, const float* eH, int pitch_c, void* stream) {
  return march_abi<float>(A, xin, xout, b, reverse, eH, pitch_c, stream);
}

extern "C" int mgk_smooth_march_f64(const mgk_op_f64* A, const double* xin, double* xout, const double* b,
                                    int reverse, const double* eH, int pitch_c, void* stream) {
  return march_abi<double>(A, xin, xout, b, reverse, eH, pitch_c, stream);
}

extern "C" int mgk_march_sweeps(void) { return march_sweeps<float>(); }
extern "C" int mgk_march_sweeps_f64(void) { return march_sweeps<double>(); }

template <typename T>
static int variant_count(int family) {
  switch (family) {
    case SK_FUSED: return fused_variants<T>();
    case SK_PIPE: return pipe_variants<T>();
    case SK_MARCH: return march_variants<T>();
    default: return 0;
  }
}

extern "C" int mgk_smooth_variant_info(int f32, int family, int variant, int* tile_x, int* tile_y,
                                       int* sweeps) {
  const int n = f32 ? variant_count<float>(family) : variant_count<double>(family);
  if (variant < 0 || variant >= n) return 1;
  SmoothVariant v{};
  if (family == SK_FUSED) v = f32 ? fused_variant<float>(variant) : fused_variant<double>(variant);
  if (family == SK_PIPE) v = f32 ? pipe_variant<float>(variant) : pipe_variant<double>(variant);
  if (family == SK_MARCH) v = f32 ? march_variant<float>(variant) : march_variant<double>(variant);
  if (tile_x) *tile_x = v.tx;
  if (tile_y) *tile_y = v.ty;
  if (sweeps) *sweeps = v.ns;
  return 0;
}

template <typename T, typename OPK>
static int variant_abi(const OPK* A, int family, int variant, const T* xin, T* xout, const T* b, int reverse,
                       const T* eH, int pitch_c, int* err, void* stream) {
  if (!A || A->nx < 3 || A->ny < 3 || A->pitch < A->nx || !xin || !xout || !b || xin == xout) return 1;
  if (variant < 0 || variant >= variant_count<T>(family)) return 1;
  if (A->periodic && (A->ny - 1) % 2) return 1;
  if (eH && ((A->nx - 1) % 2 || (A->ny - 1) % 2 || pitch_c < (A->nx - 1) / 2 + 1)) return 1;
  const Op<T> op = op_from(*A);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (family == SK_FUSED) e = launch_smooth_fused<T>(op, xin, xout, b, reverse, eH, pitch_c, nullptr, s, variant);
  else if (family == SK_PIPE) e = launch_smooth_pipe<T>(op, xin, xout, b, reverse, eH, pitch_c, nullptr, err, s, variant);
  else e = launch_smooth_march<T>(op, xin, xout, b, reverse, eH, pitch_c, nullptr, s, variant);
  if (e == cudaErrorInvalidValue) return 1;
  return e == cudaSuccess ? 0 : 4;
}

extern "C" int mgk_smooth_variant_f64(const mgk_op_f64* A, int family, int variant, const double* xin,
                                      double* xout, const double* b, int reverse, const double* eH,
                                      int pitch_c, int* err, void* stream) {
  return variant_abi<double>(A, family, variant, xin, xout, b, reverse, eH, pitch_c, err, stream);
}

extern "C" int mgk_smooth_variant_f32(const mgk_op_f32* A, int family, int variant, const float* xin,
                                      float* xout, const float* b, int reverse, const float* eH,
                                      int pitch_c, int* err, void* stream) {
  return variant_abi<float>(A, family, variant, xin, xout, b, reverse, eH, pitch_c, err, stream);
}
