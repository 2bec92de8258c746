// Shapes of the tile and row-marching smoothers that the autotuner chooses among
// (k_fused.cu, k_pipe.cu, k_march.cu).  Every variant performs the same colour phases and
// the same operations per node in the same order, so a variant changes the time of a
// smoothing pass, not its values.
#pragma once

namespace mg {

// tx x ty: tile of owned nodes (fused, pipelined), or tx owned columns of a marching strip
// (ty = 0); ns: Gauss-Seidel sweeps one launch performs.
struct SmoothVariant {
  int tx, ty, ns;
};

// Number of variants of a family for precision T, and variant v (v < 0: the family's
// default variant, also what v out of range gives).  Families: SK_FUSED, SK_PIPE, SK_MARCH.
template <typename T>
int fused_variants();
template <typename T>
SmoothVariant fused_variant(int v);
template <typename T>
int pipe_variants();
template <typename T>
SmoothVariant pipe_variant(int v);
template <typename T>
int march_variants();
template <typename T>
SmoothVariant march_variant(int v);

}  // namespace mg
