// Fused coarse-grid V-cycle (see coarse_cycle.cu): host-visible parameter structs.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace irk {

constexpr int kMaxFusedLevels = 4;
constexpr int kMaxChebDegree = 8;
constexpr size_t kCoarseCycleMaxSmem = 200 * 1024;
// A level joins the fused cycle when it has at most this many nodes per block.  In 3D one CTA per
// block runs a 17^3 level slower than its level-by-level launches replayed from the graph (measured
// at degree 4: 18.74 -> 18.31 ms per step with 9^3 as the largest fused level).
constexpr int kFusedMaxNodes3D = 729;
constexpr int kFusedMaxNodes2D = 4913;

struct CoarseLevel {
  int N, n1, n;                         // cells per axis, nodes per axis, nodes
  unsigned magic;                       // coarse_cycle_magic(n1): q / n1 by a high multiply
  float me[5][5], ke[5][5];             // element matrices scaled by h and 1/h
  float dmr[kMaxDeg], dkr[kMaxDeg];     // 1D diagonals by node position mod k
  float c1[kMaxChebDegree][kMaxStages], c2[kMaxChebDegree][kMaxStages];  // Chebyshev recurrence per step, block
};

struct CoarseParams {
  int nlev, nb, m, nci;
  float cm[kMaxStages];
  float taus[kMaxStages];                // stiffness coefficient tau of each block
  CoarseLevel lv[kMaxFusedLevels];      // lv[0] = the finest fused level
  float pc[(2 * kMaxDeg + 1) * (kMaxDeg + 1)];
  const double* ainv;                   // [nb][nci][nci] dense coarse inverse (FP64, applied in FP64)
  const int* map;                       // interior index -> node of the coarsest level
  const void* b_in;                     // level-lc right-hand sides [nb][ld]
  void* x_out;                          // level-lc result [nb][ld]
  long long ld;
};

size_t coarse_cycle_smem(const CoarseParams& P, int elem_size);
unsigned coarse_cycle_magic(int n);   // ceil(2^32 / n) for n >= 2
template <typename T>
cudaError_t launch_coarse_cycle(const CoarseParams& P, int dim, int k, cudaStream_t st);

}  // namespace irk
