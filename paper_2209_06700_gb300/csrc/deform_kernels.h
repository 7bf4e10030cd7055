// Curved-mesh stage operator kernels (see deform.cu): host-visible parameters.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"

namespace irk {

struct DeformParams {
  int N = 0, n1 = 0;
  double B[kMaxDeg + 1][kMaxDeg + 1];  // basis i at Gauss point q, [q][i] (unit cell)
  double D[kMaxDeg + 1][kMaxDeg + 1];  // its derivative
  double cm[kMaxStages], ck[kMaxStages];
  float Bh[kMaxDeg + 1][kMaxDeg + 1], Bl[kMaxDeg + 1][kMaxDeg + 1];  // hi + lo splits (ff, FP32)
  float Dh[kMaxDeg + 1][kMaxDeg + 1], Dl[kMaxDeg + 1][kMaxDeg + 1];
  float cmh[kMaxStages], cml[kMaxStages], ckh[kMaxStages], ckl[kMaxStages];
};

// Device data of one curved mesh: mapping data [cell][1 + d(d+1)/2][(k+1)^d] (element type T)
// and the cell-wise result buffers eM, eK [cell][max_ns][(k+1)^d] (8-byte elements for T = double:
// FP64 or ff, 4-byte for T = float).  B, D: host tables [q][i].
template <typename T>
struct DeformDevice {
  int dim = 0, N = 0, k = 0, max_ns = 0;
  int ff = 0;                     // T = double: 1 float-float arithmetic (FP32 pipe), 0 native FP64
  long long ncell = 0;
  const T* geo = nullptr;
  T* eM = nullptr;
  T* eK = nullptr;
  const double* B = nullptr;
  const double* D = nullptr;
};

// out_s = cm[s] M u_s + ck[s] K u_s (EPI_STORE) or out_s = M u_s, out2_s = K u_s (EPI_DUAL) for
// s < ns, on all nodes (boundary rows written as zero); u's boundary entries are read as given
// (zero for Dirichlet vectors).  Stage stride ld for u, out and out2.
template <typename T>
cudaError_t launch_deformed(const DeformDevice<T>& G, int ns, const T* u, long long ld, int epi, const double* cm,
                            const double* ck, T* out, T* out2, cudaStream_t st);

}  // namespace irk
