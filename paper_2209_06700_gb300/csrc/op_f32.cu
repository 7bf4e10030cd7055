// FP32 operator launches (multigrid level operators, Chebyshev smoother, residual, and the dual
// products M x, K x of the coupled 2x2 level operator); 3D levels of at most kCellKernelMaxN
// cells per axis go to the cell kernel of op_cell.cuh.
#include "op_cell.cuh"
#include "op_kernels.cuh"

namespace irk {

void op_tile_shape(int dim, int k, int* cx, int* cy) { op_tile_shape_impl(dim, k, cx, cy); }

template <>
cudaError_t launch_op<float>(int dim, int k, int nstage, const float* u, const OpParams<float>& P, int epi,
                             const EpiParams<float>& E, cudaStream_t st) {
  if (dim == 3 && P.N <= kCellKernelMaxN && epi != EPI_DUAL) {  // few cells per axis: cell kernel
    switch (epi) {
      case EPI_STORE: return launch_cell_op<float, EPI_STORE>(k, nstage, u, P, E, st);
      case EPI_RESID: return launch_cell_op<float, EPI_RESID>(k, nstage, u, P, E, st);
      case EPI_CHEB: return launch_cell_op<float, EPI_CHEB>(k, nstage, u, P, E, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (epi) {
    case EPI_STORE: return launch_op_e<float, EPI_STORE>(dim, k, nstage, u, P, E, st);
    case EPI_DUAL: return launch_op_e<float, EPI_DUAL>(dim, k, nstage, u, P, E, st);
    case EPI_RESID: return launch_op_e<float, EPI_RESID>(dim, k, nstage, u, P, E, st);
    case EPI_CHEB: return launch_op_e<float, EPI_CHEB>(dim, k, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t tune_op<float>(int dim, int k, int nstage, const float* u, const OpParams<float>& P, int epi,
                         const EpiParams<float>& E, cudaStream_t st) {
  if (dim == 3 && P.N <= kCellKernelMaxN && epi != EPI_DUAL) return cudaSuccess;  // cell kernel: no shapes
  switch (epi) {
    case EPI_STORE: return tune_op_e<float, EPI_STORE>(dim, k, nstage, u, P, E, st);
    case EPI_DUAL: return tune_op_e<float, EPI_DUAL>(dim, k, nstage, u, P, E, st);
    case EPI_RESID: return tune_op_e<float, EPI_RESID>(dim, k, nstage, u, P, E, st);
    case EPI_CHEB: return tune_op_e<float, EPI_CHEB>(dim, k, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace irk
