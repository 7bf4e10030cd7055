// FP64 operator launches (the stage operator of Eq. (irk:A), K y_n, and the FP64 multigrid mode).
#include "op_kernels.cuh"

namespace irk {

template <>
cudaError_t launch_op<double>(int dim, int k, int nstage, const double* u, const OpParams<double>& P, int epi,
                              const EpiParams<double>& E, cudaStream_t st) {
  switch (epi) {
    case EPI_STORE: return launch_op_e<double, EPI_STORE>(dim, k, nstage, u, P, E, st);
    case EPI_DUAL: return launch_op_e<double, EPI_DUAL>(dim, k, nstage, u, P, E, st);
    case EPI_RESID: return launch_op_e<double, EPI_RESID>(dim, k, nstage, u, P, E, st);
    case EPI_CHEB: return launch_op_e<double, EPI_CHEB>(dim, k, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t tune_op<double>(int dim, int k, int nstage, const double* u, const OpParams<double>& P, int epi,
                         const EpiParams<double>& E, cudaStream_t st) {
  switch (epi) {
    case EPI_STORE: return tune_op_e<double, EPI_STORE>(dim, k, nstage, u, P, E, st);
    case EPI_DUAL: return tune_op_e<double, EPI_DUAL>(dim, k, nstage, u, P, E, st);
    case EPI_RESID: return tune_op_e<double, EPI_RESID>(dim, k, nstage, u, P, E, st);
    case EPI_CHEB: return tune_op_e<double, EPI_CHEB>(dim, k, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace irk
