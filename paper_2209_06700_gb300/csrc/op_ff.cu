// Float-float operator launches: the FP64-accurate stage operator of Eq. (irk:A)
// and K y_n evaluated on the FP32 pipe (about 48 significant bits; inputs and
// outputs are ff vectors).
#include "op_kernels.cuh"

namespace irk {

template <>
cudaError_t launch_op<ff>(int dim, int k, int nstage, const ff* u, const OpParams<ff>& P, int epi,
                          const EpiParams<ff>& E, cudaStream_t st) {
  switch (epi) {
    case EPI_STORE: return launch_op_e<ff, EPI_STORE>(dim, k, nstage, u, P, E, st);
    case EPI_DUAL: return launch_op_e<ff, EPI_DUAL>(dim, k, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}

template <>
cudaError_t tune_op<ff>(int dim, int k, int nstage, const ff* u, const OpParams<ff>& P, int epi,
                         const EpiParams<ff>& E, cudaStream_t st) {
  switch (epi) {
    case EPI_STORE: return tune_op_e<ff, EPI_STORE>(dim, k, nstage, u, P, E, st);
    case EPI_DUAL: return tune_op_e<ff, EPI_DUAL>(dim, k, nstage, u, P, E, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace irk
