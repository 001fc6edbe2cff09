// Lane-team product (matvec_reg.cuh) instantiated for complex double-float
// (dfloat.cuh), the arithmetic of the outer residual.
#include "matvec_reg.cuh"

namespace gsm {

GSM_EXTERN_REG_PASSES(dfl)

template cudaError_t launch_matvec_reg<dfl>(const MatvecArgs<dfl> &, cudaStream_t, Profiler *, const int *);

}  // namespace gsm
