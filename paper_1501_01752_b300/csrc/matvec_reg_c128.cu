// Lane-team product (matvec_reg.cuh) instantiated for complex128.
#include "matvec_reg.cuh"

namespace gsm {

GSM_EXTERN_REG_PASSES(double)

template cudaError_t launch_matvec_reg<double>(const MatvecArgs<double> &, cudaStream_t, Profiler *, const int *);
template cudaError_t launch_reg_pass<double>(int, int, const MatvecArgs<double> &, cudaStream_t);

}  // namespace gsm
