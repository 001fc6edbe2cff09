// Lane-team product (matvec_reg.cuh): pass 3 instantiated for complex128.
#include "matvec_reg.cuh"

namespace gsm {

template cudaError_t reg_pass<double, 3>(int, const MatvecArgs<double> &, cudaStream_t);

}  // namespace gsm
