// Lane-team product (matvec_reg.cuh): pass 1 instantiated for complex128.
#include "matvec_reg.cuh"

namespace gsm {

template cudaError_t reg_pass<double, 1>(int, const MatvecArgs<double> &, cudaStream_t);

}  // namespace gsm
