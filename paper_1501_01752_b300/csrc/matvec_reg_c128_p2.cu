// Lane-team product (matvec_reg.cuh): pass 2 instantiated for complex128.
#include "matvec_reg.cuh"

namespace gsm {

template cudaError_t reg_pass<double, 2>(int, const MatvecArgs<double> &, cudaStream_t);

}  // namespace gsm
