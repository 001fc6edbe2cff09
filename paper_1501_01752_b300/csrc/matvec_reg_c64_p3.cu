// Lane-team product (matvec_reg.cuh): pass 3 instantiated for complex64.
#include "matvec_reg.cuh"

namespace gsm {

template cudaError_t reg_pass<float, 3>(int, const MatvecArgs<float> &, cudaStream_t);

}  // namespace gsm
