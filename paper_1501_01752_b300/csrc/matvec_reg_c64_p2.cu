// Lane-team product (matvec_reg.cuh): pass 2 instantiated for complex64.
#include "matvec_reg.cuh"

namespace gsm {

template cudaError_t reg_pass<float, 2>(int, const MatvecArgs<float> &, cudaStream_t);

}  // namespace gsm
