// Lane-team product (matvec_reg.cuh): pass 2 instantiated for complex double-float.
#include "matvec_reg.cuh"

namespace gsm {

template cudaError_t reg_pass<dfl, 2>(int, const MatvecArgs<dfl> &, cudaStream_t);

}  // namespace gsm
