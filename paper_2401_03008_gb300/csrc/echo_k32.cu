// FP32 instantiation of the substep kernels (the mixed-precision path: single
// precision reconstruction, fluxes, DER and constrained transport).
#include "echo_kernels.cuh"

namespace echo {

template struct Path<float>;

}  // namespace echo
