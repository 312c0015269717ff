// residual_hex6.cu -- the residual kernels instantiated for hexahedra, order 6.
#include "residual_impl.cuh"

namespace hfv {

template int run_residual<Cfg<3, 5, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
template int run_residual<Cfg<3, 5, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);

}  // namespace hfv
