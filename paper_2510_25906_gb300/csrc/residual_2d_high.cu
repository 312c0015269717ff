// residual_2d_high.cu -- the residual kernels instantiated for 2D meshes, orders 6-7.
#include "residual_impl.cuh"

namespace hfv {

template int run_residual<Cfg<2, 5, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
template int run_residual<Cfg<2, 5, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
template int run_residual<Cfg<2, 6, 0>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
template int run_residual<Cfg<2, 6, 0>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);

}  // namespace hfv
