// residual_3d.cu -- the residual kernels instantiated for 3D meshes of tetrahedra and of mixed elements, orders 2-3.
#include "residual_impl.cuh"

namespace hfv {

template int run_residual<Cfg<3, 1, 1>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
template int run_residual<Cfg<3, 1, 1>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
template int run_residual<Cfg<3, 2, 1>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
template int run_residual<Cfg<3, 2, 1>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
template int run_residual<Cfg<3, 1, 2>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
template int run_residual<Cfg<3, 1, 2>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);
template int run_residual<Cfg<3, 2, 2>, float>(hfv_scheme*, const float*, float*, const uint8_t*, uint8_t*, cudaStream_t, const float*, const StageRK*);
template int run_residual<Cfg<3, 2, 2>, double>(hfv_scheme*, const double*, double*, const uint8_t*, uint8_t*, cudaStream_t, const double*, const StageRK*);

}  // namespace hfv
