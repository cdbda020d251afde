// Element kernels of Morinishi's split form (Sec. 3.5): all degrees, both
// precisions, Euler and Navier-Stokes.
#include "volume_dev.cuh"
#include "volume_kernel.cuh"

namespace hs3d {
HS3D_VOLUME_FORM_TU(HS3D_VOL_MORINISHI)
HS3D_VOLUME_DEV_FORM_TU(HS3D_VOL_MORINISHI)
}  // namespace hs3d
