// Element kernels of the Ducros split form (Sec. 3.5): all degrees, both
// precisions, Euler and Navier-Stokes.
#include "volume_dev.cuh"
#include "volume_kernel.cuh"

namespace hs3d {
HS3D_VOLUME_FORM_TU(HS3D_VOL_DUCROS)
HS3D_VOLUME_DEV_FORM_TU(HS3D_VOL_DUCROS)
}  // namespace hs3d
