// Element kernels of the entropy-conserving (Ismail-Roe) split form (Sec. 3.5): all degrees, both
// precisions, Euler and Navier-Stokes.
#include "volume_dev.cuh"
#include "volume_kernel.cuh"

namespace hs3d {
HS3D_VOLUME_FORM_TU(HS3D_VOL_IR)
HS3D_VOLUME_DEV_FORM_TU(HS3D_VOL_IR)
}  // namespace hs3d
