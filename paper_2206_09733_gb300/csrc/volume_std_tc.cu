// Element kernels of the standard form (Sec. 3.5) with the derivative-matrix
// contraction on the tensor cores (precision HS3D_MIXED_TC): all degrees,
// Euler and Navier-Stokes.
#include "volume_dev.cuh"
#include "volume_kernel.cuh"

namespace hs3d {
HS3D_VOLUME_FORM_TU(kVolStdTC)
HS3D_VOLUME_DEV_FORM_TU(kVolStdTC)
}  // namespace hs3d
