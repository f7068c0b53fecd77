// Adjoint column stage (transpose of Eq. 21), double instances.
#include "spectral_launch.cuh"

namespace grav {
GRAV_COLUMN_LAUNCHER(launch_adjoint_columns, adjoint_impl, double)
}  // namespace grav
