// Forward column stage (Eq. 21), double instances.
#include "spectral_launch.cuh"

namespace grav {
GRAV_COLUMN_LAUNCHER(launch_forward_columns, forward_impl, double)
}  // namespace grav
