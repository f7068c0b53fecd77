// Forward column stage (Eq. 21), float instances.
#include "spectral_launch.cuh"

namespace grav {
GRAV_COLUMN_LAUNCHER(launch_forward_columns, forward_impl, float)
}  // namespace grav
