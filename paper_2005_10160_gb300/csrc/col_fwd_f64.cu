// Forward column stage (Eq. 21), double instances.
#include "spectral_launch.cuh"

namespace grav {
GRAV_FORWARD_LAUNCHER(double)
}  // namespace grav
