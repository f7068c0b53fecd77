// Forward column stage (Eq. 21), float instances.
#include "spectral_launch.cuh"

namespace grav {
GRAV_FORWARD_LAUNCHER(float)
}  // namespace grav
