// Adjoint column stage (transpose of Eq. 21), float instances.
#include "spectral_launch.cuh"

namespace grav {
GRAV_COLUMN_LAUNCHER(launch_adjoint_columns, adjoint_impl, float)

bool adjoint_tiled_ok(int log_n, int log_px, int nx, const ColumnArgs& a) {
    return log_n == 10 && log_px == 11 && nx <= 1024 && a.ny_pad % 8 == 0 && a.kx_count == 1025 &&
           aw_smem(a.ny_pad, a.ncomp, a.jp, a.ncomp, kMaxSmemOptin).dz != 0;
}
}  // namespace grav
