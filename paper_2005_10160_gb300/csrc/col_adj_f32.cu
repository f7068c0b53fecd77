// Adjoint column stage (transpose of Eq. 21), float instances.
#include "spectral_launch.cuh"

namespace grav {
GRAV_COLUMN_LAUNCHER(launch_adjoint_columns, adjoint_impl, float)

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
EncodeTiled encode_tiled() {
    static EncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}
}  // namespace

cudaError_t make_ztile_map(CUtensorMap* map, void* Z, int nz, int ny_pad, int kx_count, int batch,
                           size_t z_bstride) {
    const EncodeTiled enc = encode_tiled();
    if (!enc || ny_pad % 8 || (reinterpret_cast<uintptr_t>(Z) & 15) || (z_bstride * 8) % 16) return cudaErrorInvalidValue;
    const cuuint64_t e = 8;  // bytes per element (one complex FP32 value)
    const cuuint64_t nyb = (cuuint64_t)ny_pad / 8;
    const cuuint64_t dims[5] = {8, (cuuint64_t)kx_count, nyb, 2 * (cuuint64_t)nz, (cuuint64_t)(batch > 0 ? batch : 1)};
    const cuuint64_t strides[4] = {8 * e, (cuuint64_t)kx_count * 8 * e, nyb * kx_count * 8 * e,
                                   (cuuint64_t)(batch > 1 ? z_bstride * e : 2 * nz * nyb * kx_count * 8 * e)};
    const cuuint32_t box[5] = {8, 1, 128, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 5, Z, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool adjoint_tiled_ok(int log_n, int log_px, int nx, const ColumnArgs& a) {
    return log_n == 10 && log_px == 11 && nx <= 1024 && a.ny_pad % 8 == 0 && a.kx_count == 1025 &&
           aw_smem(a.ny_pad, a.ncomp, a.jp, a.ncomp, kMaxSmemOptin).dz != 0;
}
}  // namespace grav
