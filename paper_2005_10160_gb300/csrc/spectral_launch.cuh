// Launch helpers for the column kernels: one template instance per
// (transform length, components per thread group).
#pragma once
#include "spectral.cuh"
#include "spectral_adj_wf.cuh"
#include "spectral_wf.cuh"
#include "spectral_ws.cuh"

namespace grav {

template <typename R, int LOGN, int NC>
cudaError_t forward_impl(const ColumnArgs& a, const void* X, const R* spec, void* Y, const void* tw, int* err,
                         cudaStream_t s, Batch b) {
    using C = typename cplx<R>::type;
    if constexpr (sizeof(R) == 4 && LOGN == 10 && NC <= WfShape::FWARPS) {
        // 1024-point FP32 columns: one warp per layer transform
        const WfSmem W = wf_smem(a.ny_pad, a.ncomp, a.jp, NC, kMaxSmemOptin);
        if (W.df != 0) {
            constexpr auto kw = forward_column_wf_kernel<NC>;
            cudaError_t e = ensure_smem_limit<kw>();
            if (e != cudaSuccess) return e;
            kw<<<dim3(2 * a.kx_count, b.count), WfShape::NT, W.total, s>>>(
                a, W, (const float2*)X, (const float*)spec, (float2*)Y, (const float2*)tw, err, b.in, b.out);
            return cudaGetLastError();
        }
    }
    if constexpr (sizeof(R) == 4 && LOGN == 9) {
        // 512-point FP32 columns: both parities of a column per CTA, two
        // transforms per warp (col_fwd512_f32.cu)
        const cudaError_t e = launch_forward_wf512(a, X, (const float*)spec, Y, tw, err, s, b);
        if (e != cudaErrorNotSupported) return e;
    }
    if constexpr (sizeof(R) == 4 && (LOGN == 9 || LOGN == 10)) {
        // large FP32 transforms: the warp-specialised kernel
        const WsSmem W = ws_smem<LOGN>(a.ny_pad, a.ncomp, a.jp, NC, kMaxSmemOptin);
        if (W.ds != 0) {
            constexpr auto kw = forward_column_ws_kernel<LOGN, NC>;
            cudaError_t e = ensure_smem_limit<kw>();
            if (e != cudaSuccess) return e;
            kw<<<dim3(2 * a.kx_count, b.count), WsShape<LOGN>::NT, W.total, s>>>(
                a, W, (const float2*)X, (const float*)spec, (float2*)Y, (const float2*)tw, err, b.in, b.out);
            return cudaGetLastError();
        }
    }
    const FwdSmem L = forward_smem<R>(LOGN, a.ny_pad, a.ncomp, a.jp, kMaxSmemOptin);
    if (L.depth == 0) return cudaErrorInvalidConfiguration;
    constexpr auto k = forward_column_kernel<R, LOGN, NC>;
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    k<<<dim3(2 * a.kx_count, b.count), ColShape<LOGN>::J, L.total, s>>>(a, L, (const C*)X, spec, (C*)Y, (const C*)tw,
                                                                         err, b.in, b.out);
    return cudaGetLastError();
}

#define GRAV_NC_SWITCH(R, L)                                                     \
    switch (nc_for(a.ncomp)) {                                                   \
        case 1: return forward_impl<R, L, 1>(a, in, spec, out, tw, err, s, b);   \
        case 2: return forward_impl<R, L, 2>(a, in, spec, out, tw, err, s, b);   \
        case 3: return forward_impl<R, L, 3>(a, in, spec, out, tw, err, s, b);   \
        case 4: return forward_impl<R, L, 4>(a, in, spec, out, tw, err, s, b);   \
        case 5: return forward_impl<R, L, 5>(a, in, spec, out, tw, err, s, b);   \
        case 6: return forward_impl<R, L, 6>(a, in, spec, out, tw, err, s, b);   \
        case 7: return forward_impl<R, L, 7>(a, in, spec, out, tw, err, s, b);   \
        default: return forward_impl<R, L, 8>(a, in, spec, out, tw, err, s, b);  \
    }

#define GRAV_FORWARD_LAUNCHER(R)                                                                        \
    template <>                                                                                         \
    cudaError_t launch_forward_columns<R>(int log_n, const ColumnArgs& a, const void* in, const R* spec, \
                                          void* out, const void* tw, int* err, cudaStream_t s, Batch b) { \
        switch (log_n) {                                                                                \
            case 1: GRAV_NC_SWITCH(R, 1)                                                                \
            case 2: GRAV_NC_SWITCH(R, 2)                                                                \
            case 3: GRAV_NC_SWITCH(R, 3)                                                                \
            case 4: GRAV_NC_SWITCH(R, 4)                                                                \
            case 5: GRAV_NC_SWITCH(R, 5)                                                                \
            case 6: GRAV_NC_SWITCH(R, 6)                                                                \
            case 7: GRAV_NC_SWITCH(R, 7)                                                                \
            case 8: GRAV_NC_SWITCH(R, 8)                                                                \
            case 9: GRAV_NC_SWITCH(R, 9)                                                                \
            case 10: GRAV_NC_SWITCH(R, 10)                                                              \
            default: return cudaErrorInvalidValue;                                                      \
        }                                                                                               \
    }

template <int NC, unsigned IM = kRuntimeMask, unsigned OV = kRuntimeMask>
cudaError_t adjoint_wf_launch(const ColumnArgs& a, const AwSmem& L, const void* Xr, const float* spec, void* Z,
                              const void* tw, int* err, cudaStream_t s, Batch b) {
    constexpr auto k = adjoint_column_wf_kernel<NC, IM, OV>;
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    CUtensorMap zmap{};
    if (a.z_tiled && (e = make_ztile_map(&zmap, Z, a.nz, a.ny_pad, a.kx_count, b.count, b.out)) != cudaSuccess)
        return e;
    k<<<dim3(2 * a.kx_count, b.count), AwShape::NT, L.total, s>>>(a, L, (const float2*)Xr, spec, (float2*)Z,
                                                                   (const float2*)tw, err, b.in, b.out, zmap);
    return cudaGetLastError();
}

template <typename R, int LOGN, int CPG>
cudaError_t adjoint_impl(const ColumnArgs& a, const void* Xr, const R* spec, void* Z, const void* tw, int* err,
                         cudaStream_t s, Batch b) {
    using C = typename cplx<R>::type;
    if constexpr (sizeof(R) == 4 && LOGN == 10) {
        // 1024-point FP32 columns: one warp per layer transform
        const AwSmem L = aw_smem(a.ny_pad, a.ncomp, a.jp, a.ncomp, kMaxSmemOptin);
        if (L.dz != 0 && err) {
            switch (a.ncomp) {
                case 1: return adjoint_wf_launch<1>(a, L, Xr, spec, Z, tw, err, s, b);
                case 2: return adjoint_wf_launch<2>(a, L, Xr, spec, Z, tw, err, s, b);
                case 3: return adjoint_wf_launch<3>(a, L, Xr, spec, Z, tw, err, s, b);
                case 4: return adjoint_wf_launch<4>(a, L, Xr, spec, Z, tw, err, s, b);
                case 5: return adjoint_wf_launch<5>(a, L, Xr, spec, Z, tw, err, s, b);
                case 6:
                    // all six components (gz, gxx, gxy, gxz, gyy, gyz): gxz and gyz have
                    // imaginary spectra, gxy and gyz are odd in y; masks known at compile time
                    if (a.imag_mask == 0x28u && a.oddv_mask == 0x24u)
                        return adjoint_wf_launch<6, 0x28u, 0x24u>(a, L, Xr, spec, Z, tw, err, s, b);
                    return adjoint_wf_launch<6>(a, L, Xr, spec, Z, tw, err, s, b);
                case 7:
                    // all seven components (gzz adds an even, real spectrum): same masks
                    if (a.imag_mask == 0x28u && a.oddv_mask == 0x24u)
                        return adjoint_wf_launch<7, 0x28u, 0x24u>(a, L, Xr, spec, Z, tw, err, s, b);
                    return adjoint_wf_launch<7>(a, L, Xr, spec, Z, tw, err, s, b);
                case 8: return adjoint_wf_launch<8>(a, L, Xr, spec, Z, tw, err, s, b);
                default: break;
            }
        }
    }
    if constexpr (sizeof(R) == 4 && LOGN == 9) {
        // 512-point FP32 columns: both parities of a column per CTA, two
        // transforms per warp (col_adj512_f32.cu)
        const cudaError_t e = launch_adjoint_wf512(a, Xr, (const float*)spec, Z, tw, err, s, b);
        if (e != cudaErrorNotSupported) return e;
    }
    constexpr auto k = adjoint_column_kernel<R, LOGN, CPG>;
    const size_t smem = column_smem_bytes<R>(LOGN);
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    k<<<dim3(a.kx_count, 2, b.count), ColShape<LOGN>::NT, smem, s>>>(a, (const C*)Xr, spec, (C*)Z, (const C*)tw, b.in,
                                                                       b.out);
    return cudaGetLastError();
}

#define GRAV_CPG_SWITCH(FN, R, L, ...)                       \
    switch (cpg_for(a.ncomp)) {                              \
        case 1: return FN<R, L, 1>(__VA_ARGS__);             \
        case 2: return FN<R, L, 2>(__VA_ARGS__);             \
        case 3: return FN<R, L, 3>(__VA_ARGS__);             \
        default: return FN<R, L, 4>(__VA_ARGS__);            \
    }

#define GRAV_COLUMN_LAUNCHER(NAME, IMPL, R)                                                              \
    template <>                                                                                          \
    cudaError_t NAME<R>(int log_n, const ColumnArgs& a, const void* in, const R* spec, void* out,       \
                        const void* tw, int* err, cudaStream_t s, Batch b) {                             \
        switch (log_n) {                                                                                 \
            case 1: GRAV_CPG_SWITCH(IMPL, R, 1, a, in, spec, out, tw, err, s, b)                                 \
            case 2: GRAV_CPG_SWITCH(IMPL, R, 2, a, in, spec, out, tw, err, s, b)                                 \
            case 3: GRAV_CPG_SWITCH(IMPL, R, 3, a, in, spec, out, tw, err, s, b)                                 \
            case 4: GRAV_CPG_SWITCH(IMPL, R, 4, a, in, spec, out, tw, err, s, b)                                 \
            case 5: GRAV_CPG_SWITCH(IMPL, R, 5, a, in, spec, out, tw, err, s, b)                                 \
            case 6: GRAV_CPG_SWITCH(IMPL, R, 6, a, in, spec, out, tw, err, s, b)                                 \
            case 7: GRAV_CPG_SWITCH(IMPL, R, 7, a, in, spec, out, tw, err, s, b)                                 \
            case 8: GRAV_CPG_SWITCH(IMPL, R, 8, a, in, spec, out, tw, err, s, b)                                 \
            case 9: GRAV_CPG_SWITCH(IMPL, R, 9, a, in, spec, out, tw, err, s, b)                                 \
            case 10: GRAV_CPG_SWITCH(IMPL, R, 10, a, in, spec, out, tw, err, s, b)                               \
            default: return cudaErrorInvalidValue;                                                       \
        }                                                                                                \
    }

}  // namespace grav
