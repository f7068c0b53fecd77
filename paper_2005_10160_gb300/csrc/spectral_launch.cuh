// Launch helpers for the column kernels: one template instance per
// (transform length, components per thread group).
#pragma once
#include "spectral.cuh"

namespace grav {

constexpr int kMaxSmemPerCta = 227 * 1024;

template <typename R, int LOGN, int NC>
cudaError_t forward_impl(const ColumnArgs& a, const void* X, const R* spec, void* Y, const void* tw, int* err,
                         cudaStream_t s) {
    using C = typename cplx<R>::type;
    const FwdSmem L = forward_smem<R>(LOGN, a.ny_pad, a.ncomp, a.jp, kMaxSmemPerCta);
    if (L.depth == 0) return cudaErrorInvalidConfiguration;
    auto k = forward_column_kernel<R, LOGN, NC>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    k<<<dim3(2 * a.kx_count), ColShape<LOGN>::J, L.total, s>>>(a, L, (const C*)X, spec, (C*)Y, (const C*)tw, err);
    return cudaGetLastError();
}

#define GRAV_NC_SWITCH(R, L)                                                     \
    switch (nc_for(a.ncomp)) {                                                   \
        case 1: return forward_impl<R, L, 1>(a, in, spec, out, tw, err, s);      \
        case 2: return forward_impl<R, L, 2>(a, in, spec, out, tw, err, s);      \
        case 3: return forward_impl<R, L, 3>(a, in, spec, out, tw, err, s);      \
        case 4: return forward_impl<R, L, 4>(a, in, spec, out, tw, err, s);      \
        case 5: return forward_impl<R, L, 5>(a, in, spec, out, tw, err, s);      \
        case 6: return forward_impl<R, L, 6>(a, in, spec, out, tw, err, s);      \
        default: return forward_impl<R, L, 7>(a, in, spec, out, tw, err, s);     \
    }

#define GRAV_FORWARD_LAUNCHER(R)                                                                        \
    template <>                                                                                         \
    cudaError_t launch_forward_columns<R>(int log_n, const ColumnArgs& a, const void* in, const R* spec, \
                                          void* out, const void* tw, int* err, cudaStream_t s) {        \
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

template <typename R, int LOGN, int CPG>
cudaError_t adjoint_impl(const ColumnArgs& a, const void* Xr, const R* spec, void* Z, const void* tw, cudaStream_t s) {
    using C = typename cplx<R>::type;
    auto k = adjoint_column_kernel<R, LOGN, CPG>;
    const size_t smem = column_smem_bytes<R>(LOGN);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<dim3(a.kx_count, 2), ColShape<LOGN>::NT, smem, s>>>(a, (const C*)Xr, spec, (C*)Z, (const C*)tw);
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
                        const void* tw, cudaStream_t s) {                                                \
        switch (log_n) {                                                                                 \
            case 1: GRAV_CPG_SWITCH(IMPL, R, 1, a, in, spec, out, tw, s)                                 \
            case 2: GRAV_CPG_SWITCH(IMPL, R, 2, a, in, spec, out, tw, s)                                 \
            case 3: GRAV_CPG_SWITCH(IMPL, R, 3, a, in, spec, out, tw, s)                                 \
            case 4: GRAV_CPG_SWITCH(IMPL, R, 4, a, in, spec, out, tw, s)                                 \
            case 5: GRAV_CPG_SWITCH(IMPL, R, 5, a, in, spec, out, tw, s)                                 \
            case 6: GRAV_CPG_SWITCH(IMPL, R, 6, a, in, spec, out, tw, s)                                 \
            case 7: GRAV_CPG_SWITCH(IMPL, R, 7, a, in, spec, out, tw, s)                                 \
            case 8: GRAV_CPG_SWITCH(IMPL, R, 8, a, in, spec, out, tw, s)                                 \
            case 9: GRAV_CPG_SWITCH(IMPL, R, 9, a, in, spec, out, tw, s)                                 \
            case 10: GRAV_CPG_SWITCH(IMPL, R, 10, a, in, spec, out, tw, s)                               \
            default: return cudaErrorInvalidValue;                                                       \
        }                                                                                                \
    }

}  // namespace grav
