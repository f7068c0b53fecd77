// Self-test of the bounded pipeline wait used by the column kernels: one
// thread waits on an mbarrier that nothing ever arrives at, with a short
// limit, and must give up and report it.  This exercises the failure path
// (a copy that never lands) without faulting or hanging the GPU.
#include "async_copy.cuh"
#include "grav_internal.h"

namespace grav {
namespace {

__global__ void bounded_wait_selftest(uint64_t limit_ns, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    const uint64_t t0 = global_ns();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    const uint64_t dt = global_ns() - t0;
    status[0] = ok ? 0 : 1;
    status[1] = (int)(dt / 1000ull);  // microseconds waited
}

}  // namespace
}  // namespace grav

using namespace grav;

extern "C" int grav_selftest_bounded_wait(double limit_ms, double* waited_ms) {
    if (!(limit_ms > 0) || limit_ms > 10000.0) {
        set_error("grav_selftest_bounded_wait: limit must be in (0, 10000] ms");
        return GRAV_EINVAL;
    }
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(selftest status)");
    bounded_wait_selftest<<<1, 32>>>((uint64_t)(limit_ms * 1e6), d);
    int h[2] = {0, 0};
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait selftest");
    if (waited_ms) *waited_ms = h[1] / 1000.0;
    if (h[0]) {
        set_error("bounded wait gave up after %.3f ms (expected)", h[1] / 1000.0);
        return GRAV_ETIMEOUT;
    }
    return GRAV_OK;
}
