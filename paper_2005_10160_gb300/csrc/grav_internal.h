// Internal plan structure and kernel launchers of the GB300 forward library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/grav.h"

namespace grav {

constexpr int kMaxComp = 9;        // component bits 0 .. 8 (gz ... gzz, gx, gy)
constexpr int kMaxPlanComp = 8;    // components one plan may hold
constexpr unsigned kCompBits = (1u << kMaxComp) - 1;
constexpr double kUpsilon = 6.672e-11;  // gravitational constant of Sec. 2.1

// Parity of each component's kernel under x -> -x and y -> -y (the
// symmetries of Sec. 2.2): gz, gxx, gxy, gxz, gyy, gyz, gzz, gx, gy.
// Bit c set = component c is odd in that direction.
constexpr unsigned kOddUMask = 0x8Cu;   // gxy, gxz, gx
constexpr unsigned kOddVMask = 0x124u;  // gxy, gyz, gy
__host__ __device__ constexpr bool odd_u(int c) { return (kOddUMask >> c) & 1u; }
__host__ __device__ constexpr bool odd_v(int c) { return (kOddVMask >> c) & 1u; }

// Geometry shared by the kernel-generation launches.
struct Geometry {
    int nx, ny, nz;
    double dx, dy, dz, h;
};

// Layout of the resident kernel spectra.  Column kernels run one CTA per
// (kx, r) with r the parity of ky; the spectrum of every component is real
// or purely imaginary and even or odd in ky (exact consequences of the
// kernel's reflection symmetry), so a CTA needs one real number per
// mirror pair (ky, Py - ky):
//   spec[((r * kx_count + kx) * nz + n) * ncomp + c) * jp + q]
// q < J = Py / 4 is the pair index (ky = 2q + r); for r = 0, q = J holds the
// Nyquist row ky = Py / 2.  jp = J + 1 rounded up to a multiple of 4.

struct ColumnArgs {
    int ny;            // valid input / output rows
    int ny_pad;        // row stride of the workspaces
    int nz;
    int ncomp;
    int kx_count;
    int jp;
    unsigned imag_mask;  // bit s: component slot s has an imaginary spectrum
    unsigned oddv_mask;  // bit s: component slot s is odd in y
    int tw_shift_n;      // log2(T / N) for the half-length column transform
    int tw_shift_p;      // log2(T / Py) for the parity fold twiddles
    int z_tiled;         // adjoint output layout: 0 = Z[r][kx][n][y] (row stride ny_pad),
                         // 1 = Z[r][n][y / 8][kx][8], row pair (y % 8) / 2 at 16-byte position
                         // ((y % 8) / 2 + kx / 2) % 4 of the run (ny_pad a multiple of 8;
                         // see launch_row_c2r_tiled)
    // Batched calls across plans of equal sizes and components: request b
    // reads the kernel spectra at spec_of[b] (spec_count > 0); with
    // spec_count == 0 every request reads the kernel's spec argument.
    int spec_count;
    const void* spec_of[16];
};
constexpr int kMaxSpecPlans = 16;

// Spectra of the request a CTA works on (batch index b).
template <typename R>
__device__ __forceinline__ const R* request_spec(const ColumnArgs& a, const R* spec, int b) {
    return a.spec_count ? reinterpret_cast<const R*>(a.spec_of[b]) : spec;
}

}  // namespace grav

struct grav_plan {
    int kind;  // 0: stations on a plane above the mesh; 1: a station at every cell centre (grav_plan_create3d)
    int nx, ny, nz;
    double dx, dy, dz, h;
    unsigned comps;
    int fp64;
    int ncomp;
    int comp_id[grav::kMaxComp];
    int log_px, log_py, px, py;
    int kx_count;  // px / 2 + 1
    int J, jp;
    int ny_pad;
    unsigned imag_mask, oddv_mask;
    int log_t;      // twiddle table length T = max(px, py)
    void* spec;     // resident spectra (float or double)
    void* tw;       // twiddle table in the plan's precision
    void* ws_a;     // workspace: forward row transforms / adjoint column outputs
    void* ws_b;     // workspace: forward column outputs / adjoint row transforms
    size_t spec_bytes, tw_bytes, ws_a_bytes, ws_b_bytes;
    int* err_flag;  // device int: a pipeline wait ran out
    int device;
    // equal-dimension plans (kind 1): circulant size along z and the z parity
    // of each component slot; spec holds spec3[c][kx][jy][jz] (see volume.cu)
    int pz, log_pz;
    unsigned oddw_mask;   // bit s: component slot s is odd in the layer offset
    unsigned imag3_mask;  // bit s: the three-level spectrum of slot s is imaginary
    // stage timing (grav_plan_set_timing)
    int timing;
    std::vector<cudaEvent_t> ev_pool;
    struct TimedCall {
        int kind;  // 0 forward, 1 adjoint
        cudaEvent_t ev[4];
    };
    std::vector<TimedCall> timed;
};

namespace grav {

// Largest dynamic shared memory a CTA may use on sm_103a.
constexpr int kMaxSmemOptin = 227 * 1024;

// Raise a kernel's dynamic shared-memory limit to kMaxSmemOptin once per
// device (a kernel instance needs it before its first launch with more than
// 48 KB); later launches, including ones being captured into a CUDA graph,
// make no attribute call.
template <auto Kernel>
inline cudaError_t ensure_smem_limit() {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmemOptin);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Per-request strides of a batched call (elements of the buffer's own type);
// unused when batch == 1.
struct Batch {
    int count = 1;
    size_t in = 0, out = 0;
};

// Thread-local error message and CUDA check helpers (capi.cu).
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// Plan helpers shared by the plane and equal-dimension plans (capi.cu).
int ilog2(int v);
// Smallest power of two >= max(4, 2n - 1).
int circulant_size(int n);
size_t round_up(size_t v, size_t m);
// GRAV_EINVAL (with the message set) unless the sizes, spacings, height and
// component mask are valid for a plan.
int check_geometry(int nx, int ny, int nz, double dx, double dy, double dz, double h, unsigned components);
int dev_alloc_raw(void** p, size_t bytes, const char* what);
// Twiddle table W_T[e] = exp(-2 pi i e / T), T = 2^log_t, in FP64 (fp64 = 1)
// or FP32, on the device.
int build_twiddles(int log_t, int fp64, void** dev, size_t* bytes);
// Frees every device buffer and event of the plan, and the plan.
void free_plan(grav_plan* p);

// ---- kernel generation (kernel_gen.cu) ----
// mode 0: embed into a circulant array E[(c * nzc + n) * py + b][a] of size
//         py x px per (component, layer); E must be zeroed beforehand.
// mode 2: the same, rows b < py / 2 only, E[(c * nzc + n) * (py / 2) + b][a]
//         (the embedded kernel is even or odd in y, so row py - b is row b
//         times the component's sign, and row py / 2 is zero).
// mode 1: dense offset grid K[c][n][2ny-1][2nx-1].
cudaError_t launch_kernel_gen(const Geometry& g, unsigned comps, int n0, int n1, int mode,
                              int px, int py, double* out, cudaStream_t s);

// ---- row transforms (fft_rows.cu) ----
// Real rows -> half spectra, written transposed:
//   in  row (o, i) at in + o * in_ostride + i * in_istride, l_in valid values
//   out[(kx * O + o) * i_pad + i], kx in [0, P/2]
// err: device int set to 1 when a bounded wait of a pipelined variant ran out
// (nullptr: only variants without waits are used).
template <typename R>
cudaError_t launch_row_r2c(int log_p, const R* in, size_t in_ostride, size_t in_istride,
                           int l_in, int I, int O, void* out, int i_pad, const void* tw,
                           int log_t, cudaStream_t s, Batch b = Batch(), int* err = nullptr);
// Half spectra (the sum of in0 and in1, layout as above) -> real rows:
//   out row (o, i) at out + (o * I + i) * out_stride, first l_out values.
template <typename R>
cudaError_t launch_row_c2r(int log_p, const void* in0, const void* in1, int I, int O, int i_pad,
                           R* out, size_t out_stride, int l_out, const void* tw, int log_t,
                           cudaStream_t s, Batch b = Batch());

// Forward column stage for 512-point FP32 columns (Py = 1024) with both ky
// parities of a column in one CTA and two transforms per warp
// (col_fwd512_f32.cu).  Same arguments and layouts as the column launchers
// below; cudaErrorNotSupported when the sizes do not fit it (ny_pad > 512,
// more than 7 components) or err is null, and the caller takes another kernel.
cudaError_t launch_forward_wf512(const ColumnArgs& a, const void* X, const float* spec, void* Y, const void* tw,
                                 int* err, cudaStream_t s, Batch b);
// The adjoint counterpart (col_adj512_f32.cu), writing the untiled column
// output; cudaErrorNotSupported when ny_pad > 512, more than 8 components,
// err is null or a.z_tiled is set.
cudaError_t launch_adjoint_wf512(const ColumnArgs& a, const void* Xr, const float* spec, void* Z, const void* tw,
                                 int* err, cudaStream_t s, Batch b);

// Adjoint inverse rows from the tiled column output (ColumnArgs::z_tiled):
// in_r[n][y / 8][kx][8] (swizzled as described there) for r = 0, 1 (in1 = in0 + one half), summed, kx
// in [0, 1024]; in1 = nullptr: the single input in0.  Out row (n, y) at
// out + (n * ny + y) * out_stride, first l_out <= 1024 values.  FP32,
// P = 2048.  err as for the column kernels.
cudaError_t launch_row_c2r_tiled(const void* in0, const void* in1, int ny, int nz, int kx_count, float* out,
                                 size_t out_stride, int l_out, const void* tw, int log_t, cudaStream_t s,
                                 Batch b, int* err);
// Whether the FP32 adjoint of a plan with these sizes runs the tiled column
// output and launch_row_c2r_tiled (log_n: column transform length, log_px:
// row transform length).
bool adjoint_tiled_ok(int log_n, int log_px, int nx, const ColumnArgs& a);
// Tensor map of the tiled adjoint column output Z (see ColumnArgs::z_tiled)
// for tensor stores of one layer's column: 8-byte elements, dims (8, kx,
// y / 8, 2 nz, batch), box (8, 1, 128, 1, 1).  z_bstride: complex elements
// between the requests of a batched call.
cudaError_t make_ztile_map(CUtensorMap* map, void* Z, int nz, int ny_pad, int kx_count, int batch,
                           size_t z_bstride);

// ---- column kernels (spectral.cuh, col_*.cu) ----
// err: device int set to 1 when a pipeline wait ran out (the kernel then
// leaves early and its output is invalid).
template <typename R>
cudaError_t launch_forward_columns(int log_n, const ColumnArgs& a, const void* X, const R* spec,
                                   void* Y, const void* tw, int* err, cudaStream_t s, Batch b);
template <typename R>
cudaError_t launch_adjoint_columns(int log_n, const ColumnArgs& a, const void* Xr, const R* spec,
                                   void* Z, const void* tw, int* err, cudaStream_t s, Batch b);
template <> cudaError_t launch_forward_columns<float>(int, const ColumnArgs&, const void*, const float*, void*,
                                                     const void*, int*, cudaStream_t, Batch);
template <> cudaError_t launch_forward_columns<double>(int, const ColumnArgs&, const void*, const double*, void*,
                                                      const void*, int*, cudaStream_t, Batch);
template <> cudaError_t launch_adjoint_columns<float>(int, const ColumnArgs&, const void*, const float*, void*,
                                                     const void*, int*, cudaStream_t, Batch);
template <> cudaError_t launch_adjoint_columns<double>(int, const ColumnArgs&, const void*, const double*, void*,
                                                      const void*, int*, cudaStream_t, Batch);
// Column FFT of embedded kernel row transforms and extraction of the stored
// real numbers.  Ehat[kx][o][b] for b < py / 2 (row stride py / 2), o = c *
// nzc + n; row py - b is row b times -1 for components odd in y (bit s of
// oddv_mask), row py / 2 is zero.
template <typename RO>
cudaError_t launch_spec_extract(int log_n, const void* ehat, int kx_count, int nzc, int ncomp,
                                int n0, int nz, int jp, unsigned imag_mask, unsigned oddv_mask, double scale,
                                RO* spec, const void* tw64, int log_t, cudaStream_t s);

}  // namespace grav
