// Kernel spectra at plan time: the column half of the 2D FFT of every
// embedded kernel (the stored vector a of Eq. 19, transformed as in Eq. 18),
// done in FP64 and reduced to the real numbers the column stage needs.
//
// Input: Ehat[kx][o][b], the row transforms (along x) of the circulant
// kernels of layer n = n0 + o % nzc and component slot o / nzc, rows b < py/2
// only (the embedded kernel is even or odd in y, so row py - b is row b times
// the component's sign and row py/2 is zero).  One CTA per (kx, r) and four
// columns o folds each column for ky parity r,
// a[m] = (x[m] + (-1)^r x[m + N]) W_Py^(m r), runs the N = py/2 point FFT,
// and stores Re S (real-spectrum components: gz, gxx, gyy, gzz, gxy) or
// Im S (gxz, gyz) of the bins ky = 2q + r, q < J, plus the Nyquist bin
// ky = py/2 for r = 0, scaled by 1/(px py) (the inverse-FFT normalisation).
// The discarded part is zero up to rounding because the embedded kernel is
// exactly even or odd in x and y.
#include "fft_block.cuh"
#include "grav_internal.h"

namespace grav {

namespace {

// Columns per CTA: four (about 74 KB of FP64 transform buffers).
constexpr int kSpecSeqs = 4;

template <typename RO, int LOGN, int NT, int NSEQ>
__global__ void __launch_bounds__(NT) spec_extract_kernel(const double2* __restrict__ ehat, int kx_count, int nzc,
                                                          int ncomp, int n0, int nz, int jp, unsigned imag_mask,
                                                          unsigned oddv_mask, double scale, RO* __restrict__ spec,
                                                          const double2* __restrict__ tw, int tw_shift_n,
                                                          int tw_shift_p) {
    constexpr int N = 1 << LOGN;
    constexpr int J = N / 2 > 0 ? N / 2 : 1;
    constexpr int SSTR = seq_stride<double2>(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int tid = threadIdx.x;
    const int kx = blockIdx.x, r = blockIdx.y, o0 = blockIdx.z * NSEQ;
    const int O = ncomp * nzc;

    // fold for ky parity r: a[m] = (x[m] + (-1)^r x[m + N]) W_Py^(m r), with
    // x[m + N] = x[Py - (N - m)] = sign * x[N - m] (m >= 1) and x[N] = 0
    for (int e = tid; e < NSEQ * N; e += NT) {
        const int sq = e / N, m = e - sq * N, o = o0 + sq;
        double2 v = cmk<double2>(0, 0);
        if (o < O) {
            const double2* col = ehat + ((size_t)kx * O + o) * N;
            const double sgn = ((oddv_mask >> (o / nzc)) & 1u) ? -1.0 : 1.0;
            const double2 x0 = col[m];
            const double2 x1 = m ? cscale(col[N - m], sgn) : cmk<double2>(0, 0);
            v = r ? cmul(csub(x0, x1), tw[m << tw_shift_p]) : cadd(x0, x1);
        }
        buf[sq * SSTR + sidx<double2>(m)] = v;
    }
    __syncthreads();
    block_fft<double2, LOGN, NSEQ, NT, false>(buf, SSTR, tw, tw_shift_n, tid);

    const int nvals = (r == 0) ? J + 1 : J;
#pragma unroll
    for (int sq = 0; sq < NSEQ; ++sq) {
        const int o = o0 + sq;
        if (o >= O) break;
        const int slot = o / nzc, n = n0 + (o - slot * nzc);
        const bool imag = (imag_mask >> slot) & 1u;
        RO* dst = spec + (size_t)((size_t)(r * kx_count + kx) * nz + n) * ncomp * jp + (size_t)slot * jp;
        for (int q = tid; q < jp; q += NT) {
            double val = 0.0;
            if (q < nvals) {
                const int k = (q == J) ? N / 2 : q;
                const double2 z = buf[sq * SSTR + sidx<double2>(k)];
                val = (imag ? z.y : z.x) * scale;
            }
            dst[q] = (RO)val;
        }
    }
}

template <typename RO, int LOGN>
cudaError_t extract_impl(const void* ehat, int kx_count, int nzc, int ncomp, int n0, int nz, int jp,
                         unsigned imag_mask, unsigned oddv_mask, double scale, RO* spec, const void* tw64, int log_t,
                         cudaStream_t s) {
    constexpr int NT = 256, NSEQ = kSpecSeqs;
    const size_t smem = (size_t)NSEQ * seq_stride<double2>(1 << LOGN) * sizeof(double2);
    constexpr auto k = spec_extract_kernel<RO, LOGN, NT, NSEQ>;
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    dim3 grid(kx_count, 2, (ncomp * nzc + NSEQ - 1) / NSEQ);
    k<<<grid, NT, smem, s>>>((const double2*)ehat, kx_count, nzc, ncomp, n0, nz, jp, imag_mask, oddv_mask, scale,
                             spec, (const double2*)tw64, log_t - LOGN, log_t - (LOGN + 1));
    return cudaGetLastError();
}

}  // namespace

template <typename RO>
cudaError_t launch_spec_extract(int log_n, const void* ehat, int kx_count, int nzc, int ncomp, int n0, int nz, int jp,
                                unsigned imag_mask, unsigned oddv_mask, double scale, RO* spec, const void* tw64,
                                int log_t, cudaStream_t s) {
    switch (log_n) {
#define CASE(L) \
    case L: \
        return extract_impl<RO, L>(ehat, kx_count, nzc, ncomp, n0, nz, jp, imag_mask, oddv_mask, scale, spec, tw64, \
                                   log_t, s);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_spec_extract<float>(int, const void*, int, int, int, int, int, int, unsigned, unsigned,
                                                double, float*, const void*, int, cudaStream_t);
template cudaError_t launch_spec_extract<double>(int, const void*, int, int, int, int, int, int, unsigned, unsigned,
                                                 double, double*, const void*, int, cudaStream_t);

}  // namespace grav
