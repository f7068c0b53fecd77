// Row transforms along x: the first and last stage of the 2D circulant
// product of Eq. 18 applied to each layer (the BTTB form of Eq. 20).
//
// row_r2c: real rows, zero-padded from l_in to P points, become half spectra
// (kx = 0 .. P/2).  Two real rows a, b travel as one complex sequence
// z = a + i b; after the FFT  A(k) = (Z(k) + conj Z(-k)) / 2 and
// B(k) = (Z(k) - conj Z(-k)) / (2i).  Results are written transposed,
// [kx][o][i], so that the column stage reads one contiguous run of rows per
// frequency column.
//
// row_c2r: the inverse.  Half spectra (optionally the sum of two partial
// inputs: the even-ky and odd-ky halves of the column stage) are extended
// by Hermitian symmetry, two rows are packed as A + i B, inverse FFT'd, and
// the first l_out points of each row are kept (the crop back to the
// stations).
#include "fft_block.cuh"
#include "grav_internal.h"

namespace grav {

namespace {

template <typename R, int LOGP, int NSEQ, int NT, bool VEC>
__global__ void __launch_bounds__(NT, 2) row_r2c_kernel(const R* __restrict__ in, size_t in_ostride, size_t in_istride,
                                                      int l_in, int I, int O,
                                                      typename cplx<R>::type* __restrict__ out, int i_pad,
                                                      const typename cplx<R>::type* __restrict__ tw, int tw_shift,
                                                      size_t in_bstride, size_t out_bstride) {
    using C = typename cplx<R>::type;
    constexpr int P = 1 << LOGP;
    constexpr int SSTR = seq_stride<C>(P);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x;
    const int o = blockIdx.y;
    const int i_base = blockIdx.x * (2 * NSEQ);
    in += blockIdx.z * in_bstride;
    out += blockIdx.z * out_bstride;
    const R* in_o = in + (size_t)o * in_ostride;

    if constexpr (VEC) {
        // Rows of at most P/2 values, an even number, 8-byte aligned: every
        // thread loads element pairs (x, x+1) of both rows with all its loads
        // issued before any is used, and stores the two complex values with
        // one 16-byte shared store.
        static_assert(sizeof(R) == 4, "vector path is for float rows");
        constexpr int KMAX = (NSEQ * (P / 2) / 2 + NT - 1) / NT;
        const int npair = l_in >> 1;
        float2 va[KMAX], vb[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int e = tid + k * NT;
            va[k] = vb[k] = make_float2(0.f, 0.f);
            if (e < NSEQ * npair) {
                const int s = e / npair, xp = e - s * npair;
                const int i0 = i_base + 2 * s, i1 = i0 + 1;
                if (i0 < I) va[k] = __ldg(reinterpret_cast<const float2*>(in_o + (size_t)i0 * in_istride) + xp);
                if (i1 < I) vb[k] = __ldg(reinterpret_cast<const float2*>(in_o + (size_t)i1 * in_istride) + xp);
            }
        }
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            const int e = tid + k * NT;
            if (e < NSEQ * npair) {
                const int s = e / npair, x = 2 * (e - s * npair);
                *reinterpret_cast<float4*>(buf + s * SSTR + sidx<C>(x)) = make_float4(va[k].x, vb[k].x, va[k].y, vb[k].y);
            }
        }
        const int pad = P - 2 * npair;
        for (int e = tid; e < NSEQ * pad; e += NT) {
            const int s = e / pad, x = 2 * npair + (e - s * pad);
            buf[s * SSTR + sidx<C>(x)] = cmk<C>(0, 0);
        }
    } else {
        for (int e = tid; e < NSEQ * P; e += NT) {
            const int s = e / P, x = e - s * P;
            const int i0 = i_base + 2 * s, i1 = i0 + 1;
            R a = 0, b = 0;
            if (x < l_in) {
                if (i0 < I) a = in_o[(size_t)i0 * in_istride + x];
                if (i1 < I) b = in_o[(size_t)i1 * in_istride + x];
            }
            buf[s * SSTR + sidx<C>(x)] = cmk<C>(a, b);
        }
    }
    __syncthreads();
    block_fft<C, LOGP, NSEQ, NT, false>(buf, SSTR, tw, tw_shift, tid);

    constexpr int KX = P / 2 + 1;
    for (int e = tid; e < NSEQ * KX; e += NT) {
        const int s = e % NSEQ, kx = e / NSEQ;
        const int i0 = i_base + 2 * s, i1 = i0 + 1;
        if (i0 >= I) continue;
        const C zk = buf[s * SSTR + sidx<C>(kx)];
        const C zm = cconj(buf[s * SSTR + sidx<C>((P - kx) & (P - 1))]);
        const R half = (R)0.5;
        const C A = cmk<C>(half * (zk.x + zm.x), half * (zk.y + zm.y));
        const C d = csub(zk, zm);
        const C B = cmk<C>(half * d.y, -half * d.x);
        C* dst = out + ((size_t)kx * O + o) * i_pad + i0;
        if (VEC && i1 < I) {
            *reinterpret_cast<float4*>(dst) = make_float4(A.x, A.y, B.x, B.y);
        } else {
            dst[0] = A;
            if (i1 < I) dst[1] = B;
        }
    }
}

template <typename R, int LOGP, int NSEQ, int NT>
__global__ void __launch_bounds__(NT, 2) row_c2r_kernel(const typename cplx<R>::type* __restrict__ in0,
                                                      const typename cplx<R>::type* __restrict__ in1, int I, int O,
                                                      int i_pad, R* __restrict__ out, size_t out_stride, int l_out,
                                                      const typename cplx<R>::type* __restrict__ tw, int tw_shift,
                                                      size_t in_bstride, size_t out_bstride) {
    using C = typename cplx<R>::type;
    constexpr int P = 1 << LOGP;
    constexpr int SSTR = seq_stride<C>(P);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x;
    const int o = blockIdx.y;
    const int i_base = blockIdx.x * (2 * NSEQ);
    in0 += blockIdx.z * in_bstride;
    if (in1) in1 += blockIdx.z * in_bstride;
    out += blockIdx.z * out_bstride;

    for (int e = tid; e < NSEQ * P; e += NT) {
        const int s = e % NSEQ, k = e / NSEQ;
        const int i0 = i_base + 2 * s, i1 = i0 + 1;
        const bool upper = k > P / 2;
        const int kk = upper ? P - k : k;
        const size_t base = ((size_t)kk * O + o) * i_pad;
        C A = cmk<C>(0, 0), B = cmk<C>(0, 0);
        if (i0 < I) {
            A = in0[base + i0];
            if (in1) A = cadd(A, in1[base + i0]);
        }
        if (i1 < I) {
            B = in0[base + i1];
            if (in1) B = cadd(B, in1[base + i1]);
        }
        if (kk == 0 || kk == P / 2) { A.y = 0; B.y = 0; }  // real DC and Nyquist
        if (upper) { A = cconj(A); B = cconj(B); }
        // z = A + i B
        buf[s * SSTR + sidx<C>(k)] = cmk<C>(A.x - B.y, A.y + B.x);
    }
    __syncthreads();
    block_fft<C, LOGP, NSEQ, NT, true>(buf, SSTR, tw, tw_shift, tid);

    for (int e = tid; e < NSEQ * l_out; e += NT) {
        const int s = e / l_out, x = e - s * l_out;
        const int i0 = i_base + 2 * s, i1 = i0 + 1;
        const C z = buf[s * SSTR + sidx<C>(x)];
        if (i0 < I) out[((size_t)o * I + i0) * out_stride + x] = z.x;
        if (i1 < I) out[((size_t)o * I + i1) * out_stride + x] = z.y;
    }
}

// Rows per CTA: about 64-70 KB of shared memory per CTA.
template <typename R> constexpr int nseq_for(int logp) {
    const int bytes = (int)sizeof(typename cplx<R>::type) << logp;
    const int n = 65536 / bytes;
    return n < 1 ? 1 : (n > 8 ? 8 : n);
}

template <typename R, int LOGP, bool VEC>
cudaError_t r2c_launch(const R* in, size_t in_ostride, size_t in_istride, int l_in, int I, int O, void* out, int i_pad,
                       const void* tw, int log_t, cudaStream_t s, Batch b) {
    using C = typename cplx<R>::type;
    constexpr int NSEQ = nseq_for<R>(LOGP);
    constexpr int NT = 512;
    const size_t smem = (size_t)NSEQ * seq_stride<C>(1 << LOGP) * sizeof(C);
    constexpr auto k = row_r2c_kernel<R, LOGP, NSEQ, NT, VEC>;
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    dim3 grid((I + 2 * NSEQ - 1) / (2 * NSEQ), O, b.count);
    k<<<grid, NT, smem, s>>>(in, in_ostride, in_istride, l_in, I, O, (C*)out, i_pad, (const C*)tw, log_t - LOGP, b.in,
                             b.out);
    return cudaGetLastError();
}

template <typename R, int LOGP>
cudaError_t r2c_impl(const R* in, size_t in_ostride, size_t in_istride, int l_in, int I, int O, void* out, int i_pad,
                     const void* tw, int log_t, cudaStream_t s, Batch b) {
    // float rows of at most P/2 values, whole 16-byte vectors, aligned
    if constexpr (sizeof(R) == 4) {
        const bool vec = l_in <= (1 << LOGP) / 2 && l_in % 2 == 0 && in_istride % 2 == 0 && in_ostride % 2 == 0 &&
                         b.in % 2 == 0 && (reinterpret_cast<uintptr_t>(in) & 7) == 0 && i_pad % 2 == 0;
        if (vec) return r2c_launch<R, LOGP, true>(in, in_ostride, in_istride, l_in, I, O, out, i_pad, tw, log_t, s, b);
    }
    return r2c_launch<R, LOGP, false>(in, in_ostride, in_istride, l_in, I, O, out, i_pad, tw, log_t, s, b);
}

template <typename R, int LOGP>
cudaError_t c2r_impl(const void* in0, const void* in1, int I, int O, int i_pad, R* out, size_t out_stride, int l_out,
                     const void* tw, int log_t, cudaStream_t s, Batch b) {
    using C = typename cplx<R>::type;
    constexpr int NSEQ = nseq_for<R>(LOGP);
    constexpr int NT = 512;
    const size_t smem = (size_t)NSEQ * seq_stride<C>(1 << LOGP) * sizeof(C);
    constexpr auto k = row_c2r_kernel<R, LOGP, NSEQ, NT>;
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    dim3 grid((I + 2 * NSEQ - 1) / (2 * NSEQ), O, b.count);
    k<<<grid, NT, smem, s>>>((const C*)in0, (const C*)in1, I, O, i_pad, out, out_stride, l_out, (const C*)tw,
                             log_t - LOGP, b.in, b.out);
    return cudaGetLastError();
}

}  // namespace

#define GRAV_LOGP_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12)

template <typename R>
cudaError_t launch_row_r2c(int log_p, const R* in, size_t in_ostride, size_t in_istride, int l_in, int I, int O,
                           void* out, int i_pad, const void* tw, int log_t, cudaStream_t s, Batch b) {
    switch (log_p) {
#define CASE(L) \
    case L: return r2c_impl<R, L>(in, in_ostride, in_istride, l_in, I, O, out, i_pad, tw, log_t, s, b);
        GRAV_LOGP_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename R>
cudaError_t launch_row_c2r(int log_p, const void* in0, const void* in1, int I, int O, int i_pad, R* out,
                           size_t out_stride, int l_out, const void* tw, int log_t, cudaStream_t s, Batch b) {
    switch (log_p) {
#define CASE(L) \
    case L: return c2r_impl<R, L>(in0, in1, I, O, i_pad, out, out_stride, l_out, tw, log_t, s, b);
        GRAV_LOGP_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_row_r2c<float>(int, const float*, size_t, size_t, int, int, int, void*, int, const void*,
                                           int, cudaStream_t, Batch);
template cudaError_t launch_row_r2c<double>(int, const double*, size_t, size_t, int, int, int, void*, int,
                                            const void*, int, cudaStream_t, Batch);
template cudaError_t launch_row_c2r<float>(int, const void*, const void*, int, int, int, float*, size_t, int,
                                           const void*, int, cudaStream_t, Batch);
template cudaError_t launch_row_c2r<double>(int, const void*, const void*, int, int, int, double*, size_t, int,
                                            const void*, int, cudaStream_t, Batch);

}  // namespace grav
