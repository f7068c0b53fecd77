// Column stage of the 2D circulant product (Eqs. 18-21) and the kernel
// spectra it consumes.
//
// One CTA owns one frequency column kx of the row transforms and one parity
// r of ky.  Splitting ky by parity is the first decimation-in-frequency step
// of the Py-point column FFT: the rows m < ny <= Py/2 are folded to
// a[m] = x[m] W_Py^(m r) and an N = Py/2 point FFT gives the bins ky = 2k + r.
// Each pair of mirror bins (ky, Py - ky) has the same parity, so one CTA
// sees both members of every pair and needs one stored real number per
// pair and component (see SpecLayout): the kernel spectra are real or purely
// imaginary and even or odd in ky because the embedded kernel is exactly
// even or odd under reflection (Sec. 2.2).
//
// Forward (Eq. 21): for every layer n the CTA transforms the density column,
// multiplies by S_{c,n} and accumulates over n in registers (FP32 with a
// Kahan-compensated layer sum, or FP64); at the end it inverse-transforms
// each component's accumulator and writes the rows y < ny.  The threads are
// split into two groups that own different components, so each thread keeps
// the accumulators of at most CPG components for H mirror pairs.
//
// Adjoint (transpose of Eq. 21): the residual of every component is
// transformed once; per layer the CTA forms sum_c conj(S_{c,n}) R_c,
// inverse-transforms it and writes that layer's rows.
#pragma once
#include "fft_block.cuh"
#include "grav_internal.h"

namespace grav {

template <int LOGN> struct ColShape {
    static constexpr int N = 1 << LOGN;
    static constexpr int J = N / 2 > 0 ? N / 2 : 1;  // mirror pairs per CTA
    static constexpr int H = J >= 2 ? 2 : 1;         // pairs per thread
    static constexpr int TG = J / H;                 // threads per component group
    static constexpr int NT = 2 * TG;
    static constexpr int XPT = (N + NT - 1) / NT;    // input rows per thread
};

// Bin positions (k indices, ky = 2k + r) of mirror pair q.
template <int N> __device__ __forceinline__ void pair_pos(int q, int r, int& k1, int& k2) {
    if (r == 0) {
        k1 = q;
        k2 = (q == 0) ? N / 2 : N - q;
    } else {
        k1 = q;
        k2 = N - 1 - q;
    }
}

template <typename C> __device__ __forceinline__ C spec_term(decltype(C::x) s, C v, bool imag) {
    // S v with S = s (real spectrum) or i s (imaginary spectrum)
    return imag ? cmk<C>(-s * v.y, s * v.x) : cmk<C>(s * v.x, s * v.y);
}
template <typename C> __device__ __forceinline__ C spec_term_conj(decltype(C::x) s, C v, bool imag) {
    // conj(S) v
    return imag ? cmk<C>(s * v.y, -s * v.x) : cmk<C>(s * v.x, s * v.y);
}

template <typename R> __device__ __forceinline__ void kahan_add(R& sum, R& comp, R x) {
    const R y = x - comp;
    const R t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

template <typename R, int LOGN, int CPG, bool KAHAN>
__global__ void __launch_bounds__(ColShape<LOGN>::NT, 1)
    forward_column_kernel(ColumnArgs a, const typename cplx<R>::type* __restrict__ X, const R* __restrict__ spec,
                          typename cplx<R>::type* __restrict__ Y, const typename cplx<R>::type* __restrict__ tw) {
    using C = typename cplx<R>::type;
    using S = ColShape<LOGN>;
    constexpr int N = S::N, J = S::J, H = S::H, TG = S::TG, NT = S::NT, XPT = S::XPT;
    constexpr int SSTR = spad_len<C>(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);

    const int tid = threadIdx.x;
    const int g = tid / TG, lt = tid - g * TG;
    const int kx = blockIdx.x, r = blockIdx.y;
    const C* Xc = X + (size_t)kx * a.nz * a.ny_pad;
    const R* sp = spec + (size_t)(r * a.kx_count + kx) * a.nz * a.ncomp * a.jp;
    const bool has_nyq = (r == 0 && lt == 0);

    R acc[CPG][H][2][2];
    R cmp[CPG][H][2][2];
#pragma unroll
    for (int c = 0; c < CPG; ++c)
#pragma unroll
        for (int s = 0; s < H; ++s)
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                acc[c][s][m][0] = acc[c][s][m][1] = 0;
                cmp[c][s][m][0] = cmp[c][s][m][1] = 0;
            }

    C xv[XPT];
    R sv[CPG][H], se[CPG];
    auto load_x = [&](int n) {
#pragma unroll
        for (int j = 0; j < XPT; ++j) {
            const int m = tid + j * NT;
            xv[j] = (m < a.ny) ? Xc[(size_t)n * a.ny_pad + m] : cmk<C>(0, 0);
        }
    };
    auto load_s = [&](int n) {
#pragma unroll
        for (int c = 0; c < CPG; ++c) {
            const int slot = g * CPG + c;
            const R* row = sp + ((size_t)n * a.ncomp + slot) * a.jp;
#pragma unroll
            for (int s = 0; s < H; ++s) sv[c][s] = (slot < a.ncomp) ? row[lt * H + s] : (R)0;
            se[c] = (slot < a.ncomp && has_nyq) ? row[J] : (R)0;
        }
    };
    load_x(0);
    load_s(0);

    for (int n = 0; n < a.nz; ++n) {
        // fold for ky parity r: a[m] = x[m] W_Py^(m r)
#pragma unroll
        for (int j = 0; j < XPT; ++j) {
            const int m = tid + j * NT;
            if (m < N) buf[sidx<C>(m)] = r ? cmul(xv[j], tw[m << a.tw_shift_p]) : xv[j];
        }
        if (n + 1 < a.nz) load_x(n + 1);  // in flight during this layer's FFT
        __syncthreads();
        block_fft<C, LOGN, 1, NT, false>(buf, SSTR, tw, a.tw_shift_n, tid);
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int q = lt * H + s;
            int k1, k2;
            pair_pos<N>(q, r, k1, k2);
            const C v1 = buf[sidx<C>(k1)], v2 = buf[sidx<C>(k2)];
#pragma unroll
            for (int c = 0; c < CPG; ++c) {
                const int slot = g * CPG + c;
                const bool imag = (a.imag_mask >> slot) & 1u;
                const R s1 = sv[c][s];
                const R s2 = (r == 0 && q == 0) ? se[c] : (((a.oddv_mask >> slot) & 1u) ? -s1 : s1);
                const C t1 = spec_term<C>(s1, v1, imag), t2 = spec_term<C>(s2, v2, imag);
                if (KAHAN) {
                    kahan_add(acc[c][s][0][0], cmp[c][s][0][0], t1.x);
                    kahan_add(acc[c][s][0][1], cmp[c][s][0][1], t1.y);
                    kahan_add(acc[c][s][1][0], cmp[c][s][1][0], t2.x);
                    kahan_add(acc[c][s][1][1], cmp[c][s][1][1], t2.y);
                } else {
                    acc[c][s][0][0] += t1.x; acc[c][s][0][1] += t1.y;
                    acc[c][s][1][0] += t2.x; acc[c][s][1][1] += t2.y;
                }
            }
        }
        if (n + 1 < a.nz) load_s(n + 1);  // in flight during the next layer's FFT
        __syncthreads();
    }

    // Inverse column transform of every component, crop to y < ny.
    C* gb = buf + g * SSTR;
#pragma unroll
    for (int c = 0; c < CPG; ++c) {
        const int slot = g * CPG + c;
#pragma unroll
        for (int s = 0; s < H; ++s) {
            int k1, k2;
            pair_pos<N>(lt * H + s, r, k1, k2);
            R e0 = acc[c][s][0][0], e1 = acc[c][s][0][1], e2 = acc[c][s][1][0], e3 = acc[c][s][1][1];
            if (KAHAN) { e0 -= cmp[c][s][0][0]; e1 -= cmp[c][s][0][1]; e2 -= cmp[c][s][1][0]; e3 -= cmp[c][s][1][1]; }
            gb[sidx<C>(k1)] = cmk<C>(e0, e1);
            gb[sidx<C>(k2)] = cmk<C>(e2, e3);
        }
        __syncthreads();
        block_fft<C, LOGN, 1, TG, true>(gb, SSTR, tw, a.tw_shift_n, lt);
        if (slot < a.ncomp) {
            C* dst = Y + ((size_t)(r * a.kx_count + kx) * a.ncomp + slot) * a.ny_pad;
            for (int y = lt; y < a.ny; y += TG) {
                C v = gb[sidx<C>(y)];
                if (r) v = cmul(v, cconj(tw[y << a.tw_shift_p]));
                dst[y] = v;
            }
        }
        __syncthreads();
    }
}

template <typename R, int LOGN, int CPG>
__global__ void __launch_bounds__(ColShape<LOGN>::NT, 1)
    adjoint_column_kernel(ColumnArgs a, const typename cplx<R>::type* __restrict__ Xr, const R* __restrict__ spec,
                          typename cplx<R>::type* __restrict__ Z, const typename cplx<R>::type* __restrict__ tw) {
    using C = typename cplx<R>::type;
    using S = ColShape<LOGN>;
    constexpr int N = S::N, J = S::J, H = S::H, TG = S::TG, NT = S::NT, XPT = S::XPT;
    constexpr int SSTR = spad_len<C>(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf + SSTR;

    const int tid = threadIdx.x;
    const int g = tid / TG, lt = tid - g * TG;
    const int kx = blockIdx.x, r = blockIdx.y;
    const R* sp = spec + (size_t)(r * a.kx_count + kx) * a.nz * a.ncomp * a.jp;
    const bool has_nyq = (r == 0 && lt == 0);

    C fold[XPT];
#pragma unroll
    for (int j = 0; j < XPT; ++j) {
        const int m = tid + j * NT;
        fold[j] = (r && m < N) ? tw[m << a.tw_shift_p] : cmk<C>(1, 0);
    }

    // Transform every component's residual column once.
    C rc[CPG][H][2];
#pragma unroll
    for (int c = 0; c < CPG; ++c)
#pragma unroll
        for (int s = 0; s < H; ++s) rc[c][s][0] = rc[c][s][1] = cmk<C>(0, 0);
    for (int slot = 0; slot < a.ncomp; ++slot) {
        const C* col = Xr + ((size_t)kx * a.ncomp + slot) * a.ny_pad;
#pragma unroll
        for (int j = 0; j < XPT; ++j) {
            const int m = tid + j * NT;
            if (m < N) buf[sidx<C>(m)] = (m < a.ny) ? cmul(col[m], fold[j]) : cmk<C>(0, 0);
        }
        __syncthreads();
        block_fft<C, LOGN, 1, NT, false>(buf, SSTR, tw, a.tw_shift_n, tid);
        if (slot / CPG == g) {
            const int ci = slot - g * CPG;
#pragma unroll
            for (int c = 0; c < CPG; ++c) {
                if (c != ci) continue;
#pragma unroll
                for (int s = 0; s < H; ++s) {
                    int k1, k2;
                    pair_pos<N>(lt * H + s, r, k1, k2);
                    rc[c][s][0] = buf[sidx<C>(k1)];
                    rc[c][s][1] = buf[sidx<C>(k2)];
                }
            }
        }
        __syncthreads();
    }

    R sv[CPG][H], se[CPG];
    auto load_layer = [&](int n) {
#pragma unroll
        for (int c = 0; c < CPG; ++c) {
            const int slot = g * CPG + c;
            const R* row = sp + ((size_t)n * a.ncomp + slot) * a.jp;
#pragma unroll
            for (int s = 0; s < H; ++s) sv[c][s] = (slot < a.ncomp) ? row[lt * H + s] : (R)0;
            se[c] = (slot < a.ncomp && has_nyq) ? row[J] : (R)0;
        }
    };
    load_layer(0);

    for (int n = 0; n < a.nz; ++n) {
        C part[H][2];
#pragma unroll
        for (int s = 0; s < H; ++s) part[s][0] = part[s][1] = cmk<C>(0, 0);
#pragma unroll
        for (int s = 0; s < H; ++s) {
            const int q = lt * H + s;
#pragma unroll
            for (int c = 0; c < CPG; ++c) {
                const int slot = g * CPG + c;
                const bool imag = (a.imag_mask >> slot) & 1u;
                const R s1 = sv[c][s];
                const R s2 = (r == 0 && q == 0) ? se[c] : (((a.oddv_mask >> slot) & 1u) ? -s1 : s1);
                part[s][0] = cadd(part[s][0], spec_term_conj<C>(s1, rc[c][s][0], imag));
                part[s][1] = cadd(part[s][1], spec_term_conj<C>(s2, rc[c][s][1], imag));
            }
        }
        if (n + 1 < a.nz) load_layer(n + 1);
        if (g == 1) {
#pragma unroll
            for (int s = 0; s < H; ++s) {
                int k1, k2;
                pair_pos<N>(lt * H + s, r, k1, k2);
                buf1[sidx<C>(k1)] = part[s][0];
                buf1[sidx<C>(k2)] = part[s][1];
            }
        }
        __syncthreads();
        if (g == 0) {
#pragma unroll
            for (int s = 0; s < H; ++s) {
                int k1, k2;
                pair_pos<N>(lt * H + s, r, k1, k2);
                buf[sidx<C>(k1)] = cadd(part[s][0], buf1[sidx<C>(k1)]);
                buf[sidx<C>(k2)] = cadd(part[s][1], buf1[sidx<C>(k2)]);
            }
        }
        __syncthreads();
        block_fft<C, LOGN, 1, NT, true>(buf, SSTR, tw, a.tw_shift_n, tid);
        C* dst = Z + ((size_t)(r * a.kx_count + kx) * a.nz + n) * a.ny_pad;
        for (int y = tid; y < a.ny; y += NT) {
            C v = buf[sidx<C>(y)];
            if (r) v = cmul(v, cconj(tw[y << a.tw_shift_p]));
            dst[y] = v;
        }
        __syncthreads();
    }
}

template <typename R>
size_t column_smem_bytes(int log_n) {
    using C = typename cplx<R>::type;
    return 2 * (size_t)spad_len<C>(1 << log_n) * sizeof(C);
}

inline int cpg_for(int ncomp) { return (ncomp + 1) / 2; }

}  // namespace grav
