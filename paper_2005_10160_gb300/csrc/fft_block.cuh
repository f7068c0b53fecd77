// Shared-memory FFT building blocks for the spectral BTTB product.
//
// The Toeplitz (Eq. 17) and BTTB (Eq. 20) matrix-vector products are formed
// by circulant embedding and FFT (Eqs. 18-19).  These device routines run the
// FFTs inside the calling kernel: complex radix-2/4/8 butterflies in
// registers, Stockham autosort passes (natural order in and out) through one
// padded shared-memory buffer, twiddles read from a per-plan table
// W_T[e] = exp(-2 pi i e / T) with T the largest transform size of the plan.
//
// Conventions: forward transforms use exp(-2 pi i jk/N), inverse ones
// exp(+2 pi i jk/N); neither is normalised (the 1/(Px Py) of the inverse is
// folded into the stored kernel spectra).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace grav {

template <typename R> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
// FP32: one packed two-wide instruction per complex add or subtract
// (sm_100 family); a - b as fma(b, -1, a) rounds exactly like the
// subtraction, so results are bit for bit those of the scalar form.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
// Multiply by -i (forward sign) or +i (inverse sign).
template <typename C, bool INV> __device__ __forceinline__ C cmul_ni(C a) {
    return INV ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

// Padded shared-memory index: 16 spare bytes per 128 (8-byte elements: two
// per 16, which keeps even indices 16-byte aligned; 16-byte elements: one
// per 8) keep the strided Stockham stores at (or near) the minimum number
// of wavefronts.
template <typename C> __host__ __device__ __forceinline__ constexpr int sidx(int e) {
    return sizeof(C) == 8 ? e + 2 * (e >> 4) : e + (e >> 3);
}
template <typename C> __host__ __device__ constexpr int spad_len(int n) {
    return sizeof(C) == 8 ? n + 2 * (n >> 4) + 2 : n + (n >> 3) + 1;
}

// Stride between sequences that sit back to back: the padded length rounded
// so that the same element of consecutive sequences falls in different
// banks (8-byte elements: stride = 4 mod 16; 16-byte elements: 2 mod 8).
template <typename C> __host__ __device__ constexpr int seq_stride(int n) {
    const int len = spad_len<C>(n);
    return sizeof(C) == 8 ? len + ((4 - len % 16) + 16) % 16 : len + ((2 - len % 8) + 8) % 8;
}

// In-register DFTs of size 2, 4, 8.
template <typename C, bool INV> __device__ __forceinline__ void dft2(C& a, C& b) {
    C t = a; a = cadd(t, b); b = csub(t, b);
}
template <typename C, bool INV> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2);
    C t2 = cadd(a1, a3), t3 = cmul_ni<C, INV>(csub(a1, a3));
    a0 = cadd(t0, t2); a2 = csub(t0, t2);
    a1 = cadd(t1, t3); a3 = csub(t1, t3);
}
template <typename C, bool INV> __device__ __forceinline__ void dft8(C* u) {
    using R = decltype(C::x);
    const R h = (R)0.70710678118654752440;
    dft4<C, INV>(u[0], u[2], u[4], u[6]);
    dft4<C, INV>(u[1], u[3], u[5], u[7]);
    // odd half times w8^k, w8 = exp(-+ 2 pi i / 8)
    C o1 = u[3], o2 = u[5], o3 = u[7];
    C w1 = INV ? cmk<C>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : cmk<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
    C w2 = cmul_ni<C, INV>(o2);
    C w3 = INV ? cmk<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : cmk<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    C e0 = u[0], e1 = u[2], e2 = u[4], e3 = u[6], o0 = u[1];
    u[0] = cadd(e0, o0); u[4] = csub(e0, o0);
    u[1] = cadd(e1, w1); u[5] = csub(e1, w1);
    u[2] = cadd(e2, w2); u[6] = csub(e2, w2);
    u[3] = cadd(e3, w3); u[7] = csub(e3, w3);
}
template <typename C, int R, bool INV> __device__ __forceinline__ void dftR(C* u) {
    if constexpr (R == 2) dft2<C, INV>(u[0], u[1]);
    else if constexpr (R == 4) dft4<C, INV>(u[0], u[1], u[2], u[3]);
    else dft8<C, INV>(u);
}

// Twiddles w^1 .. w^(R-1) of a butterfly from w = W^k alone: powers by
// products of depth <= 3 (w2 = w w, w3 = w2 w, w4 = w2 w2, w5 = w4 w,
// w6 = w3 w3, w7 = w4 w3), so each costs at most a few roundings.
template <typename C, int R> __device__ __forceinline__ void twiddle_powers(C w, C* p) {
    p[1] = w;
    if constexpr (R >= 4) {
        p[2] = cmul(w, w);
        p[3] = cmul(p[2], w);
    }
    if constexpr (R >= 8) {
        p[4] = cmul(p[2], p[2]);
        p[5] = cmul(p[4], w);
        p[6] = cmul(p[3], p[3]);
        p[7] = cmul(p[4], p[3]);
    }
}

// Radix of pass p for a 2^LOGN transform: the first pass takes LOGN mod 3
// (radix 2 or 4), the rest are radix 8.
__host__ __device__ constexpr int pass_radix(int logn, int p) {
    return (logn % 3 != 0 && p == 0) ? (1 << (logn % 3)) : 8;
}
__host__ __device__ constexpr int num_passes(int logn) {
    return logn / 3 + (logn % 3 != 0 ? 1 : 0);
}
// Product of the radices of the passes before p.
__host__ __device__ constexpr int pass_ls(int logn, int p) {
    int ls = 1;
    for (int q = 0; q < p; ++q) ls *= pass_radix(logn, q);
    return ls;
}

// One Stockham pass of radix R over NSEQ sequences of length N = 2^LOGN that
// sit back to back (stride SSTR padded elements) in shared memory.  Threads
// tid < NT take butterflies tid, tid + NT, ... and hold them in registers
// across the barrier, so one buffer suffices.  Every thread of the block
// calls this (it contains __syncthreads()).
template <typename C, int LOGN, int P, int NSEQ, int NT, bool INV>
__device__ __forceinline__ void fft_pass(C* buf, int sstr, const C* __restrict__ tw, int tw_shift, int tid) {
    constexpr int N = 1 << LOGN;
    constexpr int R = pass_radix(LOGN, P);
    constexpr int LS = pass_ls(LOGN, P);
    constexpr int NR = N / R;
    constexpr int TOTAL = NSEQ * NR;
    constexpr int BPT = (TOTAL + NT - 1) / NT;
    constexpr bool LIN_LD = NR % 16 == 0, LIN_ST = LS % 16 == 0 || LS == 1;
    C u[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = tid + b * NT;
        if (tid < NT && g < TOTAL) {
            const int s = g / NR, i = g - s * NR;
            const C* x = buf + s * sstr;
            if constexpr (LIN_LD) {
                const C* xb = x + sidx<C>(i);
#pragma unroll
                for (int r = 0; r < R; ++r) u[b][r] = xb[r * sidx<C>(NR)];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) u[b][r] = x[sidx<C>(i + r * NR)];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = tid + b * NT;
        if (tid < NT && g < TOTAL) {
            const int s = g / NR, i = g - s * NR;
            const int k = i & (LS - 1);
            if constexpr (LS > 1) {
                // twiddles W_{LS R}^{r k} = (W_N^{k N / (LS R)})^r
                C w = tw[(k * (N / (LS * R))) << tw_shift];
                if (INV) w.y = -w.y;
                C pw[R];
                twiddle_powers<C, R>(w, pw);
#pragma unroll
                for (int r = 1; r < R; ++r) u[b][r] = cmul(u[b][r], pw[r]);
            }
            dftR<C, R, INV>(u[b]);
            C* y = buf + s * sstr;
            const int j = (i - k) * R + k;
            if constexpr (LIN_ST) {
                // LS == 1: the R outputs are contiguous inside one pad group
                C* yb = y + sidx<C>(j);
#pragma unroll
                for (int r = 0; r < R; ++r) yb[LS == 1 ? r : r * sidx<C>(LS)] = u[b][r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) y[sidx<C>(j + r * LS)] = u[b][r];
            }
        }
    }
    __syncthreads();
}

// Barrier over the whole block.
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
// Named barrier `id` (1..15) over `count` threads (whole warps) of the block.
struct GroupSync {
    int id, count;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
    }
};

// Per-pass twiddle tables.  Pass p >= 1 of a 2^LOGN transform multiplies
// input r of butterfly k (k < ls) by W_{ls R}^{r k}; the table keeps these at
// tab[tw_tab_off(p) + (r - 1) ls + k], so the threads of a warp (consecutive
// k) read consecutive entries, or one broadcast entry when ls is small.
__host__ __device__ constexpr int tw_tab_off(int logn, int p) {
    int off = 0;
    for (int q = 1; q < p; ++q) off += pass_ls(logn, q) * (pass_radix(logn, q) - 1);
    return off;
}
__host__ __device__ constexpr int tw_tab_len(int logn) { return tw_tab_off(logn, num_passes(logn)); }

// Fill the table from W_T (T = N << tw_shift); all threads of the block call it.
template <typename C, int LOGN, int NT>
__device__ __forceinline__ void build_tw_tab(C* tab, const C* __restrict__ tw, int tw_shift, int tid) {
    constexpr int N = 1 << LOGN;
#pragma unroll
    for (int p = 1; p < num_passes(LOGN); ++p) {
        const int ls = pass_ls(LOGN, p), R = pass_radix(LOGN, p), off = tw_tab_off(LOGN, p);
        for (int e = tid; e < ls * (R - 1); e += NT) {
            const int r = e / ls + 1, k = e - (r - 1) * ls;
            tab[off + e] = tw[(r * k * (N / (ls * R))) << tw_shift];
        }
    }
}

// Stockham pass p >= 1 with twiddles from the per-pass table.
template <typename C, int LOGN, int P, int NSEQ, int NT, bool INV, typename Sync = BlockSync>
__device__ __forceinline__ void fft_pass_tab(C* buf, int sstr, const C* tab, int tid, Sync sync = Sync()) {
    constexpr int N = 1 << LOGN;
    constexpr int R = pass_radix(LOGN, P);
    constexpr int LS = pass_ls(LOGN, P);
    constexpr int OFF = tw_tab_off(LOGN, P);
    constexpr int NR = N / R;
    constexpr int TOTAL = NSEQ * NR;
    constexpr int BPT = (TOTAL + NT - 1) / NT;
    // padded offsets are linear when the stride is a whole number of pad
    // groups (16 elements): sidx(e + r S) = sidx(e) + r sidx(S)
    constexpr bool LIN_LD = NR % 16 == 0, LIN_ST = LS % 16 == 0;
    C u[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = tid + b * NT;
        if (tid < NT && g < TOTAL) {
            const int s = g / NR, i = g - s * NR;
            const C* x = buf + s * sstr;
            if constexpr (LIN_LD) {
                const C* xb = x + sidx<C>(i);
#pragma unroll
                for (int r = 0; r < R; ++r) u[b][r] = xb[r * sidx<C>(NR)];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) u[b][r] = x[sidx<C>(i + r * NR)];
            }
        }
    }
    sync();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = tid + b * NT;
        if (tid < NT && g < TOTAL) {
            const int s = g / NR, i = g - s * NR;
            const int k = i & (LS - 1);
            const C* t = tab + OFF + k;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = t[(r - 1) * LS];
                if (INV) w.y = -w.y;
                u[b][r] = cmul(u[b][r], w);
            }
            dftR<C, R, INV>(u[b]);
            C* y = buf + s * sstr;
            const int j = (i - k) * R + k;
            if constexpr (LIN_ST) {
                C* yb = y + sidx<C>(j);
#pragma unroll
                for (int r = 0; r < R; ++r) yb[r * sidx<C>(LS)] = u[b][r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) y[sidx<C>(j + r * LS)] = u[b][r];
            }
        }
    }
    sync();
}

template <typename C, int LOGN, int NSEQ, int NT, bool INV, typename Sync = BlockSync>
__device__ __forceinline__ void fft_tail_tab(C* buf, int sstr, const C* tab, int tid, Sync sync = Sync()) {
    constexpr int NP = num_passes(LOGN);
    if constexpr (NP > 1) fft_pass_tab<C, LOGN, 1, NSEQ, NT, INV>(buf, sstr, tab, tid, sync);
    if constexpr (NP > 2) fft_pass_tab<C, LOGN, 2, NSEQ, NT, INV>(buf, sstr, tab, tid, sync);
    if constexpr (NP > 3) fft_pass_tab<C, LOGN, 3, NSEQ, NT, INV>(buf, sstr, tab, tid, sync);
    if constexpr (NP > 4) fft_pass_tab<C, LOGN, 4, NSEQ, NT, INV>(buf, sstr, tab, tid, sync);
}

// First Stockham pass (no twiddles) taking its inputs from a functor
// load(s, m) -> element m of sequence s, and writing to the shared buffer.
template <typename C, int LOGN, int R, int NSEQ, int NT, bool INV, typename Load, typename Sync = BlockSync>
__device__ __forceinline__ void fft_first_pass_from(C* buf, int sstr, int tid, Load load, Sync sync = Sync()) {
    constexpr int N = 1 << LOGN;
    constexpr int NR = N / R;
    constexpr int TOTAL = NSEQ * NR;
    constexpr int BPT = (TOTAL + NT - 1) / NT;
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = tid + b * NT;
        if (tid < NT && g < TOTAL) {
            const int s = g / NR, i = g - s * NR;
            C u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = load(s, i + r * NR);
            dftR<C, R, INV>(u);
            C* yb = buf + s * sstr + sidx<C>(i * R);  // R <= 8 outputs inside one pad group
#pragma unroll
            for (int r = 0; r < R; ++r) yb[r] = u[r];
        }
    }
    sync();
}

// FFT of NSEQ sequences whose inputs come from load(s, m); the result is in
// buf (natural order).
template <typename C, int LOGN, int NSEQ, int NT, bool INV, typename Load>
__device__ __forceinline__ void block_fft_from(C* buf, int sstr, const C* __restrict__ tw, int tw_shift, int tid,
                                               Load load) {
    constexpr int NP = num_passes(LOGN);
    static_assert(NP <= 5, "transform too long");
    fft_first_pass_from<C, LOGN, pass_radix(LOGN, 0), NSEQ, NT, INV>(buf, sstr, tid, load);
    if constexpr (NP > 1) fft_pass<C, LOGN, 1, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
    if constexpr (NP > 2) fft_pass<C, LOGN, 2, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
    if constexpr (NP > 3) fft_pass<C, LOGN, 3, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
    if constexpr (NP > 4) fft_pass<C, LOGN, 4, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
}

// The same with table twiddles: inputs from load(s, m), result in buf.
template <typename C, int LOGN, int NSEQ, int NT, bool INV, typename Load, typename Sync = BlockSync>
__device__ __forceinline__ void block_fft_tab_from(C* buf, int sstr, const C* tab, int tid, Load load,
                                                   Sync sync = Sync()) {
    static_assert(num_passes(LOGN) <= 5, "transform too long");
    fft_first_pass_from<C, LOGN, pass_radix(LOGN, 0), NSEQ, NT, INV>(buf, sstr, tid, load, sync);
    fft_tail_tab<C, LOGN, NSEQ, NT, INV>(buf, sstr, tab, tid, sync);
}

// In-place FFT of NSEQ sequences in buf with table twiddles.
template <typename C, int LOGN, int NSEQ, int NT, bool INV, typename Sync = BlockSync>
__device__ __forceinline__ void block_fft_tab(C* buf, int sstr, const C* tab, int tid, Sync sync = Sync()) {
    constexpr int N = 1 << LOGN;
    constexpr int R = pass_radix(LOGN, 0);
    constexpr int NR = N / R;
    constexpr int TOTAL = NSEQ * NR;
    constexpr int BPT = (TOTAL + NT - 1) / NT;
    C u[BPT][R];
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = tid + b * NT;
        if (tid < NT && g < TOTAL) {
            const int s = g / NR, i = g - s * NR;
#pragma unroll
            for (int r = 0; r < R; ++r) u[b][r] = buf[s * sstr + sidx<C>(i + r * NR)];
        }
    }
    sync();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int g = tid + b * NT;
        if (tid < NT && g < TOTAL) {
            const int s = g / NR, i = g - s * NR;
            dftR<C, R, INV>(u[b]);
            C* yb = buf + s * sstr + sidx<C>(i * R);
#pragma unroll
            for (int r = 0; r < R; ++r) yb[r] = u[b][r];
        }
    }
    sync();
    fft_tail_tab<C, LOGN, NSEQ, NT, INV>(buf, sstr, tab, tid, sync);
}

// Full in-place FFT of NSEQ sequences of 2^LOGN points in shared memory
// (natural order in, natural order out).  tw is W_T with T = N << tw_shift.
template <typename C, int LOGN, int NSEQ, int NT, bool INV>
__device__ __forceinline__ void block_fft(C* buf, int sstr, const C* __restrict__ tw, int tw_shift, int tid) {
    constexpr int NP = num_passes(LOGN);
    static_assert(NP <= 5, "transform too long");
    if constexpr (NP > 0) fft_pass<C, LOGN, 0, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
    if constexpr (NP > 1) fft_pass<C, LOGN, 1, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
    if constexpr (NP > 2) fft_pass<C, LOGN, 2, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
    if constexpr (NP > 3) fft_pass<C, LOGN, 3, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
    if constexpr (NP > 4) fft_pass<C, LOGN, 4, NSEQ, NT, INV>(buf, sstr, tw, tw_shift, tid);
}

}  // namespace grav
