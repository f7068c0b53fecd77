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
// Forward (Eq. 21): the row transforms of each layer's column and that
// layer's spectra slab stream into a shared-memory ring through bulk
// asynchronous copies; NSEQ layers at a time are transformed, multiplied by
// S_{c,n} and accumulated over n in registers (FP32 with a Kahan-compensated
// layer sum, or FP64).  Each thread owns one mirror pair (two bins) for every
// component.  At the end each component's accumulator is inverse-
// transformed and the rows y < ny are written.
//
// Adjoint (transpose of Eq. 21): the residual of every component is
// transformed once; per layer the CTA forms sum_c conj(S_{c,n}) R_c,
// inverse-transforms it and writes that layer's rows.
#pragma once
#include "async_copy.cuh"
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

// Shared-memory layout of the forward column kernel, chosen on the host.
// A ring of `depth` stages, each holding one layer's row-transform column
// (x_bytes) and that layer's kernel-spectra slab (s_bytes), is filled by
// bulk copies; NSEQ layers are transformed per round in the FFT buffers.
struct FwdSmem {
    int depth;
    uint32_t x_bytes, s_bytes, stage_bytes;
    uint32_t fft_off, tw_off, bar_off, total;
};

template <typename R> struct FwdCfg {
    static constexpr int NSEQ = sizeof(R) == 4 ? 4 : 2;  // layers per round
};

// Forward column stage, one CTA per (kx, r) with blockIdx.x = 2 kx + r (the
// two parities of a column run side by side and share its row transforms
// through L2).  Thread q owns mirror pair q and accumulates every component
// for both of its bins; thread 0 also issues the bulk copies.  When each
// layer of a round has at least a warp of threads, the NSEQ layers are
// transformed by separate warp groups that synchronise on their own named
// barriers, so only three block-wide barriers remain per round.
//
// The per-layer product is S v with S = s or i s (imaginary spectra) and,
// for the mirror bin, S = +-s (odd components).  Both factors are constant
// over the layers, so the loop accumulates s v for every component and the
// epilogue applies i and the sign once: sum_n (i s_n) v_n = i sum_n s_n v_n.
// The layer sum is compensated per round of NSEQ layers: the round's terms
// are added in plain arithmetic and the round total enters a Kahan sum.
template <typename R, int LOGN, int NC>
__global__ void __launch_bounds__(ColShape<LOGN>::J, ColShape<LOGN>::J <= 256 ? 2 : 1)
    forward_column_kernel(ColumnArgs a, FwdSmem L, const typename cplx<R>::type* __restrict__ X,
                          const R* __restrict__ spec, typename cplx<R>::type* __restrict__ Y,
                          const typename cplx<R>::type* __restrict__ tw, int* __restrict__ err, size_t x_bstride,
                          size_t y_bstride) {
    using C = typename cplx<R>::type;
    constexpr int N = 1 << LOGN, J = ColShape<LOGN>::J, NT = J;
    constexpr int NSEQ = FwdCfg<R>::NSEQ;
    constexpr int NTG = NT / NSEQ;  // threads per layer group
    constexpr bool GROUPED = NTG >= 32 && NTG % 32 == 0;
    constexpr bool KAHAN = sizeof(R) == 4;
    constexpr int SSTR = spad_len<C>(N);
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    C* fbuf = reinterpret_cast<C*>(smem + L.fft_off);
    C* tws = reinterpret_cast<C*>(smem + L.tw_off);  // fold twiddles W_Py^m, m < N
    C* ttab = tws + N;                                  // per-pass FFT twiddles

    const int tid = threadIdx.x;
    const int grp = tid / NTG, lt = tid - grp * NTG;
    const int r = blockIdx.x & 1, kx = blockIdx.x >> 1;
    const int nz = a.nz, ny = a.ny, depth = L.depth;
    X += blockIdx.y * x_bstride;  // request of a batched call
    Y += blockIdx.y * y_bstride;
    const C* Xk = X + (size_t)kx * nz * a.ny_pad;
    const size_t s_row = (size_t)a.ncomp * a.jp;
    const R* Sk = request_spec(a, spec, blockIdx.y) + (size_t)(r * a.kx_count + kx) * nz * s_row;
    auto stage_x = [&](int s) { return reinterpret_cast<const C*>(smem + (size_t)s * L.stage_bytes); };
    auto stage_s = [&](int s) { return reinterpret_cast<const R*>(smem + (size_t)s * L.stage_bytes + L.x_bytes); };
    auto issue = [&](int n) {
        const int s = n % depth;
        unsigned char* dst = smem + (size_t)s * L.stage_bytes;
        mbar_arrive_expect_tx(&bars[s], L.x_bytes + L.s_bytes);
        bulk_g2s(dst, Xk + (size_t)n * a.ny_pad, L.x_bytes, &bars[s]);
        bulk_g2s(dst + L.x_bytes, Sk + (size_t)n * s_row, L.s_bytes, &bars[s]);
    };

    if (tid == 0) {
        for (int s = 0; s < depth; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    for (int e = tid; e < N; e += NT) tws[e] = tw[e << a.tw_shift_p];
    build_tw_tab<C, LOGN, NT>(ttab, tw, a.tw_shift_n, tid);
    __syncthreads();
    const int first = nz < depth ? nz : depth;
    if (tid == 0)
        for (int n = 0; n < first; ++n) issue(n);

    R acc[NC][4], cmp[NC][4];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[c][j] = cmp[c][j] = 0;
    const int q = tid;
    int k1, k2;
    pair_pos<N>(q, r, k1, k2);
    const bool nyq = (r == 0 && q == 0);

    for (int n0 = 0; n0 < nz; n0 += NSEQ) {
        const int cnt = nz - n0 < NSEQ ? nz - n0 : NSEQ;
        int st[NSEQ];
#pragma unroll
        for (int l = 0; l < NSEQ; ++l) st[l] = (n0 + l) % depth;
        bool ok = true;
        for (int l = 0; l < cnt; ++l)
            ok = ok && mbar_wait_bounded(&bars[st[l]], (uint32_t)(((n0 + l) / depth) & 1), kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            // A copy never arrived: record it, let the copies still in
            // flight land (bounded), and leave.
            if (tid == 0) {
                atomicExch(err, 1);
                const int last = n0 + depth < nz ? n0 + depth : nz;
                for (int n = n0; n < last; ++n)
                    mbar_wait_bounded(&bars[n % depth], (uint32_t)((n / depth) & 1), kWaitLimitNs);
            }
            return;
        }
        // Column FFTs of the round's layers; the first pass reads the staged
        // rows and folds them for ky parity r: a[m] = x[m] W_Py^(m r).
        if constexpr (GROUPED) {
            if (grp < cnt) {
                const C* xs = stage_x((n0 + grp) % depth);
                block_fft_tab_from<C, LOGN, 1, NTG, false>(
                    fbuf + grp * SSTR, SSTR, ttab, lt,
                    [&](int, int m) {
                        C v = cmk<C>(0, 0);
                        if (m < ny) {
                            v = xs[m];
                            if (r) v = cmul(v, tws[m]);
                        }
                        return v;
                    },
                    GroupSync{1 + grp, NTG});
            }
            __syncthreads();
        } else {
            block_fft_tab_from<C, LOGN, NSEQ, NT, false>(fbuf, SSTR, ttab, tid, [&](int l, int m) {
                C v = cmk<C>(0, 0);
                if (l < cnt && m < ny) {
                    v = stage_x(st[l])[m];
                    if (r) v = cmul(v, tws[m]);
                }
                return v;
            });
        }
        R part[NC][4];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[c][j] = 0;
        if (!nyq) {
#pragma unroll
            for (int l = 0; l < NSEQ; ++l) {
                if (l < cnt) {
                    const C v1 = fbuf[l * SSTR + sidx<C>(k1)], v2 = fbuf[l * SSTR + sidx<C>(k2)];
                    const R* Ss = stage_s(st[l]) + q;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const R s1 = Ss[c * a.jp];
                        part[c][0] += s1 * v1.x;
                        part[c][1] += s1 * v1.y;
                        part[c][2] += s1 * v2.x;
                        part[c][3] += s1 * v2.y;
                    }
                }
            }
        } else {
            // pair 0 of the even parity holds ky = 0 and the Nyquist row
            // ky = Py/2, each with its own stored value
            for (int l = 0; l < cnt; ++l) {
                const C v1 = fbuf[l * SSTR + sidx<C>(k1)], v2 = fbuf[l * SSTR + sidx<C>(k2)];
                const R* Ss = stage_s(st[l]);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const R s1 = Ss[c * a.jp], s2 = Ss[c * a.jp + J];
                    part[c][0] += s1 * v1.x;
                    part[c][1] += s1 * v1.y;
                    part[c][2] += s2 * v2.x;
                    part[c][3] += s2 * v2.y;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (KAHAN) kahan_add(acc[c][j], cmp[c][j], part[c][j]);
                else acc[c][j] += part[c][j];
            }
        __syncthreads();  // stages and FFT buffers free again
        if (tid == 0) {
            fence_proxy_async_smem();
            for (int l = 0; l < cnt; ++l)
                if (n0 + l + depth < nz) issue(n0 + l + depth);
        }
    }

    // Apply i (imaginary spectra) and the mirror sign (odd in y), then the
    // inverse column transforms, NSEQ components per round; crop to y < ny.
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += NSEQ) {
#pragma unroll
        for (int l = 0; l < NSEQ; ++l) {
            const int c = c0 + l;
            if (c < NC) {
                R e[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) e[j] = KAHAN ? acc[c][j] - cmp[c][j] : acc[c][j];
                const bool imag = (a.imag_mask >> c) & 1u;
                const bool flip = !nyq && ((a.oddv_mask >> c) & 1u);
                C b1 = cmk<C>(e[0], e[1]), b2 = cmk<C>(e[2], e[3]);
                if (flip) b2 = cmk<C>(-b2.x, -b2.y);
                if (imag) {
                    b1 = cmk<C>(-b1.y, b1.x);
                    b2 = cmk<C>(-b2.y, b2.x);
                }
                fbuf[l * SSTR + sidx<C>(k1)] = b1;
                fbuf[l * SSTR + sidx<C>(k2)] = b2;
            }
        }
        __syncthreads();
        if constexpr (GROUPED) {
            const int c = c0 + grp;
            if (c < NC) {
                C* fb = fbuf + grp * SSTR;
                block_fft_tab<C, LOGN, 1, NTG, true>(fb, SSTR, ttab, lt, GroupSync{1 + grp, NTG});
                C* dst = Y + ((size_t)(r * a.kx_count + kx) * a.ncomp + c) * a.ny_pad;
                for (int y = lt; y < ny; y += NTG) {
                    C v = fb[sidx<C>(y)];
                    if (r) v = cmul(v, cconj(tws[y]));
                    dst[y] = v;
                }
            }
        } else {
            block_fft_tab<C, LOGN, NSEQ, NT, true>(fbuf, SSTR, ttab, tid);
            for (int e = tid; e < NSEQ * ny; e += NT) {
                const int l = e / ny, y = e - l * ny;
                const int c = c0 + l;
                if (c < NC) {
                    C v = fbuf[l * SSTR + sidx<C>(y)];
                    if (r) v = cmul(v, cconj(tws[y]));
                    Y[((size_t)(r * a.kx_count + kx) * a.ncomp + c) * a.ny_pad + y] = v;
                }
            }
        }
        __syncthreads();
    }
}

template <typename R, int LOGN, int CPG>
__global__ void __launch_bounds__(ColShape<LOGN>::NT, 1)
    adjoint_column_kernel(ColumnArgs a, const typename cplx<R>::type* __restrict__ Xr, const R* __restrict__ spec,
                          typename cplx<R>::type* __restrict__ Z, const typename cplx<R>::type* __restrict__ tw,
                          size_t x_bstride, size_t z_bstride) {
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
    Xr += blockIdx.z * x_bstride;  // request of a batched call
    Z += blockIdx.z * z_bstride;
    const R* sp = request_spec(a, spec, blockIdx.z) + (size_t)(r * a.kx_count + kx) * a.nz * a.ncomp * a.jp;
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

// Ring depth and offsets for the forward column kernel; depth is 0 when even
// NSEQ stages do not fit in the shared memory a CTA may use.
template <typename R>
FwdSmem forward_smem(int log_n, int ny_pad, int ncomp, int jp, int max_bytes) {
    using C = typename cplx<R>::type;
    constexpr int NSEQ = FwdCfg<R>::NSEQ;
    FwdSmem L{};
    L.x_bytes = (uint32_t)(ny_pad * sizeof(C));
    L.s_bytes = (uint32_t)(ncomp * jp * sizeof(R));
    L.stage_bytes = (L.x_bytes + L.s_bytes + 127u) & ~127u;
    const uint32_t fft_bytes = (uint32_t)(NSEQ * spad_len<C>(1 << log_n) * sizeof(C));
    const uint32_t tw_bytes = (uint32_t)(((1u << log_n) + tw_tab_len(log_n)) * sizeof(C));  // fold + pass tables
    int depth = 2 * NSEQ;
    while (depth >= NSEQ && (size_t)depth * L.stage_bytes + fft_bytes + tw_bytes + depth * 8 + 128 > (size_t)max_bytes)
        --depth;
    if (depth < NSEQ) return FwdSmem{};
    L.depth = depth;
    L.fft_off = depth * L.stage_bytes;
    L.tw_off = L.fft_off + fft_bytes;
    L.bar_off = (L.tw_off + tw_bytes + 7u) & ~7u;
    L.total = L.bar_off + depth * 8;
    return L;
}

inline int cpg_for(int ncomp) { return (ncomp + 1) / 2; }

// Components per thread instantiated for the forward kernel (exactly ncomp).
inline int nc_for(int ncomp) { return ncomp; }

}  // namespace grav
