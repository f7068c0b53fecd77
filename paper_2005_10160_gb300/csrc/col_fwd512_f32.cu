// Forward column stage for 512-point FP32 column transforms (Py = 1024,
// 257 <= ny <= 512): both ky parities of a kx column in one CTA, each warp
// transform doing the two parities of one layer at once.
//
// The layout is that of the 1024-point kernel (spectral_wf.cuh): 24 warps at
// 80 registers, warps 0-15 accumulate (thread q: parity q / 256, mirror pair
// q % 256, every component), warps 16-23 transform layers f, f + 8, ... from
// their own X slot, which they refill by bulk copy.  A layer's F slot holds
// both parities' 512 bins (parity r at offset 512 r) and, in its tail, the
// Nyquist-row spectra values (bin ky = Py / 2 of parity 0, the second bin of
// thread 0).  The accumulate threads keep only the plain sums of the current
// 32-layer block in registers; the compensated sums and their corrections
// live in shared memory (the X slots are half the size of the 1024-point
// kernel's), which leaves the transforms enough registers.  The thread of
// pair 0 of each parity prefetches that parity's spectra into L2 eight layers
// ahead of the one-layer-ahead register loads.
//
// The column x[m] (m < 512, zero-padded to Py) has ky = 2k + r bins
// X_r[k] = sum_m x[m] W_1024^(m r) W_512^(m k): parity 0 is the 512-point
// FFT of x, parity 1 that of the folded column x[m] W_1024^m.  With
// m = 32 n1 + n2 the fold factor is W_32^n1 (a constant of register n1) times
// W_1024^n2 (constant over n1, so it moves past the first 16-point pass into
// the transpose twiddles of the parity-1 transform): t2 = W_1024^(n2 (2 k1 +
// r)).  The inverse transforms cancel the extra W_1024^-n2 of these twiddles
// by scaling the parity-1 input by W_1024^n2, and unfold the parity-1 output
// y = k1 + 16 k2 by W_1024^-k1 W_64^-k2.
#include "async_copy.cuh"
#include "grav_internal.h"
#include "spectral.cuh"
#include "spectral_ws.cuh"
#include "warp_fft.cuh"

namespace grav {

namespace {

struct W5Shape {
    static constexpr int N = 512;          // transform length (per parity)
    static constexpr int NB = 2 * N;       // bins per F slot (both parities)
    static constexpr int JH = N / 2;       // mirror pairs per parity
    static constexpr int J = 2 * JH;       // accumulate threads (16 warps)
    static constexpr int FWARPS = 8;       // FFT warps
    static constexpr int NT = J + 32 * FWARPS;
    static constexpr int FSLOT = kWarpFftSlot;  // complex values per F slot (transpose area)
    static constexpr int REGS = 80;
    static constexpr int DX = FWARPS;      // one X slot per FFT warp
    static constexpr int PF = 8;           // spectra prefetch distance (layers)
    static constexpr int JP = 260;         // spectra row pitch: JH + 1 rounded up to 4
    static constexpr int BLOCK = 32;       // layers per compensated block
};
static_assert(W5Shape::NB + W5Shape::FWARPS <= W5Shape::FSLOT, "Nyquist values fit in the F slot tail");

struct W5Smem {
    int df;
    uint32_t x_bytes, s_bytes, f_bytes;
    uint32_t f_off, t2_off, cmp_off, acc_off, bar_off, flag_off, total;
};

template <int NC>
__global__ void __maxnreg__(W5Shape::REGS)
    forward_column_wf512_kernel(ColumnArgs a, W5Smem L, const float2* __restrict__ X, const float* __restrict__ spec,
                                float2* __restrict__ Y, const float2* __restrict__ tw, int* __restrict__ err,
                                size_t x_bstride, size_t y_bstride) {
    using C = float2;
    constexpr int N = W5Shape::N, NB = W5Shape::NB, JH = W5Shape::JH, J = W5Shape::J, FW = W5Shape::FWARPS;
    constexpr int NT = W5Shape::NT, FS = W5Shape::FSLOT, DX = W5Shape::DX, PF = W5Shape::PF, JP = W5Shape::JP;
    constexpr int S_ROW = NC * JP;  // floats per layer of spectra (one parity)
    static_assert(NC <= FW, "one inverse transform pair per FFT warp");
    static_assert(NC <= 7, "compensated sums of up to 7 components fit in shared memory");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* xring = smem;
    C* fring = reinterpret_cast<C*>(smem + L.f_off);
    C* t2 = reinterpret_cast<C*>(smem + L.t2_off);  // W_1024^(n2 (2 k1 + r)) at [16 r + k1][n2]
    float* cmp = reinterpret_cast<float*>(smem + L.cmp_off);  // Kahan corrections [c][j][q]
    float* accs = reinterpret_cast<float*>(smem + L.acc_off); // compensated sums [c][j][q]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* xfull = bars;
    uint64_t* ffull = xfull + DX;
    uint64_t* fempty = ffull + L.df;
    volatile int* abort = reinterpret_cast<volatile int*>(smem + L.flag_off);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kx = blockIdx.x;
    const int nz = a.nz, ny = a.ny;
    X += blockIdx.y * x_bstride;  // request of a batched call
    Y += blockIdx.y * y_bstride;
    const C* Xk = X + (size_t)kx * nz * a.ny_pad;
    const float* specb = request_spec(a, spec, blockIdx.y);
    const float* Sk0 = specb + (size_t)kx * nz * S_ROW;                   // parity 0
    const float* Sk1 = specb + (size_t)(a.kx_count + kx) * nz * S_ROW;    // parity 1

    if (tid == 0) {
        for (int s = 0; s < DX; ++s) mbar_init(&xfull[s], 1);
        for (int s = 0; s < L.df; ++s) {
            mbar_init(&ffull[s], 32);
            mbar_init(&fempty[s], J);
        }
        *abort = 0;
        fence_mbar_init();
    }
    for (int e = tid; e < 2 * N; e += NT) {
        const int K = e >> 5, n2 = e & 31, h = K >> 4, k1 = K & 15;
        t2[e] = tw[((n2 * (2 * k1 + h)) & (2 * N - 1)) << a.tw_shift_p];
    }
    for (int e = tid; e < 4 * NC * J; e += NT) cmp[e] = accs[e] = 0.f;
    __syncthreads();
    if (tid == 0) {
        // first layer of every X slot, and the first PF layers' spectra into L2
        for (int n = 0; n < DX && n < nz; ++n) {
            mbar_arrive_expect_tx(&xfull[n], L.x_bytes);
            bulk_g2s(xring + (size_t)n * L.x_bytes, Xk + (size_t)n * a.ny_pad, L.x_bytes, &xfull[n]);
        }
        for (int n = 0; n < PF && n < nz; ++n) {
            bulk_prefetch_l2(Sk0 + (size_t)n * S_ROW, L.s_bytes);
            bulk_prefetch_l2(Sk1 + (size_t)n * S_ROW, L.s_bytes);
        }
    }

    bool failed = false;
    const bool is_mac = tid < J;
    const bool nyq = tid == 0;  // parity 0, pair 0: bins ky = 0 and ky = Py / 2

    if (!is_mac) {
        // ---------------- FFT warp f: layers f, f + FW, ... ----------------
        const int f = warp - (J >> 5);
        unsigned char* xslot = xring + (size_t)f * L.x_bytes;
        const C* xs = reinterpret_cast<const C*>(xslot);
        int pending = f < nz ? f : -1;  // layer of the copy in flight into X slot f
        // Nyquist-row spectra value of component `lane`, one iteration ahead
        const bool has_nyq = lane < NC;
        float snyq_next = (has_nyq && f < nz) ? __ldg(Sk0 + (size_t)f * S_ROW + lane * JP + JH) : 0.f;
        for (int n = f; n < nz; n += FW) {
            const int sf = n % L.df;
            int ok = 1;
            if (lane == 0) {
                ok = ws_wait(&xfull[f], (uint32_t)((n / DX) & 1), abort);
                if (ok) pending = -1;
                if (ok && n >= L.df) ok = ws_wait(&fempty[sf], (uint32_t)((n / L.df - 1) & 1), abort);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                failed = true;
                break;
            }
            const float snyq = snyq_next;
            if (has_nyq && n + FW < nz) snyq_next = __ldg(Sk0 + (size_t)(n + FW) * S_ROW + lane * JP + JH);
            // u[n1]: parity 0, u[16 + n1]: parity 1 with its fold factor W_32^n1
            float2 u[32];
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
                const int m = 32 * n1 + lane;
                const C v = m < ny ? xs[m] : make_float2(0.f, 0.f);
                u[n1] = v;
                u[16 + n1] = tw32<false>(v, n1);
            }
            __syncwarp();  // every lane's reads of X slot f are done
            if (lane == 0 && n + FW < nz) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&xfull[f], L.x_bytes);
                bulk_g2s(xslot, Xk + (size_t)(n + FW) * a.ny_pad, L.x_bytes, &xfull[f]);
                pending = n + FW;
            }
            C* fb = fring + sf * FS;
            warp_fft512x2<false>(u, fb, t2, lane);
            // lane: parity lane / 16, k1 = lane % 16, bins k1 + 16 bitrev5(j)
            const int base = (lane >> 4) * N + (lane & 15);
#pragma unroll
            for (int j = 0; j < 32; ++j) fb[base + 16 * bitrev5(j)] = u[j];
            if (lane < NC) fb[NB + lane] = make_float2(snyq, 0.f);
            mbar_arrive(&ffull[sf]);  // this lane's writes of the F slot are done
        }
        if (lane == 0 && pending >= 0) {
            // a copy that will not be consumed (failure path): let it land
            // (bounded) before the CTA's shared memory is released
            mbar_wait_bounded(&xfull[f], (uint32_t)((pending / DX) & 1), kWaitLimitNs);
        }
        if (cta_sync_or(failed || *abort)) return;
        cta_sync();  // the accumulate threads have written the sums
        // inverse column transforms of component f, both parities (F slot f)
        const int c = f;
        if (c < NC) {
            C* fb = fring + c * FS;
            float2 u[32];
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
                u[n1] = fb[32 * n1 + lane];
                u[16 + n1] = fb[N + 32 * n1 + lane];
            }
            __syncwarp();
            {
                const C w = __ldg(tw + (lane << a.tw_shift_p));  // W_1024^n2, n2 = lane
#pragma unroll
                for (int n1 = 0; n1 < 16; ++n1) u[16 + n1] = cmul(u[16 + n1], w);
            }
            warp_fft512x2<true>(u, fb, t2, lane);
            const int h = lane >> 4, k1 = lane & 15;
            C* dst = Y + ((size_t)(h * a.kx_count + kx) * a.ncomp + c) * a.ny_pad;
            const C wu = cconj(__ldg(tw + (k1 << a.tw_shift_p)));  // W_1024^-k1
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int y = k1 + 16 * bitrev5(j);
                if (y < ny) dst[y] = h ? tw64(cmul(u[j], wu), 64 - bitrev5(j)) : u[j];
            }
        }
    } else {
        // ---------------- accumulate: thread q owns parity q / 256, pair q % 256 ----------------
        const int q = tid, rq = q / JH, p = q % JH;
        int k1 = 0, k2 = 0;
        pair_pos<N>(p, rq, k1, k2);
        k1 += rq * N;
        k2 += rq * N;
        float part[NC][4];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[c][j] = 0.f;
        // this thread's spectra values S[n][c][p] of its parity, one layer ahead
        const float* Sq = (rq ? Sk1 : Sk0) + p;
        float sv[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) sv[c] = nz > 0 ? __ldg(Sq + c * JP) : 0.f;
        int sf = 0, wrap = 0;  // F slot of layer n (n % df) and n / df, stepped with n
        for (int n = 0; n < nz; ++n) {
            if (!ws_wait(&ffull[sf], (uint32_t)(wrap & 1), abort)) {
                failed = true;
                break;
            }
            const C* fb = fring + sf * FS;
            const C v1 = fb[k1], v2 = fb[k2];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float s2 = nyq ? fb[NB + c].x : sv[c];
                part[c][0] += sv[c] * v1.x;
                part[c][1] += sv[c] * v1.y;
                part[c][2] += s2 * v2.x;
                part[c][3] += s2 * v2.y;
            }
            mbar_arrive(&fempty[sf]);
            // the spectra of this parity PF layers ahead into L2 (pair 0's thread)
            if (p == 0 && n + PF < nz) bulk_prefetch_l2(Sq + (size_t)(n + PF) * S_ROW, L.s_bytes);
            if (++sf == L.df) {
                sf = 0;
                ++wrap;
            }
            if (n + 1 < nz) {
                const float* row = Sq + (size_t)(n + 1) * S_ROW;
#pragma unroll
                for (int c = 0; c < NC; ++c) sv[c] = __ldg(row + c * JP);
            }
            if ((n % W5Shape::BLOCK) == W5Shape::BLOCK - 1 || n == nz - 1) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float* aj = accs + (c * 4 + j) * J + q;
                        float* cj = cmp + (c * 4 + j) * J + q;
                        float sum = *aj, cc = *cj;
                        kahan_add(sum, cc, part[c][j]);
                        *aj = sum;
                        *cj = cc;
                        part[c][j] = 0.f;
                    }
            }
        }
        if (cta_sync_or(failed || *abort)) {
            if (tid == 0) atomicExch(err, 1);
            return;
        }
        // the compensated sums (times i for imaginary spectra, with the
        // mirror sign for odd components) into F slot c, natural order
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float e[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) e[j] = accs[(c * 4 + j) * J + q] - cmp[(c * 4 + j) * J + q];
            const bool imag = (a.imag_mask >> c) & 1u;
            const bool flip = !nyq && ((a.oddv_mask >> c) & 1u);
            C b1 = make_float2(e[0], e[1]), b2 = make_float2(e[2], e[3]);
            if (flip) b2 = make_float2(-b2.x, -b2.y);
            if (imag) {
                b1 = make_float2(-b1.y, b1.x);
                b2 = make_float2(-b2.y, b2.x);
            }
            C* fb = fring + c * FS;
            fb[k1] = b1;
            fb[k2] = b2;
        }
        cta_sync();
    }
}

// Shared-memory layout; df == 0 when it does not fit.
W5Smem wf512_smem(int ny_pad, int ncomp, int jp, int max_bytes) {
    W5Smem L{};
    L.x_bytes = (uint32_t)(ny_pad * sizeof(float2));
    L.s_bytes = (uint32_t)(ncomp * jp * sizeof(float));
    L.f_bytes = (uint32_t)(W5Shape::FSLOT * sizeof(float2));
    if (ny_pad > W5Shape::N || ny_pad < 1 || ncomp > 7 || jp != W5Shape::JP || (L.x_bytes & 15u) ||
        (L.s_bytes & 15u))
        return W5Smem{};
    for (int df = 12; df >= W5Shape::FWARPS + 1; --df) {
        W5Smem l = L;
        l.df = df;
        l.f_off = (uint32_t)(W5Shape::DX * L.x_bytes + 127) & ~127u;
        l.t2_off = l.f_off + df * L.f_bytes;
        l.cmp_off = l.t2_off + 2 * W5Shape::N * sizeof(float2);
        l.acc_off = l.cmp_off + 4 * ncomp * W5Shape::J * sizeof(float);
        l.bar_off = l.acc_off + 4 * ncomp * W5Shape::J * sizeof(float);
        l.flag_off = l.bar_off + (W5Shape::DX + 2 * df) * 8;
        l.total = l.flag_off + 16;
        if ((int)l.total <= max_bytes) return l;
    }
    return W5Smem{};
}

template <int NC>
cudaError_t launch_nc(const ColumnArgs& a, const W5Smem& L, const void* X, const float* spec, void* Y, const void* tw,
                      int* err, cudaStream_t s, Batch b) {
    constexpr auto k = forward_column_wf512_kernel<NC>;
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    k<<<dim3(a.kx_count, b.count), W5Shape::NT, L.total, s>>>(a, L, (const float2*)X, spec, (float2*)Y,
                                                              (const float2*)tw, err, b.in, b.out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_forward_wf512(const ColumnArgs& a, const void* X, const float* spec, void* Y, const void* tw,
                                 int* err, cudaStream_t s, Batch b) {
    const W5Smem L = wf512_smem(a.ny_pad, a.ncomp, a.jp, kMaxSmemOptin);
    if (L.df == 0 || !err) return cudaErrorNotSupported;
    switch (a.ncomp) {
        case 1: return launch_nc<1>(a, L, X, spec, Y, tw, err, s, b);
        case 2: return launch_nc<2>(a, L, X, spec, Y, tw, err, s, b);
        case 3: return launch_nc<3>(a, L, X, spec, Y, tw, err, s, b);
        case 4: return launch_nc<4>(a, L, X, spec, Y, tw, err, s, b);
        case 5: return launch_nc<5>(a, L, X, spec, Y, tw, err, s, b);
        case 6: return launch_nc<6>(a, L, X, spec, Y, tw, err, s, b);
        case 7: return launch_nc<7>(a, L, X, spec, Y, tw, err, s, b);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace grav
