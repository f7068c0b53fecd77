// Forward column stage for 1024-point FP32 column transforms (Py = 2048)
// with one warp per layer transform.
//
// 24 warps at 80 registers a thread (the whole register file: 768 x 80, six
// warps per SM sub-partition).  Warps 0-15 accumulate: thread q owns mirror
// pair q for every component (the layer sum of Eq. 20 in the Fourier
// domain).  Warps 16-23 transform: each layer's 1024-point FFT is done by a
// single warp in registers, 32 values a lane, as 1024 = 32 x 32 (the
// four-step form):
//   x[32 n1 + n2] -> 32-point DFTs over n1 (lane n2) -> twiddle W_1024^(n2 k1)
//   -> transpose through shared memory -> 32-point DFTs over n2 (lane k1).
// A warp transform needs no block or group barrier, so eight layers are in
// flight at once and the transform costs about a third of the instructions
// of a shared-memory radix-8 transform by a thread group.
//
// Data movement: FFT warp f handles layers f, f + 8, ...; X slot f is its
// own, so after reading layer n it refills the slot with layer n + 8 itself
// (bulk copy) and prefetches a later layer's spectra into L2.  The
// accumulate threads read their spectra values from global memory one layer
// ahead, in registers.  The spectra value of the Nyquist row (one per
// component, used by one thread of the even-ky CTA) rides in the spare tail
// of the layer's F slot.  Every wait is bounded.
//
// The odd-ky CTA transforms the folded column x[m] W_Py^m (Py = 2N).  With
// m = 32 n1 + n2 the fold factor is W_64^n1 W_2048^n2: the first factor is a
// constant of register n1, the second is constant over n1 and so moves past
// the first 32-point pass into the transpose twiddles, t2 = W_2048^((2 k1 +
// r) n2).  The inverse transform cancels the extra W_2048^-n2 that these
// twiddles carry by scaling its input by W_2048^n2 first, and unfolds its
// output y = n2 + 32 k by W_2048^-n2 W_64^-k.
#pragma once
#include "async_copy.cuh"
#include "fft_block.cuh"
#include "grav_internal.h"
#include "spectral.cuh"
#include "spectral_ws.cuh"
#include "warp_fft.cuh"

namespace grav {

struct WfShape {
    static constexpr int N = 1024;
    static constexpr int J = 512;          // accumulate threads (16 warps)
    static constexpr int FWARPS = 8;       // FFT warps (2 warpgroups)
    static constexpr int NT = J + 32 * FWARPS;
    static constexpr int FSLOT = kWarpFftSlot;  // complex values per F slot (transpose area)
    static constexpr int REGS = 80;        // registers a thread: NT x REGS = 61440
    static constexpr int DX = FWARPS;      // one X slot per FFT warp
    static constexpr int PF = 8;           // spectra prefetch distance (layers)
    static constexpr int JP = 516;         // spectra row pitch: J + 1 rounded up to 4
    static constexpr int BLOCK = 32;       // layers per compensated block
};

struct WfSmem {
    int df;
    uint32_t x_bytes, s_bytes, f_bytes;
    uint32_t f_off, t2_off, cmp_off, bar_off, flag_off, total;
};

template <int NC>
__global__ void __maxnreg__(WfShape::REGS)
    forward_column_wf_kernel(ColumnArgs a, WfSmem L, const float2* __restrict__ X, const float* __restrict__ spec,
                             float2* __restrict__ Y, const float2* __restrict__ tw, int* __restrict__ err,
                             size_t x_bstride, size_t y_bstride) {
    using C = float2;
    constexpr int N = WfShape::N, J = WfShape::J, FW = WfShape::FWARPS, NT = WfShape::NT;
    constexpr int FS = WfShape::FSLOT, DX = WfShape::DX, PF = WfShape::PF, JP = WfShape::JP;
    constexpr int S_ROW = NC * JP;  // floats per layer of spectra
    static_assert(NC <= FW, "one inverse transform per FFT warp");
    static_assert(NC <= FS - N, "Nyquist spectra values fit in the F slot tail");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* xring = smem;
    C* fring = reinterpret_cast<C*>(smem + L.f_off);
    C* t2 = reinterpret_cast<C*>(smem + L.t2_off);  // W_2048^((2 k1 + r) n2) at [k1][n2]
    float* cmp = reinterpret_cast<float*>(smem + L.cmp_off);  // Kahan corrections [c][j][q]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* xfull = bars;
    uint64_t* ffull = xfull + DX;
    uint64_t* fempty = ffull + L.df;
    volatile int* abort = reinterpret_cast<volatile int*>(smem + L.flag_off);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = blockIdx.x & 1, kx = blockIdx.x >> 1;
    const int nz = a.nz, ny = a.ny;
    X += blockIdx.y * x_bstride;  // request of a batched call
    Y += blockIdx.y * y_bstride;
    const C* Xk = X + (size_t)kx * nz * a.ny_pad;
    const float* Sk = request_spec(a, spec, blockIdx.y) + (size_t)(r * a.kx_count + kx) * nz * S_ROW;

    if (tid == 0) {
        for (int s = 0; s < DX; ++s) mbar_init(&xfull[s], 1);
        for (int s = 0; s < L.df; ++s) {
            mbar_init(&ffull[s], 32);
            mbar_init(&fempty[s], J);
        }
        *abort = 0;
        fence_mbar_init();
    }
    for (int e = tid; e < N; e += NT) {
        const int k1 = e >> 5, n2 = e & 31;
        t2[e] = tw[(((2 * k1 + r) * n2) & (2 * N - 1)) << a.tw_shift_p];
    }
    for (int e = tid; e < 4 * NC * J; e += NT) cmp[e] = 0.f;
    __syncthreads();
    if (tid == 0) {
        // first layer of every X slot, and the first PF layers' spectra into L2
        for (int n = 0; n < DX && n < nz; ++n) {
            mbar_arrive_expect_tx(&xfull[n], L.x_bytes);
            bulk_g2s(xring + (size_t)n * L.x_bytes, Xk + (size_t)n * a.ny_pad, L.x_bytes, &xfull[n]);
        }
        for (int n = 0; n < PF && n < nz; ++n) bulk_prefetch_l2(Sk + (size_t)n * S_ROW, L.s_bytes);
    }

    bool failed = false;
    const bool is_mac = tid < J;
    const bool nyq = is_mac && r == 0 && tid == 0;

    if (!is_mac) {
        // ---------------- FFT warp f: layers f, f + FW, ... ----------------
        const int f = warp - (J >> 5);
        unsigned char* xslot = xring + (size_t)f * L.x_bytes;
        const C* xs = reinterpret_cast<const C*>(xslot);
        int pending = f < nz ? f : -1;  // layer of the copy in flight into X slot f
        // Nyquist-row spectra value of component `lane` (even-ky CTA), loaded
        // one iteration ahead so that its latency is never waited on
        const bool has_nyq = r == 0 && lane < NC;
        float snyq_next = (has_nyq && f < nz) ? __ldg(Sk + (size_t)f * S_ROW + lane * JP + J) : 0.f;
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
            if (has_nyq && n + FW < nz) snyq_next = __ldg(Sk + (size_t)(n + FW) * S_ROW + lane * JP + J);
            float2 u[32];
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) {
                const int m = 32 * n1 + lane;
                C v = make_float2(0.f, 0.f);
                if (m < ny) v = xs[m];
                u[n1] = v;
            }
            __syncwarp();  // every lane's reads of X slot f are done
            if (lane == 0) {
                if (n + FW < nz) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&xfull[f], L.x_bytes);
                    bulk_g2s(xslot, Xk + (size_t)(n + FW) * a.ny_pad, L.x_bytes, &xfull[f]);
                    pending = n + FW;
                }
                if (n + PF < nz) bulk_prefetch_l2(Sk + (size_t)(n + PF) * S_ROW, L.s_bytes);
            }
            if (r) {
#pragma unroll
                for (int n1 = 0; n1 < 32; ++n1) u[n1] = tw64(u[n1], n1);  // fold factor W_64^n1
            }
            C* fb = fring + sf * FS;
            warp_fft1024<false, false>(u, fb, t2, lane);  // scalar butterflies: 80 registers
#pragma unroll
            for (int j = 0; j < 32; ++j) fb[lane + 32 * bitrev5(j)] = u[j];
            if (lane < NC) fb[N + lane] = make_float2(snyq, 0.f);
            mbar_arrive(&ffull[sf]);  // this lane's writes of the F slot are done
        }
        if (lane == 0 && pending >= 0) {
            // a copy that will not be consumed (failure path): let it land
            // (bounded) before the CTA's shared memory is released
            mbar_wait_bounded(&xfull[f], (uint32_t)((pending / DX) & 1), kWaitLimitNs);
        }
        if (cta_sync_or(failed || *abort)) return;
        cta_sync();  // the accumulate threads have written the sums
        // inverse column transform of component f (F slot f)
        const int c = f;
        if (c < NC) {
            C* fb = fring + c * FS;
            float2 u[32];
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) u[n1] = fb[32 * n1 + lane];
            __syncwarp();
            if (r) {
                const C w = __ldg(tw + (lane << a.tw_shift_p));  // W_2048^n2, n2 = lane
#pragma unroll
                for (int n1 = 0; n1 < 32; ++n1) u[n1] = cmul(u[n1], w);
            }
            warp_fft1024<true, false>(u, fb, t2, lane);
            C* dst = Y + ((size_t)(r * a.kx_count + kx) * a.ncomp + c) * a.ny_pad;
            if (r) {
                // unfold: W_2048^-y with y = lane + 32 k is W_2048^-lane W_64^-k
                const C w = cconj(__ldg(tw + (lane << a.tw_shift_p)));
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int y = lane + 32 * bitrev5(j);
                    if (y < ny) dst[y] = tw64(cmul(u[j], w), 64 - bitrev5(j));
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int y = lane + 32 * bitrev5(j);
                    if (y < ny) dst[y] = u[j];
                }
            }
        }
    } else {
        // ---------------- accumulate: thread q owns mirror pair q ----------------
        const int q = tid;
        int k1 = 0, k2 = 0;
        pair_pos<N>(q, r, k1, k2);
        float acc[NC][4];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[c][j] = 0.f;
        float part[NC][4];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[c][j] = 0.f;
        // this thread's spectra values Sk[n][c][q], loaded one layer ahead
        const float* Sq = Sk + q;
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
                const float s2 = nyq ? fb[N + c].x : sv[c];
                part[c][0] += sv[c] * v1.x;
                part[c][1] += sv[c] * v1.y;
                part[c][2] += s2 * v2.x;
                part[c][3] += s2 * v2.y;
            }
            mbar_arrive(&fempty[sf]);
            if (++sf == L.df) {
                sf = 0;
                ++wrap;
            }
            if (n + 1 < nz) {
                const float* row = Sq + (size_t)(n + 1) * S_ROW;
#pragma unroll
                for (int c = 0; c < NC; ++c) sv[c] = __ldg(row + c * JP);
            }
            if ((n % WfShape::BLOCK) == WfShape::BLOCK - 1 || n == nz - 1) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float* cj = cmp + (c * 4 + j) * J + q;
                        float cc = *cj;
                        kahan_add(acc[c][j], cc, part[c][j]);
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
            for (int j = 0; j < 4; ++j) e[j] = acc[c][j] - cmp[(c * 4 + j) * J + q];
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

// Shared-memory layout; df == 0 when it does not fit.  The F ring holds
// one slot per FFT warp plus the accumulate threads' lag.
inline WfSmem wf_smem(int ny_pad, int ncomp, int jp, int nc_inst, int max_bytes) {
    WfSmem L{};
    L.x_bytes = (uint32_t)(ny_pad * sizeof(float2));
    L.s_bytes = (uint32_t)(ncomp * jp * sizeof(float));
    L.f_bytes = (uint32_t)(WfShape::FSLOT * sizeof(float2));
    if (ny_pad > WfShape::N || nc_inst > WfShape::FWARPS || ncomp != nc_inst || jp != WfShape::JP ||
        (L.x_bytes & 15u) || (L.s_bytes & 15u))
        return WfSmem{};
    for (int df = 12; df >= WfShape::FWARPS + 1; --df) {
        WfSmem l = L;
        l.df = df;
        l.f_off = (uint32_t)(WfShape::DX * L.x_bytes + 127) & ~127u;
        l.t2_off = l.f_off + df * L.f_bytes;
        l.cmp_off = l.t2_off + WfShape::N * sizeof(float2);
        l.bar_off = l.cmp_off + 4 * nc_inst * WfShape::J * sizeof(float);
        l.flag_off = l.bar_off + (WfShape::DX + 2 * df) * 8;
        l.total = l.flag_off + 16;
        if ((int)l.total <= max_bytes) return l;
    }
    return WfSmem{};
}

}  // namespace grav
