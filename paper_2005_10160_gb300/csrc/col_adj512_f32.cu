// Adjoint column stage for 512-point FP32 column transforms (Py = 1024,
// 257 <= ny <= 512), the transpose of Eq. 21 on one kx column:
//   Z_n = IFFT_y( sum_c conj(S_c,n) . FFT_y(R_c) )   for every layer n,
// with both ky parities in one CTA and every warp transform doing the two
// parities at once (warp_fft512x2).
//
// The layout is that of the 1024-point adjoint kernel (spectral_adj_wf.cuh):
// 24 warps at 80 registers.  Warps 16-23 first transform the residual
// columns (component c in warp c, both parities) into slots 0 .. NC-1; thread
// q of warps 0-15 keeps both bins of mirror pair q % 256 of parity q / 256
// for every component in registers.  Then, layer by layer, the combine
// threads form the layer's spectrum from their bins and the layer's spectra
// values (read one layer ahead, after an L2 prefetch eight layers ahead) and
// write it into a ring slot (parity r at offset 512 r); FFT warp f
// inverse-transforms layers f, f + 8, ... from the slot and writes rows
// y < ny of both parities.  Every wait is bounded.
//
// Parity 1 is the folded column, x[m] W_1024^m.  As in the forward kernel the
// fold rides in the transpose twiddles t2 = W_1024^(n2 (2 k1 + r)) and in
// compile-time constants: the forward residual transform multiplies
// register n1 by W_32^n1; the inverse layer transform unfolds its output
// y = k1 + 16 k2 by W_1024^-k1 W_64^-k2.  Its input must be scaled by
// W_1024^(k mod 32) (bin k of parity 1) to cancel the extra factor of the
// conjugate twiddles; as a layer's spectrum is complex-linear in the
// residual bins, the combine threads scale their parity-1 bins once instead.
#include "async_copy.cuh"
#include "grav_internal.h"
#include "spectral.cuh"
#include "spectral_ws.cuh"
#include "warp_fft.cuh"

namespace grav {

namespace {

struct A5Shape {
    static constexpr int N = 512;     // transform length (per parity)
    static constexpr int NB = 2 * N;  // bins per slot (both parities)
    static constexpr int JH = N / 2;  // mirror pairs per parity
    static constexpr int J = 2 * JH;  // combine threads (16 warps)
    static constexpr int FWARPS = 8;  // FFT warps
    static constexpr int NT = J + 32 * FWARPS;
    static constexpr int SLOT = kWarpFftSlot;
    static constexpr int REGS = 80;
    static constexpr int JP = 260;    // spectra row pitch: JH + 1 rounded up to 4
    static constexpr int PF = 8;      // spectra prefetch distance into L2 (layers)
};

struct A5Smem {
    int dz;
    uint32_t slot_off, t2_off, bar_off, flag_off, total;
};

template <int NC>
__global__ void __maxnreg__(A5Shape::REGS)
    adjoint_column_wf512_kernel(ColumnArgs a, A5Smem L, const float2* __restrict__ Xr, const float* __restrict__ spec,
                                float2* __restrict__ Z, const float2* __restrict__ tw, int* __restrict__ err,
                                size_t x_bstride, size_t z_bstride) {
    using C = float2;
    constexpr int N = A5Shape::N, JH = A5Shape::JH, J = A5Shape::J, FW = A5Shape::FWARPS, NT = A5Shape::NT;
    constexpr int FS = A5Shape::SLOT, JP = A5Shape::JP, S_ROW = NC * JP, PF = A5Shape::PF;
    static_assert(NC <= FW, "one residual transform pair per FFT warp");
    extern __shared__ __align__(128) unsigned char smem[];
    C* ring = reinterpret_cast<C*>(smem + L.slot_off);
    C* t2 = reinterpret_cast<C*>(smem + L.t2_off);  // W_1024^(n2 (2 k1 + r)) at [16 r + k1][n2]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* zfull = bars;
    uint64_t* zempty = zfull + L.dz;
    volatile int* abort = reinterpret_cast<volatile int*>(smem + L.flag_off);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kx = blockIdx.x;
    const int nz = a.nz, ny = a.ny;
    Xr += blockIdx.y * x_bstride;  // request of a batched call
    Z += blockIdx.y * z_bstride;
    const float* specb = request_spec(a, spec, blockIdx.y);
    const float* Sk0 = specb + (size_t)kx * nz * S_ROW;                 // parity 0
    const float* Sk1 = specb + (size_t)(a.kx_count + kx) * nz * S_ROW;  // parity 1

    if (tid == 0) {
        for (int s = 0; s < L.dz; ++s) {
            mbar_init(&zfull[s], J);
            mbar_init(&zempty[s], 32);
        }
        *abort = 0;
        fence_mbar_init();
    }
    for (int e = tid; e < 2 * N; e += NT) {
        const int K = e >> 5, n2 = e & 31, h = K >> 4, k1 = K & 15;
        t2[e] = tw[((n2 * (2 * k1 + h)) & (2 * N - 1)) << a.tw_shift_p];
    }
    __syncthreads();

    // FFT_y of every component's residual column, both parities, into slots 0 .. NC-1
    if (warp >= J / 32 && warp - J / 32 < NC) {
        const int c = warp - J / 32;
        const C* col = Xr + ((size_t)kx * a.ncomp + c) * a.ny_pad;
        float2 u[32];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            const int m = 32 * n1 + lane;
            const C v = m < ny ? col[m] : make_float2(0.f, 0.f);
            u[n1] = v;
            u[16 + n1] = tw32<false>(v, n1);  // parity 1: fold factor W_32^n1
        }
        C* fb = ring + c * FS;
        warp_fft512x2<false, false>(u, fb, t2, lane);  // scalar butterflies: register cap
        const int base = (lane >> 4) * N + (lane & 15);
#pragma unroll
        for (int j = 0; j < 32; ++j) fb[base + 16 * bitrev5(j)] = u[j];
    }
    __syncthreads();

    bool failed = false;
    if (tid < J) {
        // ---------------- combine: thread q owns parity q / 256, pair q % 256 ----------------
        const int q = tid, rq = q / JH, p = q % JH;
        int k1, k2;
        pair_pos<N>(p, rq, k1, k2);
        k1 += rq * N;
        k2 += rq * N;
        const bool nyq = q == 0;  // second bin is the Nyquist row, with spectra values of its own
        C rc[NC][2];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            rc[c][0] = ring[c * FS + k1];
            rc[c][1] = ring[c * FS + k2];
        }
        if (rq) {
            // W_1024^(k mod 32) for the inverse layer transforms (see above)
            const C w1 = __ldg(tw + ((k1 & 31) << a.tw_shift_p)), w2 = __ldg(tw + ((k2 & 31) << a.tw_shift_p));
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                rc[c][0] = cmul(rc[c][0], w1);
                rc[c][1] = cmul(rc[c][1], w2);
            }
        }
        const unsigned imag = a.imag_mask, oddv = a.oddv_mask;
        cta_sync();  // every combine thread has its bins: the slots become the ring
        const float* Sq = (rq ? Sk1 : Sk0) + p;
        float sv[NC], se[NC];
        auto load = [&](int n) {
            const float* row = Sq + (size_t)n * S_ROW;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                sv[c] = __ldg(row + c * JP);
                se[c] = nyq ? __ldg(row + c * JP + JH) : 0.f;
            }
        };
        // spectra of the first PF layers into L2 (pair 0 of each parity),
        // then one layer more each iteration
        if (p == 0)
            for (int n = 0; n < PF && n < nz; ++n) bulk_prefetch_l2(Sq + (size_t)n * S_ROW, S_ROW * sizeof(float));
        if (nz > 0) load(0);
        int sz = 0, wrap = 0;  // ring slot of layer n (n % dz) and n / dz, stepped with n
        for (int n = 0; n < nz; ++n) {
            if (p == 0 && n + PF < nz) bulk_prefetch_l2(Sq + (size_t)(n + PF) * S_ROW, S_ROW * sizeof(float));
            if (n >= L.dz && !ws_wait(&zempty[sz], (uint32_t)((wrap - 1) & 1), abort)) {
                failed = true;
                break;
            }
            C z1 = make_float2(0.f, 0.f), z2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float s1 = sv[c];
                const float s2 = nyq ? se[c] : (((oddv >> c) & 1u) ? -s1 : s1);
                const C v1 = rc[c][0], v2 = rc[c][1];
                // conj(S) v with S = s (real spectrum) or i s (imaginary spectrum)
                if ((imag >> c) & 1u) {
                    z1.x += s1 * v1.y;
                    z1.y -= s1 * v1.x;
                    z2.x += s2 * v2.y;
                    z2.y -= s2 * v2.x;
                } else {
                    z1.x += s1 * v1.x;
                    z1.y += s1 * v1.y;
                    z2.x += s2 * v2.x;
                    z2.y += s2 * v2.y;
                }
            }
            if (n + 1 < nz) load(n + 1);
            C* zb = ring + sz * FS;
            zb[k1] = z1;
            zb[k2] = z2;
            mbar_arrive(&zfull[sz]);
            if (++sz == L.dz) {
                sz = 0;
                ++wrap;
            }
        }
        if (cta_sync_or(failed || *abort)) {
            if (tid == 0) atomicExch(err, 1);
        }
    } else {
        // ---------------- FFT warp f: inverse transforms of layers f, f + 8, ... ----------------
        const int f = warp - J / 32;
        const int h = lane >> 4, k1 = lane & 15;  // output parity and low index of this lane
        cta_sync();
        for (int n = f; n < nz; n += FW) {
            const int sz = n % L.dz;
            int ok = 1;
            if (lane == 0) ok = ws_wait(&zfull[sz], (uint32_t)((n / L.dz) & 1), abort);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                failed = true;
                break;
            }
            C* zb = ring + sz * FS;
            float2 u[32];
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1) {
                u[n1] = zb[32 * n1 + lane];
                u[16 + n1] = zb[N + 32 * n1 + lane];
            }
            __syncwarp();
            warp_fft512x2<true, false>(u, zb, t2, lane);
            mbar_arrive(&zempty[sz]);  // this lane is done with the slot (transposes included)
            C* dst = Z + ((size_t)(h * a.kx_count + kx) * nz + n) * a.ny_pad;
            if (h) {
                const C wu = cconj(__ldg(tw + (k1 << a.tw_shift_p)));  // W_1024^-k1
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int y = k1 + 16 * bitrev5(j);
                    if (y < ny) dst[y] = tw64(cmul(u[j], wu), 64 - bitrev5(j));
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int y = k1 + 16 * bitrev5(j);
                    if (y < ny) dst[y] = u[j];
                }
            }
        }
        cta_sync_or(failed || *abort);
    }
}

// Ring depth and offsets; dz == 0 when the kernel does not apply.
A5Smem aw512_smem(int ny_pad, int ncomp, int jp, int max_bytes) {
    if (ny_pad > A5Shape::N || ny_pad < 1 || ncomp > A5Shape::FWARPS || ncomp < 1 || jp != A5Shape::JP)
        return A5Smem{};
    for (int dz = 16; dz >= A5Shape::FWARPS + 2; --dz) {
        A5Smem l{};
        l.dz = dz;
        l.slot_off = 0;
        l.t2_off = (uint32_t)(dz * A5Shape::SLOT * sizeof(float2));
        l.bar_off = l.t2_off + 2 * A5Shape::N * sizeof(float2);
        l.flag_off = l.bar_off + 2 * dz * 8;
        l.total = l.flag_off + 16;
        if ((int)l.total <= max_bytes) return l;
    }
    return A5Smem{};
}

template <int NC>
cudaError_t launch_nc(const ColumnArgs& a, const A5Smem& L, const void* Xr, const float* spec, void* Z,
                      const void* tw, int* err, cudaStream_t s, Batch b) {
    constexpr auto k = adjoint_column_wf512_kernel<NC>;
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    k<<<dim3(a.kx_count, b.count), A5Shape::NT, L.total, s>>>(a, L, (const float2*)Xr, spec, (float2*)Z,
                                                              (const float2*)tw, err, b.in, b.out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_wf512(const ColumnArgs& a, const void* Xr, const float* spec, void* Z, const void* tw,
                                 int* err, cudaStream_t s, Batch b) {
    const A5Smem L = aw512_smem(a.ny_pad, a.ncomp, a.jp, kMaxSmemOptin);
    if (L.dz == 0 || !err || a.z_tiled) return cudaErrorNotSupported;
    switch (a.ncomp) {
        case 1: return launch_nc<1>(a, L, Xr, spec, Z, tw, err, s, b);
        case 2: return launch_nc<2>(a, L, Xr, spec, Z, tw, err, s, b);
        case 3: return launch_nc<3>(a, L, Xr, spec, Z, tw, err, s, b);
        case 4: return launch_nc<4>(a, L, Xr, spec, Z, tw, err, s, b);
        case 5: return launch_nc<5>(a, L, Xr, spec, Z, tw, err, s, b);
        case 6: return launch_nc<6>(a, L, Xr, spec, Z, tw, err, s, b);
        case 7: return launch_nc<7>(a, L, Xr, spec, Z, tw, err, s, b);
        case 8: return launch_nc<8>(a, L, Xr, spec, Z, tw, err, s, b);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace grav
