// Adjoint column stage for 1024-point FP32 column transforms (Py = 2048),
// the transpose of Eq. 21: for every layer n,
//   Z_n = IFFT_y( sum_c conj(S_c,n) . FFT_y(R_c) )
// on one kx column and one ky parity (the same parity split as the forward).
//
// 24 warps at 80 registers a thread.  Warps 16-23 first transform the
// residual's row-transform columns (component f in warp f), one warp each,
// in registers (warp_fft1024); thread q of warps 0-15 keeps both bins of
// mirror pair q of every component in registers.  Then, layer by layer, the
// combine threads form the layer's spectrum from their bins and the layer's
// spectra values (read from global memory one layer ahead, after a bulk L2
// prefetch eight layers ahead: the combine threads run ahead of the
// transforms, so a load from DRAM would stall every layer) and write it
// into a ring slot; FFT warp f inverse-transforms layers f, f + 8, ... from
// the slot (which is also its transpose area) and writes the rows y < ny.
// The combine threads run up to (ring depth - 8) layers ahead of the
// transforms.  Every wait is bounded.
#pragma once
#include "async_copy.cuh"
#include "grav_internal.h"
#include "spectral.cuh"
#include "spectral_ws.cuh"
#include "warp_fft.cuh"

namespace grav {

struct AwShape {
    static constexpr int N = 1024;
    static constexpr int J = 512;     // combine threads (16 warps), one mirror pair each
    static constexpr int FWARPS = 8;  // FFT warps
    static constexpr int NT = J + 32 * FWARPS;
    static constexpr int SLOT = kWarpFftSlot;
    static constexpr int REGS = 80;
    static constexpr int JP = 516;    // spectra row pitch: J + 1 rounded up to 4
    static constexpr int PF = 8;      // spectra prefetch distance into L2 (layers)
};

struct AwSmem {
    int dz;
    uint32_t slot_off, tw_off, t2_off, stage_off, bar_off, flag_off, total;
};

// IM, OV: the plan's imaginary-spectrum and odd-in-y component masks when
// known at compile time (the all-six-components request), else kRuntimeMask.
constexpr unsigned kRuntimeMask = ~0u;

template <int NC, unsigned IM = kRuntimeMask, unsigned OV = kRuntimeMask>
__global__ void __maxnreg__(AwShape::REGS)
    adjoint_column_wf_kernel(ColumnArgs a, AwSmem L, const float2* __restrict__ Xr, const float* __restrict__ spec,
                             float2* __restrict__ Z, const float2* __restrict__ tw, int* __restrict__ err,
                             size_t x_bstride, size_t z_bstride, const __grid_constant__ CUtensorMap zmap) {
    using C = float2;
    constexpr int N = AwShape::N, J = AwShape::J, FW = AwShape::FWARPS, NT = AwShape::NT;
    constexpr int FS = AwShape::SLOT, JP = AwShape::JP, S_ROW = NC * JP;
    static_assert(NC <= FW, "one residual transform per FFT warp");
    extern __shared__ __align__(128) unsigned char smem[];
    C* ring = reinterpret_cast<C*>(smem + L.slot_off);
    C* tws = reinterpret_cast<C*>(smem + L.tw_off);  // fold twiddles W_Py^m, m < N
    C* t2 = reinterpret_cast<C*>(smem + L.t2_off);   // W_1024^(n2 k1) at [k1][n2]
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* zfull = bars;
    uint64_t* zempty = zfull + L.dz;
    volatile int* abort = reinterpret_cast<volatile int*>(smem + L.flag_off);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = blockIdx.x & 1, kx = blockIdx.x >> 1;
    const int nz = a.nz, ny = a.ny;
    Xr += blockIdx.y * x_bstride;  // request of a batched call
    Z += blockIdx.y * z_bstride;
    const float* Sk = request_spec(a, spec, blockIdx.y) + (size_t)(r * a.kx_count + kx) * nz * S_ROW;

    if (tid == 0) {
        for (int s = 0; s < L.dz; ++s) {
            mbar_init(&zfull[s], J);
            mbar_init(&zempty[s], 32);
        }
        *abort = 0;
        fence_mbar_init();
    }
    for (int e = tid; e < N; e += NT) {
        tws[e] = tw[e << a.tw_shift_p];
        const int k1 = e >> 5, n2 = e & 31;
        t2[e] = tw[((k1 * n2) & (N - 1)) << a.tw_shift_n];
    }
    __syncthreads();

    // FFT_y of every component's residual column, into slots 0 .. NC-1
    if (warp >= J / 32 && warp - J / 32 < NC) {
        const int c = warp - J / 32;
        const C* col = Xr + ((size_t)kx * a.ncomp + c) * a.ny_pad;
        float2 u[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) {
            const int m = 32 * n1 + lane;
            C v = make_float2(0.f, 0.f);
            if (m < ny) {
                v = col[m];
                if (r) v = cmul(v, tws[m]);  // fold for ky parity r
            }
            u[n1] = v;
        }
        C* fb = ring + c * FS;
        warp_fft1024<false>(u, fb, t2, lane);
#pragma unroll
        for (int j = 0; j < 32; ++j) fb[lane + 32 * bitrev5(j)] = u[j];
    }
    __syncthreads();

    bool failed = false;
    if (tid < J) {
        // ---------------- combine: thread q owns mirror pair q ----------------
        const int q = tid;
        int k1, k2;
        pair_pos<N>(q, r, k1, k2);
        const bool nyq = r == 0 && q == 0;  // second bin is the Nyquist row, with spectra values of its own
        C rc[NC][2];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            rc[c][0] = ring[c * FS + k1];
            rc[c][1] = ring[c * FS + k2];
        }
        const unsigned imag = IM == kRuntimeMask ? a.imag_mask : IM;
        const unsigned oddv = OV == kRuntimeMask ? a.oddv_mask : OV;
        cta_sync();  // every combine thread has its bins: the slots become the ring
        const float* Sq = Sk + q;
        float sv[NC], se[NC];
        auto load = [&](int n) {
            const float* row = Sq + (size_t)n * S_ROW;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                sv[c] = __ldg(row + c * JP);
                se[c] = nyq ? __ldg(row + c * JP + (J - q)) : 0.f;
            }
        };
        // spectra of the first PF layers into L2 (thread 0), then one layer
        // more each iteration, so that the one-layer-ahead loads hit L2
        constexpr int PF = AwShape::PF;
        if (q == 0)
            for (int n = 0; n < PF && n < nz; ++n) bulk_prefetch_l2(Sk + (size_t)n * S_ROW, S_ROW * sizeof(float));
        if (nz > 0) load(0);
        int sz = 0, wrap = 0;  // ring slot of layer n (n % dz) and n / dz, stepped with n
        for (int n = 0; n < nz; ++n) {
            if (q == 0 && n + PF < nz) bulk_prefetch_l2(Sk + (size_t)(n + PF) * S_ROW, S_ROW * sizeof(float));
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
        cta_sync();
        // ring slot of layer n (n % dz) and the parity of n / dz, stepped with
        // n (n advances by FW < dz)
        int sz = f, wrap = 0;
        for (int n = f; n < nz; n += FW) {
            int ok = 1;
            if (lane == 0) ok = ws_wait(&zfull[sz], (uint32_t)(wrap & 1), abort);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                failed = true;
                break;
            }
            C* zb = ring + sz * FS;
            float2 u[32];
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) u[n1] = zb[32 * n1 + lane];
            __syncwarp();
            warp_fft1024<true>(u, zb, t2, lane);
            if (a.z_tiled) {
                // The slot was only the transform's transpose area: free it now.  Stage the
                // layer in this warp's own buffer in the order of its tiles, Z[.][.][y / 8][kx][8]
                // with row pair (y % 8) / 2 at 16-byte position ((y % 8) / 2 + kx / 2) % 4,
                // and write it with one tensor store (zmap: 8 x kx x y/8 x (r, n) x request)
                // that is not waited for: the next layer waits, before it restages, until
                // this store has read the buffer.
                mbar_arrive(&zempty[sz]);
                C* stg = reinterpret_cast<C*>(smem + L.stage_off) + f * N;
                if (lane == 0) bulk_wait_read_all();  // the previous layer's store has read the buffer
                __syncwarp();
                const int pos = 2 * ((((lane & 7) >> 1) + (kx >> 1)) & 3) + (lane & 1);  // y % 8 = lane % 8
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int y = lane + 32 * bitrev5(j);
                    C v = u[j];
                    if (r) v = cmul(v, cconj(tws[y]));
                    stg[(y & ~7) + pos] = v;
                }
                fence_proxy_async_smem();  // these writes before the tensor store's reads
                __syncwarp();
                if (lane == 0) {
                    tma_store_5d(&zmap, stg, 0, kx, 0, r * nz + n, blockIdx.y);
                    bulk_commit();
                }
            } else {
                mbar_arrive(&zempty[sz]);  // this lane is done with the slot (transposes included)
                C* dst = Z + ((size_t)(r * a.kx_count + kx) * nz + n) * a.ny_pad;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int y = lane + 32 * bitrev5(j);
                    if (y < ny) {
                        C v = u[j];
                        if (r) v = cmul(v, cconj(tws[y]));
                        dst[y] = v;
                    }
                }
            }
            sz += FW;
            if (sz >= L.dz) {
                sz -= L.dz;
                ++wrap;
            }
        }
        if (a.z_tiled && lane == 0) bulk_wait_all();  // every tensor store has landed
        cta_sync_or(failed || *abort);
    }
}

// Ring depth and offsets; dz == 0 when the kernel does not apply.
inline AwSmem aw_smem(int ny_pad, int ncomp, int jp, int nc_inst, int max_bytes) {
    if (ny_pad > AwShape::N || nc_inst > AwShape::FWARPS || ncomp != nc_inst || jp != AwShape::JP) return AwSmem{};
    for (int dz = 16; dz >= AwShape::FWARPS + 2; --dz) {
        AwSmem l{};
        l.dz = dz;
        l.slot_off = 0;
        l.tw_off = (uint32_t)(dz * AwShape::SLOT * sizeof(float2));
        l.t2_off = l.tw_off + AwShape::N * sizeof(float2);
        l.stage_off = (l.t2_off + AwShape::N * sizeof(float2) + 127) & ~127u;  // tensor-store sources: 128-byte aligned
        l.bar_off = l.stage_off + AwShape::FWARPS * AwShape::N * sizeof(float2);
        l.flag_off = l.bar_off + 2 * dz * 8;
        l.total = l.flag_off + 16;
        if ((int)l.total <= max_bytes) return l;
    }
    return AwSmem{};
}

}  // namespace grav
