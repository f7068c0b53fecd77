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
#include <climits>
#include <algorithm>

#include "async_copy.cuh"
#include "fft_block.cuh"
#include "grav_internal.h"
#include "warp_fft.cuh"

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

// FP32 rows of length P = 2048 with at most 1024 nonzero values (the row
// stages of every mesh with 513 <= nx <= 1024): the even and the odd outputs
// are two independent 1024-point transforms,
//   Z(2k + p) = sum_{x < 1024} z[x] W_2048^(p x) W_1024^(x k),   p = 0, 1,
// one warp each (warp_fft.cuh).  Conjugate partners k and P - k have the
// same parity, so splitting Z into the spectra of the two packed real rows
// only needs one warp's output.
//
// Persistent CTAs, two per SM.  A tile is 8 rows of one layer (4 packed
// sequences, two warps each).  The tile's rows are brought into shared
// memory by bulk copies (TMA) on an mbarrier; as soon as every warp has read
// them into registers, the copies of the CTA's next tile are issued, so
// they land while this tile is transformed and written.  The CTA writes its
// rows transposed, [kx][o][i], 64 bytes per kx, next to the 64 bytes of the
// CTA holding the neighbouring tile.  Every wait is bounded.
__host__ __device__ inline int ny_blocks(int ny) { return (ny + 7) / 8; }

constexpr int kRwSeqs = 4;                       // packed sequences per tile
constexpr int kRwRows = 2 * kRwSeqs;             // rows per tile
constexpr int kRwThreads = 64 * kRwSeqs;         // two warps per sequence
constexpr int kRwPitch = 1024;                   // floats per staged row
// Complex values per warp area: the transpose area plus 2, so that the eight
// areas start 4 banks apart and the output pass reads them without conflicts.
constexpr int kRwArea = kWarpFftSlot + 2;
constexpr size_t kRwAreaOff = (size_t)kRwRows * kRwPitch * sizeof(float);
constexpr size_t kRwT2Off = kRwAreaOff + (size_t)kRwRows * kRwArea * sizeof(float2);
constexpr size_t kRwBarOff = kRwT2Off + 1024 * sizeof(float2);
constexpr size_t kRwSmem = kRwBarOff + 16;

__global__ void __launch_bounds__(kRwThreads, 2)
    row_r2c_warp_kernel(const float* __restrict__ in, size_t in_ostride, size_t in_istride, int l_in, int I, int O,
                        float2* __restrict__ out, int i_pad, const float2* __restrict__ tw, int log_t,
                        size_t in_bstride, size_t out_bstride, int nbatch, int* __restrict__ err) {
    constexpr int N = 1024, FS = kRwArea;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* sin = reinterpret_cast<float*>(smem_raw);                  // [row][kRwPitch]
    float2* zs = reinterpret_cast<float2*>(smem_raw + kRwAreaOff);    // per warp: transpose area, then Z_p
    float2* t2 = reinterpret_cast<float2*>(smem_raw + kRwT2Off);      // W_1024^(k1 n2) at [k1][n2]
    uint64_t* inb = reinterpret_cast<uint64_t*>(smem_raw + kRwBarOff);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // tile t = (bz O + o) rbs + rb, in 32 bits (the launch checks the count)
    const unsigned rbs = (unsigned)(I + kRwRows - 1) / kRwRows;  // row blocks per layer
    const unsigned ntiles = (unsigned)nbatch * (unsigned)O * rbs;

    // bulk copies of tile t's rows (thread 0)
    auto issue = [&](unsigned t) {
        const unsigned rest = t / rbs;
        const int rb = (int)(t - rest * rbs);
        const int bz = (int)(rest / (unsigned)O), o = (int)(rest - (unsigned)bz * (unsigned)O);
        const int i0 = rb * kRwRows, nrows = min(kRwRows, I - i0);
        const uint32_t row_bytes = (uint32_t)l_in * sizeof(float);
        const float* src = in + bz * in_bstride + (size_t)o * in_ostride + (size_t)i0 * in_istride;
        mbar_arrive_expect_tx(inb, row_bytes * nrows);
        for (int j = 0; j < nrows; ++j) bulk_g2s(sin + j * kRwPitch, src + (size_t)j * in_istride, row_bytes, inb);
    };

    if (tid == 0) {
        mbar_init(inb, 1);
        fence_mbar_init();
    }
    for (int e = tid; e < N; e += kRwThreads) t2[e] = tw[(((e >> 5) * (e & 31)) & (N - 1)) << (log_t - 10)];
    __syncthreads();
    if (tid == 0 && blockIdx.x < ntiles) issue(blockIdx.x);

    const int sq = warp >> 1, p = warp & 1;
    // odd outputs: z[x] W_2048^x with x = 32 n1 + lane, W_2048^x = W_64^n1 W_2048^lane
    const float2 wl = tw[lane << (log_t - 11)];
    int it = 0;
    for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const unsigned rest = t / rbs;
        const int rb = (int)(t - rest * rbs);
        const int bz = (int)(rest / (unsigned)O), o = (int)(rest - (unsigned)bz * (unsigned)O);
        const int ib = rb * kRwRows;
        const bool ok = mbar_wait_bounded(inb, (uint32_t)(it & 1), kWaitLimitNs);
        const int i0 = ib + 2 * sq;
        const bool ha = ok && i0 < I, hb = ok && i0 + 1 < I;
        const float* ra = sin + (2 * sq) * kRwPitch;
        const float* rbp = ra + kRwPitch;
        float2 u[32];
        // all of the tile's loads first, the odd-output fold factor after
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) {
            const int x = 32 * n1 + lane;
            float2 v = make_float2(0.f, 0.f);
            if (x < l_in) {
                if (ha) v.x = ra[x];
                if (hb) v.y = rbp[x];
            }
            u[n1] = v;
        }
        if (p) {
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) u[n1] = cmul(tw64(u[n1], n1), wl);
        }
        if (__syncthreads_or(!ok)) {
            // a copy did not land in time: record it, let the copy land
            // (bounded) before the shared memory is released, and leave
            if (tid == 0) {
                atomicExch(err, 1);
                mbar_wait_bounded(inb, (uint32_t)(it & 1), kWaitLimitNs);
            }
            return;
        }
        // every warp has read the staged rows: bring in the next tile's
        if (tid == 0 && t + gridDim.x < ntiles) {
            fence_proxy_async_smem();
            issue(t + gridDim.x);
        }
        float2* zw = zs + warp * FS;
        warp_fft1024<false>(u, zw, t2, lane);
#pragma unroll
        for (int j = 0; j < 32; ++j) zw[lane + 32 * bitrev5(j)] = u[j];
        __syncthreads();

        // A(kx) = (Z(kx) + conj Z(P - kx)) / 2, B(kx) = (Z(kx) - conj Z(P - kx)) / (2i).
        // Thread t writes packed sequence t % 4 for kx = t / 4, t / 4 + 64, ...: its
        // row pair and output parity stay fixed (a warp writes 8 kx x 64 bytes).
        {
            constexpr int KSTEP = kRwThreads / kRwSeqs;  // 64, even: the parity of kx stays fixed
            const int s = tid % kRwSeqs, kx0 = tid / kRwSeqs, q = kx0 & 1;
            const int j0 = ib + 2 * s;
            if (j0 < I) {
                const float2* zp = zs + (2 * s + q) * FS;
                const bool pair = j0 + 1 < I;
                const size_t dstep = (size_t)KSTEP * O * i_pad;
                float2* dst = out + bz * out_bstride + ((size_t)kx0 * O + o) * i_pad + j0;
#pragma unroll 4
                for (int kx = kx0; kx <= N; kx += KSTEP, dst += dstep) {
                    const int k = kx >> 1;
                    const float2 zk = zp[k];
                    const float2 zm = cconj(zp[q ? N - 1 - k : (N - k) & (N - 1)]);
                    const float2 A = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
                    const float2 d = csub(zk, zm);
                    const float2 B = make_float2(0.5f * d.y, -0.5f * d.x);
                    if (pair) {
                        *reinterpret_cast<float4*>(dst) = make_float4(A.x, A.y, B.x, B.y);
                    } else {
                        dst[0] = A;
                    }
                }
            }
        }
    }
}

// Adjoint inverse rows, FP32, P = 2048, from the tiled column output
// in_r[n][y / 8][kx][8] of both ky parities (summed here); within a kx run,
// row pair j (rows 2j, 2j + 1 of the tile) is at 16-byte position
// (j + kx / 2) % 4.  Only the
// first 1024 outputs of each length-2048 inverse transform are kept, so the
// transform is split by output parity (decimation in frequency):
//   z[2m]     = sum_{k < 1024} (Z(k) + Z(k + 1024))            W_1024^(-m k)
//   z[2m + 1] = sum_{k < 1024} (Z(k) - Z(k + 1024)) W_2048^(-k) W_1024^(-m k)
// one 1024-point warp transform each (warp_fft1024), with Z(k) = A(k) + i B(k)
// for the packed rows a, b and Z(k) for k > 1024 from Hermitian symmetry.
// Persistent CTAs, two per SM.  A tile is 8 rows of one layer: one
// contiguous run per input (the two ky parities of the plane adjoint, or a
// single input) brought in by a bulk copy on an mbarrier, the inputs one
// after the other through one buffer: every warp adds its share of the
// first input to its registers (the packed spectrum is linear in the input)
// before the second input's copy is issued.  The warps' transpose areas
// share that buffer, so the next tile's copy is issued once every transform
// is done.  Warp w handles rows 2 (w / 2), 2 (w / 2) + 1 and output parity
// w % 2, and stores its outputs straight to the rows.
constexpr int kCtRows = 8;                         // rows per tile
constexpr int kCtThreads = 32 * kCtRows;           // two warps per packed row pair
constexpr int kCtKx = 1025;                        // P / 2 + 1
constexpr size_t kCtHalf = (size_t)kCtKx * kCtRows * sizeof(float2);  // bytes of one input's tile
constexpr size_t kCt1Region = (size_t)kCtRows * kWarpFftSlot * sizeof(float2);
static_assert(kCt1Region >= kCtHalf, "one input's tile fits in the transpose areas");
constexpr size_t kCt1T2Off = kCt1Region;
constexpr size_t kCt1BarOff = kCt1T2Off + 1024 * sizeof(float2);
constexpr size_t kCt1Smem = kCt1BarOff + 16;

template <bool TWO>
__global__ void __launch_bounds__(kCtThreads, 2)
    row_c2r_tiled_kernel(const float2* __restrict__ in0, const float2* __restrict__ in1, int ny, int nz,
                         float* __restrict__ out, size_t out_stride, int l_out, const float2* __restrict__ tw,
                         int log_t, size_t in_bstride, size_t out_bstride, int nbatch, int* __restrict__ err) {
    constexpr int N = 1024, NPH = TWO ? 2 : 1;  // inputs, brought in one after the other
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const float2* t0 = reinterpret_cast<const float2*>(smem_raw);  // the input of this phase, [kx][8]
    float2* areas = reinterpret_cast<float2*>(smem_raw);           // transpose areas, once t0 is read
    float2* t2 = reinterpret_cast<float2*>(smem_raw + kCt1T2Off);
    uint64_t* inb = reinterpret_cast<uint64_t*>(smem_raw + kCt1BarOff);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ybs = ny_blocks(ny);
    // tile t = (bz nz + n) ybs + yb, in 32 bits (the launch checks the count)
    const unsigned per_b = (unsigned)nz * (unsigned)ybs;
    const unsigned ntiles = (unsigned)nbatch * per_b;

    auto issue = [&](unsigned t, int ph) {  // thread 0: input ph's run of tile t
        const unsigned bz = t / per_b, rest = t - bz * per_b;  // rest = n * ybs + yb
        const size_t off = (size_t)rest * kCtKx * kCtRows;
        mbar_arrive_expect_tx(inb, (uint32_t)kCtHalf);
        bulk_g2s(smem_raw, (ph ? in1 : in0) + bz * in_bstride + off, (uint32_t)kCtHalf, inb);
    };

    if (tid == 0) {
        mbar_init(inb, 1);
        fence_mbar_init();
    }
    for (int e = tid; e < N; e += kCtThreads) t2[e] = tw[(((e >> 5) * (e & 31)) & (N - 1)) << (log_t - 10)];
    __syncthreads();
    if (tid == 0 && blockIdx.x < ntiles) issue(blockIdx.x, 0);

    const int sq = warp >> 1, p = warp & 1;
    // odd outputs: W_2048^(-k) with k = 32 n1 + lane = W_64^(-n1) W_2048^(-lane)
    const float2 wl = cconj(tw[lane << (log_t - 11)]);
    uint32_t waits = 0;  // completed phases of inb
    for (unsigned t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const unsigned bz = t / per_b, rest = t - bz * per_b;
        const int n = (int)(rest / (unsigned)ybs), yb = (int)(rest - (unsigned)n * (unsigned)ybs);
        const int ya = yb * kCtRows + 2 * sq;
        // v[n1] = Z(k) +- Z(k + 1024) (output parity p), k = 32 n1 + lane, for the
        // packed spectrum Z = A + i B of rows ya, ya + 1: linear in the input, so
        // each input's share is added in turn
        float2 u[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) u[n1] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int ph = 0; ph < NPH; ++ph) {
            const bool ok = mbar_wait_bounded(inb, waits & 1u, kWaitLimitNs);
            ++waits;
            const bool ha = ok && ya < ny, hb = ok && ya + 1 < ny;
            auto zk = [&](int kx) {  // (A, B) of this input at kx
                const int pos = 2 * ((sq + (kx >> 1)) & 3);  // row pair sq's 16-byte position in the run
                const float4 v0 = *reinterpret_cast<const float4*>(t0 + kx * kCtRows + pos);
                float2 A = make_float2(v0.x, v0.y), B = make_float2(v0.z, v0.w);
                if (!ha) A = make_float2(0.f, 0.f);
                if (!hb) B = make_float2(0.f, 0.f);
                if (kx == 0 || kx == kCtKx - 1) A.y = B.y = 0.f;  // real DC and Nyquist
                return make_float4(A.x, A.y, B.x, B.y);
            };
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) {
                const int k = 32 * n1 + lane;
                const float4 a1 = zk(k);
                const float2 z1 = make_float2(a1.x - a1.w, a1.y + a1.z);  // A + i B
                const float4 a2 = zk(N - k);                                // k = 0: the Nyquist bin itself
                // Z(k + 1024) = conj A(1024 - k) + i conj B(1024 - k) (k > 0), A + i B at the Nyquist bin (k = 0)
                const float2 z2 = k ? make_float2(a2.x + a2.w, a2.z - a2.y) : make_float2(a2.x - a2.w, a2.y + a2.z);
                const float2 v = p ? make_float2(z1.x - z2.x, z1.y - z2.y) : make_float2(z1.x + z2.x, z1.y + z2.y);
                u[n1] = make_float2(u[n1].x + v.x, u[n1].y + v.y);
            }
            if (__syncthreads_or(!ok)) {
                // a copy did not land in time: record it, let the copy land
                // (bounded) before the shared memory is released, and leave
                if (tid == 0) {
                    atomicExch(err, 1);
                    mbar_wait_bounded(inb, (waits - 1) & 1u, kWaitLimitNs);
                }
                return;
            }
            if (ph + 1 < NPH && tid == 0) {  // every warp has read this input: the next one
                fence_proxy_async_smem();
                issue(t, ph + 1);
            }
        }
        if (p) {
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) u[n1] = cmul(tw64(u[n1], -n1), wl);
        }
        warp_fft1024<true>(u, areas + warp * kWarpFftSlot, t2, lane);
        __syncthreads();  // every transform is done with the areas (the tile buffer)
        if (tid == 0 && t + gridDim.x < ntiles) {
            fence_proxy_async_smem();
            issue(t + gridDim.x, 0);
        }
        // u[j] = z[2 m + p], m = lane + 32 bitrev5(j)
        float* oa = out + bz * out_bstride + ((size_t)n * ny + ya) * out_stride;
        float* ob = oa + out_stride;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int x = 2 * (lane + 32 * bitrev5(j)) + p;
            if (x < l_out) {
                if (ya < ny) oa[x] = u[j].x;
                if (ya + 1 < ny) ob[x] = u[j].y;
            }
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

#pragma unroll
    for (int s = 0; s < NSEQ; ++s) {
        const int i0 = i_base + 2 * s, i1 = i0 + 1;
        if (i0 >= I) break;
        R* oa = out + ((size_t)o * I + i0) * out_stride;
        R* ob = oa + out_stride;
        const C* bs = buf + s * SSTR;
        for (int x = tid; x < l_out; x += NT) {
            const C z = bs[sidx<C>(x)];
            oa[x] = z.x;
            if (i1 < I) ob[x] = z.y;
        }
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

// SMs of the current device (cached per device).
inline int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    int n = cache[dev & 63].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cache[dev & 63].store(n, std::memory_order_relaxed);
    }
    return n;
}

template <typename R, int LOGP>
cudaError_t r2c_impl(const R* in, size_t in_ostride, size_t in_istride, int l_in, int I, int O, void* out, int i_pad,
                     const void* tw, int log_t, cudaStream_t s, Batch b, int* err) {
    if constexpr (sizeof(R) == 4 && LOGP == 11) {
        // 2048-point float rows, at most 1024 nonzero, 16-byte aligned rows:
        // two warp transforms per row pair, rows staged by bulk copies
        const int sms = sm_count();
        const long ntiles = (long)b.count * O * ((I + kRwRows - 1) / kRwRows);
        const bool fits = err && sms > 0 && l_in <= kRwPitch && l_in % 4 == 0 && in_istride % 4 == 0 &&
                          in_ostride % 4 == 0 && b.in % 4 == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0 &&
                          i_pad % 2 == 0 && b.out % 2 == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0 &&
                          ntiles <= INT_MAX;  // the kernel counts tiles in 32 bits
        if (fits) {
            constexpr auto k = row_r2c_warp_kernel;
            cudaError_t e = ensure_smem_limit<k>();
            if (e != cudaSuccess) return e;
            const int grid = (int)std::min<long>(ntiles, 2L * sms);
            if (grid == 0) return cudaSuccess;
            k<<<grid, kRwThreads, kRwSmem, s>>>(in, in_ostride, in_istride, l_in, I, O, (float2*)out, i_pad,
                                                (const float2*)tw, log_t, b.in, b.out, b.count, err);
            return cudaGetLastError();
        }
    }
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
                           void* out, int i_pad, const void* tw, int log_t, cudaStream_t s, Batch b, int* err) {
    switch (log_p) {
#define CASE(L) \
    case L: return r2c_impl<R, L>(in, in_ostride, in_istride, l_in, I, O, out, i_pad, tw, log_t, s, b, err);
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

namespace {
template <bool TWO>
cudaError_t c2r_tiled_launch(int grid, const void* in0, const void* in1, int ny, int nz, float* out, size_t out_stride,
                             int l_out, const void* tw, int log_t, cudaStream_t s, Batch b, int* err) {
    constexpr auto k = row_c2r_tiled_kernel<TWO>;
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    k<<<grid, kCtThreads, kCt1Smem, s>>>((const float2*)in0, (const float2*)in1, ny, nz, out, out_stride, l_out,
                                        (const float2*)tw, log_t, b.in, b.out, b.count, err);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_row_c2r_tiled(const void* in0, const void* in1, int ny, int nz, int kx_count, float* out,
                                 size_t out_stride, int l_out, const void* tw, int log_t, cudaStream_t s, Batch b,
                                 int* err) {
    if (kx_count != kCtKx || l_out > 1024 || !err || (reinterpret_cast<uintptr_t>(in0) & 15) ||
        (reinterpret_cast<uintptr_t>(in1) & 15) || (b.in * sizeof(float2)) % 16)
        return cudaErrorInvalidValue;
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorInvalidValue;
    const long ntiles = (long)b.count * nz * ny_blocks(ny);
    if (ntiles > INT_MAX) return cudaErrorInvalidValue;  // the kernel counts tiles in 32 bits
    const int grid = (int)std::min<long>(ntiles, 2L * sms);
    if (grid == 0) return cudaSuccess;
    return in1 ? c2r_tiled_launch<true>(grid, in0, in1, ny, nz, out, out_stride, l_out, tw, log_t, s, b, err)
               : c2r_tiled_launch<false>(grid, in0, in1, ny, nz, out, out_stride, l_out, tw, log_t, s, b, err);
}

template cudaError_t launch_row_r2c<float>(int, const float*, size_t, size_t, int, int, int, void*, int, const void*,
                                           int, cudaStream_t, Batch, int*);
template cudaError_t launch_row_r2c<double>(int, const double*, size_t, size_t, int, int, int, void*, int,
                                            const void*, int, cudaStream_t, Batch, int*);
template cudaError_t launch_row_c2r<float>(int, const void*, const void*, int, int, int, float*, size_t, int,
                                           const void*, int, cudaStream_t, Batch);
template cudaError_t launch_row_c2r<double>(int, const void*, const void*, int, int, int, double*, size_t, int,
                                            const void*, int, cudaStream_t, Batch);

}  // namespace grav
