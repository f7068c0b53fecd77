// 1024-point FFT by a single warp, 32 complex values a lane, in registers
// (FP32), as 1024 = 32 x 32 (the four-step form):
//   x[32 n1 + n2] -> 32-point DFTs over n1 (lane n2) -> twiddle W_1024^(n2 k1)
//   -> transpose through shared memory -> 32-point DFTs over n2 (lane k1).
// A warp transform needs no block or group barrier, only __syncwarp.
#pragma once
#include "fft_block.cuh"

namespace grav {

constexpr int kWarpFftSlot = 32 * 33;  // complex values of a warp's transpose area

// cos(2 pi j / 32) for any integer j (exact symmetries of the first octant).
__device__ __forceinline__ float cos32(int j) {
    const float b[9] = {1.0f,
                        0.980785280403230449126f,
                        0.923879532511286756128f,
                        0.831469612302545237079f,
                        0.707106781186547524401f,
                        0.555570233019602224743f,
                        0.382683432365089771729f,
                        0.195090322016128267848f,
                        0.0f};
    j &= 31;
    if (j <= 8) return b[j];
    if (j <= 16) return -b[16 - j];
    if (j <= 24) return -b[j - 16];
    return b[32 - j];
}

// a * W_32^j with W_32 = exp(-+ 2 pi i / 32) (inverse: +); j is a constant
// after unrolling, so the branches and the cosines fold away.
template <bool INV> __device__ __forceinline__ float2 tw32(float2 a, int j) {
    j &= 31;
    if (j == 0) return a;
    if (j == 16) return make_float2(-a.x, -a.y);
    if (j == 8) return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    if (j == 24) return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    const float c = cos32(j), s = INV ? cos32(j - 8) : -cos32(j - 8);  // sin(2 pi j/32) = cos(2 pi (j-8)/32)
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

// cos(2 pi j / 64) for any integer j (first-quadrant values and symmetries).
__device__ __forceinline__ float cos64(int j) {
    const float b[17] = {1.0f,
                         0.995184726672196886245f,
                         0.980785280403230449126f,
                         0.956940335732208864936f,
                         0.923879532511286756128f,
                         0.881921264348355029713f,
                         0.831469612302545237079f,
                         0.773010453362736960810f,
                         0.707106781186547524401f,
                         0.634393284163645498215f,
                         0.555570233019602224743f,
                         0.471396736825997648556f,
                         0.382683432365089771729f,
                         0.290284677254462367636f,
                         0.195090322016128267848f,
                         0.098017140329560601994f,
                         0.0f};
    j &= 63;
    if (j <= 16) return b[j];
    if (j <= 32) return -b[32 - j];
    if (j <= 48) return -b[j - 32];
    return b[64 - j];
}

// a * W_64^j, W_64 = exp(-2 pi i / 64); j is a constant after unrolling.
__device__ __forceinline__ float2 tw64(float2 a, int j) {
    j &= 63;
    if (j == 0) return a;
    if (j == 16) return make_float2(a.y, -a.x);
    if (j == 32) return make_float2(-a.x, -a.y);
    if (j == 48) return make_float2(-a.y, a.x);
    const float c = cos64(j), s = -cos64(j - 16);  // sin(2 pi j/64) = cos(2 pi (j-16)/64)
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

__host__ __device__ constexpr int bitrev5(int j) {
    return ((j & 1) << 4) | ((j & 2) << 2) | (j & 4) | ((j & 8) >> 2) | ((j & 16) >> 4);
}

// 32-point DFT in registers, radix-2 decimation in frequency: natural order
// in, u[j] = X[bitrev5(j)] out.  PACKED: each complex add and subtract is
// one two-wide FP32 instruction (same roundings as the scalar form); a
// kernel at a tight register cap may take the scalar form, which needs no
// aligned register pairs.
template <bool INV, bool PACKED = true> __device__ __forceinline__ void dft32(float2 (&u)[32]) {
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < 32; b += 2 * h) {
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float2 a = u[b + i], c = u[b + i + h];
                const int j = i * (16 / h);
                if constexpr (PACKED) {
                    u[b + i] = cadd(a, c);
                    // twiddle -1 folds into the subtraction; the others act on a - c
                    u[b + i + h] = j == 16 ? csub(c, a) : tw32<INV>(csub(a, c), j);
                } else {
                    u[b + i] = make_float2(a.x + c.x, a.y + c.y);
                    u[b + i + h] = tw32<INV>(make_float2(a.x - c.x, a.y - c.y), j);
                }
            }
        }
    }
}

// 1024-point FFT by one warp.  In: u[n1] = x[32 n1 + lane].  Out: u[j] =
// X[lane + 32 bitrev5(j)].  tr: the warp's 32 x 33 transpose area; t2[k1 32 +
// lane] = W_1024^(lane k1).  tr may be overwritten by the caller afterwards.
template <bool INV, bool PACKED = true>
__device__ __forceinline__ void warp_fft1024(float2 (&u)[32], float2* tr, const float2* t2, int lane) {
    dft32<INV, PACKED>(u);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int k1 = bitrev5(j);
        float2 w = t2[k1 * 32 + lane];
        if (INV) w.y = -w.y;
        tr[k1 * 33 + lane] = cmul(u[j], w);
    }
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) u[n2] = tr[lane * 33 + n2];
    __syncwarp();
    dft32<INV, PACKED>(u);
}

__host__ __device__ constexpr int bitrev4(int j) { return ((j & 1) << 3) | ((j & 2) << 1) | ((j & 4) >> 1) | ((j & 8) >> 3); }

// 16-point DFT of u[OFF .. OFF + 15] in registers, radix-2 decimation in
// frequency (W_16^k = W_32^(2k)): natural order in, u[OFF + j] = X[bitrev4(j)]
// out.
template <bool INV, int OFF, bool PACKED = true> __device__ __forceinline__ void dft16(float2 (&u)[32]) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < 16; b += 2 * h) {
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float2 a = u[OFF + b + i], c = u[OFF + b + i + h];
                if constexpr (PACKED) {
                    u[OFF + b + i] = cadd(a, c);
                    u[OFF + b + i + h] = tw32<INV>(csub(a, c), 2 * i * (8 / h));
                } else {
                    u[OFF + b + i] = make_float2(a.x + c.x, a.y + c.y);
                    u[OFF + b + i + h] = tw32<INV>(make_float2(a.x - c.x, a.y - c.y), 2 * i * (8 / h));
                }
            }
        }
    }
}

// Two 512-point FFTs by one warp, 512 = 16 x 32: x[32 n1 + n2] (n1 < 16) ->
// 16-point DFTs over n1 (lane n2) -> twiddle -> transpose -> 32-point DFTs
// over n2.  In: u[n1] = a[32 n1 + lane], u[16 + n1] = b[32 n1 + lane].  Out:
// lane L holds transform L / 16 (0: a, 1: b) at k1 = L % 16, u[j] = X[k1 +
// 16 bitrev5(j)].  t2[(16 h + k1) 32 + lane] is the twiddle of transform h
// at (k1, n2 = lane), W_512^(n2 k1) for a plain pair of transforms (a caller
// may fold a factor constant over n1 into it).  tr: the warp's 32 x 33
// transpose area, free for the caller afterwards.
template <bool INV, bool PACKED = true>
__device__ __forceinline__ void warp_fft512x2(float2 (&u)[32], float2* tr, const float2* t2, int lane) {
    dft16<INV, 0, PACKED>(u);
    dft16<INV, 16, PACKED>(u);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int K = 16 * h + bitrev4(j);
            float2 w = t2[K * 32 + lane];
            if (INV) w.y = -w.y;
            tr[K * 33 + lane] = cmul(u[16 * h + j], w);
        }
    }
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) u[n2] = tr[lane * 33 + n2];
    __syncwarp();
    dft32<INV, PACKED>(u);
}

}  // namespace grav
