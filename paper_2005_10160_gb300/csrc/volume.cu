// Equal-dimension variant (Sec. 2.2, Eqs. 10-11): a station at the centre of
// every cell, so the data are as three-dimensional as the mesh and G is
// block Toeplitz in all three cell offsets (the block matrix of G_{t,n}
// after Eq. 22): G(station (p,q,t), cell (l,m,n)) = K(l-p, m-q, n-t), with
// (2nx-1)(2ny-1)(2nz-1) distinct values.
//
// The product is a three-level circulant embedding plus FFT: K(u,v,w) sits at
// ((-u) mod Px, (-v) mod Py, (-w) mod Pz) (the correlation form of Eq. 19 on
// every axis), each P a power of two >= 2n-1.  The embedded kernel is even or
// odd in every axis (the reflection symmetries of Sec. 2.2; along w: gz, gxz
// and gyz change sign when the station and the cell swap sides, the rest do
// not), so its spectrum is purely real or purely imaginary and even or odd in
// kx, ky and kz: the plan stores one real number per mirror triple,
//   spec3[c][kx][jy][jz],  kx <= Px/2, jy <= Py/2, jz <= Pz/2,
// with S_c(kx, ky, kz) = +-v (real) or +-i v (imaginary), the signs given by
// the component's parity in y and z for ky > Py/2, kz > Pz/2, and the
// 1/(Px Py Pz) of the inverse transforms folded in.
//
// Plan creation (FP64).  K(u,v,w) for a station at a cell centre is the
// plane kernel of kernel_gen.cu for 2nz-1 "layers" j = w + nz - 1 seen from
// the height h' = -(nz - 1/2) dz: its z-levels (nz - 1/2 - j) dz and
// (nz - 3/2 - j) dz are the station-minus-corner depths (1/2 - w) dz and
// (-1/2 - w) dz.  Per component and chunk of layers: generate and embed
// the rows b < Py/2 (kernel_gen; the other rows mirror them), transform
// them along x (row_r2c), transform the columns (y) by the parity fold and
// keep the real or imaginary part of ky <= Py/2 per layer; then transform
// each (kx, ky) sequence over the layers along z and keep the real or
// imaginary part of kz <= Pz/2.
//
// Forward, per call (five passes through HBM; B = ncomp):
//   A  x: row transforms of rho (R2C, row_r2c)          -> X[kx][n][y]
//   B  y: column FFTs of every (kx, n) row (length Py)    -> U[kx][n][ky]
//   C  z: per kx and tile of ky columns, FFT along n (length Pz), product with
//         S_c, inverse FFT, the nz stations kept, for every component c
//                                                         -> W[kx][c][t][ky]
//   D  y: inverse column FFTs, the ny stations kept       -> V[kx][c][t][y]
//   E  x: inverse row transforms (C2R, row_c2r)           -> out[c][t][y][x]
// The adjoint runs the same passes from r[c][t][y][x], multiplies by the
// conjugate spectra and sums over components in pass C (the transpose).
// Generic block-FFT kernels serve every size; FP32 plans at the common sizes
// take register-resident kernels instead: pass C for Pz = 256
// (vol_z256_kernel), passes B and D for Py = 2048 (vol_yfwd2048_kernel,
// vol_yinv2048_tiled_kernel) and, with Px = 2048, D writes the tiled layout
// V[c t][y / 8][kx][8] that pass E reads by bulk copies
// (launch_row_c2r_tiled).
#include <algorithm>
#include <new>
#include <type_traits>

#include "async_copy.cuh"
#include "fft_block.cuh"
#include "grav_internal.h"
#include "warp_fft.cuh"

namespace grav {

namespace {

constexpr int kVolMaxNx = 1024, kVolMaxNy = 1024, kVolMaxNz = 512;
constexpr int kVolThreads = 256;
// gz, gxz and gyz are odd in the layer offset w (the field of a cell below a
// station is the mirror image of one above it with the vertical sense flipped).
constexpr unsigned kOddWMask = 0x29u;
__host__ __device__ constexpr bool odd_w(int c) { return (kOddWMask >> c) & 1u; }

// Sequences per CTA of the row FFT kernels: about 64 KB (FP32) / 128 KB
// (FP64) of shared memory.
template <typename C> constexpr int rows_nseq(int logn) {
    const int n = 8192 >> logn;
    return n < 1 ? 1 : (n > 64 ? 64 : n);
}
// Columns per CTA of the z kernel: two buffers of TI sequences of Pz points,
// 4096 (FP32) or 2048 (FP64) points each, about 76 KB in all, so that two
// CTAs share an SM.
template <typename C> constexpr int z_tile(int logz) {
    const int cap = sizeof(C) == 8 ? 32 : 16;
    const int n = (sizeof(C) == 8 ? 4096 : 2048) >> logz;
    return n < 1 ? 1 : (n > cap ? cap : n);
}

// Columns per warp of the z kernel: an eighth of the tile, and at least
// enough that every lane owns an element (Pz < 32); warps = TI / columns.
constexpr int z_cols_per_warp(int ti, int logz) {
    const int by_warps = ti / 8 > 1 ? ti / 8 : 1;
    const int by_lanes = (32 + (1 << logz) - 1) >> logz;
    const int c = by_warps > by_lanes ? by_warps : by_lanes;
    return c < ti ? c : ti;
}
// Whether each warp transforms its own columns (a lane then holds at most 16
// FP32 or 8 FP64 values of them) or, for long columns, the whole CTA of 256
// threads transforms the tile together.
constexpr bool z_warp_mode(int ti, int logz, bool fp64) {
    return z_cols_per_warp(ti, logz) * (1 << logz) / 32 <= (fp64 ? 8 : 16);
}
constexpr int z_threads(int ti, int logz, bool fp64) {
    return z_warp_mode(ti, logz, fp64) ? 32 * (ti / z_cols_per_warp(ti, logz)) : 256;
}

// ---------------------------------------------------------------------------
// Pass B / D (and the plan's column step): FFTs of `rows` contiguous rows.
//   in row k: in[k * in_stride + m], m < l_in (zero beyond); out row k:
//   out[k * out_stride + m], m < l_out.
template <typename C, int LOGN, int NSEQ, bool INV>
__global__ void __launch_bounds__(kVolThreads) vol_rows_kernel(const C* __restrict__ in, size_t in_stride, int l_in,
                                                               C* __restrict__ out, size_t out_stride, int l_out,
                                                               long rows, const C* __restrict__ tw, int tw_shift) {
    constexpr int N = 1 << LOGN, SSTR = seq_stride<C>(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x;
    const long row0 = (long)blockIdx.x * NSEQ;
    block_fft_from<C, LOGN, NSEQ, kVolThreads, INV>(buf, SSTR, tw, tw_shift, tid, [&](int s, int m) {
        const long k = row0 + s;
        return (k < rows && m < l_in) ? in[k * in_stride + m] : cmk<C>(0, 0);
    });
#pragma unroll
    for (int s = 0; s < NSEQ; ++s) {
        const long k = row0 + s;
        if (k >= rows) break;
        C* dst = out + k * out_stride;
        const C* bs = buf + s * SSTR;
        for (int m = tid; m < l_out; m += kVolThreads) dst[m] = bs[sidx<C>(m)];
    }
}

// Pass D when pass E runs the tiled inverse row kernel (FP32, Px = 2048):
// inverse column FFTs of the rows W[kx][r][ky] (r = c nz + t: R rows per kx),
// the ny stations kept and written as V[r][y / 8][kx][8], row pair j of each
// block of 8 rows at 16-byte position (j + kx / 2) % 4 of its kx run (rows
// beyond ny zero): the layout launch_row_c2r_tiled reads with one bulk copy
// per block.  A CTA transforms four kx of one r and writes 256 contiguous
// bytes per block.
constexpr int kYtSeqs = 4;
template <int LOGN>
__global__ void __launch_bounds__(kVolThreads) vol_yinv_tiled_kernel(const float2* __restrict__ in, int R, int kx_count,
                                                                     int ny, float2* __restrict__ out,
                                                                     const float2* __restrict__ tw, int tw_shift) {
    constexpr int N = 1 << LOGN, SSTR = seq_stride<float2>(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    const int tid = threadIdx.x;
    const int kx0 = blockIdx.x * kYtSeqs, r = blockIdx.y;
    block_fft_from<float2, LOGN, kYtSeqs, kVolThreads, true>(buf, SSTR, tw, tw_shift, tid, [&](int sq, int m) {
        const int kx = kx0 + sq;
        return kx < kx_count ? in[((size_t)kx * R + r) * N + m] : make_float2(0.f, 0.f);
    });
    const int ybs = (ny + 7) >> 3;
    for (int e = tid; e < ybs * kYtSeqs * 8; e += kVolThreads) {
        const int slot = e & 7, sq = (e >> 3) & (kYtSeqs - 1), yb = e / (8 * kYtSeqs);
        const int kx = kx0 + sq;
        if (kx >= kx_count) continue;
        const int j = ((slot >> 1) - (kx >> 1)) & 3;  // the row pair at this 16-byte position
        const int y = 8 * yb + 2 * j + (slot & 1);
        out[(((size_t)r * ybs + yb) * kx_count + kx) * 8 + slot] =
            y < ny ? buf[sq * SSTR + sidx<float2>(y)] : make_float2(0.f, 0.f);
    }
}

// Passes B and D for Py = 2048 in FP32 (meshes with 513 <= ny <= 1024), a
// pair of warps per row, each running one 1024-point transform in
// registers (warp_fft1024).
//   forward (ny <= 1024 nonzero inputs -> 2048 outputs): warp p computes
//     Z(2k + p) = sum_{y < 1024} (z[y] W_2048^(p y)) W_1024^(y k);
//   inverse (2048 inputs -> the first 1024 outputs): warp p transforms the
//     samples Z(2k + p), and z[m] = E(m) + W_2048^(-m) O(m) for the even (E)
//     and odd (O) sample transforms.
// The two halves meet in shared memory: the forward writes each row as
// (Z(2k), Z(2k + 1)) pairs of 16 bytes, the inverse writes the tiled layout
// of vol_yinv_tiled_kernel (four kx of one r per group).  Persistent CTAs,
// two per SM.
constexpr int kYwRows = 4, kYwThreads = 64 * kYwRows;
constexpr int kYwArea = kWarpFftSlot + 2;  // areas 4 banks apart
constexpr size_t kYwSmem = (size_t)(2 * kYwRows * kYwArea + 2 * 1024) * sizeof(float2);

// barrier of the two warps of row pair `id` (ids 1 .. 4; 0 is __syncthreads)
__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// t2[k1 32 + n] = W_1024^(k1 n) (warp_fft1024), t1[y] = W_2048^y (y < 1024)
__device__ __forceinline__ void yw_tables(float2* t2, float2* t1, const float2* __restrict__ tw, int log_t, int tid) {
    for (int e = tid; e < 1024; e += kYwThreads) {
        t2[e] = tw[(((e >> 5) * (e & 31)) & 1023) << (log_t - 10)];
        t1[e] = tw[e << (log_t - 11)];
    }
}

__global__ void __launch_bounds__(kYwThreads, 2)
    vol_yfwd2048_kernel(const float2* __restrict__ in, size_t in_stride, int l_in, float2* __restrict__ out,
                        size_t out_stride, long rows, const float2* __restrict__ tw, int log_t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* areas = reinterpret_cast<float2*>(smem_raw);
    float2* t2 = areas + 2 * kYwRows * kYwArea;
    float2* t1 = t2 + 1024;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sq = warp >> 1, p = warp & 1;
    yw_tables(t2, t1, tw, log_t, tid);
    __syncthreads();
    float2* tr = areas + warp * kYwArea;
    const float2* za = areas + 2 * sq * kYwArea;  // Z(2k) of this row
    const float2* zb = za + kYwArea;              // Z(2k + 1)
    for (long g = blockIdx.x; g * kYwRows < rows; g += gridDim.x) {
        const long row = g * kYwRows + sq;
        const bool ok = row < rows;
        const float2* src = in + (size_t)(ok ? row : 0) * in_stride;
        float2 u[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) {
            const int y = 32 * n1 + lane;
            u[n1] = (ok && y < l_in) ? src[y] : make_float2(0.f, 0.f);
        }
        if (p) {
#pragma unroll
            for (int n1 = 0; n1 < 32; ++n1) u[n1] = cmul(u[n1], t1[32 * n1 + lane]);
        }
        warp_fft1024<false>(u, tr, t2, lane);  // u[j] = Z(2 (lane + 32 bitrev5(j)) + p)
#pragma unroll
        for (int j = 0; j < 32; ++j) tr[lane + 32 * bitrev5(j)] = u[j];
        pair_sync(1 + sq);
        if (ok) {
            float4* dst = reinterpret_cast<float4*>(out + (size_t)row * out_stride);
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
                const int k = 512 * p + 32 * i + lane;
                const float2 a = za[k], b = zb[k];
                dst[k] = make_float4(a.x, a.y, b.x, b.y);
            }
        }
        pair_sync(1 + sq);  // both halves are read before the areas are reused
    }
}

__global__ void __launch_bounds__(kYwThreads, 2)
    vol_yinv2048_tiled_kernel(const float2* __restrict__ in, int R, int kx_count, int ny, float2* __restrict__ out,
                              const float2* __restrict__ tw, int log_t) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* areas = reinterpret_cast<float2*>(smem_raw);
    float2* t2 = areas + 2 * kYwRows * kYwArea;
    float2* t1 = t2 + 1024;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sq = warp >> 1, p = warp & 1;
    yw_tables(t2, t1, tw, log_t, tid);
    __syncthreads();
    float2* tr = areas + warp * kYwArea;
    const int kxg = (kx_count + kYwRows - 1) / kYwRows;
    const int ybs = (ny + 7) >> 3;
    const unsigned groups = (unsigned)kxg * (unsigned)R;  // at most 257 x 4608
    for (unsigned g = blockIdx.x; g < groups; g += gridDim.x) {
        const int r = (int)(g / (unsigned)kxg), kx0 = (int)(g - (unsigned)r * (unsigned)kxg) * kYwRows;
        const int kx = kx0 + sq;
        const bool ok = kx < kx_count;
        const float2* src = in + ((size_t)(ok ? kx : 0) * R + r) * 2048 + p;
        float2 u[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) u[n1] = ok ? src[2 * (32 * n1 + lane)] : make_float2(0.f, 0.f);
        warp_fft1024<true>(u, tr, t2, lane);  // u[j] = E or O at m = lane + 32 bitrev5(j)
        if (p) {
#pragma unroll
            for (int j = 0; j < 32; ++j) u[j] = cmul(u[j], cconj(t1[lane + 32 * bitrev5(j)]));
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) tr[lane + 32 * bitrev5(j)] = u[j];
        __syncthreads();  // E and W^-m O of all four rows are in place
        {
            // thread tid writes slot tid % 8 of row kx0 + (tid / 8) % 4 in the
            // blocks yb = tid / 32, tid / 32 + 8, ...: only yb moves
            constexpr int YBSTEP = kYwThreads / (8 * kYwRows);
            const int slot = tid & 7, s = (tid >> 3) & (kYwRows - 1);
            const int kxs = kx0 + s;
            if (kxs < kx_count) {
                const int jj = ((slot >> 1) - (kxs >> 1)) & 3;  // the row pair at this 16-byte position
                const float2* ea = areas + 2 * s * kYwArea;
                const float2* eb = ea + kYwArea;
                int yb = tid / (8 * kYwRows);
                int y = 8 * yb + 2 * jj + (slot & 1);
                float2* dst = out + (((size_t)r * ybs + yb) * kx_count + kxs) * 8 + slot;
                const size_t dstep = (size_t)YBSTEP * kx_count * 8;
                for (; yb < ybs; yb += YBSTEP, y += 8 * YBSTEP, dst += dstep)
                    *dst = y < ny ? cadd(ea[y], eb[y]) : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();  // the areas are rewritten by the next group
    }
}

struct ZArgs {
    int nz, py, kx_count, ncomp;
    int jyc, jzc;          // stored spectra extents per kx: Py/2 + 1, Pz/2 + 1
    unsigned imag3_mask;   // slot s: imaginary three-level spectrum
    unsigned oddv_mask;    // slot s: odd in y
    unsigned oddw_mask;    // slot s: odd in the layer offset
    int tw_shift;          // log2(T / Pz)
};

// Pass C.  Forward (ADJ = false): in = U[kx][n][py], out = W[kx][c][t][py].
// Adjoint: in = U'[kx][c][t][py], out = W'[kx][n][py] = sum_c conj(S_c) . in_c
// transformed back.  One CTA per kx and tile of TI columns ky0 .. ky0 + TI.
// The tile is loaded and stored by the whole CTA (rows of TI consecutive
// columns, coalesced); in between each warp transforms, multiplies and
// transforms back its own SPW columns with warp-level syncs only, on per-pass
// twiddle tables in shared memory.  A lane reads every spectrum value it needs
// for one component before it uses any, so those loads overlap.
struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

template <typename R, int LOGZ, int TI, bool ADJ>
__global__ void __launch_bounds__(z_threads(TI, LOGZ, sizeof(R) == 8), 2)
    vol_z_kernel(ZArgs a, const typename cplx<R>::type* __restrict__ in, typename cplx<R>::type* __restrict__ out,
                 const R* __restrict__ spec3, const typename cplx<R>::type* __restrict__ tw) {
    using C = typename cplx<R>::type;
    constexpr int PZ = 1 << LOGZ, SSTR = seq_stride<C>(PZ);
    constexpr bool WARP = z_warp_mode(TI, LOGZ, sizeof(R) == 8);
    constexpr int NT = z_threads(TI, LOGZ, sizeof(R) == 8);
    // a group transforms its columns together: one warp (WARP) or the CTA
    constexpr int GT = WARP ? 32 : NT;                                // threads of a group
    constexpr int GC = WARP ? z_cols_per_warp(TI, LOGZ) : TI;         // columns of a group
    constexpr int IT = GC * PZ / GT;  // elements a thread multiplies per component
    using Sync = typename std::conditional<WARP, WarpSync, BlockSync>::type;
    static_assert(GC * PZ % GT == 0 && IT > 0, "whole elements per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* F = reinterpret_cast<C*>(smem_raw);
    C* G = F + TI * SSTR;
    C* tab = G + TI * SSTR;  // per-pass twiddles (fft_block.cuh)
    const int tid = threadIdx.x;
    const int grp = WARP ? tid >> 5 : 0, gtid = WARP ? (tid & 31) : tid;
    const int kx = blockIdx.y, ky0 = blockIdx.x * TI;  // the ky tiles of one kx run together
    const int nz = a.nz, py = a.py;
    C* Fw = F + grp * GC * SSTR;  // this group's columns
    C* Gw = G + grp * GC * SSTR;

    build_tw_tab<C, LOGZ, NT>(tab, tw, a.tw_shift, tid);
    // column tile (TI columns of nz values, zero-padded to Pz) into buf
    auto load_tile = [&](C* buf, const C* src) {
        for (int e = tid; e < TI * PZ; e += NT) {
            const int i = e % TI, n = e / TI;
            C v = cmk<C>(0, 0);
            if (n < nz && ky0 + i < py) v = src[(size_t)n * py + ky0 + i];
            buf[i * SSTR + sidx<C>(n)] = v;
        }
    };
    auto store_tile = [&](const C* buf, C* dst) {
        for (int e = tid; e < TI * nz; e += NT) {
            const int i = e % TI, t = e / TI;
            if (ky0 + i < py) dst[(size_t)t * py + i] = buf[i * SSTR + sidx<C>(t)];
        }
    };
    // the spectrum values of slot c at this thread's elements e = gtid + GT it
    // of its group's columns (i = e / PZ, kz = e % PZ), as the real numbers v
    // with S = v or S = i v
    auto load_spec = [&](int c, R (&v)[IT]) {
        const R* base = spec3 + ((size_t)c * a.kx_count + kx) * a.jyc * a.jzc;
        const bool ov = (a.oddv_mask >> c) & 1u, ow = (a.oddw_mask >> c) & 1u;
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int e = gtid + GT * it;
            const int i = e / PZ, kz = e - i * PZ;
            const int ky = ky0 + grp * GC + i;
            R val = 0;
            if (ky < py) {
                const bool fy = ky > py / 2, fz = kz > PZ / 2;
                const int jy = fy ? py - ky : ky, jz = fz ? PZ - kz : kz;
                val = __ldg(base + (size_t)jy * a.jzc + jz);
                if ((fy && ov) != (fz && ow)) val = -val;
            }
            v[it] = val;
        }
    };

    if constexpr (!ADJ) {
        load_tile(F, in + (size_t)kx * nz * py);
        __syncthreads();  // the tile and the twiddle table are in place
        block_fft_tab<C, LOGZ, GC, GT, false>(Fw, SSTR, tab, gtid, Sync{});
        R v[IT];
        load_spec(0, v);
        for (int c = 0; c < a.ncomp; ++c) {
            const bool imag = (a.imag3_mask >> c) & 1u;
#pragma unroll
            for (int it = 0; it < IT; ++it) {
                const int e = gtid + GT * it;
                const int i = e / PZ, kz = e - i * PZ;
                const C f = Fw[i * SSTR + sidx<C>(kz)];
                Gw[i * SSTR + sidx<C>(kz)] = imag ? cmk<C>(-v[it] * f.y, v[it] * f.x)
                                                  : cmk<C>(v[it] * f.x, v[it] * f.y);
            }
            if (c + 1 < a.ncomp) load_spec(c + 1, v);  // in flight during the transform
            Sync{}();  // the group's products are in G
            block_fft_tab<C, LOGZ, GC, GT, true>(Gw, SSTR, tab, gtid, Sync{});
            __syncthreads();  // every warp's columns are transformed back
            store_tile(G, out + (((size_t)kx * a.ncomp + c) * nz) * py + ky0);
            __syncthreads();  // G is rewritten by the next component
        }
    } else {
        C g[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) g[it] = cmk<C>(0, 0);
        R v[IT];
        for (int c = 0; c < a.ncomp; ++c) {
            load_tile(F, in + (((size_t)kx * a.ncomp + c) * nz) * py);
            load_spec(c, v);  // in flight during the transform
            __syncthreads();  // the tile (and, the first time, the twiddle table) is in place
            block_fft_tab<C, LOGZ, GC, GT, false>(Fw, SSTR, tab, gtid, Sync{});
            const bool imag = (a.imag3_mask >> c) & 1u;
#pragma unroll
            for (int it = 0; it < IT; ++it) {
                const int e = gtid + GT * it;
                const int i = e / PZ, kz = e - i * PZ;
                const C f = Fw[i * SSTR + sidx<C>(kz)];
                // conj(S) f: S = v or S = i v
                g[it] = imag ? cmk<C>(g[it].x + v[it] * f.y, g[it].y - v[it] * f.x)
                             : cmk<C>(g[it].x + v[it] * f.x, g[it].y + v[it] * f.y);
            }
            __syncthreads();  // F is reloaded for the next component
        }
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int e = gtid + GT * it;
            const int i = e / PZ, kz = e - i * PZ;
            Gw[i * SSTR + sidx<C>(kz)] = g[it];
        }
        Sync{}();
        block_fft_tab<C, LOGZ, GC, GT, true>(Gw, SSTR, tab, gtid, Sync{});
        __syncthreads();
        store_tile(G, out + (size_t)kx * nz * py + ky0);
    }
}

// Pass C for Pz = 256 in FP32, transforms in registers.  A warp owns two
// columns of the tile; lane L works on column L / 16 with q = L % 16 and
// holds 16 of its values.  256 = 16 x 16 (the four-step form):
//   forward  x[q + 16 n2] -> 16-point DFT over n2 -> twiddle W_256^(q k2)
//            -> transpose through the warp's shared area (q <-> k2)
//            -> 16-point DFT over n1: lane q = k2 holds X[k2 + 16 k1] with
//            k1 = bitrev4(j) in register j;
//   inverse  from that layout: 16-point DFT over k1 -> twiddle W_256^(-a k2)
//            -> transpose -> 16-point DFT over k2: lane q = a holds
//            x[a + 16 b], b = bitrev4(j).
// Pz = 256 >= 2 nz - 1 gives nz <= 128, so the inputs x[q + 16 n2] with
// n2 >= 8 are zero (the first stage of the forward DFT only twiddles) and
// the stations kept are x[a + 16 b] with b < 8 (the even registers: the last
// stage of the inverse DFT keeps its sums).  Tiles of nz rows x 8 columns
// (a CTA of four warps) move between HBM and shared memory in rows of 64
// bytes; the CTA grid runs the ky tiles of one kx next to each other, so each
// kx's spectra are read from HBM once and served from L2 to both halves of
// every mirror pair.
constexpr int kZ2Warps = 4, kZ2Ti = 2 * kZ2Warps, kZ2Threads = 32 * kZ2Warps;
constexpr int kZ2Str = kZ2Ti + 1;              // staging tile row stride (complex)
constexpr int kZ2TrStr = 17;                   // transpose area row stride
constexpr int kZ2TrWarp = 2 * 16 * kZ2TrStr;   // complex values of a warp's transpose area
constexpr int kZ2MaxNz = 128;
constexpr int kZ2Stage = kZ2MaxNz * kZ2Str;    // complex values of one staging tile
// spectra of one component for the tile's columns, one row of Pz/2 + 1 = 129
// values per column (both mirror halves of kz read the same row), two
// components in flight
constexpr int kZ2SpS = 145;                    // floats per staged spectra row (129 used)
constexpr int kZ2Spec = kZ2Ti * kZ2SpS;        // floats of one component's staged spectra
constexpr size_t kZ2Smem = (size_t)(256 + kZ2Warps * kZ2TrWarp + 2 * kZ2Stage) * sizeof(float2) +
                           (size_t)2 * kZ2Spec * sizeof(float);
static_assert(kZ2Threads == 16 * kZ2Ti, "sixteen threads stage each spectra row");

// 16-point DFT in registers, radix-2 decimation in frequency: natural order
// in, u[j] = X[bitrev4(j)] out.  HALF: u[8..15] are zero on entry.  LOW:
// only X[m] with m < 8 (the even registers) are wanted on exit.
template <bool INV, bool HALF, bool LOW> __device__ __forceinline__ void dft16r(float2 (&u)[16]) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
#pragma unroll
        for (int b = 0; b < 16; b += 2 * h) {
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float2 x0 = u[b + i];
                if (HALF && h == 8) {
                    u[b + i + h] = tw32<INV>(x0, 2 * i);
                } else if (LOW && h == 1) {
                    u[b + i] = cadd(x0, u[b + i + h]);
                } else {
                    const float2 x1 = u[b + i + h];
                    u[b + i] = cadd(x0, x1);
                    u[b + i + h] = tw32<INV>(csub(x0, x1), 2 * i * (8 / h));
                }
            }
        }
    }
}

template <bool ADJ>
__global__ void __launch_bounds__(kZ2Threads, 16 / kZ2Warps)
    vol_z256_kernel(ZArgs a, const float2* __restrict__ in, float2* __restrict__ out, const float* __restrict__ spec3,
                    const float2* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* tab = reinterpret_cast<float2*>(smem_raw);  // tab[r * 16 + c] = W_256^(r c)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int col = lane >> 4, q = lane & 15;
    float2* tr = tab + 256 + warp * kZ2TrWarp + col * 16 * kZ2TrStr;  // this column's transpose area
    float2* stage = tab + 256 + kZ2Warps * kZ2TrWarp;                 // two [t][kZ2Str] tiles
    const int ky0 = blockIdx.x * kZ2Ti, kx = blockIdx.y;
    const int nz = a.nz, py = a.py;
    const int ci = 2 * warp + col, ky = ky0 + ci;
    const bool fy = ky > py / 2;

    for (int e = tid; e < 256; e += kZ2Threads) tab[e] = tw[((e >> 4) * (e & 15)) << a.tw_shift];

    // nz rows of the tile's 16 columns (zero beyond py) into a staging tile
    // A thread moves column ti = tid % kZ2Ti of the tile, rows tr0, tr0 +
    // kZ2Rs, ...: its shared and global addresses advance by fixed strides.
    constexpr int kZ2Rs = kZ2Threads / kZ2Ti;  // rows per pass of the CTA
    const int ti = tid % kZ2Ti, tr0 = tid / kZ2Ti;
    const bool ti_ok = ky0 + ti < py;
    const size_t gstep = (size_t)kZ2Rs * py;
    auto load_tile = [&](float2* st, const float2* src) {
        float2* sp = st + tr0 * kZ2Str + ti;
        const float2* gp = src + (size_t)tr0 * py + ky0 + ti;
        for (int n = tr0; n < nz; n += kZ2Rs, sp += kZ2Rs * kZ2Str, gp += gstep)
            *sp = ti_ok ? *gp : make_float2(0.f, 0.f);
    };
    // the same by per-thread asynchronous copies (one group per call)
    auto issue_tile = [&](float2* st, const float2* src) {
        float2* sp = st + tr0 * kZ2Str + ti;
        const float2* gp = src + (size_t)tr0 * py + (ti_ok ? ky0 + ti : 0);
        for (int n = tr0; n < nz; n += kZ2Rs, sp += kZ2Rs * kZ2Str, gp += gstep) async8_g2s(sp, gp, ti_ok);
        async8_commit();
    };
    auto store_tile = [&](const float2* st, float2* dst) {
        if (!ti_ok) return;
        const float2* sp = st + tr0 * kZ2Str + ti;
        float2* gp = dst + (size_t)tr0 * py + ky0 + ti;
        for (int t = tr0; t < nz; t += kZ2Rs, sp += kZ2Rs * kZ2Str, gp += gstep) *gp = *sp;
    };
    // forward transform of this lane's column from a staging tile
    auto fwd_fft = [&](const float2* st, float2 (&u)[16]) {
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            const int n = q + 16 * n2;
            u[n2] = n < nz ? st[n * kZ2Str + ci] : make_float2(0.f, 0.f);
        }
        dft16r<false, true, false>(u);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int k2 = bitrev4(j);
            tr[k2 * kZ2TrStr + q] = cmul(u[j], tab[k2 * 16 + q]);
        }
        __syncwarp();
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) u[n1] = tr[q * kZ2TrStr + n1];
        __syncwarp();
        dft16r<false, false, false>(u);
    };
    // inverse transform in place; the stations t = q + 16 bitrev4(j) < 128
    // are in the even registers j on exit
    auto inv_fft = [&](float2 (&g)[16]) {
        float2 h[16];
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) h[k1] = g[bitrev4(k1)];
        dft16r<true, false, false>(h);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int aa = bitrev4(j);
            tr[aa * kZ2TrStr + q] = cmul(h[j], cconj(tab[aa * 16 + q]));
        }
        __syncwarp();
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) g[k2] = tr[q * kZ2TrStr + k2];
        __syncwarp();
        dft16r<true, false, true>(g);
    };
    auto put_stations = [&](float2* st, const float2 (&g)[16]) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
            const int t = q + 16 * bitrev4(j);
            if (t < nz) st[t * kZ2Str + ci] = g[j];
        }
    };
    // spectrum of slot c at (ky, kz = q + 16 bitrev4(j)) as the real v with
    // S = v or S = i v
    // Spectra come into shared memory by per-thread asynchronous copies one
    // component ahead: thread tid stages row sr = tid / 16 (column ky0 + sr)
    // at jz = tid % 16 + 16 m; a row beyond py is zero-filled.
    float* specb = reinterpret_cast<float*>(stage + 2 * kZ2Stage);  // two [kZ2Ti][kZ2SpS]
    const int sr = tid >> 4, sz = tid & 15;
    const int sky = ky0 + sr;
    const bool s_ok = sky < py;
    const float* spec_row = spec3 + ((size_t)kx * a.jyc + (!s_ok ? 0 : (sky > py / 2 ? py - sky : sky))) * a.jzc;
    const size_t spec_slot = (size_t)a.kx_count * a.jyc * a.jzc;
    auto issue_spec = [&](int c, float* sb) {
        const float* src = spec_row + c * spec_slot + sz;
        uint32_t dst = smem_u32(sb + sr * kZ2SpS + sz);
        const uint32_t nb = s_ok ? 4u : 0u;
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            if (m < 8 || sz == 0)  // jz = sz + 16 m <= 128
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + 64u * m), "l"(src + 16 * m),
                             "r"(nb)
                             : "memory");
        }
        async8_commit();
    };
    // spectrum of slot c at (ky, kz = q + 16 bitrev4(j)) from staged row ci
    auto load_spec = [&](int c, const float* sb, float (&v)[16]) {
        const float* row = sb + ci * kZ2SpS;
        // the sign of S(ky, kz) against the stored value: flipped by the
        // y parity for ky > Py/2 and by the w parity for kz > Pz/2
        const bool s_lo = fy && ((a.oddv_mask >> c) & 1u);
        const bool s_hi = s_lo != (((a.oddw_mask >> c) & 1u) != 0);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int kz = q + 16 * bitrev4(j);
            const bool fz = kz > 128;
            const float val = row[fz ? 256 - kz : kz];
            v[j] = (fz ? s_hi : s_lo) ? -val : val;
        }
    };

    if constexpr (!ADJ) {
        float2* st_in = stage + kZ2Stage;
        issue_spec(0, specb);
        load_tile(st_in, in + (size_t)kx * nz * py);
        async8_wait_all();
        __syncthreads();  // the tile, component 0's spectra and the twiddle table are in place
        float2 X[16];
        fwd_fft(st_in, X);
        for (int c = 0; c < a.ncomp; ++c) {
            // the other spectra buffer was last read by component c - 1,
            // before the previous barrier
            if (c + 1 < a.ncomp) issue_spec(c + 1, specb + ((c + 1) & 1) * kZ2Spec);
            float v[16];
            load_spec(c, specb + (c & 1) * kZ2Spec, v);
            float2 g[16];
            if ((a.imag3_mask >> c) & 1u) {  // S = i v
#pragma unroll
                for (int j = 0; j < 16; ++j) g[j] = make_float2(-v[j] * X[j].y, v[j] * X[j].x);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) g[j] = make_float2(v[j] * X[j].x, v[j] * X[j].y);
            }
            inv_fft(g);
            // staging tile c % 2: its last reader (the store of component
            // c - 2, or the input read for c = 1) finished before the
            // previous barrier
            float2* st = stage + (c & 1) * kZ2Stage;
            put_stations(st, g);
            async8_wait_all();  // component c + 1's spectra, visible after the barrier
            __syncthreads();
            store_tile(st, out + ((size_t)kx * a.ncomp + c) * nz * py);
        }
    } else {
        float2 acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = make_float2(0.f, 0.f);
        // component c's tile is copied into staging tile c % 2 while
        // component c - 1 is transformed
        issue_tile(stage, in + (size_t)kx * a.ncomp * nz * py);
        issue_spec(0, specb);
        for (int c = 0; c < a.ncomp; ++c) {
            float2* st = stage + (c & 1) * kZ2Stage;
            async8_wait_all();
            // tile c and its spectra have landed everywhere, and every read of
            // tile c - 1 and its spectra (the other buffers) is done
            __syncthreads();
            if (c + 1 < a.ncomp) {
                issue_tile(stage + ((c + 1) & 1) * kZ2Stage, in + ((size_t)kx * a.ncomp + c + 1) * nz * py);
                issue_spec(c + 1, specb + ((c + 1) & 1) * kZ2Spec);
            }
            float2 f[16];
            fwd_fft(st, f);
            float v[16];
            load_spec(c, specb + (c & 1) * kZ2Spec, v);
            if ((a.imag3_mask >> c) & 1u) {  // conj(S) f with S = i v
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = make_float2(acc[j].x + v[j] * f[j].y, acc[j].y - v[j] * f[j].x);
            } else {  // S = v
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[j] = make_float2(acc[j].x + v[j] * f[j].x, acc[j].y + v[j] * f[j].y);
            }
        }
        inv_fft(acc);
        float2* st = stage + (a.ncomp & 1) * kZ2Stage;  // not the tile the last component read
        put_stations(st, acc);
        __syncthreads();
        store_tile(st, out + (size_t)kx * nz * py);
    }
}

// Plan creation, column step from half rows: Ehat[kx][o][b] holds only the
// rows b < N = Py/2 of each embedded kernel (row Py - b is row b times the
// component's sign in y, row Py/2 is zero).  CTA (kx, r, group of NSEQ
// layers) folds each column for ky parity r,
//   a[m] = (x[m] + (-1)^r x[m + N]) W_Py^(m r),  x[m + N] = sign x[N - m],
// runs the N-point FFT (bin q is ky = 2q + r) and stores the real or
// imaginary part of ky <= Py/2 as T[(kx * jyc + ky) * nzw + j0 + o].
template <int LOGN, int NSEQ>
__global__ void __launch_bounds__(kVolThreads) vol_spec_y2_kernel(const double2* __restrict__ ehat, int cnt, int j0,
                                                                  int nzw, bool imag2, bool oddv,
                                                                  double* __restrict__ T,
                                                                  const double2* __restrict__ tw, int tw_shift_n,
                                                                  int tw_shift_p) {
    constexpr int N = 1 << LOGN, SSTR = seq_stride<double2>(N), JYC = N + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int tid = threadIdx.x;
    const int kx = blockIdx.x, r = blockIdx.y, o0 = blockIdx.z * NSEQ;
    const double sgn = oddv ? -1.0 : 1.0;
    for (int e = tid; e < NSEQ * N; e += kVolThreads) {
        const int sq = e / N, m = e - sq * N, o = o0 + sq;
        double2 v = cmk<double2>(0, 0);
        if (o < cnt) {
            const double2* col = ehat + ((size_t)kx * cnt + o) * N;
            const double2 x0 = col[m];
            const double2 x1 = m ? cscale(col[N - m], sgn) : cmk<double2>(0, 0);
            v = r ? cmul(csub(x0, x1), tw[m << tw_shift_p]) : cadd(x0, x1);
        }
        buf[sq * SSTR + sidx<double2>(m)] = v;
    }
    __syncthreads();
    block_fft<double2, LOGN, NSEQ, kVolThreads, false>(buf, SSTR, tw, tw_shift_n, tid);
    const int nq = r ? N / 2 : N / 2 + 1;  // the bins 2q + r <= Py/2
#pragma unroll
    for (int sq = 0; sq < NSEQ; ++sq) {
        const int o = o0 + sq;
        if (o >= cnt) break;
        for (int q = tid; q < nq; q += kVolThreads) {
            const double2 z = buf[sq * SSTR + sidx<double2>(q)];
            T[((size_t)kx * JYC + 2 * q + r) * nzw + j0 + o] = imag2 ? z.y : z.x;
        }
    }
}

// Plan creation, z step: for every (kx, jy) row of T (2nz - 1 layer values,
// j = w + nz - 1), embed K(w) at (-w) mod Pz, transform (length Pz), and keep
// the real or imaginary part of kz <= Pz/2, scaled, as spec3[kx][jy][jz] of
// one component (S = imag2 ? i T : T per layer, so the transform gives the
// complex three-level spectrum itself).
template <typename RO, int LOGZ, int NSEQ>
__global__ void __launch_bounds__(kVolThreads) vol_spec_z_kernel(const double* __restrict__ T, long rows, int nz,
                                                                 bool imag2, bool imag3, double scale,
                                                                 RO* __restrict__ spec3,
                                                                 const double2* __restrict__ tw, int tw_shift) {
    constexpr int PZ = 1 << LOGZ, SSTR = seq_stride<double2>(PZ), JZC = PZ / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int tid = threadIdx.x;
    const int nzw = 2 * nz - 1;
    const long row0 = (long)blockIdx.x * NSEQ;
    block_fft_from<double2, LOGZ, NSEQ, kVolThreads, false>(buf, SSTR, tw, tw_shift, tid, [&](int s, int m) {
        const long k = row0 + s;
        int w;
        bool live = k < rows;
        if (m <= nz - 1) w = -m;
        else if (m >= PZ - nz + 1) w = PZ - m;
        else live = false;
        if (!live) return cmk<double2>(0, 0);
        const double v = T[k * nzw + w + nz - 1];
        return imag2 ? cmk<double2>(0, v) : cmk<double2>(v, 0);
    });
    for (int e = tid; e < NSEQ * JZC; e += kVolThreads) {
        const int s = e / JZC, kz = e - s * JZC;
        const long k = row0 + s;
        if (k >= rows) continue;
        const double2 v = buf[s * SSTR + sidx<double2>(kz)];
        spec3[k * JZC + kz] = (RO)((imag3 ? v.y : v.x) * scale);
    }
}

template <typename C, int LOGN, bool INV>
cudaError_t rows_launch(const void* in, size_t in_stride, int l_in, void* out, size_t out_stride, int l_out, long rows,
                        const void* tw, int tw_shift, cudaStream_t s) {
    constexpr int NSEQ = rows_nseq<C>(LOGN);
    constexpr auto k = vol_rows_kernel<C, LOGN, NSEQ, INV>;
    const size_t smem = (size_t)NSEQ * seq_stride<C>(1 << LOGN) * sizeof(C);
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    const long blocks = (rows + NSEQ - 1) / NSEQ;
    if (blocks == 0) return cudaSuccess;
    k<<<(unsigned)blocks, kVolThreads, smem, s>>>((const C*)in, in_stride, l_in, (C*)out, out_stride, l_out, rows,
                                                   (const C*)tw, tw_shift);
    return cudaGetLastError();
}

#define GRAV_VOL_LOG_CASES(X) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11)

template <int LOGN>
cudaError_t yinv_tiled_launch(const void* in, int R, int kx_count, int ny, void* out, const void* tw, int tw_shift,
                              cudaStream_t s) {
    constexpr auto k = vol_yinv_tiled_kernel<LOGN>;
    const size_t smem = (size_t)kYtSeqs * seq_stride<float2>(1 << LOGN) * sizeof(float2);
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    const dim3 grid((kx_count + kYtSeqs - 1) / kYtSeqs, R);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    k<<<grid, kVolThreads, smem, s>>>((const float2*)in, R, kx_count, ny, (float2*)out, (const float2*)tw, tw_shift);
    return cudaGetLastError();
}

// persistent grid: two CTAs per SM, at most one per group of rows
int yw_grid(long groups) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return (int)std::min<long>(groups, 2L * sms);
}

cudaError_t launch_vol_yinv_tiled(int logn, const void* in, int R, int kx_count, int ny, void* out, const void* tw,
                                  int log_t, cudaStream_t s) {
    if (logn == 11 && ny <= 1024) {
        constexpr auto k = vol_yinv2048_tiled_kernel;
        cudaError_t e = ensure_smem_limit<k>();
        if (e != cudaSuccess) return e;
        const int grid = yw_grid((long)((kx_count + kYwRows - 1) / kYwRows) * R);
        if (grid <= 0) return R ? cudaErrorInvalidValue : cudaSuccess;
        k<<<grid, kYwThreads, kYwSmem, s>>>((const float2*)in, R, kx_count, ny, (float2*)out, (const float2*)tw, log_t);
        return cudaGetLastError();
    }
    switch (logn) {
#define CASE(L) \
    case L: return yinv_tiled_launch<L>(in, R, kx_count, ny, out, tw, log_t - L, s);
        GRAV_VOL_LOG_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename C, bool INV>
cudaError_t launch_vol_rows(int logn, const void* in, size_t in_stride, int l_in, void* out, size_t out_stride,
                            int l_out, long rows, const void* tw, int log_t, cudaStream_t s) {
    switch (logn) {
#define CASE(L) \
    case L: return rows_launch<C, L, INV>(in, in_stride, l_in, out, out_stride, l_out, rows, tw, log_t - L, s);
        GRAV_VOL_LOG_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

// Pass B (and the adjoint's): column FFTs of `rows` rows of l_in <= ny
// values (row stride in_stride) into rows of Py values (stride out_stride).
template <typename C>
cudaError_t launch_vol_yfwd(int logn, const void* in, size_t in_stride, int l_in, void* out, size_t out_stride,
                            long rows, const void* tw, int log_t, cudaStream_t s) {
    if constexpr (std::is_same<C, float2>::value) {
        if (logn == 11 && l_in <= 1024 && out_stride % 2 == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
            constexpr auto k = vol_yfwd2048_kernel;
            cudaError_t e = ensure_smem_limit<k>();
            if (e != cudaSuccess) return e;
            const int grid = yw_grid((rows + kYwRows - 1) / kYwRows);
            if (grid <= 0) return rows ? cudaErrorInvalidValue : cudaSuccess;
            k<<<grid, kYwThreads, kYwSmem, s>>>((const float2*)in, in_stride, l_in, (float2*)out, out_stride, rows,
                                                (const float2*)tw, log_t);
            return cudaGetLastError();
        }
    }
    return launch_vol_rows<C, false>(logn, in, in_stride, l_in, out, out_stride, (int)out_stride, rows, tw, log_t, s);
}

template <typename R, int LOGZ, bool ADJ>
cudaError_t z_launch(const ZArgs& a, const void* in, void* out, const R* spec3, const void* tw, cudaStream_t s) {
    using C = typename cplx<R>::type;
    if constexpr (std::is_same<R, float>::value && LOGZ == 8) {
        constexpr auto k = vol_z256_kernel<ADJ>;
        cudaError_t e = ensure_smem_limit<k>();
        if (e != cudaSuccess) return e;
        k<<<dim3((a.py + kZ2Ti - 1) / kZ2Ti, a.kx_count), kZ2Threads, kZ2Smem, s>>>(a, (const float2*)in, (float2*)out,
                                                                                   spec3, (const float2*)tw);
        return cudaGetLastError();
    } else {
        constexpr int TI = z_tile<C>(LOGZ);
        constexpr int NT = z_threads(TI, LOGZ, sizeof(R) == 8);
        constexpr auto k = vol_z_kernel<R, LOGZ, TI, ADJ>;
        const size_t smem = ((size_t)2 * TI * seq_stride<C>(1 << LOGZ) + tw_tab_len(LOGZ)) * sizeof(C);
        cudaError_t e = ensure_smem_limit<k>();
        if (e != cudaSuccess) return e;
        k<<<dim3((a.py + TI - 1) / TI, a.kx_count), NT, smem, s>>>(a, (const C*)in, (C*)out, spec3, (const C*)tw);
        return cudaGetLastError();
    }
}

template <typename R, bool ADJ>
cudaError_t launch_vol_z(int logz, const ZArgs& a, const void* in, void* out, const R* spec3, const void* tw,
                         cudaStream_t s) {
    switch (logz) {
#define CASE(L) \
    case L: return z_launch<R, L, ADJ>(a, in, out, spec3, tw, s);
        GRAV_VOL_LOG_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

constexpr int kSpecY2Seqs = 4;

template <int LOGN>
cudaError_t spec_y2_launch(const void* ehat, int cnt, int kx_count, int j0, int nzw, bool imag2, bool oddv, double* T,
                           const void* tw64, int log_t, cudaStream_t s) {
    constexpr auto k = vol_spec_y2_kernel<LOGN, kSpecY2Seqs>;
    const size_t smem = (size_t)kSpecY2Seqs * seq_stride<double2>(1 << LOGN) * sizeof(double2);
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    const dim3 grid(kx_count, 2, (cnt + kSpecY2Seqs - 1) / kSpecY2Seqs);
    k<<<grid, kVolThreads, smem, s>>>((const double2*)ehat, cnt, j0, nzw, imag2, oddv, T, (const double2*)tw64,
                                      log_t - LOGN, log_t - (LOGN + 1));
    return cudaGetLastError();
}

// log_n = log2(Py / 2)
cudaError_t launch_spec_y2(int log_n, const void* ehat, int cnt, int kx_count, int j0, int nzw, bool imag2, bool oddv,
                           double* T, const void* tw64, int log_t, cudaStream_t s) {
    switch (log_n) {
#define CASE(L) \
    case L: return spec_y2_launch<L>(ehat, cnt, kx_count, j0, nzw, imag2, oddv, T, tw64, log_t, s);
        CASE(1) GRAV_VOL_LOG_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

template <typename RO, int LOGZ>
cudaError_t spec_z_launch(const double* T, long rows, int nz, bool imag2, bool imag3, double scale, RO* spec3,
                          const void* tw64, int log_t, cudaStream_t s) {
    constexpr int NSEQ = rows_nseq<double2>(LOGZ);
    constexpr auto k = vol_spec_z_kernel<RO, LOGZ, NSEQ>;
    const size_t smem = (size_t)NSEQ * seq_stride<double2>(1 << LOGZ) * sizeof(double2);
    cudaError_t e = ensure_smem_limit<k>();
    if (e != cudaSuccess) return e;
    k<<<(unsigned)((rows + NSEQ - 1) / NSEQ), kVolThreads, smem, s>>>(T, rows, nz, imag2, imag3, scale, spec3,
                                                                       (const double2*)tw64, log_t - LOGZ);
    return cudaGetLastError();
}


template <typename RO>
cudaError_t launch_spec_z(int logz, const double* T, long rows, int nz, bool imag2, bool imag3, double scale,
                          RO* spec3, const void* tw64, int log_t, cudaStream_t s) {
    switch (logz) {
#define CASE(L) \
    case L: return spec_z_launch<RO, L>(T, rows, nz, imag2, imag3, scale, spec3, tw64, log_t, s);
        GRAV_VOL_LOG_CASES(CASE)
#undef CASE
        default: return cudaErrorInvalidValue;
    }
}

// Per-call workspaces (complex elements of the plan's type): A holds X then
// W (forward) or X' then W' (adjoint); B holds U then V (forward) or U' then
// V' (adjoint).
size_t vol_ws_a_elems(const grav_plan* p) {
    const size_t kx = p->kx_count, nz = p->nz, nc = p->ncomp;
    const size_t x = kx * nc * nz * p->ny_pad;  // X' (the larger of X and X')
    const size_t w = kx * nc * nz * p->py;      // W (the larger of W and W')
    return x > w ? x : w;
}
size_t vol_ws_b_elems(const grav_plan* p) {
    const size_t kx = p->kx_count, nz = p->nz, nc = p->ncomp;
    const size_t u = kx * nc * nz * p->py;                          // U' (the largest of U, U', V and V')
    const size_t v = kx * nc * nz * (((size_t)p->ny + 7) / 8 * 8);  // V in the tiled layout
    return u > v ? u : v;
}

// Whether passes D and E take the tiled layout and the tiled inverse row
// kernel (FP32 plans with Px = 2048).
bool vol_tiled_rows(const grav_plan* p) { return !p->fp64 && p->kx_count == 1025 && p->nx <= 1024; }

template <typename R>
int make_spectra3(grav_plan* p) {
    const int nzw = 2 * p->nz - 1;
    const int jyc = p->py / 2 + 1, jzc = p->pz / 2 + 1;
    // FP64 staging per chunk of layers of one component: the rows b < Py/2
    // of the embedded kernels and their row transforms, bounded to about
    // 2 GB; plus the column-step output T of one component.
    const int hy = p->py / 2;
    const size_t per_layer = (size_t)hy * p->px * sizeof(double) + (size_t)p->kx_count * hy * 2 * sizeof(double);
    int nzc = (int)(((size_t)2 << 30) / per_layer);
    if (nzc < 1) nzc = 1;
    if (nzc > nzw) nzc = nzw;
    if (nzc > 65535) nzc = 65535;
    void* tw64 = nullptr;
    size_t tw64_bytes = 0;
    int rc = GRAV_OK;
    if (p->fp64) {
        tw64 = p->tw;
    } else if ((rc = build_twiddles(p->log_t, 1, &tw64, &tw64_bytes)) != GRAV_OK) {
        return rc;
    }
    void *E = nullptr, *Ehat = nullptr, *T = nullptr;
    const size_t e_bytes = (size_t)nzc * hy * p->px * sizeof(double);
    const size_t eh_bytes = (size_t)p->kx_count * nzc * hy * 2 * sizeof(double);
    const size_t t_bytes = (size_t)p->kx_count * jyc * nzw * sizeof(double);
    if ((rc = dev_alloc_raw(&E, e_bytes, "kernel staging")) == GRAV_OK &&
        (rc = dev_alloc_raw(&Ehat, eh_bytes, "kernel row-transform staging")) == GRAV_OK &&
        (rc = dev_alloc_raw(&T, t_bytes, "kernel column-transform staging")) == GRAV_OK) {
        cudaStream_t s;
        cudaError_t ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            rc = cuda_fail(ce, "cudaStreamCreate");
        } else {
            // the plane generator with 2nz - 1 layers seen from h' = -(nz - 1/2) dz
            const Geometry g{p->nx, p->ny, nzw, p->dx, p->dy, p->dz, -(p->nz - 0.5) * p->dz};
            const double scale = 1.0 / ((double)p->px * (double)p->py * (double)p->pz);
            for (int slot = 0; slot < p->ncomp && rc == GRAV_OK; ++slot) {
                const int c = p->comp_id[slot];
                const bool imag2 = odd_u(c) != odd_v(c);
                const bool imag3 = (p->imag3_mask >> slot) & 1u;
                for (int j0 = 0; j0 < nzw && rc == GRAV_OK; j0 += nzc) {
                    const int j1 = j0 + nzc < nzw ? j0 + nzc : nzw;
                    const int cnt = j1 - j0;
                    if ((ce = cudaMemsetAsync(E, 0, (size_t)cnt * hy * p->px * sizeof(double), s)) != cudaSuccess) {
                        rc = cuda_fail(ce, "cudaMemsetAsync(kernel staging)");
                        break;
                    }
                    if ((ce = launch_kernel_gen(g, 1u << c, j0, j1, 2, p->px, p->py, (double*)E, s)) != cudaSuccess) {
                        rc = cuda_fail(ce, "kernel generation launch");
                        break;
                    }
                    if ((ce = launch_row_r2c<double>(p->log_px, (const double*)E, (size_t)hy * p->px, (size_t)p->px,
                                                     p->px, hy, cnt, Ehat, hy, tw64, p->log_t, s)) != cudaSuccess) {
                        rc = cuda_fail(ce, "kernel row transform launch");
                        break;
                    }
                    if ((ce = launch_spec_y2(p->log_py - 1, Ehat, cnt, p->kx_count, j0, nzw, imag2, odd_v(c),
                                             (double*)T, tw64, p->log_t, s)) != cudaSuccess) {
                        rc = cuda_fail(ce, "kernel column transform launch");
                        break;
                    }
                }
                if (rc != GRAV_OK) break;
                R* dst = (R*)p->spec + (size_t)slot * p->kx_count * jyc * jzc;
                if ((ce = launch_spec_z<R>(p->log_pz, (const double*)T, (long)p->kx_count * jyc, p->nz, imag2, imag3,
                                           scale, dst, tw64, p->log_t, s)) != cudaSuccess) {
                    rc = cuda_fail(ce, "kernel layer transform launch");
                    break;
                }
            }
            ce = cudaStreamSynchronize(s);
            if (rc == GRAV_OK && ce != cudaSuccess) rc = cuda_fail(ce, "plan construction");
            cudaStreamDestroy(s);
        }
    }
    cudaFree(E);
    cudaFree(Ehat);
    cudaFree(T);
    if (!p->fp64) cudaFree(tw64);
    return rc;
}

ZArgs z_args(const grav_plan* p) {
    ZArgs a{};
    a.nz = p->nz;
    a.py = p->py;
    a.kx_count = p->kx_count;
    a.ncomp = p->ncomp;
    a.jyc = p->py / 2 + 1;
    a.jzc = p->pz / 2 + 1;
    a.imag3_mask = p->imag3_mask;
    a.oddv_mask = p->oddv_mask;
    a.oddw_mask = p->oddw_mask;
    a.tw_shift = p->log_t - p->log_pz;
    return a;
}

template <typename R>
int run_forward3d(grav_plan* p, const void* rho, void* out, cudaStream_t s) {
    using C = typename cplx<R>::type;
    const size_t kx = p->kx_count, nz = p->nz, nc = p->ncomp;
    void* A = p->ws_a;
    void* B = p->ws_b;
    cudaError_t e;
    // A: x
    e = launch_row_r2c<R>(p->log_px, (const R*)rho, (size_t)p->ny * p->nx, (size_t)p->nx, p->nx, p->ny, p->nz, A,
                          p->ny_pad, p->tw, p->log_t, s, Batch(), p->err_flag);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension forward: row transforms");
    // B: y
    e = launch_vol_yfwd<C>(p->log_py, A, p->ny_pad, p->ny, B, p->py, (long)(kx * nz), p->tw, p->log_t, s);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension forward: column transforms");
    // C: z, product, inverse z
    e = launch_vol_z<R, false>(p->log_pz, z_args(p), B, A, (const R*)p->spec, p->tw, s);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension forward: layer transforms");
    if constexpr (std::is_same<R, float>::value) {
        if (vol_tiled_rows(p)) {
            // D: inverse y into the tiled layout; E: inverse x from it
            e = launch_vol_yinv_tiled(p->log_py, A, (int)(nc * nz), p->kx_count, p->ny, B, p->tw, p->log_t, s);
            if (e != cudaSuccess) return cuda_fail(e, "equal-dimension forward: inverse column transforms");
            e = launch_row_c2r_tiled(B, nullptr, p->ny, (int)(nc * nz), p->kx_count, (float*)out, (size_t)p->nx,
                                     p->nx, p->tw, p->log_t, s, Batch(), p->err_flag);
            if (e != cudaSuccess) return cuda_fail(e, "equal-dimension forward: inverse row transforms");
            return GRAV_OK;
        }
    }
    // D: inverse y
    e = launch_vol_rows<C, true>(p->log_py, A, p->py, p->py, B, p->ny_pad, p->ny, (long)(kx * nc * nz), p->tw,
                                 p->log_t, s);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension forward: inverse column transforms");
    // E: inverse x
    e = launch_row_c2r<R>(p->log_px, B, nullptr, p->ny, (int)(nc * nz), p->ny_pad, (R*)out, (size_t)p->nx, p->nx,
                          p->tw, p->log_t, s);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension forward: inverse row transforms");
    return GRAV_OK;
}

template <typename R>
int run_adjoint3d(grav_plan* p, const void* r, void* grad, cudaStream_t s) {
    using C = typename cplx<R>::type;
    const size_t kx = p->kx_count, nz = p->nz, nc = p->ncomp;
    void* A = p->ws_a;
    void* B = p->ws_b;
    cudaError_t e;
    e = launch_row_r2c<R>(p->log_px, (const R*)r, (size_t)p->ny * p->nx, (size_t)p->nx, p->nx, p->ny, (int)(nc * nz),
                          A, p->ny_pad, p->tw, p->log_t, s, Batch(), p->err_flag);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension adjoint: row transforms");
    e = launch_vol_yfwd<C>(p->log_py, A, p->ny_pad, p->ny, B, p->py, (long)(kx * nc * nz), p->tw, p->log_t, s);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension adjoint: column transforms");
    e = launch_vol_z<R, true>(p->log_pz, z_args(p), B, A, (const R*)p->spec, p->tw, s);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension adjoint: layer transforms");
    if constexpr (std::is_same<R, float>::value) {
        if (vol_tiled_rows(p)) {
            e = launch_vol_yinv_tiled(p->log_py, A, (int)nz, p->kx_count, p->ny, B, p->tw, p->log_t, s);
            if (e != cudaSuccess) return cuda_fail(e, "equal-dimension adjoint: inverse column transforms");
            e = launch_row_c2r_tiled(B, nullptr, p->ny, p->nz, p->kx_count, (float*)grad, (size_t)p->nx, p->nx,
                                     p->tw, p->log_t, s, Batch(), p->err_flag);
            if (e != cudaSuccess) return cuda_fail(e, "equal-dimension adjoint: inverse row transforms");
            return GRAV_OK;
        }
    }
    e = launch_vol_rows<C, true>(p->log_py, A, p->py, p->py, B, p->ny_pad, p->ny, (long)(kx * nz), p->tw, p->log_t, s);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension adjoint: inverse column transforms");
    e = launch_row_c2r<R>(p->log_px, B, nullptr, p->ny, p->nz, p->ny_pad, (R*)grad, (size_t)p->nx, p->nx, p->tw,
                          p->log_t, s);
    if (e != cudaSuccess) return cuda_fail(e, "equal-dimension adjoint: inverse row transforms");
    return GRAV_OK;
}

int check_volume_call(grav_plan* plan, const void* in, void* out, const char* name) {
    if (!plan || !in || !out) {
        set_error("%s: null plan or buffer", name);
        return GRAV_EINVAL;
    }
    if (plan->kind != 1) {
        set_error("%s: the plan was made by grav_plan_create, not grav_plan_create3d", name);
        return GRAV_EINVAL;
    }
    return GRAV_OK;
}

}  // namespace

}  // namespace grav

using namespace grav;

extern "C" {

grav_plan* grav_plan_create3d(int nx, int ny, int nz, double dx, double dy, double dz, unsigned components) {
    set_error("%s", "");
    if (check_geometry(nx, ny, nz, dx, dy, dz, 1.0, components)) return nullptr;
    if (nx > kVolMaxNx || ny > kVolMaxNy || nz > kVolMaxNz) {
        set_error("equal-dimension mesh %dx%dx%d beyond %dx%dx%d", nx, ny, nz, kVolMaxNx, kVolMaxNy, kVolMaxNz);
        return nullptr;
    }
    grav_plan* p = new (std::nothrow) grav_plan();
    if (!p) {
        set_error("host allocation of the plan failed");
        return nullptr;
    }
    p->kind = 1;
    p->nx = nx; p->ny = ny; p->nz = nz;
    p->dx = dx; p->dy = dy; p->dz = dz; p->h = 0.0;
    p->comps = components & kCompBits;
    p->fp64 = (components & GRAV_FP64_SPECTRAL) ? 1 : 0;
    for (int c = 0; c < kMaxComp; ++c) {
        if (p->comps & (1u << c)) {
            const int s = p->ncomp++;
            p->comp_id[s] = c;
            if (odd_u(c) != odd_v(c)) p->imag_mask |= 1u << s;
            if (odd_v(c)) p->oddv_mask |= 1u << s;
            if (odd_w(c)) p->oddw_mask |= 1u << s;
            if ((int)odd_u(c) + (int)odd_v(c) + (int)odd_w(c) == 1 ||
                (int)odd_u(c) + (int)odd_v(c) + (int)odd_w(c) == 3)
                p->imag3_mask |= 1u << s;
        }
    }
    p->px = circulant_size(nx);
    p->py = circulant_size(ny);
    p->pz = circulant_size(nz);
    p->log_px = ilog2(p->px);
    p->log_py = ilog2(p->py);
    p->log_pz = ilog2(p->pz);
    p->log_t = p->log_px;
    if (p->log_py > p->log_t) p->log_t = p->log_py;
    if (p->log_pz > p->log_t) p->log_t = p->log_pz;
    p->kx_count = p->px / 2 + 1;
    p->ny_pad = (int)round_up((size_t)ny, 4);
    cudaGetDevice(&p->device);

    const size_t real = p->fp64 ? sizeof(double) : sizeof(float);
    p->spec_bytes = (size_t)p->ncomp * p->kx_count * (p->py / 2 + 1) * (p->pz / 2 + 1) * real;
    p->ws_a_bytes = vol_ws_a_elems(p) * 2 * real;
    p->ws_b_bytes = vol_ws_b_elems(p) * 2 * real;

    size_t free_b = 0, total_b = 0;
    cudaError_t ce = cudaMemGetInfo(&free_b, &total_b);
    if (ce != cudaSuccess) {
        cuda_fail(ce, "cudaMemGetInfo");
        delete p;
        return nullptr;
    }
    const size_t need = p->spec_bytes + p->ws_a_bytes + p->ws_b_bytes;
    if (need > free_b) {
        set_error("plan needs %zu bytes of device memory, %zu free", need, free_b);
        delete p;
        return nullptr;
    }
    int rc = build_twiddles(p->log_t, p->fp64, &p->tw, &p->tw_bytes);
    if (!rc) rc = dev_alloc_raw(&p->spec, p->spec_bytes, "kernel spectra");
    if (!rc) rc = dev_alloc_raw(&p->ws_a, p->ws_a_bytes, "workspace A");
    if (!rc) rc = dev_alloc_raw(&p->ws_b, p->ws_b_bytes, "workspace B");
    if (!rc) rc = dev_alloc_raw((void**)&p->err_flag, 256, "error flag");
    if (!rc) {
        cudaError_t me = cudaMemset(p->err_flag, 0, 256);
        if (me != cudaSuccess) rc = cuda_fail(me, "cudaMemset(error flag)");
    }
    if (!rc) rc = p->fp64 ? make_spectra3<double>(p) : make_spectra3<float>(p);
    if (rc) {
        free_plan(p);
        return nullptr;
    }
    return p;
}

int grav_forward3d(grav_plan* plan, const void* rho_dev, void* out_dev, void* stream) {
    int rc = check_volume_call(plan, rho_dev, out_dev, "grav_forward3d");
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    return plan->fp64 ? run_forward3d<double>(plan, rho_dev, out_dev, s)
                      : run_forward3d<float>(plan, rho_dev, out_dev, s);
}

int grav_adjoint3d(grav_plan* plan, const void* r_dev, void* grad_dev, void* stream) {
    int rc = check_volume_call(plan, r_dev, grad_dev, "grav_adjoint3d");
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    return plan->fp64 ? run_adjoint3d<double>(plan, r_dev, grad_dev, s)
                      : run_adjoint3d<float>(plan, r_dev, grad_dev, s);
}

}  // extern "C"
