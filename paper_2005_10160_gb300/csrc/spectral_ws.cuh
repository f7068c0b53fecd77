// Warp-specialised forward column stage for the large transforms (N = Py/2
// of 512 or 1024 points, FP32): the same arithmetic as forward_column_kernel
// (column FFT of each layer's row transforms, product with the stored
// spectra, compensated sum over layers, Eq. 21), split across three roles
// that run concurrently inside one CTA and hand data over through
// shared-memory rings guarded by mbarriers:
//
//   producer warp   lane 0 streams each layer's row-transform column (X ring)
//                   and spectra slab (S ring) with bulk asynchronous copies,
//                   as far ahead as the rings allow;
//   FFT groups      GROUPS groups of NTG threads; group g transforms layers
//                   g, g + GROUPS, ... from the X ring into the F ring, with
//                   barriers among its own warps only;
//   MAC warps       J threads, thread q owning mirror pair q for every
//                   component, consume the F and S rings layer by layer.
//
// The main loop has no block-wide barrier, so the waits of one role overlap
// with the work of the others.  Every wait is bounded; a wait that runs out
// sets a shared abort flag that every other wait checks, so all roles leave
// promptly, the copies still in flight are allowed to land, and the plan's
// error flag records the failure.
//
// The layer sum is compensated per block of eight layers: each block's terms
// are added in registers and the block total enters a Kahan sum whose
// correction terms live in shared memory (they are touched once per block).
#pragma once
#include "async_copy.cuh"
#include "fft_block.cuh"
#include "grav_internal.h"
#include "spectral.cuh"

namespace grav {

template <int LOGN> struct WsShape {
    static constexpr int N = 1 << LOGN;
    static constexpr int J = N / 2;          // MAC threads: one mirror pair each
    static constexpr int GROUPS = 4;         // FFT groups, one layer each in flight
    static constexpr int NTG = N / 16;       // threads per group: two radix-8 butterflies each
    static constexpr int NF = GROUPS * NTG;  // FFT threads
    static constexpr int NT = J + NF + 32;   // plus the producer warp
};

// Shared-memory layout, chosen on the host (depths of the three rings).
struct WsSmem {
    int dx, ds, df;
    uint32_t x_bytes, s_bytes, f_bytes;
    uint32_t s_off, f_off, tw_off, cmp_off, bar_off, flag_off, total;
};

constexpr int kBlockLayers = 8;  // layers per compensated block

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up as soon as another thread has aborted.
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        if (mbar_try_wait_sleep(bar, parity, kSleepHintNs)) return true;
        if (*abort) return false;
        if (global_ns() - t0 > kWaitLimitNs) break;
    }
    *abort = 1;
    return false;
}

template <int LOGN, int NC>
__global__ void __launch_bounds__(WsShape<LOGN>::NT, 1) __maxnreg__(65536 / WsShape<LOGN>::NT / 8 * 8)
    forward_column_ws_kernel(ColumnArgs a, WsSmem L, const float2* __restrict__ X, const float* __restrict__ spec,
                             float2* __restrict__ Y, const float2* __restrict__ tw, int* __restrict__ err,
                             size_t x_bstride, size_t y_bstride) {
    using C = float2;
    using S = WsShape<LOGN>;
    constexpr int N = S::N, J = S::J, GROUPS = S::GROUPS, NTG = S::NTG, NF = S::NF, NT = S::NT;
    constexpr int SSTR = spad_len<C>(N);
    static_assert(NTG % 32 == 0, "FFT groups are whole warps");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* xring = smem;
    unsigned char* sring = smem + L.s_off;
    C* fring = reinterpret_cast<C*>(smem + L.f_off);
    C* tws = reinterpret_cast<C*>(smem + L.tw_off);  // fold twiddles W_Py^m, m < N
    C* ttab = tws + N;                                  // per-pass FFT twiddles
    float* cmp = reinterpret_cast<float*>(smem + L.cmp_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* xfull = bars;
    uint64_t* xempty = xfull + L.dx;
    uint64_t* sfull = xempty + L.dx;
    uint64_t* sempty = sfull + L.ds;
    uint64_t* ffull = sempty + L.ds;
    uint64_t* fempty = ffull + L.df;
    volatile int* abort = reinterpret_cast<volatile int*>(smem + L.flag_off);
    volatile int* gflag = abort + 1;  // per FFT group: the leader's wait result

    const int tid = threadIdx.x;
    const int r = blockIdx.x & 1, kx = blockIdx.x >> 1;
    const int nz = a.nz, ny = a.ny;
    X += blockIdx.y * x_bstride;  // request of a batched call
    Y += blockIdx.y * y_bstride;
    const C* Xk = X + (size_t)kx * nz * a.ny_pad;
    const size_t s_row = (size_t)a.ncomp * a.jp;
    const float* Sk = request_spec(a, spec, blockIdx.y) + (size_t)(r * a.kx_count + kx) * nz * s_row;

    if (tid == 0) {
        for (int s = 0; s < L.dx; ++s) {
            mbar_init(&xfull[s], 1);
            mbar_init(&xempty[s], NTG);
        }
        for (int s = 0; s < L.ds; ++s) {
            mbar_init(&sfull[s], 1);
            mbar_init(&sempty[s], J);
        }
        for (int s = 0; s < L.df; ++s) {
            mbar_init(&ffull[s], NTG);
            mbar_init(&fempty[s], J);
        }
        *abort = 0;
        fence_mbar_init();
    }
    for (int e = tid; e < N; e += NT) tws[e] = tw[e << a.tw_shift_p];
    build_tw_tab<C, LOGN, NT>(ttab, tw, a.tw_shift_n, tid);
    for (int e = tid; e < 4 * NC * J; e += NT) cmp[e] = 0.f;
    __syncthreads();

    bool failed = false;
    int nx_i = 0, ns_i = 0;  // producer: copies issued so far
    float acc[NC][4];
    int k1 = 0, k2 = 0;
    const bool is_mac = tid < J;
    const bool nyq = is_mac && r == 0 && tid == 0;

    if (tid >= J + NF) {
        // ---------------- producer: lane 0 of the last warp ----------------
        if (tid == J + NF) {
            uint64_t t_last = global_ns();
            while (nx_i < nz || ns_i < nz) {
                bool progressed = false;
                if (nx_i < nz) {
                    const int s = nx_i % L.dx, use = nx_i / L.dx;
                    if (use == 0 || mbar_try_wait(&xempty[s], (uint32_t)((use - 1) & 1))) {
                        fence_proxy_async_smem();
                        mbar_arrive_expect_tx(&xfull[s], L.x_bytes);
                        bulk_g2s(xring + (size_t)s * L.x_bytes, Xk + (size_t)nx_i * a.ny_pad, L.x_bytes, &xfull[s]);
                        ++nx_i;
                        progressed = true;
                    }
                }
                if (ns_i < nz) {
                    const int s = ns_i % L.ds, use = ns_i / L.ds;
                    if (use == 0 || mbar_try_wait(&sempty[s], (uint32_t)((use - 1) & 1))) {
                        fence_proxy_async_smem();
                        mbar_arrive_expect_tx(&sfull[s], L.s_bytes);
                        bulk_g2s(sring + (size_t)s * L.s_bytes, Sk + (size_t)ns_i * s_row, L.s_bytes, &sfull[s]);
                        ++ns_i;
                        progressed = true;
                    }
                }
                if (progressed) {
                    t_last = global_ns();
                } else {
                    __nanosleep(256);  // both rings full: back off
                    if (*abort) break;
                    if (global_ns() - t_last > kWaitLimitNs) {
                        *abort = 1;
                        break;
                    }
                }
            }
            failed = *abort != 0;
        }
    } else if (!is_mac) {
        // ---------------- FFT group g ----------------
        const int g = (tid - J) / NTG, lt = (tid - J) - g * NTG;
        const GroupSync gs{1 + g, NTG};
        for (int n = g; n < nz; n += GROUPS) {
            const int sx = n % L.dx, sf = n % L.df;
            if (lt == 0) {
                bool ok = ws_wait(&xfull[sx], (uint32_t)((n / L.dx) & 1), abort);
                if (ok && n >= L.df) ok = ws_wait(&fempty[sf], (uint32_t)((n / L.df - 1) & 1), abort);
                gflag[g] = ok ? 1 : 0;
            }
            gs();
            if (!gflag[g]) {
                failed = true;
                break;
            }
            const C* xs = reinterpret_cast<const C*>(xring + (size_t)sx * L.x_bytes);
            C* fb = fring + sf * SSTR;
            fft_first_pass_from<C, LOGN, pass_radix(LOGN, 0), 1, NTG, false>(
                fb, SSTR, lt,
                [&](int, int m) {
                    C v = make_float2(0.f, 0.f);
                    if (m < ny) {
                        v = xs[m];
                        if (r) v = cmul(v, tws[m]);
                    }
                    return v;
                },
                gs);
            mbar_arrive(&xempty[sx]);  // this thread's reads of the X slot are done
            fft_tail_tab<C, LOGN, 1, NTG, false>(fb, SSTR, ttab, lt, gs);
            mbar_arrive(&ffull[sf]);  // this thread's writes of the F slot are done
        }
    } else {
        // ---------------- MAC: thread q owns mirror pair q ----------------
        const int q = tid;
        pair_pos<N>(q, r, k1, k2);
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[c][j] = 0.f;
        float part[NC][4];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[c][j] = 0.f;
        for (int n = 0; n < nz; ++n) {
            const int sf = n % L.df, ss = n % L.ds;
            if (!ws_wait(&ffull[sf], (uint32_t)((n / L.df) & 1), abort) ||
                !ws_wait(&sfull[ss], (uint32_t)((n / L.ds) & 1), abort)) {
                failed = true;
                break;
            }
            const C* fb = fring + sf * SSTR;
            const C v1 = fb[sidx<C>(k1)], v2 = fb[sidx<C>(k2)];
            const float* Ss = reinterpret_cast<const float*>(sring + (size_t)ss * L.s_bytes) + q;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const float s1 = Ss[c * a.jp];
                const float s2 = nyq ? Ss[c * a.jp + J] : s1;
                part[c][0] += s1 * v1.x;
                part[c][1] += s1 * v1.y;
                part[c][2] += s2 * v2.x;
                part[c][3] += s2 * v2.y;
            }
            mbar_arrive(&fempty[sf]);
            mbar_arrive(&sempty[ss]);
            if ((n % kBlockLayers) == kBlockLayers - 1 || n == nz - 1) {
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
    }

    if (__syncthreads_or(failed || *abort)) {
        if (tid == J + NF) {
            // let the copies that were issued land (bounded) before the CTA's
            // shared memory is released
            atomicExch(err, 1);
            // the most recent copy issued into each slot
            for (int n = nx_i - L.dx < 0 ? 0 : nx_i - L.dx; n < nx_i; ++n)
                mbar_wait_bounded(&xfull[n % L.dx], (uint32_t)((n / L.dx) & 1), kWaitLimitNs);
            for (int n = ns_i - L.ds < 0 ? 0 : ns_i - L.ds; n < ns_i; ++n)
                mbar_wait_bounded(&sfull[n % L.ds], (uint32_t)((n / L.ds) & 1), kWaitLimitNs);
        }
        return;
    }

    // Inverse column transforms, GROUPS components per round: the MAC threads
    // write their compensated sums (times i for imaginary spectra, with the
    // mirror sign for odd components) into the F slots, the FFT groups
    // transform them and write the rows y < ny.
#pragma unroll
    for (int c0 = 0; c0 < NC; c0 += GROUPS) {
        if (is_mac) {
#pragma unroll
            for (int l = 0; l < GROUPS; ++l) {
                const int c = c0 + l;
                if (c < NC) {
                    float e[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) e[j] = acc[c][j] - cmp[(c * 4 + j) * J + tid];
                    const bool imag = (a.imag_mask >> c) & 1u;
                    const bool flip = !nyq && ((a.oddv_mask >> c) & 1u);
                    C b1 = make_float2(e[0], e[1]), b2 = make_float2(e[2], e[3]);
                    if (flip) b2 = make_float2(-b2.x, -b2.y);
                    if (imag) {
                        b1 = make_float2(-b1.y, b1.x);
                        b2 = make_float2(-b2.y, b2.x);
                    }
                    C* fb = fring + l * SSTR;
                    fb[sidx<C>(k1)] = b1;
                    fb[sidx<C>(k2)] = b2;
                }
            }
        }
        __syncthreads();
        if (!is_mac && tid < J + NF) {
            const int g = (tid - J) / NTG, lt = (tid - J) - g * NTG;
            const int c = c0 + g;
            if (c < NC) {
                C* fb = fring + g * SSTR;
                block_fft_tab<C, LOGN, 1, NTG, true>(fb, SSTR, ttab, lt, GroupSync{1 + g, NTG});
                C* dst = Y + ((size_t)(r * a.kx_count + kx) * a.ncomp + c) * a.ny_pad;
                for (int y = lt; y < ny; y += NTG) {
                    C v = fb[sidx<C>(y)];
                    if (r) v = cmul(v, cconj(tws[y]));
                    dst[y] = v;
                }
            }
        }
        __syncthreads();
    }
}

// Ring depths and offsets; ds == 0 when nothing fits.
template <int LOGN>
WsSmem ws_smem(int ny_pad, int ncomp, int jp, int nc_inst, int max_bytes) {
    using S = WsShape<LOGN>;
    WsSmem L{};
    L.x_bytes = (uint32_t)(ny_pad * sizeof(float2));
    L.s_bytes = (uint32_t)(ncomp * jp * sizeof(float));
    L.f_bytes = (uint32_t)(spad_len<float2>(S::N) * sizeof(float2));
    const uint32_t tw_bytes = (uint32_t)((S::N + tw_tab_len(LOGN)) * sizeof(float2));
    const uint32_t cmp_bytes = (uint32_t)(4 * nc_inst * S::J * sizeof(float));
    auto layout = [&](int dx, int ds, int df) {
        WsSmem l = L;
        l.dx = dx;
        l.ds = ds;
        l.df = df;
        l.s_off = (uint32_t)(dx * L.x_bytes + 127) & ~127u;
        l.f_off = (uint32_t)(l.s_off + ds * L.s_bytes + 127) & ~127u;
        l.tw_off = l.f_off + df * L.f_bytes;
        l.cmp_off = (l.tw_off + tw_bytes + 15u) & ~15u;
        l.bar_off = (l.cmp_off + cmp_bytes + 7u) & ~7u;
        l.flag_off = l.bar_off + 2 * (dx + ds + df) * 8;
        l.total = l.flag_off + (1 + S::GROUPS) * 4;
        return l;
    };
    const int cands[][3] = {{8, 6, 6}, {6, 6, 6}, {6, 4, 6}, {6, 4, 5}, {4, 4, 5}, {4, 3, 4}, {4, 2, 4}};
    for (const auto& c : cands) {
        WsSmem l = layout(c[0], c[1], c[2]);
        if ((int)l.total <= max_bytes) return l;
    }
    return WsSmem{};
}

}  // namespace grav
