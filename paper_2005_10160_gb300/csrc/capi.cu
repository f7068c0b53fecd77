// C ABI of the library (include/grav.h): plan construction (kernel
// generation, circulant embedding and kernel spectra, Eqs. 10, 19, 22) and
// the per-call forward (Eq. 21) and adjoint pipelines.
//
// Forward, per call, on the caller's stream:
//   1. row transforms of every density row (R2C along x, zero-padded to px),
//      written column-major per frequency column             [row stage]
//   2. per (kx, ky parity): column FFT of each layer, multiply by the
//      kernel spectra, sum over layers, inverse column FFT   [column stage]
//   3. inverse row transforms (C2R) cropped to the stations  [row stage]
// The adjoint runs the same three stages in mirror image.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "grav_internal.h"

namespace grav {

namespace {
thread_local char g_err[512] = "";

template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
}  // namespace

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Smallest power of two >= max(4, 2n - 1): the circulant size of one axis
// (Eq. 19 embeds 2n - 1 kernel values; any size >= 2n - 1 gives the exact
// product).
int circulant_size(int n) {
    int p = 4;
    while (p < 2 * n - 1) p *= 2;
    return p;
}

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

namespace {

// exp(-2 pi i e / T) with exact quadrant symmetry; T is a power of two >= 4.
void unit_root(long e, long T, double* re, double* im) {
    e = ((e % T) + T) % T;
    const long quarter = T / 4;
    const long q = e / quarter, rr = e - q * quarter;
    double c, s;
    if (2 * rr <= quarter) {
        const double phi = 2.0 * M_PI * (double)rr / (double)T;
        c = cos(phi);
        s = sin(phi);
    } else {
        const double phi = 2.0 * M_PI * (double)(quarter - rr) / (double)T;
        c = sin(phi);
        s = cos(phi);
    }
    double ct, st;  // cos and sin of the full angle 2 pi e / T
    switch (q) {
        case 0: ct = c; st = s; break;
        case 1: ct = -s; st = c; break;
        case 2: ct = -c; st = -s; break;
        default: ct = s; st = -c; break;
    }
    *re = ct;
    *im = -st;
}

}  // namespace

int check_geometry(int nx, int ny, int nz, double dx, double dy, double dz, double h, unsigned components) {
    if (nx < 1 || ny < 1 || nz < 1 || nx > GRAV_MAX_NX || ny > GRAV_MAX_NY) {
        set_error("mesh size %dx%dx%d outside 1..%d x 1..%d x >=1", nx, ny, nz, GRAV_MAX_NX, GRAV_MAX_NY);
        return GRAV_EINVAL;
    }
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !isfinite(dx) || !isfinite(dy) || !isfinite(dz)) {
        set_error("cell sizes must be finite and > 0 (got %g, %g, %g)", dx, dy, dz);
        return GRAV_EINVAL;
    }
    if (!(h > 0) || !isfinite(h)) {
        set_error("station height h must be finite and > 0 (got %g)", h);
        return GRAV_EINVAL;
    }
    if ((components & kCompBits) == 0 || (components & ~(kCompBits | (unsigned)GRAV_FP64_SPECTRAL))) {
        set_error("component mask 0x%x selects no component or has unknown bits", components);
        return GRAV_EINVAL;
    }
    if (__builtin_popcount(components & kCompBits) > kMaxPlanComp) {
        set_error("component mask 0x%x selects more than %d components; split it into two plans", components,
                  kMaxPlanComp);
        return GRAV_EINVAL;
    }
    if ((size_t)nz * (size_t)ny * (size_t)nx > (size_t)1 << 31) {
        set_error("mesh has more than 2^31 cells");
        return GRAV_EINVAL;
    }
    return GRAV_OK;
}

int dev_alloc_raw(void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GRAV_ENOMEM : GRAV_ECUDA;
    }
    return GRAV_OK;
}

namespace {

template <typename T>
int dev_alloc(T** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? GRAV_ENOMEM : GRAV_ECUDA;
    }
    return GRAV_OK;
}

}  // namespace

void free_plan(grav_plan* p) {
    if (!p) return;
    for (auto& t : p->timed)
        for (cudaEvent_t e : t.ev) p->ev_pool.push_back(e);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    cudaFree(p->spec);
    cudaFree(p->tw);
    cudaFree(p->ws_a);
    cudaFree(p->ws_b);
    cudaFree(p->err_flag);
    delete p;
}

int build_twiddles(int log_t, int fp64, void** dev, size_t* bytes) {
    const long T = 1L << log_t;
    const size_t elem = fp64 ? 16 : 8;
    *bytes = (size_t)T * elem;
    unsigned char* host = (unsigned char*)malloc(*bytes);
    if (!host) {
        set_error("host allocation of the twiddle table failed");
        return GRAV_ENOMEM;
    }
    for (long e = 0; e < T; ++e) {
        double re, im;
        unit_root(e, T, &re, &im);
        if (fp64) {
            double* d = (double*)host + 2 * e;
            d[0] = re; d[1] = im;
        } else {
            float* f = (float*)host + 2 * e;
            f[0] = (float)re; f[1] = (float)im;
        }
    }
    int rc = dev_alloc(dev, *bytes, "twiddle table");
    if (rc == GRAV_OK) {
        cudaError_t e = cudaMemcpy(*dev, host, *bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpy(twiddles)");
    }
    free(host);
    return rc;
}

namespace {

template <typename R>
int make_spectra(grav_plan* p) {
    // FP64 staging: the embedded kernels of a chunk of layers and their row
    // transforms, bounded to about 2 GB.
    // rows b < py / 2 of each embedded kernel (the other half mirrors them)
    const int hy = p->py / 2;
    const size_t per_layer = (size_t)p->ncomp * hy * p->px * sizeof(double) +
                             (size_t)p->kx_count * p->ncomp * hy * 2 * sizeof(double);
    const size_t budget = (size_t)2 << 30;
    int nzc = (int)(budget / per_layer);
    if (nzc < 1) nzc = 1;
    if (nzc > p->nz) nzc = p->nz;
    if (nzc * p->ncomp > 65535) nzc = 65535 / p->ncomp;

    void* tw64 = nullptr;
    size_t tw64_bytes = 0;
    int rc = GRAV_OK;
    if (p->fp64) {
        tw64 = p->tw;
    } else {
        rc = build_twiddles(p->log_t, 1, &tw64, &tw64_bytes);
        if (rc) return rc;
    }
    double* E = nullptr;
    void* Ehat = nullptr;
    const size_t e_bytes = (size_t)nzc * p->ncomp * hy * p->px * sizeof(double);
    const size_t eh_bytes = (size_t)p->kx_count * nzc * p->ncomp * hy * 2 * sizeof(double);
    if ((rc = dev_alloc(&E, e_bytes, "kernel staging")) == GRAV_OK &&
        (rc = dev_alloc(&Ehat, eh_bytes, "kernel row-transform staging")) == GRAV_OK) {
        cudaStream_t s;
        cudaError_t ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            rc = cuda_fail(ce, "cudaStreamCreate");
        } else {
            Geometry g{p->nx, p->ny, p->nz, p->dx, p->dy, p->dz, p->h};
            const double scale = 1.0 / ((double)p->px * (double)p->py);
            for (int n0 = 0; n0 < p->nz && rc == GRAV_OK; n0 += nzc) {
                const int n1 = n0 + nzc < p->nz ? n0 + nzc : p->nz;
                const int cnt = n1 - n0;
                const int O = cnt * p->ncomp;
                if ((ce = cudaMemsetAsync(E, 0, (size_t)O * hy * p->px * sizeof(double), s)) != cudaSuccess) {
                    rc = cuda_fail(ce, "cudaMemsetAsync(kernel staging)");
                    break;
                }
                if ((ce = launch_kernel_gen(g, p->comps, n0, n1, 2, p->px, p->py, E, s)) != cudaSuccess) {
                    rc = cuda_fail(ce, "kernel generation launch");
                    break;
                }
                // rows o = slot * cnt + (n - n0) of length px, py / 2 of them per o
                if ((ce = launch_row_r2c<double>(p->log_px, E, (size_t)hy * p->px, (size_t)p->px, p->px, hy, O,
                                                 Ehat, hy, tw64, p->log_t, s)) != cudaSuccess) {
                    rc = cuda_fail(ce, "kernel row transform launch");
                    break;
                }
                if ((ce = launch_spec_extract<R>(p->log_py - 1, Ehat, p->kx_count, cnt, p->ncomp, n0, p->nz, p->jp,
                                                 p->imag_mask, p->oddv_mask, scale, (R*)p->spec, tw64, p->log_t,
                                                 s)) != cudaSuccess) {
                    rc = cuda_fail(ce, "kernel spectra launch");
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
    if (!p->fp64) cudaFree(tw64);
    return rc;
}

constexpr size_t kMaxTimedCalls = 65536;

// Events of one timed call, or nullptr when timing is off or full.
grav_plan::TimedCall* begin_timed(grav_plan* p, int kind) {
    if (!p->timing || p->timed.size() >= kMaxTimedCalls) return nullptr;
    grav_plan::TimedCall t;
    t.kind = kind;
    for (int i = 0; i < 4; ++i) {
        if (!p->ev_pool.empty()) {
            t.ev[i] = p->ev_pool.back();
            p->ev_pool.pop_back();
        } else if (cudaEventCreate(&t.ev[i]) != cudaSuccess) {
            cudaGetLastError();
            for (int j = 0; j < i; ++j) p->ev_pool.push_back(t.ev[j]);
            return nullptr;
        }
    }
    p->timed.push_back(t);
    return &p->timed.back();
}

inline void mark(grav_plan::TimedCall* t, int i, cudaStream_t s) {
    if (t) cudaEventRecord(t->ev[i], s);
}

// Per-request workspace of a batched call: [A][B], each rounded to 256 bytes.
size_t ws_a_part(const grav_plan* p) { return round_up(p->ws_a_bytes, 256); }
size_t ws_req_bytes(const grav_plan* p) { return ws_a_part(p) + round_up(p->ws_b_bytes, 256); }

// spec_of: per-request spectra of a batched call across plans (nullptr: the
// plan's own for every request).
template <typename R>
int run_forward(grav_plan* p, const void* rho, void* out, void* wa, void* wb, int batch, size_t ws_stride,
                cudaStream_t s, const void* const* spec_of = nullptr) {
    using C = typename cplx_of<R>::type;
    const size_t cs = ws_stride / sizeof(C);  // workspace stride in complex elements
    cudaError_t e;
    grav_plan::TimedCall* tc = batch == 1 ? begin_timed(p, 0) : nullptr;
    mark(tc, 0, s);
    e = launch_row_r2c<R>(p->log_px, (const R*)rho, (size_t)p->ny * p->nx, (size_t)p->nx, p->nx, p->ny, p->nz, wa,
                          p->ny_pad, p->tw, p->log_t, s, Batch{batch, (size_t)p->nz * p->ny * p->nx, cs}, p->err_flag);
    if (e != cudaSuccess) return cuda_fail(e, "forward row transform");
    mark(tc, 1, s);
    ColumnArgs a{p->ny, p->ny_pad, p->nz, p->ncomp, p->kx_count, p->jp, p->imag_mask, p->oddv_mask,
                 p->log_t - (p->log_py - 1), p->log_t - p->log_py};
    if (spec_of) {
        a.spec_count = batch;
        for (int i = 0; i < batch; ++i) a.spec_of[i] = spec_of[i];
    }
    e = launch_forward_columns<R>(p->log_py - 1, a, wa, (const R*)p->spec, wb, p->tw, p->err_flag, s,
                                  Batch{batch, cs, cs});
    if (e != cudaSuccess) return cuda_fail(e, "forward column stage");
    mark(tc, 2, s);
    const size_t half = (size_t)p->kx_count * p->ncomp * p->ny_pad * 2 * sizeof(R);
    e = launch_row_c2r<R>(p->log_px, wb, (const unsigned char*)wb + half, p->ny, p->ncomp, p->ny_pad, (R*)out,
                          (size_t)p->nx, p->nx, p->tw, p->log_t, s,
                          Batch{batch, cs, (size_t)p->ncomp * p->ny * p->nx});
    if (e != cudaSuccess) return cuda_fail(e, "forward inverse row transform");
    mark(tc, 3, s);
    return GRAV_OK;
}

template <typename R>
int run_adjoint(grav_plan* p, const void* r, void* grad, void* wa, void* wb, int batch, size_t ws_stride,
                cudaStream_t s, const void* const* spec_of = nullptr) {
    using C = typename cplx_of<R>::type;
    const size_t cs = ws_stride / sizeof(C);
    cudaError_t e;
    grav_plan::TimedCall* tc = batch == 1 ? begin_timed(p, 1) : nullptr;
    mark(tc, 0, s);
    e = launch_row_r2c<R>(p->log_px, (const R*)r, (size_t)p->ny * p->nx, (size_t)p->nx, p->nx, p->ny, p->ncomp, wb,
                          p->ny_pad, p->tw, p->log_t, s, Batch{batch, (size_t)p->ncomp * p->ny * p->nx, cs},
                          p->err_flag);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint row transform");
    mark(tc, 1, s);
    ColumnArgs a{p->ny, p->ny_pad, p->nz, p->ncomp, p->kx_count, p->jp, p->imag_mask, p->oddv_mask,
                 p->log_t - (p->log_py - 1), p->log_t - p->log_py};
    // FP32 2048 x 2048 plans: tile-major column output, read back by whole tiles
    if constexpr (sizeof(R) == 4) a.z_tiled = adjoint_tiled_ok(p->log_py - 1, p->log_px, p->nx, a) ? 1 : 0;
    if (spec_of) {
        a.spec_count = batch;
        for (int i = 0; i < batch; ++i) a.spec_of[i] = spec_of[i];
    }
    e = launch_adjoint_columns<R>(p->log_py - 1, a, wb, (const R*)p->spec, wa, p->tw, p->err_flag, s,
                                  Batch{batch, cs, cs});
    if (e != cudaSuccess) return cuda_fail(e, "adjoint column stage");
    mark(tc, 2, s);
    const size_t half = (size_t)p->kx_count * p->nz * p->ny_pad * 2 * sizeof(R);
    if (a.z_tiled) {
        e = launch_row_c2r_tiled(wa, (const unsigned char*)wa + half, p->ny, p->nz, p->kx_count, (float*)grad,
                                 (size_t)p->nx, p->nx, p->tw, p->log_t, s,
                                 Batch{batch, cs, (size_t)p->nz * p->ny * p->nx}, p->err_flag);
    } else {
        e = launch_row_c2r<R>(p->log_px, wa, (const unsigned char*)wa + half, p->ny, p->nz, p->ny_pad, (R*)grad,
                              (size_t)p->nx, p->nx, p->tw, p->log_t, s,
                              Batch{batch, cs, (size_t)p->nz * p->ny * p->nx});
    }
    if (e != cudaSuccess) return cuda_fail(e, "adjoint inverse row transform");
    mark(tc, 3, s);
    return GRAV_OK;
}

// Requests on different plans share a batched call when the plans agree in
// everything but their kernel spectra: mesh sizes, components, precision
// (hence the same circulant sizes, workspace layout and twiddles).
bool same_shape(const grav_plan* a, const grav_plan* b) {
    return a->kind == 0 && b->kind == 0 && a->nx == b->nx && a->ny == b->ny && a->nz == b->nz &&
           a->comps == b->comps && a->fp64 == b->fp64 && a->device == b->device;
}

int batch_plans_call(int batch, grav_plan* const* plans, const void* in, void* out, void* ws, void* stream,
                     bool adjoint) {
    const char* name = adjoint ? "grav_adjoint_batch_plans" : "grav_forward_batch_plans";
    if (!plans || !in || !out || !ws || batch < 1 || batch > kMaxSpecPlans) {
        set_error("%s: null argument, or batch outside 1..%d", name, kMaxSpecPlans);
        return GRAV_EINVAL;
    }
    const void* spec_of[kMaxSpecPlans];
    for (int i = 0; i < batch; ++i) {
        if (!plans[i] || !same_shape(plans[0], plans[i])) {
            set_error("%s: plan %d is null or differs from plan 0 in mesh size, components, precision or kind",
                      name, i);
            return GRAV_EINVAL;
        }
        spec_of[i] = plans[i]->spec;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) {
        set_error("%s: workspace must be 256-byte aligned", name);
        return GRAV_EINVAL;
    }
    grav_plan* p = plans[0];
    void* wa = ws;
    void* wb = (unsigned char*)ws + ws_a_part(p);
    const size_t stride = ws_req_bytes(p);
    cudaStream_t s = (cudaStream_t)stream;
    if (adjoint)
        return p->fp64 ? run_adjoint<double>(p, in, out, wa, wb, batch, stride, s, spec_of)
                       : run_adjoint<float>(p, in, out, wa, wb, batch, stride, s, spec_of);
    return p->fp64 ? run_forward<double>(p, in, out, wa, wb, batch, stride, s, spec_of)
                   : run_forward<float>(p, in, out, wa, wb, batch, stride, s, spec_of);
}

int batch_call(grav_plan* plan, int batch, const void* in, void* out, void* ws, void* stream, bool adjoint) {
    const char* name = adjoint ? "grav_adjoint_batch" : "grav_forward_batch";
    if (!plan || !in || !out || batch < 1 || batch > 65535) {
        set_error("%s: null plan or buffer, or batch outside 1..65535", name);
        return GRAV_EINVAL;
    }
    if (plan->kind != 0) {
        set_error("%s: the plan was made by grav_plan_create3d; use grav_forward3d / grav_adjoint3d", name);
        return GRAV_EINVAL;
    }
    if (!ws && batch > 1) {
        set_error("%s: a batch of %d needs a workspace of %d x grav_workspace_bytes", name, batch, batch);
        return GRAV_EINVAL;
    }
    if (ws && (reinterpret_cast<uintptr_t>(ws) & 255)) {
        set_error("%s: workspace must be 256-byte aligned", name);
        return GRAV_EINVAL;
    }
    void* wa = ws ? ws : plan->ws_a;
    void* wb = ws ? (unsigned char*)ws + ws_a_part(plan) : plan->ws_b;
    const size_t stride = ws_req_bytes(plan);
    cudaStream_t s = (cudaStream_t)stream;
    if (adjoint)
        return plan->fp64 ? run_adjoint<double>(plan, in, out, wa, wb, batch, stride, s)
                          : run_adjoint<float>(plan, in, out, wa, wb, batch, stride, s);
    return plan->fp64 ? run_forward<double>(plan, in, out, wa, wb, batch, stride, s)
                      : run_forward<float>(plan, in, out, wa, wb, batch, stride, s);
}

}  // namespace

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GRAV_ENOMEM : GRAV_ECUDA;
}

}  // namespace grav

using namespace grav;

extern "C" {

const char* grav_last_error(void) { return g_err; }

grav_plan* grav_plan_create(int nx, int ny, int nz, double dx, double dy, double dz, double h, unsigned components) {
    g_err[0] = 0;
    if (check_geometry(nx, ny, nz, dx, dy, dz, h, components)) return nullptr;
    grav_plan* p = new (std::nothrow) grav_plan();
    if (!p) {
        set_error("host allocation of the plan failed");
        return nullptr;
    }
    p->nx = nx; p->ny = ny; p->nz = nz;
    p->dx = dx; p->dy = dy; p->dz = dz; p->h = h;
    p->comps = components & kCompBits;
    p->fp64 = (components & GRAV_FP64_SPECTRAL) ? 1 : 0;
    for (int c = 0; c < kMaxComp; ++c) {
        if (p->comps & (1u << c)) {
            const int s = p->ncomp++;
            p->comp_id[s] = c;
            if (odd_u(c) != odd_v(c)) p->imag_mask |= 1u << s;
            if (odd_v(c)) p->oddv_mask |= 1u << s;
        }
    }
    p->px = circulant_size(nx);
    p->py = circulant_size(ny);
    p->log_px = ilog2(p->px);
    p->log_py = ilog2(p->py);
    p->log_t = p->log_px > p->log_py ? p->log_px : p->log_py;
    p->kx_count = p->px / 2 + 1;
    p->J = p->py / 4;
    p->jp = (int)round_up((size_t)p->J + 1, 4);
    p->ny_pad = (int)round_up((size_t)ny, 4);
    cudaGetDevice(&p->device);

    const size_t real = p->fp64 ? sizeof(double) : sizeof(float);
    p->spec_bytes = (size_t)2 * p->kx_count * nz * p->ncomp * p->jp * real;
    p->ws_a_bytes = (size_t)2 * p->kx_count * nz * p->ny_pad * 2 * real;
    p->ws_b_bytes = (size_t)2 * p->kx_count * p->ncomp * p->ny_pad * 2 * real;

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
    if (!rc) rc = dev_alloc(&p->spec, p->spec_bytes, "kernel spectra");
    if (!rc) rc = dev_alloc(&p->ws_a, p->ws_a_bytes, "workspace A");
    if (!rc) rc = dev_alloc(&p->ws_b, p->ws_b_bytes, "workspace B");
    if (!rc) rc = dev_alloc(&p->err_flag, 256, "error flag");
    if (!rc) {
        cudaError_t me = cudaMemset(p->err_flag, 0, 256);
        if (me != cudaSuccess) rc = cuda_fail(me, "cudaMemset(error flag)");
    }
    if (!rc) rc = p->fp64 ? make_spectra<double>(p) : make_spectra<float>(p);
    if (rc) {
        free_plan(p);
        return nullptr;
    }
    return p;
}

int grav_forward(grav_plan* plan, const void* rho_dev, void* out_dev, void* stream) {
    if (!plan || !rho_dev || !out_dev) {
        set_error("grav_forward: null plan or buffer");
        return GRAV_EINVAL;
    }
    return batch_call(plan, 1, rho_dev, out_dev, nullptr, stream, false);
}

int grav_adjoint(grav_plan* plan, const void* r_dev, void* grad_dev, void* stream) {
    if (!plan || !r_dev || !grad_dev) {
        set_error("grav_adjoint: null plan or buffer");
        return GRAV_EINVAL;
    }
    return batch_call(plan, 1, r_dev, grad_dev, nullptr, stream, true);
}

size_t grav_workspace_bytes(const grav_plan* plan) { return plan ? ws_req_bytes(plan) : 0; }

int grav_forward_batch(grav_plan* plan, int batch, const void* rho_dev, void* out_dev, void* workspace_dev,
                       void* stream) {
    return batch_call(plan, batch, rho_dev, out_dev, workspace_dev, stream, false);
}

int grav_adjoint_batch(grav_plan* plan, int batch, const void* r_dev, void* grad_dev, void* workspace_dev,
                       void* stream) {
    return batch_call(plan, batch, r_dev, grad_dev, workspace_dev, stream, true);
}

int grav_forward_batch_plans(int batch, grav_plan* const* plans, const void* rho_dev, void* out_dev,
                             void* workspace_dev, void* stream) {
    return batch_plans_call(batch, plans, rho_dev, out_dev, workspace_dev, stream, false);
}

int grav_adjoint_batch_plans(int batch, grav_plan* const* plans, const void* r_dev, void* grad_dev,
                             void* workspace_dev, void* stream) {
    return batch_plans_call(batch, plans, r_dev, grad_dev, workspace_dev, stream, true);
}

void grav_plan_destroy(grav_plan* plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan(plan);
}

size_t grav_plan_bytes(const grav_plan* plan) {
    if (!plan) return 0;
    return plan->spec_bytes + plan->tw_bytes + plan->ws_a_bytes + plan->ws_b_bytes;
}

int grav_plan_info(const grav_plan* plan, grav_plan_info_t* info) {
    if (!plan || !info) {
        set_error("grav_plan_info: null argument");
        return GRAV_EINVAL;
    }
    info->nx = plan->nx; info->ny = plan->ny; info->nz = plan->nz;
    info->px = plan->px; info->py = plan->py;
    info->ncomp = plan->ncomp;
    info->fp64 = plan->fp64;
    info->spectra_bytes = plan->spec_bytes;
    info->workspace_bytes = plan->ws_a_bytes + plan->ws_b_bytes;
    info->pz = plan->kind == 1 ? plan->pz : 0;
    info->equal_dim = plan->kind == 1 ? 1 : 0;
    return GRAV_OK;
}

int grav_kernel_values(int nx, int ny, int nz, double dx, double dy, double dz, double h, unsigned components,
                       double* K_dev, void* stream) {
    int rc = check_geometry(nx, ny, nz, dx, dy, dz, h, components);
    if (rc) return rc;
    if (!K_dev) {
        set_error("grav_kernel_values: null output");
        return GRAV_EINVAL;
    }
    Geometry g{nx, ny, nz, dx, dy, dz, h};
    cudaError_t e = launch_kernel_gen(g, components & kCompBits, 0, nz, 1, 0, 0, K_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "kernel generation launch");
    return GRAV_OK;
}

int grav_plan_check(grav_plan* plan) {
    if (!plan) {
        set_error("grav_plan_check: null plan");
        return GRAV_EINVAL;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, plan->err_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(error flag)");
    if (flag) {
        cudaMemset(plan->err_flag, 0, sizeof(int));
        set_error("a pipeline wait of an earlier call on this plan ran out; its output is invalid");
        return GRAV_ETIMEOUT;
    }
    return GRAV_OK;
}

int grav_plan_set_timing(grav_plan* plan, int enable) {
    if (!plan) {
        set_error("grav_plan_set_timing: null plan");
        return GRAV_EINVAL;
    }
    plan->timing = enable ? 1 : 0;
    return GRAV_OK;
}

int grav_plan_stage_times(grav_plan* plan, double ms[6], long long calls[2]) {
    if (!plan || !ms || !calls) {
        set_error("grav_plan_stage_times: null argument");
        return GRAV_EINVAL;
    }
    for (int i = 0; i < 6; ++i) ms[i] = 0.0;
    calls[0] = calls[1] = 0;
    int rc = GRAV_OK;
    for (auto& t : plan->timed) {
        cudaError_t e = cudaEventSynchronize(t.ev[3]);
        if (e != cudaSuccess && rc == GRAV_OK) rc = cuda_fail(e, "cudaEventSynchronize(stage timing)");
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
            float v = 0.f;
            if (cudaEventElapsedTime(&v, t.ev[i], t.ev[i + 1]) == cudaSuccess) ms[3 * t.kind + i] += v;
        }
        calls[t.kind] += 1;
        for (cudaEvent_t ev : t.ev) plan->ev_pool.push_back(ev);
    }
    plan->timed.clear();
    return rc;
}

}  // extern "C"
