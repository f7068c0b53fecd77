/*
 * grav.h - C ABI of the GB300 fast forward library for gravity (gz) and the
 * gravity-gradient tensor (gxx, gxy, gxz, gyy, gyz, gzz) of a right-prism
 * density mesh observed on a horizontal plane.
 *
 * Method (Cao, "Rapid forward of gravity and tensor gravity data"):
 *   d = G M (Eqs. 3-4).  By translation equivalence (Eq. 7, Eq. 10) each
 *   depth layer's block of G is block Toeplitz with Toeplitz blocks
 *   (Sec. 2.2.3, Eqs. 17 and 20), fixed by its (2nx-1)(2ny-1) offset values;
 *   the product with a layer of densities is a circulant embedding plus FFT
 *   (Eqs. 18-19), and the layers add up (Eq. 21).  The plan stores only the
 *   kernel spectra (Eq. 22) instead of G.
 *
 * Geometry (Fig. 1; cell order j = l + nx m + nx ny n, Sec. 2.2):
 *   z is positive down.  Cell (l, m, n) spans [l dx, (l+1) dx] x
 *   [m dy, (m+1) dy] x [n dz, (n+1) dz].  Station (p, q) is at
 *   ((p + 1/2) dx, (q + 1/2) dy, -h) with h > 0: one station above every
 *   column of cells.  Units are SI: density kg/m^3, gz m/s^2, gradients 1/s^2;
 *   the gravitational constant is 6.672e-11 (Sec. 2.1).
 *
 * Layouts (row-major, x fastest):
 *   rho  [nz][ny][nx]      density (forward input)
 *   out  [ncomp][ny][nx]   one plane per selected component, in ascending
 *                          bit order of the component mask
 *   r    [ncomp][ny][nx]   residual / data-space vector (adjoint input)
 *   grad [nz][ny][nx]      G^T r (adjoint output)
 *   Element type: float, or double when GRAV_FP64_SPECTRAL is set.
 *
 * Ownership and ordering: the caller owns every device buffer passed in;
 * the plan owns its kernel spectra and workspaces.  grav_forward and
 * grav_adjoint are asynchronous on the given CUDA stream (NULL = legacy
 * default stream) and never synchronise on success.  One plan runs one
 * call at a time: calls on different streams that overlap on the device
 * share the plan's workspaces and race.  Every entry point may be called
 * from any host thread; the error message is thread-local.
 *
 * Errors: entry points returning int give GRAV_OK (0) or a negative code;
 * grav_plan_create returns NULL on error.  grav_last_error() then holds a
 * message.  Invalid arguments never touch the device.
 */
#ifndef GRAV_H
#define GRAV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grav_plan grav_plan;

/* Component mask bits (Eq. 1): the five independent gradient components,
 * gz (Eq. 2) and the derived gzz = -(gxx + gyy); and the horizontal first
 * derivatives gx, gy (also block Toeplitz, shown in Fig. 6), positive towards
 * +x and +y.  One plan holds at most 8 components (GRAV_EINVAL above that:
 * split the request over two plans). */
enum {
    GRAV_GZ = 1,
    GRAV_GXX = 2,
    GRAV_GXY = 4,
    GRAV_GXZ = 8,
    GRAV_GYY = 16,
    GRAV_GYZ = 32,
    GRAV_GZZ = 64,
    GRAV_GX = 128,
    GRAV_GY = 256,
    GRAV_ALL6 = 63,
    /* Precision flag: FP64 input, spectra, FFTs and output.  Without it the
     * spectra are stored as FP32 and the per-call arithmetic is FP32 with a
     * compensated (Kahan) sum over the depth layers. */
    GRAV_FP64_SPECTRAL = 1 << 16
};

/* Status codes. */
enum {
    GRAV_OK = 0,
    GRAV_EINVAL = -1,   /* bad size, spacing, height, mask or null pointer */
    GRAV_ENOMEM = -2,   /* device memory (HBM) exhausted */
    GRAV_ECUDA = -3,    /* a CUDA call failed; the message names it */
    GRAV_ETIMEOUT = -4  /* a bounded device wait gave up (grav_plan_check) */
};

/* Limits of this implementation.  They differ per axis on purpose: the row
 * stage (x) streams rows of up to 4096 points through registers, while the
 * column stage (y) keeps a whole half-length column transform of every layer
 * in one CTA's shared memory, which caps Py at 2048 (ny <= 1024).  A mesh
 * with ny > 1024 and nx <= 1024 is computed with the axes exchanged:
 * transpose rho's x and y, swap dx and dy, and read gxx as gyy, gxz as gyz,
 * gx as gy (and back); gz, gxy and gzz are unchanged.  A 2048 x 2048 mesh is
 * beyond this version. */
#define GRAV_MAX_NX 2048
#define GRAV_MAX_NY 1024

/* Build a plan: generate the kernel of every layer over the offset grid in
 * FP64 (Eq. 2 and the gradient closed forms, translation form Eq. 10),
 * embed it in a circulant (Eq. 19), transform it and keep the spectra
 * resident on the current device (Eq. 22).  Blocks until done.
 *   nx, ny, nz  cells per axis: 1 <= nx <= GRAV_MAX_NX, 1 <= ny <= GRAV_MAX_NY,
 *               nz >= 1
 *   dx, dy, dz  cell size in metres, > 0
 *   h           station height above the mesh top in metres, > 0
 *   components  OR of GRAV_GZ ... GRAV_GY (at most 8 of them), optionally
 *               | GRAV_FP64_SPECTRAL
 * Returns NULL on error (GRAV_EINVAL or GRAV_ENOMEM class, see
 * grav_last_error). */
grav_plan* grav_plan_create(int nx, int ny, int nz, double dx, double dy, double dz,
                            double h, unsigned components);

/* Forward d_c = sum_n G_{c,n} rho_n (Eq. 21) for every selected component.
 *   rho_dev  device [nz][ny][nx], float (double with GRAV_FP64_SPECTRAL)
 *   out_dev  device [ncomp][ny][nx], same type; fully overwritten
 *   stream   cudaStream_t or NULL
 * Returns GRAV_OK, GRAV_EINVAL (null plan or pointer) or GRAV_ECUDA. */
int grav_forward(grav_plan* plan, const void* rho_dev, void* out_dev, void* stream);

/* Adjoint grad = sum_c G_c^T r_c: the transpose of Eq. 21, a per-layer
 * product with the conjugate kernel spectra and no sum over layers.
 *   r_dev     device [ncomp][ny][nx]
 *   grad_dev  device [nz][ny][nx]; fully overwritten
 * Same types, stream and status codes as grav_forward. */
int grav_adjoint(grav_plan* plan, const void* r_dev, void* grad_dev, void* stream);

/* Device bytes of scratch one request of a batched call needs (the plan's
 * own workspaces hold exactly one request).  0 for NULL. */
size_t grav_workspace_bytes(const grav_plan* plan);

/* Forward of `batch` independent density models on one plan with one launch
 * per stage (Eq. 21 for each; a serving loop groups requests on the same
 * mesh this way).
 *   batch          1 .. 65535
 *   rho_dev        device [batch][nz][ny][nx]
 *   out_dev        device [batch][ncomp][ny][nx]
 *   workspace_dev  device scratch of batch * grav_workspace_bytes(plan) bytes,
 *                  256-byte aligned, owned by the caller; NULL only for
 *                  batch == 1 (then the plan's own workspaces are used).
 *                  Calls with different workspaces may overlap on the GPU.
 * Returns GRAV_OK, GRAV_EINVAL or GRAV_ECUDA. */
int grav_forward_batch(grav_plan* plan, int batch, const void* rho_dev, void* out_dev, void* workspace_dev,
                       void* stream);

/* Adjoint (transpose of Eq. 21) of `batch` data-space vectors:
 * r_dev [batch][ncomp][ny][nx] -> grad_dev [batch][nz][ny][nx]; workspace as
 * for grav_forward_batch. */
int grav_adjoint_batch(grav_plan* plan, int batch, const void* r_dev, void* grad_dev, void* workspace_dev,
                       void* stream);

/* Forward of `batch` requests on `batch` plans (one plan per request) with
 * one launch per stage (Eq. 21 for each).  The plans may differ only in their
 * kernel spectra, i.e. in cell sizes and station height: mesh sizes,
 * components and precision must be equal (a serving loop batches requests on
 * the same model seen from several heights this way).
 *   batch          1 .. 16
 *   plans          host array of `batch` plans made by grav_plan_create
 *   rho_dev        device [batch][nz][ny][nx], request b on plans[b]
 *   out_dev        device [batch][ncomp][ny][nx]
 *   workspace_dev  device scratch of batch * grav_workspace_bytes(plans[0])
 *                  bytes, 256-byte aligned, owned by the caller (required)
 * Returns GRAV_OK, GRAV_EINVAL (null argument, plans that differ in more
 * than their spectra) or GRAV_ECUDA. */
int grav_forward_batch_plans(int batch, grav_plan* const* plans, const void* rho_dev, void* out_dev,
                             void* workspace_dev, void* stream);

/* Adjoint counterpart: r_dev [batch][ncomp][ny][nx] -> grad_dev
 * [batch][nz][ny][nx], request b on plans[b]; rules as above. */
int grav_adjoint_batch_plans(int batch, grav_plan* const* plans, const void* r_dev, void* grad_dev,
                             void* workspace_dev, void* stream);

/* Release the plan and its device memory (waits for the device first).
 * NULL is ignored. */
void grav_plan_destroy(grav_plan* plan);

/* Message of the last failing call on this host thread ("" if none). */
const char* grav_last_error(void);

/* Device bytes the plan holds (spectra + workspaces + tables): the figure an
 * HBM-budget admission check needs.  0 for NULL. */
size_t grav_plan_bytes(const grav_plan* plan);

/* Sizes chosen by the plan. */
typedef struct {
    int nx, ny, nz;
    int px, py;              /* circulant (FFT) sizes per axis, powers of 2 >= 2n-1 */
    int ncomp;               /* selected components */
    int fp64;                /* 1 with GRAV_FP64_SPECTRAL */
    size_t spectra_bytes;    /* resident kernel spectra */
    size_t workspace_bytes;  /* per-call scratch owned by the plan */
    int pz;                  /* circulant size along z (equal-dimension plans), else 0 */
    int equal_dim;           /* 1 for a plan made by grav_plan_create3d */
} grav_plan_info_t;

/* Fill *info.  Returns GRAV_OK or GRAV_EINVAL. */
int grav_plan_info(const grav_plan* plan, grav_plan_info_t* info);

/* The kernel values themselves (the first row and column of every Toeplitz
 * block, Eqs. 17 and 19), as the plan generates them in FP64:
 *   K_dev  device double [ncomp][nz][2ny-1][2nx-1]; entry
 *          [c][n][v + ny - 1][u + nx - 1] is G_c for a station and the
 *          cell offset by (u, v) columns in layer n (Eq. 10).
 * Asynchronous on stream.  Same argument rules as grav_plan_create.
 * Returns GRAV_OK, GRAV_EINVAL or GRAV_ECUDA. */
int grav_kernel_values(int nx, int ny, int nz, double dx, double dy, double dz, double h,
                       unsigned components, double* K_dev, void* stream);

/* Stage timing, for tracing and roofline measurement.  While enabled, every
 * grav_forward / grav_adjoint records CUDA events on its stream before and
 * after each of its three stages (row transforms, column stage, inverse row
 * transforms).  Enabling adds four event records per call and no
 * synchronisation.  Returns GRAV_OK, GRAV_EINVAL or GRAV_ECUDA. */
int grav_plan_set_timing(grav_plan* plan, int enable);

/* Waits for the recorded events, adds up the device time of each stage since
 * the previous read, and resets the record.
 *   ms[0..2]  forward: row transforms, column stage, inverse row transforms
 *   ms[3..5]  adjoint: the same three stages
 *   calls[0]  forward calls timed, calls[1] adjoint calls timed
 * At most 65536 calls are kept between reads; later calls are not timed.
 * Returns GRAV_OK, GRAV_EINVAL or GRAV_ECUDA. */
int grav_plan_stage_times(grav_plan* plan, double ms[6], long long calls[2]);

/* Waits for the device, then reports whether a bounded wait inside an
 * earlier call on this plan ran out (the column stage streams its inputs
 * through asynchronous copies and gives up after one second instead of
 * hanging).  Returns GRAV_OK, GRAV_ETIMEOUT (that call's output is invalid;
 * the flag is cleared) or GRAV_ECUDA. */
int grav_plan_check(grav_plan* plan);

/* Failure-path self-test: one GPU thread waits, with the same bounded wait
 * the pipelines use, on a barrier that nothing completes, for limit_ms
 * milliseconds (0 < limit_ms <= 10000).  Expected result: GRAV_ETIMEOUT, with
 * the time actually waited in *waited_ms (may be NULL); the CUDA context
 * stays usable.  GRAV_OK would mean the wait did not run out. */
int grav_selftest_bounded_wait(double limit_ms, double* waited_ms);

/* ---- Equal-dimension variant (Sec. 2.2, Eqs. 10-11) ----
 *
 * A station at the centre of every cell: station (p, q, t) sits at
 * ((p + 1/2) dx, (q + 1/2) dy, (t + 1/2) dz), inside the mesh, and the data are
 * as three-dimensional as the model (the case the paper sizes at 1024 x 1024 x
 * 100 cells).  G(station (p,q,t), cell (l,m,n)) depends only on the offset
 * (l-p, m-q, n-t), so G is block Toeplitz on all three levels (the block
 * matrix of G_{t,n} after Eq. 22) with (2nx-1)(2ny-1)(2nz-1) distinct values.
 * The plan embeds them in a three-level circulant (Eq. 19 on every axis) and
 * keeps its spectra; a forward is a three-dimensional FFT product.  At a
 * station's own cell the closed forms give the field inside the prism.
 *
 * Layouts: rho and grad [nz][ny][nx]; out and r [ncomp][nz][ny][nx] (one
 * value per station and component, components in ascending bit order).
 * Precision flag, units, streams, ownership and errors as for the plane
 * plans.  Limits: nx, ny <= 1024, nz <= 512, at most 8 components. */

/* Build an equal-dimension plan (kernel over the offsets of Eq. 10 with
 * the layer offset as a third index, Eq. 11; three-level circulant spectra).
 * Blocks until done.  Arguments as grav_plan_create without h.  Returns NULL
 * on error (see grav_last_error).  Release it with grav_plan_destroy;
 * grav_plan_bytes and grav_plan_info apply; grav_forward, grav_adjoint and
 * the batched and static-scratch calls reject it with GRAV_EINVAL. */
grav_plan* grav_plan_create3d(int nx, int ny, int nz, double dx, double dy, double dz, unsigned components);

/* d_c(p,q,t) = sum_{l,m,n} K_c(l-p, m-q, n-t) rho(l,m,n) at every cell centre.
 *   rho_dev  device [nz][ny][nx]
 *   out_dev  device [ncomp][nz][ny][nx]; fully overwritten
 * Returns GRAV_OK, GRAV_EINVAL (null pointer, or not an equal-dimension
 * plan) or GRAV_ECUDA. */
int grav_forward3d(grav_plan* plan, const void* rho_dev, void* out_dev, void* stream);

/* Transpose: grad(l,m,n) = sum_c sum_{p,q,t} K_c(l-p, m-q, n-t) r_c(p,q,t).
 *   r_dev     device [ncomp][nz][ny][nx]
 *   grad_dev  device [nz][ny][nx]; fully overwritten
 * Status codes as grav_forward3d. */
int grav_adjoint3d(grav_plan* plan, const void* r_dev, void* grad_dev, void* stream);

/* Size of the library's static device scratch area (16 MiB per GPU). */
#define GRAV_STATIC_SCRATCH_BYTES (16u << 20)

/* Forward for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a library convenience.
 *
 * A caller whose device memory is all reserved by another framework's
 * allocator, or a serving loop that must not call cudaMalloc (it can
 * synchronise the device), creates its plans at start-up and may then need
 * scratch for a forward without asking for memory, for instance to run a
 * second forward on the same plan on another stream.  This entry point
 * computes exactly what grav_forward computes, with the same arguments,
 * types and status codes, but takes its per-call scratch from one static
 * array of GRAV_STATIC_SCRATCH_BYTES that the library holds on every GPU it
 * is loaded on, instead of the plan's workspaces.  It allocates nothing.
 *
 * Limits and rules:
 *   - the plan's scratch need, (px/2 + 1) ny' (nz + 2 ncomp) complex values
 *     (ny' = ny rounded up to a multiple of 4, FP32 or FP64 as the plan),
 *     must fit in GRAV_STATIC_SCRATCH_BYTES; otherwise GRAV_EINVAL with the
 *     sizes in grav_last_error().  FP32 meshes up to 128 x 128 x 32 fit.
 *   - the current device must be the plan's device (GRAV_EINVAL otherwise).
 *   - the first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *     The address is looked up again whenever the device's CUDA context is
 *     a new one (after cudaDeviceReset), on the first call made after that.
 *   - every call, on any plan, shares the one array: calls whose work
 *     overlaps on the GPU race and give wrong results.  Order them on one
 *     stream or with events.  No contents need clearing between calls. */
int grav_forward_static_scratch(grav_plan* plan, const void* rho_dev, void* out_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GRAV_H */
