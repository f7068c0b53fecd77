/*
 * Test infrastructure, not product code: the plain FP64 CPU oracle for the
 * right-prism gravity / gravity-gradient forward model.  Only tests/, the
 * smoke check and the CPU-baseline leg of bench.py use it.  It shares no
 * code, header or table with the CUDA library.
 *
 * What it computes is the plain definition of the method's result, d = G M
 * (Eqs. 3-4, Sec. 2.1): every station/cell pair gets its own kernel value
 * from the eight-corner closed form, with no offset reuse, no symmetry and no
 * FFT.  Each kernel value is
 *
 *     G_c(P, Q) = upsilon * sum_{i,j,k in {1,2}} mu_ijk F_c(x_i, y_j, z_k)
 *
 * with x_i = x - xi_i, y_j = y - eta_j, z_k = z - zeta_k (station minus
 * prism corner, z positive down), r = sqrt(x^2 + y^2 + z^2) and
 * mu_ijk = (-1)^(i+j+k) (Eq. 2).  Index 1 is the lower coordinate.
 *
 *   gz  (Eq. 2): F = -[x asinh(y/sqrt(x^2+z^2)) + y asinh(x/sqrt(y^2+z^2))
 *                     - z atan(x y / (z r))]
 *   The paper prints ln(t + sqrt(1 + t^2)); that is asinh(t) exactly, and the
 *   asinh spelling avoids the cancellation the ln form suffers for t << 0.
 *
 *   Gradient components: the paper names them (Eq. 1) but prints only gz
 *   (Sec. 2.1).  The standard prism forms (Nagy, Papp and Benedek 2000,
 *   J. Geodesy 74) are used:
 *   gxx: F =  atan(y z / (x r))      gyy: F = atan(x z / (y r))
 *   gzz: F =  atan(x y / (z r))      gxy: F = -asinh(z / sqrt(x^2 + y^2))
 *   gxz: F = -asinh(y / sqrt(x^2 + z^2))
 *   gyz: F = -asinh(x / sqrt(y^2 + z^2))
 *   The horizontal first derivatives gx, gy (the x and y counterparts of gz,
 *   positive towards +x and +y) are the same eight-corner form with the axes
 *   permuted cyclically (z -> x, resp. z -> y, as the distinguished axis):
 *   gx:  F = -[y asinh(z/sqrt(x^2+y^2)) + z asinh(y/sqrt(x^2+z^2))
 *              - x atan(y z / (x r))]
 *   gy:  F = -[z asinh(x/sqrt(y^2+z^2)) + x asinh(z/sqrt(x^2+y^2))
 *              - y atan(x z / (y r))]
 *
 * Geometry (the mesh of Fig. 1 and the index order of Sec. 2.2,
 * j = l + nx*m + nx*ny*n):
 *   cell (l, m, n) spans [l dx, (l+1) dx] x [m dy, (m+1) dy] x [n dz, (n+1) dz]
 *   station (p, q) sits at ((p + 1/2) dx, (q + 1/2) dy, -h), h > 0
 *   In the equal-dimension variant (Sec. 2.2, Eqs. 10-11: data as
 *   three-dimensional as the mesh) station (p, q, t) sits at the centre of
 *   cell (p, q, t), index i = p + nx*q + nx*ny*t.  A cell centre is never on
 *   a corner plane of any cell, so every term of the closed forms is
 *   finite; at the station's own cell they give the interior field.
 *   upsilon = 6.672e-11 N m^2 / kg^2 (Sec. 2.1, below Eq. 2).
 * Units: density kg/m^3, gz in m/s^2, gradients in 1/s^2.
 *
 * Component bits (ascending bit order is the output row order):
 *   1 gz, 2 gxx, 4 gxy, 8 gxz, 16 gyy, 32 gyz, 64 gzz, 128 gx, 256 gy.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_UPSILON 6.672e-11
#define ORC_NCOMP_MAX 9

/* Eight-corner sums for one prism seen from one station, all nine
 * components, per unit density and including upsilon.  out[0..8] =
 * gz, gxx, gxy, gxz, gyy, gyz, gzz, gx, gy. */
void orc_prism(double x, double y, double z,
               double xi1, double xi2, double eta1, double eta2,
               double zeta1, double zeta2, double out[ORC_NCOMP_MAX])
{
    const double xs[2] = {x - xi1, x - xi2};
    const double ys[2] = {y - eta1, y - eta2};
    const double zs[2] = {z - zeta1, z - zeta2};
    double acc[ORC_NCOMP_MAX] = {0};
    for (int i = 0; i < 2; ++i) {
        for (int j = 0; j < 2; ++j) {
            for (int k = 0; k < 2; ++k) {
                /* mu = (-1)^(i+j+k) with 1-based indices = (-1)^(i+j+k+3) */
                const double mu = ((i + j + k) % 2 == 0) ? -1.0 : 1.0;
                const double xi = xs[i], yj = ys[j], zk = zs[k];
                const double r = sqrt(xi * xi + yj * yj + zk * zk);
                const double rxz = sqrt(xi * xi + zk * zk);
                const double ryz = sqrt(yj * yj + zk * zk);
                const double rxy = sqrt(xi * xi + yj * yj);
                const double a_y = asinh(yj / rxz);
                const double a_x = asinh(xi / ryz);
                const double a_z = asinh(zk / rxy);
                const double t_z = atan(xi * yj / (zk * r));
                const double t_x = atan(yj * zk / (xi * r));
                const double t_y = atan(xi * zk / (yj * r));
                acc[0] += mu * -(xi * a_y + yj * a_x - zk * t_z);
                acc[1] += mu * t_x;
                acc[2] += mu * -a_z;
                acc[3] += mu * -a_y;
                acc[4] += mu * t_y;
                acc[5] += mu * -a_x;
                acc[6] += mu * t_z;
                acc[7] += mu * -(yj * a_z + zk * a_y - xi * t_x);
                acc[8] += mu * -(zk * a_x + xi * a_z - yj * t_y);
            }
        }
    }
    for (int c = 0; c < ORC_NCOMP_MAX; ++c) out[c] = ORC_UPSILON * acc[c];
}

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, h;
    unsigned comps;
} orc_mesh;

static int orc_comp_list(unsigned comps, int list[ORC_NCOMP_MAX])
{
    int nc = 0;
    for (int c = 0; c < ORC_NCOMP_MAX; ++c)
        if (comps & (1u << c)) list[nc++] = c;
    return nc;
}

/* Kernel value of every selected component for station (p, q) and cell
 * (l, m, n): one row of G (Eq. 3). */
static void orc_pair(const orc_mesh* g, int p, int q, int l, int m, int n,
                     double out[ORC_NCOMP_MAX])
{
    const double x = (p + 0.5) * g->dx, y = (q + 0.5) * g->dy, z = -g->h;
    orc_prism(x, y, z, l * g->dx, (l + 1) * g->dx, m * g->dy, (m + 1) * g->dy,
              n * g->dz, (n + 1) * g->dz, out);
}

/* Kernel value for station (p, q, t) at the centre of cell (p, q, t) and
 * cell (l, m, n): the equal-dimension variant. */
static void orc_pair3d(const orc_mesh* g, int p, int q, int t, int l, int m, int n,
                       double out[ORC_NCOMP_MAX])
{
    const double x = (p + 0.5) * g->dx, y = (q + 0.5) * g->dy, z = (t + 0.5) * g->dz;
    orc_prism(x, y, z, l * g->dx, (l + 1) * g->dx, m * g->dy, (m + 1) * g->dy,
              n * g->dz, (n + 1) * g->dz, out);
}

typedef struct {
    const orc_mesh* g;
    const double* rho;     /* [nz][ny][nx] */
    const double* resid;   /* [ncomp][ny][nx] for the adjoint */
    const int* idx;        /* stations (forward) or cells (adjoint) */
    int n_idx;
    double* out;
    int tid, nthreads;
} orc_job;

/* d_c(station) = sum over all cells of G_c(station, cell) rho(cell), in plain
 * sequential cell order j = l + nx m + nx ny n (Eq. 3). */
static void* orc_forward_worker(void* arg)
{
    orc_job* jb = (orc_job*)arg;
    const orc_mesh* g = jb->g;
    int list[ORC_NCOMP_MAX];
    const int nc = orc_comp_list(g->comps, list);
    for (int s = jb->tid; s < jb->n_idx; s += jb->nthreads) {
        const int st = jb->idx[s];
        const int p = st % g->nx, q = st / g->nx;
        double acc[ORC_NCOMP_MAX] = {0};
        for (int n = 0; n < g->nz; ++n)
            for (int m = 0; m < g->ny; ++m)
                for (int l = 0; l < g->nx; ++l) {
                    const double rho = jb->rho[((size_t)n * g->ny + m) * g->nx + l];
                    double k[ORC_NCOMP_MAX];
                    orc_pair(g, p, q, l, m, n, k);
                    for (int c = 0; c < nc; ++c) acc[c] += k[list[c]] * rho;
                }
        for (int c = 0; c < nc; ++c) jb->out[(size_t)c * jb->n_idx + s] = acc[c];
    }
    return NULL;
}

/* The same sum for stations at cell centres (equal-dimension variant):
 * station index i = p + nx q + nx ny t. */
static void* orc_forward3d_worker(void* arg)
{
    orc_job* jb = (orc_job*)arg;
    const orc_mesh* g = jb->g;
    int list[ORC_NCOMP_MAX];
    const int nc = orc_comp_list(g->comps, list);
    for (int s = jb->tid; s < jb->n_idx; s += jb->nthreads) {
        const int st = jb->idx[s];
        const int p = st % g->nx, q = (st / g->nx) % g->ny, t = st / (g->nx * g->ny);
        double acc[ORC_NCOMP_MAX] = {0};
        for (int n = 0; n < g->nz; ++n)
            for (int m = 0; m < g->ny; ++m)
                for (int l = 0; l < g->nx; ++l) {
                    const double rho = jb->rho[((size_t)n * g->ny + m) * g->nx + l];
                    double k[ORC_NCOMP_MAX];
                    orc_pair3d(g, p, q, t, l, m, n, k);
                    for (int c = 0; c < nc; ++c) acc[c] += k[list[c]] * rho;
                }
        for (int c = 0; c < nc; ++c) jb->out[(size_t)c * jb->n_idx + s] = acc[c];
    }
    return NULL;
}

/* (G^T r)(cell) = sum over components and stations of G_c(station, cell)
 * r_c(station): the transpose of Eq. 4. */
static void* orc_adjoint_worker(void* arg)
{
    orc_job* jb = (orc_job*)arg;
    const orc_mesh* g = jb->g;
    int list[ORC_NCOMP_MAX];
    const int nc = orc_comp_list(g->comps, list);
    const size_t nd = (size_t)g->nx * g->ny;
    for (int s = jb->tid; s < jb->n_idx; s += jb->nthreads) {
        const int cell = jb->idx[s];
        const int l = cell % g->nx, m = (cell / g->nx) % g->ny, n = cell / (g->nx * g->ny);
        double acc = 0.0;
        for (int q = 0; q < g->ny; ++q)
            for (int p = 0; p < g->nx; ++p) {
                double k[ORC_NCOMP_MAX];
                orc_pair(g, p, q, l, m, n, k);
                for (int c = 0; c < nc; ++c)
                    acc += k[list[c]] * jb->resid[(size_t)c * nd + (size_t)q * g->nx + p];
            }
        jb->out[s] = acc;
    }
    return NULL;
}

/* Equal-dimension variant: (G^T r)(cell) over the stations at cell centres;
 * r: [ncomp][nz][ny][nx]. */
static void* orc_adjoint3d_worker(void* arg)
{
    orc_job* jb = (orc_job*)arg;
    const orc_mesh* g = jb->g;
    int list[ORC_NCOMP_MAX];
    const int nc = orc_comp_list(g->comps, list);
    const size_t nm = (size_t)g->nx * g->ny * g->nz;
    for (int s = jb->tid; s < jb->n_idx; s += jb->nthreads) {
        const int cell = jb->idx[s];
        const int l = cell % g->nx, m = (cell / g->nx) % g->ny, n = cell / (g->nx * g->ny);
        double acc = 0.0;
        for (int t = 0; t < g->nz; ++t)
            for (int q = 0; q < g->ny; ++q)
                for (int p = 0; p < g->nx; ++p) {
                    double k[ORC_NCOMP_MAX];
                    orc_pair3d(g, p, q, t, l, m, n, k);
                    const size_t i = ((size_t)t * g->ny + q) * g->nx + p;
                    for (int c = 0; c < nc; ++c) acc += k[list[c]] * jb->resid[(size_t)c * nm + i];
                }
        jb->out[s] = acc;
    }
    return NULL;
}

static int orc_run(void* (*fn)(void*), orc_job* proto, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    pthread_t th[512];
    orc_job jobs[512];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].tid = t;
        jobs[t].nthreads = nthreads;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) break;
        started = t;
    }
    /* Threads that failed to start have their share done here. */
    for (int t = started + 1; t < nthreads; ++t) fn(&jobs[t]);
    fn(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    return 0;
}

static int orc_check(int nx, int ny, int nz, double dx, double dy, double dz,
                     double h, unsigned comps)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    if (!(dx > 0) || !(dy > 0) || !(dz > 0) || !(h > 0)) return -1;
    if (comps == 0 || (comps & ~0x1FFu)) return -1;
    return 0;
}

/* Forward at a subset of stations.  rho: [nz][ny][nx]; st_idx: station
 * indices p + nx q; out: [ncomp][n_st].  Returns 0, or -1 on bad input. */
int orc_forward(int nx, int ny, int nz, double dx, double dy, double dz, double h,
                unsigned comps, const double* rho, int n_st, const int* st_idx,
                double* out, int nthreads)
{
    if (orc_check(nx, ny, nz, dx, dy, dz, h, comps) || n_st < 0) return -1;
    for (int s = 0; s < n_st; ++s)
        if (st_idx[s] < 0 || st_idx[s] >= nx * ny) return -1;
    orc_mesh g = {nx, ny, nz, dx, dy, dz, h, comps};
    orc_job jb;
    memset(&jb, 0, sizeof jb);
    jb.g = &g; jb.rho = rho; jb.idx = st_idx; jb.n_idx = n_st; jb.out = out;
    return orc_run(orc_forward_worker, &jb, nthreads);
}

/* Adjoint at a subset of cells.  resid: [ncomp][ny][nx]; cell_idx: cell
 * indices l + nx m + nx ny n; out: [n_cells]. */
int orc_adjoint(int nx, int ny, int nz, double dx, double dy, double dz, double h,
                unsigned comps, const double* resid, int n_cells, const int* cell_idx,
                double* out, int nthreads)
{
    if (orc_check(nx, ny, nz, dx, dy, dz, h, comps) || n_cells < 0) return -1;
    for (int s = 0; s < n_cells; ++s)
        if (cell_idx[s] < 0 || cell_idx[s] >= nx * ny * nz) return -1;
    orc_mesh g = {nx, ny, nz, dx, dy, dz, h, comps};
    orc_job jb;
    memset(&jb, 0, sizeof jb);
    jb.g = &g; jb.resid = resid; jb.idx = cell_idx; jb.n_idx = n_cells; jb.out = out;
    return orc_run(orc_adjoint_worker, &jb, nthreads);
}

/* Explicit kernel matrix G (Eqs. 3-5) for tiny meshes:
 * G[c][i][j], i = p + nx q (station), j = l + nx m + nx ny n (cell). */
int orc_gmatrix(int nx, int ny, int nz, double dx, double dy, double dz, double h,
                unsigned comps, double* G)
{
    if (orc_check(nx, ny, nz, dx, dy, dz, h, comps)) return -1;
    orc_mesh g = {nx, ny, nz, dx, dy, dz, h, comps};
    int list[ORC_NCOMP_MAX];
    const int nc = orc_comp_list(comps, list);
    const size_t nd = (size_t)nx * ny, nm = (size_t)nx * ny * nz;
    for (size_t i = 0; i < nd; ++i)
        for (size_t j = 0; j < nm; ++j) {
            double k[ORC_NCOMP_MAX];
            orc_pair(&g, (int)(i % nx), (int)(i / nx), (int)(j % nx),
                     (int)((j / nx) % ny), (int)(j / nd), k);
            for (int c = 0; c < nc; ++c) G[((size_t)c * nd + i) * nm + j] = k[list[c]];
        }
    return 0;
}

/* Equal-dimension variant: forward at a subset of the stations at cell
 * centres.  rho: [nz][ny][nx]; st_idx: station indices p + nx q + nx ny t;
 * out: [ncomp][n_st].  h is not used.  Returns 0, or -1 on bad input. */
int orc_forward3d(int nx, int ny, int nz, double dx, double dy, double dz,
                  unsigned comps, const double* rho, int n_st, const int* st_idx,
                  double* out, int nthreads)
{
    if (orc_check(nx, ny, nz, dx, dy, dz, 1.0, comps) || n_st < 0) return -1;
    for (int s = 0; s < n_st; ++s)
        if (st_idx[s] < 0 || st_idx[s] >= nx * ny * nz) return -1;
    orc_mesh g = {nx, ny, nz, dx, dy, dz, 0.0, comps};
    orc_job jb;
    memset(&jb, 0, sizeof jb);
    jb.g = &g; jb.rho = rho; jb.idx = st_idx; jb.n_idx = n_st; jb.out = out;
    return orc_run(orc_forward3d_worker, &jb, nthreads);
}

/* Equal-dimension variant: adjoint at a subset of cells.  resid:
 * [ncomp][nz][ny][nx] (one value per station at a cell centre); cell_idx:
 * cell indices l + nx m + nx ny n; out: [n_cells]. */
int orc_adjoint3d(int nx, int ny, int nz, double dx, double dy, double dz,
                  unsigned comps, const double* resid, int n_cells, const int* cell_idx,
                  double* out, int nthreads)
{
    if (orc_check(nx, ny, nz, dx, dy, dz, 1.0, comps) || n_cells < 0) return -1;
    for (int s = 0; s < n_cells; ++s)
        if (cell_idx[s] < 0 || cell_idx[s] >= nx * ny * nz) return -1;
    orc_mesh g = {nx, ny, nz, dx, dy, dz, 0.0, comps};
    orc_job jb;
    memset(&jb, 0, sizeof jb);
    jb.g = &g; jb.resid = resid; jb.idx = cell_idx; jb.n_idx = n_cells; jb.out = out;
    return orc_run(orc_adjoint3d_worker, &jb, nthreads);
}

/* Equal-dimension variant, explicit G for tiny meshes: G[c][i][j],
 * i = p + nx q + nx ny t (station at the centre of cell i), j as above. */
int orc_gmatrix3d(int nx, int ny, int nz, double dx, double dy, double dz,
                  unsigned comps, double* G)
{
    if (orc_check(nx, ny, nz, dx, dy, dz, 1.0, comps)) return -1;
    orc_mesh g = {nx, ny, nz, dx, dy, dz, 0.0, comps};
    int list[ORC_NCOMP_MAX];
    const int nc = orc_comp_list(comps, list);
    const size_t nd = (size_t)nx * ny, nm = nd * nz;
    for (size_t i = 0; i < nm; ++i)
        for (size_t j = 0; j < nm; ++j) {
            double k[ORC_NCOMP_MAX];
            orc_pair3d(&g, (int)(i % nx), (int)((i / nx) % ny), (int)(i / nd), (int)(j % nx),
                       (int)((j / nx) % ny), (int)(j / nd), k);
            for (int c = 0; c < nc; ++c) G[((size_t)c * nm + i) * nm + j] = k[list[c]];
        }
    return 0;
}
