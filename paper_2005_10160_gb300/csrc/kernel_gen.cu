// FP64 kernel generation: the translation-equivalent geometric kernel
// K_c(u, v, n) of every component c over the offset grid (Eq. 10), i.e. the
// first row and column of every Toeplitz block of G (Eqs. 17, 19).
//
// K_c(u, v, n) is the field at a station due to a unit-density cell offset
// by (u, v) columns in layer n.  With the station at the origin the cell has
// corners x_i = (1/2 - u) dx, -(1/2 + u) dx, y_j likewise, z_k = -h - zeta_k
// with zeta in {n dz, (n+1) dz}, and
//     K_c = upsilon * sum_{ijk} mu_ijk F_c(x_i, y_j, z_k),  mu_ijk = (-1)^(i+j+k)
// (Eq. 2).  F_c is the closed form of Eq. 2 for gz (its logarithms written
// as asinh, which is the same function and keeps far offsets accurate) and
// the standard prism forms for the gradient components:
//     gxx: atan(yz/(xr))   gyy: atan(xz/(yr))   gzz: atan(xy/(zr))
//     gxy: -asinh(z/sqrt(x^2+y^2))   gxz: -asinh(y/sqrt(x^2+z^2))
//     gyz: -asinh(x/sqrt(y^2+z^2))
// and for the horizontal first derivatives the gz form with x (resp. y) as
// the distinguished axis:
//     gx: -[y asinh(z/sqrt(x^2+y^2)) + z asinh(y/sqrt(x^2+z^2)) - x atan(yz/(xr))]
//     gy: -[z asinh(x/sqrt(y^2+z^2)) + x asinh(z/sqrt(x^2+y^2)) - y atan(xz/(yr))]
// FP64 throughout: the eight corner terms cancel to a few parts in 1e7 at
// the far offsets of a 1024-cell mesh, so FP32 generation is unusable.
//
// One thread per offset (u, v) of the quadrant u, v >= 0, in tiles that
// share their corner terms (see kernel_gen below).  Walking down the layers,
// each thread writes the four mirrored offsets (+-u, +-v) using the
// component's parity under reflection (Sec. 2.2), so the stored kernel is
// exactly even or odd.
#include "grav_internal.h"

namespace grav {

namespace {

// NC: components kept per corner, 7 (gz ... gzz) or 9 (with gx, gy); plans
// without gx, gy use 7 so that the kernel keeps fewer registers.
template <int NC>
__device__ __forceinline__ void corner_terms(double x, double y, double z, unsigned comps, double (&F)[NC]) {
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double r = sqrt(x2 + y2 + z2);
    double ay = 0.0, ax = 0.0, az = 0.0, tz = 0.0, tx = 0.0, ty = 0.0;
    if (comps & (GRAV_GZ | GRAV_GXZ | GRAV_GX)) ay = asinh(y / sqrt(x2 + z2));
    if (comps & (GRAV_GZ | GRAV_GYZ | GRAV_GY)) ax = asinh(x / sqrt(y2 + z2));
    if (comps & (GRAV_GXY | GRAV_GX | GRAV_GY)) az = asinh(z / sqrt(x2 + y2));
    if (comps & (GRAV_GZ | GRAV_GZZ)) tz = atan(x * y / (z * r));
    if (comps & (GRAV_GXX | GRAV_GX)) tx = atan(y * z / (x * r));
    if (comps & (GRAV_GYY | GRAV_GY)) ty = atan(x * z / (y * r));
    F[0] = -(x * ay + y * ax - z * tz);
    F[1] = tx;
    F[2] = -az;
    F[3] = -ay;
    F[4] = ty;
    F[5] = -ax;
    F[6] = tz;
    if constexpr (NC > 7) {
        F[7] = -(y * az + z * ay - x * tx);  // gx: the gz form with x as the distinguished axis
        F[8] = -(z * ax + x * az - y * ty);  // gy: the same with y
    }
}

// Offsets per CTA: a kGenTX x kGenTY tile of the quadrant.  Neighbouring
// offsets share prism corners (the far x-corner of offset u is the near one
// of u + 1), so the CTA evaluates the corner terms of its (kGenTX + 1) x
// (kGenTY + 1) corners once per z-level into shared memory (two levels kept:
// the bottom of layer n is the top of layer n + 1) and every thread forms
// its offset's kernel values from its eight corners.  The FP64 work per
// offset and level drops from four corner evaluations to about 1.2.
constexpr int kGenTX = 32, kGenTY = 8;

template <int NC>
__global__ void __launch_bounds__(kGenTX * kGenTY)
    kernel_gen(Geometry g, unsigned comps, int n0, int n1, int mode, int px, int py, double* __restrict__ out) {
    constexpr int CX = kGenTX + 1, CY = kGenTY + 1, NCOR = CX * CY, NT = kGenTX * kGenTY;
    __shared__ double F[2][CY][CX][NC];  // corner terms of two z-levels
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kGenTX + tx;
    const int u0 = blockIdx.x * kGenTX, v0 = blockIdx.y * kGenTY;
    const int u = u0 + tx, v = v0 + ty;

    // corner terms of z-level z into buffer buf: corner (cu, cv) sits at
    // x = (1/2 - cu) dx, y = (1/2 - cv) dy (station at the origin)
    auto level = [&](int buf, double z) {
        for (int e = tid; e < NCOR; e += NT) {
            const int cy = e / CX, cx = e - cy * CX;
            const int cu = u0 + cx, cv = v0 + cy;
            double t[NC];
            if (cu <= g.nx && cv <= g.ny) {
                corner_terms<NC>((0.5 - cu) * g.dx, (0.5 - cv) * g.dy, z, comps, t);
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) t[c] = 0.0;
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) F[buf][cy][cx][c] = t[c];
        }
    };

    const int nzc = n1 - n0;
    const int wx = 2 * g.nx - 1, wy = 2 * g.ny - 1;
    int cur = 0;
    level(cur, -g.h - n0 * g.dz);
    for (int n = n0; n < n1; ++n) {
        level(cur ^ 1, -g.h - (n + 1) * g.dz);
        __syncthreads();
        if (u < g.nx && v < g.ny) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if (!(comps & (1u << c))) continue;
                const int s = __popc(comps & ((1u << c) - 1u));  // output slot of component c
                // mu_ijk: +1 for the bottom z-level when i + j is even; corners
                // (u + i, v + j)
                const double d00 = F[cur ^ 1][ty][tx][c] - F[cur][ty][tx][c];
                const double d01 = F[cur ^ 1][ty + 1][tx][c] - F[cur][ty + 1][tx][c];
                const double d10 = F[cur ^ 1][ty][tx + 1][c] - F[cur][ty][tx + 1][c];
                const double d11 = F[cur ^ 1][ty + 1][tx + 1][c] - F[cur][ty + 1][tx + 1][c];
                const double K = kUpsilon * ((d00 - d01) - (d10 - d11));
                for (int mu = 0; mu < (u > 0 ? 2 : 1); ++mu) {
                    for (int mv = 0; mv < (v > 0 ? 2 : 1); ++mv) {
                        double val = K;
                        if (mu && odd_u(c)) val = -val;
                        if (mv && odd_v(c)) val = -val;
                        if ((u == 0 && odd_u(c)) || (v == 0 && odd_v(c))) val = 0.0;
                        const int U = mu ? -u : u, V = mv ? -v : v;
                        size_t idx;
                        if (mode == 0) {
                            const int a = (px - U) & (px - 1), b = (py - V) & (py - 1);
                            idx = (((size_t)s * nzc + (n - n0)) * py + b) * px + a;
                        } else if (mode == 2) {
                            // rows b = -V < py / 2 only (V <= 0): the rest mirror them
                            if (V > 0) continue;
                            const int a = (px - U) & (px - 1), b = -V;
                            idx = (((size_t)s * nzc + (n - n0)) * (py / 2) + b) * px + a;
                        } else {
                            idx = (((size_t)s * g.nz + n) * wy + (V + g.ny - 1)) * wx + (U + g.nx - 1);
                        }
                        out[idx] = val;
                    }
                }
            }
        }
        __syncthreads();  // the next level overwrites this level's top buffer
        cur ^= 1;
    }
}

}  // namespace

cudaError_t launch_kernel_gen(const Geometry& g, unsigned comps, int n0, int n1, int mode, int px, int py,
                              double* out, cudaStream_t s) {
    const dim3 block(kGenTX, kGenTY);
    const dim3 grid((g.nx + kGenTX - 1) / kGenTX, (g.ny + kGenTY - 1) / kGenTY);
    comps &= kCompBits;
    if (comps & (GRAV_GX | GRAV_GY))
        kernel_gen<9><<<grid, block, 0, s>>>(g, comps, n0, n1, mode, px, py, out);
    else
        kernel_gen<7><<<grid, block, 0, s>>>(g, comps, n0, n1, mode, px, py, out);
    return cudaGetLastError();
}

}  // namespace grav
