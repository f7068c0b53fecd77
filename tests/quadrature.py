"""Brute-force Gauss-Legendre quadrature of the Newtonian volume integrals of
a uniform right prism: an independent check of the oracle's closed forms.

With d = Q - P (source point minus station, z positive down) and r = |d|:
    g_a  = upsilon rho int d_a / r^3 dV    (a = z, x, y)
    g_ab = upsilon rho int (3 d_a d_b - r^2 delta_ab) / r^5 dV
(the first and second derivatives of the potential upsilon rho int 1/r dV).
"""
import numpy as np

UPSILON = 6.672e-11


def _nodes(a, b, nsub, order):
    xg, wg = np.polynomial.legendre.leggauss(order)
    e = np.linspace(a, b, nsub + 1)
    xs, ws = [], []
    for i in range(nsub):
        lo, hi = e[i], e[i + 1]
        xs.append(0.5 * (hi - lo) * xg + 0.5 * (hi + lo))
        ws.append(0.5 * (hi - lo) * wg)
    return np.concatenate(xs), np.concatenate(ws)


def prism_quadrature(station, box, nsub=8, order=16):
    """[gz, gxx, gxy, gxz, gyy, gyz, gzz, gx, gy] per unit density."""
    X, WX = _nodes(box[0], box[1], nsub, order)
    Y, WY = _nodes(box[2], box[3], nsub, order)
    Z, WZ = _nodes(box[4], box[5], nsub, order)
    dx = X[:, None, None] - station[0]
    dy = Y[None, :, None] - station[1]
    dz = Z[None, None, :] - station[2]
    w = WX[:, None, None] * WY[None, :, None] * WZ[None, None, :]
    r2 = dx * dx + dy * dy + dz * dz
    r = np.sqrt(r2)
    r3 = r2 * r
    r5 = r3 * r2
    out = [
        (w * dz / r3).sum(),
        (w * (3 * dx * dx - r2) / r5).sum(),
        (w * 3 * dx * dy / r5).sum(),
        (w * 3 * dx * dz / r5).sum(),
        (w * (3 * dy * dy - r2) / r5).sum(),
        (w * 3 * dy * dz / r5).sum(),
        (w * (3 * dz * dz - r2) / r5).sum(),
        (w * dx / r3).sum(),
        (w * dy / r3).sum(),
    ]
    return UPSILON * np.array(out)


def point_mass(station, centre, mass):
    """Point-mass field [gz, gxx, gxy, gxz, gyy, gyz, gzz, gx, gy] of ``mass`` kg."""
    d = np.asarray(centre, float) - np.asarray(station, float)
    R2 = float(d @ d)
    R = np.sqrt(R2)
    g = UPSILON * mass
    T = g * (3 * np.outer(d, d) - R2 * np.eye(3)) / R ** 5
    return np.array([g * d[2] / R ** 3, T[0, 0], T[0, 1], T[0, 2], T[1, 1], T[1, 2], T[2, 2],
                     g * d[0] / R ** 3, g * d[1] / R ** 3])
