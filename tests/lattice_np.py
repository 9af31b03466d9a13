"""Closed-form bond endpoints of the pyrochlore lattice in numpy, for tests
at sizes where the oracle's geometric tables do not fit (L = 256).  Pinned
against the oracle's geometric bond list at small L (test_lattice_np.py).

Bond 12 r + k, r = 4 c + f: k < 6 pairs basis vertices (a, b) of the
tetrahedron of FCC point r; k >= 6 the same pairs of the tetrahedron through
site 4 r whose vertex v (v > 0) sits in cell c - h(f, v), FCC point f ^ v."""
import numpy as np

PA = np.array([0, 0, 0, 1, 1, 2])
PB = np.array([1, 2, 3, 2, 3, 3])


def _a(f, d):
    f = np.asarray(f)
    return np.where(d == 0, (f >> 1) & 1, np.where(d == 1, f & 1, (f & 1) ^ ((f >> 1) & 1)))


def _vertex_site(L, c, f, v):
    """Global site of vertex v of the down tetrahedron of FCC point (c, f)."""
    x, y, z = c % L, (c // L) % L, c // (L * L)
    out = np.empty_like(c)
    for axis, coord in enumerate((x, y, z)):
        step = ((_a(f, axis) == 0) & (_a(v, axis) == 1) & (v > 0)).astype(np.int64)
        coord_new = (coord - step) % L
        if axis == 0:
            xn = coord_new
        elif axis == 1:
            yn = coord_new
        else:
            zn = coord_new
    cell = xn + L * (yn + L * zn)
    out = np.where(v == 0, 16 * c + 4 * f, 16 * cell + 4 * (f ^ v) + v)
    return out


def bond_endpoints(L: int, b: np.ndarray):
    b = np.asarray(b, dtype=np.int64)
    r, k = b // 12, b % 12
    c, f = r >> 2, r & 3
    kk = np.where(k < 6, k, k - 6)
    va, vb = PA[kk], PB[kk]
    up_i, up_j = 4 * r + va, 4 * r + vb
    dn_i = _vertex_site(L, c, f, va)
    dn_j = _vertex_site(L, c, f, vb)
    return np.where(k < 6, up_i, dn_i), np.where(k < 6, up_j, dn_j)
