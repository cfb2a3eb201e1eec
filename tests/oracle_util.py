"""Small helpers shared by the oracle pin tests (no model arithmetic here)."""
import numpy as np

# D3Q19 velocity set, written out again for the tests so that the checks do
# not borrow the oracle's own table.
C19 = np.array([
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=np.float64)


def momentum(f, mask=None):
    """Total momentum sum_x sum_i f_i c_i (fluid nodes only if mask given)."""
    w = np.ones(f.shape[1:]) if mask is None else (mask == 0).astype(np.float64)
    return np.array([np.sum(np.tensordot(C19[:, a], f, axes=(0, 0)) * w) for a in range(3)])


def neighbours_inside(shape, periodic, X, R):
    """Boolean field: fluid node with at least one D3Q19 neighbour strictly
    inside the sphere (brute force over all nodes and directions)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def inside(xx, yy, zz):
        d = []
        for c, L, Xa, per in ((xx, nx, X[0], periodic[0]), (yy, ny, X[1], periodic[1]),
                              (zz, nz, X[2], periodic[2])):
            dd = c - Xa
            if per:
                dd = np.where(dd > 0.5 * L, dd - L, np.where(dd < -0.5 * L, dd + L, dd))
            d.append(dd)
        return d[0] ** 2 + d[1] ** 2 + d[2] ** 2 < R * R

    solid = inside(x.astype(float), y.astype(float), z.astype(float))
    adj = np.zeros(shape, dtype=bool)
    for c in C19[1:]:
        xs, ys, zs = (x + int(c[0])), (y + int(c[1])), (z + int(c[2]))
        ok = np.ones(shape, dtype=bool)
        for arr, L, per in ((xs, nx, periodic[0]), (ys, ny, periodic[1]), (zs, nz, periodic[2])):
            if per:
                arr %= L
            else:
                ok &= (arr >= 0) & (arr < L)
        xs, ys, zs = np.clip(xs, 0, nx - 1), np.clip(ys, 0, ny - 1), np.clip(zs, 0, nz - 1)
        adj |= ok & solid[zs, ys, xs]
    return adj & ~solid, solid
