"""Particle kernel, interpolation J and spreading S on the staggered grid.

Grid convention (App. A.1): scalar fields live at cell centres r_i = h i; the
alpha component of a vector field lives on the alpha-face r_i + (h/2) e_alpha.
Arrays are indexed [z, y, x] (x fastest), periodic in every direction.

The kernel is the tensor product delta_h(r) = h^-3 prod_alpha phi(r_alpha / h)
with the 3-point Roma-Peskin function phi (App. A.1), so each particle touches
27 points of each location set.  Following Eq. (Jdis) the h^3 of the cell
volume cancels the h^-3 of the kernel: J f = sum_i w_i f_i with the
dimensionless weights w_i = prod_alpha phi(.), while S F puts w_i F / h^3 on
point i (Eq. (Sdis)).
"""
import numpy as np

# offsets (in units of h) of the four location sets, ordered (x, y, z)
CENTRE = (0.0, 0.0, 0.0)
FACE = ((0.5, 0.0, 0.0), (0.0, 0.5, 0.0), (0.0, 0.0, 0.5))


def phi(r):
    """3-point Roma-Peskin function (App. A.1)."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    inner = a <= 0.5
    outer = (a > 0.5) & (a <= 1.5)
    out[inner] = (1.0 + np.sqrt(1.0 - 3.0 * a[inner] ** 2)) / 3.0
    out[outer] = (5.0 - 3.0 * a[outer] - np.sqrt(1.0 - 3.0 * (1.0 - a[outer]) ** 2)) / 6.0
    return out


def stencil_1d(q, h, offset, n):
    """Indices and 1D weights of the 3 points nearest to q along one axis.

    The grid points of this location set sit at (i + offset) h.  With
    s = q/h - offset the nearest point is i0 = floor(s + 1/2) (a tie at a
    half-integer s is harmless: phi(1.5) = 0).  Returns (idx (..., 3) int,
    w (..., 3) float64) with idx taken modulo n.
    """
    s = np.asarray(q, dtype=np.float64) / h - offset
    i0 = np.floor(s + 0.5).astype(np.int64)
    d = np.arange(-1, 2)
    pts = i0[..., None] + d
    w = phi(pts - s[..., None])
    return np.mod(pts, n), w


class Stencils:
    """Cached 27-point stencils of a set of particles for one location set.

    q : (np, 3) positions (x, y, z); shape : grid shape (nz, ny, nx).
    ``flat`` (np, 27) linear indices into the [z, y, x] array and ``w`` (np, 27)
    the dimensionless tensor-product weights.
    """

    def __init__(self, q, h, shape, offset):
        q = np.atleast_2d(np.asarray(q, dtype=np.float64))
        nz, ny, nx = shape
        ix, wx = stencil_1d(q[:, 0], h, offset[0], nx)
        iy, wy = stencil_1d(q[:, 1], h, offset[1], ny)
        iz, wz = stencil_1d(q[:, 2], h, offset[2], nz)
        # point order: x fastest, then y, then z (c = a + 3 b + 9 d)
        self.flat = (iz[:, :, None, None] * ny + iy[:, None, :, None]) * nx + ix[:, None, None, :]
        self.w = wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
        self.flat = self.flat.reshape(q.shape[0], 27)
        self.w = self.w.reshape(q.shape[0], 27)

    def interp(self, field):
        """J f for every particle: sum_i w_i f_i (Eq. (Jdis))."""
        return np.sum(self.w * field.reshape(-1)[self.flat], axis=1)

    def spread(self, values, shape, h):
        """S F summed over particles: point i receives w_i F_p / h^3 (Eq. (Sdis)).

        Contributions are added in particle order, then point order.
        """
        out = np.zeros(int(np.prod(shape)))
        np.add.at(out, self.flat.reshape(-1),
                  (self.w * (np.asarray(values, dtype=np.float64)[:, None] / h ** 3)).reshape(-1))
        return out.reshape(shape)


def all_stencils(q, h, shape):
    """Stencils for the centre set and the three face sets."""
    return (Stencils(q, h, shape, CENTRE),
            tuple(Stencils(q, h, shape, FACE[a]) for a in range(3)))


def kernel_volume(h):
    """V = 1 / (J S) = 8 h^3 for the 3-point kernel (Eq. (kvol), Sec. 2.1)."""
    return 8.0 * h ** 3
