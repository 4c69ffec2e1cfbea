"""Pins of the oracle's particle kernel, J and S (Sec. 2, App. A.1).

Checked against what the paper fixes: the moment conditions (Eqs. (k1),
(k2)), the position-independent norm 1/V with V = 8 h^3 (Eq. (kvol), Sec. 2.1),
the adjointness of J and S (Eq. (adj)), and a brute-force evaluation of the
kernel over every grid point with minimum-image distances.
"""
import numpy as np
import pytest

from oracle import peskin


def test_phi_closed_form_values():
    # phi(0) = 2/3, phi(1/2) = 1/2 from both branches, phi(1) = 1/6, phi(3/2) = 0
    assert peskin.phi(0.0) == pytest.approx(2.0 / 3.0, abs=1e-15)
    assert peskin.phi(0.5) == pytest.approx(0.5, abs=1e-15)
    assert peskin.phi(np.nextafter(0.5, 1.0)) == pytest.approx(0.5, abs=1e-7)
    assert peskin.phi(1.0) == pytest.approx(1.0 / 6.0, abs=1e-15)
    assert peskin.phi(-1.0) == pytest.approx(1.0 / 6.0, abs=1e-15)
    assert peskin.phi(1.5) == pytest.approx(0.0, abs=1e-15)
    assert peskin.phi(1.7) == 0.0


@pytest.mark.parametrize("seed", range(4))
def test_moment_conditions_1d(seed):
    """sum phi = 1, sum (r - q) phi = 0, sum phi^2 = 1/2 for any shift."""
    s = np.random.default_rng(seed).uniform(-3.0, 3.0, 2000)
    s = np.concatenate([s, [0.0, 0.5, -0.5, 1.5, 0.25]])
    idx, w = peskin.stencil_1d(s, 1.0, 0.0, 10 ** 6)
    pts = np.floor(s + 0.5)[:, None] + np.arange(-1, 2)
    assert np.allclose(w.sum(1), 1.0, atol=2e-15, rtol=0)
    assert np.allclose(((pts - s[:, None]) * w).sum(1), 0.0, atol=2e-15)
    assert np.allclose((w ** 2).sum(1), 0.5, atol=2e-15)


def test_kernel_volume_3d():
    """sum w^2 = 1/8 for all location sets, hence V = 1/(J S) = 8 h^3."""
    rng = np.random.default_rng(7)
    h = 0.7
    q = rng.uniform(0, 10 * h, (200, 3))
    c, faces = peskin.all_stencils(q, h, (10, 10, 10))
    for st in (c,) + faces:
        assert np.allclose(st.w.sum(1), 1.0, atol=1e-14)
        assert np.allclose((st.w ** 2).sum(1), 1.0 / 8.0, atol=1e-14)
    assert peskin.kernel_volume(h) == pytest.approx(8 * h ** 3)


def test_linear_fields_interpolated_exactly():
    """Eqs. (k1)-(k2): J of f(r) = a + b . r is f(q) (away from the periodic seam)."""
    h, n = 0.5, 16
    shape = (n, n, n)
    rng = np.random.default_rng(3)
    q = rng.uniform(3 * h, (n - 4) * h, (50, 3))
    a, b = 0.3, np.array([1.5, -0.7, 2.2])
    for off in (peskin.CENTRE,) + peskin.FACE:
        zz, yy, xx = np.meshgrid(*(h * (np.arange(n) + off[2 - i]) for i in range(3)), indexing="ij")
        f = a + b[0] * xx + b[1] * yy + b[2] * zz
        st = peskin.Stencils(q, h, shape, off)
        assert np.allclose(st.interp(f), a + q @ b, atol=1e-12)


def brute_force_kernel(q, h, shape, offset):
    """delta_h(q - r_i) h^3 at every grid point, minimum-image distances."""
    nz, ny, nx = shape
    out = np.zeros(shape)
    L = np.array([nx, ny, nz]) * h
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = (np.array([i, j, k]) + np.array(offset)) * h
                d = q - r
                d -= L * np.round(d / L)
                out[k, j, i] = np.prod(peskin.phi(d / h))
    return out


@pytest.mark.parametrize("offset", [peskin.CENTRE] + list(peskin.FACE))
def test_stencil_matches_brute_force_with_wraparound(offset):
    h, shape = 1.3, (4, 5, 6)
    rng = np.random.default_rng(11)
    qs = np.vstack([rng.uniform(0, 1, (5, 3)) * np.array([6, 5, 4]) * h,
                    [[0.02 * h, 0.01 * h, 3.99 * h]]])      # next to the periodic seam
    for q in qs:
        st = peskin.Stencils(q[None], h, shape, offset)
        dense = np.zeros(int(np.prod(shape)))
        np.add.at(dense, st.flat[0], st.w[0])
        assert np.allclose(dense.reshape(shape), brute_force_kernel(q, h, shape, offset), atol=1e-14)


def test_j_and_s_are_adjoint():
    """Eq. (adj): (J v) . u = sum_i h^3 v_i (S u)_i, checked as dense matrices."""
    h, shape = 0.9, (4, 4, 4)
    rng = np.random.default_rng(5)
    q = rng.uniform(0, 4 * h, (6, 3))
    ncell = 64
    for off in (peskin.CENTRE,) + peskin.FACE:
        st = peskin.Stencils(q, h, shape, off)
        jmat = np.stack([st.interp(np.eye(ncell)[i].reshape(shape)) for i in range(ncell)], axis=1)
        smat = np.stack([st.spread(np.eye(6)[p], shape, h).reshape(-1) for p in range(6)], axis=1)
        assert np.allclose(jmat, h ** 3 * smat.T, atol=1e-14)
        v = rng.normal(size=shape)
        u = rng.normal(size=6)
        assert np.dot(st.interp(v), u) == pytest.approx(h ** 3 * np.sum(v * st.spread(u, shape, h)),
                                                        rel=1e-13)


def test_half_integer_tie_is_continuous():
    """At s = k + 1/2 both neighbouring stencils give the same weights (phi(1.5) = 0)."""
    n = 8
    for s0 in (2.5, 3.5, 0.5):
        eps = 1e-12
        a_idx, a_w = peskin.stencil_1d(np.array([s0 - eps]), 1.0, 0.0, n)
        b_idx, b_w = peskin.stencil_1d(np.array([s0 + eps]), 1.0, 0.0, n)
        da = np.zeros(n)
        db = np.zeros(n)
        np.add.at(da, a_idx[0], a_w[0])
        np.add.at(db, b_idx[0], b_w[0])
        assert np.allclose(da, db, atol=1e-6)
