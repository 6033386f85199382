"""Pins of the oracle's further Laplacian stencils (Sec. 2.2.2: the isotropic 9-point 2D and
19- and 27-point 3D second-order stencils, the fourth-order 9-point 2D stencil) against
closed forms:
Fourier symbols, exactness on polynomials, isotropy of the leading error, and the structure
of the stencil matrix."""
import itertools

import numpy as np
import pytest

import oracle


def _symbol(stencil, k, h):
    """Closed-form eigenvalue of the stencil on the Fourier mode exp(i k.x)."""
    a = [ki * h for ki in k]
    if stencil == "9iso":
        ca, cb = np.cos(a[0]), np.cos(a[1])
        return (8.0 * (ca + cb) + 4.0 * ca * cb - 20.0) / (6.0 * h * h)
    if stencil == "9o4":
        return sum(32.0 * np.cos(t) - 2.0 * np.cos(2.0 * t) - 30.0 for t in a) / (12.0 * h * h)
    if stencil == "19iso":
        c = [np.cos(t) for t in a]
        return (4.0 * sum(c) + 4.0 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2]) - 24.0) / (6.0 * h * h)
    if stencil == "27iso":
        # faces 2 cos, edges 4 cos cos per axis pair, corners 8 cos cos cos
        c = [np.cos(t) for t in a]
        pairs = c[0] * c[1] + c[0] * c[2] + c[1] * c[2]
        return (28.0 * sum(c) + 12.0 * pairs + 8.0 * c[0] * c[1] * c[2] - 128.0) / (30.0 * h * h)
    return -(4.0 / (h * h)) * sum(np.sin(t / 2) ** 2 for t in a)


@pytest.mark.parametrize("stencil,shape,h", [("9iso", (16, 12), 0.7), ("9o4", (14, 18), 1.3),
                                             ("19iso", (8, 10, 6), 0.9), ("std", (8, 6, 10), 1.0),
                                             ("27iso", (6, 8, 10), 1.1)])
def test_fourier_symbol(stencil, shape, h):
    rng = np.random.default_rng(1)
    coords = np.meshgrid(*[np.arange(n) * h for n in shape], indexing="ij")
    for _ in range(6):
        m = [int(rng.integers(0, n)) for n in shape]
        k = [2 * np.pi * mi / (n * h) for mi, n in zip(m, shape)]
        phase = sum(ki * c for ki, c in zip(k, coords)) + 0.4
        phi = np.cos(phase)
        lam = _symbol(stencil, k, h)
        got = oracle.laplacian_stencil(phi, h, stencil)
        np.testing.assert_allclose(got, lam * phi, rtol=0, atol=1e-12 * max(1.0, abs(lam)))


def _interior(shape, r):
    return tuple(slice(r, n - r) for n in shape)


def test_second_order_stencils_are_exact_on_quadratics():
    h = 0.5
    y, x = np.meshgrid(np.arange(32) * h, np.arange(32) * h, indexing="ij")
    f = 1.5 * x * x - 0.5 * x * y + 2.0 * y * y + 0.3 * x - 0.7 * y
    for st in ("std", "9iso", "9o4"):
        lap = oracle.laplacian_stencil(f, h, st)
        np.testing.assert_allclose(lap[_interior(f.shape, 2)], 2 * 1.5 + 2 * 2.0, rtol=0,
                                   atol=1e-9)
    z, y, x = np.meshgrid(*[np.arange(20) * h] * 3, indexing="ij")
    g = x * x + 2.0 * y * y - z * z + x * y + y * z
    for st in ("19iso", "27iso"):
        lap = oracle.laplacian_stencil(g, h, st)
        np.testing.assert_allclose(lap[_interior(g.shape, 1)], 2 + 4 - 2, rtol=0, atol=1e-9)


def test_fourth_order_stencil_is_exact_on_quartics():
    h = 0.25
    y, x = np.meshgrid(np.arange(40) * h, np.arange(40) * h, indexing="ij")
    f = x ** 4 + y ** 4 + x * x * y * y - 3.0 * x ** 3
    exact = 12 * x * x + 12 * y * y + 2 * y * y + 2 * x * x - 18.0 * x
    sl = _interior(f.shape, 2)
    np.testing.assert_allclose(oracle.laplacian_stencil(f, h, "9o4")[sl], exact[sl], rtol=0,
                               atol=1e-8)
    # while the 5-point stencil is not (its error is h^2/12 times the fourth derivatives)
    assert np.abs(oracle.laplacian_stencil(f, h, "std")[sl] - exact[sl]).max() > 1e-3


@pytest.mark.parametrize("iso,std,dim", [("9iso", "std", 2), ("19iso", "std", 3),
                                         ("27iso", "std", 3)])
def test_isotropic_stencils_have_isotropic_leading_error(iso, std, dim):
    # eigenvalue along an axis vs along a diagonal at the same |k|: the isotropic stencils
    # agree to O(k^6), the standard one differs at O(k^4)
    kk = 0.15
    axis = [kk] + [0.0] * (dim - 1)
    diag = [kk / np.sqrt(dim)] * dim
    aniso_iso = abs(_symbol(iso, axis, 1.0) - _symbol(iso, diag, 1.0))
    aniso_std = abs(_symbol(std, axis, 1.0) - _symbol(std, diag, 1.0))
    assert aniso_iso < 1e-6 < aniso_std
    # and both approximate -k^2
    assert abs(_symbol(iso, diag, 1.0) + kk * kk) < 1e-4
    # isotropy at O(k^4) holds along every direction, not only the two above
    rng = np.random.default_rng(5)
    for _ in range(4):
        u = rng.standard_normal(dim)
        u *= kk / np.linalg.norm(u)
        assert abs(_symbol(iso, u, 1.0) - _symbol(iso, axis, 1.0)) < 1e-6


@pytest.mark.parametrize("stencil,shape,points", [("9iso", (6, 7), 9), ("9o4", (7, 6), 9),
                                                  ("19iso", (5, 5, 6), 19),
                                                  ("27iso", (5, 6, 5), 27)])
def test_stencil_matrix_support_symmetry_and_zero_row_sums(stencil, shape, points):
    n = int(np.prod(shape))
    L = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        L[:, j] = oracle.laplacian_stencil(e.reshape(shape), 1.0, stencil).ravel()
    assert np.all(np.count_nonzero(L, axis=1) == points)
    np.testing.assert_allclose(L, L.T, atol=1e-15)
    np.testing.assert_allclose(L.sum(axis=1), 0.0, atol=1e-12)


def test_allen_cahn_linear_closed_form_with_isotropic_stencil():
    shape, h = (16, 20), 0.8
    m = (3, 2)
    coords = np.meshgrid(*[np.arange(n) * h for n in shape], indexing="ij")
    k = [2 * np.pi * mi / (n * h) for mi, n in zip(m, shape)]
    phi0 = 0.2 * np.cos(sum(ki * c for ki, c in zip(k, coords)))
    c1, dt, n = 0.6, 0.03, 30
    out, = oracle.run("ac", (phi0,), (c1, 0.0), dt, n, h, stencil="9iso")
    g = 1.0 + dt * (_symbol("9iso", k, h) + c1)
    np.testing.assert_allclose(out, g ** n * phi0, rtol=0, atol=1e-12)


def test_27_point_weights_by_direction_class():
    # a unit impulse: the stencil's value at each offset is its weight; 14/3/1 per face, edge
    # and corner neighbour and -128 at the centre, over 30 h^2
    h = 0.5
    e = np.zeros((5, 5, 5))
    e[2, 2, 2] = 1.0
    L = oracle.laplacian_stencil(e, h, "27iso") * (30.0 * h * h)
    for o in itertools.product((-1, 0, 1), repeat=3):
        w = {0: -128.0, 1: 14.0, 2: 3.0, 3: 1.0}[sum(1 for x in o if x)]
        assert L[2 + o[0], 2 + o[1], 2 + o[2]] == w
    assert np.count_nonzero(L) == 27
