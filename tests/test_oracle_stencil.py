"""Pins of the oracle's periodic Laplacian (Sec. 2.2.2) against things other than itself:
hand-derived fixtures, closed forms, a brute-force dense matrix and Fourier eigenvalues."""
import itertools
import os

import numpy as np
import pytest

import oracle


def _read_blocks(path):
    """Numeric blocks of a golden file, split at comment lines."""
    blocks, cur = [], []
    for line in open(path):
        line = line.strip()
        if not line:
            continue
        if line.startswith("#"):
            if cur:
                blocks.append(np.array(cur, dtype=np.float64))
                cur = []
            continue
        cur.append([float(t) for t in line.split()])
    if cur:
        blocks.append(np.array(cur, dtype=np.float64))
    return blocks


def test_laplacian_golden_ramp_4x4(golden_dir):
    phi, expected = _read_blocks(os.path.join(golden_dir, "laplacian_ramp_4x4.txt"))
    np.testing.assert_array_equal(oracle.laplacian(phi), expected)


@pytest.mark.parametrize("shape", [(3, 4, 5), (5, 2, 3), (7, 6), (2, 9)])
def test_laplacian_ramp_closed_form(shape):
    # phi = sum_ax w_ax * i_ax; along a periodic axis of n points the ramp's second
    # difference is n at i = 0, -n at i = n - 1 and 0 elsewhere.
    d = len(shape)
    w = [10.0 ** (d - 1 - ax) for ax in range(d)]
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    phi = sum(wi * g for wi, g in zip(w, grids))
    expect = np.zeros(shape)
    for ax, n in enumerate(shape):
        a = np.zeros(n)
        a[0] += n
        a[n - 1] -= n
        if n == 1:
            a[:] = 0
        sh = [1] * d
        sh[ax] = n
        expect = expect + w[ax] * a.reshape(sh)
    h = 0.5
    np.testing.assert_allclose(oracle.laplacian(phi, h), expect / h ** 2, rtol=0, atol=1e-12)


def _dense_laplacian(shape, h):
    """Dense periodic Laplacian built by enumerating each site's +-1 neighbours."""
    n = int(np.prod(shape))
    L = np.zeros((n, n))
    strides = [int(np.prod(shape[ax + 1:])) for ax in range(len(shape))]
    for site in itertools.product(*[range(s) for s in shape]):
        i = sum(c * st for c, st in zip(site, strides))
        for ax in range(len(shape)):
            for sgn in (-1, 1):
                nb = list(site)
                nb[ax] = (nb[ax] + sgn) % shape[ax]
                j = sum(c * st for c, st in zip(nb, strides))
                L[i, j] += 1.0 / h ** 2
                L[i, i] -= 1.0 / h ** 2
    return L


@pytest.mark.parametrize("shape,h", [((8, 8), 1.0), ((4, 4, 4), 1.0), ((5, 7), 0.5),
                                     ((3, 4, 5), 0.7)])
def test_laplacian_matches_dense_matrix(shape, h):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(shape)
    L = _dense_laplacian(shape, h)
    np.testing.assert_allclose(oracle.laplacian(x, h).ravel(), L @ x.ravel(), rtol=0, atol=1e-12)
    # periodic Laplacian: symmetric, rows sum to zero
    np.testing.assert_array_equal(L, L.T)
    np.testing.assert_allclose(L.sum(axis=1), 0.0, atol=1e-12)


@pytest.mark.parametrize("shape,h", [((16, 12), 1.0), ((8, 6, 10), 1.0), ((12, 10), 0.7),
                                     ((6, 8, 4), 0.25)])
def test_laplacian_fourier_eigenvalue(shape, h):
    # For phi = cos(k . x), k_i = 2 pi m_i / (N_i h):  lap_h phi = -(4/h^2) sum sin^2(k_i h/2) phi
    rng = np.random.default_rng(3)
    coords = np.meshgrid(*[np.arange(n) * h for n in shape], indexing="ij")
    for _ in range(5):
        m = [int(rng.integers(0, n)) for n in shape]
        k = [2 * np.pi * mi / (n * h) for mi, n in zip(m, shape)]
        phase = sum(ki * c for ki, c in zip(k, coords)) + 0.3
        phi = np.cos(phase)
        lam = -(4.0 / h ** 2) * sum(np.sin(ki * h / 2) ** 2 for ki in k)
        np.testing.assert_allclose(oracle.laplacian(phi, h), lam * phi, rtol=0,
                                   atol=1e-12 * max(1.0, abs(lam)))


def test_bilaplacian_is_13_point_stencil(golden_dir):
    rows = _read_blocks(os.path.join(golden_dir, "bilaplacian_13pt.txt"))[0]
    n = 9
    delta = np.zeros((n, n))
    delta[0, 0] = 1.0
    f = oracle.rhs_cahn_hilliard(delta, c1=0.0, c2=0.0, M=1.0)
    expect = np.zeros((n, n))
    for dx, dy, w in rows:
        expect[int(dy) % n, int(dx) % n] = -w
    np.testing.assert_array_equal(f, expect)
