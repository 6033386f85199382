"""Pins of the oracle's semi-implicit Fourier spectral solver (Sec. 2.4.2) and structure
factor (Sec. 3): the scheme is exact on linear problems for any dt, conserves the conserved
fields exactly, keeps the uniform fixed point, agrees with an explicit step to O(dt^2), and
the wavenumber layout matches an explicit DFT; S(k) obeys Parseval and peaks at a stripe
pattern's wavenumber."""
import itertools

import numpy as np
import pytest

import oracle


def _mode(shape, m, h, amp):
    coords = np.meshgrid(*[np.arange(n) * h for n in shape], indexing="ij")
    k = [2 * np.pi * mi / (n * h) for mi, n in zip(m, shape)]
    return amp * np.cos(sum(ki * c for ki, c in zip(k, coords)) + 0.3), sum(ki * ki for ki in k)


@pytest.mark.parametrize("shape,h", [((12, 10), 0.7), ((6, 8, 10), 1.2)])
def test_wavenumber_layout_matches_explicit_dft(shape, h):
    # rfftn index (i, ..., j) carries frequency m with e^{-2 pi i m x / n}; check |k|^2 against
    # the explicit DFT sum of a single random coefficient on a small grid
    k2 = oracle.wavenumber_sq(shape, h)
    rng = np.random.default_rng(0)
    for _ in range(5):
        idx = tuple(int(rng.integers(0, s)) for s in k2.shape)
        freqs = [i if i <= n // 2 else i - n for i, n in zip(idx[:-1], shape[:-1])] + [idx[-1]]
        kk = sum((2 * np.pi * f / (n * h)) ** 2 for f, n in zip(freqs, shape))
        assert abs(k2[idx] - kk) <= 1e-12 * max(1.0, kk)
    # and the transform itself: an explicit DFT sum of a random field at one index
    f = rng.standard_normal(shape)
    idx = tuple(min(1, s - 1) for s in k2.shape)
    acc = 0.0 + 0.0j
    for site in itertools.product(*[range(n) for n in shape]):
        acc += f[site] * np.exp(-2j * np.pi * sum(i * x / n for i, x, n in zip(idx, site, shape)))
    assert abs(np.fft.rfftn(f)[idx] - acc) <= 1e-9


@pytest.mark.parametrize("shape,h", [((16, 12), 1.0), ((8, 10, 6), 0.8)])
def test_spectral_laplacian_of_a_mode(shape, h):
    phi, kk = _mode(shape, (1,) * len(shape), h, 1.0)
    ax = tuple(range(len(shape)))
    lap = np.fft.irfftn(-oracle.wavenumber_sq(shape, h) * np.fft.rfftn(phi), s=shape, axes=ax)
    np.testing.assert_allclose(lap, -kk * phi, rtol=0, atol=1e-11)


@pytest.mark.parametrize("model,coeffs", [("ac", (0.8, 0.0)), ("ch", (0.9, 0.0, 1.3))])
def test_linear_problems_are_integrated_exactly(model, coeffs):
    shape, h = (16, 20), 0.9
    phi, kk = _mode(shape, (2, 3), h, 0.1)
    dt, n = 0.37, 9  # any dt: the linear part is integrated exactly
    out, = oracle.spectral_run(model, (phi,), coeffs, dt, n, h)
    if model == "ac":
        L = -kk + coeffs[0]
    else:
        L = coeffs[2] * (-kk * kk + coeffs[0] * kk)
    np.testing.assert_allclose(out, np.exp(L * dt * n) * phi, rtol=0, atol=1e-12)


def test_model_c_uncoupled_fields_evolve_exactly():
    shape, h = (12, 16), 1.0
    p0, k1 = _mode(shape, (1, 2), h, 0.1)
    m0, k2 = _mode(shape, (3, 1), h, 0.05)
    c1, c3, dt, n = 0.7, 0.6, 0.2, 7
    psi, m = oracle.spectral_run("c", (p0, m0), (c1, 0.0, c3, 0.0, 0.0), dt, n, h)
    np.testing.assert_allclose(psi, np.exp((-k1 + c1) * dt * n) * p0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(m, np.exp((-k2 * k2 + c3 * k2) * dt * n) * m0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("model,coeffs,nf", [("ch", (1.0, 1.0, 1.0), 1), ("c", (1.0,) * 5, 2)])
def test_conserved_fields_keep_their_mass(model, coeffs, nf):
    rng = np.random.default_rng(4)
    x0 = tuple(rng.uniform(-0.5, 0.5, (24, 20)) + 0.1 for _ in range(nf))
    out = oracle.spectral_run(model, x0, coeffs, 0.05, 40)
    conserved = out[-1]  # m (Model B's only field, Model C's second)
    assert abs(conserved.sum() - x0[-1].sum()) <= 1e-11 * np.abs(x0[-1]).sum()
    assert np.abs(conserved - x0[-1]).max() > 1e-3


def test_uniform_fixed_point_of_model_a():
    c1, c2 = 0.8, 1.3
    psi0 = np.full((10, 12), np.sqrt(c1 / c2))
    out, = oracle.spectral_run("ac", (psi0,), (c1, c2), 0.5, 20)
    np.testing.assert_allclose(out, psi0, rtol=0, atol=1e-13)


@pytest.mark.parametrize("model,coeffs", [("ac", (1.0, 1.0)), ("ch", (1.0, 1.0, 0.8)),
                                          ("c", (0.9, 1.1, 0.8, 1.2, 0.7))])
def test_small_dt_agrees_with_explicit_step_to_second_order(model, coeffs):
    # one spectral step minus one explicit Euler step with the spectral Laplacian is O(dt^2);
    # the right-hand sides are the paper's equations written out here (Sec. 3)
    rng = np.random.default_rng(7)
    shape = (16, 16)
    x = rng.uniform(-0.4, 0.4, shape)
    y = rng.uniform(-0.4, 0.4, shape)
    k2 = oracle.wavenumber_sq(shape)
    lap = lambda a: np.fft.irfftn(-k2 * np.fft.rfftn(a), s=shape, axes=(0, 1))
    if model == "ac":
        fields, f = (x,), [lap(x) + coeffs[0] * x - coeffs[1] * x ** 3]
    elif model == "ch":
        c1, c2, M = coeffs
        fields, f = (x,), [-M * lap(lap(x)) - M * lap(c1 * x - c2 * x ** 3)]
    else:
        c1, c2, c3, c4, c5 = coeffs
        fields = (x, y)
        f = [lap(x) + c1 * x - c2 * x ** 3 + 2 * c5 * x * y,
             -lap(lap(y)) - lap(c3 * y - c4 * y ** 3 + c5 * x ** 2)]
    errs = []
    for dt in (1e-3, 5e-4):
        sp = oracle.spectral_run(model, fields, coeffs, dt, 1)
        errs.append(max(np.abs(s_ - (a + dt * fa)).max() for s_, a, fa in zip(sp, fields, f)))
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_structure_factor_parseval_and_stripe_peak():
    n, lam = 64, 8
    x = np.arange(n)
    psi = np.tile(np.cos(2 * np.pi * (x + 0.5) / lam), (n, 1))
    centres, mean, counts = oracle.structure_factor(psi, 1.0, n_bins=64)
    rho = (psi > 0).astype(float)
    total = (mean * counts).sum() + rho.sum() ** 2 / rho.size  # S(0) is excluded from bins
    assert abs(total - rho.sum()) <= 1e-9 * rho.sum()
    k0 = 2 * np.pi / lam
    assert abs(centres[np.argmax(mean)] - k0) <= (centres[1] - centres[0])
