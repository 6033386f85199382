"""Pins of the oracle's forward-Euler models (Sec. 2.4.1, Sec. 3 equations, Gray-Scott
in its standard form): linear closed forms, fixed point, conservation, energy decrease,
energy-gradient identity, symmetry, and a per-site brute force on tiny grids."""
import itertools

import numpy as np
import pytest

import oracle
import synthetic


def _mode(shape, m, h, amp=1.0, phase=0.2):
    coords = np.meshgrid(*[np.arange(n) * h for n in shape], indexing="ij")
    k = [2 * np.pi * mi / (n * h) for mi, n in zip(m, shape)]
    lam = -(4.0 / h ** 2) * sum(np.sin(ki * h / 2) ** 2 for ki in k)
    return amp * np.cos(sum(ki * c for ki, c in zip(k, coords)) + phase), lam


@pytest.mark.parametrize("shape,m,h", [((16, 16), (3, 1), 1.0), ((8, 10, 6), (1, 2, 1), 0.8)])
def test_allen_cahn_linear_closed_form(shape, m, h):
    # c2 = 0: a Fourier mode is multiplied by g = 1 + dt (lam + c1) per step.
    phi0, lam = _mode(shape, m, h, amp=0.3)
    c1, dt, n = 0.7, 0.05, 40
    out, = oracle.run("ac", (phi0,), (c1, 0.0), dt, n, h)
    g = 1.0 + dt * (lam + c1)
    np.testing.assert_allclose(out, g ** n * phi0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape,m,h", [((16, 12), (2, 3), 1.0), ((8, 8, 6), (1, 1, 1), 1.0)])
def test_cahn_hilliard_linear_closed_form(shape, m, h):
    # c2 = 0: g = 1 + dt M (-lam^2 - c1 lam).
    phi0, lam = _mode(shape, m, h, amp=0.1)
    c1, M, dt, n = 1.0, 0.8, 0.005, 50
    out, = oracle.run("ch", (phi0,), (c1, 0.0, M), dt, n, h)
    g = 1.0 + dt * M * (-lam * lam - c1 * lam)
    np.testing.assert_allclose(out, g ** n * phi0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [(16, 16), (6, 8, 10)])
def test_gray_scott_v_zero_closed_form(shape):
    # v = 0 stays exactly 0, and u - 1 decays per Fourier mode by g = 1 + dt (Du lam - F).
    mode, lam = _mode(shape, (1,) * len(shape), 1.0, amp=1e-2)
    Du, Dv, F, k, dt, n = 0.2, 0.1, 0.04, 0.06, 0.5, 30
    u, v = oracle.run("gs", (1.0 + mode, np.zeros(shape)), (Du, Dv, F, k), dt, n)
    assert np.all(v == 0.0)
    g = 1.0 + dt * (Du * lam - F)
    np.testing.assert_allclose(u - 1.0, g ** n * mode, rtol=0, atol=1e-14)


def test_gray_scott_fixed_point():
    u = np.ones((5, 6, 7))
    v = np.zeros((5, 6, 7))
    u1, v1 = oracle.run("gs", (u, v), (0.2, 0.1, 0.04, 0.06), 0.5, 10)
    assert np.all(u1 == 1.0) and np.all(v1 == 0.0)


@pytest.mark.parametrize("shape", [(32, 24), (10, 12, 8)])
def test_cahn_hilliard_conserves_mass(shape):
    phi0 = synthetic.cahn_hilliard_init(shape, seed=11, amp=0.3).astype(np.float64) + 0.1
    m0 = oracle.mass(phi0)
    out, = oracle.run("ch", (phi0,), (1.0, 1.0, 1.0), 0.01, 300)
    assert abs(oracle.mass(out) - m0) <= 1e-12 * np.abs(phi0).sum()
    assert np.abs(out - phi0).max() > 1e-3  # it did evolve


def test_allen_cahn_energy_decreases_at_config_dt():
    # dt = 0.05 < 2 / (4d/h^2 + 3 c2 - c1) = 0.2 with |phi| <= 1: E^{n+1} <= E^n every step.
    phi = synthetic.allen_cahn_init((128, 128), seed=1).astype(np.float64)
    e_prev = oracle.energy(phi)
    for _ in range(1000):
        phi, = oracle.euler_step("ac", (phi,), (1.0, 1.0), 0.05)
        e = oracle.energy(phi)
        assert e <= e_prev + 1e-12 * abs(e_prev)
        e_prev = e
    assert np.abs(phi).max() <= 1.0


@pytest.mark.parametrize("shape,h", [((6, 5), 1.0), ((4, 3, 5), 0.6)])
def test_energy_gradient_is_allen_cahn_rhs(shape, h):
    # Complex-step derivative: -Im E(phi + i eps e_x) / eps / h^d == rhs_AC(phi)_x.
    rng = np.random.default_rng(5)
    phi = rng.uniform(-0.8, 0.8, shape)
    c1, c2, eps = 0.9, 1.3, 1e-30
    f = oracle.rhs_allen_cahn(phi, c1, c2, h)
    for site in itertools.islice(itertools.product(*[range(n) for n in shape]), 0, None, 3):
        z = phi.astype(np.complex128)
        z[site] += 1j * eps
        dE = np.imag(oracle.energy(z, c1, c2, h)) / eps
        assert abs(-dE / h ** len(shape) - f[site]) <= 1e-12 * max(1.0, abs(f[site]))


def _brute_force_step(model, fields, coeffs, dt, h):
    """Per-site loops with explicit neighbour indices; CH computes mu everywhere first."""
    shape = fields[0].shape
    d = len(shape)
    sites = list(itertools.product(*[range(n) for n in shape]))

    def lap(a, s):
        acc = 0.0
        for ax in range(d):
            for sgn in (-1, 1):
                nb = list(s)
                nb[ax] = (nb[ax] + sgn) % shape[ax]
                acc += a[tuple(nb)] - a[s]
        return acc / (h * h)

    out = [f.copy() for f in fields]
    if model == "ac":
        c1, c2 = coeffs
        p = fields[0]
        for s in sites:
            out[0][s] = p[s] + dt * (lap(p, s) + c1 * p[s] - c2 * p[s] ** 3)
    elif model == "ch":
        c1, c2, M = coeffs
        p = fields[0]
        mu = np.zeros(shape)
        for s in sites:
            mu[s] = c2 * p[s] ** 3 - c1 * p[s] - lap(p, s)
        for s in sites:
            out[0][s] = p[s] + dt * M * lap(mu, s)
    elif model == "c":
        c1, c2, c3, c4, c5 = coeffs
        p, q = fields
        mu = np.zeros(shape)
        for s in sites:
            mu[s] = c4 * q[s] ** 3 - c3 * q[s] - c5 * p[s] ** 2 - lap(q, s)
        for s in sites:
            out[0][s] = p[s] + dt * (lap(p, s) + c1 * p[s] - c2 * p[s] ** 3 + 2 * c5 * p[s] * q[s])
            out[1][s] = q[s] + dt * lap(mu, s)
    else:
        Du, Dv, F, k = coeffs
        u, v = fields
        for s in sites:
            r = u[s] * v[s] * v[s]
            out[0][s] = u[s] + dt * (Du * lap(u, s) - r + F * (1 - u[s]))
            out[1][s] = v[s] + dt * (Dv * lap(v, s) + r - (F + k) * v[s])
    return tuple(out)


@pytest.mark.parametrize("model,coeffs", [("ac", (1.0, 1.0)), ("ch", (0.8, 1.2, 0.9)),
                                          ("gs", (0.2, 0.1, 0.04, 0.06)),
                                          ("c", (0.9, 1.1, 0.8, 1.2, 0.7))])
@pytest.mark.parametrize("shape", [(3, 4), (5, 5), (2, 3, 4)])
def test_step_matches_per_site_brute_force(model, coeffs, shape):
    rng = np.random.default_rng(17)
    nf = 2 if model in ("gs", "c") else 1
    fields = tuple(rng.uniform(-0.5, 1.0, shape) for _ in range(nf))
    h, dt = 0.9, 0.01
    ref = _brute_force_step(model, fields, coeffs, dt, h)
    got = oracle.euler_step(model, fields, coeffs, dt, h)
    for r, g in zip(ref, got):
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-13)


@pytest.mark.parametrize("model,coeffs", [("ac", (1.0, 1.0)), ("ch", (1.0, 1.0, 1.0)),
                                          ("gs", (0.2, 0.1, 0.04, 0.06)),
                                          ("c", (1.0, 1.0, 1.0, 1.0, 1.0))])
def test_step_commutes_with_grid_symmetries(model, coeffs):
    # Periodic translations, axis reflections and the transpose of a square grid commute
    # with the step: catches a wrong axis, sign or transposed operand.
    rng = np.random.default_rng(23)
    nf = 2 if model in ("gs", "c") else 1
    fields = tuple(rng.uniform(0.0, 1.0, (12, 12)) for _ in range(nf))
    base = oracle.euler_step(model, fields, coeffs, 0.01)
    for op in (lambda a: np.roll(a, 3, axis=0), lambda a: np.roll(a, -5, axis=1),
               lambda a: a[::-1, :], lambda a: a[:, ::-1], lambda a: a.T):
        moved = oracle.euler_step(model, tuple(op(f) for f in fields), coeffs, 0.01)
        for b, m in zip(base, moved):
            np.testing.assert_allclose(m, op(b), rtol=0, atol=1e-15)


# ------------------------------------------------------------------------ Model C

@pytest.mark.parametrize("shape,m_", [((16, 12), (2, 3)), ((8, 6, 10), (1, 1, 2))])
def test_model_c_uncoupled_linear_closed_forms(shape, m_):
    # c2 = c4 = c5 = 0: psi modes grow by 1 + dt (lam + c1), m modes by 1 + dt (-lam^2 - c3 lam)
    mode, lam = _mode(shape, m_, 1.0, amp=0.1)
    c1, c3, dt, n = 0.7, 0.9, 0.004, 40
    psi, m = oracle.run("c", (mode, 0.5 * mode), (c1, 0.0, c3, 0.0, 0.0), dt, n)
    np.testing.assert_allclose(psi, (1 + dt * (lam + c1)) ** n * mode, rtol=0, atol=1e-12)
    np.testing.assert_allclose(m, (1 + dt * (-lam * lam - c3 * lam)) ** n * 0.5 * mode, rtol=0,
                               atol=1e-12)


def test_model_c_reduces_to_models_a_and_b_without_coupling():
    rng = np.random.default_rng(31)
    psi, m = rng.uniform(-0.5, 0.5, (12, 10)), rng.uniform(-0.5, 0.5, (12, 10))
    fp, fm = oracle.rhs_model_c(psi, m, 0.8, 1.3, 0.6, 1.1, 0.0)
    np.testing.assert_allclose(fp, oracle.rhs_allen_cahn(psi, 0.8, 1.3), rtol=0, atol=1e-13)
    np.testing.assert_allclose(fm, oracle.rhs_cahn_hilliard(m, 0.6, 1.1, 1.0), rtol=0, atol=1e-13)


def test_model_c_conserves_m_and_its_energy_decreases():
    rng = np.random.default_rng(37)
    psi, m = rng.uniform(-0.3, 0.3, (32, 32)), rng.uniform(-0.3, 0.3, (32, 32)) + 0.1
    coeffs = (1.0, 1.0, 1.0, 1.0, 1.0)
    m0 = oracle.mass(m)
    e_prev = oracle.energy_model_c(psi, m, *coeffs)
    x = (psi, m)
    for _ in range(300):
        x = oracle.euler_step("c", x, coeffs, 0.005)
        e = oracle.energy_model_c(*x, *coeffs)
        assert e <= e_prev + 1e-12 * abs(e_prev)
        e_prev = e
    assert abs(oracle.mass(x[1]) - m0) <= 1e-12 * np.abs(m).sum()


@pytest.mark.parametrize("shape", [(5, 6), (3, 4, 5)])
def test_model_c_energy_gradients_by_complex_step(shape):
    # -dE/dpsi = f_psi and dE/dm = mu_m (whose Laplacian is f_m)
    rng = np.random.default_rng(41)
    psi, m = rng.uniform(-0.8, 0.8, shape), rng.uniform(-0.8, 0.8, shape)
    c = (0.9, 1.2, 0.7, 1.3, 0.6)
    fp, _ = oracle.rhs_model_c(psi, m, *c)
    mu = c[3] * m ** 3 - c[2] * m - c[4] * psi ** 2 - oracle.laplacian(m)
    eps = 1e-30
    for site in itertools.islice(itertools.product(*[range(n) for n in shape]), 0, None, 4):
        zp = psi.astype(np.complex128)
        zp[site] += 1j * eps
        dpsi = np.imag(oracle.energy_model_c(zp, m, *c)) / eps
        zm = m.astype(np.complex128)
        zm[site] += 1j * eps
        dm = np.imag(oracle.energy_model_c(psi, zm, *c)) / eps
        assert abs(-dpsi - fp[site]) <= 1e-12 * max(1.0, abs(fp[site]))
        assert abs(dm - mu[site]) <= 1e-12 * max(1.0, abs(mu[site]))
