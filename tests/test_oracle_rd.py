"""Pins of the oracle's N-species reaction-diffusion right-hand side (any number of coupled
fields, Sec. 2.3; Gray-Scott of Sec. 1 is its two-species case):
  du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j^E[m][j].

Each pin comes from outside the function: closed forms of linear systems, an independently
written model (Gray-Scott), conservation laws of mass-action kinetics, and a per-site loop."""
import itertools

import numpy as np
import pytest

import oracle


def mode(shape, ks, h=1.0):
    grids = np.meshgrid(*[np.arange(n) * h for n in shape], indexing="ij")
    phase = sum(2 * np.pi * k * g / (n * h) for k, g, n in zip(ks, grids, shape))
    lam = -(4.0 / h ** 2) * sum(np.sin(np.pi * k / n) ** 2 for k, n in zip(ks, shape))
    return np.cos(phase), lam


@pytest.mark.parametrize("shape,ks", [((12, 16), (2, 3)), ((6, 8, 10), (1, 2, 3))])
def test_pure_diffusion_of_a_mode_is_exact(shape, ks):
    # K = 0: each field decays independently, a Fourier mode by (1 + dt D_i lambda)^n
    D = (0.3, 0.1, 0.05)
    c = oracle.rd_pack(D, np.zeros((1, 3)), np.zeros((3, 1)))
    phi, lam = mode(shape, ks, h=0.7)
    amps = (1.0, -0.5, 2.0)
    x0 = tuple(a * phi for a in amps)
    dt, n = 0.2, 13
    got = oracle.run("rd", x0, c, dt, n, h=0.7)
    for a, d, g in zip(amps, D, got):
        assert np.allclose(g, a * (1 + dt * d * lam) ** n * phi, rtol=0, atol=1e-13)


def test_linear_reactions_follow_the_matrix_power():
    # degree-1 monomials u_j with rates B: each Fourier mode's amplitude vector evolves by
    # (I + dt (B + lambda diag(D)))^n; a uniform state by (I + dt B)^n
    rng = np.random.default_rng(1)
    N = 4
    B = rng.uniform(-0.5, 0.5, (N, N))
    D = rng.uniform(0.0, 0.2, N)
    E = np.eye(N)
    c = oracle.rd_pack(D, E, B)
    shape = (8, 10)
    phi, lam = mode(shape, (1, 2))
    a0 = rng.uniform(-1, 1, N)
    b0 = rng.uniform(-1, 1, N)
    x0 = tuple(a0[i] + b0[i] * phi for i in range(N))
    dt, n = 0.1, 9
    got = oracle.run("rd", x0, c, dt, n)
    Au = np.linalg.matrix_power(np.eye(N) + dt * B, n)
    Am = np.linalg.matrix_power(np.eye(N) + dt * (B + lam * np.diag(D)), n)
    a_n, b_n = Au @ a0, Am @ b0
    for i in range(N):
        assert np.allclose(got[i], a_n[i] + b_n[i] * phi, rtol=0, atol=1e-12)


@pytest.mark.parametrize("shape", [(16, 12), (5, 6, 7)])
def test_gray_scott_is_a_two_species_case(shape):
    # monomials 1, u, v, u v^2: f_u = F - F u - u v^2, f_v = -(F + k) v + u v^2
    Du, Dv, F, k = 0.2, 0.1, 0.04, 0.06
    E = [[0, 0], [1, 0], [0, 1], [1, 2]]
    K = [[F, -F, 0.0, -1.0], [0.0, 0.0, -(F + k), 1.0]]
    c = oracle.rd_pack((Du, Dv), E, K)
    rng = np.random.default_rng(2)
    x0 = (rng.uniform(0.3, 1.0, shape), rng.uniform(0.0, 0.4, shape))
    a = oracle.run("rd", x0, c, 0.5, 6)
    b = oracle.run("gs", x0, (Du, Dv, F, k), 0.5, 6)
    for p, q in zip(a, b):
        assert np.abs(p - q).max() <= 1e-14


def test_mass_action_conserves_its_invariants():
    # A + B -> C at rate r, plus a spectator species S: sum(A + C), sum(B + C) and sum(S)
    # are conserved by both the reaction and the diffusion
    r = 1.3
    D = (0.2, 0.15, 0.05, 0.1)
    E = [[1, 1, 0, 0]]
    K = [[-r], [-r], [r], [0.0]]
    c = oracle.rd_pack(D, E, K)
    rng = np.random.default_rng(3)
    shape = (7, 9, 6)
    x = tuple(rng.uniform(0.0, 1.0, shape) for _ in range(4))
    inv0 = ((x[0] + x[2]).sum(), (x[1] + x[2]).sum(), x[3].sum())
    x = oracle.run("rd", x, c, 0.05, 60)
    inv = ((x[0] + x[2]).sum(), (x[1] + x[2]).sum(), x[3].sum())
    for a, b in zip(inv, inv0):
        assert abs(a - b) <= 1e-12 * abs(b)
    assert (x[2].sum() > 0.0) and (x[0].sum() < inv0[0])  # something reacted


def test_per_site_loop_on_a_tiny_grid():
    # three fields, cubic and mixed monomials: the right-hand side written as a loop over
    # sites and neighbours
    D = (0.3, 0.0, 0.7)
    E = [[0, 0, 0], [2, 1, 0], [0, 0, 3], [1, 1, 1], [0, 2, 0]]
    K = [[0.5, -1.0, 0.2, 0.0, 0.3], [0.0, 0.4, -0.6, 1.1, 0.0], [-0.2, 0.0, 0.0, 0.9, -0.7]]
    c = oracle.rd_pack(D, E, K)
    rng = np.random.default_rng(4)
    shape = (3, 4)
    u = [rng.uniform(-1, 1, shape) for _ in range(3)]
    h = 0.8
    got = oracle.rhs("rd", u, c, h)
    for i in range(3):
        for y, x in itertools.product(range(3), range(4)):
            nb = [u[i][(y + dy) % 3, (x + dx) % 4] for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1))]
            lap = (sum(nb) - 4 * u[i][y, x]) / h ** 2
            reac = 0.0
            for mm in range(len(E)):
                p = 1.0
                for j in range(3):
                    p *= u[j][y, x] ** E[mm][j]
                reac += K[i][mm] * p
            assert abs(got[i][y, x] - (D[i] * lap + reac)) <= 1e-13


def test_coefficient_layout_is_validated():
    with pytest.raises(ValueError):
        oracle.rd_unpack((0.1, 0.2, 1.0, 4, 0, 1.0, 1.0), 2)  # exponent 4
    with pytest.raises(ValueError):
        oracle.rd_unpack((0.1, 0.2, 1.5), 2)  # non-integer monomial count
    with pytest.raises(ValueError):
        oracle.rd_unpack((0.1,) * 6, 5)  # five fields
    D, E, K = oracle.rd_unpack(oracle.rd_pack((1.0, 2.0), [[1, 0]], [[3.0], [4.0]]), 2)
    assert list(D) == [1.0, 2.0] and E.tolist() == [[1, 0]] and K.tolist() == [[3.0], [4.0]]
