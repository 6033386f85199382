"""Pins of the oracle's Gray-Scott discrete adjoint: complex-step Jacobians of the forward
step, the dot-product identity, complex-step and FP64 central finite differences of the
whole time loop (the 32x32 copy of the 512x512 adjoint workload, 2000 steps)."""
import numpy as np
import pytest

import oracle
import synthetic

COEFFS = (0.2, 0.1, 0.04, 0.06)  # Du, Dv, F, k
DT = 0.5


def _cs_step_jvp(u, v, du, dv, coeffs=COEFFS, dt=DT, eps=1e-30):
    """J(x) dx of one forward step by the complex-step derivative (exact to roundoff)."""
    u1, v1 = oracle.euler_step("gs", (u + 1j * eps * du, v + 1j * eps * dv), coeffs, dt)
    return np.imag(u1) / eps, np.imag(v1) / eps


def test_adjoint_step_is_jacobian_transpose():
    rng = np.random.default_rng(1)
    shape = (4, 5)
    u, v = rng.uniform(0.3, 1.0, shape), rng.uniform(0.0, 0.4, shape)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    n = u.size
    # dense J by columns, then J^T lambda
    J = np.zeros((2 * n, 2 * n))
    for j in range(2 * n):
        e = np.zeros(2 * n)
        e[j] = 1.0
        ju, jv = _cs_step_jvp(u, v, e[:n].reshape(shape), e[n:].reshape(shape))
        J[:, j] = np.concatenate([ju.ravel(), jv.ravel()])
    lam = np.concatenate([a.ravel(), b.ravel()])
    expect = J.T @ lam
    a0, b0, _ = oracle.gray_scott_adjoint_step(u, v, a, b, *COEFFS, DT)
    np.testing.assert_allclose(np.concatenate([a0.ravel(), b0.ravel()]), expect, rtol=0,
                               atol=1e-12)


def test_adjoint_step_parameter_gradient():
    # d/dtheta <lambda, step(x; theta)> by complex step on each coefficient.
    rng = np.random.default_rng(2)
    shape = (6, 7)
    u, v = rng.uniform(0.3, 1.0, shape), rng.uniform(0.0, 0.4, shape)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    _, _, g = oracle.gray_scott_adjoint_step(u, v, a, b, *COEFFS, DT)
    eps = 1e-30
    for i in range(4):
        th = np.array(COEFFS, dtype=np.complex128)
        th[i] += 1j * eps
        u1, v1 = oracle.euler_step("gs", (u, v), tuple(th), DT)
        d = np.imag((a * u1).sum() + (b * v1).sum()) / eps
        assert abs(g[i] - d) <= 1e-12 * max(1.0, abs(d))


def test_dot_product_identity():
    rng = np.random.default_rng(3)
    shape = (9, 8)
    u, v = rng.uniform(0.3, 1.0, shape), rng.uniform(0.0, 0.4, shape)
    for _ in range(3):
        du, dv = rng.standard_normal(shape), rng.standard_normal(shape)
        a, b = rng.standard_normal(shape), rng.standard_normal(shape)
        ju, jv = _cs_step_jvp(u, v, du, dv)
        a0, b0, _ = oracle.gray_scott_adjoint_step(u, v, a, b, *COEFFS, DT)
        # lambda^n = lambda + dt J^T lambda is the transpose of x -> x + dt f(x)
        lhs = (ju * a).sum() + (jv * b).sum()
        rhs = (du * a0).sum() + (dv * b0).sum()
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def _target(u0, v0, n_steps, shape=None):
    Du, Dv, F, k = COEFFS
    return oracle.run("gs", (u0, v0), (Du, Dv, F + 0.002, k - 0.001), DT, n_steps)


def _loss_complex(u0, v0, coeffs, n_steps, ut, vt):
    u, v = oracle.run("gs", (u0, v0), coeffs, DT, n_steps)
    return 0.5 * (((u - ut) ** 2).sum() + ((v - vt) ** 2).sum())


@pytest.fixture(scope="module")
def adjoint_32():
    shape = (32, 32)
    u0, v0 = synthetic.workload_init("gs2d_adjoint_512", shape=shape)
    u0, v0 = u0.astype(np.float64), v0.astype(np.float64)
    n = 2000
    ut, vt = _target(u0, v0, n)
    uN, vN = oracle.run("gs", (u0, v0), COEFFS, DT, n)
    gu0, gv0, gth = oracle.gray_scott_adjoint(u0, v0, COEFFS, DT, n, uN - ut, vN - vt)
    return dict(u0=u0, v0=v0, n=n, ut=ut, vt=vt, gu0=gu0, gv0=gv0, gth=gth)


def test_adjoint_vs_complex_step_theta(adjoint_32):
    d = adjoint_32
    eps = 1e-30
    for i in range(4):
        th = np.array(COEFFS, dtype=np.complex128)
        th[i] += 1j * eps
        L = _loss_complex(d["u0"], d["v0"], tuple(th), d["n"], d["ut"], d["vt"])
        dL = np.imag(L) / eps
        assert abs(d["gth"][i] - dL) <= 1e-9 * max(1e-3, abs(dL)), (i, d["gth"][i], dL)


def test_adjoint_vs_central_differences(adjoint_32):
    # FP64 central differences, eps = 1e-6 max(1, |theta|): all four coefficients and
    # 16 random directions in (u0, v0).
    d = adjoint_32
    rng = np.random.default_rng(99)

    def loss(u0, v0, coeffs):
        return oracle.gray_scott_final_and_loss(u0, v0, coeffs, DT, d["n"], d["ut"], d["vt"])[2]

    for i in range(4):
        eps = 1e-6 * max(1.0, abs(COEFFS[i]))
        tp = list(COEFFS); tp[i] += eps
        tm = list(COEFFS); tm[i] -= eps
        fd = (loss(d["u0"], d["v0"], tuple(tp)) - loss(d["u0"], d["v0"], tuple(tm))) / (2 * eps)
        assert abs(d["gth"][i] - fd) <= 1e-6 * max(1e-3, abs(fd)), (i, d["gth"][i], fd)
    for _ in range(16):
        du, dv = rng.standard_normal(d["u0"].shape), rng.standard_normal(d["u0"].shape)
        eps = 1e-6
        fp = loss(d["u0"] + eps * du, d["v0"] + eps * dv, COEFFS)
        fm = loss(d["u0"] - eps * du, d["v0"] - eps * dv, COEFFS)
        fd = (fp - fm) / (2 * eps)
        ad = (d["gu0"] * du).sum() + (d["gv0"] * dv).sum()
        assert abs(ad - fd) <= 1e-6 * max(1e-3, abs(fd)), (ad, fd)


# ------------------------------------------------------------ Models A and B (c1, c2, M)

PF_CASES = [("ac", (0.9, 1.2), 0.02), ("ch", (0.8, 1.1, 0.7), 0.004)]


@pytest.mark.parametrize("model,coeffs,dt", PF_CASES)
def test_phase_field_adjoint_step_is_jacobian_transpose(model, coeffs, dt):
    rng = np.random.default_rng(5)
    shape = (5, 6)
    phi = rng.uniform(-0.9, 0.9, shape)
    lam = rng.standard_normal(shape)
    n = phi.size
    J = np.zeros((n, n))
    eps = 1e-30
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        out, = oracle.euler_step(model, (phi + 1j * eps * e.reshape(shape),), coeffs, dt)
        J[:, j] = (np.imag(out) / eps).ravel()
    if model == "ac":
        got, _ = oracle.allen_cahn_adjoint_step(phi, lam, *coeffs, dt)
    else:
        got, _ = oracle.cahn_hilliard_adjoint_step(phi, lam, *coeffs, dt)
    np.testing.assert_allclose(got.ravel(), J.T @ lam.ravel(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("model,coeffs,dt", PF_CASES)
def test_phase_field_adjoint_step_parameter_gradient(model, coeffs, dt):
    rng = np.random.default_rng(6)
    shape = (7, 6)
    phi = rng.uniform(-0.9, 0.9, shape)
    lam = rng.standard_normal(shape)
    if model == "ac":
        _, g = oracle.allen_cahn_adjoint_step(phi, lam, *coeffs, dt)
    else:
        _, g = oracle.cahn_hilliard_adjoint_step(phi, lam, *coeffs, dt)
    eps = 1e-30
    for i in range(len(coeffs)):
        th = np.array(coeffs, dtype=np.complex128)
        th[i] += 1j * eps
        out, = oracle.euler_step(model, (phi,), tuple(th), dt)
        d = np.imag((lam * out).sum()) / eps
        assert abs(g[i] - d) <= 1e-12 * max(1.0, abs(d))


@pytest.mark.parametrize("model,coeffs,dt", PF_CASES)
def test_phase_field_adjoint_vs_complex_step_of_the_loop(model, coeffs, dt):
    # the whole time loop: dL/dtheta and a direction of dL/dphi0 by complex step
    phi0 = synthetic.allen_cahn_init((24, 20), seed=3, lo=-0.6, hi=0.6).astype(np.float64)
    target = oracle.run(model, (phi0 * 0.9,), coeffs, dt, 150)[0]
    n = 150
    phiN = oracle.run(model, (phi0,), coeffs, dt, n)[0]
    g0, gth = oracle.phase_field_adjoint(model, phi0, coeffs, dt, n, phiN - target)
    eps = 1e-30

    def loss(p0, th):
        p = oracle.run(model, (p0,), th, dt, n)[0]
        return 0.5 * ((p - target) ** 2).sum()

    for i in range(len(coeffs)):
        th = np.array(coeffs, dtype=np.complex128)
        th[i] += 1j * eps
        d = np.imag(loss(phi0.astype(np.complex128), tuple(th))) / eps
        assert abs(gth[i] - d) <= 1e-9 * max(1e-6, abs(d)), (i, gth[i], d)
    dirn = np.random.default_rng(7).standard_normal(phi0.shape)
    d = np.imag(loss(phi0 + 1j * eps * dirn, coeffs)) / eps
    assert abs((g0 * dirn).sum() - d) <= 1e-9 * max(1.0, abs(d))
