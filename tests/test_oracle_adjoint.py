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
