"""GPU adjoint of the forward-Euler Gray-Scott loop (through the C ABI) against the FP64
oracle adjoint (itself pinned by complex-step and central differences), the checkpoint
schedule invariance, the autograd Function, and central differences at full size.

Bars: relative L2 of dL/d(u0, v0) <= 1e-3 and relative error of dL/dtheta <= 1e-3."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

COEFFS = (0.2, 0.1, 0.04, 0.06)  # Du, Dv, F, k
DT = 0.5


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02598_gb300.build import build
    build()
    import paper_2109_02598_gb300 as pf
    return pf


def target(u0, v0, n):
    Du, Dv, F, k = COEFFS
    return oracle.run("gs", (u0, v0), (Du, Dv, F + 0.002, k - 0.001), DT, n)


def gpu_adjoint(pf, u0, v0, n, ckpt, ut, vt, coeffs=COEFFS):
    """GPU forward (checkpointed) + backward with dL/dx_N = x_N - x* (host arrays)."""
    g = pf.Grid(u0.shape, 2).set_model("gs", coeffs, DT)
    g.write_fields((u0, v0))
    from paper_2109_02598_gb300 import _lib
    import ctypes
    _lib.check(g._lib.pf_adj_forward(g.handle, n, ckpt))
    uN, vN = g.read_fields()
    du = (uN.astype(np.float64) - ut).astype(np.float32)
    dv = (vN.astype(np.float64) - vt).astype(np.float32)
    gu0 = np.empty_like(du)
    gv0 = np.empty_like(dv)
    dth = (ctypes.c_double * 4)()
    _lib.check(g._lib.pf_adj_backward(g.handle, du.ctypes.data_as(ctypes.c_void_p),
                                      dv.ctypes.data_as(ctypes.c_void_p), 0,
                                      gu0.ctypes.data_as(ctypes.c_void_p),
                                      gv0.ctypes.data_as(ctypes.c_void_p), dth))
    # the grid still holds x_N: the backward pass does not change the state
    uN2, vN2 = g.read_fields()
    assert np.array_equal(uN, uN2) and np.array_equal(vN, vN2)
    g.close()
    return (uN, vN), (gu0, gv0), np.array(list(dth))


def rel_l2(got, ref):
    num = np.sqrt(sum(((g.astype(np.float64) - r) ** 2).sum() for g, r in zip(got, ref)))
    return num / np.sqrt(sum((r ** 2).sum() for r in ref))


def check_against_oracle(pf, shape, n, ckpt, seed):
    u0, v0 = synthetic.gray_scott_init(shape, seed=seed, n_seeds=max(1, shape[0] * shape[1] // 400),
                                       side=4, noise=0.05)
    ut, vt = target(u0, v0, n)
    (uN, vN), gx0, gth = gpu_adjoint(pf, u0, v0, n, ckpt, ut, vt)
    ouN, ovN = oracle.run("gs", (u0, v0), COEFFS, DT, n)
    ru, rv, rth = oracle.gray_scott_adjoint(u0, v0, COEFFS, DT, n, ouN - ut, ovN - vt)
    assert rel_l2(gx0, (ru, rv)) <= 1e-3
    assert np.all(np.abs(gth - rth) <= 1e-3 * np.abs(rth) + 1e-9 * np.abs(rth).max())
    return gth


@pytest.mark.parametrize("shape,n,ckpt", [((40, 56), 60, 7), ((33, 70), 25, 0), ((9, 5), 12, 12)])
def test_adjoint_matches_oracle_small(pf, shape, n, ckpt):
    check_against_oracle(pf, shape, n, ckpt, seed=61)


def test_adjoint_32x32_copy_2000_steps(pf):
    # the 32x32 copy of the 512^2 adjoint workload, 2000 steps, sqrt(N) checkpoints
    u0, v0 = synthetic.workload_init("gs2d_adjoint_512", shape=(32, 32))
    n = 2000
    ut, vt = target(u0, v0, n)
    _, gx0, gth = gpu_adjoint(pf, u0, v0, n, 0, ut, vt)
    ouN, ovN = oracle.run("gs", (u0, v0), COEFFS, DT, n)
    ru, rv, rth = oracle.gray_scott_adjoint(u0, v0, COEFFS, DT, n, ouN - ut, ovN - vt)
    assert rel_l2(gx0, (ru, rv)) <= 1e-3
    assert np.all(np.abs(gth - rth) <= 1e-3 * np.abs(rth))


def test_adjoint_512_short_run_matches_oracle(pf):
    u0, v0 = synthetic.workload_init("gs2d_adjoint_512")
    n = 60
    ut, vt = target(u0, v0, n)
    _, gx0, gth = gpu_adjoint(pf, u0, v0, n, 0, ut, vt)
    ouN, ovN = oracle.run("gs", (u0, v0), COEFFS, DT, n)
    ru, rv, rth = oracle.gray_scott_adjoint(u0, v0, COEFFS, DT, n, ouN - ut, ovN - vt)
    assert rel_l2(gx0, (ru, rv)) <= 1e-3
    assert np.all(np.abs(gth - rth) <= 1e-3 * np.abs(rth))


def test_checkpoint_schedule_does_not_change_gradients(pf):
    u0, v0 = synthetic.gray_scott_init((48, 40), seed=71, n_seeds=4, side=4, noise=0.05)
    n = 50
    ut, vt = target(u0, v0, n)
    _, base_x, base_th = gpu_adjoint(pf, u0, v0, n, 1, ut, vt)
    for ckpt in (0, 7, 50):
        _, gx, gth = gpu_adjoint(pf, u0, v0, n, ckpt, ut, vt)
        assert np.array_equal(gx[0], base_x[0]) and np.array_equal(gx[1], base_x[1])
        assert np.array_equal(gth, base_th)


def test_autograd_function(pf):
    import torch
    u0, v0 = synthetic.gray_scott_init((36, 44), seed=81, n_seeds=3, side=4, noise=0.05)
    n = 40
    ut, vt = target(u0, v0, n)
    U0 = torch.tensor(u0, device="cuda", requires_grad=True)
    V0 = torch.tensor(v0, device="cuda", requires_grad=True)
    th = torch.tensor(COEFFS, dtype=torch.float64, device="cuda", requires_grad=True)
    uN, vN = pf.GrayScottAdjoint.apply(U0, V0, th, n, DT)
    Ut = torch.tensor(ut, device="cuda", dtype=torch.float32)
    Vt = torch.tensor(vt, device="cuda", dtype=torch.float32)
    loss = 0.5 * ((uN - Ut) ** 2).sum() + 0.5 * ((vN - Vt) ** 2).sum()
    loss.backward()
    ouN, ovN = oracle.run("gs", (u0, v0), COEFFS, DT, n)
    ru, rv, rth = oracle.gray_scott_adjoint(u0, v0, COEFFS, DT, n, ouN - ut, ovN - vt)
    assert rel_l2((U0.grad.cpu().numpy(), V0.grad.cpu().numpy()), (ru, rv)) <= 1e-3
    assert np.all(np.abs(th.grad.cpu().numpy() - rth) <= 1e-3 * np.abs(rth))


def test_full_size_theta_gradient_vs_central_differences(pf):
    # 512^2, 2000 steps, sqrt(N) checkpoints: dL/dF and dL/dk against FP64 central
    # differences of the oracle's loss (eps = 1e-6).
    u0, v0 = synthetic.workload_init("gs2d_adjoint_512")
    n = 2000
    ut, vt = target(u0, v0, n)
    _, _, gth = gpu_adjoint(pf, u0, v0, n, 0, ut, vt)
    for i in (2, 3):
        eps = 1e-6
        cp = list(COEFFS); cp[i] += eps
        cm = list(COEFFS); cm[i] -= eps
        lp = oracle.gray_scott_final_and_loss(u0, v0, tuple(cp), DT, n, ut, vt)[2]
        lm = oracle.gray_scott_final_and_loss(u0, v0, tuple(cm), DT, n, ut, vt)[2]
        fd = (lp - lm) / (2 * eps)
        assert abs(gth[i] - fd) <= 1e-3 * abs(fd), (i, gth[i], fd)
