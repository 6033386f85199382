"""GPU adjoint of the forward-Euler Gray-Scott loop (through the C ABI) against the FP64
oracle adjoint (itself pinned by complex-step and central differences), the checkpoint
schedule invariance, the autograd Function, and central differences at full size.

Bars: relative L2 of dL/d(u0, v0) <= 1e-3 and relative error of dL/dtheta <= 1e-3."""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

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


def _loss(u0, v0, coeffs, n, ut, vt):
    return oracle.gray_scott_final_and_loss(u0, v0, coeffs, DT, n, ut, vt)[2]


def test_full_size_gradients_vs_central_differences(pf):
    # 512^2, 2000 steps, sqrt(N) checkpoints: every parameter gradient (D_u, D_v, F, k) and
    # the initial-state gradient along one seeded random direction in (u0, v0), against FP64
    # central differences of the oracle's loss (eps = 1e-6). The twelve oracle runs go to
    # worker processes (spawned: this process already holds a CUDA context).
    u0, v0 = synthetic.workload_init("gs2d_adjoint_512")
    n = 2000
    eps = 1e-6
    rng = np.random.default_rng(2000)
    du, dv = rng.standard_normal(u0.shape), rng.standard_normal(v0.shape)
    u64, v64 = u0.astype(np.float64), v0.astype(np.float64)
    with ProcessPoolExecutor(min(12, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        ut, vt = target(u0, v0, n)
        jobs = {}
        for i in range(4):
            cp = list(COEFFS); cp[i] += eps
            cm = list(COEFFS); cm[i] -= eps
            jobs[i] = (ex.submit(_loss, u0, v0, tuple(cp), n, ut, vt),
                       ex.submit(_loss, u0, v0, tuple(cm), n, ut, vt))
        jobs["x0"] = (ex.submit(_loss, u64 + eps * du, v64 + eps * dv, COEFFS, n, ut, vt),
                      ex.submit(_loss, u64 - eps * du, v64 - eps * dv, COEFFS, n, ut, vt))
        _, (gu0, gv0), gth = gpu_adjoint(pf, u0, v0, n, 0, ut, vt)
        for key, (plus, minus) in jobs.items():
            fd = (plus.result() - minus.result()) / (2 * eps)
            if key == "x0":
                ad = float((gu0.astype(np.float64) * du).sum() + (gv0.astype(np.float64) * dv).sum())
            else:
                ad = gth[key]
            assert abs(ad - fd) <= 1e-3 * abs(fd), (key, ad, fd)


# --------------------------------------------- Models A and B: dL/d(c1, c2) and mobility M

PF = {"ac": ((0.9, 1.1), 0.02), "ch": ((0.8, 1.1, 0.7), 0.004)}


def pf_gpu_adjoint(pf, model, phi0, n, ckpt, target):
    import ctypes
    from paper_2109_02598_gb300 import _lib
    coeffs, dt = PF[model]
    g = pf.Grid(phi0.shape, 1).set_model(model, coeffs, dt)
    g.write_field(0, phi0)
    _lib.check(g._lib.pf_adj_forward(g.handle, n, ckpt))
    phiN = g.read_field(0)
    d = (phiN.astype(np.float64) - target).astype(np.float32)
    g0 = np.empty_like(d)
    dth = (ctypes.c_double * 4)()
    _lib.check(g._lib.pf_adj_backward(g.handle, d.ctypes.data_as(ctypes.c_void_p), None, 0,
                                      g0.ctypes.data_as(ctypes.c_void_p), None, dth))
    g.close()
    return g0, np.array(list(dth)[:len(coeffs)])


@pytest.mark.parametrize("model", ["ac", "ch"])
@pytest.mark.parametrize("shape,n,ckpt", [((40, 48), 60, 7), ((33, 70), 25, 0)])
def test_phase_field_adjoint_matches_oracle(pf, model, shape, n, ckpt):
    coeffs, dt = PF[model]
    phi0 = synthetic.allen_cahn_init(shape, seed=91, lo=-0.6, hi=0.6)
    target = oracle.run(model, (phi0.astype(np.float64) * 0.9,), coeffs, dt, n)[0]
    g0, gth = pf_gpu_adjoint(pf, model, phi0, n, ckpt, target)
    phiN = oracle.run(model, (phi0,), coeffs, dt, n)[0]
    r0, rth = oracle.phase_field_adjoint(model, phi0, coeffs, dt, n, phiN - target)
    assert rel_l2((g0,), (r0,)) <= 1e-3
    assert np.all(np.abs(gth - rth) <= 1e-3 * np.abs(rth)), (gth, rth)


def test_mobility_gradient_autograd_vs_central_differences(pf):
    # Model B 128^2, 400 steps: torch loss through PhaseFieldAdjoint; dL/dM and dL/dc1
    # against FP64 central differences of the oracle's loss
    import torch
    coeffs, dt = PF["ch"]
    n = 400
    phi0 = synthetic.cahn_hilliard_init((128, 128), seed=93, amp=0.3)
    target = oracle.run("ch", (phi0.astype(np.float64) * 0.8,), coeffs, dt, n)[0]
    P0 = torch.tensor(phi0, device="cuda", requires_grad=True)
    th = torch.tensor(coeffs, dtype=torch.float64, device="cuda", requires_grad=True)
    out = pf.PhaseFieldAdjoint.apply(P0, th, "ch", n, dt)
    T = torch.tensor(target, device="cuda", dtype=torch.float32)
    loss = 0.5 * ((out - T) ** 2).sum()
    loss.backward()
    gth = th.grad.cpu().numpy()

    def L(c):
        p = oracle.run("ch", (phi0,), c, dt, n)[0]
        return 0.5 * ((p - target) ** 2).sum()

    for i in (0, 2):
        eps = 1e-6
        cp = list(coeffs); cp[i] += eps
        cm = list(coeffs); cm[i] -= eps
        fd = (L(tuple(cp)) - L(tuple(cm))) / (2 * eps)
        assert abs(gth[i] - fd) <= 1e-3 * abs(fd), (i, gth[i], fd)
    # and the initial-field gradient in one direction
    d = np.random.default_rng(3).standard_normal(phi0.shape)
    eps = 1e-6
    p_plus = oracle.run("ch", (phi0 + eps * d,), coeffs, dt, n)[0]
    p_minus = oracle.run("ch", (phi0 - eps * d,), coeffs, dt, n)[0]
    fd = (0.5 * ((p_plus - target) ** 2).sum() - 0.5 * ((p_minus - target) ** 2).sum()) / (2 * eps)
    ad = float((P0.grad.cpu().numpy().astype(np.float64) * d).sum())
    assert abs(ad - fd) <= 1e-3 * abs(fd), (ad, fd)
