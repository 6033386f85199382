"""N coupled species of reaction-diffusion type on the GPU (PF_MODEL_RD, up to 4 fields):
du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j^E[m][j], through the C ABI, against the FP64
oracle. Bars as for the other models: one step rel L-inf <= 1e-6, 1000 steps rel L2 <= 1e-3."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02598_gb300.build import build
    build()
    import paper_2109_02598_gb300 as pf
    return pf


# three species: a constant source, cubic, quadratic and mixed monomials
SYS3 = dict(D=(0.2, 0.05, 0.12),
            E=[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 2, 0], [2, 0, 1], [0, 0, 3]],
            K=[[0.03, -0.03, 0.0, 0.1, -1.0, 0.0, 0.0],
               [0.0, 0.0, -0.09, 0.0, 1.0, -0.4, 0.0],
               [0.0, 0.05, 0.0, -0.2, 0.0, 0.4, -0.3]])
# four species: A + B <-> C (rates 1.2 and 0.5), C -> D (0.2), D -> A (0.3), A decays (0.05)
# and B is fed (0.05); monomials AB, C, D, A, 1
SYS4 = dict(D=(0.1, 0.15, 0.05, 0.02),
            E=[[1, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 0, 0, 0]],
            K=[[-1.2, 0.5, 0.3, -0.05, 0.0], [-1.2, 0.5, 0.0, 0.0, 0.05],
               [1.2, -0.7, 0.0, 0.0, 0.0], [0.0, 0.2, -0.3, 0.0, 0.0]])


def coeffs(sys):
    return oracle.rd_pack(sys["D"], sys["E"], sys["K"])


def init(shape, n, seed):
    return tuple(synthetic.uniform(seed, 60 + i, int(np.prod(shape)), 0.05, 0.9)
                 .reshape(shape).astype(np.float32) for i in range(n))


def run(pf, x0, c, dt, n, h=1.0):
    g = pf.Grid(x0[0].shape, len(x0), h).set_model("rd", c, dt)
    g.write_fields(x0)
    g.step(n)
    out = g.read_fields()
    g.close()
    return out


def rel_linf(got, ref):
    return max(np.abs(a.astype(np.float64) - b).max() for a, b in zip(got, ref)) / \
        max(np.abs(b).max() for b in ref)


def rel_l2(got, ref):
    num = np.sqrt(sum(((a.astype(np.float64) - b) ** 2).sum() for a, b in zip(got, ref)))
    return num / np.sqrt(sum((b ** 2).sum() for b in ref))


@pytest.mark.parametrize("sys,nf", [(SYS3, 3), (SYS4, 4)])
@pytest.mark.parametrize("shape", [(37, 150), (64, 64), (5, 7), (1, 9), (9, 20, 70), (4, 4, 4),
                                   (3, 17, 33)])
def test_single_step_and_twenty_steps(pf, sys, nf, shape):
    c = coeffs(sys)
    x0 = init(shape, nf, seed=len(shape) * 10 + nf)
    one = run(pf, x0, c, 0.5, 1)
    assert rel_linf(one, oracle.euler_step("rd", x0, c, 0.5)) <= 1e-6
    twenty = run(pf, x0, c, 0.5, 20)
    assert rel_linf(twenty, oracle.run("rd", x0, c, 0.5, 20)) <= 1e-5


@pytest.mark.parametrize("shape,h", [((96, 80), 1.0), ((16, 20, 24), 0.8)])
def test_thousand_steps(pf, shape, h):
    c = coeffs(SYS4)
    x0 = init(shape, 4, seed=7)
    ref = oracle.run("rd", x0, c, 0.1, 1000, h)
    got = run(pf, x0, c, 0.1, 1000, h)
    assert rel_l2(got, ref) <= 1e-3


def test_mass_action_invariants(pf):
    # A + B -> C with a spectator S: sum(A + C), sum(B + C), sum(S) are conserved
    c = oracle.rd_pack((0.2, 0.15, 0.05, 0.1), [[1, 1, 0, 0]], [[-1.3], [-1.3], [1.3], [0.0]])
    x0 = init((64, 48), 4, seed=9)
    x = run(pf, x0, c, 0.2, 300)
    x0d = [a.astype(np.float64) for a in x0]
    xd = [a.astype(np.float64) for a in x]
    for a, b in (((xd[0] + xd[2]).sum(), (x0d[0] + x0d[2]).sum()),
                 ((xd[1] + xd[2]).sum(), (x0d[1] + x0d[2]).sum()), (xd[3].sum(), x0d[3].sum())):
        assert abs(a - b) <= 1e-5 * abs(b)
    assert xd[2].sum() > x0d[2].sum()


def test_gray_scott_as_two_species(pf):
    # the same equations as PF_MODEL_GS, written as monomials; a different operation order,
    # so within the float32 tolerance rather than bitwise
    Du, Dv, F, k = 0.2, 0.1, 0.04, 0.06
    c = oracle.rd_pack((Du, Dv), [[0, 0], [1, 0], [0, 1], [1, 2]],
                       [[F, -F, 0.0, -1.0], [0.0, 0.0, -(F + k), 1.0]])
    x0 = synthetic.gray_scott_init((64, 96), seed=11, n_seeds=6, side=4, noise=0.05)
    a = run(pf, x0, c, 0.5, 200)
    g = pf.Grid(x0[0].shape, 2).set_model("gs", (Du, Dv, F, k), 0.5).write_fields(x0)
    g.step(200)
    b = g.read_fields()
    g.close()
    assert rel_l2(a, b) <= 1e-5
    assert rel_l2(a, oracle.run("gs", x0, (Du, Dv, F, k), 0.5, 200)) <= 1e-4


def test_rules(pf):
    from paper_2109_02598_gb300 import PfError, rd_coeffs
    g = pf.Grid((16, 16), 3)
    with pytest.raises(PfError, match="exponents"):
        g.set_model("rd", (0.1, 0.1, 0.1, 1.0, 4.0, 0.0, 0.0, 1.0, 1.0, 1.0), 0.1)
    with pytest.raises(PfError, match="takes"):
        g.set_model("rd", (0.1, 0.1, 0.1, 1.0, 1.0, 0.0, 0.0), 0.1)
    with pytest.raises(PfError, match="D_1"):
        g.set_model("rd", rd_coeffs((0.1, -0.1, 0.1), [[1, 0, 0]], [[1.0], [0.0], [0.0]]), 0.1)
    with pytest.raises(PfError, match="stability"):
        g.set_model("rd", rd_coeffs((1.0, 0.1, 0.1), [], [[], [], []]), 1.0)
    g.set_model("rd", rd_coeffs((0.1, 0.1, 0.1), [[1, 1, 0]], [[-1.0], [-1.0], [1.0]]), 0.1)
    with pytest.raises(PfError, match="one step per launch"):
        g.set_tuning(64, 16, 2)
    with pytest.raises(PfError, match="stencil"):
        g.set_stencil("iso")
    with pytest.raises(PfError):
        g.set_model("gs", (0.2, 0.1, 0.04, 0.06), 0.5)  # Gray-Scott needs 2 fields
    with pytest.raises(PfError):
        g.energy()
    assert g.mass(2) == 0.0
    g.close()
    with pytest.raises(PfError, match="n_fields"):
        pf.Grid((8, 8), 5)
