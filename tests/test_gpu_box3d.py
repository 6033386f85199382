"""The 3D box kernel for the radius-2 models (3D tile 32x8: Models B and C, whole 32 x 8 x 8
boxes per CTA, k = 1 or 2 steps per launch): the bits of the general z-streaming kernel on
every shape (boxes past the grid's edges, grids smaller than a box, the paper's 64^3) and at
both depths, the oracle's single-step bar (rel L-inf <= 1e-6) and 1000-step bar (rel L2 <=
1e-3), and its rules."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

COEFFS = {"ch": (1.0, 1.0, 1.0), "c": (1.0, 1.0, 1.0, 1.0, 1.0)}
DT = {"ch": 0.01, "c": 0.005}


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02598_gb300.build import build
    build()
    import paper_2109_02598_gb300 as pf
    return pf


def fields_for(model, shape, seed=0):
    if model == "ch":
        return (synthetic.cahn_hilliard_init(shape, seed=900 + seed, amp=0.3),)
    return (synthetic.allen_cahn_init(shape, seed=910 + seed, lo=-0.5, hi=0.5),
            synthetic.cahn_hilliard_init(shape, seed=920 + seed, amp=0.4))


def run(pf, model, x0, n, tuning, h=1.0):
    g = pf.Grid(x0[0].shape, len(x0), h).set_model(model, COEFFS[model], DT[model])
    g.set_tuning(*tuning)
    assert g.tuning == tuning
    g.write_fields(x0).step(n)
    out = g.read_fields()
    g.close()
    return out


@pytest.mark.parametrize("model", ["ch", "c"])
@pytest.mark.parametrize("shape", [(64, 64, 64), (20, 12, 44), (9, 10, 8), (5, 3, 4),
                                   (17, 40, 96), (8, 8, 32)])
def test_box_kernel_is_bitwise_the_general_kernel(pf, model, shape):
    x0 = fields_for(model, shape)
    ref = run(pf, model, x0, 7, (32, 16, 1))
    for k in (1, 2):
        got = run(pf, model, x0, 7, (32, 8, k))
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), (model, shape, k)


@pytest.mark.parametrize("model", ["ch", "c"])
def test_box_kernel_against_the_oracle(pf, model):
    shape = (24, 20, 36)
    x0 = fields_for(model, shape, seed=1)
    h = 0.9 if model == "c" else 1.0  # Model B's stability limit scales with h^4
    one = run(pf, model, x0, 1, (32, 8, 1), h=h)
    ref1 = oracle.euler_step(model, x0, COEFFS[model], DT[model], h)
    assert max(np.abs(a.astype(np.float64) - b).max() / np.abs(b).max()
               for a, b in zip(one, ref1)) <= 1e-6
    got = run(pf, model, x0, 1000, (32, 8, 2))
    ref = oracle.run(model, x0, COEFFS[model], DT[model], 1000)
    num = np.sqrt(sum(((a.astype(np.float64) - b) ** 2).sum() for a, b in zip(got, ref)))
    assert num / np.sqrt(sum((b ** 2).sum() for b in ref)) <= 1e-3


def test_box_kernel_rules(pf):
    g = pf.Grid((8, 8, 8), 1).set_model("ac", (1.0, 1.0), 0.05)
    with pytest.raises(pf.PfError, match="box kernel"):
        g.set_tuning(32, 8, 1)  # Models B and C only
    g.close()
    g = pf.Grid((8, 8, 10), 1).set_model("ch", (1.0, 1.0, 1.0), 0.01)
    with pytest.raises(pf.PfError, match="box kernel"):
        g.set_tuning(32, 8, 1)  # nx % 4 != 0
    g.close()
    g = pf.Grid((8, 8, 8), 1).set_model("ch", (1.0, 1.0, 1.0), 0.01)
    with pytest.raises(pf.PfError):
        g.set_tuning(32, 8, 3)
    g.set_tuning(32, 8, 2)
    assert g.tuning == (32, 8, 2)
    g.close()
