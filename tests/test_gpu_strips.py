"""The 2D strip kernel (tile 128 or 64 x PF_TILE_STRIPS): one warp per strip of columns, the
k steps pipelined in registers. It must give the tiled kernels' bits for every model, width,
depth and grid shape, with the 5-point stencil and (Models A and Gray-Scott) the isotropic
9-point one (ragged widths, grids narrower than a strip, fewer rows than a task, a
single row or column), and meet the oracle bars: one step rel L-inf <= 1e-6, 1000 steps rel
L2 <= 1e-3."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

COEFFS = {"ac": (1.0, 1.0), "gs": (0.2, 0.1, 0.04, 0.06), "ch": (1.0, 1.0, 1.0),
          "c": (1.0, 1.0, 1.0, 1.0, 1.0)}
DT = {"ac": 0.05, "gs": 0.5, "ch": 0.01, "c": 0.005}
KS = {"ac": (1, 2, 4), "gs": (1, 2, 4), "ch": (1, 2), "c": (1, 2)}


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
    if model == "ac":
        return (synthetic.allen_cahn_init(shape, seed=500 + seed, lo=-0.5, hi=0.5),)
    if model == "ch":
        return (synthetic.cahn_hilliard_init(shape, seed=700 + seed, amp=0.3),)
    if model == "c":
        return (synthetic.allen_cahn_init(shape, seed=800 + seed, lo=-0.5, hi=0.5),
                synthetic.cahn_hilliard_init(shape, seed=850 + seed, amp=0.4))
    n_seeds = max(2, int(np.prod(shape)) // 2000)
    return synthetic.gray_scott_init(shape, seed=600 + seed, n_seeds=n_seeds, side=4,
                                     noise=0.05)


def run(pf, model, x0, n, tuning, h=1.0):
    g = pf.Grid(x0[0].shape, len(x0), h).set_model(model, COEFFS[model], DT[model])
    g.set_tuning(*tuning)
    assert g.tuning == tuning
    g.write_fields(x0)
    g.step(n)
    out = g.read_fields()
    g.close()
    return out


SHAPES = [(200, 300), (37, 131), (64, 64), (5, 7), (1, 9), (9, 1), (130, 120), (97, 250),
          (300, 61)]


@pytest.mark.parametrize("model", ["ac", "gs", "ch", "c"])
@pytest.mark.parametrize("shape", SHAPES)
def test_strips_are_bitwise_the_tiled_kernel(pf, model, shape):
    x0 = fields_for(model, shape)
    for k in KS[model]:
        ref = run(pf, model, x0, 12, (64, 16, k))
        for width in (128, 64):
            got = run(pf, model, x0, 12, (width, pf.PF_TILE_STRIPS, k))
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), (model, shape, k, width)


@pytest.mark.parametrize("model", ["ac", "gs", "ch", "c"])
def test_strips_single_step_and_1000_steps_vs_oracle(pf, model):
    shape = (96, 260)
    x0 = fields_for(model, shape, seed=3)
    one = run(pf, model, x0, 1, (128, pf.PF_TILE_STRIPS, 1))
    ref1 = oracle.euler_step(model, x0, COEFFS[model], DT[model])
    assert max(np.abs(a.astype(np.float64) - b).max() / np.abs(b).max()
               for a, b in zip(one, ref1)) <= 1e-6
    got = run(pf, model, x0, 1000, (128, pf.PF_TILE_STRIPS, KS[model][-1]))
    ref = oracle.run(model, x0, COEFFS[model], DT[model], 1000)
    num = np.sqrt(sum(((a.astype(np.float64) - b) ** 2).sum() for a, b in zip(got, ref)))
    assert num / np.sqrt(sum((b ** 2).sum() for b in ref)) <= 1e-3


@pytest.mark.parametrize("model,shape,k", [("gs", (4096, 4096), 4), ("ch", (8192, 8192), 2),
                                           ("ac", (4096, 4096), 4)])
def test_strips_full_size_bitwise_tiled(pf, model, shape, k):
    # the plain 2D grids the bench quotes, 8 steps at the strip kernel's depth, both strip
    # widths (the autotuner takes 64 columns for Gray-Scott 4096^2, 128 for the others):
    # every site
    x0 = fields_for(model, shape, seed=5)
    ref = run(pf, model, x0, 8, (128, 32, k))
    for width in (128, 64):
        got = run(pf, model, x0, 8, (width, pf.PF_TILE_STRIPS, k))
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), width


def test_strips_spacing_and_rules(pf):
    x0 = fields_for("ac", (80, 90))
    a = run(pf, "ac", x0, 7, (128, pf.PF_TILE_STRIPS, 2), h=0.7)
    b = run(pf, "ac", x0, 7, (128, 16, 2), h=0.7)
    assert np.array_equal(a[0], b[0])
    g = pf.Grid((64, 64), 1).set_model("ch", (1.0, 1.0, 1.0), 0.01)
    with pytest.raises(pf.PfError, match="strip kernel"):
        g.set_tuning(128, pf.PF_TILE_STRIPS, 4)  # Model B: k = 1 or 2
    g.close()
    g = pf.Grid((64, 64), 2).set_model("rd", pf.rd_coeffs((0.1, 0.1), [[1, 1]], [[-1.0], [1.0]]),
                                       0.1)
    g.set_tuning(128, pf.PF_TILE_STRIPS, 1)  # the N-species model keeps its own kernel
    assert g.tuning == (64, 16, 1)
    g.close()
    g = pf.Grid((64, 64), 1).set_model("ac", (1.0, 1.0), 0.05)
    with pytest.raises(pf.PfError, match="strip kernel"):
        g.set_tuning(96, pf.PF_TILE_STRIPS, 1)  # widths 128 and 64 only
    with pytest.raises(pf.PfError, match="strip kernel"):
        g.set_tuning(128, pf.PF_TILE_STRIPS, 8)
    g.set_stencil("4th")  # radius 2: the three-row windows do not hold it
    with pytest.raises(pf.PfError, match="strip kernel"):
        g.set_tuning(128, pf.PF_TILE_STRIPS, 1)
    g.set_stencil("iso")
    g.set_tuning(128, pf.PF_TILE_STRIPS, 4)
    assert g.tuning == (128, pf.PF_TILE_STRIPS, 4)
    g.set_stencil("4th")  # the strip tuning no longer applies: back to the default tile
    assert g.tuning[1] != pf.PF_TILE_STRIPS
    g.close()
    g = pf.Grid((64, 64), 1).set_model("ch", (1.0, 1.0, 1.0), 0.01).set_stencil("iso")
    with pytest.raises(pf.PfError, match="strip kernel"):
        g.set_tuning(128, pf.PF_TILE_STRIPS, 1)  # Model B: the 5-point stencil only
    g.close()


# ---------------------------------------------------------------- isotropic 9-point stencil

def run_iso(pf, model, x0, n, tuning, dt, h=0.9):
    g = pf.Grid(x0[0].shape, len(x0), h).set_stencil("iso")
    g.set_model(model, COEFFS[model], dt)
    g.set_tuning(*tuning)
    assert g.tuning == tuning
    g.write_fields(x0)
    g.step(n)
    out = g.read_fields()
    g.close()
    return out


@pytest.mark.parametrize("model", ["ac", "gs"])
@pytest.mark.parametrize("shape", SHAPES)
def test_iso_strips_are_bitwise_the_tiled_kernel(pf, model, shape):
    # the tiled kernels take the 9-point stencil at k = 1 and 2; the strips at k = 1, 2, 4
    # give their bits at the same step count
    x0 = fields_for(model, shape, seed=7)
    dt = DT[model] * 0.5
    ref = run_iso(pf, model, x0, 12, (64, 16, 1), dt)
    for k in (1, 2, 4):
        for width in (128, 64):
            got = run_iso(pf, model, x0, 12, (width, pf.PF_TILE_STRIPS, k), dt)
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), (model, shape, k, width)


@pytest.mark.parametrize("model", ["ac", "gs"])
def test_iso_strips_vs_oracle(pf, model):
    shape = (96, 260)
    x0 = fields_for(model, shape, seed=8)
    dt, h = DT[model] * 0.5, 0.9
    one = run_iso(pf, model, x0, 1, (64, pf.PF_TILE_STRIPS, 1), dt, h)
    ref1 = oracle.euler_step(model, x0, COEFFS[model], dt, h, stencil="9iso")
    assert max(np.abs(a.astype(np.float64) - b).max() / np.abs(b).max()
               for a, b in zip(one, ref1)) <= 1e-6
    got = run_iso(pf, model, x0, 1000, (64, pf.PF_TILE_STRIPS, 4), dt, h)
    ref = oracle.run(model, x0, COEFFS[model], dt, 1000, h, stencil="9iso")
    num = np.sqrt(sum(((a.astype(np.float64) - b) ** 2).sum() for a, b in zip(got, ref)))
    assert num / np.sqrt(sum((b ** 2).sum() for b in ref)) <= 1e-3


def test_iso_strips_full_size_bitwise_tiled(pf):
    # Gray-Scott 4096^2 with the 9-point stencil, 8 steps: every site, both widths, k = 4
    x0 = fields_for("gs", (4096, 4096), seed=9)
    ref = run_iso(pf, "gs", x0, 8, (128, 32, 2), DT["gs"], 1.0)
    for width in (128, 64):
        got = run_iso(pf, "gs", x0, 8, (width, pf.PF_TILE_STRIPS, 4), DT["gs"], 1.0)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), width
