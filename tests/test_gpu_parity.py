"""Parity of the CUDA forward-Euler step (through the C ABI) with the FP64 oracle.

Bars (float32 kernels against the FP64 oracle from the same float32 initial array):
  one step            relative L-inf  <= 1e-6   (||x_gpu - x_ora||_inf / ||x_ora||_inf)
  1000 steps          relative L2     <= 1e-3
Every tile shape and temporal-blocking depth must give bitwise-identical results.
Shapes span several tiles with ragged tails, grids smaller than a tile, and the full
workload sizes (one step, every site)."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

COEFFS = {"ac": (1.0, 1.0), "ch": (1.0, 1.0, 1.0), "gs": (0.2, 0.1, 0.04, 0.06),
          "c": (1.0, 1.0, 1.0, 1.0, 1.0)}
DT = {"ac": 0.05, "ch": 0.01, "gs": 0.5, "c": 0.005}
MODELS = ["ac", "ch", "gs", "c"]


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02598_gb300.build import build
    build()
    import paper_2109_02598_gb300 as pf
    return pf


def init_fields(model, shape, seed=0):
    if model == "ac":
        return (synthetic.allen_cahn_init(shape, seed=100 + seed, lo=-0.5, hi=0.5),)
    if model == "ch":
        return (synthetic.cahn_hilliard_init(shape, seed=200 + seed, amp=0.3),)
    if model == "c":
        return (synthetic.allen_cahn_init(shape, seed=400 + seed, lo=-0.5, hi=0.5),
                synthetic.cahn_hilliard_init(shape, seed=450 + seed, amp=0.4))
    n_seeds = max(2, int(np.prod(shape)) // 2000)
    return synthetic.gray_scott_init(shape, seed=300 + seed, n_seeds=n_seeds, side=4,
                                     noise=0.05)


def gpu_run(pf, model, fields, n, coeffs=None, dt=None, h=1.0, tuning=None):
    coeffs = COEFFS[model] if coeffs is None else coeffs
    dt = DT[model] if dt is None else dt
    g = pf.Grid(fields[0].shape, n_fields=len(fields), h=h)
    g.set_model(model, coeffs, dt, force=True)
    if tuning is not None:
        g.set_tuning(*tuning)
    g.write_fields(fields)
    g.step(n)
    out = g.read_fields()
    g.close()
    return out


def rel_linf(got, ref):
    num = max(np.abs(g.astype(np.float64) - r).max() for g, r in zip(got, ref))
    den = max(np.abs(r).max() for r in ref)
    return num / den


def rel_l2(got, ref):
    num = np.sqrt(sum(((g.astype(np.float64) - r) ** 2).sum() for g, r in zip(got, ref)))
    den = np.sqrt(sum((r ** 2).sum() for r in ref))
    return num / den


SHAPES_2D = [(37, 150), (64, 64), (5, 7), (1, 9), (130, 33)]
# the last three take the TMA-staged kernel for AC/GS (nx % 64 == 0, ny % 16 == 0)
SHAPES_3D = [(9, 20, 70), (4, 4, 4), (3, 17, 33), (17, 5, 130), (5, 48, 192), (1, 16, 64),
             (2, 32, 128)]


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", SHAPES_2D + SHAPES_3D)
def test_single_step_parity(pf, model, shape):
    x0 = init_fields(model, shape)
    h = 0.9
    ref = oracle.euler_step(model, x0, COEFFS[model], DT[model] * 0.5, h)
    got = gpu_run(pf, model, x0, 1, dt=DT[model] * 0.5, h=h)
    assert rel_linf(got, ref) <= 1e-6


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", [(37, 150), (6, 11, 40)])
def test_twenty_steps_parity(pf, model, shape):
    x0 = init_fields(model, shape, seed=1)
    ref = oracle.run(model, x0, COEFFS[model], DT[model], 20)
    got = gpu_run(pf, model, x0, 20)
    assert rel_linf(got, ref) <= 2e-5


@pytest.mark.parametrize("model", MODELS)
def test_tiles_and_temporal_blocking_are_bitwise_identical(pf, model):
    x0 = init_fields(model, (70, 200), seed=2)
    base = gpu_run(pf, model, x0, 12, tuning=(64, 16, 1))
    ks = (1, 2) if model in ("ch", "c") else (1, 2, 4)
    for tile in [(64, 16), (128, 16), (32, 32), (128, 32)]:
        for k in ks:
            got = gpu_run(pf, model, x0, 12, tuning=(tile[0], tile[1], k))
            for a, b in zip(base, got):
                assert np.array_equal(a, b), (tile, k)
    # n not a multiple of k: remainder launches with smaller k
    got = gpu_run(pf, model, x0, 12, tuning=(128, 16, 2 if model in ("ch", "c") else 4))
    for a, b in zip(base, got):
        assert np.array_equal(a, b)
    # 3D tiles: general kernel on a ragged grid
    y0 = init_fields(model, (12, 19, 70), seed=3)
    b3 = gpu_run(pf, model, y0, 5, tuning=(32, 16, 1))
    g3 = gpu_run(pf, model, y0, 5, tuning=(64, 8, 1))
    for a, b in zip(b3, g3):
        assert np.array_equal(a, b)
    # 3D tiles on a grid the TMA kernel accepts: general and TMA kernels agree bitwise
    y1 = init_fields(model, (12, 32, 128), seed=4)
    b3 = gpu_run(pf, model, y1, 7, tuning=(32, 16, 1))
    tiles = [(64, 8)] + ([] if model in ("ch", "c") else [(64, 16), (128, 8), (128, 16)])
    for t in tiles:
        got = gpu_run(pf, model, y1, 7, tuning=(t[0], t[1], 1))
        for a, b in zip(b3, got):
            assert np.array_equal(a, b), t


@pytest.mark.parametrize("shape", [(40, 72), (6, 32, 64)])
def test_recorded_step_graphs_follow_model_and_tuning_changes(pf, shape):
    # pf_step replays recorded CUDA graphs for long launch sequences; changing the
    # coefficients or the tuning must not replay a stale graph
    (x0,) = init_fields("ac", shape, seed=9)
    g = pf.Grid(shape, 1).set_model("ac", (1.0, 1.0), 0.05)
    g.write_field(0, x0)
    g.step(30)
    g.step(30)  # replay from the other buffer
    g.set_model("ac", (0.5, 2.0), 0.02)
    g.step(30)
    g.set_tuning(32, 16, 1) if len(shape) == 3 else g.set_tuning(32, 32, 2)
    g.step(30)
    got = g.read_field(0)
    g.close()
    ref = oracle.run("ac", (x0,), (1.0, 1.0), 0.05, 60)
    ref = oracle.run("ac", ref, (0.5, 2.0), 0.02, 60)
    assert rel_linf((got,), ref) <= 5e-5


@pytest.mark.parametrize("model", ["ac", "gs"])
@pytest.mark.parametrize("shape,tile", [((12, 32, 128), (128, 8)), ((6, 16, 256), (256, 8)),
                                        ((9, 40, 128), (128, 8))])
def test_depth2_3d_kernel_is_bitwise_depth1(pf, model, shape, tile):
    # two time steps per pass (temporal blocking in 3D); odd step counts end with a
    # depth-1 launch; every result equals the depth-1 kernels' bit for bit
    x0 = init_fields(model, shape, seed=12)
    for n in (8, 7, 1):
        base = gpu_run(pf, model, x0, n, tuning=(32, 16, 1))
        got = gpu_run(pf, model, x0, n, tuning=(tile[0], tile[1], 2))
        for a, b in zip(base, got):
            assert np.array_equal(a, b), (n, tile)
    ref = oracle.run(model, x0, COEFFS[model], DT[model], 8)
    got = gpu_run(pf, model, x0, 8, tuning=(tile[0], tile[1], 2))
    assert rel_linf(got, ref) <= 1e-5


@pytest.mark.parametrize("model", ["ac", "gs"])
@pytest.mark.parametrize("shape,tile", [((160, 256, 256), 256), ((256, 256, 256), 256),
                                        ((8, 1280, 128), 128)])
def test_depth2_3d_work_splits_are_bitwise_depth1(pf, model, shape, tile):
    # The host splits the (row tile, plane) work of the depth-2 kernel over the SMs three ways.
    # 256 x 256 rows (32 row tiles) with 160 or 256 planes: four rows of one CTA per tile, each
    # a chunk of planes, and the remaining CTAs share the top chunk of every tile (ROWS).
    # 1280 x 128 rows (160 tiles, more than the SMs) with 8 planes: equal ranges of the
    # (tile, plane) sequence that cross tile boundaries (BALANCED). Either way, the same bits
    # as the depth-1 kernel.
    x0 = init_fields(model, shape, seed=13)
    base = gpu_run(pf, model, x0, 4, tuning=(64, 16, 1))
    got = gpu_run(pf, model, x0, 4, tuning=(tile, 8, 2))
    for a, b in zip(base, got):
        assert np.array_equal(a, b)


def test_depth2_3d_rejected_where_unsupported(pf):
    from paper_2109_02598_gb300 import PfError
    g = pf.Grid((8, 16, 64), 2).set_model("gs", COEFFS["gs"], DT["gs"])
    with pytest.raises(PfError):
        g.set_tuning(128, 8, 2)  # nx != 128
    g.close()
    h = pf.Grid((8, 16, 128), 1).set_model("ch", COEFFS["ch"], DT["ch"])
    with pytest.raises(PfError):
        h.set_tuning(128, 8, 2)  # no depth-2 kernel for Model B
    h.close()


def test_tma_tile_rejected_when_grid_does_not_divide(pf):
    from paper_2109_02598_gb300 import PfError
    g = pf.Grid((8, 20, 64), 2).set_model("gs", COEFFS["gs"], DT["gs"])
    with pytest.raises(PfError, match="ny"):
        g.set_tuning(64, 16, 1)  # ny = 20 is not a multiple of 16
    g.set_tuning(64, 8, 1)  # the general kernel takes any size
    g.close()
    h = pf.Grid((8, 40, 64), 1).set_model("ch", COEFFS["ch"], DT["ch"])
    with pytest.raises(PfError, match="ny"):
        h.set_tuning(64, 16, 1)  # Model B on the TMA tiles too, but ny = 40 % 16 != 0
    h.close()


@pytest.mark.parametrize("model", ["ch", "c"])
@pytest.mark.parametrize("shape,tiles", [((12, 32, 128), [(64, 16), (128, 8), (128, 16)]),
                                         ((5, 16, 64), [(64, 16)]),
                                         ((3, 8, 128), [(128, 8)]),
                                         ((64, 64, 64), [(64, 16)])])
def test_radius2_tma_kernel_is_bitwise_general(pf, model, shape, tiles):
    # Models B and C on the TMA z-streaming tiles (the chemical potential on chip, one ring
    # wider than the tile): the general kernel's bits for every tile and step count, and the
    # oracle within the single-step bar
    x0 = init_fields(model, shape, seed=14)
    for n in (1, 2, 7):
        base = gpu_run(pf, model, x0, n, tuning=(32, 16, 1))
        for t in tiles:
            got = gpu_run(pf, model, x0, n, tuning=(t[0], t[1], 1))
            for a, b in zip(base, got):
                assert np.array_equal(a, b), (n, t)
    t = tiles[0]
    one = gpu_run(pf, model, x0, 1, tuning=(t[0], t[1], 1))
    assert rel_linf(one, oracle.euler_step(model, x0, COEFFS[model], DT[model])) <= 1e-6


def test_default_tuning_picks_tma_for_the_3d_workload(pf):
    g = pf.Grid((256, 256, 256), 2).set_model("gs", COEFFS["gs"], DT["gs"])
    assert g.tuning == (128, 16, 1)
    g.close()
    g = pf.Grid((8, 48, 192), 2).set_model("gs", COEFFS["gs"], DT["gs"])
    assert g.tuning == (64, 16, 1)
    g.close()


# ---------------------------------------------------------------- workload configurations

def test_ac2d_128_1000_steps(pf):
    w = synthetic.WORKLOADS["ac2d_128"]
    x0 = synthetic.workload_init("ac2d_128")
    ref = oracle.run("ac", x0, w["coeffs"], w["dt"], 1000, w["h"])
    got = gpu_run(pf, "ac", x0, 1000, w["coeffs"], w["dt"], w["h"])
    assert rel_l2(got, ref) <= 1e-3
    one = gpu_run(pf, "ac", x0, 1, w["coeffs"], w["dt"], w["h"])
    assert rel_linf(one, oracle.euler_step("ac", x0, w["coeffs"], w["dt"])) <= 1e-6


@pytest.mark.parametrize("bands", [False, True])
def test_ch2d_1000_steps_256(pf, bands):
    # the 2048^2 recipe at 256^2 so the oracle finishes 1000 steps in seconds; also on the
    # band kernel (64 bands of 4 rows)
    w = synthetic.WORKLOADS["ch2d_2048"]
    x0 = synthetic.workload_init("ch2d_2048", shape=(256, 256))
    ref = oracle.run("ch", x0, w["coeffs"], w["dt"], 1000, w["h"])
    tuning = (256, pf.PF_TILE_BANDS, 1) if bands else None
    got = gpu_run(pf, "ch", x0, 1000, w["coeffs"], w["dt"], w["h"], tuning=tuning)
    assert rel_l2(got, ref) <= 1e-3


def test_gs3d_1000_steps_48(pf):
    w = synthetic.WORKLOADS["gs3d_256"]
    x0 = synthetic.workload_init("gs3d_256", shape=(48, 48, 48))
    ref = oracle.run("gs", x0, w["coeffs"], w["dt"], 1000, w["h"])
    got = gpu_run(pf, "gs", x0, 1000, w["coeffs"], w["dt"], w["h"])
    assert rel_l2(got, ref) <= 1e-3


@pytest.mark.parametrize("shape,tunings", [
    ((48, 32, 128), [(128, 8, 2), (64, 16, 1)]),
    ((16, 16, 256), [(256, 8, 2), (128, 16, 1)])])
def test_gs3d_1000_steps_on_the_timed_3d_kernels(pf, shape, tunings):
    # the 3D Gray-Scott recipe on grids the depth-2 kernel (full x-rows, 8-row tiles) and the
    # TMA z-streaming kernel both take, each pinned to the oracle directly: one launch's steps
    # (two for depth 2) within the single-step bar, 1000 steps within the 1000-step bar
    w = synthetic.WORKLOADS["gs3d_256"]
    x0 = synthetic.workload_init("gs3d_256", shape=shape)
    ref = oracle.run("gs", x0, w["coeffs"], w["dt"], 1000, w["h"])
    for t in tunings:
        k = t[2]
        one = gpu_run(pf, "gs", x0, k, w["coeffs"], w["dt"], w["h"], tuning=t)
        assert rel_linf(one, oracle.run("gs", x0, w["coeffs"], w["dt"], k, w["h"])) <= 1e-6, t
        got = gpu_run(pf, "gs", x0, 1000, w["coeffs"], w["dt"], w["h"], tuning=t)
        assert rel_l2(got, ref) <= 1e-3, (t, rel_l2(got, ref))


@pytest.mark.parametrize("name", ["ch2d_2048", "gs3d_256"])
def test_full_size_single_step(pf, name):
    w = synthetic.WORKLOADS[name]
    x0 = synthetic.workload_init(name)
    ref = oracle.euler_step(w["model"], x0, w["coeffs"], w["dt"], w["h"])
    got = gpu_run(pf, w["model"], x0, 1, w["coeffs"], w["dt"], w["h"])
    assert rel_linf(got, ref) <= 1e-6


def test_full_size_ch2d_mass_conserved(pf):
    # 2000 steps of the 2048^2 configuration on the default tiled kernel and on the band
    # kernel (the autotuner's choice for this grid): mass conserved, and the same bits
    w = synthetic.WORKLOADS["ch2d_2048"]
    (x0,) = synthetic.workload_init("ch2d_2048")
    phis = []
    for tuning in (None, (2048, pf.PF_TILE_BANDS, 1)):
        g = pf.Grid(x0.shape, 1, w["h"]).set_model("ch", w["coeffs"], w["dt"])
        if tuning:
            g.set_tuning(*tuning)
        g.write_field(0, x0)
        m0 = g.mass()
        assert abs(m0 - oracle.mass(x0)) <= 1e-9 * np.abs(x0.astype(np.float64)).sum()
        g.step(2000)
        m1 = g.mass()
        assert abs(m1 - m0) / x0.size <= 1e-6  # mean drift per site
        phi = g.read_field(0)
        assert np.isfinite(phi).all() and phi.std() > x0.std()  # spinodal growth happened
        g.close()
        phis.append(phi)
    assert np.array_equal(phis[0], phis[1])


def test_full_length_ch2d_on_the_band_kernel(pf):
    # the whole Model B configuration (2048^2, 20000 steps) on the kernel the autotuner
    # picks for it: mass conserved to float32 round-off, the field finite, the free energy
    # lower than at the start (the scheme is the energy's H^-1 gradient flow)
    w = synthetic.WORKLOADS["ch2d_2048"]
    (x0,) = synthetic.workload_init("ch2d_2048")
    g = pf.Grid(x0.shape, 1, w["h"]).set_model("ch", w["coeffs"], w["dt"])
    g.set_tuning(2048, pf.PF_TILE_BANDS, 1)
    g.write_field(0, x0)
    m0, e0 = g.mass(), g.energy()
    g.step(w["steps"])
    m1, e1 = g.mass(), g.energy()
    phi = g.read_field(0)
    g.close()
    assert w["steps"] == 20000
    assert abs(m1 - m0) / x0.size <= 1e-6
    assert np.isfinite(phi).all() and np.abs(phi).max() < 1.5
    assert e1 < e0


def test_full_size_gs3d_stays_bounded(pf):
    # the whole 3D Gray-Scott configuration (256^3, 5000 steps) on the default depth-1 TMA
    # kernel and on the depth-2 kernel the autotuner picks: finite, within [-0.01, 1.01],
    # and the same bits
    w = synthetic.WORKLOADS["gs3d_256"]
    x0 = synthetic.workload_init("gs3d_256")
    out = []
    for tuning in (None, (256, 8, 2)):
        g = pf.Grid(x0[0].shape, 2, w["h"]).set_model("gs", w["coeffs"], w["dt"])
        if tuning:
            g.set_tuning(*tuning)
        g.write_fields(x0)
        g.step(w["steps"])
        u, v = g.read_fields()
        g.close()
        assert np.isfinite(u).all() and np.isfinite(v).all()
        assert u.min() >= -0.01 and u.max() <= 1.01 and v.min() >= -0.01 and v.max() <= 1.01
        out.append((u, v))
    assert w["steps"] == 5000
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


# ---------------------------------------------------------------- invariants on the GPU

def test_gs_fixed_point_is_bitwise(pf):
    for shape in [(33, 70), (5, 9, 13)]:
        u = np.ones(shape, np.float32)
        v = np.zeros(shape, np.float32)
        out = gpu_run(pf, "gs", (u, v), 25)
        assert np.array_equal(out[0], u) and np.array_equal(out[1], v)


def test_ac_energy_decreases(pf):
    w = synthetic.WORKLOADS["ac2d_128"]
    x0 = synthetic.workload_init("ac2d_128")
    g = pf.Grid(x0[0].shape, 1, w["h"]).set_model("ac", w["coeffs"], w["dt"])
    g.write_fields(x0)
    e_prev = g.energy()
    assert abs(e_prev - oracle.energy(x0[0])) <= 1e-10 * abs(e_prev)
    for _ in range(100):
        g.step(10)
        e = g.energy()
        assert e <= e_prev + 1e-6 * abs(e_prev)
        e_prev = e
    g.close()


@pytest.mark.parametrize("shape", [(37, 150), (9, 20, 70)])
def test_reductions_match_oracle(pf, shape):
    (phi,) = init_fields("ac", shape, seed=5)
    g = pf.Grid(shape, 1, 0.7).set_model("ac", (0.9, 1.1), 0.01)
    g.write_field(0, phi)
    assert abs(g.mass() - oracle.mass(phi, 0.7)) <= 1e-12 * oracle.mass(np.abs(phi), 0.7)
    e = oracle.energy(phi, 0.9, 1.1, 0.7)
    assert abs(g.energy() - e) <= 1e-12 * abs(e)
    g.close()


def test_device_tensor_io(pf):
    import torch
    shape = (40, 72)
    (x0,) = init_fields("ac", shape, seed=6)
    g = pf.Grid(shape, 1).set_model("ac", COEFFS["ac"], DT["ac"])
    g.write_field(0, torch.from_numpy(x0).cuda())
    g.step(3)
    t = g.read_field(0, device=True)
    assert t.is_cuda
    ref = oracle.run("ac", (x0,), COEFFS["ac"], DT["ac"], 3)
    assert rel_linf((t.cpu().numpy(),), ref) <= 1e-6
    g.close()


def test_errors_are_reported(pf):
    from paper_2109_02598_gb300 import PfError
    g = pf.Grid((16, 16), 1)
    with pytest.raises(PfError, match="no model"):
        g.step(1)
    with pytest.raises(PfError, match="stability"):
        g.set_model("ac", (1.0, 1.0), 1.0)
    with pytest.raises(PfError):
        g.set_model("gs", (0.2, 0.1, 0.04, 0.06), 0.5)  # needs 2 fields
    g.set_model("ac", (1.0, 1.0), 2.0, force=True)
    g.write_field(0, np.full((16, 16), 1e30, np.float32))
    g.step(5)
    with pytest.raises(PfError, match="not finite"):
        g.mass()
    g.close()


# ---------------------------------------------------------------- Model C (eutectic)

@pytest.mark.parametrize("shape", [(96, 80), (16, 24, 20)])
def test_model_c_invariants_and_energy(pf, shape):
    x0 = init_fields("c", shape, seed=11)
    g = pf.Grid(shape, 2).set_model("c", COEFFS["c"], DT["c"])
    g.write_fields(x0)
    m0 = g.mass(1)
    e0 = g.energy()
    assert abs(e0 - oracle.energy_model_c(*x0, *COEFFS["c"])) <= 1e-10 * abs(e0)
    e_prev = e0
    for _ in range(20):
        g.step(10)
        e = g.energy()
        assert e <= e_prev + 1e-6 * abs(e_prev)
        e_prev = e
    assert abs(g.mass(1) - m0) / np.prod(shape) <= 1e-6
    got = g.read_fields()
    g.close()
    ref = oracle.run("c", x0, COEFFS["c"], DT["c"], 200)
    assert rel_l2(got, ref) <= 1e-4


# ---------------------------------------------------------------- further stencils

STENCIL_MAP = {"iso": "9iso", "4th": "9o4"}


def gpu_run_st(pf, model, fields, n, stencil, dt, h=1.0, tuning=None):
    g = pf.Grid(fields[0].shape, n_fields=len(fields), h=h)
    g.set_stencil(stencil)
    g.set_model(model, COEFFS[model], dt, force=True)
    if tuning is not None:
        g.set_tuning(*tuning)
    g.write_fields(fields)
    g.step(n)
    out = g.read_fields()
    g.close()
    return out


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("stencil", ["iso", "4th"])
@pytest.mark.parametrize("shape", [(37, 150), (70, 33), (5, 7)])
def test_2d_stencils_single_step_and_bitwise(pf, model, stencil, shape):
    x0 = init_fields(model, shape, seed=21)
    dt, h = DT[model] * 0.5, 0.9
    ref = oracle.euler_step(model, x0, COEFFS[model], dt, h, stencil=STENCIL_MAP[stencil])
    got = gpu_run_st(pf, model, x0, 1, stencil, dt, h)
    assert rel_linf(got, ref) <= 1e-6
    # every supported tile and depth gives the same bits
    base = gpu_run_st(pf, model, x0, 6, stencil, dt, h, tuning=(64, 16, 1))
    for t in [(64, 16, 2), (128, 32, 1), (128, 32, 2)]:
        got = gpu_run_st(pf, model, x0, 6, stencil, dt, h, tuning=t)
        for a, b in zip(base, got):
            assert np.array_equal(a, b), t
    ref6 = oracle.run(model, x0, COEFFS[model], dt, 6, h, stencil=STENCIL_MAP[stencil])
    assert rel_linf(base, ref6) <= 1e-5


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", [(9, 20, 70), (4, 4, 4), (6, 17, 33)])
@pytest.mark.parametrize("stencil,oname", [("iso", "19iso"), ("iso27", "27iso")])
def test_3d_isotropic_stencil(pf, model, shape, stencil, oname):
    x0 = init_fields(model, shape, seed=22)
    dt, h = DT[model] * 0.5, 0.9
    ref = oracle.euler_step(model, x0, COEFFS[model], dt, h, stencil=oname)
    got = gpu_run_st(pf, model, x0, 1, stencil, dt, h)
    assert rel_linf(got, ref) <= 1e-6
    a = gpu_run_st(pf, model, x0, 5, stencil, dt, h, tuning=(32, 16, 1))
    b = gpu_run_st(pf, model, x0, 5, stencil, dt, h, tuning=(64, 8, 1))
    for p, q in zip(a, b):
        assert np.array_equal(p, q)
    ref5 = oracle.run(model, x0, COEFFS[model], dt, 5, h, stencil=oname)
    assert rel_linf(a, ref5) <= 1e-5


def test_stencil_rules(pf):
    from paper_2109_02598_gb300 import PfError
    g = pf.Grid((8, 16, 64), 2).set_model("gs", COEFFS["gs"], DT["gs"])
    with pytest.raises(PfError):
        g.set_stencil("4th")  # 2D only
    g.set_stencil("iso")
    assert g.tuning == (32, 16, 1)  # the general 3D kernel
    g.set_stencil("iso27")
    assert g.tuning == (32, 16, 1)
    with pytest.raises(PfError):
        g.set_tuning(64, 16, 1)  # no TMA kernel with this stencil
    g.close()
    h = pf.Grid((64, 64), 1).set_model("ch", (1.0, 1.0, 1.0), 0.03, force=True)
    with pytest.raises(PfError, match="stability"):
        h.set_stencil("4th")  # dt beyond the fourth-order bound
    with pytest.raises(PfError, match="3D grids only"):
        h.set_stencil("iso27")
    h.close()


def test_bounded_wait_times_out_and_reports(pf):
    # a wait that nothing completes gives up after its budget and the status says so;
    # the context stays usable afterwards
    import torch
    from paper_2109_02598_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.pf_selftest_wait_timeout(200000, None) == _lib.PF_ERR_TIMEOUT
    assert b"bounded wait ran out" in lib.pf_last_error()
    assert lib.pf_selftest_wait_timeout(200000, stream) == _lib.PF_ERR_TIMEOUT
    x0 = init_fields("gs", (6, 16, 64), seed=30)
    ref = oracle.euler_step("gs", x0, COEFFS["gs"], DT["gs"])
    assert rel_linf(gpu_run(pf, "gs", x0, 1), ref) <= 1e-6


def set_cluster_tuning(g, k):
    """Select the on-chip cluster kernel (tile = full rows x ny / CS); CS is 16 or 8."""
    from paper_2109_02598_gb300 import PfError
    ny, nx = g.shape
    for cs in (16, 8):
        if ny % cs:
            continue
        try:
            g.set_tuning(nx, ny // cs, k)
            return cs
        except PfError:
            continue
    raise AssertionError("no cluster tuning accepted")


@pytest.mark.parametrize("model,k", [("ac", 1), ("ac", 2), ("ac", 4), ("ac", 8), ("gs", 1),
                                     ("gs", 4), ("gs", 8), ("ch", 1), ("ch", 2), ("c", 1),
                                     ("c", 2)])
@pytest.mark.parametrize("shape", [(128, 128), (64, 96)])
def test_cluster_kernel_bitwise_and_oracle(pf, model, k, shape):
    # 37 steps: super-steps of k and a shorter last one; same bits as the tiled kernel
    radius = 2 if model in ("ch", "c") else 1
    if k * radius > shape[0] // 16:
        pytest.skip("the k-row halo is wider than a 16-CTA cluster's band of rows")
    x0 = init_fields(model, shape, seed=40)
    n = 37
    g = pf.Grid(shape, n_fields=len(x0)).set_model(model, COEFFS[model], DT[model], force=True)
    set_cluster_tuning(g, k)
    assert g.tuning[0] == shape[1]
    g.write_fields(x0)
    g.step(n)
    a = g.read_fields()
    g.close()
    b = gpu_run(pf, model, x0, n, tuning=(64, 16, 1))
    for p, q in zip(a, b):
        assert np.array_equal(p, q)
    ref = oracle.run(model, x0, COEFFS[model], DT[model], n)
    assert rel_linf(a, ref) <= 1e-5


def test_cluster_kernel_rules_and_autotune(pf):
    from paper_2109_02598_gb300 import PfError
    g = pf.Grid((128, 128), 1).set_model("ac", COEFFS["ac"], DT["ac"])
    g.write_fields(init_fields("ac", (128, 128), seed=41))
    t = g.autotune(3)  # the cluster kernel is a candidate
    g.step(10)
    g.close()
    h = pf.Grid((128, 128), 1).set_model("ac", COEFFS["ac"], DT["ac"]).set_stencil("iso")
    with pytest.raises(PfError, match="cluster"):
        set_cluster_tuning_strict(h)
    h.close()
    assert len(t) == 3


def set_cluster_tuning_strict(g):
    ny, nx = g.shape
    g.set_tuning(nx, ny // 16, 1)


@pytest.mark.parametrize("model,shape", [
    ("ch", (256, 512)),   # 64 bands of exactly 2R = 4 rows: edge rows only
    ("ch", (333, 388)),   # 83 bands of 4-5 rows; 97 threads (a partial warp)
    ("ch", (1000, 1024)), # one band per SM, 6-7 rows
    ("ac", (304, 128)),   # bands of 2 rows
    ("ac", (77, 388)),    # 38 bands of 2-3 rows
    ("ac", (1000, 512)),
    ("ch", (608, 2560)),  # four columns per thread (nx > 2048), bands of 4 rows
    ("ac", (304, 4096))])
def test_band_kernel_bitwise_and_oracle(pf, model, shape):
    # the grid held in the SMs' shared memory, bands exchanging edge rows every step:
    # 1 and 37 steps give the tiled kernel's bits; 37 steps also meet the oracle
    x0 = init_fields(model, shape, seed=60)
    for n in (1, 37):
        g = pf.Grid(shape, 1).set_model(model, COEFFS[model], DT[model], force=True)
        g.set_tuning(shape[1], pf.PF_TILE_BANDS, 1)
        assert g.tuning == (shape[1], pf.PF_TILE_BANDS, 1)
        g.write_fields(x0)
        g.step(n)
        a = g.read_fields()
        g.close()
        b = gpu_run(pf, model, x0, n, tuning=(64, 16, 1))
        for p, q in zip(a, b):
            assert np.array_equal(p, q)
    ref = oracle.run(model, x0, COEFFS[model], DT[model], 37)
    assert rel_linf(a, ref) <= 1e-5


@pytest.mark.parametrize("model,coeffs,dt", [("ch", (0.8, 1.2, 0.6), 0.0012),
                                              ("ac", (0.7, 1.3), 0.02)])
def test_band_kernel_spacing_and_coefficients(pf, model, coeffs, dt):
    # h = 0.5 (Laplacian factor 4) and non-unit coefficients: the tiled kernel's bits
    shape = (300, 256)
    x0 = init_fields(model, shape, seed=65)
    a = gpu_run(pf, model, x0, 23, coeffs, dt, h=0.5, tuning=(256, pf.PF_TILE_BANDS, 1))
    b = gpu_run(pf, model, x0, 23, coeffs, dt, h=0.5, tuning=(64, 16, 1))
    assert np.array_equal(a[0], b[0])
    ref = oracle.run(model, x0, coeffs, dt, 23, 0.5)
    assert rel_linf(a, ref) <= 1e-5


def test_band_kernel_model_b_2048_and_repeated_calls(pf):
    # the Model B configuration's grid: one step against the oracle; three calls of 5 steps
    # equal one call of 15 (step counters restart with every launch) and the tiled kernel
    shape = (2048, 2048)
    x0 = (synthetic.cahn_hilliard_init(shape, seed=2),)
    g = pf.Grid(shape, 1).set_model("ch", COEFFS["ch"], DT["ch"])
    g.set_tuning(2048, pf.PF_TILE_BANDS, 1)
    g.write_fields(x0)
    g.step(1)
    one = g.read_fields()
    ref = oracle.euler_step("ch", x0, COEFFS["ch"], DT["ch"])
    assert rel_linf(one, ref) <= 1e-6
    g.write_fields(x0)
    for _ in range(3):
        g.step(5)
    a = g.read_fields()
    g.write_fields(x0)
    g.step(15)
    b = g.read_fields()
    g.close()
    c = gpu_run(pf, "ch", x0, 15, tuning=(128, 16, 2))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[0], c[0])


def test_band_kernel_rules_and_autotune(pf):
    from paper_2109_02598_gb300 import PfError
    g = pf.Grid((512, 512), 1).set_model("ch", COEFFS["ch"], DT["ch"])
    with pytest.raises(PfError, match="band kernel"):
        g.set_tuning(512, pf.PF_TILE_BANDS, 2)  # k = 1 only
    g.set_stencil("iso")
    with pytest.raises(PfError, match="band kernel"):
        g.set_tuning(512, pf.PF_TILE_BANDS, 1)
    g.close()
    for model, shape in (("gs", (512, 512)), ("ac", (512, 60)), ("ac", (3, 512))):
        h = pf.Grid(shape, 2 if model == "gs" else 1).set_model(model, COEFFS[model], DT[model])
        with pytest.raises(PfError, match="band kernel"):
            h.set_tuning(shape[1], pf.PF_TILE_BANDS, 1)
        h.close()
    g = pf.Grid((1024, 1024), 1).set_model("ch", COEFFS["ch"], DT["ch"])
    x0 = (synthetic.cahn_hilliard_init((1024, 1024), seed=61),)
    g.write_fields(x0)
    t = g.autotune(3)  # the band kernel is a candidate; the state is left as it was
    g.step(7)
    a = g.read_fields()
    g.close()
    assert len(t) == 3
    assert np.array_equal(a[0], gpu_run(pf, "ch", x0, 7)[0])


def test_autotune_cache_file(pf, tmp_path):
    # the first autotune stores its choice; a second grid of the same kind takes it from the
    # file; an entry the library rejects is tuned again and overwritten
    from paper_2109_02598_gb300 import tunecache
    path = str(tmp_path / "tune.json")
    x0 = init_fields("ch", (256, 256), seed=62)
    g = pf.Grid((256, 256), 1).set_model("ch", COEFFS["ch"], DT["ch"]).write_fields(x0)
    t1 = g.autotune(3, cache=path)
    g.close()
    data = tunecache.read(path)
    assert list(data.values()) == [list(t1)]
    key = next(iter(data))
    h = pf.Grid((256, 256), 1).set_model("ch", COEFFS["ch"], DT["ch"]).write_fields(x0)
    assert h.autotune(3, cache=path) == t1
    h.close()
    tunecache.put(path, key, (7, 7, 1))  # no such tile
    h = pf.Grid((256, 256), 1).set_model("ch", COEFFS["ch"], DT["ch"]).write_fields(x0)
    t3 = h.autotune(3, cache=path)
    h.close()
    assert tunecache.get(path, key) == tuple(t3) != (7, 7, 1)


def test_run_series_mass_and_energy(pf):
    # Model B conserves mass; Model A's discrete energy does not increase at a stable dt
    x0 = init_fields("ch", (128, 128), seed=63)
    g = pf.Grid((128, 128), 1).set_model("ch", COEFFS["ch"], DT["ch"]).write_fields(x0)
    s = g.run_series(200, 25)
    g.close()
    assert [r["step"] for r in s] == list(range(0, 201, 25))
    assert max(abs(r["mass"][0] - s[0]["mass"][0]) for r in s) / x0[0].size <= 1e-6
    x0 = init_fields("ac", (128, 128), seed=64)
    g = pf.Grid((128, 128), 1).set_model("ac", COEFFS["ac"], DT["ac"]).write_fields(x0)
    s = g.run_series(100, 10, energy=True)
    g.close()
    e = [r["energy"] for r in s]
    assert all(b <= a * (1 + 1e-6) + 1e-6 for a, b in zip(e, e[1:]))
    assert e[-1] < e[0]


@pytest.mark.parametrize("model,shape,tuning", [("gs", (6, 32, 128), None),
                                                 ("ch", (256, 256), (256, -1, 1)),
                                                 ("c", (40, 36), (64, 16, 2))])
def test_checkpoint_resume_is_bitwise(pf, tmp_path, model, shape, tuning):
    # 12 steps, save, load into a new grid, 18 more: the bits of 30 steps without a stop
    x0 = init_fields(model, shape, seed=66)
    g = pf.Grid(shape, len(x0)).set_model(model, COEFFS[model], DT[model], force=True)
    if tuning:
        g.set_tuning(*tuning)
    g.write_fields(x0).step(12)
    g.save(str(tmp_path / "c.npz"), extra={"note": "half way"})
    g.close()
    h = pf.Grid.load(str(tmp_path / "c.npz"))
    assert h.steps_done == 12 and h.model == model and h.checkpoint_extra == {"note": "half way"}
    if tuning:
        assert h.tuning == tuning
    h.step(18)
    a = h.read_fields()
    h.close()
    b = gpu_run(pf, model, x0, 30, tuning=tuning)
    for p, q in zip(a, b):
        assert np.array_equal(p, q)


def test_config_runner_series_checkpoints_and_resume(pf, tmp_path):
    # a run from a configuration: series every 20 steps, checkpoints every 30; resuming from
    # the step-30 checkpoint for 30 more steps writes the step-60 checkpoint's bits
    from paper_2109_02598_gb300 import checkpoint, run
    cfg = {"grid": {"shape": [128, 128]},
           "model": {"name": "ch", "coeffs": [1.0, 1.0, 1.0], "dt": 0.01},
           "init": {"synthetic": "cahn_hilliard_init", "args": {"seed": 67, "amp": 0.3}},
           "run": {"steps": 60, "tuning": [64, 16, 2], "series_every": 20,
                   "checkpoint_every": 30, "series_path": str(tmp_path / "a" / "series.json"),
                   "checkpoint_path": str(tmp_path / "a" / "ckpt_{step}.npz")}}
    s = run.run(cfg)
    assert s["steps_done"] == 60 and s["series"] == 4 and len(s["checkpoints"]) == 2
    series = __import__("json").load(open(tmp_path / "a" / "series.json"))
    assert [r["step"] for r in series] == [0, 20, 40, 60]
    assert max(abs(r["mass"][0] - series[0]["mass"][0]) for r in series) <= 1e-6 * 128 * 128
    cfg2 = dict(cfg, init={"checkpoint": str(tmp_path / "a" / "ckpt_30.npz")},
                run=dict(cfg["run"], steps=30, series_path=None,
                         checkpoint_path=str(tmp_path / "b" / "ckpt_{step}.npz")))
    s2 = run.run(cfg2)
    assert s2["steps_done"] == 60 and s2["checkpoints"] == [str(tmp_path / "b" / "ckpt_60.npz")]
    _, a = checkpoint.load_state(str(tmp_path / "a" / "ckpt_60.npz"))
    _, b = checkpoint.load_state(str(tmp_path / "b" / "ckpt_60.npz"))
    assert np.array_equal(a[0], b[0])


def test_async_host_copies_pipeline_jobs_on_two_grids(pf):
    # the pattern of a caller that overlaps copies with steps: jobs alternate between two
    # grids on two streams, each job uploading, stepping and downloading without waiting;
    # every job's result equals the synchronous path's bit for bit
    import torch
    shape = (6, 32, 128)
    x0 = init_fields("gs", shape, seed=50)
    ref = gpu_run(pf, "gs", x0, 10)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    grids = [pf.Grid(shape, 2, stream=s).set_model("gs", COEFFS["gs"], DT["gs"]) for s in streams]
    ins = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in x0]
    outs = [[torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(2)]
            for _ in range(4)]
    for j in range(4):
        g = grids[j % 2]
        for f in range(2):
            g.write_field_async(f, ins[f])
        g.step(10)
        for f in range(2):
            g.read_field_async(f, outs[j][f])
    for g in grids:
        g.synchronize()
        g.close()
    for o in outs:
        for f in range(2):
            assert np.array_equal(o[f].numpy(), ref[f])
