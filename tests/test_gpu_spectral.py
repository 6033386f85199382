"""Parity of the GPU semi-implicit spectral solver (Sec. 2.4.2) and structure factor (Sec. 3)
with the FP64 oracle, through the C ABI.

Bars (float32 transforms and kernels against the FP64 oracle from the same float32 array;
a float32 emulation of the scheme on the CPU stays below half of each):
  one step            relative L-inf <= 2e-6
  20 steps            relative L-inf <= 2e-5
  200 steps           relative L2    <= 1e-3
  structure factor    bin counts and centres bit-exact (the bin of a mode is decided in
                      float64 by the same operations on both sides); mean S within
                      1e-10 of max S (both transforms are float64)."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

COEFFS = {"ac": (1.0, 1.0), "ch": (1.0, 1.0, 1.0), "c": (1.0, 1.0, 1.0, 1.0, 1.0)}
DT = {"ac": 0.05, "ch": 0.05, "c": 0.005}
MODELS = ["ac", "ch", "c"]
# ragged and odd sizes: nx odd (scalar nonlinear path), an odd mode count (update tail),
# unit axes, and the paper's 2D size
SHAPES = [(48, 40), (30, 27), (1, 16), (16, 12, 20), (3, 5, 4), (5, 9, 7), (1, 6, 10),
          (128, 128)]


@pytest.fixture(scope="module")
def pf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02598_gb300.build import build
    build()
    import paper_2109_02598_gb300 as pf
    return pf


def init(model, shape, seed=0):
    return synthetic.paper_timing_init("ac" if model != "c" else "c", shape, seed=50 + seed)


def gpu_spectral(pf, model, fields, n, coeffs=None, dt=None, h=1.0, chunks=None, engine="auto"):
    s = pf.Spectral(fields[0].shape, model, COEFFS[model] if coeffs is None else coeffs,
                    DT[model] if dt is None else dt, h=h)
    s.set_engine(engine)
    s.write_fields(fields)
    for k in (chunks or [n]):
        s.step(k)
    out = s.read_fields()
    s.close()
    return out


def rel_linf(got, ref):
    num = max(np.abs(g.astype(np.float64) - r).max() for g, r in zip(got, ref))
    return num / max(np.abs(r).max() for r in ref)


def rel_l2(got, ref):
    num = np.sqrt(sum(((g.astype(np.float64) - r) ** 2).sum() for g, r in zip(got, ref)))
    return num / np.sqrt(sum((r ** 2).sum() for r in ref))


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", SHAPES)
def test_single_step(pf, model, shape):
    x0 = init(model, shape)
    ref = oracle.spectral_run(model, x0, COEFFS[model], DT[model], 1)
    assert rel_linf(gpu_spectral(pf, model, x0, 1, engine="cufft"), ref) <= 2e-6


# the fused engine: power-of-two sides, from the smallest it takes (4 x 2) to 1024; in 3D,
# (y, z) slabs from 2 x 2 to the paper's 64 x 64, and rows up to 256
FUSED_SHAPES = [(2, 4), (16, 16), (32, 64), (64, 8), (128, 128), (256, 1024),
                (2, 2, 4), (4, 8, 16), (16, 2, 32), (8, 32, 256), (64, 64, 64)]


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", FUSED_SHAPES)
def test_fused_engine_single_and_twenty_steps(pf, model, shape):
    x0 = init(model, shape, seed=9)
    for n, bar in ((1, 2e-6), (20, 2e-5)):
        ref = oracle.spectral_run(model, x0, COEFFS[model], DT[model], n)
        assert rel_linf(gpu_spectral(pf, model, x0, n, engine="fused"), ref) <= bar, n


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", [(64, 128), (16, 32, 8)])
def test_fused_and_cufft_engines_agree_and_interleave(pf, model, shape):
    x0 = init(model, shape, seed=10)
    a = gpu_spectral(pf, model, x0, 60, engine="fused")
    b = gpu_spectral(pf, model, x0, 60, engine="cufft")
    assert rel_linf(a, b) <= 2e-5
    # engines can alternate on one solver: the state is shared
    s = pf.Spectral(shape, model, COEFFS[model], DT[model]).write_fields(x0)
    for i in range(6):
        s.set_engine("fused" if i % 2 else "cufft").step(10)
    c = s.read_fields()
    s.close()
    assert rel_linf(c, b) <= 2e-5


def test_engine_selection(pf):
    s = pf.Spectral((64, 32), "ac", COEFFS["ac"], 0.05)
    assert s.engine == "fused"
    assert s.set_engine("cufft").engine == "cufft"
    s.close()
    # auto: fused wherever it takes the grid, except Model C with a 1024 side in 2D; in 3D
    # only slabs that fit a CTA's shared memory
    for shape, model, want in [((256, 256), "c", "fused"), ((512, 512), "ac", "fused"),
                               ((512, 512), "c", "fused"), ((1024, 1024), "ac", "fused"),
                               ((1024, 1024), "c", "cufft"),
                               ((64, 64, 64), "c", "fused"), ((8, 16, 32), "ac", "fused"),
                               ((256, 256, 256), "ac", "cufft")]:
        s = pf.Spectral(shape, model, COEFFS[model], DT[model])
        assert s.engine == want, (shape, model)
        s.close()
    for shape in [(48, 40), (16, 12, 20), (2048, 8)]:
        s = pf.Spectral(shape, "ac", COEFFS["ac"], 0.05)
        assert s.engine == "cufft"
        with pytest.raises(pf.PfError, match="power-of-two"):
            s.set_engine("fused")
        s.close()


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape", [(48, 40), (30, 27), (16, 12, 20), (3, 5, 4)])
def test_twenty_steps(pf, model, shape):
    x0 = init(model, shape, seed=1)
    ref = oracle.spectral_run(model, x0, COEFFS[model], DT[model], 20)
    assert rel_linf(gpu_spectral(pf, model, x0, 20, engine="cufft"), ref) <= 2e-5


@pytest.mark.parametrize("model,shape,dt", [("ac", (128, 128), 0.05), ("ch", (64, 64), 0.05),
                                            ("c", (32, 32, 32), 0.05), ("c", (128, 64), 0.02)])
@pytest.mark.parametrize("engine", ["cufft", "auto"])
def test_two_hundred_steps(pf, model, shape, dt, engine):
    x0 = init(model, shape, seed=2)
    ref = oracle.spectral_run(model, x0, COEFFS[model], dt, 200)
    assert rel_l2(gpu_spectral(pf, model, x0, 200, dt=dt, engine=engine), ref) <= 1e-3


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("shape,engine", [((24, 40), "cufft"), ((32, 64), "fused"),
                                          ((8, 16, 32), "fused")])
def test_one_call_equals_single_steps(pf, model, shape, engine):
    # cuFFT: two recorded 32-step graphs and 6 direct steps against 70 single calls; fused:
    # one 70-step launch against 70 one-step launches
    x0 = init(model, shape, seed=3)
    a = gpu_spectral(pf, model, x0, 70, engine=engine)
    b = gpu_spectral(pf, model, x0, 70, chunks=[1] * 70, engine=engine)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("model,shape,dt,steps", [("ac", (128, 128), 0.2, 2000),
                                                  ("c", (512, 512), 0.005, 10000),
                                                  ("c", (64, 64, 64), 0.005, 10000)])
def test_long_runs_stay_bounded(pf, model, shape, dt, steps):
    # the paper's run length: the fields stay finite and within reach of the wells, and
    # Model C's m keeps its mean (the k = 0 mode of a conserved field never changes).
    # Wells with all coefficients 1: Model A psi = +-1; Model C m = 1.879 (largest root of
    # m^3 - 3m - 1, from the equal chemical potentials) and psi^2 = 1 + 2m, |psi| = 2.175
    bound = 1.01 if model == "ac" else 2.25
    x0 = synthetic.paper_timing_init(model, shape)
    out = gpu_spectral(pf, model, x0, steps, dt=dt)
    for x in out:
        assert np.isfinite(x).all()
        assert np.abs(x).max() < bound
    if model == "c":
        assert abs(out[1].astype(np.float64).mean() - x0[1].astype(np.float64).mean()) < 1e-5


@pytest.mark.parametrize("model,coeffs", [("ac", (0.7, 0.0)), ("ch", (0.9, 0.0, 1.3))])
def test_linear_mode_evolves_by_exp_of_L_dt(pf, model, coeffs):
    shape, h, dt, n = (32, 48), 0.8, 0.4, 25
    coords = np.meshgrid(*[np.arange(s) * h for s in shape], indexing="ij")
    k = [2 * np.pi * m / (s * h) for m, s in zip((3, 2), shape)]
    kk = sum(ki * ki for ki in k)
    phi0 = (0.2 * np.cos(sum(ki * c for ki, c in zip(k, coords)) + 0.3)).astype(np.float32)
    L = -kk + coeffs[0] if model == "ac" else coeffs[2] * (-kk * kk + coeffs[0] * kk)
    got, = gpu_spectral(pf, model, (phi0,), n, coeffs=coeffs, dt=dt, h=h)
    exact = np.exp(L * dt * n) * phi0.astype(np.float64)
    assert np.abs(got - exact).max() <= 1e-5 * max(1.0, np.abs(exact).max())


@pytest.mark.parametrize("model", ["ch", "c"])
def test_conserved_field_keeps_its_mean(pf, model):
    x0 = init(model, (40, 36), seed=4)
    out = gpu_spectral(pf, model, x0, 100)
    m0, m1 = x0[-1].astype(np.float64), out[-1].astype(np.float64)
    assert abs(m1.mean() - m0.mean()) <= 1e-6
    assert np.abs(m1 - m0).max() > 1e-2  # it did evolve


def test_write_read_round_trip_and_zero_steps(pf):
    x0 = init("c", (20, 30), seed=5)
    out = gpu_spectral(pf, "c", x0, 0)
    assert rel_linf(out, x0) <= 1e-6
    # device-side tensors in and out
    import torch
    s = pf.Spectral((20, 30), "c", COEFFS["c"], DT["c"])
    s.write_fields([torch.from_numpy(x).cuda() for x in x0])
    s.step(3)
    d = s.read_field(1, device=True)
    h = s.read_field(1)
    assert np.array_equal(d.cpu().numpy(), h)
    s.close()


def test_rejects_bad_arguments(pf):
    with pytest.raises(pf.PfError, match="Models A, B and C"):
        pf.Spectral((16, 16), "gs", (0.2, 0.1, 0.04, 0.06), 0.5)
    with pytest.raises(pf.PfError, match="nx >= 2"):
        pf.Spectral((16, 1), "ac", COEFFS["ac"], 0.1)
    s = pf.Spectral((8, 8), "ac", COEFFS["ac"], 0.1)
    with pytest.raises(pf.PfError, match="out of range"):
        s.read_field(1)
    with pytest.raises(pf.PfError):
        s.step(-1)
    s.close()


@pytest.mark.parametrize("shape,n_bins,h", [((64, 64), 32, 1.0), ((30, 27), 7, 0.7),
                                            ((16, 12, 20), 1024, 1.0), ((5, 9, 7), 16, 1.3),
                                            ((1, 6, 10), 5, 1.0), ((256, 256), 64, 1.0)])
def test_structure_factor_matches_oracle(pf, shape, n_bins, h):
    psi = synthetic.paper_timing_init("ac", shape, seed=7)[0]
    c_ref, m_ref, n_ref = oracle.structure_factor(psi, h, n_bins)
    c, m, n = pf.structure_factor(psi, h, n_bins)
    assert np.array_equal(n, n_ref)
    assert np.array_equal(c, c_ref)
    assert np.abs(m - m_ref).max() <= 1e-10 * m_ref.max()
    # run to run: the same bits
    c2, m2, n2 = pf.structure_factor(psi, h, n_bins)
    assert np.array_equal(m, m2)


def test_structure_factor_of_a_padded_grid_and_an_evolved_state(pf):
    # nx = 27 has a row pitch of 28 in the grid's layout; the field is read in place
    x0 = init("ac", (30, 27), seed=8)
    s = pf.Spectral((30, 27), "ac", COEFFS["ac"], 0.1)
    s.write_fields(x0).step(50)
    psi = s.read_field(0)
    s.close()
    g = pf.Grid((30, 27), n_fields=1).set_model("ac", COEFFS["ac"], 0.05).write_fields((psi,))
    c, m, n = g.structure_factor(0, n_bins=12)
    g.close()
    c_ref, m_ref, n_ref = oracle.structure_factor(psi, 1.0, 12)
    assert np.array_equal(n, n_ref)
    assert np.abs(m - m_ref).max() <= 1e-10 * m_ref.max()


@pytest.mark.parametrize("model,shape", [("ac", (512, 512)), ("c", (64, 64, 64))])
def test_paper_sizes_one_step_every_site(pf, model, shape):
    x0 = synthetic.paper_timing_init(model, shape)
    ref = oracle.spectral_run(model, x0, COEFFS[model], DT[model], 1)
    assert rel_linf(gpu_spectral(pf, model, x0, 1), ref) <= 2e-6


@pytest.mark.parametrize("solver,dim,n,dt,steps,seeds", [
    ("spectral", 2, 512, 0.2, 500, 4), ("spectral", 3, 96, 0.2, 300, 2),
    ("euler", 2, 512, 0.05, 2000, 4)])
def test_porod_law(pf, solver, dim, n, dt, steps, seeds):
    # the paper's validation (Sec. 3): Model A quenched from U(-1, 1) to t = 100 (2D) or 60
    # (3D); the radially averaged S(k), averaged over independent runs, falls off as
    # k^-(d+1) between twice the peak wavenumber and k = 1.5
    shape = (n,) * dim
    Ss = []
    for seed in range(seeds):
        x0 = synthetic.paper_timing_init("ac", shape, seed=seed)
        if solver == "spectral":
            s = pf.Spectral(shape, "ac", COEFFS["ac"], dt).write_fields(x0).step(steps)
            c, m, cnt = pf.structure_factor(s.read_field(0, device=True), 1.0, 64)
        else:
            s = pf.Grid(shape, 1).set_model("ac", COEFFS["ac"], dt).write_fields(x0)
            s.step(steps)
            c, m, cnt = s.structure_factor(0, n_bins=64)
        s.close()
        Ss.append(m)
    slope, _, used = pf.porod_fit(c, np.mean(Ss, axis=0), cnt, 0.4, 1.5)
    assert used >= 8
    assert abs(slope + (dim + 1)) < 0.3, slope
